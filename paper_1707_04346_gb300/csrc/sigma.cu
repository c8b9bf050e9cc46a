// sigma = H c as sigma_1 + sigma_2 + sigma_3 (Eq. 8), string driven (Section 3.3).
//
// Layout: C and sigma are row-major [N_alpha][N_beta] (Eq. 4).
//  sigma_1 (beta-beta, I_alpha = J_alpha): gather inside C rows
//      sigma(Ia, Ib) = sum_J G_b(Ib, J) C(Ia, J)
//    with R rows of C staged in shared memory, so each entry of the beta
//    same-spin Hamiltonian (ELL) is read once per R rows.
//  sigma_2 (alpha-alpha, I_beta = J_beta): the same gather along columns
//      sigma(Ia, Ib) += sum_J G_a(Ia, J) C(J, Ib)
//    with R beta columns of C staged in shared memory (read and written as
//    runs of R consecutive elements of each row).
//  sigma_3 (alpha-beta): with W[(ij),(kl)] = (ij|kl) and the replacement
//    lists of both strings,
//      sigma(Ia, Ib) += sum_{a in E(Ia)} s_a sum_{b in E(Ib)} s_b W[p_a][p_b] C(J_a, J_b)
//    (the alpha-beta part of 1/2 sum (ij|kl) E_ij E_kl, where the alpha-beta
//    and beta-alpha halves coincide).  FP64: one CTA owns an output row; for
//    each alpha replacement a it stages C(J_a, :) and W[p_a, :] in shared
//    memory and accumulates the row of sigma in shared memory (diagonal
//    replacements merged, see k_sigma3_exact).  FP32: sigma_tc.cu.
#include "internal.cuh"

namespace fci {

constexpr int kEnt = 8;  // ELL entries whose table loads are issued together (FP32)

// Table loads issued as volatile asm, so that a batch of them stays together in
// program order ahead of its first use whatever the compiler's scheduling (the
// fused FP32 kernel lost a third of its speed to a schedule change once).
__device__ __forceinline__ int32_t ld_batch_s32(const int32_t *p) {
    int32_t v;
    asm volatile("ld.global.nc.s32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ float ld_batch_f32(const float *p) {
    float v;
    asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}

template <typename T>
__device__ __forceinline__ T gval_of(const SpinTables &S, int64_t idx);
template <>
__device__ __forceinline__ double gval_of<double>(const SpinTables &S, int64_t idx) {
    return S.gval[idx];
}
template <>
__device__ __forceinline__ float gval_of<float>(const SpinTables &S, int64_t idx) {
    return S.gvalf[idx];
}

// sigma_1 (beta-beta, I_alpha = J_alpha): R rows of C in shared memory,
//   sigma(Ia, Ib) = sum_e G_b[e][Ib] * C(Ia, col_e)   (overwrites sigma, or adds when add != 0)
// Each ELL entry of a beta string is read once per block of R rows.
template <typename T, int R>
__global__ void __launch_bounds__(512) k_sigma1_rows(const T *__restrict__ C, T *__restrict__ sig, SpinTables B,
                                                     int64_t nsa, int add) {
    constexpr int U = sizeof(T) == 4 ? kEnt : 1;  // FP64 is bound by its FMA pipe
    extern __shared__ unsigned char smem_raw[];
    T *rows = reinterpret_cast<T *>(smem_raw);
    const int64_t nsb = B.ns;
    const int64_t r0 = (int64_t)blockIdx.x * R;
    for (int64_t t = threadIdx.x; t < (int64_t)R * nsb; t += blockDim.x) {
        const int64_t r = t / nsb, j = t % nsb;
        rows[t] = (r0 + r < nsa) ? C[(r0 + r) * nsb + j] : T(0);
    }
    __syncthreads();
    for (int64_t ib = threadIdx.x; ib < nsb; ib += blockDim.x) {
        T acc[R];
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = 0;
        // ELL entries in batches of U: all table loads of a batch are in
        // flight before the first staged value is read
        for (int e0 = 0; e0 < B.nsame; e0 += U) {
            int32_t col[U];
            T v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const bool ok = e0 + u < B.nsame;
                const int64_t idx = (int64_t)(ok ? e0 + u : 0) * nsb + ib;
                col[u] = ok ? B.gcol[idx] : 0;
                v[u] = ok ? gval_of<T>(B, idx) : T(0);
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int r = 0; r < R; ++r) acc[r] = fma(v[u], rows[(int64_t)r * nsb + col[u]], acc[r]);
        }
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (r0 + r < nsa) sig[(r0 + r) * nsb + ib] = add ? sig[(r0 + r) * nsb + ib] + acc[r] : acc[r];
    }
}

// sigma_2 (alpha-alpha, I_beta = J_beta): R beta columns of C in shared memory,
//   sigma(Ia, Ib) += sum_e G_a[e][Ia] * C(col_e, Ib)
// Columns are loaded and written as runs of R consecutive elements of a row.
template <typename T, int R>
__global__ void __launch_bounds__(512) k_sigma2_cols(const T *__restrict__ C, T *__restrict__ sig, SpinTables A,
                                                     int64_t nsb) {
    constexpr int U = sizeof(T) == 4 ? kEnt : 1;  // FP64 is bound by its FMA pipe
    extern __shared__ unsigned char smem_raw[];
    T *cols = reinterpret_cast<T *>(smem_raw);  // [R][nsa]
    const int64_t nsa = A.ns;
    const int64_t c0 = (int64_t)blockIdx.x * R;
    for (int64_t ia = threadIdx.x; ia < nsa; ia += blockDim.x) {
#pragma unroll
        for (int r = 0; r < R; ++r) cols[(int64_t)r * nsa + ia] = (c0 + r < nsb) ? C[ia * nsb + c0 + r] : T(0);
    }
    __syncthreads();
    for (int64_t ia = threadIdx.x; ia < nsa; ia += blockDim.x) {
        T acc[R];
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = 0;
        for (int e0 = 0; e0 < A.nsame; e0 += U) {
            int32_t col[U];
            T v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const bool ok = e0 + u < A.nsame;
                const int64_t idx = (int64_t)(ok ? e0 + u : 0) * nsa + ia;
                col[u] = ok ? A.gcol[idx] : 0;
                v[u] = ok ? gval_of<T>(A, idx) : T(0);
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int r = 0; r < R; ++r) acc[r] = fma(v[u], cols[(int64_t)r * nsa + col[u]], acc[r]);
        }
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (c0 + r < nsb) sig[ia * nsb + c0 + r] += acc[r];
    }
}

// ---- FP64 same-spin terms in double-float arithmetic ----
// GB300 issues FP32 operations 64 times faster than FP64 ones, so the FP64
// sigma_1 and sigma_2 carry every FP64 value x as the FP32 pair
// (h, l) = (fl(x), fl(x - h)), 48 significant bits.  A term v c is formed as
// h_v h_c exactly (the product and its rounding error, recovered by an FMA)
// plus the cross terms h_v l_c + l_v h_c (l_v l_c, below 2^-48 of the term, is
// left out), and added to the running pair (s_h, s_l) by TwoSum: twelve FP32
// operations per term, exact in s_h + s_l up to the FP32 roundings of the
// low-order parts, i.e. within a few units of 2^-48 of sum |terms|.
__device__ __forceinline__ float2 df_split(double x) {
    const float h = __double2float_rn(x);
    return make_float2(h, __double2float_rn(x - (double)h));
}

__device__ __forceinline__ void df_mac(float vh, float vl, float2 c, float &sh, float &sl) {
    const float ph = vh * c.x;
    const float pl = fmaf(vh, c.y, fmaf(vl, c.x, fmaf(vh, c.x, -ph)));
    const float t = sh + ph;
    const float bp = t - sh;
    sl += ((sh - (t - bp)) + (ph - bp)) + pl;
    sh = t;
}


// Staging of R (4 or 8) double-float values per string for the double-float
// kernels: one record of R float2 per string, whose 16-byte chunk k (values 2k
// and 2k + 1) sits at chunk position k ^ (x mod R/2).  An ELL entry then reads
// R/2 16-byte chunks of one record, and the lanes of a warp, which read the same
// chunk of different records, spread over all banks; with R rows of pairs
// staged one after the other each entry took R 8-byte loads that collided in
// the banks about 2.5 times.
template <int R>
__device__ __forceinline__ float4 *stage_chunk(float4 *base, int64_t x, int k) {
    return base + x * (R / 2) + (k ^ (int)(x & (R / 2 - 1)));
}

// sigma_1 in double-float: R rows of C staged as pairs; sigma overwritten or
// (add != 0) added to.
template <int R, int U = 8>
__global__ void __launch_bounds__(512, 1) k_sigma1_rows_df(const double *__restrict__ C, double *__restrict__ sig,
                                                           SpinTables B, int64_t nsa, int add,
                                                           const int *__restrict__ active) {
    if (active != nullptr && *active == 0) return;  // gated launch (batched engine)
    extern __shared__ float4 stage4[];  // R >= 4: [nsb] records of R pairs; else [R][nsb] pairs
    float2 *rows2 = reinterpret_cast<float2 *>(stage4);
    const int64_t nsb = B.ns;
    const int64_t r0 = (int64_t)blockIdx.x * R;
    if constexpr (R >= 4) {
        for (int64_t j = threadIdx.x; j < nsb; j += blockDim.x)
#pragma unroll
            for (int k = 0; k < R / 2; ++k) {
                const float2 a = (r0 + 2 * k < nsa) ? df_split(C[(r0 + 2 * k) * nsb + j]) : make_float2(0.f, 0.f);
                const float2 b = (r0 + 2 * k + 1 < nsa) ? df_split(C[(r0 + 2 * k + 1) * nsb + j]) : make_float2(0.f, 0.f);
                *stage_chunk<R>(stage4, j, k) = make_float4(a.x, a.y, b.x, b.y);
            }
    } else {
        for (int64_t t = threadIdx.x; t < (int64_t)R * nsb; t += blockDim.x) {
            const int64_t r = t / nsb, j = t % nsb;
            rows2[t] = (r0 + r < nsa) ? df_split(C[(r0 + r) * nsb + j]) : make_float2(0.f, 0.f);
        }
    }
    __syncthreads();
    for (int64_t ib = threadIdx.x; ib < nsb; ib += blockDim.x) {
        float sh[R], sl[R];
#pragma unroll
        for (int r = 0; r < R; ++r) sh[r] = sl[r] = 0.f;
        for (int e0 = 0; e0 < B.nsame; e0 += U) {
            int32_t col[U];
            float vh[U], vl[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const bool ok = e0 + u < B.nsame;
                const int64_t idx = (int64_t)(ok ? e0 + u : 0) * nsb + ib;
                col[u] = ok ? B.gcol[idx] : 0;
                vh[u] = ok ? B.gvalf[idx] : 0.f;
                vl[u] = ok ? B.gvall[idx] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if constexpr (R >= 4) {
#pragma unroll
                    for (int k = 0; k < R / 2; ++k) {
                        const float4 q = *stage_chunk<R>(stage4, col[u], k);
                        df_mac(vh[u], vl[u], make_float2(q.x, q.y), sh[2 * k], sl[2 * k]);
                        df_mac(vh[u], vl[u], make_float2(q.z, q.w), sh[2 * k + 1], sl[2 * k + 1]);
                    }
                } else {
#pragma unroll
                    for (int r = 0; r < R; ++r) df_mac(vh[u], vl[u], rows2[(int64_t)r * nsb + col[u]], sh[r], sl[r]);
                }
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (r0 + r < nsa) {
                const int64_t o = (r0 + r) * nsb + ib;
                const double v = (double)sh[r] + (double)sl[r];
                sig[o] = add ? sig[o] + v : v;
            }
    }
}

// sigma_2 in double-float: R beta columns of C staged as pairs; adds to sigma.
template <int R, int U = 8>
__global__ void __launch_bounds__(512, 1) k_sigma2_cols_df(const double *__restrict__ C, double *__restrict__ sig,
                                                           SpinTables A, int64_t nsb, const int *__restrict__ active) {
    if (active != nullptr && *active == 0) return;
    extern __shared__ float4 stage4[];  // R >= 4: [nsa] records of R pairs; else [R][nsa] pairs
    float2 *cols2 = reinterpret_cast<float2 *>(stage4);
    const int64_t nsa = A.ns;
    const int64_t c0 = (int64_t)blockIdx.x * R;
    for (int64_t ia = threadIdx.x; ia < nsa; ia += blockDim.x) {
        if constexpr (R >= 4) {
#pragma unroll
            for (int k = 0; k < R / 2; ++k) {
                const float2 a = (c0 + 2 * k < nsb) ? df_split(C[ia * nsb + c0 + 2 * k]) : make_float2(0.f, 0.f);
                const float2 b = (c0 + 2 * k + 1 < nsb) ? df_split(C[ia * nsb + c0 + 2 * k + 1]) : make_float2(0.f, 0.f);
                *stage_chunk<R>(stage4, ia, k) = make_float4(a.x, a.y, b.x, b.y);
            }
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r)
                cols2[(int64_t)r * nsa + ia] = (c0 + r < nsb) ? df_split(C[ia * nsb + c0 + r]) : make_float2(0.f, 0.f);
        }
    }
    __syncthreads();
    for (int64_t ia = threadIdx.x; ia < nsa; ia += blockDim.x) {
        float sh[R], sl[R];
#pragma unroll
        for (int r = 0; r < R; ++r) sh[r] = sl[r] = 0.f;
        for (int e0 = 0; e0 < A.nsame; e0 += U) {
            int32_t col[U];
            float vh[U], vl[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const bool ok = e0 + u < A.nsame;
                const int64_t idx = (int64_t)(ok ? e0 + u : 0) * nsa + ia;
                col[u] = ok ? A.gcol[idx] : 0;
                vh[u] = ok ? A.gvalf[idx] : 0.f;
                vl[u] = ok ? A.gvall[idx] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if constexpr (R >= 4) {
#pragma unroll
                    for (int k = 0; k < R / 2; ++k) {
                        const float4 q = *stage_chunk<R>(stage4, col[u], k);
                        df_mac(vh[u], vl[u], make_float2(q.x, q.y), sh[2 * k], sl[2 * k]);
                        df_mac(vh[u], vl[u], make_float2(q.z, q.w), sh[2 * k + 1], sl[2 * k + 1]);
                    }
                } else {
#pragma unroll
                    for (int r = 0; r < R; ++r) df_mac(vh[u], vl[u], cols2[(int64_t)r * nsa + col[u]], sh[r], sl[r]);
                }
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (c0 + r < nsb) sig[ia * nsb + c0 + r] += (double)sh[r] + (double)sl[r];
    }
}

// FP32 sigma_1 + sigma_2 in one pass when both spins share one string space
// (n_alpha = n_beta, identical same-spin tables): a block stages R rows and
// the same R columns of C, and every ELL entry it reads updates both,
//   sigma(r0+r, x) += G[x][col] C(r0+r, col)      (sigma_1, row r0+r)
//   sigma(x, r0+r) += G[x][col] C(col, r0+r)      (sigma_2, column r0+r)
// which halves the table traffic that bounds the separate FP32 kernels.  Two
// blocks meet on each element (its row block and its column block), so sigma
// starts at zero and both adds are atomic; two addends onto zero give the
// same sum in either order.
template <int R>
__global__ void __launch_bounds__(512) k_sigma12_f32(const float *__restrict__ C, float *__restrict__ sig,
                                                     SpinTables S, const int *__restrict__ active) {
    if (active != nullptr && *active == 0) return;  // gated launch (batched engine): instance not active
    extern __shared__ float smf[];
    const int64_t ns = S.ns;
    float *rows = smf;           // [R][ns]
    float *cols = smf + R * ns;  // [R][ns]
    const int64_t r0 = (int64_t)blockIdx.x * R;
    for (int64_t t = threadIdx.x; t < (int64_t)R * ns; t += blockDim.x) {
        const int64_t r = t / ns, j = t % ns;
        rows[t] = (r0 + r < ns) ? C[(r0 + r) * ns + j] : 0.f;
    }
    for (int64_t i = threadIdx.x; i < ns; i += blockDim.x) {
#pragma unroll
        for (int r = 0; r < R; ++r) cols[(int64_t)r * ns + i] = (r0 + r < ns) ? C[i * ns + r0 + r] : 0.f;
    }
    __syncthreads();
    for (int64_t x = threadIdx.x; x < ns; x += blockDim.x) {
        float ar[R], ac[R];
#pragma unroll
        for (int r = 0; r < R; ++r) ar[r] = ac[r] = 0.f;
        for (int e0 = 0; e0 < S.nsame; e0 += kEnt) {
            int32_t col[kEnt];
            float v[kEnt];
#pragma unroll
            for (int u = 0; u < kEnt; ++u) {  // in-range addresses; padding slots zeroed after the loads
                const int64_t idx = (int64_t)(e0 + u < S.nsame ? e0 + u : 0) * ns + x;
                col[u] = ld_batch_s32(S.gcol + idx);
                v[u] = ld_batch_f32(S.gvalf + idx);
            }
#pragma unroll
            for (int u = 0; u < kEnt; ++u)
                if (e0 + u >= S.nsame) {
                    col[u] = 0;
                    v[u] = 0.f;
                }
#pragma unroll
            for (int u = 0; u < kEnt; ++u)
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    ar[r] = fmaf(v[u], rows[(int64_t)r * ns + col[u]], ar[r]);
                    ac[r] = fmaf(v[u], cols[(int64_t)r * ns + col[u]], ac[r]);
                }
        }
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (r0 + r < ns) {
                atomicAdd(sig + (r0 + r) * ns + x, ar[r]);
                atomicAdd(sig + x * ns + r0 + r, ac[r]);
            }
    }
}

// out[c][r] = in[r][c] (ADD: out[c][r] += in[r][c]) for a rows x cols matrix,
// through 32 x 32 tiles in shared memory (block 32 x 8).
template <bool ADD>
__global__ void k_transpose_f32(const float *__restrict__ in, float *__restrict__ out, int64_t rows, int64_t cols) {
    __shared__ float tile[32][33];
    const int64_t c0 = (int64_t)blockIdx.x * 32, r0 = (int64_t)blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int64_t r = r0 + i, c = c0 + threadIdx.x;
        if (r < rows && c < cols) tile[i][threadIdx.x] = in[r * cols + c];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int64_t c = c0 + i, r = r0 + threadIdx.x;
        if (c < cols && r < rows) {
            const float v = tile[threadIdx.x][i];
            out[c * rows + r] = ADD ? out[c * rows + r] + v : v;
        }
    }
}

__device__ __forceinline__ double flip_sign(double x, uint32_t signbit) {
    return __longlong_as_double(__double_as_longlong(x) ^ ((long long)signbit << 32));
}

// FP64 sigma_3, exact sparse, with the diagonal replacements merged:
//  * the n_alpha entries E_kk (k in I_a) all map I_a onto itself with sign +1;
//    they form one pass over C(I_a, :) with the integral row sum_k (kk|q);
//  * for every other alpha entry, the n_beta entries E_ll (l in I_b) of the
//    beta list contribute sum_l (p_a|ll) C(J_a, I_b) = wdiag_b[p_a][I_b] C(J_a, I_b).
// Each remaining (alpha, beta) replacement pair is one DFMA, the beta sign
// applied by flipping the sign bit:
//   2 * (s_b + (s_a - n_a)(s_b - n_b + 1)) FLOP per determinant.
__global__ void __launch_bounds__(512) k_sigma3_exact(const double *__restrict__ C, double *__restrict__ sig,
                                                      SpinTables A, SpinTables B, const double *__restrict__ W,
                                                      int npair) {
    extern __shared__ unsigned char smem_raw[];
    const int64_t nsb = B.ns;
    double *crow = reinterpret_cast<double *>(smem_raw);
    double *acc = crow + nsb;
    double *wrow = acc + nsb;
    uint32_t *ea = reinterpret_cast<uint32_t *>(wrow + npair);
    const int64_t ia = blockIdx.x;
    const int noff_b = B.ne * (int)(B.nsingle / (B.ne > 0 ? B.ne : 1) - 1);  // n_b (norb - n_b)
    for (int e = threadIdx.x; e < A.nsingle; e += blockDim.x) ea[e] = A.tab[(int64_t)e * A.ns + ia];
    for (int64_t j = threadIdx.x; j < nsb; j += blockDim.x) crow[j] = C[ia * nsb + j];
    __syncthreads();
    // merged alpha-diagonal pass
    for (int q = threadIdx.x; q < npair; q += blockDim.x) {
        double w = 0.0;
        for (int a = 0; a < A.nsingle; ++a)
            if ((int64_t)ent_target(ea[a]) == ia) w += W[(int64_t)ent_pair(ea[a]) * npair + q];
        wrow[q] = w;
    }
    __syncthreads();
    for (int64_t ib = threadIdx.x; ib < nsb; ib += blockDim.x) {
        double v = 0.0;
        for (int b = 0; b < B.nsingle; ++b) {
            const uint32_t entb = B.tab[(int64_t)b * nsb + ib];
            v = fma(flip_sign(wrow[ent_pair(entb)], entb & 0x80000000u), crow[ent_target(entb)], v);
        }
        acc[ib] = v;
    }
    // off-diagonal alpha entries
    for (int a = 0; a < A.nsingle; ++a) {
        const uint32_t enta = ea[a];
        const int64_t ja = ent_target(enta);
        if (ja == ia) continue;
        const int pa = ent_pair(enta);
        __syncthreads();  // previous pass finished with crow / wrow
        for (int64_t j = threadIdx.x; j < nsb; j += blockDim.x) crow[j] = C[ja * nsb + j];
        for (int q = threadIdx.x; q < npair; q += blockDim.x) wrow[q] = W[(int64_t)pa * npair + q];
        __syncthreads();
        const double *wd = B.wdiag + (int64_t)pa * nsb;
        for (int64_t ib = threadIdx.x; ib < nsb; ib += blockDim.x) {
            double v = wd[ib] * crow[ib];
            for (int b = 0; b < noff_b; ++b) {
                const uint32_t entb = B.tabo[(int64_t)b * nsb + ib];
                v = fma(flip_sign(wrow[ent_pair(entb)], entb & 0x80000000u), crow[ent_target(entb)], v);
            }
            acc[ib] += ent_negative(enta) ? -v : v;
        }
    }
    __syncthreads();
    for (int64_t j = threadIdx.x; j < nsb; j += blockDim.x) sig[ia * nsb + j] += acc[j];
}

// y <- y + sgn y^T (half = 0) or (y + sgn y^T) / 2 (half = 1), in place, for a
// square n x n matrix: a block takes the 32 x 32 tile (bi, bj), bi <= bj, and
// its mirror (bj, bi), reads both into shared memory and writes both (a
// diagonal tile once).  With c^T = sgn c this forms sigma_1 = sgn sigma_2^T
// from sigma_2 (Eq. 8 with the alpha and beta strings of one space), and it
// projects a vector onto the Ms = 0 combinations of one spin parity.
template <typename T>
__global__ void k_sym_pairs(T *__restrict__ y, int64_t n, int sgn, int half) {
    const int64_t bi = blockIdx.y, bj = blockIdx.x;
    if (bi > bj) return;
    __shared__ T a[32][33], b[32][33];
    const int tx = threadIdx.x;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t i = bi * 32 + r, j = bj * 32 + tx, i2 = bj * 32 + r, j2 = bi * 32 + tx;
        a[r][tx] = (i < n && j < n) ? y[i * n + j] : T(0);    // tile (bi, bj)
        b[r][tx] = (i2 < n && j2 < n) ? y[i2 * n + j2] : T(0);  // tile (bj, bi)
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t i = bi * 32 + r, j = bj * 32 + tx;
        T v = sgn > 0 ? T(a[r][tx] + b[tx][r]) : T(a[r][tx] - b[tx][r]);
        if (half) v = v / T(2);
        if (i < n && j < n) y[i * n + j] = v;
        if (bi != bj) {
            const int64_t i2 = bj * 32 + r, j2 = bi * 32 + tx;
            T w = sgn > 0 ? T(b[r][tx] + a[tx][r]) : T(b[r][tx] - a[tx][r]);
            if (half) w = w / T(2);
            if (i2 < n && j2 < n) y[i2 * n + j2] = w;
        }
    }
}

int sym_pairs(void *y, int64_t n, int elem, int sgn, int half, cudaStream_t s) {
    const dim3 grid(ceil_div(n, 32), ceil_div(n, 32)), block(32, 8);
    if (grid.y > 65535) return fail(FCI_ERR_ARG, "spin parity: more than 2097120 strings");
    if (elem == 8)
        k_sym_pairs<double><<<grid, block, 0, s>>>((double *)y, n, sgn, half);
    else if (elem == 4)
        k_sym_pairs<float><<<grid, block, 0, s>>>((float *)y, n, sgn, half);
    else if (elem == -8 && !half)
        k_sym_pairs<long long><<<grid, block, 0, s>>>((long long *)y, n, sgn, 0);
    else
        return fail(FCI_ERR_ARG, "sym_pairs: bad element kind");
    FCI_CUDA(cudaGetLastError());
    return FCI_OK;
}

static size_t smem_limit() {
    static int lim = -1;
    if (lim < 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&lim, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    }
    return (size_t)lim;
}

// Whether FP32 sigma_1/sigma_2 run through intermediate strings on the tensor
// cores (asked for, or the staged same-spin kernels do not fit); that path
// needs the 2N-float workspace ws32, which fci_init allocates.
bool f32_same_spin_tc(const fci_ctx *ctx) {
    const SpinTables &A = ctx->A, &B = ctx->B;
    const size_t lim = smem_limit();
    auto fits = [&](int r, int64_t len) { return (size_t)r * len * sizeof(float) <= lim; };
    const bool fused = A.ne == B.ne && A.ns == B.ns && fits(8, A.ns);  // 2 x 4 rows of the fused kernel
    const bool tc_ok = A.nsingle > 0 && B.nsingle > 0 && ctx->npair + 1 <= 256 && A.nsingle <= 96 &&
                       B.nsingle <= 96;
    return tc_ok && (ctx->opt.same_spin_tc == 1 || (!fused && (A.ne == B.ne || !fits(4, B.ns) || !fits(4, A.ns))));
}

int alloc_sigma_workspace(fci_ctx *ctx) {
    if (!f32_same_spin_tc(ctx) || ctx->ws32) return FCI_OK;
    int rc = FCI_OK;
    ctx->ws32 = (float *)dalloc(ctx, sizeof(float) * 2 * (size_t)ctx->ndet, &rc);
    return rc;
}

template <typename T>
static int sigma_impl(fci_ctx *ctx, const T *C, T *sig, cudaStream_t s, int parity) {
    const SpinTables &A = ctx->A, &B = ctx->B;
    // a vector of known spin parity (C^T = parity C, one string space): sigma_1 from sigma_2
    if (A.ne != B.ne || A.ns != B.ns) parity = 0;
    if constexpr (sizeof(T) == 8)
        if (sigma_wide_ok(ctx)) return launch_sigma_f64_wide(ctx, C, sig, s, parity);
    const int64_t nsa = A.ns, nsb = B.ns;
    const size_t lim = smem_limit();
    // sigma_1 then sigma_2: R rows / columns per block, the largest R whose block fits
    auto pick_r = [&](int64_t len) -> int {
        for (int r = 8; r >= 1; r >>= 1)
            if ((size_t)r * len * sizeof(T) <= lim) return r;
        return 0;
    };
    // FP32 with one string space for both spins: fused sigma_1 + sigma_2
    int fusedR = 0;
    if (sizeof(T) == 4 && A.ne == B.ne && nsa == nsb)
        for (int r : {8, 4})
            if (!fusedR && (size_t)2 * r * nsa * sizeof(float) <= lim) fusedR = r;
    // FP32 same-spin terms through intermediate strings on the tensor cores: when
    // asked for, or when the staged kernels above do not fit (large string spaces)
    const bool same_tc = sizeof(T) == 4 && f32_same_spin_tc(ctx);
    // profiled kernels (fci_profile_read): two slots when fused, else three
    static const char *const names3[3] = {"sigma1_rows", "sigma2_cols", sizeof(T) == 4 ? "sigma3_tc" : "sigma3_exact"};
    static const char *const names3tc[3] = {"sigma2_tc", "sigma1_tc", "sigma3_tc"};
    static const char *const names2[2] = {"sigma12_f32", "sigma3_tc"};
    static const char *const names4[4] = {"slice_c", "sigma3_sliced", "sigma1_rows", "sigma2_cols"};
    // FP64 with the sliced tensor-core sigma_3: it runs first and overwrites sigma
    const bool sliced = sizeof(T) == 8 && A.nsingle > 0 && B.nsingle > 0 && ctx->opt.f64_kernels != FCI_F64_FMA &&
                        sigma3_sliced_ok(ctx);
    if (parity != 0 && A.nsingle > 0) {
        // sigma = sigma_2 + parity sigma_2^T + sigma_3: FP64 with the sliced sigma_3 and the
        // double-float sigma_2, FP32 with the tensor-core kernels of large spaces
        if constexpr (sizeof(T) == 8) {
            if (sliced && sigma_ss_ok(ctx)) {  // sigma_2 as a dense sliced product
                static const char *const namesp[4] = {"sigma2_ss", "sigma1_sym", "slice_c", "sigma3_sliced"};
                const int rec = prof_begin(ctx, s, 4, namesp);
                FCI_CUDA(cudaMemsetAsync(sig, 0, sizeof(T) * (size_t)ctx->ndet, s));
                if (int rc = launch_sigma_ss(ctx, (const double *)C, (double *)sig, 2, s, rec, 0)) return rc;
                if (int rc = sym_pairs(sig, nsa, 8, parity, 0, s)) return rc;
                prof_mark(ctx, rec, 1, s);
                return launch_sigma3_sliced(ctx, C, sig, s, rec, 2, nullptr, 1);
            }
            if (sliced) {
                static const char *const namesp[4] = {"sigma2_cols", "sigma1_sym", "slice_c", "sigma3_sliced"};
                const int rec = prof_begin(ctx, s, 4, namesp);
                FCI_CUDA(cudaMemsetAsync(sig, 0, sizeof(T) * (size_t)ctx->ndet, s));
                const int R = pick_r(nsa);
                if (!R) return fail(FCI_ERR_ARG, "alpha string count too large for the sigma_2 kernel");
                void *k = R == 8 ? (void *)k_sigma2_cols_df<8> : R == 4 ? (void *)k_sigma2_cols_df<4>
                          : R == 2 ? (void *)k_sigma2_cols_df<2> : (void *)k_sigma2_cols_df<1>;
                FCI_CUDA(opt_in_max_smem(k, ctx->device));
                int64_t nsb_ = nsb;
                SpinTables At = A;
                const int *no_gate = nullptr;
                void *args[] = {(void *)&C, (void *)&sig, (void *)&At, (void *)&nsb_, (void *)&no_gate};
                FCI_CUDA(cudaLaunchKernel(k, dim3(ceil_div(nsb, R)), dim3(512), args, (size_t)R * nsa * sizeof(T), s));
                prof_mark(ctx, rec, 0, s);
                if (int rc = sym_pairs(sig, nsa, 8, parity, 0, s)) return rc;
                prof_mark(ctx, rec, 1, s);
                return launch_sigma3_sliced(ctx, C, sig, s, rec, 2, nullptr, 1);
            }
        } else if (same_tc) {
            static const char *const namesp[3] = {"sigma2_tc", "sigma1_sym", "sigma3_tc"};
            const int rec = prof_begin(ctx, s, 3, namesp);
            FCI_CUDA(cudaMemsetAsync(sig, 0, sizeof(float) * (size_t)ctx->ndet, s));
            if (int rc = launch_same_spin_tc(ctx, (const float *)C, (float *)sig, A, B, s)) return rc;
            prof_mark(ctx, rec, 0, s);
            if (int rc = sym_pairs(sig, nsa, 4, parity, 0, s)) return rc;
            prof_mark(ctx, rec, 1, s);
            if (int rc = launch_sigma3_tc(ctx, (const float *)C, (float *)sig, ctx->opt.f32_splits, s)) return rc;
            prof_mark(ctx, rec, 2, s);
            return FCI_OK;
        }
    }
    static const char *const names4ss[4] = {"slice_c", "sigma3_sliced", "sigma1_ss", "sigma2_ss"};
    const bool ss = sliced && sigma_ss_ok(ctx);
    const int rec = ss ? prof_begin(ctx, s, 4, names4ss)
                    : sliced ? prof_begin(ctx, s, 4, names4)
                    : same_tc ? prof_begin(ctx, s, 3, names3tc)
                    : fusedR ? prof_begin(ctx, s, 2, names2) : prof_begin(ctx, s, 3, names3);
    const int slot3 = (fusedR && !same_tc) ? 1 : 2;
    int slot = 0;  // next profiling slot of the staged same-spin kernels
    int add1 = 0;  // sigma_1 adds to what sigma_3 wrote
    if (sliced) {
        if constexpr (sizeof(T) == 8) {
            if (int rc = launch_sigma3_sliced(ctx, C, sig, s, rec, 0)) return rc;
            if (ss) return launch_sigma_ss(ctx, (const double *)C, (double *)sig, 3, s, rec, 2);
        }
        slot = 2;
        add1 = 1;
    }
    if (same_tc) {
        if constexpr (sizeof(T) == 4) {
            if (!ctx->ws32) return fail(FCI_ERR_STATE, "FP32 same-spin workspace missing (made at fci_init)");
            float *Ct = ctx->ws32, *Tt = ctx->ws32 + ctx->ndet;
            FCI_CUDA(cudaMemsetAsync(sig, 0, sizeof(float) * (size_t)ctx->ndet, s));
            // sigma_2: intermediate alpha strings, rows of C
            if (int rc = launch_same_spin_tc(ctx, (const float *)C, (float *)sig, A, B, s)) return rc;
            prof_mark(ctx, rec, 0, s);
            // sigma_1: intermediate beta strings, rows of C transposed
            const dim3 tb(32, 8);
            k_transpose_f32<false><<<dim3(ceil_div(nsb, 32), ceil_div(nsa, 32)), tb, 0, s>>>((const float *)C, Ct, nsa, nsb);
            FCI_CUDA(cudaMemsetAsync(Tt, 0, sizeof(float) * (size_t)ctx->ndet, s));
            if (int rc = launch_same_spin_tc(ctx, Ct, Tt, B, A, s)) return rc;
            k_transpose_f32<true><<<dim3(ceil_div(nsa, 32), ceil_div(nsb, 32)), tb, 0, s>>>(Tt, (float *)sig, nsb, nsa);
            FCI_CUDA(cudaGetLastError());
            prof_mark(ctx, rec, 1, s);
        }
    } else if (fusedR) {
        const size_t sm = (size_t)2 * fusedR * nsa * sizeof(float);
        void *k = fusedR == 8 ? (void *)k_sigma12_f32<8> : (void *)k_sigma12_f32<4>;
        FCI_CUDA(opt_in_max_smem(k, ctx->device));
        FCI_CUDA(cudaMemsetAsync(sig, 0, sizeof(float) * (size_t)nsa * (size_t)nsb, s));
        SpinTables St = A;
        const int *no_gate = nullptr;
        void *args[] = {(void *)&C, (void *)&sig, (void *)&St, (void *)&no_gate};
        FCI_CUDA(cudaLaunchKernel(k, dim3(ceil_div(nsa, fusedR)), dim3(512), args, sm, s));
        prof_mark(ctx, rec, 0, s);
    } else {
        {
            const int R = pick_r(nsb);
            if (!R) return fail(FCI_ERR_ARG, "beta string count too large for the sigma_1 kernel");
            const size_t sm = (size_t)R * nsb * sizeof(T);
            void *k = (sizeof(T) == 8 && ctx->opt.f64_kernels != FCI_F64_FMA)
                          ? (R == 8 ? (void *)k_sigma1_rows_df<8> : R == 4 ? (void *)k_sigma1_rows_df<4>
                             : R == 2 ? (void *)k_sigma1_rows_df<2> : (void *)k_sigma1_rows_df<1>)
                          : (R == 8 ? (void *)k_sigma1_rows<T, 8> : R == 4 ? (void *)k_sigma1_rows<T, 4>
                             : R == 2 ? (void *)k_sigma1_rows<T, 2> : (void *)k_sigma1_rows<T, 1>);
            FCI_CUDA(opt_in_max_smem(k, ctx->device));
            int64_t nsa_ = nsa;
            SpinTables Bt = B;
            const int *no_gate = nullptr;  // the double-float kernel's gate (others take one argument fewer)
            void *args[] = {(void *)&C, (void *)&sig, (void *)&Bt, (void *)&nsa_, (void *)&add1, (void *)&no_gate};
            FCI_CUDA(cudaLaunchKernel(k, dim3(ceil_div(nsa, R)), dim3(512), args, sm, s));
            prof_mark(ctx, rec, slot, s);
        }
        {
            const int R = pick_r(nsa);
            if (!R) return fail(FCI_ERR_ARG, "alpha string count too large for the sigma_2 kernel");
            const size_t sm = (size_t)R * nsa * sizeof(T);
            void *k = (sizeof(T) == 8 && ctx->opt.f64_kernels != FCI_F64_FMA)
                          ? (R == 8 ? (void *)k_sigma2_cols_df<8> : R == 4 ? (void *)k_sigma2_cols_df<4>
                             : R == 2 ? (void *)k_sigma2_cols_df<2> : (void *)k_sigma2_cols_df<1>)
                          : (R == 8 ? (void *)k_sigma2_cols<T, 8> : R == 4 ? (void *)k_sigma2_cols<T, 4>
                             : R == 2 ? (void *)k_sigma2_cols<T, 2> : (void *)k_sigma2_cols<T, 1>);
            FCI_CUDA(opt_in_max_smem(k, ctx->device));
            int64_t nsb_ = nsb;
            SpinTables At = A;
            const int *no_gate = nullptr;
            void *args[] = {(void *)&C, (void *)&sig, (void *)&At, (void *)&nsb_, (void *)&no_gate};
            FCI_CUDA(cudaLaunchKernel(k, dim3(ceil_div(nsb, R)), dim3(512), args, sm, s));
            prof_mark(ctx, rec, slot + 1, s);
        }
    }
    // sigma_3
    if (sliced) return FCI_OK;
    if (A.nsingle > 0 && B.nsingle > 0 && sizeof(T) == 4) {
        if (int rc = launch_sigma3_tc(ctx, (const float *)C, (float *)sig, ctx->opt.f32_splits, s)) return rc;
    } else if (A.nsingle > 0 && B.nsingle > 0) {
        if constexpr (sizeof(T) == 8) {
            size_t sm = sizeof(double) * (2 * nsb + ctx->npair) + sizeof(uint32_t) * A.nsingle;
            if (sm > lim) return fail(FCI_ERR_ARG, "beta string count too large for the FP64 sigma_3 row kernel");
            if (sm > 48 * 1024)
                FCI_CUDA(opt_in_max_smem((const void *)k_sigma3_exact, ctx->device));
            k_sigma3_exact<<<(unsigned)nsa, 512, sm, s>>>(C, sig, A, B, ctx->W, ctx->npair);
            FCI_CUDA(cudaGetLastError());
        }
    }
    prof_mark(ctx, rec, slot3, s);
    return FCI_OK;
}

// FP32 sigma of one instance of the batched engine, skipped on the device
// when *active == 0 (so that a captured graph serves any active set).  Only
// for one string space (fused sigma_1 + sigma_2) with the tensor-core sigma_3;
// sigma is zeroed even when the instance is skipped.  The kernels' shared
// memory limits are set once by prepare_sigma_f32_gated (outside any capture).
bool sigma_f32_gated_ok(const fci_ctx *ctx) {
    const SpinTables &A = ctx->A, &B = ctx->B;
    if (A.ne != B.ne || A.ns != B.ns || A.nsingle == 0 || B.nsingle == 0) return false;
    if ((size_t)2 * 4 * A.ns * sizeof(float) > smem_limit()) return false;
    return sigma3_tc_smem(ctx, ctx->opt.f32_splits) > 0;
}

static void *gated_sigma12(int64_t ns, size_t *sm) {
    const int R = (size_t)2 * 8 * ns * sizeof(float) <= smem_limit() ? 8 : 4;
    *sm = (size_t)2 * R * ns * sizeof(float);
    return R == 8 ? (void *)k_sigma12_f32<8> : (void *)k_sigma12_f32<4>;
}

int prepare_sigma_f32_gated(const fci_ctx *ctx) {
    size_t sm = 0;
    void *k = gated_sigma12(ctx->A.ns, &sm);
    FCI_CUDA(opt_in_max_smem(k, ctx->device));
    return prepare_sigma3_tc(ctx, ctx->opt.f32_splits);
}

int launch_sigma_f32_gated(fci_ctx *ctx, const float *C, float *sig, const int *active, cudaStream_t s) {
    const int64_t ns = ctx->A.ns;
    size_t sm = 0;
    void *k = gated_sigma12(ns, &sm);
    const int R = sm == (size_t)2 * 8 * ns * sizeof(float) ? 8 : 4;
    FCI_CUDA(cudaMemsetAsync(sig, 0, sizeof(float) * (size_t)ns * (size_t)ns, s));
    SpinTables St = ctx->A;
    void *args[] = {(void *)&C, (void *)&sig, (void *)&St, (void *)&active};
    FCI_CUDA(cudaLaunchKernel(k, dim3(ceil_div(ns, R)), dim3(512), args, sm, s));
    return launch_sigma3_tc(ctx, C, sig, ctx->opt.f32_splits, s, active);
}

// FP64 sigma of one batched instance with the single-instance kernels (sliced
// sigma_3, then the double-float sigma_1 and sigma_2 adding to it), every
// kernel skipped on the device when *active == 0, so that a captured graph
// serves any active set.  Shared-memory opt-ins: prepare_sigma_f64_gated.
static int df_rows(int64_t len) {
    for (int r = 8; r >= 1; r >>= 1)
        if ((size_t)r * len * sizeof(double) <= smem_limit()) return r;
    return 0;
}

static void *df_kernel1(int R) {
    return R == 8 ? (void *)k_sigma1_rows_df<8> : R == 4 ? (void *)k_sigma1_rows_df<4>
           : R == 2 ? (void *)k_sigma1_rows_df<2> : (void *)k_sigma1_rows_df<1>;
}
static void *df_kernel2(int R) {
    return R == 8 ? (void *)k_sigma2_cols_df<8> : R == 4 ? (void *)k_sigma2_cols_df<4>
           : R == 2 ? (void *)k_sigma2_cols_df<2> : (void *)k_sigma2_cols_df<1>;
}

bool sigma_f64_gated_ok(const fci_ctx *ctx) {
    return sigma3_sliced_ok(ctx) && df_rows(ctx->A.ns) > 0 && df_rows(ctx->B.ns) > 0;
}

int prepare_sigma_f64_gated(const fci_ctx *ctx) {
    if (int rc = prepare_sigma3_sliced(ctx)) return rc;
    FCI_CUDA(opt_in_max_smem(df_kernel1(df_rows(ctx->B.ns)), ctx->device));
    FCI_CUDA(opt_in_max_smem(df_kernel2(df_rows(ctx->A.ns)), ctx->device));
    return FCI_OK;
}

int launch_sigma_f64_gated(fci_ctx *ctx, const double *C, double *sig, const int *active, cudaStream_t s) {
    if (int rc = launch_sigma3_sliced(ctx, C, sig, s, -1, 0, active)) return rc;
    const SpinTables &A = ctx->A, &B = ctx->B;
    int64_t nsa = A.ns, nsb = B.ns;
    int add = 1;
    SpinTables At = A, Bt = B;
    const int R1 = df_rows(nsb), R2 = df_rows(nsa);
    void *a1[] = {(void *)&C, (void *)&sig, (void *)&Bt, (void *)&nsa, (void *)&add, (void *)&active};
    FCI_CUDA(cudaLaunchKernel(df_kernel1(R1), dim3(ceil_div(nsa, R1)), dim3(512), a1, (size_t)R1 * nsb * 8, s));
    void *a2[] = {(void *)&C, (void *)&sig, (void *)&At, (void *)&nsb, (void *)&active};
    FCI_CUDA(cudaLaunchKernel(df_kernel2(R2), dim3(ceil_div(nsb, R2)), dim3(512), a2, (size_t)R2 * nsa * 8, s));
    return FCI_OK;
}

int launch_sigma(fci_ctx *ctx, const void *c, void *sigma, int dtype, cudaStream_t s, int parity) {
    if (dtype == FCI_F64) return sigma_impl<double>(ctx, (const double *)c, (double *)sigma, s, parity);
    if (dtype == FCI_F32) return sigma_impl<float>(ctx, (const float *)c, (float *)sigma, s, parity);
    return fail(FCI_ERR_ARG, "dtype must be FCI_F64 or FCI_F32");
}

}  // namespace fci
