// Batched CASCI: many independent determinant-CI problems (different active
// spaces and integrals) solved together on one GPU.
//
// The paper reaches parallelism by cutting one CI vector into many TTSS
// batches and handing them to processors (Section 3.1); here the independent
// units are whole CASCI instances.  All instances run the Davidson scheme of
// Section 3.3 in lock-step (same subspace size m), so every step is one launch
// over all instances:
//  * vectors of all instances are stored back to back ("batch vectors"); the
//    element-wise and reduction kernels walk a list of <=256-element chunks,
//    each inside one instance, and reduce per instance in a fixed order;
//  * sigma of every instance comes from one persistent launch whose CTAs pull
//    (instance, alpha-row group) items, largest instances first, from a device
//    work counter; a row group of `tpr` threads builds sigma_1 + sigma_2 +
//    sigma_3 (Eq. 8) of one output alpha row with the same string-driven
//    formulas as the single-instance kernels;
//  * `tpr` is tuned per (norb, precision) at init by timing 32/64/128/256 on
//    the first instance of that size;
//  * the iterations are captured in CUDA graphs, up to eight iterations (to
//    the next thick restart) per graph, with every per-instance parameter and
//    every decision (convergence, refinement, expansion) in device memory; the
//    host launches one graph per chunk of iterations and reads back one
//    counter (the converged instances).
// An instance that converged is masked off; a slot an instance does not fill
// in an iteration (dropped correction, refinement step, or converged) is a
// zero vector whose projected-matrix diagonal is set to 1e30, so it never
// mixes into the lowest Ritz pairs.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "internal.cuh"

namespace fci {
namespace bt {

constexpr int kBlock = 256;
constexpr int kMaxSub = 32;
constexpr int kMaxRoots = 8;
constexpr int kChunk = 256;    // elementwise kernels: one CTA per chunk of <= kChunk elements
constexpr int kDChunk = 8192;  // dot products: 32 elements per thread before the block reduction
constexpr double kPad = 1e30;
constexpr int64_t kHybridMinDets = 32768;  // FP32 sigma of instances this large: single-instance kernels
constexpr int kRefinePeriod = 4;           // mixed precision: refinements on every 4th non-restart iteration

struct InstDev {
    SpinTables A, B;
    const double *W;
    const float *Wf;
    const double *hdiag;
    int64_t ndet, off;
    int npair, tpr;
    int stage_all;  // FP32: all off-diagonal alpha rows of an output row fit in shared memory at once
};

struct Chunk {
    int inst, len;
    int64_t start;
};

struct Item {
    int inst, row0;
};

__device__ __forceinline__ double flipb(double x, uint32_t sb) {
    return __longlong_as_double(__double_as_longlong(x) ^ ((long long)sb << 32));
}
__device__ __forceinline__ float flipb(float x, uint32_t sb) { return __int_as_float(__float_as_int(x) ^ (int)sb); }

template <typename T>
__device__ __forceinline__ T gv(const SpinTables &S, int64_t i);
template <>
__device__ __forceinline__ double gv<double>(const SpinTables &S, int64_t i) { return S.gval[i]; }
template <>
__device__ __forceinline__ float gv<float>(const SpinTables &S, int64_t i) { return S.gvalf[i]; }

template <typename T>
__device__ __forceinline__ T wv(const InstDev &d, int64_t i);
template <>
__device__ __forceinline__ double wv<double>(const InstDev &d, int64_t i) { return d.W[i]; }
template <>
__device__ __forceinline__ float wv<float>(const InstDev &d, int64_t i) { return d.Wf[i]; }

__device__ __forceinline__ void group_sync(int g, int tpr) {
    if (tpr == 32) {
        __syncwarp();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(tpr) : "memory");
    }
}

// Persistent batched sigma.  cin/cout: per-instance vector pointers; on:
// per-instance enable flags; row_elems: shared-memory elements per row group.
template <typename T>
__global__ void __launch_bounds__(kBlock, 1) k_bsigma(const InstDev *__restrict__ D, const Item *__restrict__ items,
                                                       int nitems, int *__restrict__ counter, const T *const *cin,
                                                       T *const *cout, const int *__restrict__ on, int row_elems) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *base = reinterpret_cast<T *>(smem_raw);
    __shared__ int s_item;
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= nitems) break;
        const Item I = items[it];
        if (!on[I.inst]) continue;
        const InstDev d = D[I.inst];
        const int tpr = d.tpr, g = tid / tpr, lt = tid % tpr;
        const int64_t row = (int64_t)I.row0 + g;
        if (row >= d.A.ns) continue;  // whole group idle; its barrier is private
        const int64_t nsb = d.B.ns;
        const int64_t nsa = d.A.ns;
        const T *C = cin[I.inst];
        T *S = cout[I.inst];
        T *cself = base + (int64_t)g * row_elems;
        T *ca = cself + nsb;
        T *acc = ca + nsb;
        T *wrow = acc + nsb;
        for (int64_t j = lt; j < nsb; j += tpr) cself[j] = C[row * nsb + j];
        group_sync(g, tpr);
        // sigma_2 (alpha-alpha rows of C) and sigma_1 (inside the row)
        for (int64_t j = lt; j < nsb; j += tpr) {
            T a = 0;
            for (int e = 0; e < d.A.nsame; ++e) {
                const int64_t ix = (int64_t)e * nsa + row;
                a = fma(gv<T>(d.A, ix), C[(int64_t)d.A.gcol[ix] * nsb + j], a);
            }
            for (int e = 0; e < d.B.nsame; ++e) {
                const int64_t ix = (int64_t)e * nsb + j;
                a = fma(gv<T>(d.B, ix), cself[d.B.gcol[ix]], a);
            }
            acc[j] = a;
        }
        if constexpr (sizeof(T) == 4) {
            if (d.stage_all && tpr == kBlock) {
                // FP32, one row group per CTA: stage every off-diagonal alpha row
                // C(J_a, :) and its signed integral row s_a (p_a|q) once, so each beta
                // entry is loaded once per determinant
                const int noff_a = d.A.ne * (d.A.nsingle / (d.A.ne > 0 ? d.A.ne : 1) - 1);
                const int noff_b = d.B.ne * (d.B.nsingle / (d.B.ne > 0 ? d.B.ne : 1) - 1);
                const int na4 = (noff_a + 3) & ~3;             // row length padded for float4
                // 16-byte aligned start (float4 loads): offset rounded up to 4 elements
                T *sR = cself + ((3 * nsb + d.npair + 3) & ~(int64_t)3);  // [nsb][na4]: C(J_a, j) at [j][a]
                T *sW = sR + (int64_t)na4 * nsb;               // [npair][na4]: s_a (p_a|q) at [q][a]
                int *sP = reinterpret_cast<int *>(sW + (int64_t)na4 * d.npair);  // [noff_a] entry of a
                group_sync(g, tpr);
                if (lt == 0) {
                    int o = 0;
                    for (int a = 0; a < d.A.nsingle; ++a) {
                        const uint32_t ea = d.A.tab[(int64_t)a * nsa + row];
                        if ((int64_t)ent_target(ea) != row) sP[o++] = (int)ea;
                    }
                }
                for (int q = lt; q < d.npair; q += tpr) {
                    T w = 0;
                    for (int a = 0; a < d.A.nsingle; ++a) {
                        const uint32_t ea = d.A.tab[(int64_t)a * nsa + row];
                        if ((int64_t)ent_target(ea) == row) w += wv<T>(d, (int64_t)ent_pair(ea) * d.npair + q);
                    }
                    wrow[q] = w;
                }
                group_sync(g, tpr);
                for (int64_t t = lt; t < (int64_t)na4 * nsb; t += tpr) {
                    const int a = (int)(t / nsb);
                    const int64_t j = t % nsb;
                    sR[j * na4 + a] = a < noff_a ? C[(int64_t)ent_target((uint32_t)sP[a]) * nsb + j] : T(0);
                }
                for (int t = lt; t < na4 * d.npair; t += tpr) {
                    const int a = t / d.npair, q = t % d.npair;
                    T w = 0;
                    if (a < noff_a) {
                        const uint32_t ea = (uint32_t)sP[a];
                        w = wv<T>(d, (int64_t)ent_pair(ea) * d.npair + q);
                        if (ent_negative(ea)) w = -w;
                    }
                    sW[q * na4 + a] = w;
                }
                group_sync(g, tpr);
                for (int64_t j = lt; j < nsb; j += tpr) {
                    T v = acc[j];
                    // merged alpha diagonal against every beta entry
                    for (int b = 0; b < d.B.nsingle; ++b) {
                        const uint32_t eb = d.B.tab[(int64_t)b * nsb + j];
                        v = fma(flipb(wrow[ent_pair(eb)], eb & 0x80000000u), cself[ent_target(eb)], v);
                    }
                    // off-diagonal alpha against the merged beta diagonal
                    for (int a = 0; a < noff_a; ++a) {
                        const uint32_t ea = (uint32_t)sP[a];
                        const T w = (T)d.B.wdiag[(int64_t)ent_pair(ea) * nsb + j];
                        v = fma(ent_negative(ea) ? -w : w, sR[j * na4 + a], v);
                    }
                    // off-diagonal alpha against off-diagonal beta: contiguous over a
                    for (int b = 0; b < noff_b; ++b) {
                        const uint32_t eb = d.B.tabo[(int64_t)b * nsb + j];
                        const float4 *wq = reinterpret_cast<const float4 *>(sW + (int64_t)ent_pair(eb) * na4);
                        const float4 *rq = reinterpret_cast<const float4 *>(sR + (int64_t)ent_target(eb) * na4);
                        float t = 0.f;
                        for (int a4 = 0; a4 < na4 / 4; ++a4) {
                            const float4 x = wq[a4], y = rq[a4];
                            t = fmaf(x.x, y.x, t);
                            t = fmaf(x.y, y.y, t);
                            t = fmaf(x.z, y.z, t);
                            t = fmaf(x.w, y.w, t);
                        }
                        v += ent_negative(eb) ? -t : t;
                    }
                    S[row * nsb + j] = v;
                }
                group_sync(g, tpr);
                continue;
            }
        }
        // sigma_3 with the diagonal replacements merged (as in the single-instance
        // FP64 kernel): first one pass over C(I_a, :) with the summed integral
        // rows of the alpha E_kk, then the off-diagonal alpha entries against the
        // off-diagonal beta entries plus sum_l (p_a|ll) C(J_a, I_b)
        group_sync(g, tpr);
        for (int q = lt; q < d.npair; q += tpr) {
            T w = 0;
            for (int a = 0; a < d.A.nsingle; ++a) {
                const uint32_t ea = d.A.tab[(int64_t)a * nsa + row];
                if ((int64_t)ent_target(ea) == row) w += wv<T>(d, (int64_t)ent_pair(ea) * d.npair + q);
            }
            wrow[q] = w;
        }
        group_sync(g, tpr);
        for (int64_t j = lt; j < nsb; j += tpr) {
            T v = 0;
            for (int b = 0; b < d.B.nsingle; ++b) {
                const uint32_t eb = d.B.tab[(int64_t)b * nsb + j];
                v = fma(flipb(wrow[ent_pair(eb)], eb & 0x80000000u), cself[ent_target(eb)], v);
            }
            acc[j] += v;
        }
        const int noff_b = d.B.ne * (int)(d.npair > 0 ? (d.B.nsingle / (d.B.ne > 0 ? d.B.ne : 1) - 1) : 0);
        for (int a = 0; a < d.A.nsingle; ++a) {
            const uint32_t ea = d.A.tab[(int64_t)a * nsa + row];
            const int64_t ja = ent_target(ea);
            if (ja == row) continue;
            const int pa = ent_pair(ea);
            group_sync(g, tpr);
            for (int64_t j = lt; j < nsb; j += tpr) ca[j] = C[ja * nsb + j];
            for (int q = lt; q < d.npair; q += tpr) wrow[q] = wv<T>(d, (int64_t)pa * d.npair + q);
            group_sync(g, tpr);
            const double *wd = d.B.wdiag + (int64_t)pa * nsb;
            for (int64_t j = lt; j < nsb; j += tpr) {
                T v = (T)wd[j] * ca[j];
                for (int b = 0; b < noff_b; ++b) {
                    const uint32_t eb = d.B.tabo[(int64_t)b * nsb + j];
                    v = fma(flipb(wrow[ent_pair(eb)], eb & 0x80000000u), ca[ent_target(eb)], v);
                }
                acc[j] += ent_negative(ea) ? -v : v;
            }
        }
        for (int64_t j = lt; j < nsb; j += tpr) S[row * nsb + j] = acc[j];
        group_sync(g, tpr);
    }
}

// ---- flat batch-vector kernels (one CTA per chunk) ---------------------------

// partial[c][g*8 + j] = sum over chunk c of X_{g*8+j} . y (j < 8); block
// index = c * G + g.  As in the single-instance solver the FP64 pipe bounds
// these products, so every element costs one FMA and a block keeps only 8
// accumulators per thread.
__global__ void __launch_bounds__(kBlock) k_bdots(const Chunk *__restrict__ ch, const int *__restrict__ on,
                                                  const double *__restrict__ X, int64_t ntot, int m, int G,
                                                  const double *__restrict__ y, double *__restrict__ partial) {
    const int cidx = blockIdx.x / G, g = blockIdx.x % G;
    const Chunk c = ch[cidx];
    const int i0 = g * 8, mg = m - i0 < 8 ? m - i0 : 8;
    double acc[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j] = 0.0;
    if (on[c.inst])
        for (int t = threadIdx.x; t < c.len; t += kBlock) {
            const int64_t idx = c.start + t;
            const double yv = y[idx];
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (j < mg) acc[j] = fma(X[(int64_t)(i0 + j) * ntot + idx], yv, acc[j]);
        }
    __shared__ double red[8][kBlock / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        double v = acc[j];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[j][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < mg) {
        double v = 0.0;
        for (int w = 0; w < kBlock / 32; ++w) v += red[threadIdx.x][w];
        partial[(int64_t)cidx * 32 + i0 + threadIdx.x] = v;
    }
}

// out[i*os + j*js] = sum of partial[c*STRIDE + j] over instance i's chunks:
// one CTA per instance, a strided sum per thread and a fixed-order tree.
template <int STRIDE>
__global__ void __launch_bounds__(kBlock) k_breduce(const int *__restrict__ cfirst, const int *__restrict__ on,
                                                    const double *__restrict__ partial, int m,
                                                    double *__restrict__ out, int64_t os, int64_t js) {
    const int i = blockIdx.x;
    if (!on[i]) return;
    __shared__ double red[kBlock / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c0 = cfirst[i], c1 = cfirst[i + 1];
    for (int j = 0; j < m; ++j) {
        double v = 0.0;
        for (int c = c0 + threadIdx.x; c < c1; c += kBlock) v += partial[(int64_t)c * STRIDE + j];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < kBlock / 32; ++w) t += red[w];
            out[i * os + j * js] = t;
        }
        __syncthreads();
    }
}

// y = beta*y + alpha * sum_j coef[i*cs + j*cj] X_j     (masked by on)
__global__ void __launch_bounds__(kBlock) k_blincomb(const Chunk *__restrict__ ch, const int *__restrict__ on,
                                                     const double *__restrict__ X, int64_t ntot, int m,
                                                     const double *__restrict__ coef, int64_t cs, int64_t cj,
                                                     double alpha, double beta, double *__restrict__ y) {
    const Chunk c = ch[blockIdx.x];
    if (!on[c.inst] || threadIdx.x >= c.len) return;
    const int64_t idx = c.start + threadIdx.x;
    const double *cf = coef + c.inst * cs;
    double v = 0.0;
    for (int j = 0; j < m; ++j) v += cf[j * cj] * X[(int64_t)j * ntot + idx];
    y[idx] = (beta == 0.0 ? 0.0 : beta * y[idx]) + alpha * v;
}

// r = hx - w x ; t = -r/(diag - w) with the 1e-8 floor; partial[c] = |r|^2 over the chunk
__global__ void __launch_bounds__(kBlock) k_bresid(const Chunk *__restrict__ ch, const int *__restrict__ on,
                                                   const InstDev *__restrict__ D, const double *__restrict__ x,
                                                   const double *__restrict__ hx, const double *__restrict__ w,
                                                   int wstride, double *__restrict__ t, double *__restrict__ partial) {
    const Chunk c = ch[blockIdx.x];
    double a = 0.0;
    if (on[c.inst] && threadIdx.x < c.len) {
        const int64_t idx = c.start + threadIdx.x;
        const double e = w[(int64_t)c.inst * wstride];
        const double r = hx[idx] - e * x[idx];
        double dd = D[c.inst].hdiag[idx - D[c.inst].off] - e;
        if (fabs(dd) < 1e-8) dd = dd < 0 ? -1e-8 : 1e-8;
        t[idx] = -r / dd;
        a = r * r;
    }
    __shared__ double red[kBlock / 32];
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = 0.0;
        for (int k = 0; k < kBlock / 32; ++k) v += red[k];
        partial[(int64_t)blockIdx.x * 8] = v;
    }
}

// y *= 1/sqrt(nrm2[i]) if the norm is at least 1e-10, else y = 0 (keep[i] = 0)
__global__ void __launch_bounds__(kBlock) k_bnormalise(const Chunk *__restrict__ ch, const int *__restrict__ on,
                                                       const double *__restrict__ nrm2, double *__restrict__ y) {
    const Chunk c = ch[blockIdx.x];
    if (!on[c.inst] || threadIdx.x >= c.len) return;
    const int64_t idx = c.start + threadIdx.x;
    const double nn = sqrt(nrm2[c.inst]);
    y[idx] = nn >= 1e-10 ? y[idx] / nn : 0.0;
}

__global__ void __launch_bounds__(kBlock) k_bcopy(const Chunk *__restrict__ ch, const int *__restrict__ on,
                                                  const double *__restrict__ a, double *__restrict__ b,
                                                  int zero_when_off) {
    const Chunk c = ch[blockIdx.x];
    if (threadIdx.x >= c.len) return;
    const int64_t idx = c.start + threadIdx.x;
    if (on[c.inst]) b[idx] = a[idx];
    else if (zero_when_off) b[idx] = 0.0;
}

__global__ void k_d2f(const double *__restrict__ a, float *__restrict__ b, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}
__global__ void k_f2d(const float *__restrict__ a, double *__restrict__ b, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (double)a[i];
}

// S_j += V_i[j][k] * delta for j < m (rank-1 refinement), masked
__global__ void __launch_bounds__(kBlock) k_brank1(const Chunk *__restrict__ ch, const int *__restrict__ on,
                                                   double *__restrict__ S, int64_t ntot, int m,
                                                   const double *__restrict__ V, int k,
                                                   const double *__restrict__ delta) {
    const Chunk c = ch[blockIdx.x];
    if (!on[c.inst] || threadIdx.x >= c.len) return;
    const int64_t idx = c.start + threadIdx.x;
    const double dl = delta[idx];
    const double *Vi = V + (int64_t)c.inst * kMaxSub * kMaxSub;
    for (int j = 0; j < m; ++j) S[(int64_t)j * ntot + idx] += Vi[j * m + k] * dl;
}

// A_i[r][c] += g_i[r] * V_i[c][k]
__global__ void k_brank1_proj(const int *__restrict__ on, double *__restrict__ A, const double *__restrict__ g,
                              const double *__restrict__ V, int m, int k) {
    const int i = blockIdx.x;
    if (!on[i]) return;
    double *Ai = A + (int64_t)i * kMaxSub * kMaxSub;
    const double *gi = g + (int64_t)i * kMaxSub;
    const double *Vi = V + (int64_t)i * kMaxSub * kMaxSub;
    for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
        const int r = t / m, cc = t % m;
        Ai[r * kMaxSub + cc] += gi[r] * Vi[cc * m + k];
    }
}

// slot j of instance i: if the new vector was dropped (norm below 1e-10) or the
// instance is masked, make it a padding slot: A[j][*] = A[*][j] = 0, A[j][j] = kPad
__global__ void k_bpad(const int *__restrict__ on, const double *__restrict__ nrm2, double *__restrict__ A, int j,
                       int ninst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ninst) return;
    const bool pad = !on[i] || !(sqrt(nrm2[i]) >= 1e-10);
    if (!pad) return;
    double *Ai = A + (int64_t)i * kMaxSub * kMaxSub;
    for (int t = 0; t < kMaxSub; ++t) {
        Ai[j * kMaxSub + t] = 0.0;
        Ai[t * kMaxSub + j] = 0.0;
    }
    Ai[j * kMaxSub + j] = kPad;
}

// Cyclic Jacobi per instance (textbook; ascending order, stable).
__global__ void k_bjacobi(const int *__restrict__ on, const double *__restrict__ Aall, int m,
                          double *__restrict__ wall, double *__restrict__ Vall) {
    const int i = blockIdx.x;
    if (!on[i]) return;
    const double *A = Aall + (int64_t)i * kMaxSub * kMaxSub;
    double *w = wall + (int64_t)i * kMaxSub;
    double *V = Vall + (int64_t)i * kMaxSub * kMaxSub;
    __shared__ double a[kMaxSub][kMaxSub + 1];
    __shared__ double v[kMaxSub][kMaxSub + 1];
    __shared__ int order[kMaxSub];
    const int tid = threadIdx.x;
    for (int t = tid; t < m * m; t += blockDim.x) {
        const int r = t / m, c = t % m;
        a[r][c] = 0.5 * (A[r * kMaxSub + c] + A[c * kMaxSub + r]);
        v[r][c] = (r == c) ? 1.0 : 0.0;
    }
    __syncthreads();
    // Parallel cyclic Jacobi with round-robin pair ordering: each step rotates
    // m/2 disjoint pairs at once (rotations on disjoint index pairs commute).
    // A rotation is skipped when |a_pq| < 1e-14 (|a_pp| + |a_qq|); the sweeps
    // stop after a sweep without rotation (60 at most).
    __shared__ int rotated;
    __shared__ int pos[kMaxSub + 1];
    __shared__ int pp[kMaxSub / 2 + 1], pq[kMaxSub / 2 + 1];
    __shared__ double pc[kMaxSub / 2 + 1], psn[kMaxSub / 2 + 1];
    const int me = m + (m & 1);  // even number of players; index m is a dummy when m is odd
    const int half = me / 2;
    for (int t = tid; t < me; t += blockDim.x) pos[t] = t;
    __syncthreads();
    for (int sweep = 0; sweep < 60; ++sweep) {
        if (tid == 0) rotated = 0;
        __syncthreads();
        for (int step = 0; step < me - 1; ++step) {
            for (int k = tid; k < half; k += blockDim.x) {
                int p = pos[k], q = pos[me - 1 - k];
                if (p > q) { const int t2 = p; p = q; q = t2; }
                double c = 1.0, sn = 0.0;
                if (q < m) {
                    const double apq = a[p][q];
                    if (fabs(apq) > 1e-14 * (fabs(a[p][p]) + fabs(a[q][q]))) {
                        rotated = 1;
                        const double theta = (a[q][q] - a[p][p]) / (2.0 * apq);
                        const double tt = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                        c = 1.0 / sqrt(tt * tt + 1.0);
                        sn = tt * c;
                    }
                }
                pp[k] = p;
                pq[k] = q;
                pc[k] = c;
                psn[k] = sn;
            }
            __syncthreads();
            // columns: a <- a J
            for (int t = tid; t < half * m; t += blockDim.x) {
                const int k = t / m, r = t % m;
                if (psn[k] == 0.0) continue;
                const int p = pp[k], q = pq[k];
                const double c = pc[k], sn = psn[k];
                const double arp = a[r][p], arq = a[r][q];
                a[r][p] = c * arp - sn * arq;
                a[r][q] = sn * arp + c * arq;
            }
            __syncthreads();
            // rows: a <- J^T a ; eigenvectors v <- v J
            for (int t = tid; t < half * m; t += blockDim.x) {
                const int k = t / m, r = t % m;
                if (psn[k] == 0.0) continue;
                const int p = pp[k], q = pq[k];
                const double c = pc[k], sn = psn[k];
                const double apr = a[p][r], aqr = a[q][r];
                a[p][r] = c * apr - sn * aqr;
                a[q][r] = sn * apr + c * aqr;
                const double vrp = v[r][p], vrq = v[r][q];
                v[r][p] = c * vrp - sn * vrq;
                v[r][q] = sn * vrp + c * vrq;
            }
            __syncthreads();
            // next round-robin pairing: player 0 stays, the others rotate
            if (tid == 0) {
                const int last = pos[me - 1];
                for (int t = me - 1; t > 1; --t) pos[t] = pos[t - 1];
                pos[1] = last;
            }
            __syncthreads();
        }
        if (!rotated) break;
    }
    if (tid == 0) {
        for (int r = 0; r < m; ++r) order[r] = r;
        for (int r = 1; r < m; ++r) {
            const int o = order[r];
            int j = r - 1;
            while (j >= 0 && a[order[j]][order[j]] > a[o][o]) {
                order[j + 1] = order[j];
                --j;
            }
            order[j + 1] = o;
        }
    }
    __syncthreads();
    for (int t = tid; t < m; t += blockDim.x) w[t] = a[order[t]][order[t]];
    for (int t = tid; t < m * m; t += blockDim.x) {
        const int r = t / m, k = t % m;
        V[r * m + k] = v[r][order[k]];
    }
}

// nroots smallest diagonal entries per instance (ties: lower index) -> unit vectors in B_k
__global__ void k_bguess(const InstDev *__restrict__ D, int nroots, double *__restrict__ Bv, int64_t ntot) {
    const int i = blockIdx.x;
    const InstDev d = D[i];
    __shared__ double sb[256];
    __shared__ int64_t si[256];
    __shared__ int64_t chosen[kMaxRoots];
    for (int k = 0; k < nroots; ++k) {
        double best = INFINITY;
        int64_t bi = INT64_MAX;
        for (int64_t r = threadIdx.x; r < d.ndet; r += blockDim.x) {
            bool skip = false;
            for (int c = 0; c < k; ++c) skip |= chosen[c] == r;
            const double v = d.hdiag[r];
            if (!skip && (v < best || (v == best && r < bi))) {
                best = v;
                bi = r;
            }
        }
        sb[threadIdx.x] = best;
        si[threadIdx.x] = bi;
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) {
                const double v = sb[threadIdx.x + s];
                const int64_t j = si[threadIdx.x + s];
                if (v < sb[threadIdx.x] || (v == sb[threadIdx.x] && j < si[threadIdx.x])) {
                    sb[threadIdx.x] = v;
                    si[threadIdx.x] = j;
                }
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) chosen[k] = si[0];
        __syncthreads();
        double *b = Bv + (int64_t)k * ntot + d.off;
        for (int64_t r = threadIdx.x; r < d.ndet; r += blockDim.x) b[r] = (r == chosen[k]) ? 1.0 : 0.0;
        __syncthreads();
    }
}

}  // namespace bt
}  // namespace fci

using namespace fci;
using namespace fci::bt;

struct fci_batch {
    int device = 0;
    cudaStream_t stream = nullptr;
    fci_options opt{};
    std::vector<fci_ctx *> ctx;
    std::vector<int64_t> off;  // ninst + 1
    int64_t ntot = 0;
    int ninst = 0, nsm = 0;
    InstDev *d_inst = nullptr;
    std::vector<InstDev> h_inst;
    Chunk *d_chunks = nullptr;   // <= 256 elements each (element-wise kernels)
    int nchunks = 0;
    int *d_cfirst = nullptr;
    Chunk *d_dchunks = nullptr;  // <= kDChunk elements each (reductions)
    int ndchunks = 0;
    int *d_dcfirst = nullptr;
    Item *d_items = nullptr;
    int nitems = 0;
    int *d_counter = nullptr;
    int row_elems64 = 0, row_elems32 = 0;
    size_t smem64 = 0, smem32 = 0;
    std::vector<int> tune;  // triples (norb, dtype, tpr)
    // instances whose sigma runs the single-instance kernels gated by their
    // active flag (FP32: fused sigma_1 + sigma_2, tensor-core sigma_3; FP64:
    // sliced sigma_3, double-float sigma_1 and sigma_2); their work items come
    // first in d_items
    std::vector<int> hyb;
    int nitems_hyb = 0;
    // sigma call plumbing
    void **d_cin = nullptr, **d_cout = nullptr;
    int *d_on_all = nullptr;
    int64_t stats[4] = {0, 0, 0, 0};  // iterations, sigma launches, graph launches, host synchronisations
    std::vector<std::pair<void *, size_t>> allocs;
};

namespace {

template <typename P>
P *balloc(fci_batch *b, size_t count, int *rc) {
    if (*rc || count == 0) return nullptr;
    b->allocs.push_back({nullptr, 0});  // the slot exists before the allocation (a throw leaks nothing)
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, sizeof(P) * count);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *rc = fail(FCI_ERR_OOM, "batched CASCI: device allocation failed");
        return nullptr;
    }
    b->allocs.back() = {p, sizeof(P) * count};
    return (P *)p;
}

unsigned grid_flat(int64_t n) {
    int64_t g = (n + 255) / 256;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, 4 * 152));
}

// Work items with the instances' current tpr: the single-instance-kernel
// instances first, then the others, largest instances first in each group.
int build_items(fci_batch *b, int *rc) {
    std::vector<int> order(b->ninst), is_hyb(b->ninst, 0);
    for (int i : b->hyb) is_hyb[i] = 1;
    for (int i = 0; i < b->ninst; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        if (is_hyb[x] != is_hyb[y]) return is_hyb[x] > is_hyb[y];
        return b->h_inst[x].ndet > b->h_inst[y].ndet;
    });
    std::vector<Item> items;
    b->nitems_hyb = 0;
    for (int i : order) {
        const int R = kBlock / b->h_inst[i].tpr;
        for (int64_t r = 0; r < b->h_inst[i].A.ns; r += R) {
            items.push_back({i, (int)r});
            if (is_hyb[i]) ++b->nitems_hyb;
        }
    }
    b->nitems = (int)items.size();
    if (!b->d_items) b->d_items = balloc<Item>(b, items.size(), rc);
    if (*rc) return *rc;
    FCI_CUDA(cudaMemcpy(b->d_items, items.data(), sizeof(Item) * items.size(), cudaMemcpyHostToDevice));
    FCI_CUDA(cudaMemcpy(b->d_inst, b->h_inst.data(), sizeof(InstDev) * b->ninst, cudaMemcpyHostToDevice));
    return FCI_OK;
}

template <typename T>
int launch_bsigma(fci_batch *b, const int *d_on, const T *const *d_in, T *const *d_out, cudaStream_t s,
                  const Item *items, int nitems) {
    FCI_CUDA(cudaMemsetAsync(b->d_counter, 0, sizeof(int), s));
    const size_t smem = sizeof(T) == 8 ? b->smem64 : b->smem32;
    const int re = sizeof(T) == 8 ? b->row_elems64 : b->row_elems32;
    k_bsigma<T><<<b->nsm, kBlock, smem, s>>>(b->d_inst, items, nitems, b->d_counter, d_in, d_out, d_on, re);
    FCI_CUDA(cudaGetLastError());
    return FCI_OK;
}

}  // namespace

extern "C" {

int fci_batch_free(fci_batch *b) {
    if (!b) return FCI_OK;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (auto &a : b->allocs)
        if (a.first) cudaFree(a.first);
    for (auto *c : b->ctx) fci_free(c);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
    return FCI_OK;
}

int64_t fci_batch_offset(fci_batch *b, int i) {
    if (!b || i < 0 || i > b->ninst) return -1;
    return b->off[i];
}

int fci_batch_tuning(fci_batch *b, int *out, int cap, int *count) {
    if (!b) return fail(FCI_ERR_ARG, "batch is NULL");
    const int n = (int)b->tune.size() / 3;
    if (count) *count = n;
    if (out)
        for (int i = 0; i < n && i < cap; ++i)
            for (int k = 0; k < 3; ++k) out[3 * i + k] = b->tune[3 * i + k];
    return FCI_OK;
}

int64_t fci_batch_stats(fci_batch *b, int what) {
    if (!b || what < 0 || what > 3) return -1;
    return b->stats[what];
}

static int batch_init_impl(fci_batch **out, int ninst, const fci_instance *inst, const fci_options *opt);

int fci_batch_init(fci_batch **out, int ninst, const fci_instance *inst, const fci_options *opt) {
    if (out) *out = nullptr;
    try {
        return batch_init_impl(out, ninst, inst, opt);
    } catch (const std::bad_alloc &) {  // host tables: no exception crosses the C ABI
        if (out && *out) {
            fci_batch_free(*out);
            *out = nullptr;
        }
        return fail(FCI_ERR_OOM, "batched CASCI: host allocation failed");
    }
}

// The batch under construction is kept in a guard that frees it (and every
// context and buffer it holds) unless initialisation completes.
struct BatchGuard {
    fci_batch *b = nullptr;
    ~BatchGuard() {
        if (b) fci_batch_free(b);
    }
};

static int batch_init_impl(fci_batch **out, int ninst, const fci_instance *inst, const fci_options *opt) {
    if (!out || !inst || ninst < 1) return fail(FCI_ERR_ARG, "batched CASCI: bad arguments");
    *out = nullptr;
    fci_options o;
    fci_default_options(&o);
    if (opt) {
        if (opt->struct_size != (int)sizeof(fci_options)) return fail(FCI_ERR_ARG, "fci_options.struct_size mismatch");
        o = *opt;
    }
    for (int i = 0; i < ninst; ++i)
        if (inst[i].norb < 1 || inst[i].norb > 16) return fail(FCI_ERR_ARG, "batched CASCI: norb must be in 1..16");
    fci_batch *b = new (std::nothrow) fci_batch();
    if (!b) return fail(FCI_ERR_OOM, "host allocation failed");
    BatchGuard guard;
    guard.b = b;
    b->opt = o;
    b->ninst = ninst;
    int rc = FCI_OK;
    {
        int dev = o.device;
        if (dev < 0) FCI_CUDA(cudaGetDevice(&dev));
        b->device = dev;
        FCI_CUDA(cudaSetDevice(dev));
        FCI_CUDA(cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev));
        FCI_CUDA(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
    }
    fci_options oi = o;
    oi.device = b->device;
    b->off.assign(ninst + 1, 0);
    int maxnsb = 0, maxnpair = 0;
    for (int i = 0; i < ninst && rc == FCI_OK; ++i) {
        fci_ctx *c = nullptr;
        rc = fci_init(&c, inst[i].norb, inst[i].nalpha, inst[i].nbeta, inst[i].h1, inst[i].eri, &oi);
        if (rc) break;
        b->ctx.push_back(c);
        InstDev d;
        d.A = c->A;
        d.B = c->B;
        d.W = c->W;
        d.Wf = c->Wf;
        d.hdiag = c->hdiag;
        d.ndet = c->ndet;
        d.off = b->off[i];
        d.npair = c->npair;
        d.tpr = 128;
        b->h_inst.push_back(d);
        b->off[i + 1] = b->off[i] + c->ndet;
        maxnsb = std::max<int>(maxnsb, (int)c->B.ns);
        maxnpair = std::max(maxnpair, c->npair);
    }
    if (rc) {
        std::string msg = fci_last_error();
        guard.b = nullptr;
        fci_batch_free(b);
        set_error(msg);
        return rc;
    }
    b->ntot = b->off[ninst];
    // chunks of <= 256 elements inside one instance
    std::vector<Chunk> ch;
    std::vector<int> cfirst(ninst + 1, 0);
    for (int i = 0; i < ninst; ++i) {
        cfirst[i] = (int)ch.size();
        for (int64_t s0 = 0; s0 < b->h_inst[i].ndet; s0 += kChunk)
            ch.push_back({i, (int)std::min<int64_t>(kChunk, b->h_inst[i].ndet - s0), b->off[i] + s0});
    }
    cfirst[ninst] = (int)ch.size();
    b->nchunks = (int)ch.size();
    std::vector<Chunk> dch;
    std::vector<int> dcfirst(ninst + 1, 0);
    for (int i = 0; i < ninst; ++i) {
        dcfirst[i] = (int)dch.size();
        for (int64_t s0 = 0; s0 < b->h_inst[i].ndet; s0 += kDChunk)
            dch.push_back({i, (int)std::min<int64_t>(kDChunk, b->h_inst[i].ndet - s0), b->off[i] + s0});
    }
    dcfirst[ninst] = (int)dch.size();
    b->ndchunks = (int)dch.size();
    b->d_chunks = balloc<Chunk>(b, ch.size(), &rc);
    b->d_cfirst = balloc<int>(b, ninst + 1, &rc);
    b->d_dchunks = balloc<Chunk>(b, dch.size(), &rc);
    b->d_dcfirst = balloc<int>(b, ninst + 1, &rc);
    b->d_inst = balloc<InstDev>(b, ninst, &rc);
    b->d_counter = balloc<int>(b, 1, &rc);
    b->d_cin = balloc<void *>(b, ninst, &rc);
    b->d_cout = balloc<void *>(b, ninst, &rc);
    b->d_on_all = balloc<int>(b, ninst, &rc);
    if (rc) return rc;
    FCI_CUDA(cudaMemcpy(b->d_chunks, ch.data(), sizeof(Chunk) * ch.size(), cudaMemcpyHostToDevice));
    FCI_CUDA(cudaMemcpy(b->d_cfirst, cfirst.data(), sizeof(int) * (ninst + 1), cudaMemcpyHostToDevice));
    FCI_CUDA(cudaMemcpy(b->d_dchunks, dch.data(), sizeof(Chunk) * dch.size(), cudaMemcpyHostToDevice));
    FCI_CUDA(cudaMemcpy(b->d_dcfirst, dcfirst.data(), sizeof(int) * (ninst + 1), cudaMemcpyHostToDevice));
    std::vector<int> ones(ninst, 1);
    FCI_CUDA(cudaMemcpy(b->d_on_all, ones.data(), sizeof(int) * ninst, cudaMemcpyHostToDevice));
    // shared memory: up to 8 row groups (tpr = 32) of 3 rows + one integral row
    b->row_elems64 = (3 * maxnsb + maxnpair + 1) & ~1;
    b->row_elems32 = (3 * maxnsb + maxnpair + 3) & ~3;
    b->smem64 = sizeof(double) * 8 * b->row_elems64;
    b->smem32 = sizeof(float) * 8 * b->row_elems32;
    // FP32 stage-all mode (one row group of 256 threads): cself, ca, acc, wrow,
    // then all off-diagonal alpha rows and their integral rows
    for (int i = 0; i < ninst; ++i) {
        const int64_t nsb_i = b->h_inst[i].B.ns;
        const int noff_a = b->h_inst[i].A.ne * ((int)b->h_inst[i].A.ns > 0 && b->h_inst[i].A.ne > 0
                                                    ? b->h_inst[i].A.nsingle / b->h_inst[i].A.ne - 1
                                                    : 0);
        const int na4 = (noff_a + 3) & ~3;
        const int64_t elems = ((3 * nsb_i + b->h_inst[i].npair + 3) & ~(int64_t)3) + (int64_t)na4 * nsb_i +
                              (int64_t)na4 * b->h_inst[i].npair + noff_a;
        const size_t bytes = sizeof(float) * (size_t)elems;
        b->h_inst[i].stage_all = (noff_a > 0 && bytes <= 200 * 1024) ? 1 : 0;
        if (b->h_inst[i].stage_all) b->smem32 = std::max(b->smem32, bytes);
    }
    {  // opted in to the device maximum: other batches launch the same kernels
        cudaError_t e1 = opt_in_max_smem((const void *)k_bsigma<double>, b->device);
        cudaError_t e2 = opt_in_max_smem((const void *)k_bsigma<float>, b->device);
        if (e1 != cudaSuccess || e2 != cudaSuccess) {
            return cuda_fail(e1 != cudaSuccess ? e1 : e2, "batched CASCI: shared-memory opt-in");
        }
    }
    if (b->smem64 > 227 * 1024) {
        return fail(FCI_ERR_ARG, "batched CASCI: an instance is too large for the batched sigma kernel");
    }

    // ---- autotuner: threads per alpha row for each (norb, dtype) ----
    {
        const int cands[4] = {32, 64, 128, 256};
        std::map<int, int> first_of;  // norb -> first instance index
        for (int i = 0; i < ninst; ++i)
            if (!first_of.count(inst[i].norb)) first_of[inst[i].norb] = i;
        // scratch vectors for the largest tuning instance
        int64_t maxn = 0;
        for (auto &kv : first_of) maxn = std::max<int64_t>(maxn, b->h_inst[kv.second].ndet);
        double *x64 = balloc<double>(b, maxn, &rc), *y64 = balloc<double>(b, maxn, &rc);
        float *x32 = balloc<float>(b, maxn, &rc), *y32 = balloc<float>(b, maxn, &rc);
        Item *titems = balloc<Item>(b, 1 << 16, &rc);
        int *ton = balloc<int>(b, ninst, &rc);
        if (rc) {
            return rc;
        }
        cudaMemsetAsync(x64, 0, sizeof(double) * maxn, b->stream);
        cudaMemsetAsync(x32, 0, sizeof(float) * maxn, b->stream);
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        std::map<int, int> best64, best32;
        for (auto &kv : first_of) {
            const int i = kv.second;
            std::vector<int> onv(ninst, 0);
            onv[i] = 1;
            FCI_CUDA(cudaMemcpy(ton, onv.data(), sizeof(int) * ninst, cudaMemcpyHostToDevice));
            std::vector<void *> pin(ninst, nullptr), pout(ninst, nullptr);
            for (int dt = 0; dt < 2; ++dt) {
                pin[i] = dt == 0 ? (void *)x64 : (void *)x32;
                pout[i] = dt == 0 ? (void *)y64 : (void *)y32;
                FCI_CUDA(cudaMemcpy(b->d_cin, pin.data(), sizeof(void *) * ninst, cudaMemcpyHostToDevice));
                FCI_CUDA(cudaMemcpy(b->d_cout, pout.data(), sizeof(void *) * ninst, cudaMemcpyHostToDevice));
                float best_ms = 1e30f;
                int best = 128;
                for (int tpr : cands) {
                    b->h_inst[i].tpr = tpr;
                    FCI_CUDA(cudaMemcpy(b->d_inst + i, &b->h_inst[i], sizeof(InstDev), cudaMemcpyHostToDevice));
                    std::vector<Item> it;
                    const int R = kBlock / tpr;
                    for (int64_t r = 0; r < b->h_inst[i].A.ns && it.size() < (1u << 16); r += R) it.push_back({i, (int)r});
                    FCI_CUDA(cudaMemcpy(titems, it.data(), sizeof(Item) * it.size(), cudaMemcpyHostToDevice));
                    float tmin = 1e30f;
                    for (int rep = 0; rep < 3; ++rep) {
                        cudaEventRecord(e0, b->stream);
                        if (dt == 0)
                            launch_bsigma<double>(b, ton, (const double *const *)b->d_cin, (double *const *)b->d_cout,
                                                  b->stream, titems, (int)it.size());
                        else
                            launch_bsigma<float>(b, ton, (const float *const *)b->d_cin, (float *const *)b->d_cout,
                                                 b->stream, titems, (int)it.size());
                        cudaEventRecord(e1, b->stream);
                        cudaEventSynchronize(e1);
                        float ms = 0.f;
                        cudaEventElapsedTime(&ms, e0, e1);
                        tmin = std::min(tmin, ms);
                    }
                    if (tmin < best_ms) {
                        best_ms = tmin;
                        best = tpr;
                    }
                }
                (dt == 0 ? best64 : best32)[kv.first] = best;
                b->tune.push_back(kv.first);
                b->tune.push_back(dt == 0 ? FCI_F64 : FCI_F32);
                b->tune.push_back(best);
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        b->stats[1] = 0;
        // the FP32 choice is used in mixed mode (most sigma calls), else FP64
        for (int i = 0; i < ninst; ++i)
            b->h_inst[i].tpr = (o.precision == FCI_PREC_MIXED ? best32 : best64)[inst[i].norb];
        // the FP32 stage-all mode uses one row group of all 256 threads
        if (o.precision == FCI_PREC_MIXED)
            for (int i = 0; i < ninst; ++i)
                if (b->h_inst[i].stage_all) b->h_inst[i].tpr = kBlock;
        if (o.precision != FCI_PREC_MIXED)
            for (int i = 0; i < ninst; ++i) b->h_inst[i].stage_all = 0;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            return cuda_fail(e, "batched CASCI tuning");
        }
    }
    // large instances run the single-instance kernels in both precisions
    for (int i = 0; i < ninst && rc == FCI_OK; ++i)
        if (b->h_inst[i].ndet >= kHybridMinDets && sigma_f32_gated_ok(b->ctx[i]) && sigma_f64_gated_ok(b->ctx[i])) {
            b->hyb.push_back(i);
            rc = prepare_sigma_f32_gated(b->ctx[i]);
            if (!rc) rc = prepare_sigma_f64_gated(b->ctx[i]);
        }
    if (rc || (rc = build_items(b, &rc))) {
        return rc;
    }
    guard.b = nullptr;  // complete: the caller owns the batch
    *out = b;
    return FCI_OK;
}

int fci_batch_sigma(fci_batch *b, const void *c, void *sigma, int dtype, void *stream) {
    if (!b || !c || !sigma) return fail(FCI_ERR_ARG, "NULL argument");
    if (dtype != FCI_F64 && dtype != FCI_F32) return fail(FCI_ERR_ARG, "dtype must be FCI_F64 or FCI_F32");
    FCI_CUDA(cudaSetDevice(b->device));
    const size_t es = dtype == FCI_F64 ? 8 : 4;
    std::vector<void *> pin(b->ninst), pout(b->ninst);
    for (int i = 0; i < b->ninst; ++i) {
        pin[i] = (char *)c + es * b->off[i];
        pout[i] = (char *)sigma + es * b->off[i];
    }
    cudaStream_t s = (cudaStream_t)stream;
    FCI_CUDA(cudaMemcpyAsync(b->d_cin, pin.data(), sizeof(void *) * b->ninst, cudaMemcpyHostToDevice, s));
    FCI_CUDA(cudaMemcpyAsync(b->d_cout, pout.data(), sizeof(void *) * b->ninst, cudaMemcpyHostToDevice, s));
    int rc;
    if (dtype == FCI_F64) {
        rc = b->nitems > b->nitems_hyb
                 ? launch_bsigma<double>(b, b->d_on_all, (const double *const *)b->d_cin, (double *const *)b->d_cout, s,
                                         b->d_items + b->nitems_hyb, b->nitems - b->nitems_hyb)
                 : FCI_OK;
        for (int i : b->hyb)
            if (!rc)
                rc = launch_sigma_f64_gated(b->ctx[i], (const double *)c + b->off[i], (double *)sigma + b->off[i],
                                            b->d_on_all + i, s);
    } else
        rc = launch_bsigma<float>(b, b->d_on_all, (const float *const *)b->d_cin, (float *const *)b->d_cout, s,
                                  b->d_items, b->nitems);
    if (rc) return rc;
    FCI_CUDA(cudaStreamSynchronize(s));  // the pointer tables are reused by the next call
    return FCI_OK;
}

}  // extern "C"

// ---- batched Davidson ----------------------------------------------------------

namespace fci {
namespace bt {

// d = d - h (masked)
__global__ void __launch_bounds__(kBlock) k_bsub(const Chunk *__restrict__ ch, const int *__restrict__ on,
                                                 double *__restrict__ d, const double *__restrict__ h) {
    const Chunk c = ch[blockIdx.x];
    if (!on[c.inst] || threadIdx.x >= c.len) return;
    const int64_t idx = c.start + threadIdx.x;
    d[idx] -= h[idx];
}
// h = h + d (masked)
__global__ void __launch_bounds__(kBlock) k_badd(const Chunk *__restrict__ ch, const int *__restrict__ on,
                                                 double *__restrict__ h, const double *__restrict__ d) {
    const Chunk c = ch[blockIdx.x];
    if (!on[c.inst] || threadIdx.x >= c.len) return;
    const int64_t idx = c.start + threadIdx.x;
    h[idx] += d[idx];
}

// Per-instance decisions of one batched Davidson iteration, on the device (one
// thread per instance), from the Ritz values w and squared residual norms rn2
// just computed: energies, convergence (only where the subspace sigma is
// FP64-exact), and whether the instance refines (mixed precision) or expands
// this iteration.  State per instance: iteration count, iterations since the
// last exact point, the energies of the last exact point, the last 16
// residuals.  *ndone counts converged instances.  Refinements happen only on
// iterations with can_refine set (every kRefinePeriod-th iteration that is not
// a thick restart): an instance whose test passes in between refines at the
// next such iteration, and the other iterations carry no refinement launches.
__global__ void k_bdecide(int ninst, int nroots, double tol, int mixed, int can_refine, const double *__restrict__ w,
                          const double *__restrict__ rn2, int *__restrict__ active, int *__restrict__ refine,
                          int *__restrict__ expand, int *__restrict__ exact, int *__restrict__ inner,
                          int *__restrict__ its, double *__restrict__ eprev, double *__restrict__ rhist,
                          double *__restrict__ energy, int *__restrict__ ndone) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ninst) return;
    refine[i] = 0;
    expand[i] = 0;
    if (!active[i]) return;
    const int it = ++its[i];
    double rmax = 0.0, demax = 0.0;
    for (int k = 0; k < nroots; ++k) {
        const double e = w[(int64_t)i * kMaxSub + k];
        rmax = fmax(rmax, sqrt(rn2[(int64_t)i * kMaxRoots + k]));
        demax = fmax(demax, fabs(e - eprev[(int64_t)i * kMaxRoots + k]));
        energy[(int64_t)i * kMaxRoots + k] = e;
    }
    double *rh = rhist + (int64_t)i * 16;
    const double r15 = rh[it % 16];  // residual 16 iterations ago
    rh[it % 16] = rmax;
    if (exact[i]) {
        if (demax < tol && rmax < sqrt(tol)) {
            active[i] = 0;
            atomicAdd(ndone, 1);
            return;
        }
        for (int k = 0; k < nroots; ++k) eprev[(int64_t)i * kMaxRoots + k] = w[(int64_t)i * kMaxSub + k];
        inner[i] = 0;
    } else if (mixed && (++inner[i] >= 60 || rmax < sqrt(tol) || (inner[i] >= 15 && rmax > 0.5 * r15)) &&
               can_refine) {
        refine[i] = 1;
    }
    expand[i] = refine[i] ? 0 : 1;
}

// exact <- 1 where the instance refined; exact <- 0 where it expanded with FP32
// sigma (mixed) or, when all is set, everywhere (a collapse kept FP32 vectors)
__global__ void k_bexact(int ninst, const int *__restrict__ refine, const int *__restrict__ expand, int all,
                         int *__restrict__ exact) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ninst) return;
    if (all) exact[i] = 0;
    else if (refine && refine[i]) exact[i] = 1;
    else if (expand && expand[i]) exact[i] = 0;
}

struct BWork {
    fci_batch *b;
    cudaStream_t s;
    int nroots, maxsub;
    bool mixed;
    double *Bv, *Sv, *X, *HX, *T;   // batch vectors: [maxsub|nroots][ntot]
    float *c32, *s32;               // [ntot]
    double *A, *w, *V, *g, *nrm2, *rn2, *partial;
    int *on, *on_exp, *on_ref;      // masks: active, expanding, refining
    int *exact, *inner, *its, *ndone;  // per-instance decision state (device)
    double *eprev, *rhist, *energy;    // [ninst][kMaxRoots], [ninst][16], [ninst][kMaxRoots]
    void **ptr32;                   // [2][ninst]: c32 / s32 per instance
    void **ptrBS;                   // [maxsub][2][ninst]: B_j -> S_j per instance
    void **ptrXT;                   // [nroots][2][ninst]: X_k -> T_k per instance
    void **ptrD2;                   // [2][ninst]: scratch for the initial guesses
    std::map<int, cudaGraphExec_t> g_chunk;  // iterations from subspace size m to the next restart (<= 8)
};

// out[i*os + j*js] = X_j . y for j < m, per instance (masked by on); one CTA
// per (kDChunk-element chunk, group of 8 vectors), then one CTA per instance
static void bdots(BWork &W, const int *on, const double *X, int m, const double *y, double *out, int64_t os,
                  int64_t js) {
    fci_batch *b = W.b;
    const int G = (m + 7) / 8;
    k_bdots<<<b->ndchunks * G, kBlock, 0, W.s>>>(b->d_dchunks, on, X, b->ntot, m, G, y, W.partial);
    k_breduce<32><<<b->ninst, kBlock, 0, W.s>>>(b->d_dcfirst, on, W.partial, m, out, os, js);
}

// hx = H x for the batch vector x (instances masked by on); FP32 arithmetic when low.
// tab: [2][ninst] FP64 in/out pointers of x and hx.
static int bsigma(BWork &W, const int *on, const double *x, double *hx, void **tab, bool low) {
    fci_batch *b = W.b;
    const int n = b->ninst;
    if (low) {
        k_d2f<<<grid_flat(b->ntot), 256, 0, W.s>>>(x, W.c32, b->ntot);
        if (b->nitems > b->nitems_hyb)
            if (int rc = launch_bsigma<float>(b, on, (const float *const *)W.ptr32, (float *const *)(W.ptr32 + n),
                                              W.s, b->d_items + b->nitems_hyb, b->nitems - b->nitems_hyb))
                return rc;
        for (int i : b->hyb)
            if (int rc = launch_sigma_f32_gated(b->ctx[i], W.c32 + b->off[i], W.s32 + b->off[i], on + i, W.s))
                return rc;
        k_f2d<<<grid_flat(b->ntot), 256, 0, W.s>>>(W.s32, hx, b->ntot);
        return FCI_OK;
    }
    if (b->nitems > b->nitems_hyb)
        if (int rc = launch_bsigma<double>(b, on, (const double *const *)tab, (double *const *)(tab + n), W.s,
                                           b->d_items + b->nitems_hyb, b->nitems - b->nitems_hyb))
            return rc;
    for (int i : b->hyb)
        if (int rc = launch_sigma_f64_gated(b->ctx[i], x + b->off[i], hx + b->off[i], on + i, W.s)) return rc;
    return FCI_OK;
}

}  // namespace bt
}  // namespace fci

namespace fci {
namespace bt {
// The Davidson iterations of fci_batch_davidson.  Every device buffer it makes
// is recorded in `mine` and every graph in W; the caller frees them on every
// return path, also when this function returns early or throws.
static int batch_davidson_run(fci_batch *b, int nroots, double tol, double *energies, BWork &W,
                              std::vector<std::pair<void *, size_t>> &mine) {
    const int ninst = b->ninst;
    const int64_t ntot = b->ntot;
    int rc = FCI_OK;
    W.b = b;
    W.s = b->stream;
    W.nroots = nroots;
    W.mixed = b->opt.precision == FCI_PREC_MIXED;
    const int maxsub = std::min(kMaxSub, std::max(b->opt.max_subspace, 2 * nroots));
    W.maxsub = maxsub;
    auto get = [&](size_t bytes) -> void * {
        if (rc) return nullptr;
        mine.push_back({nullptr, 0});  // the slot exists before the allocation
        void *p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            rc = fail(FCI_ERR_OOM, "batched Davidson: device allocation failed");
            return nullptr;
        }
        mine.back() = {p, bytes};
        return p;
    };
    W.Bv = (double *)get(sizeof(double) * maxsub * ntot);
    W.Sv = (double *)get(sizeof(double) * maxsub * ntot);
    const int keepn = std::max(nroots, std::min(8, maxsub / 2));  // thick restart
    W.X = (double *)get(sizeof(double) * keepn * ntot);
    W.HX = (double *)get(sizeof(double) * keepn * ntot);
    W.T = (double *)get(sizeof(double) * nroots * ntot);
    W.c32 = (float *)get(sizeof(float) * ntot);
    W.s32 = (float *)get(sizeof(float) * ntot);
    W.A = (double *)get(sizeof(double) * ninst * kMaxSub * kMaxSub);
    W.V = (double *)get(sizeof(double) * ninst * kMaxSub * kMaxSub);
    W.w = (double *)get(sizeof(double) * ninst * kMaxSub);
    W.g = (double *)get(sizeof(double) * ninst * kMaxSub);
    W.nrm2 = (double *)get(sizeof(double) * ninst);
    W.rn2 = (double *)get(sizeof(double) * ninst * kMaxRoots);
    W.partial = (double *)get(sizeof(double) * (size_t)std::max(b->nchunks, b->ndchunks) * 32);
    W.on = (int *)get(sizeof(int) * ninst);
    W.on_exp = (int *)get(sizeof(int) * ninst);
    W.on_ref = (int *)get(sizeof(int) * ninst);
    W.ptr32 = (void **)get(sizeof(void *) * 2 * ninst);
    W.ptrBS = (void **)get(sizeof(void *) * 2 * ninst * maxsub);
    W.ptrXT = (void **)get(sizeof(void *) * 2 * ninst * nroots);
    W.exact = (int *)get(sizeof(int) * ninst);
    W.inner = (int *)get(sizeof(int) * ninst);
    W.its = (int *)get(sizeof(int) * ninst);
    W.ndone = (int *)get(sizeof(int));
    W.eprev = (double *)get(sizeof(double) * ninst * kMaxRoots);
    W.rhist = (double *)get(sizeof(double) * ninst * 16);
    W.energy = (double *)get(sizeof(double) * ninst * kMaxRoots);
    if (rc) return rc;
    cudaStream_t s = W.s;
    {
        std::vector<void *> t(2 * ninst);
        for (int i = 0; i < ninst; ++i) {
            t[i] = W.c32 + b->off[i];
            t[ninst + i] = W.s32 + b->off[i];
        }
        FCI_CUDA(cudaMemcpy(W.ptr32, t.data(), sizeof(void *) * 2 * ninst, cudaMemcpyHostToDevice));
        std::vector<void *> u(2 * ninst * maxsub);
        for (int j = 0; j < maxsub; ++j)
            for (int i = 0; i < ninst; ++i) {
                u[(size_t)j * 2 * ninst + i] = W.Bv + (size_t)j * ntot + b->off[i];
                u[(size_t)j * 2 * ninst + ninst + i] = W.Sv + (size_t)j * ntot + b->off[i];
            }
        FCI_CUDA(cudaMemcpy(W.ptrBS, u.data(), sizeof(void *) * u.size(), cudaMemcpyHostToDevice));
        std::vector<void *> v(2 * ninst * nroots);
        for (int k = 0; k < nroots; ++k)
            for (int i = 0; i < ninst; ++i) {
                v[(size_t)k * 2 * ninst + i] = W.X + (size_t)k * ntot + b->off[i];
                v[(size_t)k * 2 * ninst + ninst + i] = W.T + (size_t)k * ntot + b->off[i];
            }
        FCI_CUDA(cudaMemcpy(W.ptrXT, v.data(), sizeof(void *) * v.size(), cudaMemcpyHostToDevice));
    }
    // decision state on the device: every instance active, exact in FP64 mode
    {
        std::vector<int> ones(ninst, 1), ex(ninst, W.mixed ? 0 : 1);
        std::vector<double> inf_r((size_t)ninst * kMaxRoots, INFINITY), inf_h((size_t)ninst * 16, INFINITY);
        FCI_CUDA(cudaMemcpy(W.on, ones.data(), sizeof(int) * ninst, cudaMemcpyHostToDevice));
        FCI_CUDA(cudaMemcpy(W.exact, ex.data(), sizeof(int) * ninst, cudaMemcpyHostToDevice));
        FCI_CUDA(cudaMemset(W.inner, 0, sizeof(int) * ninst));
        FCI_CUDA(cudaMemset(W.its, 0, sizeof(int) * ninst));
        FCI_CUDA(cudaMemset(W.ndone, 0, sizeof(int)));
        FCI_CUDA(cudaMemcpy(W.eprev, inf_r.data(), sizeof(double) * inf_r.size(), cudaMemcpyHostToDevice));
        FCI_CUDA(cudaMemcpy(W.energy, inf_r.data(), sizeof(double) * inf_r.size(), cudaMemcpyHostToDevice));
        FCI_CUDA(cudaMemcpy(W.rhist, inf_h.data(), sizeof(double) * inf_h.size(), cudaMemcpyHostToDevice));
    }
    for (int i = 0; i < 4; ++i) b->stats[i] = 0;

    // (1) initial subspace: unit vectors on the lowest diagonal elements, their sigma
    FCI_CUDA(cudaMemsetAsync(W.A, 0, sizeof(double) * ninst * kMaxSub * kMaxSub, s));
    k_bguess<<<ninst, 256, 0, s>>>(b->d_inst, nroots, W.Bv, ntot);
    for (int k = 0; k < nroots && !rc; ++k)
        rc = bsigma(W, W.on, W.Bv + (size_t)k * ntot, W.Sv + (size_t)k * ntot, W.ptrBS + (size_t)k * 2 * ninst,
                    W.mixed);
    b->stats[1] += nroots;
    int m = nroots;
    for (int j = 0; j < m && !rc; ++j)
        bdots(W, W.on, W.Bv, m, W.Sv + (size_t)j * ntot, W.A + j, kMaxSub * kMaxSub, kMaxSub);
    if (rc) return rc;

    // One iteration as a kernel sequence whose every decision lives on the
    // device: (4) diagonalise, Ritz vectors and residuals, the per-instance
    // decisions (k_bdecide), the refinement of the instances that refine
    // (mixed precision; sigma64 of the Ritz vectors corrects S along v), a thick
    // restart when the subspace is full (the subspace size m follows the same
    // sequence for every instance, so the host knows it), and (2)-(3) one new
    // preconditioned, orthonormalised vector per root with its sigma for the
    // instances that expand (padding elsewhere).  Returns m after the iteration.
    const int keep = std::min(keepn, maxsub);
    const unsigned gi = (unsigned)((ninst + 127) / 128);
    auto iteration = [&](int mi, bool can_refine, int *sig_launches) -> int {
        k_bjacobi<<<ninst, 128, 0, s>>>(W.on, W.A, mi, W.w, W.V);
        for (int k = 0; k < nroots; ++k) {
            k_blincomb<<<b->nchunks, kBlock, 0, s>>>(b->d_chunks, W.on, W.Bv, ntot, mi, W.V + k, kMaxSub * kMaxSub, mi,
                                                      1.0, 0.0, W.X + (size_t)k * ntot);
            k_blincomb<<<b->nchunks, kBlock, 0, s>>>(b->d_chunks, W.on, W.Sv, ntot, mi, W.V + k, kMaxSub * kMaxSub, mi,
                                                      1.0, 0.0, W.HX + (size_t)k * ntot);
            k_bresid<<<b->nchunks, kBlock, 0, s>>>(b->d_chunks, W.on, b->d_inst, W.X + (size_t)k * ntot,
                                                    W.HX + (size_t)k * ntot, W.w + k, kMaxSub, W.T + (size_t)k * ntot,
                                                    W.partial);
            k_breduce<8><<<ninst, kBlock, 0, s>>>(b->d_cfirst, W.on, W.partial, 1, W.rn2 + k, kMaxRoots, 1);
        }
        k_bdecide<<<gi, 128, 0, s>>>(ninst, nroots, tol, W.mixed ? 1 : 0, can_refine ? 1 : 0, W.w, W.rn2, W.on,
                                     W.on_ref, W.on_exp, W.exact, W.inner, W.its, W.eprev, W.rhist, W.energy, W.ndone);
        if (can_refine) {
            // refinement: delta = sigma64(x_k) - HX_k corrects S along v_k (rank 1)
            for (int k = 0; k < nroots && !rc; ++k) {
                double *d = W.T + (size_t)k * ntot;  // refining instances add no correction this round
                rc = bsigma(W, W.on_ref, W.X + (size_t)k * ntot, d, W.ptrXT + (size_t)k * 2 * ninst, false);
                if (rc) break;
                k_bsub<<<b->nchunks, kBlock, 0, s>>>(b->d_chunks, W.on_ref, d, W.HX + (size_t)k * ntot);
                k_badd<<<b->nchunks, kBlock, 0, s>>>(b->d_chunks, W.on_ref, W.HX + (size_t)k * ntot, d);
                bdots(W, W.on_ref, W.Bv, mi, d, W.g, kMaxSub, 1);
                k_brank1<<<b->nchunks, kBlock, 0, s>>>(b->d_chunks, W.on_ref, W.Sv, ntot, mi, W.V, k, d);
                k_brank1_proj<<<ninst, 256, 0, s>>>(W.on_ref, W.A, W.g, W.V, mi, k);
            }
            *sig_launches += nroots;
            k_bexact<<<gi, 128, 0, s>>>(ninst, W.on_ref, nullptr, 0, W.exact);
        }
        if (rc) return mi;
        if (mi + nroots > maxsub) {
            // thick restart: every active instance collapses onto its lowest
            // `keep` Ritz vectors and their sigma
            const int kk = std::min(keep, mi);
            for (int k = nroots; k < kk; ++k) {
                k_blincomb<<<b->nchunks, kBlock, 0, s>>>(b->d_chunks, W.on, W.Bv, ntot, mi, W.V + k, kMaxSub * kMaxSub,
                                                          mi, 1.0, 0.0, W.X + (size_t)k * ntot);
                k_blincomb<<<b->nchunks, kBlock, 0, s>>>(b->d_chunks, W.on, W.Sv, ntot, mi, W.V + k, kMaxSub * kMaxSub,
                                                          mi, 1.0, 0.0, W.HX + (size_t)k * ntot);
            }
            for (int k = 0; k < kk; ++k) {
                k_bcopy<<<b->nchunks, kBlock, 0, s>>>(b->d_chunks, W.on, W.X + (size_t)k * ntot, W.Bv + (size_t)k * ntot, 0);
                k_bcopy<<<b->nchunks, kBlock, 0, s>>>(b->d_chunks, W.on, W.HX + (size_t)k * ntot, W.Sv + (size_t)k * ntot, 0);
            }
            mi = kk;
            if (W.mixed && kk > nroots) k_bexact<<<gi, 128, 0, s>>>(ninst, nullptr, nullptr, 1, W.exact);  // FP32 sigma kept
            cudaMemsetAsync(W.A, 0, sizeof(double) * ninst * kMaxSub * kMaxSub, s);
            for (int j = 0; j < mi; ++j)
                bdots(W, W.on, W.Bv, mi, W.Sv + (size_t)j * ntot, W.A + j, kMaxSub * kMaxSub, kMaxSub);
        }
        // expansion: one new vector per root and instance (padding where not expanding)
        for (int k = 0, mm = mi; k < nroots && !rc; ++k, ++mm) {
            double *bv = W.Bv + (size_t)mm * ntot, *sv = W.Sv + (size_t)mm * ntot;
            k_bcopy<<<b->nchunks, kBlock, 0, s>>>(b->d_chunks, W.on_exp, W.T + (size_t)k * ntot, bv, 1);
            for (int pass = 0; pass < 2; ++pass) {
                bdots(W, W.on_exp, W.Bv, mm, bv, W.g, kMaxSub, 1);
                k_blincomb<<<b->nchunks, kBlock, 0, s>>>(b->d_chunks, W.on_exp, W.Bv, ntot, mm, W.g, kMaxSub, 1, -1.0, 1.0,
                                                          bv);
            }
            bdots(W, W.on_exp, bv, 1, bv, W.nrm2, 1, 1);
            k_bnormalise<<<b->nchunks, kBlock, 0, s>>>(b->d_chunks, W.on_exp, W.nrm2, bv);
            cudaMemsetAsync(sv, 0, sizeof(double) * ntot, s);
            rc = bsigma(W, W.on_exp, bv, sv, W.ptrBS + (size_t)mm * 2 * ninst, W.mixed);
            bdots(W, W.on_exp, W.Bv, mm + 1, sv, W.A + mm, kMaxSub * kMaxSub, kMaxSub);
            bdots(W, W.on_exp, W.Sv, mm + 1, bv, W.A + (size_t)mm * kMaxSub, kMaxSub * kMaxSub, 1);
            k_bpad<<<(ninst + 127) / 128, 128, 0, s>>>(W.on_exp, W.nrm2, W.A, mm, ninst);
        }
        *sig_launches += nroots;
        if (W.mixed) k_bexact<<<gi, 128, 0, s>>>(ninst, nullptr, W.on_exp, 0, W.exact);
        return mi + nroots;
    };
    // Refinements (mixed precision) are allowed on every kRefinePeriod-th
    // iteration that is not a thick restart (a restart keeps vectors with FP32
    // sigma, which would undo the refinement's exactness): `phase` counts the
    // non-restart iterations modulo the period.  The iterations from subspace
    // size m0 up to and including the next restart (at most 8, no more than
    // `left`), with the refinement flag of each: their count, size and phase after.
    auto chunk = [&](int m0, int ph0, int left, int *m_after, int *ph_after, std::vector<char> &refs) {
        int mm = m0, ph = ph0, L = 0;
        refs.clear();
        while (L < 8 && L < left) {
            ++L;
            const bool restart = mm + nroots > maxsub;
            refs.push_back(W.mixed && !restart && ph == 0 ? 1 : 0);
            if (!restart) ph = (ph + 1) % kRefinePeriod;
            mm = (restart ? std::min(keep, mm) : mm) + nroots;
            if (restart) break;
        }
        *m_after = mm;
        *ph_after = ph;
        return L;
    };
    // Host loop: one graph launch per chunk of iterations, then one 4-byte
    // read (the number of converged instances); nothing else returns to the host.
    int it = 0, hdone = 0, phase = 1;  // the first refinement comes after kRefinePeriod - 1 FP32 iterations
    bool all_done = false;
    std::map<int, int> chunk_sig;
    std::vector<char> refs;
    while (it < b->opt.max_iter && !rc) {
        int m_after = 0, ph_after = 0;
        const int L = chunk(m, phase, b->opt.max_iter - it, &m_after, &ph_after, refs);
        const int key = (m * 64 + L) * kRefinePeriod + phase;
        auto g = W.g_chunk.find(key);
        if (g == W.g_chunk.end()) {
            cudaGraph_t graph;
            int sl = 0;
            FCI_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
            int mm = m;
            for (int j = 0; j < L && !rc; ++j) mm = iteration(mm, refs[j] != 0, &sl);
            const cudaError_t ce = cudaStreamEndCapture(s, &graph);
            if (rc) {
                if (ce == cudaSuccess) cudaGraphDestroy(graph);
                break;
            }
            FCI_CUDA(ce);
            cudaGraphExec_t ex;
            const cudaError_t ie = cudaGraphInstantiate(&ex, graph, 0);
            cudaGraphDestroy(graph);
            FCI_CUDA(ie);
            g = W.g_chunk.emplace(key, ex).first;
            chunk_sig[key] = sl;
        }
        FCI_CUDA(cudaGraphLaunch(g->second, s));
        b->stats[1] += chunk_sig[key];
        b->stats[2]++;
        it += L;
        m = m_after;
        phase = ph_after;
        FCI_CUDA(cudaMemcpyAsync(&hdone, W.ndone, sizeof(int), cudaMemcpyDeviceToHost, s));
        FCI_CUDA(cudaStreamSynchronize(s));
        b->stats[3]++;
        if (hdone >= ninst) {
            all_done = true;
            break;
        }
    }
    if (rc) return rc;
    {
        std::vector<int> its(ninst);
        std::vector<double> en((size_t)ninst * kMaxRoots);
        FCI_CUDA(cudaMemcpy(its.data(), W.its, sizeof(int) * ninst, cudaMemcpyDeviceToHost));
        FCI_CUDA(cudaMemcpy(en.data(), W.energy, sizeof(double) * en.size(), cudaMemcpyDeviceToHost));
        b->stats[0] = *std::max_element(its.begin(), its.end());
        for (int i = 0; i < ninst; ++i)
            for (int k = 0; k < nroots; ++k) energies[(size_t)i * nroots + k] = en[(size_t)i * kMaxRoots + k];
    }
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "batched Davidson");
    for (int i : b->hyb) {  // bounded waits of the tensor-core sigma_3
        int derr = 0;
        FCI_CUDA(cudaMemcpy(&derr, b->ctx[i]->d_err, sizeof(int), cudaMemcpyDeviceToHost));
        if (derr) return fail(FCI_ERR_TIMEOUT, "batched Davidson: a bounded device wait gave up inside sigma");
    }
    if (!all_done) return fail(FCI_ERR_NOCONV, "batched Davidson: some instances did not converge within max_iter");
    return FCI_OK;
}
}  // namespace bt
}  // namespace fci

extern "C" int fci_batch_davidson(fci_batch *b, int nroots, double tol, double *energies) {
    using namespace fci::bt;
    if (!b || !energies) return fail(FCI_ERR_ARG, "NULL argument");
    if (nroots < 1 || nroots > kMaxRoots) return fail(FCI_ERR_ARG, "nroots must be in 1..8");
    for (int i = 0; i < b->ninst; ++i)
        if (b->h_inst[i].ndet < 2 * nroots) return fail(FCI_ERR_ARG, "an instance has fewer than 2*nroots determinants");
    if (!(tol > 0)) return fail(FCI_ERR_ARG, "tol must be positive");
    FCI_CUDA(cudaSetDevice(b->device));
    FCI_CUDA(cudaDeviceSynchronize());
    BWork W{};
    std::vector<std::pair<void *, size_t>> mine;
    int rc = FCI_OK;
    try {
        rc = batch_davidson_run(b, nroots, tol, energies, W, mine);
    } catch (const std::bad_alloc &) {  // host vectors: no exception crosses the C ABI
        rc = fail(FCI_ERR_OOM, "batched Davidson: host allocation failed");
    }
    // an error between stream capture begin and end leaves the stream capturing
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(b->stream, &cap) == cudaSuccess && cap != cudaStreamCaptureStatusNone) {
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(b->stream, &g);
        if (g) cudaGraphDestroy(g);
    }
    cudaStreamSynchronize(b->stream);
    for (auto &kv : W.g_chunk) cudaGraphExecDestroy(kv.second);
    for (auto &a : mine)
        if (a.first) cudaFree(a.first);
    return rc;
}
