// FP64 same-spin sigma terms (sigma_1 and sigma_2 of Eq. 8) as dense sliced
// contractions on the bf16 tensor cores.
//
// With G_s the Hamiltonian of spin s alone between the strings of that spin
// (the one-spin part of Eq. 6: diagonal, single and double replacements;
// symmetric),
//   sigma_1(I_a, I_b) = sum_{J_b} G_b(I_b, J_b) C(I_a, J_b)
//   sigma_2(I_a, I_b) = sum_{J_a} G_a(I_a, J_a) C(J_a, I_b).
// G_s has 1 + n(N-n) + C(n,2) C(N-n,2) nonzeros per row (491 of 3432 at
// CAS(14,14)).  Its diagonal (one-spin energies, tens of Eh against couplings
// well below one) is applied in FP64 separately; the off-diagonal part as a
// dense matrix makes both terms square matrix products, and
// the bf16 tensor pipe (1937 TFLOP/s measured) outruns the FP32 pipe (70) by
// far more than the zeros cost.  FP64 accuracy comes from the digit scheme of
// sliced_mma.cuh: every row of G_s and every row or column of C in 46-bit
// fixed point relative to its own largest power of two, six 8-bit digits, 21
// digit products with exact per-weight accumulation flushed into 64-bit
// integers every 256 terms, and at the end one FP64 conversion per element
// with the two scales of its row and column.
//
// One kernel computes out[n ldo + m] += sum_k A(m, k) B(n, k) for two plane
// sets A (rows m, the MMA's M: 128 per tile) and B (rows n: 48 per tile), each
// row with its own exponent:
//   sigma_1: A = G_b (m = I_b), B = C by rows (n = I_a, k = J_b);
//   sigma_2: A = C by columns (m = I_b, k = J_a), B = G_a (n = I_a);
// both write sigma(I_a, I_b) at I_a n_b + I_b, consecutive across the lanes of
// a warp.  Plane sets are laid out like the 2-RDM's digit planes: per K-step
// of 16, six planes of rows x 16 bf16 in the K-major no-swizzle core-matrix
// layout; rows padded to a multiple of 384 (both tile heights), K to 16.
// G_s's planes are built once at fci_init; C's two plane sets per call.
#include "sliced_mma.cuh"

namespace fci {
namespace ss {

using sl::kSlices;
using tc::kM;
using sm::bulk_g2s;
using sm::levels_to_int_f;
using sm::mbar_expect_tx;

constexpr int kThreads = 448;        // warp 0 copies, warp 1 issues the MMAs, warps 2-13 epilogue
constexpr int kEpiThreads = 384;
constexpr int kBN = 48;              // B rows per tile
constexpr int kStages = 6;           // K-steps of operands in flight
constexpr int kKTile = 16;           // K-steps (256 terms) per accumulator flush
constexpr int kRowPad = 384;         // plane rows: a multiple of 128 and of 48
constexpr int kF = 34;               // integer unit 2^-34 of the accumulator scale
constexpr uint32_t kBytesA = 6 * 4096;
constexpr uint32_t kBytesB = 6 * kBN * 32;
constexpr uint32_t kStageBytes = kBytesA + kBytesB;
constexpr int kBars = 2 * kStages + 5;
constexpr uint32_t kSmem = kStages * kStageBytes + kBars * 8 + 16;

inline int64_t pad_rows(int64_t r) { return (r + kRowPad - 1) / kRowPad * kRowPad; }
inline size_t plane_bytes(int64_t rows, int64_t k) { return (size_t)((k + 15) / 16) * 6 * pad_rows(rows) * 32; }

// six digits of X into the planes at (row r, column k): plane t of K-step k/16
// at byte ((k/16) 6 + t) rows_pad 32, then the core-matrix offset of (r, k%16)
__device__ __forceinline__ void put_digits(unsigned char *planes, int64_t rows_pad, int64_t r, int64_t k, long long X) {
    float f[kSlices];
    sl::digits6(X, f);
    const int64_t ks = k >> 4;
    const int kk = (int)(k & 15);
    const uint32_t off = (uint32_t)((r >> 3) * 256 + (kk >> 3) * 128 + (r & 7) * 16 + (kk & 7) * 2);
#pragma unroll
    for (int t = 0; t < kSlices; ++t) {
        const __nv_bfloat16 b = __float2bfloat16_rn(f[t]);  // exact: an 8-bit integer times a power of two
        *reinterpret_cast<__nv_bfloat16 *>(planes + ((size_t)ks * 6 + t) * rows_pad * 32 + off) = b;
    }
}

__device__ __forceinline__ long long fixed46(double x, int emax) {
    const unsigned long long b = __double_as_longlong(x);
    return sl::fixed47((uint32_t)b, (uint32_t)(b >> 32), emax + 1);
}

// largest biased exponent of the off-diagonal part of each row of the ELL
// same-spin Hamiltonian (slot 0 is the diagonal, applied separately)
__global__ void k_ss_rowexp(const double *__restrict__ gval, int64_t ns, int nsame, int *__restrict__ e) {
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= ns) return;
    unsigned m = 0;
    for (int k = 1; k < nsame; ++k)
        m = max(m, (unsigned)((__double_as_longlong(gval[(int64_t)k * ns + x]) >> 52) & 0x7FF));
    e[x] = (int)m;
}

// dense G planes: every off-diagonal ELL entry (row x, column gcol, value
// gval) scattered (each row's columns are distinct; the planes start at zero)
__global__ void k_ss_gplanes(const int32_t *__restrict__ gcol, const double *__restrict__ gval, int64_t ns, int nsame,
                             const int *__restrict__ e, int64_t rows_pad, unsigned char *__restrict__ planes) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < ns || t >= ns * (int64_t)nsame) return;  // slot 0 (t < ns): the diagonal
    const int64_t x = t % ns;
    const double v = gval[t];
    if (v == 0.0) return;
    put_digits(planes, rows_pad, x, gcol[t], fixed46(v, e[x]));
}

// largest biased exponent of each row (erow) and each column (ecol) of the
// nrows x ncols matrix C, both from one coalesced pass: block (32, 8) over a
// 32 x 32 tile, integer atomicMax into erow / ecol (zeroed beforehand)
__global__ void k_ss_cexp(const double *__restrict__ C, int64_t nrows, int64_t ncols, int *__restrict__ erow,
                          int *__restrict__ ecol) {
    __shared__ unsigned colmax[8][32];
    const int64_t c = (int64_t)blockIdx.x * 32 + threadIdx.x;
    unsigned cm = 0;
    for (int i = 0; i < 4; ++i) {
        const int64_t r = (int64_t)blockIdx.y * 32 + threadIdx.y * 4 + i;
        unsigned e = 0;
        if (r < nrows && c < ncols) e = (unsigned)((__double_as_longlong(C[r * ncols + c]) >> 52) & 0x7FF);
        cm = max(cm, e);
        unsigned rm = e;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) rm = max(rm, __shfl_xor_sync(0xFFFFFFFFu, rm, o));
        if (threadIdx.x == 0 && r < nrows) atomicMax(erow + r, (int)rm);
    }
    colmax[threadIdx.y][threadIdx.x] = cm;
    __syncthreads();
    if (threadIdx.y == 0 && c < ncols) {
        unsigned m = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) m = max(m, colmax[k][threadIdx.x]);
        atomicMax(ecol + c, (int)m);
    }
}

// C's planes by rows (row i of the planes = row i of C, k = column) or by
// columns (row j of the planes = column j of C, k = row of C): one thread per
// (plane row, 8 consecutive k), 16-byte stores of each digit plane
__global__ void k_ss_cplanes(const double *__restrict__ C, int64_t nrows, int64_t ncols, int cols,
                             const int *__restrict__ e, int64_t rows_pad, unsigned char *__restrict__ planes) {
    const int64_t prow_n = cols ? ncols : nrows, klen = cols ? nrows : ncols;
    const int64_t groups = (klen + 7) / 8;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= prow_n * groups) return;
    // cols: consecutive threads take consecutive plane rows (consecutive C columns: coalesced reads)
    const int64_t r = cols ? t % prow_n : t / groups, g = cols ? t / prow_n : t % groups;
    const int er = e[r];
    uint32_t w[kSlices][4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float f0[kSlices], f1[kSlices];
        const int64_t k0 = g * 8 + 2 * i, k1 = k0 + 1;
        const double v0 = k0 < klen ? (cols ? C[k0 * ncols + r] : C[r * ncols + k0]) : 0.0;
        const double v1 = k1 < klen ? (cols ? C[k1 * ncols + r] : C[r * ncols + k1]) : 0.0;
        sl::digits6(fixed46(v0, er), f0);
        sl::digits6(fixed46(v1, er), f1);
#pragma unroll
        for (int s = 0; s < kSlices; ++s) w[s][i] = sl::pack_bf16(f0[s], f1[s]);
    }
    const int64_t ks = g >> 1;
    const uint32_t off = (uint32_t)((r >> 3) * 256 + (g & 1) * 128 + (r & 7) * 16);
#pragma unroll
    for (int s = 0; s < kSlices; ++s)
        *reinterpret_cast<uint4 *>(planes + ((size_t)ks * 6 + s) * rows_pad * 32 + off) =
            make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
}

// sigma(I_a, I_b) += (G_a(I_a, I_a) + G_b(I_b, I_b)) C(I_a, I_b) in FP64 (the
// diagonal of the same-spin Hamiltonians, ELL slot 0; a null da or db leaves
// that spin out)
__global__ void k_ss_diag(const double *__restrict__ C, double *__restrict__ sig, const double *__restrict__ da,
                          const double *__restrict__ db, int64_t nsa, int64_t nsb) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nsa * nsb; i += stride) {
        const int64_t ia = i / nsb, ib = i - ia * nsb;
        const double d = (da ? da[ia] : 0.0) + (db ? db[ib] : 0.0);
        sig[i] = fma(d, C[i], sig[i]);
    }
}

struct SsArgs {
    const unsigned char *A, *B;  // plane sets
    int64_t rowsA, rowsB;        // padded plane rows
    int M, N;                    // rows of A (output lanes) and of B (output columns) in use
    int64_t nks;                 // K-steps
    const int *eA, *eB;          // biased exponent of each row
    double *out;
    int64_t ldo;                 // out[n ldo + m] +=
    int *err;
};

// Tiles: 128 rows of A x 48 rows of B, t = nb * nmb + mb; CTA b takes tiles
// b, b + grid, ...  (the CTAs of one wave share A and B K-steps through L2,
// advancing through K at one rate).
__global__ void __launch_bounds__(kThreads, 1) k_ss_tc(SsArgs P) {
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kStages * kStageBytes);
    volatile int *s_fail = reinterpret_cast<volatile int *>(smem + kStages * kStageBytes + kBars * 8);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + kStages * kStageBytes + kBars * 8 + 4);
    const uint32_t sbase = tc::smem_u32(smem);
    const uint32_t bar0 = tc::smem_u32(bars);
    auto full = [&](int st) { return bar0 + 8u * (uint32_t)st; };
    auto freeb = [&](int st) { return bar0 + 8u * (uint32_t)(kStages + st); };
    auto acc_full = [&](int b) { return bar0 + 8u * (uint32_t)(2 * kStages + b); };
    auto acc_empty = [&](int b) { return bar0 + 8u * (uint32_t)(2 * kStages + 2 + b); };
    const uint32_t drain = bar0 + 8u * (uint32_t)(2 * kStages + 4);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nmb = (P.M + 127) / 128, nnb = (P.N + kBN - 1) / kBN;
    const int ntiles = nmb * nnb;

    for (uint32_t i = (uint32_t)tid * 16u; i < kStages * kStageBytes; i += kThreads * 16u)
        *reinterpret_cast<uint4 *>(smem + i) = make_uint4(0u, 0u, 0u, 0u);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(tslot)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < kStages; ++i) {
            tc::mbar_init(full(i), 1);
            tc::mbar_init(freeb(i), 1);
        }
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(acc_full(b), 1);
            tc::mbar_init(acc_empty(b), kEpiThreads);
        }
        tc::mbar_init(drain, 1);
        *s_fail = 0;
    }
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tslot;

    int64_t G_copied = 0;
    if (warp == 0 && lane == 0) {
        // ---- copies: the A and B planes of one K-step per stage ----
        int64_t &G = G_copied;
        for (int t = blockIdx.x; t < ntiles && !*s_fail; t += gridDim.x) {
            const int mb = t % nmb, nb = t / nmb;
            const uint32_t ba = 128u * 32u, bb = (uint32_t)kBN * 32u;  // rows padded: whole tiles
            for (int64_t ks = 0; ks < P.nks; ++ks, ++G) {
                const int st = (int)(G % kStages);
                if (G >= kStages && !tc::mbar_wait_bounded(freeb(st), (uint32_t)((G / kStages - 1) & 1))) {
                    *s_fail = 1;
                    break;
                }
                mbar_expect_tx(full(st), 6u * (ba + bb));
                const unsigned char *sa = P.A + ((size_t)ks * 6 * P.rowsA + (size_t)mb * 128) * 32;
                const unsigned char *sb = P.B + ((size_t)ks * 6 * P.rowsB + (size_t)nb * kBN) * 32;
                const uint32_t dst = sbase + (uint32_t)st * kStageBytes;
#pragma unroll
                for (int p = 0; p < 6; ++p) {
                    bulk_g2s(dst + (uint32_t)p * 4096u, sa + (size_t)p * P.rowsA * 32, ba, full(st));
                    bulk_g2s(dst + kBytesA + (uint32_t)p * kBN * 32u, sb + (size_t)p * P.rowsB * 32, bb, full(st));
                }
            }
        }
    } else if (warp == 1 && lane == 0) {
        // ---- MMAs: A digit s times the stacked B digits 0..4-s into weights
        // s..4 (N = (5 - s) 48), then B digit 5 - s into weight 4 ----
        uint64_t ad[kSlices], bd[kSlices];
#pragma unroll
        for (int s = 0; s < kSlices; ++s) {
            ad[s] = tc::smem_desc(sbase + (uint32_t)s * 4096u, 128, 256);
            bd[s] = tc::smem_desc(sbase + kBytesA + (uint32_t)s * kBN * 32u, 128, 256);
        }
        uint32_t idn[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) idn[k] = tc::instr_desc(kM, (k + 1) * kBN);
        int64_t G = 0, Tt = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x)
            for (int64_t kt = 0; kt < P.nks && ok; kt += kKTile, ++Tt) {
                const int b = (int)(Tt & 1);
                if (Tt >= 2 && !tc::mbar_wait_bounded(acc_empty(b), (uint32_t)(((Tt - 2) >> 1) & 1))) {
                    ok = false;
                    break;
                }
                tc::fence_after();
                const int64_t ke = min(P.nks, kt + kKTile);
                for (int64_t ks = kt; ks < ke; ++ks, ++G) {
                    const int st = (int)(G % kStages);
                    if (!tc::mbar_wait_bounded(full(st), (uint32_t)((G / kStages) & 1))) {
                        ok = false;
                        break;
                    }
                    tc::fence_after();
                    const uint64_t so = (uint64_t)((st * kStageBytes) >> 4);
#pragma unroll
                    for (int sa = 0; sa < kSlices; ++sa) {
                        // the first MMA of a flush group writes every accumulator column
                        if (sa < 5)
                            tc::mma_bf16(tmem + wd::acc_col(b, sa, kBN), ad[sa] + so, bd[0] + so, idn[4 - sa],
                                         (sa == 0 && ks == kt) ? 0u : 1u);
                        tc::mma_bf16(tmem + wd::acc_col(b, 4, kBN), ad[sa] + so, bd[5 - sa] + so, idn[0], 1u);
                    }
                    tc::mma_commit(freeb(st));
                }
                if (!ok) break;
                tc::mma_commit(acc_full(b));
            }
        if (!ok) *s_fail = 1;
    } else if (warp >= 2) {
        // ---- epilogue: three warps per lane quarter (warp % 4); lane m of the
        // tile, columns 16 sub .. 16 sub + 15 read as two groups of 8 ----
        const int quarter = warp & 3, sub = (warp - 2) >> 2;
        const int ml = quarter * 32 + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
        const float two_f = __int_as_float((127 + kF) << 23);
        bool range_bad = false;
        int64_t Tt = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
            const int mb = t % nmb, nb = t / nmb;
            const int m = mb * 128 + ml;
            long long acc[2][8];
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[h][j] = 0;
            for (int64_t kt = 0; kt < P.nks; kt += kKTile, ++Tt) {
                const int b = (int)(Tt & 1);
                if (!tc::mbar_wait_bounded(acc_full(b), (uint32_t)((Tt >> 1) & 1))) {
                    ok = false;
                    break;
                }
                tc::fence_after();
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    uint32_t r[wd::kLevels][8];
#pragma unroll
                    for (int lv = 0; lv < wd::kLevels; ++lv)
                        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                                     : "=r"(r[lv][0]), "=r"(r[lv][1]), "=r"(r[lv][2]), "=r"(r[lv][3]), "=r"(r[lv][4]),
                                       "=r"(r[lv][5]), "=r"(r[lv][6]), "=r"(r[lv][7])
                                     : "r"(lane_base + wd::acc_col(b, lv, kBN) + (uint32_t)(16 * sub + 8 * h)));
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    if (h == 1) {  // the buffer is read: the next flush group may overwrite it
                        tc::fence_before();
                        tc::mbar_arrive(acc_empty(b));
                    }
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const float v2 = __uint_as_float(r[2][j]), v3 = __uint_as_float(r[3][j]);
                        range_bad |= !(fabsf(v2) <= 256.f) || !(fabsf(v3) <= 1.f);  // |.| <= 2^24 units
                        acc[h][j] += levels_to_int_f(__uint_as_float(r[0][j]), __uint_as_float(r[1][j]), v2, v3,
                                                     __uint_as_float(r[4][j]), kF, two_f);
                    }
                }
            }
            if (!ok) break;
            if (m < P.M) {
                const int eam = P.eA[m];
                const int ea = eam - 1022;
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int n = nb * kBN + 16 * sub + 8 * h + j;
                        if (n < P.N) {
                            // value = V 2^(eA + eB - 12 - f), eA/eB the unbiased exponents of the row
                            // maxima; a non-finite operand row (exponent 0x7FF) gives NaN
                            const int ebn = P.eB[n];
                            const double v = (eam == 0x7FF || ebn == 0x7FF)
                                                 ? __longlong_as_double(0x7FF8000000000000ll)
                                                 : sl::scaled_i64(acc[h][j], ea + (ebn - 1022) - 12 - kF);
                            double *o = P.out + (int64_t)n * P.ldo + m;
                            *o += v;
                        }
                    }
            }
        }
        if (!ok) *s_fail = 1;
        if (range_bad) atomicOr(P.err, 2);
    }
    // ---- exit: wait for every MMA this CTA issued and every copy it started,
    // then free tensor memory ----
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 1 && lane == 0) {
        tc::mma_commit(drain);
        if (!tc::mbar_wait_bounded(drain, 0u)) *s_fail = 1;
    }
    if (warp == 0 && lane == 0) {
        for (int st = 0; st < kStages; ++st) {
            const int64_t fills = G_copied / kStages + (st < G_copied % kStages ? 1 : 0);
            if (fills > 0 && !tc::mbar_wait_bounded(full(st), (uint32_t)((fills - 1) & 1))) *s_fail = 1;
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (*s_fail && tid == 0) atomicOr(P.err, 1);
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
}

}  // namespace ss

// The dense path applies when both spins have replacements, no string space
// exceeds 16384 strings (the planes of G stay below 2 GB) and the context asks
// for it (fci_options.f64_same_spin).
bool sigma_ss_ok(const fci_ctx *ctx) { return ctx->ssG_a != nullptr; }

int build_ss_tables(fci_ctx *ctx) {
    const SpinTables &A = ctx->A, &B = ctx->B;
    if (ctx->opt.f64_same_spin == FCI_SS_FAMILY) return FCI_OK;
    if (A.nsingle == 0 || B.nsingle == 0 || A.ns > 16384 || B.ns > 16384) return FCI_OK;
    int rc = FCI_OK;
    cudaStream_t s = ctx->stream;
    const bool shared = (&A == &B) || (A.gval == B.gval);
    auto build = [&](const SpinTables &T, unsigned char **planes, int **e) -> int {
        const size_t pb = ss::plane_bytes(T.ns, T.ns);
        *planes = (unsigned char *)dalloc(ctx, pb, &rc);
        *e = (int *)dalloc(ctx, sizeof(int) * (size_t)T.ns, &rc);
        if (rc) return rc;
        FCI_CUDA(cudaMemsetAsync(*planes, 0, pb, s));
        ss::k_ss_rowexp<<<ceil_div(T.ns, 256), 256, 0, s>>>(T.gval, T.ns, T.nsame, *e);
        ss::k_ss_gplanes<<<ceil_div(T.ns * (int64_t)T.nsame, 256), 256, 0, s>>>(T.gcol, T.gval, T.ns, T.nsame, *e,
                                                                                ss::pad_rows(T.ns), *planes);
        FCI_CUDA(cudaGetLastError());
        return FCI_OK;
    };
    if ((rc = build(A, &ctx->ssG_a, &ctx->ssE_a))) return rc;
    if (shared) {
        ctx->ssG_b = ctx->ssG_a;
        ctx->ssE_b = ctx->ssE_a;
    } else if ((rc = build(B, &ctx->ssG_b, &ctx->ssE_b))) {
        return rc;
    }
    // per-call workspace: C by rows (K = J_b) and by columns (K = J_a), and their exponents
    ctx->ssCr = (unsigned char *)dalloc(ctx, ss::plane_bytes(A.ns, B.ns), &rc);
    ctx->ssCc = (unsigned char *)dalloc(ctx, ss::plane_bytes(B.ns, A.ns), &rc);
    ctx->ssEr = (int *)dalloc(ctx, sizeof(int) * (size_t)(A.ns + B.ns + 1), &rc);
    if (rc) return rc;
    ctx->ssEc = ctx->ssEr + A.ns;
    // plane padding (rows past the strings, K past the last string) stays zero
    FCI_CUDA(cudaMemsetAsync(ctx->ssCr, 0, ss::plane_bytes(A.ns, B.ns), s));
    FCI_CUDA(cudaMemsetAsync(ctx->ssCc, 0, ss::plane_bytes(B.ns, A.ns), s));
    FCI_CUDA(opt_in_max_smem((const void *)ss::k_ss_tc, ctx->device));
    FCI_CUDA(cudaStreamSynchronize(s));
    return FCI_OK;
}

void free_ss_tables(fci_ctx *ctx) {
    const SpinTables &A = ctx->A, &B = ctx->B;
    if (ctx->ssG_b && ctx->ssG_b != ctx->ssG_a) {
        dfree(ctx, ctx->ssG_b, ss::plane_bytes(B.ns, B.ns));
        dfree(ctx, ctx->ssE_b, sizeof(int) * (size_t)B.ns);
    }
    if (ctx->ssG_a) {
        dfree(ctx, ctx->ssG_a, ss::plane_bytes(A.ns, A.ns));
        dfree(ctx, ctx->ssE_a, sizeof(int) * (size_t)A.ns);
    }
    dfree(ctx, ctx->ssCr, ss::plane_bytes(A.ns, B.ns));
    dfree(ctx, ctx->ssCc, ss::plane_bytes(B.ns, A.ns));
    dfree(ctx, ctx->ssEr, sizeof(int) * (size_t)(A.ns + B.ns + 1));
    ctx->ssG_a = ctx->ssG_b = ctx->ssCr = ctx->ssCc = nullptr;
    ctx->ssE_a = ctx->ssE_b = ctx->ssEr = ctx->ssEc = nullptr;
}

// sigma += sigma_1 (which = 1), sigma_2 (which = 2) or both (which = 3), in
// that order, from the dense planes.
static unsigned grid_stride(int64_t n) { return (unsigned)std::min<int64_t>((n + 255) / 256, 152 * 8); }

int launch_sigma_ss(fci_ctx *ctx, const double *C, double *sig, int which, cudaStream_t s, int rec, int slot) {
    const SpinTables &A = ctx->A, &B = ctx->B;
    const int64_t nsa = A.ns, nsb = B.ns;
    int nsm = 0;
    FCI_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device));
    auto gemm = [&](const unsigned char *Ap, int64_t rowsA, int M, const int *eA, const unsigned char *Bp, int64_t rowsB,
                    int N, const int *eB, int64_t K) -> int {
        ss::SsArgs P;
        P.A = Ap;
        P.B = Bp;
        P.rowsA = rowsA;
        P.rowsB = rowsB;
        P.M = M;
        P.N = N;
        P.nks = (K + 15) / 16;
        P.eA = eA;
        P.eB = eB;
        P.out = sig;
        P.ldo = nsb;
        P.err = ctx->d_err;
        const int64_t tiles = (int64_t)((M + 127) / 128) * ((N + ss::kBN - 1) / ss::kBN);
        const unsigned grid = (unsigned)std::min<int64_t>(tiles, nsm);
        ss::k_ss_tc<<<grid, ss::kThreads, ss::kSmem, s>>>(P);
        FCI_CUDA(cudaGetLastError());
        return FCI_OK;
    };
    // exponents of C's rows (I_a) and columns (I_b)
    FCI_CUDA(cudaMemsetAsync(ctx->ssEr, 0, sizeof(int) * (size_t)(nsa + nsb), s));
    ss::k_ss_cexp<<<dim3(ceil_div(nsb, 32), ceil_div(nsa, 32)), dim3(32, 8), 0, s>>>(C, nsa, nsb, ctx->ssEr, ctx->ssEc);
    FCI_CUDA(cudaGetLastError());
    if (which & 1) {  // sigma_1: A = G_b (m = I_b), B = C by rows (n = I_a), K = J_b
        ss::k_ss_cplanes<<<ceil_div(nsa * ((nsb + 7) / 8), 256), 256, 0, s>>>(C, nsa, nsb, 0, ctx->ssEr,
                                                                             ss::pad_rows(nsa), ctx->ssCr);
        FCI_CUDA(cudaGetLastError());
        if (int rc = gemm(ctx->ssG_b, ss::pad_rows(nsb), (int)nsb, ctx->ssE_b, ctx->ssCr, ss::pad_rows(nsa), (int)nsa,
                          ctx->ssEr, nsb))
            return rc;
        prof_mark(ctx, rec, slot, s);
        ++slot;
    }
    // the diagonal: both spins (which = 3), alpha only (which = 2: sigma_1 follows
    // as the parity transpose of sigma_2), beta only (which = 1)
    ss::k_ss_diag<<<grid_stride(nsa * nsb), 256, 0, s>>>(C, sig, which & 2 ? A.gval : nullptr,
                                                        which & 1 ? B.gval : nullptr, nsa, nsb);
    FCI_CUDA(cudaGetLastError());
    if (which & 2) {  // sigma_2: A = C by columns (m = I_b), B = G_a (n = I_a), K = J_a
        ss::k_ss_cplanes<<<ceil_div(nsb * ((nsa + 7) / 8), 256), 256, 0, s>>>(C, nsa, nsb, 1, ctx->ssEc,
                                                                             ss::pad_rows(nsb), ctx->ssCc);
        FCI_CUDA(cudaGetLastError());
        if (int rc = gemm(ctx->ssCc, ss::pad_rows(nsb), (int)nsb, ctx->ssEc, ctx->ssG_a, ss::pad_rows(nsa), (int)nsa,
                          ctx->ssE_a, nsa))
            return rc;
        prof_mark(ctx, rec, slot, s);
    }
    return FCI_OK;
}

}  // namespace fci
