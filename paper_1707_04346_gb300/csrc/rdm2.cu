// Spin-summed two-particle density Gamma_pqrs = <c| E_pq E_rs |c>, the
// density of the two-electron term of Eq. 6 (with gamma = <c|E_pq|c>,
// <c|H|c> = sum h_pq gamma_pq + 1/2 sum (pq|rs) (Gamma_pqrs - delta_qr gamma_ps)),
// the second half of the density step the paper runs after the Davidson
// iterations (Section 4, Table 2 "1e/2e Density Matrices").
//
// With the identity resolved over the determinants K of the space,
//   Gamma_pqrs = sum_K D_qp(K) D_rs(K),   D_rs(K) = <K| E_rs |c>,
//   gamma_pq   = sum_K c_K D_pq(K),
// so with D's rows (r, s) -> r n + s and one more row n^2 that holds c itself,
// the R x R Gram matrix G = D D^T (R = n^2 + 1) holds both densities.  For
// K = (K_a, K_b), each entry a+_k a_l |K_a> = sign |T> of K_a's
// single-replacement list (Eq. 7) gives <K_a| a+_l a_k |T> = sign, that is
// D_lk(K) += sign c(T, K_b); the entries of K_b's beta list give
// D_lk(K) += sign c(K_a, T) (k == l entries: the occupation numbers).  One
// spin's entries of one determinant have distinct (l, k), so D needs no
// atomics: the alpha entries are stored, then the beta entries added.
//
// G is a dense contraction over all N determinants, run on the bf16 tensor
// cores with FP64 accuracy in the way of the sliced sigma kernels:
//  * c in fixed point relative to its largest power of two (|c| < 2^eD),
//    X = round(c 2^(45 - eD)); D's values are exact integer sums of these
//    (|X_D| < 2^46, top digit in [-64, 64]), cut into six balanced 8-bit
//    digits that bf16 holds exactly;
//  * k_rdm2_fixed writes c's fixed-point integers once and k_rdm2_rows the D
//    row (l n + k) of every replacement-list entry;
//  * k_rdm2_digits writes, per K-step of 16 determinants, the six digit planes
//    of the R rows in the tensor cores' K-major no-swizzle layout (8 x 8 core
//    matrices of 128 bytes, 8-row groups 256 bytes apart), so that one bulk
//    copy per plane stages a whole operand tile;
//  * k_rdm2_tc computes tiles of 128 rows (A, the MMA's M) x 48 rows (B): the
//    six B planes are stacked along N and the five accumulators of an element
//    sit side by side in tensor memory, so that A digit s times B digits
//    0..4-s is one MMA writing weights s..4 and B digit 5-s one more into the
//    last accumulator (11 MMAs per K-step for the 21 digit products of weight
//    <= 5).  Weights 0-3 accumulate exact integers (at most 3 2^22 units
//    for 256 determinants, FP32 holds them up to 2^24; the first MMA of each
//    group of 256 overwrites the accumulators, so they need no resetting),
//    weights 4-5 in FP32; every 256
//    determinants the epilogue turns the five words into one 64-bit integer
//    and sums them in registers, and at the end of a work item adds them to
//    the integer G with red.global.add.u64 (exact and order-free).  The
//    256-determinant groups are fixed (K-steps 16j .. 16j + 15) and each is
//    accumulated in one order, so the result is the same bits on every run and
//    for every chunking.  Only tiles that hold some G[a][b] with
//    a <= b are computed (G is symmetric);
//  * k_rdm2_finish scales the integers to FP64 and permutes G into gamma and
//    Gamma.
// The integer unit is set per call from ||c||^2 (|G| <= 4 ||c||^2 stays below
// 2^60 units), so G is resolved to about 2^-59 ||c||^2.  Left out are the
// digit products of weight >= 6 (below 2^-46 of the leading product, zero
// mean) and c's fixed-point rounding (2^-46 of max |c|).
#include "sliced_mma.cuh"

#include <algorithm>
#include <cmath>

namespace fci {
namespace r2 {

using sl::kSlices;
using tc::kM;
using sm::bulk_g2s;
using sm::levels_to_int_f;
using sm::mbar_expect_tx;

constexpr int kThreads = 448;        // warp 0 copies, warp 1 issues the MMAs, warps 2-13 epilogue
constexpr int kEpiThreads = 384;
constexpr int kBN = 48;              // B rows per tile (the MMA's N per digit)
constexpr int kStages = 6;           // K-steps of operands in flight
constexpr int kKTile = 16;           // K-steps (256 determinants) per accumulator flush
constexpr int kKRange = 16;          // K-steps per work item (all tiles of one range meet in L2)
constexpr uint32_t kBytesA = 6 * 4096;       // six planes of 128 rows x 16
constexpr uint32_t kBytesB = 6 * kBN * 32;   // six planes of 48 rows x 16
constexpr uint32_t kStageBytes = kBytesA + kBytesB;
constexpr int kBars = 2 * kStages + 5;       // full[], free[], acc_full[2], acc_empty[2], drain
constexpr uint32_t kSmem = kStages * kStageBytes + kBars * 8 + 16;
constexpr int kStatBlocks = 1024;

// Fixed point of c relative to the largest biased exponent emax of the vector:
// round(|x| 2^(45 - eD)) with the sign of x, |x| < 2^eD.
__device__ __forceinline__ long long fixed45(double x, int emax) {
    const unsigned long long b = __double_as_longlong(x);
    return sl::fixed47((uint32_t)b, (uint32_t)(b >> 32), emax + 2);
}
__device__ __forceinline__ long long fixed45(float x, int emax) {
    const uint32_t b = __float_as_uint(x);
    const int ex = (int)((b >> 23) & 0xFFu);
    const long long m = (long long)((b & 0x7FFFFFu) | (ex ? 0x800000u : 0u));
    // x = m 2^(max(ex,1) - 150), eD = emax - 126: X = m 2^(max(ex,1) - emax + 21)
    const int sh = (ex ? ex : 1) - emax + 21;
    long long X;
    if (sh >= 0)
        X = m << sh;  // sh <= 21 since ex <= emax
    else
        X = -sh > 30 ? 0ll : (m + (1ll << (-sh - 1))) >> -sh;
    return (b >> 31) ? -X : X;
}

template <typename T>
__device__ __forceinline__ unsigned biased_exponent(T x);
template <>
__device__ __forceinline__ unsigned biased_exponent<double>(double x) {
    return (unsigned)((__double_as_longlong(x) >> 52) & 0x7FF);
}
template <>
__device__ __forceinline__ unsigned biased_exponent<float>(float x) {
    return (__float_as_uint(x) >> 23) & 0xFFu;
}

// Largest biased exponent of c (atomicMax) and per-block sums of c^2 (fixed
// grid of kStatBlocks blocks, summed on the host in block order).
template <typename T>
__global__ void __launch_bounds__(256) k_rdm2_stats(const T *__restrict__ c, int64_t n, int *__restrict__ emax,
                                                    double *__restrict__ part) {
    __shared__ double red[8];
    unsigned mx = 0;
    double s2 = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const T v = c[i];
        mx = max(mx, biased_exponent<T>(v));
        const double d = (double)v;
        s2 = fma(d, d, s2);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mx = max(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
        s2 += __shfl_xor_sync(0xFFFFFFFFu, s2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(emax, (int)mx);
        red[threadIdx.x >> 5] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}

// (l, k) of the entry a+_k a_l |x> = sign |t> (x, t bitmasks; pair index p of {k, l})
__device__ __forceinline__ void entry_orbitals(uint32_t x, uint32_t t, uint32_t p, int &l, int &k) {
    if (x != t) {
        l = __ffs(x & ~t) - 1;
        k = __ffs(t & ~x) - 1;
    } else {  // k == l: pair index l (l + 1) / 2 + l
        int o = 0;
        while ((uint32_t)(o * (o + 3) / 2) < p) ++o;
        l = k = o;
    }
}

// c in fixed point, once per call: Xc[i] = round(c_i 2^(45 - eD)).
template <typename T>
__global__ void k_rdm2_fixed(const T *__restrict__ c, int64_t n, int emax, long long *__restrict__ Xc) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) Xc[i] = fixed45(c[i], emax);
}

// rows[e * ns + x] = l n + k for the entry a+_k a_l |x> = sign |target> of
// string x (the row of D that the entry feeds), entry-major like SpinTables::tab.
__global__ void k_rdm2_rows(SpinTables S, int n, uint16_t *__restrict__ rows) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= S.ns * (int64_t)S.nsingle) return;
    const uint32_t ent = S.tab[t];
    int l, k;
    entry_orbitals(S.str[t % S.ns], S.str[ent_target(ent)], ent_pair(ent), l, k);
    rows[t] = (uint16_t)(l * n + k);
}

// One block per K-step of 16 determinants: the integers X_D of rows 0..Rd-1
// in shared memory (determinant-major with an odd stride, so that the 16
// determinants of one entry and the consecutive rows of the digit pass hit
// distinct banks), then their six digit planes into dg (K-step ks - ks0 of
// the chunk), plane t at byte (ks*6 + t) * Rd * 32, row r, determinant kk of
// the K-step at (r/8) 256 + (kk/8) 128 + (r%8) 16 + (kk%8) 2.
__global__ void __launch_bounds__(256) k_rdm2_digits(const long long *__restrict__ Xc, SpinTables A, SpinTables B,
                                                     const uint16_t *__restrict__ rows_a,
                                                     const uint16_t *__restrict__ rows_b, int n, int Rd, int64_t ks0,
                                                     int64_t N, uint4 *__restrict__ dg) {
    extern __shared__ __align__(16) long long X[];  // [16][Rd + 1]
    __shared__ int64_t s_ka[16];
    __shared__ int s_kb[16];
    const int Rs = Rd + 1;
    const int64_t ks = ks0 + blockIdx.x;
    const int64_t nsb = B.ns;
    const int crow = n * n;
    if (threadIdx.x < 16) {
        const int64_t K = ks * 16 + threadIdx.x;
        const int64_t ka = K / nsb;
        s_ka[threadIdx.x] = K < N ? ka : -1;
        s_kb[threadIdx.x] = (int)(K - ka * nsb);
    }
    for (int i = threadIdx.x; i < Rs * 16; i += blockDim.x) X[i] = 0;
    __syncthreads();
    // alpha entries (and the row of c): stored
    for (int it = threadIdx.x; it < (A.nsingle + 1) * 16; it += blockDim.x) {
        const int e = it >> 4, kk = it & 15;
        const int64_t ka = s_ka[kk];
        if (ka < 0) continue;
        const int64_t kb = s_kb[kk];
        if (e == A.nsingle) {
            X[kk * Rs + crow] = Xc[ka * nsb + kb];
            continue;
        }
        const int64_t at = (int64_t)e * A.ns + ka;
        const uint32_t ent = A.tab[at];
        const long long v = Xc[(int64_t)ent_target(ent) * nsb + kb];
        X[kk * Rs + rows_a[at]] = ent_negative(ent) ? -v : v;
    }
    __syncthreads();
    // beta entries: added
    for (int it = threadIdx.x; it < B.nsingle * 16; it += blockDim.x) {
        const int e = it >> 4, kk = it & 15;
        const int64_t ka = s_ka[kk];
        if (ka < 0) continue;
        const int64_t at = (int64_t)e * B.ns + s_kb[kk];
        const uint32_t ent = B.tab[at];
        const long long v = Xc[ka * nsb + ent_target(ent)];
        X[kk * Rs + rows_b[at]] += ent_negative(ent) ? -v : v;
    }
    __syncthreads();
    // digits: thread item it = (r/8) 16 + g 8 + r%8 owns 16 bytes at it*16 of each plane
    uint4 *base = dg + (ks - ks0) * 6 * (int64_t)Rd * 2;
    for (int it = threadIdx.x; it < Rd * 2; it += blockDim.x) {
        const int r = (it >> 4) * 8 + (it & 7), g = (it >> 3) & 1;
        uint32_t w[kSlices][4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float f0[kSlices], f1[kSlices];
            sl::digits6(X[(g * 8 + 2 * i) * Rs + r], f0);
            sl::digits6(X[(g * 8 + 2 * i + 1) * Rs + r], f1);
#pragma unroll
            for (int s = 0; s < kSlices; ++s) w[s][i] = sl::pack_bf16(f0[s], f1[s]);
        }
#pragma unroll
        for (int s = 0; s < kSlices; ++s) base[(int64_t)s * Rd * 2 + it] = make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
    }
}

// Row block rb (128 rows) and column block cb (48 rows) of tile `tile` among
// the tiles that hold some (a, b) with a <= b: cb*48 + 47 >= rb*128.
__device__ __forceinline__ void tile_blocks(int tile, int nrb, int ncb, int &rb, int &cb) {
    for (rb = 0; rb < nrb; ++rb) {
        const int c0 = rb * 128 > 47 ? (rb * 128 - 47 + kBN - 1) / kBN : 0;
        const int cnt = ncb - c0;
        if (tile < cnt) {
            cb = c0 + tile;
            return;
        }
        tile -= cnt;
    }
    cb = 0;
}

struct TcArgs {
    const unsigned char *dg;  // digit planes of the chunk
    int64_t nks;              // K-steps in the chunk
    int Rd, R, nrb, ncb, ntile;
    int f;                    // integer unit 2^-f of the accumulator scale
    unsigned long long *G;    // [Rd][Rd] integers, G[b * Rd + a] for a <= b
    int *err;
};

// Work of CTA b: with at least ntile CTAs (a multiple of ntile), CTA b keeps
// tile b % ntile for the whole launch and takes the K-ranges g, g + ng, ...
// (g = b / ntile, ng = grid / ntile), so that its sums stay in registers and
// the ntile CTAs of a group read each K-range at about the same time; with
// fewer CTAs than tiles, CTA b takes tiles b, b + grid, ... over every K-range.
struct Work {
    int t0, tstep, g, ng;
    __device__ Work(int ntile) {
        if ((int)gridDim.x >= ntile) {
            t0 = blockIdx.x % ntile;
            tstep = ntile;
            g = blockIdx.x / ntile;
            ng = gridDim.x / ntile;
        } else {
            t0 = blockIdx.x;
            tstep = gridDim.x;
            g = 0;
            ng = 1;
        }
    }
};

__global__ void __launch_bounds__(kThreads, 1) k_rdm2_tc(TcArgs P) {
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
    const int64_t nkr = (P.nks + kKRange - 1) / kKRange;
    const Work W(P.ntile);

    // zero the operand stages once: rows past the end of a partial tile then
    // hold finite digits (their lanes and columns are not read back)
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
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tslot;
    tc::fence_async_smem();  // the zeroed stages, before the bulk copies and MMAs read or write them
    tc::fence_before();
    __syncthreads();
    tc::fence_after();

    int64_t G_copied = 0;  // K-steps whose copies warp 0 issued
    if (warp == 0 && lane == 0) {
        // ---- copies: the A and B planes of one K-step per stage ----
        int64_t &G = G_copied;
        for (int t = W.t0; t < P.ntile && !*s_fail; t += W.tstep) {
            int rb, cb;
            tile_blocks(t, P.nrb, P.ncb, rb, cb);
            const uint32_t ba = (uint32_t)min(128, P.Rd - rb * 128) * 32u;
            const uint32_t bb = (uint32_t)min(kBN, P.Rd - cb * kBN) * 32u;
            for (int64_t kr = W.g; kr < nkr && !*s_fail; kr += W.ng) {
                const int64_t k1 = min(P.nks, (kr + 1) * kKRange);
                for (int64_t ks = kr * kKRange; ks < k1; ++ks, ++G) {
                    const int st = (int)(G % kStages);
                    if (G >= kStages && !tc::mbar_wait_bounded(freeb(st), (uint32_t)((G / kStages - 1) & 1))) {
                        *s_fail = 1;
                        break;
                    }
                    mbar_expect_tx(full(st), 6u * (ba + bb));
                    const unsigned char *src = P.dg + (size_t)ks * 6 * P.Rd * 32;
                    const uint32_t dst = sbase + (uint32_t)st * kStageBytes;
#pragma unroll
                    for (int p = 0; p < 6; ++p) {
                        bulk_g2s(dst + (uint32_t)p * 4096u, src + ((size_t)p * P.Rd + rb * 128) * 32, ba, full(st));
                        bulk_g2s(dst + kBytesA + (uint32_t)p * kBN * 32u, src + ((size_t)p * P.Rd + cb * kBN) * 32, bb,
                                 full(st));
                    }
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
        for (int t = W.t0; t < P.ntile && ok; t += W.tstep)
            for (int64_t kr = W.g; kr < nkr && ok; kr += W.ng) {
                const int64_t k1 = min(P.nks, (kr + 1) * kKRange);
                for (int64_t kt = kr * kKRange; kt < k1 && ok; kt += kKTile, ++Tt) {
                    const int b = (int)(Tt & 1);
                    if (Tt >= 2 && !tc::mbar_wait_bounded(acc_empty(b), (uint32_t)(((Tt - 2) >> 1) & 1))) {
                        ok = false;
                        break;
                    }
                    tc::fence_after();
                    const int64_t ke = min(k1, kt + kKTile);
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
                            // the first MMA of a flush group writes every accumulator
                            // column (weights 0..4), so it overwrites instead of adding
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
            }
        if (!ok) *s_fail = 1;
    } else if (warp >= 2) {
        // ---- epilogue: three warps per lane quarter (warp % 4); lane m of the
        // tile, columns 16 sub .. 16 sub + 15 read as two groups of 8 ----
        const int quarter = warp & 3, sub = (warp - 2) >> 2;
        const int m = quarter * 32 + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
        const float two_f = __int_as_float((127 + P.f) << 23);
        bool range_bad = false;
        int64_t Tt = 0;
        bool ok = true;
        for (int t = W.t0; t < P.ntile && ok; t += W.tstep) {
            int rb, cb;
            tile_blocks(t, P.nrb, P.ncb, rb, cb);
            const int row = rb * 128 + m;
            long long acc[2][8];
            uint32_t live = 0;  // bit 8 h + j: element (row, column 16 sub + 8 h + j) is read back
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    acc[h][j] = 0;
                    const int col = cb * kBN + 16 * sub + 8 * h + j;
                    if (row < P.R && col < P.R && col >= row) live |= 1u << (8 * h + j);
                }
            for (int64_t kr = W.g; kr < nkr && ok; kr += W.ng) {
                const int64_t k1 = min(P.nks, (kr + 1) * kKRange);
                for (int64_t kt = kr * kKRange; kt < k1; kt += kKTile, ++Tt) {
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
                                         : "=r"(r[lv][0]), "=r"(r[lv][1]), "=r"(r[lv][2]), "=r"(r[lv][3]),
                                           "=r"(r[lv][4]), "=r"(r[lv][5]), "=r"(r[lv][6]), "=r"(r[lv][7])
                                         : "r"(lane_base + wd::acc_col(b, lv, kBN) + (uint32_t)(16 * sub + 8 * h)));
                        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                        if (h == 1) {  // the buffer is read: the next flush group may overwrite it
                            tc::fence_before();
                            tc::mbar_arrive(acc_empty(b));
                        }
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            if (live >> (8 * h + j) & 1u) {
                                const float v2 = __uint_as_float(r[2][j]), v3 = __uint_as_float(r[3][j]);
                                range_bad |= !(fabsf(v2) <= 256.f) || !(fabsf(v3) <= 1.f);  // |.| <= 2^24 units
                                acc[h][j] += levels_to_int_f(__uint_as_float(r[0][j]), __uint_as_float(r[1][j]), v2, v3,
                                                             __uint_as_float(r[4][j]), P.f, two_f);
                            }
                    }
                }
            }
            if (!ok) break;
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (live >> (8 * h + j) & 1u) {
                        const int col = cb * kBN + 16 * sub + 8 * h + j;
                        atomicAdd(P.G + (size_t)col * P.Rd + row, (unsigned long long)acc[h][j]);
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
    if (warp == 0 && lane == 0) {  // at once unless a wait gave up
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

// Gamma[p][q][r][s] = G[qp][rs] and gamma[p][q] = G[c][pq] as FP64 (G[a][b]
// read at a <= b), scaled by 2^e2; NaN everywhere when c held a non-finite value.
__global__ void k_rdm2_finish(const long long *__restrict__ G, int Rd, int n, int e2, int nonfinite,
                              double *__restrict__ g2, double *__restrict__ g1) {
    const int64_t n2 = (int64_t)n * n, n4 = n2 * n2;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n4 + n2) return;
    int64_t a, b;
    if (i < n4) {
        const int p = (int)(i / (n2 * n)), q = (int)((i / n2) % n), rs = (int)(i % n2);
        a = (int64_t)q * n + p;
        b = rs;
    } else {
        a = n2;
        b = i - n4;
    }
    const int64_t lo = a < b ? a : b, hi = a < b ? b : a;
    const double v = nonfinite ? __longlong_as_double(0x7FF8000000000000ll) : sl::scaled_i64(G[hi * Rd + lo], e2);
    if (i < n4)
        g2[i] = v;
    else
        g1[i - n4] = v;
}

inline unsigned grid_blocks(int64_t n) { return (unsigned)std::min<int64_t>((n + 255) / 256, 152 * 16); }

template <typename T>
int rdm2_impl(fci_ctx *ctx, const T *C, double *g1_host, double *g2_host) {
    const int n = ctx->norb;
    const int R = n * n + 1, Rd = (R + 7) / 8 * 8;
    const int64_t N = ctx->ndet, nks = (N + 15) / 16;
    const int64_t n2 = (int64_t)n * n, n4 = n2 * n2;
    const int nrb = (Rd + 127) / 128, ncb = (Rd + kBN - 1) / kBN;
    int ntile = 0;
    for (int rb = 0; rb < nrb; ++rb) ntile += ncb - (rb * 128 > 47 ? (rb * 128 - 47 + kBN - 1) / kBN : 0);
    cudaStream_t s = ctx->stream;
    const size_t step_bytes = (size_t)6 * Rd * 32;
    size_t budget = ctx->opt.rdm2_chunk_bytes > 0 ? (size_t)ctx->opt.rdm2_chunk_bytes : ((size_t)1 << 30);
    // whole flush groups per chunk: every 256-determinant group K-steps [16j, 16j + 16)
    // is accumulated in the same order whatever the chunking, so the result is
    // the same bits for every chunk size
    int64_t chunk = (int64_t)(budget / step_bytes);
    if (chunk < nks) chunk = std::max<int64_t>(kKTile, chunk / kKTile * kKTile);
    if (chunk > nks) chunk = nks;
    const size_t gbytes = sizeof(long long) * (size_t)Rd * Rd;
    const size_t obytes = sizeof(double) * (size_t)(n4 + n2);
    const size_t sbytes = sizeof(int) * 2 + sizeof(double) * kStatBlocks;
    const size_t xbytes = sizeof(long long) * (size_t)N;
    const size_t rbytes = sizeof(uint16_t) * ((size_t)ctx->A.ns * ctx->A.nsingle + (size_t)ctx->B.ns * ctx->B.nsingle + 8);
    int rc = FCI_OK;
    unsigned char *dg = (unsigned char *)dalloc(ctx, step_bytes * (size_t)chunk, &rc);
    long long *G = rc ? nullptr : (long long *)dalloc(ctx, gbytes, &rc);
    double *out = rc ? nullptr : (double *)dalloc(ctx, obytes, &rc);
    unsigned char *stat = rc ? nullptr : (unsigned char *)dalloc(ctx, sbytes, &rc);
    long long *Xc = rc ? nullptr : (long long *)dalloc(ctx, xbytes, &rc);
    uint16_t *rows = rc ? nullptr : (uint16_t *)dalloc(ctx, rbytes, &rc);
    auto release = [&]() {
        dfree(ctx, dg, step_bytes * (size_t)chunk);
        dfree(ctx, G, gbytes);
        dfree(ctx, out, obytes);
        dfree(ctx, stat, sbytes);
        dfree(ctx, Xc, xbytes);
        dfree(ctx, rows, rbytes);
    };
    if (rc) {
        release();
        return rc;
    }
    int *d_emax = reinterpret_cast<int *>(stat), *d_err = d_emax + 1;
    double *d_part = reinterpret_cast<double *>(stat + 2 * sizeof(int));
    std::vector<double> part(kStatBlocks);
    int emax = 0, herr = 0;
    // per-kernel timing (fci_profile_*) when the call runs as one chunk
    static const char *const names[5] = {"rdm2_stats", "rdm2_prep", "rdm2_digits", "rdm2_tc", "rdm2_finish"};
    const int rec = chunk >= nks ? prof_begin(ctx, s, 5, names) : -1;
    cudaError_t e = cudaMemsetAsync(stat, 0, sbytes, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(G, 0, gbytes, s);
    if (e == cudaSuccess) {
        k_rdm2_stats<T><<<kStatBlocks, 256, 0, s>>>(C, N, d_emax, d_part);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&emax, d_emax, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(part.data(), d_part, sizeof(double) * kStatBlocks, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        release();
        return cuda_fail(e, "rdm2 statistics");
    }
    prof_mark(ctx, rec, 0, s);
    const int emax_inf = sizeof(T) == 8 ? 0x7FF : 0xFF;
    const int nonfinite = emax >= emax_inf;
    double norm2 = 0.0;
    for (double v : part) norm2 += v;
    int e2 = 0;
    if (!nonfinite && emax > 0 && norm2 > 0.0) {
        const int eD = sizeof(T) == 8 ? emax - 1022 : emax - 126;  // |c| < 2^eD
        int ex = 0;
        const double m = std::frexp(norm2, &ex);                   // norm2 = m 2^ex, m in [0.5, 1)
        const int lg = m > 0.5 ? ex : ex - 1;                      // ceil(log2 norm2)
        int f = 48 + 2 * eD - lg;                                  // 4 ||c||^2 2^(10 - 2 eD + f) <= 2^60
        if (f > 52) f = 52;
        e2 = 2 * eD - 10 - f;
        // the FP32 sums of c^2 may sit slightly below the exact norm: one bit of margin
        f -= 1;
        e2 += 1;
        FCI_CUDA(opt_in_max_smem((const void *)k_rdm2_digits, ctx->device));
        const SpinTables &SA = ctx->A, &SB = ctx->B;
        uint16_t *rows_a = rows, *rows_b = rows + (size_t)SA.ns * SA.nsingle;
        k_rdm2_fixed<T><<<grid_blocks(N), 256, 0, s>>>(C, N, emax, Xc);
        if (SA.nsingle) k_rdm2_rows<<<ceil_div(SA.ns * (int64_t)SA.nsingle, 256), 256, 0, s>>>(SA, n, rows_a);
        if (SB.nsingle) k_rdm2_rows<<<ceil_div(SB.ns * (int64_t)SB.nsingle, 256), 256, 0, s>>>(SB, n, rows_b);
        FCI_CUDA(cudaGetLastError());
        prof_mark(ctx, rec, 1, s);
        FCI_CUDA(cudaFuncSetAttribute((const void *)k_rdm2_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem));
        int nsm = 0;
        FCI_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device));
        for (int64_t k0 = 0; k0 < nks && e == cudaSuccess; k0 += chunk) {
            const int64_t kn = std::min<int64_t>(chunk, nks - k0);
            k_rdm2_digits<<<(unsigned)kn, 256, (size_t)(Rd + 1) * 16 * sizeof(long long), s>>>(
                Xc, SA, SB, rows_a, rows_b, n, Rd, k0, N, reinterpret_cast<uint4 *>(dg));
            e = cudaGetLastError();
            if (e != cudaSuccess) break;
            prof_mark(ctx, rec, 2, s);
            TcArgs P;
            P.dg = dg;
            P.nks = kn;
            P.Rd = Rd;
            P.R = R;
            P.nrb = nrb;
            P.ncb = ncb;
            P.ntile = ntile;
            P.f = f;
            P.G = reinterpret_cast<unsigned long long *>(G);
            P.err = d_err;
            // a multiple of ntile CTAs (one tile each) when the tiles fit the
            // SMs, no more groups than K-ranges
            const int64_t nkr = (kn + kKRange - 1) / kKRange;
            const unsigned grid = ntile <= nsm ? (unsigned)(ntile * std::min<int64_t>(nsm / ntile, nkr)) : (unsigned)nsm;
            k_rdm2_tc<<<grid, kThreads, kSmem, s>>>(P);
            e = cudaGetLastError();
            prof_mark(ctx, rec, 3, s);
        }
    }
    if (nonfinite || emax == 0 || !(norm2 > 0.0)) {  // nothing to contract: empty timing slots
        prof_mark(ctx, rec, 1, s);
        prof_mark(ctx, rec, 2, s);
        prof_mark(ctx, rec, 3, s);
    }
    if (e == cudaSuccess) {
        k_rdm2_finish<<<ceil_div(n4 + n2, 256), 256, 0, s>>>(G, Rd, n, e2, nonfinite, out, out + n4);
        e = cudaGetLastError();
        prof_mark(ctx, rec, 4, s);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(g2_host, out, sizeof(double) * n4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && g1_host) e = cudaMemcpyAsync(g1_host, out + n4, sizeof(double) * n2, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    release();
    if (e != cudaSuccess) return cuda_fail(e, "rdm2");
    if (herr & 1) return fail(FCI_ERR_TIMEOUT, "rdm2: a bounded wait in the tensor-core kernel gave up");
    if (herr) return fail(FCI_ERR_RANGE, "rdm2: an exact accumulator left its range");
    return FCI_OK;
}

}  // namespace r2

int run_rdm2(fci_ctx *ctx, const void *c, int dtype, double *gamma1, double *gamma2) {
    if (dtype == FCI_F64) return r2::rdm2_impl<double>(ctx, (const double *)c, gamma1, gamma2);
    return r2::rdm2_impl<float>(ctx, (const float *)c, gamma1, gamma2);
}

}  // namespace fci
