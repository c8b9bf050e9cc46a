// FP64-accurate sigma_3 (the alpha-beta term of Eq. 8) on the bf16 tensor
// cores (tcgen05, sm_103a), for FP64 CI vectors.
//
// Per output alpha string I_a with replacement list a = (J_a, p_a, s_a), as in
// the FP32 kernel (sigma_tc_kernel.cuh):
//   G[J_b][q] = sum_a C(J_a, J_b) * s_a (q | p_a)           (contraction, K = a)
//   sigma(I_a, I_b) = sum over beta replacements a+_k a_l |J_b> = s_b |I_b>,
//                     pair q = {k, l}, of s_b G[J_b][q]      (scatter)
//
// FP64-accurate contraction from 8-bit slices (Ozaki splitting):
//  * a pre-pass writes every C value in fixed point relative to the largest
//    power of two of its own row, X = round(|C| 2^(47 - e_row)) with the sign,
//    cut into six balanced 8-bit digits X = d0 2^40 + d1 2^32 + ... + d5,
//    |d_s| <= 128 (the low digits are centred on zero, so the products that
//    are left out have zero mean), stored as the bf16 values d_s 2^(-8s),
//    which bf16 holds exactly (12 bytes per determinant, two planes);
//  * per alpha row, the rows J_a it gathers share the largest of their
//    exponents, eD; the factor 2^(e_row(J_a) - eD) of each replacement is
//    folded into the integral operand, whose digits are rebuilt per row from
//    the context's fixed-point integrals round((pq|rs) 2^(47 - eW)) shifted
//    right by eD - e_row(J_a), with the sign s_a;
//  * the 21 slice products s + t <= 5 run on the tensor cores with FP32
//    accumulation in tensor memory, one accumulator per level L = s + t for
//    L = 0, 1, 2 and one shared by L >= 3.  A level-L product is an integer
//    times 2^(-8L) of magnitude <= 2^14, so with K <= 85 replacements every
//    level sum stays below 2^22 units and levels 0-2 are exact; the shared
//    accumulator rounds at 2^-24 of level 3, 2^-48 of the leading level;
//  * the epilogue turns the four level sums of G[J_b][q] into one integer
//    V = round(2^34 sum_L acc_L) (units 2^(eD + eW - 48)) without conversion
//    instructions (GB300 runs float-integer conversions on its slow FP64
//    pipe): levels 0-2 accumulate on biases that leave their integers in the
//    low mantissa bits, level 3+ is rounded with FP32 magic-number additions.
//    It adds s_b V into the target's 64-bit slot of the sigma row in shared
//    memory with an integer atomic: the adds are exact and their order does
//    not matter, so the result is bit-reproducible;
//  * at the end of the row the integers are converted to FP64 (integer
//    arithmetic only, round to nearest even) and written to sigma, which this
//    kernel overwrites (or adds to, when add != 0).
// Per product the representation and the products left out (s + t >= 6) are
// below about 2^-46 of (largest gathered |C|) x (largest |(pq|rs)|).
//
// The beta table by pair (SpinTables::tabp, 16-bit entries, npad per string)
// gives, for lane J_b and pair column q of the accumulator, the one replacement
// of J_b with pair q (if any), so the epilogue reads the accumulator lane by
// lane from tensor memory with compile-time register indices and needs no
// staging of G; one 16-byte load brings the entries of 8 columns.
//
// CTA (416 threads), one per SM, persistent over alpha rows:
//  * warps 0-3 (producers): thread m gathers the sliced values C(J_a, J_b) of
//    beta string J_b = 128 t + m and transposes them into the six A slices,
//    K-major (no swizzle) in shared memory; each K-step (16 replacements) sits
//    behind its own pair of barriers so that the next tile's slices are written
//    while the tensor cores finish this one;
//  * warp 12 (one thread) issues the MMAs: per tile, the accumulator columns
//    are split in two halves (pairs 0..N0-1 and N0..npad-1), each with its own
//    four level accumulators, so the epilogue of one half overlaps the MMAs of
//    the other;
//  * warps 4-11 (epilogue): two warps per tensor-memory lane quarter, taking
//    alternate 8-column chunks.
// All waits are bounded; a wait that gives up sets the device error word and
// the CTA drains its MMAs and frees its tensor memory.
#pragma once
#include "sigma_tc_kernel.cuh"

namespace fci {
namespace sl {

using tc::kM;

constexpr int kSlices = 6;    // 8-bit digits per FP64 operand (48 bits)
constexpr int kThreads = 416; // warps 0-3 producers, 4-11 epilogue, 12 MMA issuer
constexpr int kEpiThreads = 256;
constexpr int kMaxKSteps = 6; // K <= 96 (the exact level sums need K <= 85)
constexpr int kMaxK = 85;
constexpr int kBars = 2 * kMaxKSteps + 5;  // a_full[6], a_free[6], acc_full[2], acc_empty[2], drain

struct Layout {
    uint32_t bytesA, bytesB, offA, offAcc, offEa, offBar, total;
};

// Shared memory: B slices [6][npad x kpad], A slices [6][128 x kpad], the sigma
// row as 64-bit integers [nsb], the alpha list [nsingle_a], barriers and words.
__host__ __device__ inline Layout make_layout(int kpad, int npad, int64_t nsb, int nsingle_a) {
    Layout L;
    L.bytesB = (uint32_t)(npad * kpad * 2);
    L.bytesA = (uint32_t)(kM * kpad * 2);
    L.offA = (uint32_t)kSlices * L.bytesB;
    L.offAcc = L.offA + (uint32_t)kSlices * L.bytesA;
    L.offEa = L.offAcc + (uint32_t)(((nsb * 8) + 15) / 16 * 16);
    L.offBar = L.offEa + (uint32_t)(((nsingle_a + 3) / 4) * 16);
    L.total = L.offBar + kBars * 8 + 16;  // barriers, fail word, tmem slot, row exponent
    return L;
}

// Fixed point of an FP64 value (raw bits lo, hi) relative to the biased row
// exponent emax: round(|x| 2^(47 - eD)) with the sign of x, eD = emax - 1022
// (|x| < 2^eD, so |X| <= 2^47).
__device__ __forceinline__ long long fixed47(uint32_t lo, uint32_t hi, int emax) {
    const int ex = (int)((hi >> 20) & 0x7FFu);
    const int sh = emax + 6 - ex;  // >= 6 when ex <= emax
    unsigned long long m = ((unsigned long long)((hi & 0xFFFFFu) | 0x100000u) << 32) | lo;
    m = (ex == 0 || sh >= 60 || sh < 6) ? 0ull : ((m + (1ull << (sh - 1))) >> sh);
    const long long X = (long long)m;
    return (hi >> 31) ? -X : X;
}

// The six balanced digits of a fixed-point value |X| <= 2^47 as the floats
// d_s 2^(-8s) (exact): with X' = X + 0x8080808080, d0 = X' >> 40 in
// [-128, 128] and d_s = (byte 5-s of X') - 128 in [-128, 127].  Only FP32 and
// integer operations (no conversion instructions).
__device__ __forceinline__ void digits6(long long X, float (&f)[kSlices]) {
    X += 0x8080808080ll;
    const int h32 = (int)(X >> 32);
    const uint32_t l32 = (uint32_t)X;
    f[0] = __int_as_float(0x4B400000 + (h32 >> 8)) - 12582912.0f;  // 1.5 2^23 + d0, exact for |d0| < 2^22
    // byte b: 2^23 + b from a byte permute with the exponent byte 0x4B, then
    // (2^23 + b) 2^(-8s) - (2^23 + 128) 2^(-8s) = (b - 128) 2^(-8s) in one exact FMA
    f[1] = fmaf(__uint_as_float(__byte_perm((uint32_t)h32, 0x4B000000u, 0x7440)), 0x1p-8f, -32768.5f);
    f[2] = fmaf(__uint_as_float(__byte_perm(l32, 0x4B000000u, 0x7443)), 0x1p-16f, -(0x1p7f + 0x1p-9f));
    f[3] = fmaf(__uint_as_float(__byte_perm(l32, 0x4B000000u, 0x7442)), 0x1p-24f, -(0x1p-1f + 0x1p-17f));
    f[4] = fmaf(__uint_as_float(__byte_perm(l32, 0x4B000000u, 0x7441)), 0x1p-32f, -(0x1p-9f + 0x1p-25f));
    f[5] = fmaf(__uint_as_float(__byte_perm(l32, 0x4B000000u, 0x7440)), 0x1p-40f, -(0x1p-17f + 0x1p-33f));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&h);
}

// T * 2^e2 as FP64, by integer arithmetic (round to nearest even; results
// below the normal range flush to zero).
__device__ __forceinline__ double scaled_i64(long long T, int e2) {
    if (T == 0) return 0.0;
    const unsigned long long sgn = T < 0 ? 0x8000000000000000ull : 0ull;
    unsigned long long m = T < 0 ? (unsigned long long)(-T) : (unsigned long long)T;
    int n = 63 - __clzll((long long)m);
    if (n > 52) {
        const int sh = n - 52;
        const unsigned long long rem = m & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
        m >>= sh;
        if (rem > half || (rem == half && (m & 1ull))) {
            m += 1ull;
            if (m >> 53) {
                m >>= 1;
                n += 1;
            }
        }
    } else {
        m <<= (52 - n);
    }
    const int E = n + e2 + 1023;
    if (E <= 0) return __longlong_as_double((long long)sgn);
    if (E >= 2047) return __longlong_as_double((long long)(sgn | 0x7FF0000000000000ull));
    return __longlong_as_double((long long)(sgn | ((unsigned long long)E << 52) | (m & 0xFFFFFFFFFFFFFull)));
}

__device__ __forceinline__ void ld_early_v2(const uint2 *p, uint32_t &x, uint32_t &y) {
    asm volatile("ld.global.nc.v2.u32 {%0, %1}, [%2];" : "=r"(x), "=r"(y) : "l"(p));
}

// round(X 2^-d) for d >= 0 (zero once d >= 60)
__device__ __forceinline__ long long round_shift(long long X, int d) {
    if (d <= 0) return X;
    if (d >= 60) return 0;
    return (X + (1ll << (d - 1))) >> d;
}

// Levels 0-2 accumulate on a bias that puts their integers in the low mantissa
// bits: 1.5 2^23 (level 0, integers), 1.5 2^15 (level 1, multiples of 2^-8),
// 1.5 2^7 (level 2, multiples of 2^-16); with every level sum below 2^22 units
// the accumulator stays in [2^(e), 2^(e+1)) and its bit pattern minus the
// bias's is the integer.  Level 3 and above accumulates from zero.
constexpr uint32_t kBias0 = 0x4B400000u, kBias1 = 0x47400000u, kBias2 = 0x43400000u;

// The integer V = round(2^34 (acc0 + acc1 + acc2 + acc3)) of one accumulator
// element, times the sign of the replacement (neg = 1: negative), from the raw
// accumulator words (levels 0-2 biased): 2^34 acc0 + 2^34 acc1 = (i0 2^8 + i1)
// 2^26, 2^34 acc2 = i2 2^18, and acc3 is split into h = round(2^18 acc3) and an
// exact remainder rounded at 2^-34.
__device__ __forceinline__ long long levels_to_int(uint32_t r0, uint32_t r1, uint32_t r2, uint32_t r3, uint32_t neg) {
    constexpr float M = 12582912.0f;  // 1.5 2^23
    constexpr int MB = 0x4B400000;    // its bit pattern
    int hi = (int)(r0 * 256u + r1 - (kBias0 * 256u + kBias1));  // i0 2^8 + i1, exact modulo 2^32
    int i2 = (int)(r2 - kBias2);
    const float a3 = __uint_as_float(r3 ^ (neg << 31));
    const float t = fmaf(a3, 262144.f, M);
    const int h = __float_as_int(t) - MB;
    const float rem = fmaf(-(t - M), 0x1p-18f, a3);  // exact: a3 - h 2^-18
    const int l = __float_as_int(fmaf(rem, 0x1p34f, M)) - MB;
    if (neg) {
        hi = -hi;
        i2 = -i2;
    }
    return ((long long)hi << 26) + ((long long)(i2 * 4 + h) << 16) + l;
}

__device__ __forceinline__ uint4 ld_early_v4(const uint4 *p) {
    uint4 v;
    asm volatile("ld.global.nc.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
    return v;
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, uint32_t v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1};" ::"r"(taddr), "r"(v)
                 : "memory");
}

// tensor-memory column of level L of accumulator half h
__device__ __forceinline__ uint32_t acc_col(int h, int L, int n0, int n1) {
    return (uint32_t)(h == 0 ? L * n0 : 4 * n0 + L * n1);
}

template <int KPAD>
__global__ void __launch_bounds__(kThreads, 1)
    k_sigma3_sliced(const uint2 *__restrict__ cs0123, const uint32_t *__restrict__ cs45, double *__restrict__ sig,
                    SpinTables A, SpinTables B, const long long *__restrict__ XW, const int *__restrict__ rowexp,
                    int npair, int npad, int n0, int eW, int *err, const int *__restrict__ active, int add) {
    if (active != nullptr && *active == 0) return;  // gated launch (batched engine): instance not active
    constexpr int NKS = KPAD / 16;
    constexpr int kgroups = KPAD / 8;
    constexpr uint32_t sbo = (uint32_t)(KPAD / 8) * 128u;
    extern __shared__ __align__(1024) unsigned char smem[];
    const int64_t nsb = B.ns;
    const Layout L = make_layout(KPAD, npad, nsb, A.nsingle);
    unsigned char *sB = smem;
    unsigned char *sA = smem + L.offA;
    unsigned long long *sAcc = reinterpret_cast<unsigned long long *>(smem + L.offAcc);
    uint32_t *sEa = reinterpret_cast<uint32_t *>(smem + L.offEa);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + L.offBar);
    volatile int *s_fail = reinterpret_cast<volatile int *>(smem + L.offBar + kBars * 8);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + L.offBar + kBars * 8 + 4);
    volatile int *s_emax = reinterpret_cast<volatile int *>(smem + L.offBar + kBars * 8 + 8);
    const uint32_t bar0 = tc::smem_u32(bars);
    auto a_full = [&](int ks) { return bar0 + 8u * (uint32_t)ks; };
    auto a_free = [&](int ks) { return bar0 + 8u * (uint32_t)(kMaxKSteps + ks); };
    auto acc_full = [&](int h) { return bar0 + 8u * (uint32_t)(2 * kMaxKSteps + h); };
    auto acc_empty = [&](int h) { return bar0 + 8u * (uint32_t)(2 * kMaxKSteps + 2 + h); };
    const uint32_t drain = bar0 + 8u * (uint32_t)(2 * kMaxKSteps + 4);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int sa_n = A.nsingle;
    const int n1 = npad - n0;
    const int nh = n1 > 0 ? 2 : 1;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(tslot)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < NKS; ++i) {
            tc::mbar_init(a_full(i), 128);
            tc::mbar_init(a_free(i), 1);
        }
        for (int h = 0; h < 2; ++h) {
            tc::mbar_init(acc_full(h), 1);
            tc::mbar_init(acc_empty(h), kEpiThreads);
        }
        tc::mbar_init(drain, 1);
        *s_fail = 0;
    }
    for (int64_t j = tid; j < nsb; j += kThreads) sAcc[j] = 0ull;
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tslot;
    if (warp >= 4 && warp < 12) {  // level 0-2 biases of both accumulator halves (this warp's chunks)
        const uint32_t lb = tmem + ((uint32_t)((warp & 3) * 32) << 16);
        for (int h = 0; h < nh; ++h)
            for (int c = (warp - 4) >> 2; c < (h ? n1 : n0) / 8; c += 2) {
                tmem_st8(lb + acc_col(h, 0, n0, n1) + (uint32_t)(c * 8), kBias0);
                tmem_st8(lb + acc_col(h, 1, n0, n1) + (uint32_t)(c * 8), kBias1);
                tmem_st8(lb + acc_col(h, 2, n0, n1) + (uint32_t)(c * 8), kBias2);
                tmem_st8(lb + acc_col(h, 3, n0, n1) + (uint32_t)(c * 8), 0u);
            }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const int64_t ntiles = (nsb + kM - 1) / kM;
    int64_t T = 0;  // tiles done by this CTA (barrier phases)

    for (int64_t row = blockIdx.x; row < A.ns; row += gridDim.x) {
        // ---- row set-up: alpha list, common exponent, B slices ----
        for (int e = tid; e < sa_n; e += kThreads) sEa[e] = A.tab[(int64_t)e * A.ns + row];
        __syncthreads();
        if (warp == 0) {
            int mx = 0;
            for (int e = lane; e < sa_n; e += 32) mx = max(mx, __ldg(rowexp + ent_target(sEa[e])));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
            if (lane == 0) *s_emax = mx;
        }
        __syncthreads();
        const int emax = *s_emax;
        // B[q][a] = s_a (q | p_a) 2^(e_row(J_a) - eD): digits of the context's
        // fixed-point integrals shifted by the row's exponent gap, K-major per slice
        for (int item = tid; item < npad * kgroups; item += kThreads) {
            const int q = item / kgroups, kg = item % kgroups;
            uint32_t w[kSlices][4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                float f[2][kSlices];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int a = kg * 8 + 2 * i + u;
                    long long X = 0;
                    if (q < npair && a < sa_n) {
                        const uint32_t ea = sEa[a];
                        X = round_shift(__ldg(XW + (int64_t)q * npair + ent_pair(ea)),
                                        emax - __ldg(rowexp + ent_target(ea)));
                        if (ent_negative(ea)) X = -X;
                    }
                    digits6(X, f[u]);
                }
#pragma unroll
                for (int sl = 0; sl < kSlices; ++sl) w[sl][i] = pack_bf16(f[0][sl], f[1][sl]);
            }
            // half h keeps its six slices stacked along N: rows bh + sl nh + (q - q0h)
            const int h = q < n0 ? 0 : 1;
            const int nhh = h ? n1 : n0, rbase = h ? kSlices * n0 : 0, ql = q - (h ? n0 : 0);
#pragma unroll
            for (int sl = 0; sl < kSlices; ++sl)
                *reinterpret_cast<uint4 *>(sB + tc::kmajor_offset(rbase + sl * nhh + ql, kg, KPAD)) =
                    make_uint4(w[sl][0], w[sl][1], w[sl][2], w[sl][3]);
        }
        tc::fence_async_smem();
        tc::fence_before();
        __syncthreads();
        tc::fence_after();

        if (warp < 4) {
            // ---- producers: beta string 128 t + m, one K-group (8 values) at a time,
            // the next group's loads in flight while this one is transposed ----
            const int m = tid;
            uint32_t cx[8], cy[8], cz[8], nx[8], ny[8], nz[8];
            auto load = [&](uint32_t(&x)[8], uint32_t(&y)[8], uint32_t(&z)[8], int64_t jb, int kg) {
                const int64_t jc = jb < nsb ? jb : nsb - 1;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int a = kg * 8 + i;
                    const int64_t idx = (int64_t)ent_target(sEa[a < sa_n ? a : 0]) * nsb + jc;
                    ld_early_v2(cs0123 + idx, x[i], y[i]);
                    z[i] = tc::ld_early_u32(cs45 + idx);
                }
            };
            load(cx, cy, cz, m, 0);
            for (int64_t t = 0; t < ntiles && !*s_fail; ++t) {
                const int64_t Tt = T + t;
                const int64_t jb = t * kM + m;
                const bool live = jb < nsb;
#pragma unroll
                for (int ks = 0; ks < NKS; ++ks) {
                    if (Tt >= 1 && !tc::mbar_wait_bounded(a_free(ks), (uint32_t)((Tt - 1) & 1))) {
                        *s_fail = 1;
                        break;
                    }
#pragma unroll
                    for (int g = 0; g < 2; ++g) {
                        const int kg = 2 * ks + g;
                        if (kg + 1 < kgroups)
                            load(nx, ny, nz, jb, kg + 1);
                        else if (t + 1 < ntiles)
                            load(nx, ny, nz, jb + kM, 0);
                        if (!live || kg * 8 + 8 > sa_n) {  // dead lane or padded replacements
#pragma unroll
                            for (int i = 0; i < 8; ++i)
                                if (!(live && kg * 8 + i < sa_n)) cx[i] = cy[i] = cz[i] = 0u;
                        }
                        const uint32_t off = tc::kmajor_offset(m, kg, KPAD);
#pragma unroll
                        for (int sl = 0; sl < kSlices; ++sl) {
                            uint32_t o[4];
#pragma unroll
                            for (int i = 0; i < 4; ++i) {
                                const uint32_t x0 = sl < 2 ? cx[2 * i] : sl < 4 ? cy[2 * i] : cz[2 * i];
                                const uint32_t x1 = sl < 2 ? cx[2 * i + 1] : sl < 4 ? cy[2 * i + 1] : cz[2 * i + 1];
                                o[i] = __byte_perm(x0, x1, (sl & 1) ? 0x7632 : 0x5410);
                            }
                            *reinterpret_cast<uint4 *>(sA + (uint32_t)sl * L.bytesA + off) = make_uint4(o[0], o[1], o[2], o[3]);
                        }
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            cx[i] = nx[i];
                            cy[i] = ny[i];
                            cz[i] = nz[i];
                        }
                    }
                    tc::fence_async_smem();
                    tc::mbar_arrive(a_full(ks));
                }
            }
        } else if (warp < 12) {
            // ---- epilogue: lane m of the tile, 8-column chunks g, g+2, ... of each half ----
            const int quarter = warp & 3, grp = (warp - 4) >> 2;
            const int m = quarter * 32 + lane;
            const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
            for (int64_t t = 0; t < ntiles; ++t) {
                const int64_t Tt = T + t;
                const int64_t jb = t * kM + m;
                const bool live = jb < nsb;
                // this string's pair entries, 8 per 16-byte load (dead lanes: none)
                const uint4 *trow = reinterpret_cast<const uint4 *>(B.tabp + (live ? jb : 0) * npad);
                for (int h = 0; h < nh; ++h) {
                    const int c0 = (h ? n0 : 0) / 8, nchunks = (h ? n1 : n0) / 8;
                    auto fetch = [&](int c) {
                        return live ? ld_early_v4(trow + c0 + c) : make_uint4(~0u, ~0u, ~0u, ~0u);
                    };
                    uint4 ent = make_uint4(~0u, ~0u, ~0u, ~0u);
                    if (grp < nchunks) ent = fetch(grp);
                    if (!tc::mbar_wait_bounded(acc_full(h), (uint32_t)(Tt & 1))) {
                        *s_fail = 1;
                        break;
                    }
                    tc::fence_after();
                    if (grp >= nchunks) {
                        tc::fence_before();
                        tc::mbar_arrive(acc_empty(h));
                    }
                    for (int c = grp; c < nchunks; c += 2) {
                        uint32_t r[4][8];
#pragma unroll
                        for (int lv = 0; lv < 4; ++lv)
                            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                                         : "=r"(r[lv][0]), "=r"(r[lv][1]), "=r"(r[lv][2]), "=r"(r[lv][3]),
                                           "=r"(r[lv][4]), "=r"(r[lv][5]), "=r"(r[lv][6]), "=r"(r[lv][7])
                                         : "r"(lane_base + acc_col(h, lv, n0, n1) + (uint32_t)(c * 8)));
                        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                        // the next tile accumulates levels 0-2 onto their biases and level 3 onto zero
                        tmem_st8(lane_base + acc_col(h, 0, n0, n1) + (uint32_t)(c * 8), kBias0);
                        tmem_st8(lane_base + acc_col(h, 1, n0, n1) + (uint32_t)(c * 8), kBias1);
                        tmem_st8(lane_base + acc_col(h, 2, n0, n1) + (uint32_t)(c * 8), kBias2);
                        tmem_st8(lane_base + acc_col(h, 3, n0, n1) + (uint32_t)(c * 8), 0u);
                        if (c + 2 >= nchunks) {  // last chunk of this thread in the half: release it
                            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                            tc::fence_before();
                            tc::mbar_arrive(acc_empty(h));
                        }
                        const uint4 en = ent;
                        if (c + 2 < nchunks) ent = fetch(c + 2);
                        const uint32_t ew[4] = {en.x, en.y, en.z, en.w};
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const uint32_t v16 = (j & 1) ? (ew[j >> 1] >> 16) : (ew[j >> 1] & 0xFFFFu);
                            if (v16 == 0xFFFFu) continue;
                            const long long v = levels_to_int(r[0][j], r[1][j], r[2][j], r[3][j], v16 >> 15);
                            atomicAdd(sAcc + (v16 & 0x7FFFu), (unsigned long long)v);
                        }
                    }
                }
                if (*s_fail) break;
            }
        } else if (warp == 12 && lane == 0) {
            // ---- MMA issuer: descriptors of K-step 0, advanced by 256 bytes (16 in
            // the address field) per K-step.  A half's six B slices are stacked
            // along N and its four levels sit side by side in tensor memory, so
            // A slice s times B slices 0..3-s is one MMA of N = (4 - s) n_h writing
            // levels s..3, and the products of weight 4 and 5 are MMAs of N = n_h
            // into level 3: 15 MMAs per K-step instead of 21 (each M = 128 MMA
            // reads its 4 KB A slice from shared memory; fewer, wider MMAs read it
            // fewer times).  Level 3 starts from zero (written by the epilogue). ----
            uint64_t ad[kSlices], bd0[kSlices], bd1[kSlices];
#pragma unroll
            for (int sl = 0; sl < kSlices; ++sl) {
                ad[sl] = tc::smem_desc(tc::smem_u32(sA + sl * L.bytesA), 128, sbo);
                bd0[sl] = tc::smem_desc(tc::smem_u32(sB) + (uint32_t)(sl * n0 / 8) * sbo, 128, sbo);
                bd1[sl] = tc::smem_desc(tc::smem_u32(sB) + (uint32_t)((kSlices * n0 + sl * n1) / 8) * sbo, 128, sbo);
            }
            uint32_t id0[4], id1[4];  // N = (k + 1) n_h
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                id0[k] = tc::instr_desc(kM, (k + 1) * n0);
                id1[k] = tc::instr_desc(kM, n1 > 0 ? (k + 1) * n1 : 16);
            }
            uint32_t col0[4], col1[4];
#pragma unroll
            for (int lv = 0; lv < 4; ++lv) {
                col0[lv] = tmem + acc_col(0, lv, n0, n1);
                col1[lv] = tmem + acc_col(1, lv, n0, n1);
            }
            auto issue_half = [&](const uint64_t(&bd)[kSlices], const uint32_t(&col)[4], const uint32_t(&idn)[4],
                                  bool wait_a, bool last, int64_t Tt) -> bool {
#pragma unroll
                for (int ks = 0; ks < NKS; ++ks) {
                    if (wait_a && !tc::mbar_wait_bounded(a_full(ks), (uint32_t)(Tt & 1))) return false;
                    tc::fence_after();
#pragma unroll
                    for (int sa = 0; sa < kSlices; ++sa) {
                        const uint64_t a = ad[sa] + (uint64_t)(ks * 16);
                        const int st = sa < 4 ? 4 - sa : 0;  // stacked B slices 0..st-1 -> levels sa..3
                        if (st > 0) tc::mma_bf16(col[sa], a, bd[0] + (uint64_t)(ks * 16), idn[st - 1], 1u);
#pragma unroll
                        for (int t = st; sa + t < kSlices; ++t)  // weights 4, 5 -> level 3
                            tc::mma_bf16(col[3], a, bd[t] + (uint64_t)(ks * 16), idn[0], 1u);
                    }
                    if (last) tc::mma_commit(a_free(ks));
                }
                return true;
            };
            for (int64_t t = 0; t < ntiles; ++t) {
                const int64_t Tt = T + t;
                bool ok = !(Tt >= 1 && !tc::mbar_wait_bounded(acc_empty(0), (uint32_t)((Tt - 1) & 1)));
                ok = ok && issue_half(bd0, col0, id0, true, nh == 1, Tt);
                if (ok) tc::mma_commit(acc_full(0));
                if (ok && nh == 2) {
                    ok = !(Tt >= 1 && !tc::mbar_wait_bounded(acc_empty(1), (uint32_t)((Tt - 1) & 1)));
                    ok = ok && issue_half(bd1, col1, id1, false, true, Tt);
                    if (ok) tc::mma_commit(acc_full(1));
                }
                if (!ok) {
                    *s_fail = 1;
                    break;
                }
            }
        }
        // ---- row end: every entry of the row has been added ----
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        T += ntiles;
        if (*s_fail) break;
        const int e2 = emax - 1022 + eW - 48;
        double *out = sig + row * nsb;
        for (int64_t j = tid; j < nsb; j += kThreads) {
            const double v = emax == 0x7FF ? __longlong_as_double(0x7FF8000000000000ll) : scaled_i64((long long)sAcc[j], e2);
            out[j] = add ? out[j] + v : v;
            sAcc[j] = 0ull;
        }
        __syncthreads();
    }
    // ---- exit: wait for every MMA this CTA issued, then free tensor memory ----
    if (warp == 12 && lane == 0) {
        tc::mma_commit(drain);
        if (!tc::mbar_wait_bounded(drain, 0u)) *s_fail = 1;
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (*s_fail && tid == 0) atomicExch(err, 1);
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
}

}  // namespace sl
}  // namespace fci
