// FP64-accurate sigma terms on the bf16 tensor cores for string spaces whose
// operands do not fit the per-row kernel of sigma3_sliced_kernel.cuh
// (CAS(16,16), CAS(18,18)): the alpha-beta term sigma_3 and the same-spin
// terms sigma_1 / sigma_2 of Eq. 8, from the same 8-bit digit slices.
//
// Differences from the per-row kernel:
//  * one fixed-point scale for the whole call: every C value is written as
//    X = round(|C| 2^(47 - eD)) with the sign (top digit in [-128, 128]), eD
//    from the largest exponent of all of C, and the integral table as 46-bit
//    integers (top digit in [-64, 64]): the two-electron rows in the scale of
//    sigma_3 for (q|p) and twice that for (q|p)/2, so that one table serves
//    both terms with every bit.  All products then have one unit (sigma_3's
//    integers are doubled) and the three terms add into one 64-bit integer
//    accumulator in global memory (red.global.add.u64: exact, order-free);
//  * five accumulators per element: levels 0, 1, 2, 3 on biases (integers in
//    the low mantissa bits: exact while a level sum stays below 2^22 units,
//    which holds for K <= 170, 102, 73 replacements at levels 1, 2, 3, and at
//    level 3 is checked in the epilogue: out of range sets bit 1 of the error
//    word) and levels 4-5 in FP32 from zero.  With level 3 exact, the FP32
//    accumulator holds only terms 2^-32 below the leading ones (the tensor
//    cores' FP32 accumulation need not round to nearest, so what it holds
//    must be small);
//  * the pair columns q of the contraction are cut into parts of at most 48;
//    a work item is (row string, part), so the integral operand of one part
//    (6 slices x 48 x K) and one A tile (6 slices x 128 x K) fit in shared
//    memory together, and the five accumulators of a part fit twice in tensor
//    memory: tiles alternate between the two buffers, so the epilogue of one
//    tile runs under the MMAs of the next.  The parts of one row are
//    consecutive items, so their gathers of the same C rows meet in L2;
//  * the six B slices of a part are stacked along N (rows t np .. t np + np - 1)
//    and the five levels of an accumulator buffer sit side by side in tensor
//    memory (columns L np ..), so that A slice s times B slices 0..4-s is ONE
//    MMA of N = (5 - s) np writing levels s..4, plus one N = np MMA for
//    t = 5 - s into level 4: 11 MMAs per K-step instead of 21.  An M = 128
//    MMA reads its 4 KB A slice from shared memory each time, which at
//    N = 48 takes as long as the multiply itself; stacking amortises it.
//
// MODE 0 (sigma_3), row = output alpha string I_a with replacement list
// a = (J_a, p_a, s_a), lanes = beta strings J_b:
//   G[J_b][q] = sum_a C(J_a, J_b) s_a (q | p_a)
//   acc(I_a, I_b) += s_b G[J_b][q]  for the beta replacement of J_b with pair q
//   (tabp: [J_b][q] -> packed entry of that replacement, or none).
// MODE 1 (same-spin term of the strings of R), row = intermediate string K,
// lanes = columns J of the gathered matrix (sigma_2: C, R = alpha strings;
// sigma_1: C transposed, R = beta strings):
//   G[J][q] = sum_a C(J_a, J) s_a (q | p_a) / 2        (q < npair)
//   G[J][npair] = sum_a C(J_a, J) s_a k(p_a),  k_kl = h_kl - 1/2 sum_j (kj|jl)
//     (this column's table row is in a scale 2^shq coarser: its integers are
//     multiplied by 2^shq before they are added; in MODE 0 every integer is
//     multiplied by 2^shq = 2)
//   acc(E_q K, J) += s_q G[J][q] for each entry (E_q K, q, s_q) of K's list,
//   acc(K, J) += G[J][npair]
// i.e. 1/2 sum (ij|kl) E_ij E_kl + sum k_kl E_kl with the identity resolved
// over intermediate strings; the adds of a warp go to one row, consecutive J.
//
// CTA (416 threads), one per SM, persistent over items: warps 0-3 gather and
// transpose the A slices (as in the per-row kernel), warps 4-11 read the
// accumulators (two warps per lane quarter, alternate 8-column chunks), warp
// 12 issues the MMAs.  All waits are bounded; a wait that gives up sets the
// device error word, and the CTA drains its MMAs and frees tensor memory.
#pragma once
#include "sigma3_sliced_kernel.cuh"

namespace fci {
namespace wd {

using sl::kSlices;
using tc::kM;

constexpr int kThreads = 416;      // warps 0-3 producers, 4-11 epilogue, 12 MMA issuer
constexpr int kEpiThreads = 256;
constexpr int kMaxKSteps = 6;      // K <= 96
constexpr int kPartMax = 48;       // pair columns per part
constexpr int kLevels = 5;         // accumulators per element
constexpr int kBufCols = 256;      // tensor-memory columns of one accumulator buffer (5 x np used)
constexpr uint32_t kBias3 = 0x3F400000u;  // 1.5 2^-1: level 3 (multiples of 2^-24) in the low bits
constexpr int kBars = 2 * kMaxKSteps + 5;  // a_full[6], a_free[6], acc_full[2], acc_empty[2], drain

struct Layout {
    uint32_t bytesA, bytesB, offA, offEa, offPair, offBar, total;
};

// Shared memory: B slices stacked [6 x 48 rows][kpad], A slices [6][128 x kpad], the row's
// replacement list, its entries by pair (MODE 1), barriers and words.
__host__ __device__ inline Layout make_layout(int kpad, int npad, int nsingle) {
    Layout L;
    L.bytesB = (uint32_t)(kPartMax * kpad * 2);
    L.bytesA = (uint32_t)(kM * kpad * 2);
    L.offA = (uint32_t)kSlices * L.bytesB;
    L.offEa = L.offA + (uint32_t)kSlices * L.bytesA;
    L.offPair = L.offEa + (uint32_t)(((nsingle + 3) / 4) * 16);
    L.offBar = L.offPair + (uint32_t)(((npad + 3) / 4) * 16);
    L.total = L.offBar + kBars * 8 + 16;  // barriers, fail word, tmem slot
    return L;
}

// First pair column and width of part p when npad (a multiple of 16) is cut
// into nparts parts of whole 16-column blocks, as even as possible.
__host__ __device__ inline void part_range(int npad, int nparts, int p, int *q0, int *np) {
    const int nblk = npad / 16, base = nblk / nparts, extra = nblk % nparts;
    *q0 = 16 * (p * base + (p < extra ? p : extra));
    *np = 16 * (base + (p < extra ? 1 : 0));
}

// tensor-memory column of level L of accumulator buffer buf for parts np wide
__device__ __forceinline__ uint32_t acc_col(int buf, int L, int np) { return (uint32_t)(buf * kBufCols + L * np); }

// Write the starting words of one 8-column chunk of every level: the biases of
// levels 0-3 and zero for level 4.
__device__ __forceinline__ void init_chunk(uint32_t lane_base, int buf, int np, int c) {
    sl::tmem_st8(lane_base + acc_col(buf, 0, np) + (uint32_t)(c * 8), sl::kBias0);
    sl::tmem_st8(lane_base + acc_col(buf, 1, np) + (uint32_t)(c * 8), sl::kBias1);
    sl::tmem_st8(lane_base + acc_col(buf, 2, np) + (uint32_t)(c * 8), sl::kBias2);
    sl::tmem_st8(lane_base + acc_col(buf, 3, np) + (uint32_t)(c * 8), kBias3);
    sl::tmem_st8(lane_base + acc_col(buf, 4, np) + (uint32_t)(c * 8), 0u);
}

// The integer V = round(2^34 (acc0 + ... + acc4)) of one element, times the
// sign (neg = 1: negative), from the raw words (levels 0-3 biased):
// 2^34 (acc0 + acc1) = (i0 2^8 + i1) 2^26, 2^34 (acc2 + acc3) = (i2 2^8 + i3) 2^10,
// and acc4 split into h = round(2^18 acc4) and an exact remainder rounded at 2^-34.
__device__ __forceinline__ long long levels_to_int5(uint32_t r0, uint32_t r1, uint32_t r2, uint32_t r3, uint32_t r4,
                                                    uint32_t neg) {
    constexpr float M = 12582912.0f;  // 1.5 2^23
    constexpr int MB = 0x4B400000;
    int hi = (int)(r0 * 256u + r1 - (sl::kBias0 * 256u + sl::kBias1));  // exact modulo 2^32
    int mid = (int)(r2 * 256u + r3 - (sl::kBias2 * 256u + kBias3));
    const float a4 = __uint_as_float(r4 ^ (neg << 31));
    const float t = fmaf(a4, 262144.f, M);
    const int h = __float_as_int(t) - MB;
    const float rem = fmaf(-(t - M), 0x1p-18f, a4);  // exact: a4 - h 2^-18
    const int l = __float_as_int(fmaf(rem, 0x1p34f, M)) - MB;
    if (neg) {
        hi = -hi;
        mid = -mid;
    }
    return ((long long)hi << 26) + ((long long)mid << 10) + ((long long)h << 16) + l;
}

template <int KPAD, int MODE>
__global__ void __launch_bounds__(kThreads, 1)
    k_sigma_wide(const uint2 *__restrict__ cs0123, const uint32_t *__restrict__ cs45,
                 unsigned long long *__restrict__ acc, SpinTables R, int64_t ncols, const uint32_t *__restrict__ tabp,
                 const long long *__restrict__ XT, int npair, int npad, int nparts, int shq, int *err) {
    constexpr int NKS = KPAD / 16;
    constexpr int kgroups = KPAD / 8;
    constexpr uint32_t sbo = (uint32_t)(KPAD / 8) * 128u;
    extern __shared__ __align__(1024) unsigned char smem[];
    const int sa_n = R.nsingle;
    const Layout L = make_layout(KPAD, npad, sa_n);
    unsigned char *sB = smem;
    unsigned char *sA = smem + L.offA;
    uint32_t *sEa = reinterpret_cast<uint32_t *>(smem + L.offEa);
    uint32_t *sPair = reinterpret_cast<uint32_t *>(smem + L.offPair);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + L.offBar);
    volatile int *s_fail = reinterpret_cast<volatile int *>(smem + L.offBar + kBars * 8);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + L.offBar + kBars * 8 + 4);
    const uint32_t bar0 = tc::smem_u32(bars);
    auto a_full = [&](int ks) { return bar0 + 8u * (uint32_t)ks; };
    auto a_free = [&](int ks) { return bar0 + 8u * (uint32_t)(kMaxKSteps + ks); };
    auto acc_full = [&](int b) { return bar0 + 8u * (uint32_t)(2 * kMaxKSteps + b); };
    auto acc_empty = [&](int b) { return bar0 + 8u * (uint32_t)(2 * kMaxKSteps + 2 + b); };
    const uint32_t drain = bar0 + 8u * (uint32_t)(2 * kMaxKSteps + 4);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nq = MODE == 1 ? npair + 1 : npair;  // rows of XT

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
    const int64_t ntiles = (ncols + kM - 1) / kM;
    const int64_t nitems = R.ns * (int64_t)nparts;
    int64_t T = 0;  // tiles done by this CTA (barrier phases)

    for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int64_t row = item / nparts;
        int q0 = 0, np = 0;
        part_range(npad, nparts, (int)(item % nparts), &q0, &np);
        // ---- item set-up: replacement list, entries by pair, B slices of the part ----
        for (int e = tid; e < sa_n; e += kThreads) sEa[e] = R.tab[(int64_t)e * R.ns + row];
        if (MODE == 1)
            for (int q = tid; q < npad; q += kThreads) sPair[q] = q == npair ? (uint32_t)row : kNoEntry;
        __syncthreads();
        if (MODE == 1)
            for (int e = tid; e < sa_n; e += kThreads) sPair[ent_pair(sEa[e])] = sEa[e];
        // B[q][a] = s_a XT[q0 + q][p_a] as six digit slices, K-major
        for (int it = tid; it < np * kgroups; it += kThreads) {
            const int ql = it / kgroups, kg = it % kgroups, q = q0 + ql;
            uint32_t w[kSlices][4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                float f[2][kSlices];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int a = kg * 8 + 2 * i + u;
                    long long X = 0;
                    if (q < nq && a < sa_n) {
                        const uint32_t ea = sEa[a];
                        X = __ldg(XT + (int64_t)q * npair + ent_pair(ea));
                        if (ent_negative(ea)) X = -X;
                    }
                    sl::digits6(X, f[u]);
                }
#pragma unroll
                for (int s = 0; s < kSlices; ++s) w[s][i] = sl::pack_bf16(f[0][s], f[1][s]);
            }
#pragma unroll
            for (int s = 0; s < kSlices; ++s)
                *reinterpret_cast<uint4 *>(sB + tc::kmajor_offset(s * np + ql, kg, KPAD)) =
                    make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
        }
        if (warp >= 4 && warp < 12) {  // starting words of both buffers in this item's layout
            const uint32_t lb = tmem + ((uint32_t)((warp & 3) * 32) << 16);
            for (int b = 0; b < 2; ++b)
                for (int c = (warp - 4) >> 2; c < np / 8; c += 2) init_chunk(lb, b, np, c);
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        }
        tc::fence_async_smem();
        tc::fence_before();
        __syncthreads();
        tc::fence_after();

        if (warp < 4) {
            // ---- producers: column string 128 t + m, one K-group (8 values) at a
            // time, the next group's loads in flight while this one is transposed ----
            const int m = tid;
            uint32_t cx[8], cy[8], cz[8], nx[8], ny[8], nz[8];
            auto load = [&](uint32_t(&x)[8], uint32_t(&y)[8], uint32_t(&z)[8], int64_t jb, int kg) {
                const int64_t jc = jb < ncols ? jb : ncols - 1;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int a = kg * 8 + i;
                    const int64_t idx = (int64_t)ent_target(sEa[a < sa_n ? a : 0]) * ncols + jc;
                    sl::ld_early_v2(cs0123 + idx, x[i], y[i]);
                    z[i] = tc::ld_early_u32(cs45 + idx);
                }
            };
            load(cx, cy, cz, m, 0);
            for (int64_t t = 0; t < ntiles && !*s_fail; ++t) {
                const int64_t Tt = T + t;
                const int64_t jb = t * kM + m;
                const bool live = jb < ncols;
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
                        for (int s = 0; s < kSlices; ++s) {
                            uint32_t o[4];
#pragma unroll
                            for (int i = 0; i < 4; ++i) {
                                const uint32_t x0 = s < 2 ? cx[2 * i] : s < 4 ? cy[2 * i] : cz[2 * i];
                                const uint32_t x1 = s < 2 ? cx[2 * i + 1] : s < 4 ? cy[2 * i + 1] : cz[2 * i + 1];
                                o[i] = __byte_perm(x0, x1, (s & 1) ? 0x7632 : 0x5410);
                            }
                            *reinterpret_cast<uint4 *>(sA + (uint32_t)s * L.bytesA + off) = make_uint4(o[0], o[1], o[2], o[3]);
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
            // ---- epilogue: lane m of the tile, 8-column chunks grp, grp + 2, ... ----
            const int quarter = warp & 3, grp = (warp - 4) >> 2;
            const int m = quarter * 32 + lane;
            const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
            const int nch = np / 8;
            uint32_t range_bad = 0;
            for (int64_t t = 0; t < ntiles; ++t) {
                const int64_t Tt = T + t;
                const int b = (int)(Tt & 1);
                const int64_t jb = t * kM + m;
                const bool live = jb < ncols;
                // MODE 0: this string's entries of the part's pairs, 8 per chunk
                const uint4 *trow = MODE == 0 ? reinterpret_cast<const uint4 *>(tabp + (live ? jb : 0) * npad + q0) : nullptr;
                auto fetch = [&](int c, uint4 &e0, uint4 &e1) {
                    if (MODE == 0 && live) {
                        e0 = sl::ld_early_v4(trow + 2 * c);
                        e1 = sl::ld_early_v4(trow + 2 * c + 1);
                    } else {
                        e0 = e1 = make_uint4(kNoEntry, kNoEntry, kNoEntry, kNoEntry);
                    }
                };
                uint4 e0, e1;
                if (grp < nch) fetch(grp, e0, e1);
                if (!tc::mbar_wait_bounded(acc_full(b), (uint32_t)((Tt >> 1) & 1))) {
                    *s_fail = 1;
                    break;
                }
                tc::fence_after();
                if (grp >= nch) {
                    tc::fence_before();
                    tc::mbar_arrive(acc_empty(b));
                }
                for (int c = grp; c < nch; c += 2) {
                    uint32_t r[kLevels][8];
#pragma unroll
                    for (int lv = 0; lv < kLevels; ++lv)
                        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                                     : "=r"(r[lv][0]), "=r"(r[lv][1]), "=r"(r[lv][2]), "=r"(r[lv][3]), "=r"(r[lv][4]),
                                       "=r"(r[lv][5]), "=r"(r[lv][6]), "=r"(r[lv][7])
                                     : "r"(lane_base + acc_col(b, lv, np) + (uint32_t)(c * 8)));
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    init_chunk(lane_base, b, np, c);  // the next use of this buffer starts from these
                    if (c + 2 >= nch) {  // last chunk of this thread: release the buffer
                        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                        tc::fence_before();
                        tc::mbar_arrive(acc_empty(b));
                    }
                    const uint32_t ew[8] = {e0.x, e0.y, e0.z, e0.w, e1.x, e1.y, e1.z, e1.w};
                    if (c + 2 < nch) fetch(c + 2, e0, e1);
                    if (!live) continue;
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const uint32_t en = MODE == 0 ? ew[j] : sPair[q0 + c * 8 + j];
                        if (en == kNoEntry) continue;
                        range_bad |= (r[3][j] >> 23) ^ (kBias3 >> 23);  // level 3 left its binade
                        long long v = levels_to_int5(r[0][j], r[1][j], r[2][j], r[3][j], r[4][j], en >> 31);
                        if (MODE == 0 || q0 + c * 8 + j == npair) v *= 1ll << shq;
                        const int64_t o = MODE == 0 ? row * ncols + (int64_t)ent_target(en)
                                                    : (int64_t)ent_target(en) * ncols + jb;
                        atomicAdd(acc + o, (unsigned long long)v);
                    }
                }
                if (*s_fail) break;
            }
            if (range_bad) atomicOr(err, 2);
        } else if (warp == 12 && lane == 0) {
            // ---- MMA issuer: descriptors of K-step 0, advanced by 256 bytes (16 in
            // the address field) per K-step ----
            // A slice s: levels s..4 from B slices 0..4-s (stacked, one MMA of
            // N = (5 - s) np), then B slice 5 - s into level 4 (N = np)
            uint64_t ad[kSlices], bd[kSlices];
#pragma unroll
            for (int s = 0; s < kSlices; ++s) {
                ad[s] = tc::smem_desc(tc::smem_u32(sA + s * L.bytesA), 128, sbo);
                bd[s] = tc::smem_desc(tc::smem_u32(sB) + (uint32_t)(s * np / 8) * sbo, 128, sbo);
            }
            uint32_t idn[5];
#pragma unroll
            for (int k = 0; k < 5; ++k) idn[k] = tc::instr_desc(kM, (k + 1) * np);
            for (int64_t t = 0; t < ntiles; ++t) {
                const int64_t Tt = T + t;
                const int b = (int)(Tt & 1);
                bool ok = !(Tt >= 2 && !tc::mbar_wait_bounded(acc_empty(b), (uint32_t)(((Tt - 2) >> 1) & 1)));
#pragma unroll
                for (int ks = 0; ks < NKS; ++ks) {
                    if (ok && !tc::mbar_wait_bounded(a_full(ks), (uint32_t)(Tt & 1))) ok = false;
                    if (!ok) break;
                    tc::fence_after();
#pragma unroll
                    for (int sa = 0; sa < kSlices; ++sa) {
                        const uint64_t a = ad[sa] + (uint64_t)(ks * 16);
                        if (sa < 5)
                            tc::mma_bf16(tmem + acc_col(b, sa, np), a, bd[0] + (uint64_t)(ks * 16), idn[4 - sa], 1u);
                        tc::mma_bf16(tmem + acc_col(b, 4, np), a, bd[5 - sa] + (uint64_t)(ks * 16), idn[0], 1u);
                    }
                    tc::mma_commit(a_free(ks));
                }
                if (!ok) {
                    *s_fail = 1;
                    break;
                }
                tc::mma_commit(acc_full(b));
            }
        }
        // ---- item end: every MMA of the item has been read by the epilogue ----
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        T += ntiles;
        if (*s_fail) break;
    }
    // ---- exit: wait for every MMA this CTA issued, then free tensor memory ----
    if (warp == 12 && lane == 0) {
        tc::mma_commit(drain);
        if (!tc::mbar_wait_bounded(drain, 0u)) *s_fail = 1;
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (*s_fail && tid == 0) atomicOr(err, 1);
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
}

}  // namespace wd
}  // namespace fci
