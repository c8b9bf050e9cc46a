// sigma_3 (the alpha-beta term of Eq. 8) on the 5th-generation tensor cores
// (tcgen05, sm_103a) for FP32 CI vectors.
//
// For one output alpha string I_a with replacement list a = (J_a, p_a, s_a):
//   G[J_b][q] = sum_a D[J_b][a] * B[q][a],  D[J_b][a] = C(J_a, J_b),
//                                           B[q][a]  = s_a * (q | p_a)
//   sigma(I_a, I_b) += s_b * G[J_b][p_b]   for every beta replacement
//                                           a+_k a_l |J_b> = s_b |I_b>, p_b = {k,l}
// i.e. the gather D[kl, I_a, J_b] = sum sign * C, the dense contraction with
// the (ij|kl) pair matrix, and the scatter-add into sigma of the string-driven
// alpha-beta term.  M = 128 beta strings per tile, N = pairs (padded to 16),
// K = alpha replacements (padded to 16).
//
// Precision: FP32 operands are split into NS bf16 slices (x = x_0 + x_1 + ...),
// and the NS(NS+1)/2 slice products with i + j < NS accumulate in FP32 in
// tensor memory: NS = 2 is split-BF16x3, NS = 3 is split-BF16x6 (about FP32
// accuracy).
//
// CTA: one per SM, persistent over output alpha rows, with three roles that
// run concurrently on consecutive 128-string tiles:
//  * warps 0-3 (producers): each thread gathers the K values of one beta
//    string (the next tile's loads are in flight while the current one is
//    split into bf16 slices and stored K-major, no swizzle, into one of the A
//    buffers) and arrives on full[stage];
//  * one thread of the last warp waits for full[stage] and for a free
//    accumulator, issues the NS(NS+1)/2 x K/16 MMAs into one of two TMEM
//    accumulators and commits to done[acc];
//  * the epilogue warps wait for done[acc], read the accumulator (tcgen05.ld)
//    and add s_b G[J_b][p_b] into the sigma row held in shared memory.  The
//    default epilogue (4 warps) copies the whole accumulator tile to shared
//    memory, releases it, and then every thread gathers the entries of the
//    targets it owns in this tile from a precomputed schedule (see
//    SpinTables::tsched): no atomics, and the adds of a batch of entries hit
//    distinct slots.  When the schedule or its shared memory is missing, an
//    atomic epilogue (8 warps, two per TMEM lane quarter) or a staged-column
//    epilogue with atomics takes over.
// All waits are bounded; a wait that gives up sets the device error word and
// the CTA drains and frees its tensor memory.  The pipeline drains at the end
// of each alpha row, where the sigma row is added to the output and the B
// operand of the next row is built.
#include <cuda_bf16.h>

#include "internal.cuh"

namespace fci {
namespace tc {

constexpr int kM = 128;
constexpr long kSpinLimit = 1L << 22;  // mbarrier polls before giving up

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Byte offset of the 16-byte chunk (row r, K-group kg) in a K-major
// no-swizzle tile with kpad columns: 8-row groups are (kpad/8)*128 bytes
// apart (SBO), K-adjacent 8x8 core matrices 128 bytes apart (LBO).
__device__ __forceinline__ uint32_t kmajor_offset(int r, int kg, int kpad) {
    return (uint32_t)((r >> 3) * (kpad >> 3) * 128 + kg * 128 + (r & 7) * 16);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version 1; base offset 0; no swizzle
    return d;
}

// kind::f16 instruction descriptor: D = F32, A = B = BF16, both K-major, dense.
__device__ __forceinline__ uint32_t instr_desc(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint32_t addr, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t addr, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    return ok != 0;
}

// Global loads that stay where they are written: a volatile asm is not moved
// past the (volatile) barrier waits, so a load issued before a wait really is
// in flight during it (a plain load may be sunk to its first use).
__device__ __forceinline__ uint32_t ld_early_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.global.nc.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ float ld_early_f32(const float *p) {
    float v;
    asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}

// Bounded wait; returns false if the limit was reached.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t addr, uint32_t parity) {
    for (long it = 0; it < kSpinLimit; ++it)
        if (mbar_try_wait(addr, parity)) return true;
    return false;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&r)[16]) {
    uint32_t u[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]),
          "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) r[i] = __uint_as_float(u[i]);
}

// Split 8 floats into NS bf16 slices and store each slice's 16 bytes.
template <int NS>
__device__ __forceinline__ void store_split8(const float (&v)[8], unsigned char *base, uint32_t slice_bytes,
                                             uint32_t off) {
    float rem[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) rem[i] = v[i];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        uint32_t w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            __nv_bfloat16 lo = __float2bfloat16_rn(rem[2 * i]);
            __nv_bfloat16 hi = __float2bfloat16_rn(rem[2 * i + 1]);
            rem[2 * i] -= __bfloat162float(lo);
            rem[2 * i + 1] -= __bfloat162float(hi);
            w[i] = (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
        }
        *reinterpret_cast<uint4 *>(base + s * slice_bytes + off) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// Packed-conversion split: 8 floats -> NS bf16 slices (round to nearest), the
// remainder carried to the next slice.
template <int NS>
__device__ __forceinline__ void store_split8p(const float *v, unsigned char *base, uint32_t slice_bytes,
                                              uint32_t off) {
    float rem[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) rem[i] = v[i];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        uint32_t w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const __nv_bfloat162 h = __floats2bfloat162_rn(rem[2 * i], rem[2 * i + 1]);
            w[i] = *reinterpret_cast<const uint32_t *>(&h);
            if (s + 1 < NS) {
                rem[2 * i] -= __uint_as_float(w[i] << 16);
                rem[2 * i + 1] -= __uint_as_float(w[i] & 0xFFFF0000u);
            }
        }
        *reinterpret_cast<uint4 *>(base + s * slice_bytes + off) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

struct Layout {
    uint32_t bytesB, bytesA, offA, offG, offSig, offEa, offBar, total;
    int gcols;   // accumulator columns staged per epilogue chunk
    int stages;  // A tile buffers (1 or 2)
};

// gcols > 0: staged-column epilogue (gcols accumulator columns per chunk);
// gcols == -1: atomic epilogue (no staged accumulator, one sigma row);
// gcols == -3: gather epilogue (the whole accumulator staged, one sigma row
// with kM dummy slots); gcols == -4: gather epilogue adding into the sigma
// row in global memory (no sigma row in shared memory); gcols == -5: the
// same-spin epilogue (a pair table of npad entries, nothing staged).
__host__ __device__ inline Layout make_layout(int ns_split, int kpad, int npad, int64_t nsb, int nsingle_a, int gcols,
                                              int stages) {
    Layout L;
    L.bytesB = (uint32_t)(npad * kpad * 2);
    L.bytesA = (uint32_t)(kM * kpad * 2);
    L.gcols = gcols;
    L.stages = stages;
    L.offA = ns_split * L.bytesB;
    L.offG = L.offA + stages * ns_split * L.bytesA;
    L.offSig = L.offG + (gcols > 0 ? (uint32_t)(kM * (gcols + 1) * 4)
                         : (gcols == -3 || gcols == -4) ? (uint32_t)(kM * (npad + 1) * 4) : 0u);
    L.offSig = (L.offSig + 15u) & ~15u;
    L.offEa = L.offSig + (gcols == -4   ? 0u
                          : gcols == -5 ? (uint32_t)(((npad + 3) / 4) * 16)
                                        : (uint32_t)(((nsb + (gcols == -3 ? kM : 0) + 3) / 4) * 16));
    L.offBar = L.offEa + (uint32_t)(((nsingle_a + 3) / 4) * 16);
    L.total = L.offBar + 8 * 8 + 16;  // full[2], done[2], empty[2], fail word, tmem slot
    return L;
}

// roles: warps 0-3 producers, 4-7 epilogue (TMEM lane quarter = warp % 4), 8 issues the MMAs
constexpr int kThreads2 = 288;
// atomic epilogue: warps 0-3 producers, 4-11 epilogue (two warps per TMEM lane
// quarter, one per half of the pair columns), 12 issues the MMAs
constexpr int kThreads3 = 416;
constexpr int kColBatch = 48;  // accumulator columns loaded per tcgen05.wait
constexpr int kEntBatch = 24;  // replacement-list entries prefetched per batch
constexpr int kGatherPre = 64;  // gather epilogue: schedule entries held in registers per thread

// Fire-and-forget shared-memory add (no value returned, nothing to wait for).
__device__ __forceinline__ void red_add_shared(float *p, float v) {
    asm volatile("red.shared.add.f32 [%0], %1;" ::"r"(smem_u32(p)), "f"(v) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t addr) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(addr) : "memory");
}

// EPI: 0 staged columns with atomics, 1 atomic (eight epilogue warps), 2 gather,
// 3 gather into the sigma row in global memory, 4 same-spin (see below).
//
// EPI 4 computes the same-spin term of the strings of A instead (sigma_2 on C,
// sigma_1 on C transposed) through intermediate strings K = the rows:
//   1/2 sum (ij|kl) E_ij E_kl C:  G[J_b][q] = sum_a C(J_a, J_b) s_a (q|p_a) / 2,
//        sigma(E_q K, J_b) += s_q G[J_b][q]       for each entry (E_q K, q, s_q) of K's list
//   sum k_kl E_kl C: one more column q = npair with B[npair][a] = s_a k(p_a),
//        sigma(K, J_b) += G[J_b][npair]
// The rows of sigma it adds to belong to other intermediate strings too, so the
// adds are atomic (red.global, coalesced along J_b).
template <int NS, int KPAD, int EPI>
__global__ void __launch_bounds__(EPI == 1 ? kThreads3 : kThreads2, 1)
    k_sigma3_tc(const float *__restrict__ C, float *__restrict__ sig, SpinTables A, SpinTables B,
                const float *__restrict__ Wf, int npair, int npad, int gcols, int stages, uint32_t tmem_cols,
                int *err, const int *__restrict__ active, const float *__restrict__ kf) {
    if (active != nullptr && *active == 0) return;  // gated launch: the instance is not active
    extern __shared__ __align__(1024) unsigned char smem[];
    const int64_t nsb = B.ns;
    const Layout L = make_layout(NS, KPAD, npad, nsb, A.nsingle, gcols, stages);
    unsigned char *sB = smem;
    unsigned char *sA = smem + L.offA;
    float *sG = reinterpret_cast<float *>(smem + L.offG);
    float *sSig = reinterpret_cast<float *>(smem + L.offSig);
    uint32_t *sEa = reinterpret_cast<uint32_t *>(smem + L.offEa);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + L.offBar);
    volatile int *s_fail = reinterpret_cast<volatile int *>(smem + L.offBar + 48);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + L.offBar + 56);
    const uint32_t full0 = smem_u32(bars + 0), done0 = smem_u32(bars + 2), empty0 = smem_u32(bars + 4);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int gstride = gcols + 1;
    constexpr int kThr = EPI == 1 ? kThreads3 : kThreads2;
    constexpr int kEpiWarps = EPI == 1 ? 8 : 4;
    const int sa_n = A.nsingle, sb_n = B.nsingle;
    constexpr uint32_t sbo = (uint32_t)(KPAD / 8) * 128u;
    constexpr int kgroups = KPAD / 8;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(full0 + 8 * i, 128);
            mbar_init(done0 + 8 * i, 1);
            mbar_init(empty0 + 8 * i, 32 * kEpiWarps);
        }
        *s_fail = 0;
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t idesc = instr_desc(kM, npad);
    const int64_t ntiles = (nsb + kM - 1) / kM;
    int64_t T = 0;  // global tile counter (stage and phase bookkeeping)

    for (int64_t row = blockIdx.x; row < A.ns; row += gridDim.x) {
        // ---- row set-up (all threads): alpha list, zero sigma row, B operand ----
        for (int e = tid; e < sa_n; e += kThr) sEa[e] = A.tab[(int64_t)e * A.ns + row];
        uint32_t *sPair = reinterpret_cast<uint32_t *>(sSig);  // EPI 4: [npad] entry of K's list by pair
        if (EPI == 4)
            for (int q = tid; q < npad; q += kThr) sPair[q] = q == npair ? (uint32_t)row : kNoEntry;
        else if (EPI != 3)
            for (int64_t j = tid; j < nsb; j += kThr) sSig[j] = 0.f;
        __syncthreads();
        if (EPI == 4)
            for (int e = tid; e < sa_n; e += kThr) sPair[ent_pair(sEa[e])] = sEa[e];
        for (int item = tid; item < npad * kgroups; item += kThr) {
            const int q = item / kgroups, kg = item % kgroups;
            float v[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int a = kg * 8 + i;
                float x = 0.f;
                if (q < npair && a < sa_n) {
                    const uint32_t ea = sEa[a];
                    x = __ldg(Wf + (int64_t)q * npair + ent_pair(ea));
                    if (EPI == 4) x *= 0.5f;
                    if (ent_negative(ea)) x = -x;
                } else if (EPI == 4 && q == npair && a < sa_n) {
                    const uint32_t ea = sEa[a];
                    x = __ldg(kf + ent_pair(ea));
                    if (ent_negative(ea)) x = -x;
                }
                v[i] = x;
            }
            store_split8p<NS>(v, sB, L.bytesB, kmajor_offset(q, kg, KPAD));
        }
        fence_async_smem();
        fence_before();
        __syncthreads();
        fence_after();

        if (warp < 4) {
            // ---- producers: one beta string of the tile per thread ----
            const int m = tid;
            float pre[KPAD];
            auto gather = [&](int64_t jb) {
                // addresses clamped into range, values of padding slots zeroed after the load
                const int64_t jc = jb < nsb ? jb : nsb - 1;
#pragma unroll
                for (int a = 0; a < KPAD; ++a) {
                    const float x = ld_early_f32(C + (int64_t)ent_target(sEa[a < sa_n ? a : 0]) * nsb + jc);
                    pre[a] = (a < sa_n && jb < nsb) ? x : 0.f;
                }
            };
            gather(m);
            for (int64_t t = 0; t < ntiles; ++t) {
                const int64_t Tt = T + t;
                const int st = (int)(Tt % stages);
                if (Tt >= stages) {  // MMA of tile Tt - stages has released this A buffer
                    const int64_t Tp = Tt - stages;
                    if (!mbar_wait_bounded(done0 + 8 * (uint32_t)(Tp & 1), (uint32_t)((Tp >> 1) & 1))) {
                        *s_fail = 1;
                        break;
                    }
                }
                unsigned char *a_st = sA + (uint32_t)st * NS * L.bytesA;
#pragma unroll
                for (int kg = 0; kg < kgroups; ++kg) store_split8p<NS>(pre + kg * 8, a_st, L.bytesA, kmajor_offset(m, kg, KPAD));
                fence_async_smem();
                mbar_arrive(full0 + 8 * (uint32_t)st);
                if (t + 1 < ntiles) gather((t + 1) * kM + m);
            }
        } else if (EPI == 4 && warp < 8) {
            // ---- epilogue, same-spin: column q of the accumulator goes to the sigma
            // row of K's entry with pair q (uniform over the warp), each lane adding
            // its own J_b ----
            const int e = tid - 128;
            const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
            for (int64_t t = 0; t < ntiles; ++t) {
                const int64_t Tt = T + t;
                const uint32_t acc = tmem + (uint32_t)((Tt & 1) * npad);
                const int64_t jb = t * kM + e;
                const bool live = jb < nsb;
                if (!mbar_wait_bounded(done0 + 8 * (uint32_t)(Tt & 1), (uint32_t)((Tt >> 1) & 1))) {
                    *s_fail = 1;
                    break;
                }
                fence_after();
#pragma unroll 1
                for (int cb = 0; cb < npad; cb += 16) {
                    uint32_t u[16];
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                        : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]),
                          "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]),
                          "=r"(u[15])
                        : "r"(acc + lane_base + (uint32_t)cb));
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    if (cb + 16 >= npad) {  // accumulator fully read: release it
                        fence_before();
                        mbar_arrive(empty0 + 8 * (uint32_t)(Tt & 1));
                    }
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const uint32_t en = sPair[cb + q];
                        if (en != kNoEntry && live) {
                            const float g = __uint_as_float(u[q]);
                            atomicAdd(sig + (int64_t)ent_target(en) * nsb + jb, ent_negative(en) ? -g : g);
                        }
                    }
                }
            }
        } else if ((EPI == 2 || EPI == 3) && warp < 8) {
            // ---- epilogue, target-owned gather: the warps copy the accumulator
            // tile into shared memory (row = source string J_b, column = pair)
            // and release it; then thread k adds its share of the tile's entries
            // (each target's entries all in one share, stored step-major so that
            // a warp's loads are coalesced),
            //   sigma(I_a, I_b) += s_b G[J_b][p_b]
            // summing each target's run in a register and adding it once.  Every
            // target has one owner per tile and tiles are separated by barriers
            // of the four epilogue warps, so the sigma row needs no atomics ----
            const int e = tid - 128;
            const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
            const int gs = npad + 1;
            for (int64_t t = 0; t < ntiles; ++t) {
                const int64_t Tt = T + t;
                const uint32_t acc = tmem + (uint32_t)((Tt & 1) * npad);
                // this thread's share (step-major: coalesced across the warp),
                // loaded before the accumulator is ready; `after` is the entry
                // that follows the registers' window
                const int32_t sbase = B.toff[t];
                const int steps = (B.toff[t + 1] - sbase) / kM;
                const uint32_t *mysched = B.tsched + sbase + e;
                uint32_t en[kGatherPre];
#pragma unroll
                for (int k = 0; k < kGatherPre; ++k) en[k] = ld_early_u32(mysched + (k < steps ? k : steps - 1) * kM);
                uint32_t after = ld_early_u32(mysched + (kGatherPre < steps ? kGatherPre : steps - 1) * kM);
                if (!mbar_wait_bounded(done0 + 8 * (uint32_t)(Tt & 1), (uint32_t)((Tt >> 1) & 1))) {
                    *s_fail = 1;
                } else {
                    fence_after();
#pragma unroll 1
                    for (int cb = 0; cb < npad; cb += 16) {
                        uint32_t u[16];
                        asm volatile(
                            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                            : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]),
                              "=r"(u[7]), "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]),
                              "=r"(u[14]), "=r"(u[15])
                            : "r"(acc + lane_base + (uint32_t)cb));
                        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                        for (int q = 0; q < 16; ++q) sG[e * gs + cb + q] = __uint_as_float(u[q]);
                    }
                    fence_before();
                    mbar_arrive(empty0 + 8 * (uint32_t)(Tt & 1));
                }
                asm volatile("bar.sync 1, 128;" ::: "memory");
                if (*s_fail) break;
                // runs end where the next entry has another target; a thread's runs
                // have distinct targets and targets have one owner, so the adds of
                // a batch of 8 entries touch distinct sigma slots: all loads of the
                // batch are issued before any store
                float run = 0.f;
                for (int c0 = 0; c0 < steps; c0 += kGatherPre) {
                    if (c0 > 0) {
#pragma unroll
                        for (int k = 0; k < kGatherPre; ++k)
                            en[k] = ld_early_u32(mysched + (c0 + k < steps ? c0 + k : steps - 1) * kM);
                        after = ld_early_u32(mysched + (c0 + kGatherPre < steps ? c0 + kGatherPre : steps - 1) * kM);
                    }
                    const int nst = steps - c0 < kGatherPre ? steps - c0 : kGatherPre;
#pragma unroll
                    for (int b = 0; b < kGatherPre; b += 8) {
                        if (b >= nst) break;
                        float g[8], part[8], old[8];
                        uint32_t tg[8];
                        bool last[8];
#pragma unroll
                        for (int u = 0; u < 8; ++u)
                            g[u] = sG[(int)((en[b + u] >> 16) & 127u) * gs + (int)((en[b + u] >> 23) & 255u)];
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            const int k = b + u;
                            const uint32_t v = en[k];
                            const uint32_t nxt = k + 1 < kGatherPre ? en[k + 1 < kGatherPre ? k + 1 : k] : after;
                            const bool valid = k < nst;
                            tg[u] = v & 0xFFFFu;
                            run += valid ? ((v >> 31) ? -g[u] : g[u]) : 0.f;
                            last[u] = valid && (c0 + k + 1 >= steps || (nxt & 0xFFFFu) != tg[u]);
                            part[u] = run;
                            if (last[u]) run = 0.f;
                        }
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            if (EPI == 3) {  // sigma row in global memory (stays in L2); no dummy slots there
                                last[u] = last[u] && tg[u] < (uint32_t)nsb;
                                old[u] = last[u] ? sig[row * nsb + tg[u]] : 0.f;
                            } else {
                                old[u] = last[u] ? sSig[tg[u]] : 0.f;
                            }
                        }
#pragma unroll
                        for (int u = 0; u < 8; ++u)
                            if (last[u]) {
                                if (EPI == 3)
                                    sig[row * nsb + tg[u]] = old[u] + part[u];
                                else
                                    sSig[tg[u]] = old[u] + part[u];
                            }
                    }
                }
                asm volatile("bar.sync 1, 128;" ::: "memory");
            }
        } else if (EPI == 1 && warp < 12) {
            // ---- epilogue, shared-memory atomics: no dependency between the adds,
            // so the warp never waits on its own updates; the replacement-list
            // entries of the next columns are loaded while the current ones are
            // added, and the first batch before the accumulator is ready ----
            const int quarter = warp & 3, half = (warp - 4) >> 2;
            const int e = quarter * 32 + lane;
            const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
            const int csplit = (npad / 16) * 8;  // npad is a multiple of 16
            const int c_begin = half ? csplit : 0, c_end = half ? npad : csplit;
            for (int64_t t = 0; t < ntiles; ++t) {
                const int64_t Tt = T + t;
                const uint32_t acc = tmem + (uint32_t)((Tt & 1) * npad);
                const int64_t jb = t * kM + e;
                const bool live = jb < nsb;
                uint32_t ent[16], nxt[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int c = c_begin + q;
                    ent[q] = (live && c < c_end && c < npair) ? __ldg(B.tabp + (int64_t)c * nsb + jb) : kNoEntry;
                }
                if (!mbar_wait_bounded(done0 + 8 * (uint32_t)(Tt & 1), (uint32_t)((Tt >> 1) & 1))) {
                    *s_fail = 1;
                    break;
                }
                fence_after();
                float self = 0.f;
                for (int cb = c_begin; cb < c_end; cb += 16) {
                    uint32_t u[16];
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                        : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7])
                        : "r"(acc + lane_base + (uint32_t)cb));
                    if (cb + 8 < c_end)
                        asm volatile(
                            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                            : "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]),
                              "=r"(u[15])
                            : "r"(acc + lane_base + (uint32_t)(cb + 8)));
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const int c = cb + 16 + q;
                        nxt[q] = (live && c < c_end && c < npair) ? __ldg(B.tabp + (int64_t)c * nsb + jb) : kNoEntry;
                    }
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        if (ent[q] != kNoEntry) {
                            const float g = __uint_as_float(u[q]);
                            const float v = ent_negative(ent[q]) ? -g : g;
                            const uint32_t tg = ent_target(ent[q]);
                            if ((int64_t)tg == jb) self += v;  // diagonal pairs (kk), k in J_b
                            else red_add_shared(&sSig[tg], v);
                        }
                        ent[q] = nxt[q];
                    }
                }
                fence_before();
                mbar_arrive(empty0 + 8 * (uint32_t)(Tt & 1));
                if (live) red_add_shared(&sSig[jb], self);
            }
        } else if (warp < 8) {
            // ---- epilogue: lane e of the accumulator is beta string t*128 + e ----
            const int e = tid - 128;
            const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
            float *grow = sG + (int64_t)e * gstride;
            for (int64_t t = 0; t < ntiles; ++t) {
                const int64_t Tt = T + t;
                const uint32_t acc = tmem + (uint32_t)((Tt & 1) * npad);
                if (!mbar_wait_bounded(done0 + 8 * (uint32_t)(Tt & 1), (uint32_t)((Tt >> 1) & 1))) {
                    *s_fail = 1;
                    break;
                }
                fence_after();
                const int64_t jb = t * kM + e;
                const bool live = jb < nsb;
                for (int c_lo = 0; c_lo < npad; c_lo += gcols) {
                    const int c_hi = min(npad, c_lo + gcols);
                    for (int cb = c_lo; cb < c_hi; cb += kColBatch) {
                        uint32_t u[kColBatch];
#pragma unroll
                        for (int q = 0; q < kColBatch / 8; ++q) {
                            const int c0 = cb + q * 8;
                            if (c0 < c_hi)
                                asm volatile(
                                    "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                                    : "=r"(u[q * 8 + 0]), "=r"(u[q * 8 + 1]), "=r"(u[q * 8 + 2]), "=r"(u[q * 8 + 3]),
                                      "=r"(u[q * 8 + 4]), "=r"(u[q * 8 + 5]), "=r"(u[q * 8 + 6]), "=r"(u[q * 8 + 7])
                                    : "r"(acc + lane_base + (uint32_t)c0));
                        }
                        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                        for (int q = 0; q < kColBatch; ++q)
                            if (cb + q < c_hi) grow[cb - c_lo + q] = __uint_as_float(u[q]);
                    }
                    if (c_hi >= npad) {  // accumulator fully read: release it to the MMA warp
                        fence_before();
                        mbar_arrive(empty0 + 8 * (uint32_t)(Tt & 1));
                    }
                    // scatter this chunk's pairs: sigma(I_a, I_b) += s_b G[J_b][p_b]
                    if (live) {
                        // entries that map J_b onto itself (the diagonal pairs (kk), k in J_b)
                        // are summed in a register and added once
                        float self = 0.f;
                        for (int e0 = 0; e0 < sb_n; e0 += kEntBatch) {
                            uint32_t ent[kEntBatch];
#pragma unroll
                            for (int q = 0; q < kEntBatch; ++q)
                                ent[q] = e0 + q < sb_n ? __ldg(B.tab + (int64_t)(e0 + q) * nsb + jb) : 0u;
#pragma unroll
                            for (int q = 0; q < kEntBatch; ++q) {
                                const int pq = (int)ent_pair(ent[q]);
                                if (e0 + q < sb_n && pq >= c_lo && pq < c_hi) {
                                    const float g = grow[pq - c_lo];
                                    const float v = ent_negative(ent[q]) ? -g : g;
                                    if ((int64_t)ent_target(ent[q]) == jb) self += v;
                                    else red_add_shared(&sSig[ent_target(ent[q])], v);
                                }
                            }
                        }
                        red_add_shared(&sSig[jb], self);
                    }
                }
            }
        } else if (warp == 4 + kEpiWarps && lane == 0) {
            // ---- MMA issuer ----
            for (int64_t t = 0; t < ntiles; ++t) {
                const int64_t Tt = T + t;
                const int st = (int)(Tt % stages);
                const int64_t us = Tt / stages;
                if (!mbar_wait_bounded(full0 + 8 * (uint32_t)st, (uint32_t)(us & 1))) {
                    *s_fail = 1;
                    break;
                }
                if (Tt >= 2 && !mbar_wait_bounded(empty0 + 8 * (uint32_t)(Tt & 1), (uint32_t)(((Tt - 2) >> 1) & 1))) {
                    *s_fail = 1;
                    break;
                }
                fence_after();
                const uint32_t acc_col = tmem + (uint32_t)((Tt & 1) * npad);
                const unsigned char *a_st = sA + (uint32_t)st * NS * L.bytesA;
                uint32_t accf = 0;
#pragma unroll
                for (int i = 0; i < NS; ++i)
#pragma unroll
                    for (int j = 0; j + i < NS; ++j)
#pragma unroll
                        for (int ks = 0; ks < KPAD / 16; ++ks) {
                            const uint64_t ad = smem_desc(smem_u32(a_st + i * L.bytesA) + ks * 256, 128, sbo);
                            const uint64_t bd = smem_desc(smem_u32(sB + j * L.bytesB) + ks * 256, 128, sbo);
                            mma_bf16(acc_col, ad, bd, idesc, accf);
                            accf = 1;
                        }
                mma_commit(done0 + 8 * (uint32_t)(Tt & 1));
            }
        }
        // ---- row end: everything of this row has been scattered ----
        fence_before();
        __syncthreads();
        fence_after();
        T += ntiles;
        if (*s_fail) break;
        if (EPI != 3 && EPI != 4)
            for (int64_t j = tid; j < nsb; j += kThr) sig[row * nsb + j] += sSig[j];
        __syncthreads();
    }
    if (*s_fail && tid == 0) {
        atomicExch(err, 1);
        // let any MMA still in flight finish before the accumulator is freed
        mbar_wait_bounded(done0 + 8 * (uint32_t)((T - 1) & 1), (uint32_t)(((T - 1) >> 1) & 1));
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
}

}  // namespace tc

static int round_up(int x, int m) { return (x + m - 1) / m * m; }

// Epilogue and A buffers whose layout fits in `lim` bytes: the gather
// epilogue (gcols = -3, then -4 with the sigma row in global memory; both need
// the tile schedule), else the atomic epilogue (gcols = -1), else staged
// columns (a multiple of 16) with atomics; two A buffers preferred.
static bool pick_layout(int nsplit, int kpad, int npad, int64_t nsb, int nsa_single, int lim, bool sched, int *gcols,
                        int *stages) {
    static const int order[][2] = {{-3, 2}, {-3, 1}, {-4, 2}, {-4, 1}, {-1, 2}, {-1, 1}};  // {epilogue mode, A buffers}
    for (const auto &o : order)
        if ((o[0] > -3 || sched) && (int)tc::make_layout(nsplit, kpad, npad, nsb, nsa_single, o[0], o[1]).total <= lim) {
            *gcols = o[0];
            *stages = o[1];
            return true;
        }
    for (int st = 2; st >= 1; --st)
        for (int passes = 1; passes <= npad / 16; ++passes) {
            const int g = round_up((npad + passes - 1) / passes, 16);
            if ((int)tc::make_layout(nsplit, kpad, npad, nsb, nsa_single, g, st).total <= lim) {
                *gcols = g;
                *stages = st;
                return true;
            }
        }
    return false;
}

template <int NS, int EPI>
static void *kernel_for(int kpad) {
    switch (kpad) {
        case 16: return (void *)tc::k_sigma3_tc<NS, 16, EPI>;
        case 32: return (void *)tc::k_sigma3_tc<NS, 32, EPI>;
        case 48: return (void *)tc::k_sigma3_tc<NS, 48, EPI>;
        case 64: return (void *)tc::k_sigma3_tc<NS, 64, EPI>;
        case 80: return (void *)tc::k_sigma3_tc<NS, 80, EPI>;
        case 96: return (void *)tc::k_sigma3_tc<NS, 96, EPI>;
        default: return nullptr;
    }
}

struct TcPlan {
    void *kern = nullptr;
    int npad = 0, gcols = 0, stages = 0, threads = 0, lim = 0;
    uint32_t cols = 0, smem = 0;
};

static int tc_plan(const fci_ctx *ctx, int nsplit, TcPlan *P) {
    const int kpad = round_up(ctx->A.nsingle, 16), npad = round_up(ctx->npair, 16);
    if (npad > 256) return fail(FCI_ERR_ARG, "tensor-core sigma_3 supports at most 256 orbital pairs (norb <= 22)");
    if (kpad > 96) return fail(FCI_ERR_ARG, "tensor-core sigma_3 supports at most 96 alpha replacements per string");
    int lim = 0;
    FCI_CUDA(cudaDeviceGetAttribute(&lim, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
    int gcols = 0, stages = 0;
    if (!pick_layout(nsplit, kpad, npad, ctx->B.ns, ctx->A.nsingle, lim, ctx->B.tsched != nullptr, &gcols, &stages))
        return fail(FCI_ERR_ARG, "tensor-core sigma_3: beta string count too large for shared memory");
    const int epi = gcols == -1 ? 1 : gcols == -3 ? 2 : gcols == -4 ? 3 : 0;
    P->kern = nsplit == 2 ? (epi == 3 ? kernel_for<2, 3>(kpad) : epi == 2 ? kernel_for<2, 2>(kpad)
                             : epi == 1 ? kernel_for<2, 1>(kpad) : kernel_for<2, 0>(kpad))
                          : (epi == 3 ? kernel_for<3, 3>(kpad) : epi == 2 ? kernel_for<3, 2>(kpad)
                             : epi == 1 ? kernel_for<3, 1>(kpad) : kernel_for<3, 0>(kpad));
    P->npad = npad;
    P->lim = lim;
    P->gcols = gcols;
    P->stages = stages;
    P->threads = epi == 1 ? tc::kThreads3 : tc::kThreads2;
    P->smem = tc::make_layout(nsplit, kpad, npad, ctx->B.ns, ctx->A.nsingle, gcols, stages).total;
    uint32_t cols = 32;
    while (cols < (uint32_t)(2 * npad)) cols <<= 1;  // two accumulators
    if (cols > 512) return fail(FCI_ERR_ARG, "tensor-core sigma_3: accumulators exceed tensor memory");
    P->cols = cols;
    return FCI_OK;
}

// Opt the chosen kernel into its shared memory (not done while a stream is
// being captured: the batched engine prepares its instances beforehand).
int prepare_sigma3_tc(const fci_ctx *ctx, int nsplit) {
    TcPlan P;
    if (int rc = tc_plan(ctx, nsplit, &P)) return rc;
    FCI_CUDA(opt_in_max_smem(P.kern, ctx->device));
    return FCI_OK;
}

int launch_sigma3_tc(fci_ctx *ctx, const float *C, float *sig, int nsplit, cudaStream_t s, const int *active) {
    TcPlan P;
    if (int rc = tc_plan(ctx, nsplit, &P)) return rc;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    FCI_CUDA(cudaStreamIsCapturing(s, &cap));
    if (cap == cudaStreamCaptureStatusNone)
        FCI_CUDA(opt_in_max_smem(P.kern, ctx->device));
    int nsm = 0;
    FCI_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device));
    int64_t grid = nsm;  // one CTA per SM (launch bounds and shared memory)
    if (grid > ctx->A.ns) grid = ctx->A.ns;
    const float *no_kf = nullptr;
    void *args[] = {(void *)&C,      (void *)&sig,    (void *)&ctx->A,   (void *)&ctx->B,
                    (void *)&ctx->Wf, (void *)&ctx->npair, (void *)&P.npad, (void *)&P.gcols,
                    (void *)&P.stages, (void *)&P.cols,  (void *)&ctx->d_err, (void *)&active,
                    (void *)&no_kf};
    FCI_CUDA(cudaLaunchKernel(P.kern, dim3((unsigned)grid), dim3(P.threads), args, P.smem, s));
    return FCI_OK;
}

// Same-spin term (two-body through intermediate strings plus the one-body
// part) of the strings R, on the tensor cores: sig[R.ns][cols.ns] += ...;
// sigma_2 with (R, cols) = (alpha, beta) on C, sigma_1 with (beta, alpha) on
// C transposed.  The adds are atomic.
int launch_same_spin_tc(fci_ctx *ctx, const float *C, float *sig, const SpinTables &R, const SpinTables &cols,
                        cudaStream_t s) {
    const int nsplit = ctx->opt.f32_splits;
    const int kpad = round_up(R.nsingle, 16), npad = round_up(ctx->npair + 1, 16);
    if (npad > 256) return fail(FCI_ERR_ARG, "same-spin tensor-core sigma supports at most 255 orbital pairs");
    if (kpad > 96) return fail(FCI_ERR_ARG, "same-spin tensor-core sigma supports at most 96 replacements per string");
    int lim = 0, nsm = 0;
    FCI_CUDA(cudaDeviceGetAttribute(&lim, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
    FCI_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device));
    int gcols = -5, stages = 2;
    uint32_t smem = tc::make_layout(nsplit, kpad, npad, cols.ns, R.nsingle, gcols, stages).total;
    if ((int)smem > lim) {
        stages = 1;
        smem = tc::make_layout(nsplit, kpad, npad, cols.ns, R.nsingle, gcols, stages).total;
    }
    if ((int)smem > lim) return fail(FCI_ERR_ARG, "same-spin tensor-core sigma: operands exceed shared memory");
    void *kern = nsplit == 2 ? kernel_for<2, 4>(kpad) : kernel_for<3, 4>(kpad);
    uint32_t tcols = 32;
    while (tcols < (uint32_t)(2 * npad)) tcols <<= 1;
    if (tcols > 512) return fail(FCI_ERR_ARG, "same-spin tensor-core sigma: accumulators exceed tensor memory");
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    FCI_CUDA(cudaStreamIsCapturing(s, &cap));
    if (cap == cudaStreamCaptureStatusNone) FCI_CUDA(opt_in_max_smem(kern, ctx->device));
    int64_t grid = nsm;
    if (grid > R.ns) grid = R.ns;
    const int *no_gate = nullptr;
    SpinTables Rt = R, Ct = cols;
    void *args[] = {(void *)&C,       (void *)&sig,        (void *)&Rt,      (void *)&Ct,
                    (void *)&ctx->Wf, (void *)&ctx->npair, (void *)&npad,    (void *)&gcols,
                    (void *)&stages,  (void *)&tcols,      (void *)&ctx->d_err, (void *)&no_gate,
                    (void *)&ctx->kf};
    FCI_CUDA(cudaLaunchKernel(kern, dim3((unsigned)grid), dim3(tc::kThreads2), args, smem, s));
    return FCI_OK;
}

size_t sigma3_tc_smem(const fci_ctx *ctx, int nsplit) {
    if (ctx->A.nsingle == 0 || ctx->B.nsingle == 0) return 0;
    const int kpad = round_up(ctx->A.nsingle, 16), npad = round_up(ctx->npair, 16);
    int g = 0, st = 0;
    if (!pick_layout(nsplit, kpad, npad, ctx->B.ns, ctx->A.nsingle, 232448, ctx->B.tsched != nullptr, &g, &st)) return 0;
    return tc::make_layout(nsplit, kpad, npad, ctx->B.ns, ctx->A.nsingle, g, st).total;
}

}  // namespace fci
