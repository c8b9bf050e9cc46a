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
// CTA (288 threads): one per SM, persistent over output alpha rows, with three
// roles that run concurrently on consecutive 128-string tiles:
//  * warps 0-3 (producers): each thread gathers the K values of one beta
//    string (the next tile's loads are in flight while the current one is
//    split into bf16 slices) and stores the slices either K-major, no swizzle,
//    into one of the A buffers in shared memory, or (ATM) into the A stage's
//    tensor-memory columns with tcgen05.st; then arrives on full[stage];
//  * lane 0 of warp 8 waits for full[stage] and for a free accumulator,
//    issues the NS(NS+1)/2 x K/16 MMAs into one of two TMEM accumulators and
//    commits to done[acc];
//  * warps 4-7 (epilogue) wait for done[acc], copy the accumulator tile
//    (tcgen05.ld) to shared memory, release it, and then every thread gathers
//    the entries of the targets it owns in this tile from a precomputed
//    schedule (SpinTables::tsched) and adds s_b G[J_b][p_b] into the sigma
//    row: no atomics, and the adds of a batch of entries hit distinct slots.
//    The row is held in shared memory (EPI 2) or, when it does not fit, in
//    global memory, where it stays in L2 (EPI 3).  EPI 4 is the same-spin
//    mode described at the kernel.
// All waits are bounded; a wait that gives up sets the device error word and
// the CTA drains and frees its tensor memory.  The pipeline drains at the end
// of each alpha row, where the sigma row is added to the output and the B
// operand of the next row is built.
#pragma once
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

// A operand in tensor memory (rows = lanes, K packed two bf16 per column)
__device__ __forceinline__ void mma_bf16_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc,
                                            uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tmem_st4(uint32_t taddr, const uint32_t (&w)[4]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr), "r"(w[0]), "r"(w[1]),
                 "r"(w[2]), "r"(w[3])
                 : "memory");
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

// 8 floats -> NS bf16 slices in registers (four bf16 pairs per slice), the
// remainder carried to the next slice as in store_split8p.
template <int NS>
__device__ __forceinline__ void split8p(const float *v, uint32_t (&w)[NS][4]) {
    float rem[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) rem[i] = v[i];
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const __nv_bfloat162 h = __floats2bfloat162_rn(rem[2 * i], rem[2 * i + 1]);
            w[s][i] = *reinterpret_cast<const uint32_t *>(&h);
            if (s + 1 < NS) {
                rem[2 * i] -= __uint_as_float(w[s][i] << 16);
                rem[2 * i + 1] -= __uint_as_float(w[s][i] & 0xFFFF0000u);
            }
        }
}

struct Layout {
    uint32_t bytesB, bytesA, offA, offG, offSig, offEa, offBar, total;
    int stages;  // A tile buffers (1 or 2)
};

// Shared memory of one CTA: B operand (NS slices), A buffers (none when A is
// in tensor memory), the staged accumulator tile (gather epilogues), the sigma
// row (epi 2, with kM dummy slots) or the pair table of the intermediate
// string (epi 4), the alpha replacement list and the barriers.
__host__ __device__ inline Layout make_layout(int ns_split, int kpad, int npad, int64_t nsb, int nsingle_a, int epi,
                                              int stages, bool atm) {
    Layout L;
    L.bytesB = (uint32_t)(npad * kpad * 2);
    L.bytesA = (uint32_t)(kM * kpad * 2);
    L.stages = stages;
    L.offA = ns_split * L.bytesB;
    L.offG = L.offA + (atm ? 0u : (uint32_t)(stages * ns_split) * L.bytesA);
    L.offSig = L.offG + (epi == 2 || epi == 3 ? (uint32_t)(kM * (npad + 1) * 4) : 0u);
    L.offSig = (L.offSig + 15u) & ~15u;
    L.offEa = L.offSig + (epi == 2   ? (uint32_t)(((nsb + kM + 3) / 4) * 16)
                          : epi == 4 ? (uint32_t)(((npad + 3) / 4) * 16)
                                     : 0u);
    L.offBar = L.offEa + (uint32_t)(((nsingle_a + 3) / 4) * 16);
    L.total = L.offBar + 8 * 8 + 16;  // full[2], done[2], empty[2], fail word, tmem slot
    return L;
}

// roles: warps 0-3 producers, 4-7 epilogue (TMEM lane quarter = warp % 4), 8 issues the MMAs
constexpr int kThreads2 = 288;  // warps 0-3 producers, 4-7 epilogue, 8 issues the MMAs
constexpr int kGatherPre = 64;  // gather epilogue: schedule entries held in registers per thread

__device__ __forceinline__ void mbar_arrive(uint32_t addr) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(addr) : "memory");
}

// EPI: 2 gather into the sigma row in shared memory, 3 gather into the sigma
// row in global memory, 4 same-spin (see below).
//
// EPI 4 computes the same-spin term of the strings of A instead (sigma_2 on C,
// sigma_1 on C transposed) through intermediate strings K = the rows:
//   1/2 sum (ij|kl) E_ij E_kl C:  G[J_b][q] = sum_a C(J_a, J_b) s_a (q|p_a) / 2,
//        sigma(E_q K, J_b) += s_q G[J_b][q]       for each entry (E_q K, q, s_q) of K's list
//   sum k_kl E_kl C: one more column q = npair with B[npair][a] = s_a k(p_a),
//        sigma(K, J_b) += G[J_b][npair]
// The rows of sigma it adds to belong to other intermediate strings too, so the
// adds are atomic (red.global, coalesced along J_b).
template <int NS, int KPAD, int EPI, bool ATM>
__global__ void __launch_bounds__(kThreads2, 1)
    k_sigma3_tc(const float *__restrict__ C, float *__restrict__ sig, SpinTables A, SpinTables B,
                const float *__restrict__ Wf, int npair, int npad, int stages, uint32_t tmem_cols,
                int *err, const int *__restrict__ active, const float *__restrict__ kf) {
    if (active != nullptr && *active == 0) return;  // gated launch: the instance is not active
    extern __shared__ __align__(1024) unsigned char smem[];
    const int64_t nsb = B.ns;
    const Layout L = make_layout(NS, KPAD, npad, nsb, A.nsingle, EPI, stages, ATM);
    // ATM: A stage st, slice i at tensor-memory columns aoff + (st*NS + i)*KPAD/2
    const uint32_t aoff = (uint32_t)(2 * npad);
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
    constexpr int kThr = kThreads2;
    const int sa_n = A.nsingle;
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
            mbar_init(empty0 + 8 * i, 128);
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
        else if (EPI == 2)
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
                if (ATM) {
                    const uint32_t abase = tmem + ((uint32_t)(warp * 32) << 16) + aoff + (uint32_t)(st * NS) * (KPAD / 2);
#pragma unroll
                    for (int kg = 0; kg < kgroups; ++kg) {
                        uint32_t w[NS][4];
                        split8p<NS>(pre + kg * 8, w);
#pragma unroll
                        for (int sl = 0; sl < NS; ++sl) tmem_st4(abase + (uint32_t)sl * (KPAD / 2) + (uint32_t)kg * 4, w[sl]);
                    }
                    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                    fence_before();
                } else {
                    unsigned char *a_st = sA + (uint32_t)st * NS * L.bytesA;
#pragma unroll
                    for (int kg = 0; kg < kgroups; ++kg)
                        store_split8p<NS>(pre + kg * 8, a_st, L.bytesA, kmajor_offset(m, kg, KPAD));
                    fence_async_smem();
                }
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
        } else if (warp == 8 && lane == 0) {
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
                            const uint64_t bd = smem_desc(smem_u32(sB + j * L.bytesB) + ks * 256, 128, sbo);
                            if (ATM) {
                                const uint32_t at = tmem + aoff + (uint32_t)((st * NS + i) * (KPAD / 2) + ks * 8);
                                mma_bf16_ts(acc_col, at, bd, idesc, accf);
                            } else {
                                const uint64_t ad = smem_desc(smem_u32(a_st + i * L.bytesA) + ks * 256, 128, sbo);
                                mma_bf16(acc_col, ad, bd, idesc, accf);
                            }
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
        if (EPI == 2)
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
}  // namespace fci
