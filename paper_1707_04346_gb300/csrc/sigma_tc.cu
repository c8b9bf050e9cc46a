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
// CTA: 4 warps.  All threads gather the A tile (one beta string each) and
// write it to shared memory in the K-major no-swizzle canonical layout; one
// thread issues the MMAs and commits to an mbarrier; after the (bounded) wait
// each warp reads its 32 accumulator lanes with tcgen05.ld and scatters into
// the sigma row held in shared memory (shared-memory FP32 atomics; for a fixed
// pair the map J_b -> I_b is one-to-one, so lanes of a warp never collide).
#include <cuda_bf16.h>

#include "internal.cuh"

namespace fci {
namespace tc {

constexpr int kM = 128;
constexpr int kThreads = 128;
constexpr long kSpinLimit = 1L << 24;  // mbarrier polls before giving up

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

struct Layout {
    uint32_t bytesB, bytesA, offA, offSig, offEa, offBar, total;
};

__host__ __device__ inline Layout make_layout(int ns_split, int kpad, int npad, int64_t nsb, int nsingle_a) {
    Layout L;
    L.bytesB = (uint32_t)(npad * kpad * 2);
    L.bytesA = (uint32_t)(kM * kpad * 2);
    L.offA = ns_split * L.bytesB;
    L.offSig = L.offA + ns_split * L.bytesA;
    L.offEa = L.offSig + (uint32_t)(((nsb + 3) / 4) * 16);
    L.offBar = L.offEa + (uint32_t)(((nsingle_a + 3) / 4) * 16);
    L.total = L.offBar + 16;
    return L;
}

template <int NS>
__global__ void __launch_bounds__(kThreads) k_sigma3_tc(const float *__restrict__ C, float *__restrict__ sig, SpinTables A,
                                                        SpinTables B, const float *__restrict__ Wf, int npair, int kpad,
                                                        int npad, uint32_t tmem_cols, int *err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int64_t nsb = B.ns;
    const Layout L = make_layout(NS, kpad, npad, nsb, A.nsingle);
    unsigned char *sB = smem;
    unsigned char *sA = smem + L.offA;
    float *sSig = reinterpret_cast<float *>(smem + L.offSig);
    uint32_t *sEa = reinterpret_cast<uint32_t *>(smem + L.offEa);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + L.offBar);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + L.offBar + 8);
    const int tid = threadIdx.x, warp = tid >> 5;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) mbar_init(smem_u32(mbar), 1);
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t idesc = instr_desc(kM, npad);
    const uint32_t sbo = (uint32_t)(kpad / 8) * 128u;
    const int kgroups = kpad / 8;
    const int sa_n = A.nsingle, sb_n = B.nsingle;
    uint32_t phase = 0;
    bool failed = false;

    for (int64_t row = blockIdx.x; row < A.ns && !failed; row += gridDim.x) {
        for (int e = tid; e < sa_n; e += kThreads) sEa[e] = A.tab[(int64_t)e * A.ns + row];
        for (int64_t j = tid; j < nsb; j += kThreads) sSig[j] = 0.f;
        __syncthreads();
        // B[q][a] = s_a * (q | p_a), zero padded
        for (int item = tid; item < npad * kgroups; item += kThreads) {
            const int q = item / kgroups, kg = item % kgroups;
            float v[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int a = kg * 8 + i;
                float x = 0.f;
                if (q < npair && a < sa_n) {
                    const uint32_t ea = sEa[a];
                    x = Wf[(int64_t)q * npair + ent_pair(ea)];
                    if (ent_negative(ea)) x = -x;
                }
                v[i] = x;
            }
            store_split8<NS>(v, sB, L.bytesB, kmajor_offset(q, kg, kpad));
        }
        for (int64_t t0 = 0; t0 < nsb; t0 += kM) {
            // A tile: D[J_b][a] = C(J_a, J_b); one beta string per thread
            const int64_t jb = t0 + tid;
            for (int kg = 0; kg < kgroups; ++kg) {
                float v[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int a = kg * 8 + i;
                    v[i] = (a < sa_n && jb < nsb) ? C[(int64_t)ent_target(sEa[a]) * nsb + jb] : 0.f;
                }
                store_split8<NS>(v, sA, L.bytesA, kmajor_offset(tid, kg, kpad));
            }
            fence_async_smem();
            fence_before();
            __syncthreads();
            if (tid == 0) {
                fence_after();
                uint32_t acc = 0;
#pragma unroll
                for (int i = 0; i < NS; ++i)
#pragma unroll
                    for (int j = 0; j + i < NS; ++j)
                        for (int ks = 0; ks < kpad / 16; ++ks) {
                            const uint64_t ad = smem_desc(smem_u32(sA + i * L.bytesA) + ks * 256, 128, sbo);
                            const uint64_t bd = smem_desc(smem_u32(sB + j * L.bytesB) + ks * 256, 128, sbo);
                            mma_bf16(tmem, ad, bd, idesc, acc);
                            acc = 1;
                        }
                mma_commit(smem_u32(mbar));
            }
            __syncwarp();
            bool ok = mbar_wait_bounded(smem_u32(mbar), phase);
            phase ^= 1u;
            if (__syncthreads_or(!ok)) {
                if (tid == 0) atomicExch(err, 1);
                mbar_wait_bounded(smem_u32(mbar), phase ^ 1u);  // let the MMAs drain before freeing TMEM
                failed = true;
                break;
            }
            fence_after();
            // epilogue: lane (32*warp + l) of the accumulator is beta string t0 + tid
            const bool live = jb < nsb && sb_n > 0;
            const uint32_t *ep = B.tabq + (live ? jb : 0) * sb_n;
            int e = 0;
            uint32_t ent = live ? ep[0] : 0u;
            int np = live ? (int)ent_pair(ent) : (1 << 30);
            for (int c0 = 0; c0 < npad; c0 += 16) {
                float r[16];
                tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    if (c0 + j == np) {
                        atomicAdd(&sSig[ent_target(ent)], ent_negative(ent) ? -r[j] : r[j]);
                        ++e;
                        if (e < sb_n) {
                            ent = ep[e];
                            np = (int)ent_pair(ent);
                        } else {
                            np = 1 << 30;
                        }
                    }
                }
            }
            fence_before();
            __syncthreads();  // accumulator and A tile free for the next tile
        }
        if (failed) break;
        for (int64_t j = tid; j < nsb; j += kThreads) sig[row * nsb + j] += sSig[j];
        __syncthreads();
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
}

}  // namespace tc

static int round_up(int x, int m) { return (x + m - 1) / m * m; }

// Shared memory bytes the kernel needs, or 0 if this space has no alpha-beta term.
size_t sigma3_tc_smem(const fci_ctx *ctx, int nsplit) {
    if (ctx->A.nsingle == 0 || ctx->B.nsingle == 0) return 0;
    const int kpad = round_up(ctx->A.nsingle, 16), npad = round_up(ctx->npair, 16);
    return tc::make_layout(nsplit, kpad, npad, ctx->B.ns, ctx->A.nsingle).total;
}

int launch_sigma3_tc(fci_ctx *ctx, const float *C, float *sig, int nsplit, cudaStream_t s) {
    const int kpad = round_up(ctx->A.nsingle, 16), npad = round_up(ctx->npair, 16);
    if (npad > 256) return fail(FCI_ERR_ARG, "tensor-core sigma_3 supports at most 256 orbital pairs (norb <= 22)");
    const tc::Layout L = tc::make_layout(nsplit, kpad, npad, ctx->B.ns, ctx->A.nsingle);
    int dev = ctx->device, lim = 0, nsm = 0;
    FCI_CUDA(cudaDeviceGetAttribute(&lim, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    FCI_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    if ((int)L.total > lim) return fail(FCI_ERR_ARG, "tensor-core sigma_3: beta string count too large for shared memory");
    uint32_t cols = 32;
    while (cols < (uint32_t)npad) cols <<= 1;
    // resident CTAs per SM must not ask for more than 512 TMEM columns in total:
    // pad the shared-memory request so that at most 512/cols CTAs fit.
    int per_sm_smem = 0;
    FCI_CUDA(cudaDeviceGetAttribute(&per_sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    const int max_ctas = (int)(512 / cols);
    size_t smem = L.total;
    const size_t floor_bytes = (size_t)per_sm_smem / (size_t)(max_ctas + 1) + 1024;
    if (smem < floor_bytes) smem = floor_bytes;
    if ((int)smem > lim) smem = lim;
    auto kern = nsplit == 2 ? tc::k_sigma3_tc<2> : tc::k_sigma3_tc<3>;
    FCI_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int occ = 0;
    FCI_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, tc::kThreads, smem));
    if (occ < 1) return fail(FCI_ERR_ARG, "tensor-core sigma_3 does not fit on an SM");
    if (occ > max_ctas) occ = max_ctas;
    int64_t grid = (int64_t)nsm * occ;
    if (grid > ctx->A.ns) grid = ctx->A.ns;
    kern<<<(unsigned)grid, tc::kThreads, smem, s>>>(C, sig, ctx->A, ctx->B, ctx->Wf, ctx->npair, kpad, npad, cols,
                                                    ctx->d_err);
    FCI_CUDA(cudaGetLastError());
    return FCI_OK;
}

}  // namespace fci
