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
// CTA: 8 warps, one CTA per SM, persistent over output alpha rows.  Each beta
// string of a 128-row tile has two threads, each gathering half of its K
// values.  Per tile: the gathered values (already in registers) are split and
// stored K-major (no swizzle) into shared memory; one thread issues the
// NS(NS+1)/2 x K/16 MMAs and commits to an mbarrier; while the tensor cores
// run, every thread already loads the next tile's values; after the (bounded)
// wait the accumulator is staged from tensor memory into shared memory
// (tcgen05.ld, warp w reads lanes 32*(w%4).., the two warp groups split the
// columns), and each thread pair scatters its string's replacement-list
// entries into the sigma row held in shared memory with FP32 atomics (for a
// fixed pair the map J_b -> I_b is one-to-one).  If the staged accumulator
// would not fit, the columns are staged in several passes.
#include <cuda_bf16.h>

#include "internal.cuh"

namespace fci {
namespace tc {

constexpr int kM = 128;
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
    uint32_t bytesB, bytesA, offA, offG, offSig, offEa, offBar, total;
    int gcols;   // accumulator columns staged per epilogue pass
    int passes;  // epilogue passes over the columns
};

// gcols: columns of the accumulator staged in shared memory at once (npad when
// everything fits, else a multiple of 16 below it).
__host__ __device__ inline Layout make_layout(int ns_split, int kpad, int npad, int64_t nsb, int nsingle_a, int gcols) {
    Layout L;
    L.bytesB = (uint32_t)(npad * kpad * 2);
    L.bytesA = (uint32_t)(kM * kpad * 2);
    L.gcols = gcols;
    L.passes = (npad + gcols - 1) / gcols;
    L.offA = ns_split * L.bytesB;
    L.offG = L.offA + ns_split * L.bytesA;
    L.offSig = L.offG + (uint32_t)(kM * (gcols + 1) * 4);
    L.offSig = (L.offSig + 15u) & ~15u;
    L.offEa = L.offSig + (uint32_t)(((nsb + 3) / 4) * 16);
    L.offBar = L.offEa + (uint32_t)(((nsingle_a + 3) / 4) * 16);
    L.total = L.offBar + 16;
    return L;
}

constexpr int kThreads2 = 256;      // two threads per beta string of the tile
constexpr int kColBatch = 48;       // accumulator columns loaded per tcgen05.wait
constexpr int kEntBatch = 24;       // replacement-list entries prefetched per batch

// Gather this thread's half of the K values of tile row `jb` into registers.
template <int KH>
__device__ __forceinline__ void gather_half(float (&pre)[KH], const float *__restrict__ C, const uint32_t *sEa,
                                            int sa_n, int half, int64_t jb, int64_t nsb) {
#pragma unroll
    for (int i = 0; i < KH; ++i) {
        const int a = half * KH + i;
        pre[i] = (a < sa_n && jb < nsb) ? __ldg(C + (int64_t)ent_target(sEa[a]) * nsb + jb) : 0.f;
    }
}

template <int NS, int KPAD>
__global__ void __launch_bounds__(kThreads2, 1)
    k_sigma3_tc(const float *__restrict__ C, float *__restrict__ sig, SpinTables A, SpinTables B,
                const float *__restrict__ Wf, int npair, int npad, int gcols, uint32_t tmem_cols, int *err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    constexpr int KH = KPAD / 2;  // K values gathered per thread (multiple of 8)
    const int64_t nsb = B.ns;
    const Layout L = make_layout(NS, KPAD, npad, nsb, A.nsingle, gcols);
    unsigned char *sB = smem;
    unsigned char *sA = smem + L.offA;
    float *sG = reinterpret_cast<float *>(smem + L.offG);
    float *sSig = reinterpret_cast<float *>(smem + L.offSig);
    uint32_t *sEa = reinterpret_cast<uint32_t *>(smem + L.offEa);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + L.offBar);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + L.offBar + 8);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m = tid & (kM - 1);  // tile row (beta string) of this thread
    const int half = tid >> 7;     // which half of K it gathers / which entries it scatters
    const int gstride = gcols + 1;

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
    constexpr uint32_t sbo = (uint32_t)(KPAD / 8) * 128u;
    constexpr int kgroups = KPAD / 8;
    const int sa_n = A.nsingle, sb_n = B.nsingle;
    uint32_t phase = 0;
    bool failed = false;
    float pre[KH];

    for (int64_t row = blockIdx.x; row < A.ns && !failed; row += gridDim.x) {
        for (int e = tid; e < sa_n; e += kThreads2) sEa[e] = A.tab[(int64_t)e * A.ns + row];
        for (int64_t j = tid; j < nsb; j += kThreads2) sSig[j] = 0.f;
        __syncthreads();
        // B[q][a] = s_a * (q | p_a), zero padded, NS bf16 slices
        for (int item = tid; item < npad * kgroups; item += kThreads2) {
            const int q = item / kgroups, kg = item % kgroups;
            float v[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int a = kg * 8 + i;
                float x = 0.f;
                if (q < npair && a < sa_n) {
                    const uint32_t ea = sEa[a];
                    x = __ldg(Wf + (int64_t)q * npair + ent_pair(ea));
                    if (ent_negative(ea)) x = -x;
                }
                v[i] = x;
            }
            store_split8<NS>(v, sB, L.bytesB, kmajor_offset(q, kg, KPAD));
        }
        gather_half<KH>(pre, C, sEa, sa_n, half, m, nsb);
        for (int64_t t0 = 0; t0 < nsb; t0 += kM) {
            const int64_t jb = t0 + m;
            // A tile from the prefetched registers: D[J_b][a] = C(J_a, J_b)
#pragma unroll
            for (int kg = 0; kg < KH / 8; ++kg) {
                float v[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) v[i] = pre[kg * 8 + i];
                store_split8<NS>(v, sA, L.bytesA, kmajor_offset(m, half * (KH / 8) + kg, KPAD));
            }
            fence_async_smem();
            fence_before();
            __syncthreads();  // A tile written; previous epilogue finished with sG and TMEM
            if (tid == 0) {
                fence_after();
                uint32_t acc = 0;
#pragma unroll
                for (int i = 0; i < NS; ++i)
#pragma unroll
                    for (int j = 0; j + i < NS; ++j)
#pragma unroll
                        for (int ks = 0; ks < KPAD / 16; ++ks) {
                            const uint64_t ad = smem_desc(smem_u32(sA + i * L.bytesA) + ks * 256, 128, sbo);
                            const uint64_t bd = smem_desc(smem_u32(sB + j * L.bytesB) + ks * 256, 128, sbo);
                            mma_bf16(tmem, ad, bd, idesc, acc);
                            acc = 1;
                        }
                mma_commit(smem_u32(mbar));
            }
            __syncwarp();
            // prefetch the next tile's gather while the tensor cores run
            if (t0 + kM < nsb) gather_half<KH>(pre, C, sEa, sa_n, half, t0 + kM + m, nsb);
            const bool ok = mbar_wait_bounded(smem_u32(mbar), phase);
            phase ^= 1u;
            if (__syncthreads_or(!ok)) {
                if (tid == 0) atomicExch(err, 1);
                mbar_wait_bounded(smem_u32(mbar), phase ^ 1u);  // let the MMAs drain before freeing TMEM
                failed = true;
                break;
            }
            fence_after();
            const bool live = jb < nsb;
            for (int p = 0; p < L.passes; ++p) {
                const int c_lo = p * gcols;
                const int c_hi = min(npad, c_lo + gcols);
                // stage accumulator columns [c_lo, c_hi): warp w reads lanes 32*(w%4)..,
                // the two warp groups split the columns
                const int ncol = c_hi - c_lo;          // multiple of 16
                const int my_lo = c_lo + half * (ncol / 2);
                const int my_hi = my_lo + ncol / 2;    // multiple of 8 wide
                const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
                float *grow = sG + (int64_t)((warp & 3) * 32 + lane) * gstride;
                // column loads in batches of 48, one wait per batch (ranges are warp-uniform)
                for (int cb = my_lo; cb < my_hi; cb += kColBatch) {
                    uint32_t u[kColBatch];
#pragma unroll
                    for (int q = 0; q < kColBatch / 8; ++q) {
                        const int c0 = cb + q * 8;
                        if (c0 < my_hi)
                            asm volatile(
                                "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                                : "=r"(u[q * 8 + 0]), "=r"(u[q * 8 + 1]), "=r"(u[q * 8 + 2]), "=r"(u[q * 8 + 3]),
                                  "=r"(u[q * 8 + 4]), "=r"(u[q * 8 + 5]), "=r"(u[q * 8 + 6]), "=r"(u[q * 8 + 7])
                                : "r"(tmem + lane_base + (uint32_t)c0));
                    }
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int q = 0; q < kColBatch; ++q)
                        if (cb + q < my_hi) grow[cb - c_lo + q] = __uint_as_float(u[q]);
                }
                __syncthreads();
                // scatter: sigma(I_a, I_b) += s_b G[J_b][p_b]; the two threads of a row split the
                // entries; entry loads are issued in batches of 24 before any is used
                if (live) {
                    const float *gm = sG + (int64_t)m * gstride;
                    for (int e0 = half; e0 < sb_n; e0 += 2 * kEntBatch) {
                        uint32_t ent[kEntBatch];
#pragma unroll
                        for (int q = 0; q < kEntBatch; ++q) {
                            const int e = e0 + 2 * q;
                            ent[q] = e < sb_n ? __ldg(B.tab + (int64_t)e * nsb + jb) : 0u;
                        }
#pragma unroll
                        for (int q = 0; q < kEntBatch; ++q) {
                            const int pq = (int)ent_pair(ent[q]);
                            if (e0 + 2 * q < sb_n && pq >= c_lo && pq < c_hi) {
                                const float g = gm[pq - c_lo];
                                atomicAdd(&sSig[ent_target(ent[q])], ent_negative(ent[q]) ? -g : g);
                            }
                        }
                    }
                }
                if (p + 1 < L.passes) __syncthreads();
            }
            fence_before();
        }
        __syncthreads();
        if (failed) break;
        for (int64_t j = tid; j < nsb; j += kThreads2) sig[row * nsb + j] += sSig[j];
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

// Largest staged column count (multiple of 16, dividing the columns into
// equal-ish passes) whose layout fits in `lim` bytes; 0 if none does.
static int pick_gcols(int nsplit, int kpad, int npad, int64_t nsb, int nsa_single, int lim) {
    for (int passes = 1; passes <= npad / 16; ++passes) {
        const int g = round_up((npad + passes - 1) / passes, 16);
        if ((int)tc::make_layout(nsplit, kpad, npad, nsb, nsa_single, g).total <= lim) return g;
    }
    return 0;
}

template <int NS>
static void *kernel_for(int kpad) {
    switch (kpad) {
        case 16: return (void *)tc::k_sigma3_tc<NS, 16>;
        case 32: return (void *)tc::k_sigma3_tc<NS, 32>;
        case 48: return (void *)tc::k_sigma3_tc<NS, 48>;
        case 64: return (void *)tc::k_sigma3_tc<NS, 64>;
        case 80: return (void *)tc::k_sigma3_tc<NS, 80>;
        case 96: return (void *)tc::k_sigma3_tc<NS, 96>;
        default: return nullptr;
    }
}

int launch_sigma3_tc(fci_ctx *ctx, const float *C, float *sig, int nsplit, cudaStream_t s) {
    const int kpad = round_up(ctx->A.nsingle, 16), npad = round_up(ctx->npair, 16);
    if (npad > 256) return fail(FCI_ERR_ARG, "tensor-core sigma_3 supports at most 256 orbital pairs (norb <= 22)");
    void *kern = nsplit == 2 ? kernel_for<2>(kpad) : kernel_for<3>(kpad);
    if (!kern) return fail(FCI_ERR_ARG, "tensor-core sigma_3 supports at most 96 alpha replacements per string");
    int dev = ctx->device, lim = 0, nsm = 0;
    FCI_CUDA(cudaDeviceGetAttribute(&lim, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    FCI_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int gcols = pick_gcols(nsplit, kpad, npad, ctx->B.ns, ctx->A.nsingle, lim);
    if (gcols == 0) return fail(FCI_ERR_ARG, "tensor-core sigma_3: beta string count too large for shared memory");
    const tc::Layout L = tc::make_layout(nsplit, kpad, npad, ctx->B.ns, ctx->A.nsingle, gcols);
    uint32_t cols = 32;
    while (cols < (uint32_t)npad) cols <<= 1;
    // one CTA per SM (launch bounds); it holds `cols` of the 512 TMEM columns
    FCI_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total));
    int64_t grid = nsm;
    if (grid > ctx->A.ns) grid = ctx->A.ns;
    void *args[] = {(void *)&C, (void *)&sig, (void *)&ctx->A, (void *)&ctx->B, (void *)&ctx->Wf,
                    (void *)&ctx->npair, (void *)&npad, (void *)&gcols, (void *)&cols, (void *)&ctx->d_err};
    FCI_CUDA(cudaLaunchKernel(kern, dim3((unsigned)grid), dim3(tc::kThreads2), args, L.total, s));
    return FCI_OK;
}

size_t sigma3_tc_smem(const fci_ctx *ctx, int nsplit) {
    if (ctx->A.nsingle == 0 || ctx->B.nsingle == 0) return 0;
    const int kpad = round_up(ctx->A.nsingle, 16), npad = round_up(ctx->npair, 16);
    int lim = 232448;
    const int g = pick_gcols(nsplit, kpad, npad, ctx->B.ns, ctx->A.nsingle, lim);
    return g ? tc::make_layout(nsplit, kpad, npad, ctx->B.ns, ctx->A.nsingle, g).total : 0;
}

}  // namespace fci
