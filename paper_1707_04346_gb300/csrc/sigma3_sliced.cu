// Host side of the FP64-accurate tensor-core sigma_3 (sigma3_sliced_kernel.cuh):
// the tables it needs (built once at fci_init), the per-call row exponents of
// C, and the launch.
#include <cmath>
#include <cstring>
#include <vector>

#include "sigma3_sliced_kernel.cuh"

namespace fci {

static int round_up16(int x) { return (x + 15) / 16 * 16; }

// out[r] = largest biased FP64 exponent field over row r of C (nrows x ncols);
// one warp per row.
__global__ void k_row_exponents(const double *__restrict__ C, int64_t nrows, int64_t ncols, int *__restrict__ out,
                                const int *__restrict__ active) {
    if (active != nullptr && *active == 0) return;  // gated launch (batched engine): instance not active
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= nrows) return;
    const unsigned long long *row = reinterpret_cast<const unsigned long long *>(C + r * ncols);
    unsigned mx = 0;
    for (int64_t j = lane; j < ncols; j += 32) mx = max(mx, (unsigned)((__ldg(row + j) >> 52) & 0x7FFull));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
    if (lane == 0) out[r] = (int)mx;
}

// Replacement lists by orbital pair: tabp[x][q] = target | negative << 15 of
// the entry of string x whose orbital pair is q (a string has at most one:
// {k, l} with k == l occupied, or exactly one of k, l occupied), else 0xFFFF
// (left by the memset).
__global__ void k_pair_table(const uint32_t *__restrict__ tab, int64_t ns, int nsingle, int npad,
                             uint16_t *__restrict__ tabp) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ns * nsingle) return;
    const uint32_t v = tab[t];  // entry-major: t = e * ns + x
    const int64_t x = t % ns;
    tabp[x * npad + ent_pair(v)] = (uint16_t)(ent_target(v) | (ent_negative(v) ? 0x8000u : 0u));
}

// Six bf16 digit slices of every C value, relative to its row's exponent:
// slices 0-3 to cs0123, 4-5 to cs45 (d_s 2^(-8s), d_s balanced 8-bit digits of
// round(|C| 2^(47 - e_row)) with the sign).
__global__ void k_slice_c(const double *__restrict__ C, const int *__restrict__ rowexp, int64_t nrows, int64_t ncols,
                          uint2 *__restrict__ cs0123, uint32_t *__restrict__ cs45, const int *__restrict__ active) {
    if (active != nullptr && *active == 0) return;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nrows * ncols) return;
    const unsigned long long b = __double_as_longlong(__ldg(C + t));
    float f[sl::kSlices];
    sl::digits6(sl::fixed47((uint32_t)b, (uint32_t)(b >> 32), __ldg(rowexp + t / ncols)), f);
    cs0123[t] = make_uint2(sl::pack_bf16(f[0], f[1]), sl::pack_bf16(f[2], f[3]));
    cs45[t] = sl::pack_bf16(f[4], f[5]);
}

// Sizes of the sliced kernel for this context; false when it does not apply.
static bool sliced_shape(const fci_ctx *ctx, int *kpad, int *npad, int *n0, uint32_t *smem) {
    const SpinTables &A = ctx->A, &B = ctx->B;
    if (A.nsingle == 0 || B.nsingle == 0 || A.nsingle > sl::kMaxK || B.ns > 0x7FFF) return false;
    *kpad = round_up16(A.nsingle);
    *npad = round_up16(ctx->npair);
    if (*kpad > 16 * sl::kMaxKSteps || *npad > 128 || B.ns > kMaxStrings) return false;
    *n0 = round_up16((*npad + 1) / 2);
    if (*n0 > *npad) *n0 = *npad;
    *smem = sl::make_layout(*kpad, *npad, B.ns, A.nsingle).total;
    int lim = 0;
    if (cudaDeviceGetAttribute(&lim, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device) != cudaSuccess) return false;
    return (int)*smem <= lim;
}

bool sigma3_sliced_ok(const fci_ctx *ctx) { return ctx->XW != nullptr && ctx->B.tabp != nullptr; }

// Build, once per context: the fixed-point integrals XW = round(W 2^(47 - eW))
// (|W| < 2^eW), the pair-major beta table, and the buffers of the per-call
// pre-pass (row exponents, the C digit planes: 4 + 12 N bytes).  Contexts whose
// shapes the kernel does not cover get none of them (the FMA kernel runs).
//
// Kernel choice (fci_options.f64_kernels): FMA builds nothing; WIDE builds the
// wide kernels' tables (sigma_wide.cu) on any space they cover; AUTO and
// SLICED take this per-row kernel where it fits, else the wide kernels where
// both spins have electrons and they fit; else AUTO keeps the FMA kernels and
// SLICED and WIDE fail.
int build_sliced_tables(fci_ctx *ctx, const double *h1_host, const double *eri_host) {
    int kpad = 0, npad = 0, n0 = 0;
    uint32_t smem = 0;
    const int mode = ctx->opt.f64_kernels;
    if (mode == FCI_F64_FMA) return FCI_OK;
    if (mode == FCI_F64_WIDE || !sliced_shape(ctx, &kpad, &npad, &n0, &smem)) {
        const bool both = ctx->A.nsingle > 0 && ctx->B.nsingle > 0;
        if ((mode == FCI_F64_WIDE || both) && sigma_wide_fits(ctx)) return build_wide_tables(ctx, h1_host, eri_host);
        if (mode == FCI_F64_SLICED || mode == FCI_F64_WIDE)
            return fail(FCI_ERR_ARG, "f64_kernels: the space exceeds the tensor-core FP64 kernels' limits "
                                     "(at most 96 replacements per string and 255 orbital pairs)");
        return FCI_OK;
    }
    const int n = ctx->norb, np = ctx->npair;
    const int64_t n2 = (int64_t)n * n;
    std::vector<double> W((size_t)np * np);
    double wmax = 0.0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j <= i; ++j)
            for (int k = 0; k < n; ++k)
                for (int l = 0; l <= k; ++l) {
                    const double v = eri_host[i * n2 * n + j * n2 + (int64_t)k * n + l];
                    W[(size_t)pair_index(i, j) * np + pair_index(k, l)] = v;
                    wmax = std::fmax(wmax, std::fabs(v));
                }
    int eW = 0;
    if (wmax > 0) std::frexp(wmax, &eW);  // wmax < 2^eW
    std::vector<long long> xw(W.size());
    for (size_t e = 0; e < W.size(); ++e) xw[e] = std::llrint(std::ldexp(W[e], 47 - eW));  // |xw| <= 2^47
    int rc = FCI_OK;
    ctx->XW = (long long *)dalloc(ctx, sizeof(long long) * (size_t)np * np, &rc);
    ctx->rowexp = (int *)dalloc(ctx, sizeof(int) * (size_t)ctx->A.ns, &rc);
    ctx->cs0123 = (uint2 *)dalloc(ctx, sizeof(uint2) * (size_t)ctx->ndet, &rc);
    ctx->cs45 = (uint32_t *)dalloc(ctx, sizeof(uint32_t) * (size_t)ctx->ndet, &rc);
    SpinTables &B = ctx->B;
    B.tabp = (uint16_t *)dalloc(ctx, sizeof(uint16_t) * (size_t)npad * B.ns, &rc);
    if (rc) return rc;
    ctx->eW = eW;
    FCI_CUDA(cudaMemcpyAsync(ctx->XW, xw.data(), sizeof(long long) * xw.size(), cudaMemcpyHostToDevice, ctx->stream));
    FCI_CUDA(cudaMemsetAsync(B.tabp, 0xFF, sizeof(uint16_t) * (size_t)npad * B.ns, ctx->stream));
    k_pair_table<<<ceil_div(B.ns * B.nsingle, 256), 256, 0, ctx->stream>>>(B.tab, B.ns, B.nsingle, npad, B.tabp);
    FCI_CUDA(cudaGetLastError());
    FCI_CUDA(cudaStreamSynchronize(ctx->stream));
    return FCI_OK;
}

void free_sliced_tables(fci_ctx *ctx) {
    const int np = ctx->npair;
    if (ctx->B.tabp) dfree(ctx, ctx->B.tabp, sizeof(uint16_t) * (size_t)((np + 15) / 16 * 16) * ctx->B.ns);
    ctx->B.tabp = nullptr;
    dfree(ctx, ctx->XW, sizeof(long long) * (size_t)np * np);
    dfree(ctx, ctx->rowexp, sizeof(int) * (size_t)ctx->A.ns);
    dfree(ctx, ctx->cs0123, sizeof(uint2) * (size_t)ctx->ndet);
    dfree(ctx, ctx->cs45, sizeof(uint32_t) * (size_t)ctx->ndet);
    ctx->XW = nullptr;
    ctx->rowexp = nullptr;
    ctx->cs0123 = nullptr;
    ctx->cs45 = nullptr;
}

static void *sliced_kernel(int kpad);

// Opt the kernel into its shared memory outside any stream capture.
int prepare_sigma3_sliced(const fci_ctx *ctx) {
    int kpad = 0, npad = 0, n0 = 0;
    uint32_t smem = 0;
    if (!sigma3_sliced_ok(ctx) || !sliced_shape(ctx, &kpad, &npad, &n0, &smem))
        return fail(FCI_ERR_STATE, "sliced sigma_3 tables were not built for this context");
    FCI_CUDA(opt_in_max_smem(sliced_kernel(kpad), ctx->device));
    return FCI_OK;
}

static void *sliced_kernel(int kpad) {
    switch (kpad) {
        case 16: return (void *)sl::k_sigma3_sliced<16>;
        case 32: return (void *)sl::k_sigma3_sliced<32>;
        case 48: return (void *)sl::k_sigma3_sliced<48>;
        case 64: return (void *)sl::k_sigma3_sliced<64>;
        case 80: return (void *)sl::k_sigma3_sliced<80>;
        case 96: return (void *)sl::k_sigma3_sliced<96>;
        default: return nullptr;
    }
}

// Row exponents and digit slices of C (stream-ordered), then sigma_3 into sig,
// which is overwritten (add = 0) or added to.  prof_slot: profiling slot of the pre-pass (the kernel
// takes the next one).  active: null, or a device flag; the kernels return at
// once when it is 0 (batched engine: one captured graph for any active set).
int launch_sigma3_sliced(fci_ctx *ctx, const double *C, double *sig, cudaStream_t s, int rec, int prof_slot,
                         const int *active, int add) {
    int kpad = 0, npad = 0, n0 = 0;
    uint32_t smem = 0;
    if (!sigma3_sliced_ok(ctx) || !sliced_shape(ctx, &kpad, &npad, &n0, &smem))
        return fail(FCI_ERR_STATE, "sliced sigma_3 tables were not built for this context");
    const SpinTables &A = ctx->A, &B = ctx->B;
    k_row_exponents<<<ceil_div(A.ns * 32, 256), 256, 0, s>>>(C, A.ns, B.ns, ctx->rowexp, active);
    FCI_CUDA(cudaGetLastError());
    k_slice_c<<<ceil_div(ctx->ndet, 256), 256, 0, s>>>(C, ctx->rowexp, A.ns, B.ns, ctx->cs0123, ctx->cs45, active);
    FCI_CUDA(cudaGetLastError());
    prof_mark(ctx, rec, prof_slot, s);
    void *kern = sliced_kernel(kpad);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    FCI_CUDA(cudaStreamIsCapturing(s, &cap));
    if (cap == cudaStreamCaptureStatusNone) FCI_CUDA(opt_in_max_smem(kern, ctx->device));
    int nsm = 0;  // (a captured launch relies on prepare_sigma3_sliced having opted in)
    FCI_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device));
    int64_t grid = nsm;  // one CTA per SM
    if (grid > A.ns) grid = A.ns;
    SpinTables At = A, Bt = B;
    const uint2 *c0 = ctx->cs0123;
    const uint32_t *c4 = ctx->cs45;
    const long long *xw = ctx->XW;
    const int *rexp = ctx->rowexp;
    int npair = ctx->npair, eW = ctx->eW;
    void *args[] = {(void *)&c0,   (void *)&c4,    (void *)&sig,  (void *)&At, (void *)&Bt,         (void *)&xw,
                    (void *)&rexp, (void *)&npair, (void *)&npad, (void *)&n0, (void *)&eW, (void *)&ctx->d_err,
                    (void *)&active, (void *)&add};
    FCI_CUDA(cudaLaunchKernel(kern, dim3((unsigned)grid), dim3(sl::kThreads), args, smem, s));
    prof_mark(ctx, rec, prof_slot + 1, s);
    return FCI_OK;
}

}  // namespace fci
