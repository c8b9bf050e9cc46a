// Host side of the FP64-accurate tensor-core sigma for large string spaces
// (sigma_wide_kernel.cuh): its tables (built once at fci_init), the per-call
// pre-passes, and the sequence of one FP64 sigma = sigma_1 + sigma_2 + sigma_3
// (Eq. 8) through one 64-bit integer accumulator.
#include <cmath>
#include <vector>

#include "sigma_wide_kernel.cuh"

namespace fci {

static int round_up16(int x) { return (x + 15) / 16 * 16; }

// *eG = max(*eG, largest biased FP64 exponent field in x[0..n)).
__global__ void k_global_exponent(const double *__restrict__ x, int64_t n, int *__restrict__ eG) {
    unsigned mx = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const unsigned long long *u = reinterpret_cast<const unsigned long long *>(x);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        mx = max(mx, (unsigned)((__ldg(u + i) >> 52) & 0x7FFull));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(eG, (int)mx);
}

// Six bf16 digit slices of every value, all relative to the one exponent *eG.
__global__ void k_slice_global(const double *__restrict__ x, int64_t n, const int *__restrict__ eG,
                               uint2 *__restrict__ cs0123, uint32_t *__restrict__ cs45) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const unsigned long long b = __double_as_longlong(__ldg(x + t));
    float f[sl::kSlices];
    sl::digits6(sl::fixed47((uint32_t)b, (uint32_t)(b >> 32), *eG), f);
    cs0123[t] = make_uint2(sl::pack_bf16(f[0], f[1]), sl::pack_bf16(f[2], f[3]));
    cs45[t] = sl::pack_bf16(f[4], f[5]);
}

// out[c][r] = in[r][c] for a rows x cols matrix of 8-byte words (32 x 32 tiles).
__global__ void k_transpose_u64(const unsigned long long *__restrict__ in, unsigned long long *__restrict__ out,
                                int64_t rows, int64_t cols) {
    __shared__ unsigned long long tile[32][33];
    const int64_t c0 = (int64_t)blockIdx.x * 32, r0 = (int64_t)blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int64_t r = r0 + i, c = c0 + threadIdx.x;
        if (r < rows && c < cols) tile[i][threadIdx.x] = in[r * cols + c];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int64_t c = c0 + i, r = r0 + threadIdx.x;
        if (c < cols && r < rows) out[c * rows + r] = tile[threadIdx.x][i];
    }
}

// sigma[i] = acc[i] 2^(e2) as FP64 with e2 = *eG - 1022 + eC - 49 (NaN
// everywhere when C held a non-finite value).  acc and sigma may alias.
__global__ void k_convert_acc(const long long *acc, double *sig, int64_t n, const int *__restrict__ eG, int eC,
                              int add = 0) {
    const int e = *eG;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const long long v = acc[i];
        const double x = e == 0x7FF ? __longlong_as_double(0x7FF8000000000000ll) : sl::scaled_i64(v, e - 1022 + eC - 49);
        sig[i] = add ? sig[i] + x : x;
    }
}

// tabp32[x][q] = the packed entry of string x with orbital pair q (one at
// most), else kNoEntry (left by the memset).
__global__ void k_pair_table32(const uint32_t *__restrict__ tab, int64_t ns, int nsingle, int npad,
                               uint32_t *__restrict__ tabp32) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ns * nsingle) return;
    const uint32_t v = tab[t];  // entry-major: t = e * ns + x
    tabp32[(t % ns) * npad + ent_pair(v)] = v;
}

// Sizes of one launch of the wide kernel with row table R (MODE 1 has the
// one-body column q = npair); false when the kernel does not cover it.
struct WideShape {
    int kpad = 0, npad = 0, nparts = 0;
    uint32_t smem = 0;
};

static bool wide_shape(const fci_ctx *ctx, const SpinTables &R, int mode, WideShape *S) {
    if (R.nsingle == 0 || R.nsingle > 16 * wd::kMaxKSteps || R.ns > kMaxStrings) return false;
    S->kpad = round_up16(R.nsingle);
    S->npad = round_up16(ctx->npair + (mode == 1 ? 1 : 0));
    if (S->npad > 256) return false;
    S->nparts = (S->npad + wd::kPartMax - 1) / wd::kPartMax;
    S->smem = wd::make_layout(S->kpad, S->npad, R.nsingle).total;
    int lim = 0;
    if (cudaDeviceGetAttribute(&lim, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device) != cudaSuccess) return false;
    return (int)S->smem <= lim;
}

// Whether the wide kernels cover every term this context has.
bool sigma_wide_fits(const fci_ctx *ctx) {
    const SpinTables &A = ctx->A, &B = ctx->B;
    if (A.ns > kMaxStrings || B.ns > kMaxStrings) return false;
    WideShape S;
    if (A.nsingle > 0 && (!wide_shape(ctx, A, 0, &S) || !wide_shape(ctx, A, 1, &S))) return false;
    if (B.nsingle > 0 && !wide_shape(ctx, B, 1, &S)) return false;
    return true;
}

bool sigma_wide_ok(const fci_ctx *ctx) { return ctx->XT != nullptr; }

template <int MODE>
static void *wide_kernel(int kpad) {
    switch (kpad) {
        case 16: return (void *)wd::k_sigma_wide<16, MODE>;
        case 32: return (void *)wd::k_sigma_wide<32, MODE>;
        case 48: return (void *)wd::k_sigma_wide<48, MODE>;
        case 64: return (void *)wd::k_sigma_wide<64, MODE>;
        case 80: return (void *)wd::k_sigma_wide<80, MODE>;
        case 96: return (void *)wd::k_sigma_wide<96, MODE>;
        default: return nullptr;
    }
}

// Build, once per context: the fixed-point integral table
//   XT[q][p] = round((q|p) 2^(47 - eC))   (q < npair; |(q|p)| < 2^(eC - 1), so |XT| <= 2^46)
//   XT[npair][p] = round(k_p 2^(48 - eC - sh1))
// whose two-electron rows are sigma_3's (q|p) in the scale 2^(47 - eC) and the
// same-spin term's (q|p)/2 in the scale 2^(48 - eC), so that all products
// share the unit 2^(eD + eC - 49) once sigma_3's integers are doubled; the
// one-body row k (often the larger) is in a scale 2^sh1 coarser, sh1 <= 4
// (beyond that eC grows with max|k|, so that no sum can leave 64 bits); the
// beta pair table with 32-bit entries; the digit planes of C (12 bytes per
// determinant); and the 8-byte per determinant accumulator (the FP32
// same-spin workspace when the context has one: the two are never used in one
// call).
int build_wide_tables(fci_ctx *ctx, const double *h1_host, const double *eri_host) {
    const int n = ctx->norb, np = ctx->npair;
    const int64_t n2 = (int64_t)n * n;
    std::vector<double> W((size_t)np * np), kq((size_t)np);
    double wmax = 0.0, kmax = 0.0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j <= i; ++j)
            for (int k = 0; k < n; ++k)
                for (int l = 0; l <= k; ++l) {
                    const double v = eri_host[i * n2 * n + j * n2 + (int64_t)k * n + l];
                    W[(size_t)pair_index(i, j) * np + pair_index(k, l)] = v;
                    wmax = std::fmax(wmax, std::fabs(v));
                }
    for (int k = 0; k < n; ++k)
        for (int l = 0; l <= k; ++l) {
            double v = h1_host[k * n + l];
            for (int j = 0; j < n; ++j) v -= 0.5 * eri_host[((int64_t)k * n + j) * n2 + (int64_t)j * n + l];
            kq[pair_index(k, l)] = v;
            kmax = std::fmax(kmax, std::fabs(v));
        }
    int ew = 0, ek = 0;
    if (wmax > 0) std::frexp(wmax, &ew);  // |W| < 2^ew
    if (kmax > 0) std::frexp(kmax, &ek);  // |k| < 2^ek
    int eC = ew + 1;
    if (ek + 2 - eC > 4) eC = ek - 2;
    const int sh1 = ek + 2 - eC > 0 ? ek + 2 - eC : 0;  // |k| < 2^(eC + sh1 - 2)
    std::vector<long long> xt((size_t)(np + 1) * np);
    for (size_t i = 0; i < (size_t)np * np; ++i) xt[i] = std::llrint(std::ldexp(W[i], 47 - eC));
    for (int p = 0; p < np; ++p) xt[(size_t)np * np + p] = std::llrint(std::ldexp(kq[p], 48 - eC - sh1));
    if (int rc = alloc_sigma_workspace(ctx)) return rc;
    int rc = FCI_OK;
    SpinTables &B = ctx->B;
    const int npad0 = round_up16(np);
    ctx->XT = (long long *)dalloc(ctx, sizeof(long long) * xt.size(), &rc);
    ctx->d_eG = (int *)dalloc(ctx, sizeof(int), &rc);
    if (!ctx->cs0123) ctx->cs0123 = (uint2 *)dalloc(ctx, sizeof(uint2) * (size_t)ctx->ndet, &rc);
    if (!ctx->cs45) ctx->cs45 = (uint32_t *)dalloc(ctx, sizeof(uint32_t) * (size_t)ctx->ndet, &rc);
    if (!ctx->ws32) ctx->wsacc = (long long *)dalloc(ctx, sizeof(long long) * (size_t)ctx->ndet, &rc);
    if (B.nsingle > 0 && ctx->A.nsingle > 0)
        B.tabp32 = (uint32_t *)dalloc(ctx, sizeof(uint32_t) * (size_t)npad0 * B.ns, &rc);
    if (rc) return rc;
    ctx->eC = eC;
    ctx->sh1 = sh1;
    FCI_CUDA(cudaMemcpyAsync(ctx->XT, xt.data(), sizeof(long long) * xt.size(), cudaMemcpyHostToDevice, ctx->stream));
    if (B.tabp32) {
        FCI_CUDA(cudaMemsetAsync(B.tabp32, 0xFF, sizeof(uint32_t) * (size_t)npad0 * B.ns, ctx->stream));
        k_pair_table32<<<ceil_div(B.ns * B.nsingle, 256), 256, 0, ctx->stream>>>(B.tab, B.ns, B.nsingle, npad0,
                                                                                 B.tabp32);
        FCI_CUDA(cudaGetLastError());
    }
    FCI_CUDA(cudaStreamSynchronize(ctx->stream));
    return FCI_OK;
}

void free_wide_tables(fci_ctx *ctx) {
    const int np = ctx->npair;
    if (ctx->B.tabp32) dfree(ctx, ctx->B.tabp32, sizeof(uint32_t) * (size_t)round_up16(np) * ctx->B.ns);
    ctx->B.tabp32 = nullptr;
    dfree(ctx, ctx->XT, sizeof(long long) * (size_t)(np + 1) * np);
    dfree(ctx, ctx->d_eG, sizeof(int));
    dfree(ctx, ctx->wsacc, sizeof(long long) * (size_t)ctx->ndet);
    ctx->XT = nullptr;
    ctx->wsacc = nullptr;
    ctx->d_eG = nullptr;
}

// One launch of the wide kernel over the digit planes in ctx->cs*, adding to acc.
template <int MODE>
static int launch_wide(fci_ctx *ctx, const SpinTables &R, int64_t ncols, unsigned long long *acc, cudaStream_t s) {
    WideShape S;
    if (!wide_shape(ctx, R, MODE, &S)) return fail(FCI_ERR_STATE, "wide FP64 sigma: shape not covered");
    void *kern = wide_kernel<MODE>(S.kpad);
    FCI_CUDA(opt_in_max_smem(kern, ctx->device));
    int nsm = 0;
    FCI_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device));
    int64_t grid = nsm;  // one CTA per SM
    if (grid > R.ns * S.nparts) grid = R.ns * S.nparts;
    SpinTables Rt = R;
    const uint2 *c0 = ctx->cs0123;
    const uint32_t *c4 = ctx->cs45;
    const uint32_t *tabp = ctx->B.tabp32;
    const long long *xt = ctx->XT;
    int npair = ctx->npair, shq = MODE == 0 ? 1 : ctx->sh1;
    void *args[] = {(void *)&c0,   (void *)&c4,    (void *)&acc,   (void *)&Rt,     (void *)&ncols,
                    (void *)&tabp, (void *)&xt,    (void *)&npair, (void *)&S.npad, (void *)&S.nparts,
                    (void *)&shq,  (void *)&ctx->d_err};
    FCI_CUDA(cudaLaunchKernel(kern, dim3((unsigned)grid), dim3(wd::kThreads), args, S.smem, s));
    return FCI_OK;
}

static unsigned grid_stride_blocks(int64_t n) {
    const int64_t b = (n + 255) / 256;
    return (unsigned)(b < 8 * 152 ? (b < 1 ? 1 : b) : 8 * 152);
}

// FP64 sigma = H C through the wide kernels (sig overwritten):
//  1. eG = largest exponent of C;
//  2. sigma_1 as the same-spin term of the beta strings on C transposed (the
//     gathered rows must be contiguous): transpose C into the accumulator
//     buffer, slice it, accumulate into sig (as 64-bit integers, transposed),
//     transpose back into the accumulator buffer;
//  3. slice C; sigma_3 and sigma_2 add to the accumulator;
//  4. convert the accumulator to FP64 into sig.
// Profiling slots: transpose and slice, sigma1, sigma3 (with the slicing of C),
// sigma2, convert.
int launch_sigma_f64_wide(fci_ctx *ctx, const double *C, double *sig, cudaStream_t s, int parity) {
    if (!sigma_wide_ok(ctx)) return fail(FCI_ERR_STATE, "wide FP64 sigma tables were not built for this context");
    if (sigma_ss_ok(ctx)) {
        // sigma_3 through the wide kernel; sigma_1 and sigma_2 as dense sliced products
        const int64_t n = ctx->ndet;
        unsigned long long *acc = ctx->ws32 ? reinterpret_cast<unsigned long long *>(ctx->ws32)
                                            : reinterpret_cast<unsigned long long *>(ctx->wsacc);
        auto sigma3 = [&](int rec, int slot, int add) -> int {
            FCI_CUDA(cudaMemsetAsync(ctx->d_eG, 0, sizeof(int), s));
            k_global_exponent<<<grid_stride_blocks(n), 256, 0, s>>>(C, n, ctx->d_eG);
            k_slice_global<<<ceil_div(n, 256), 256, 0, s>>>(C, n, ctx->d_eG, ctx->cs0123, ctx->cs45);
            FCI_CUDA(cudaGetLastError());
            FCI_CUDA(cudaMemsetAsync(acc, 0, sizeof(long long) * (size_t)n, s));
            prof_mark(ctx, rec, slot, s);
            if (int rc = launch_wide<0>(ctx, ctx->A, ctx->B.ns, acc, s)) return rc;
            prof_mark(ctx, rec, slot + 1, s);
            k_convert_acc<<<grid_stride_blocks(n), 256, 0, s>>>(reinterpret_cast<const long long *>(acc), sig, n,
                                                                 ctx->d_eG, ctx->eC, add);
            FCI_CUDA(cudaGetLastError());
            prof_mark(ctx, rec, slot + 2, s);
            return FCI_OK;
        };
        if (parity != 0) {  // sigma_2, sigma_1 = parity sigma_2^T, then sigma_3 added
            static const char *const namesp[5] = {"sigma2_ss", "sigma1_sym", "slice_c", "sigma3_wide", "convert"};
            const int rec = prof_begin(ctx, s, 5, namesp);
            FCI_CUDA(cudaMemsetAsync(sig, 0, sizeof(double) * (size_t)n, s));
            if (int rc = launch_sigma_ss(ctx, C, sig, 2, s, rec, 0)) return rc;
            if (int rc = sym_pairs(sig, ctx->A.ns, 8, parity, 0, s)) return rc;
            prof_mark(ctx, rec, 1, s);
            return sigma3(rec, 2, 1);
        }
        static const char *const names[5] = {"slice_c", "sigma3_wide", "convert", "sigma1_ss", "sigma2_ss"};
        const int rec = prof_begin(ctx, s, 5, names);
        if (int rc = sigma3(rec, 0, 0)) return rc;
        return launch_sigma_ss(ctx, C, sig, 3, s, rec, 3);
    }
    if (parity != 0 && ctx->A.nsingle > 0) {
        // C^T = parity C (one string space): sigma_2 into the accumulator, sigma_1 =
        // parity sigma_2^T by one integer transpose-add, then sigma_3 adds
        static const char *const namesp[5] = {"slice_c", "sigma2_wide", "sigma1_sym", "sigma3_wide", "convert"};
        const int rec = prof_begin(ctx, s, 5, namesp);
        const int64_t ns = ctx->A.ns, n = ctx->ndet;
        unsigned long long *acc = ctx->ws32 ? reinterpret_cast<unsigned long long *>(ctx->ws32)
                                            : reinterpret_cast<unsigned long long *>(ctx->wsacc);
        FCI_CUDA(cudaMemsetAsync(ctx->d_eG, 0, sizeof(int), s));
        k_global_exponent<<<grid_stride_blocks(n), 256, 0, s>>>(C, n, ctx->d_eG);
        k_slice_global<<<ceil_div(n, 256), 256, 0, s>>>(C, n, ctx->d_eG, ctx->cs0123, ctx->cs45);
        FCI_CUDA(cudaGetLastError());
        FCI_CUDA(cudaMemsetAsync(acc, 0, sizeof(long long) * (size_t)n, s));
        prof_mark(ctx, rec, 0, s);
        if (int rc = launch_wide<1>(ctx, ctx->A, ns, acc, s)) return rc;
        prof_mark(ctx, rec, 1, s);
        if (int rc = sym_pairs(acc, ns, -8, parity, 0, s)) return rc;
        prof_mark(ctx, rec, 2, s);
        if (int rc = launch_wide<0>(ctx, ctx->A, ns, acc, s)) return rc;
        prof_mark(ctx, rec, 3, s);
        k_convert_acc<<<grid_stride_blocks(n), 256, 0, s>>>(reinterpret_cast<const long long *>(acc), sig, n,
                                                             ctx->d_eG, ctx->eC);
        FCI_CUDA(cudaGetLastError());
        prof_mark(ctx, rec, 4, s);
        return FCI_OK;
    }
    static const char *const names[5] = {"transpose_slice", "sigma1_wide", "sigma3_wide", "sigma2_wide", "convert"};
    const int rec = prof_begin(ctx, s, 5, names);
    const SpinTables &A = ctx->A, &B = ctx->B;
    const int64_t nsa = A.ns, nsb = B.ns, n = ctx->ndet;
    unsigned long long *acc = ctx->ws32 ? reinterpret_cast<unsigned long long *>(ctx->ws32)
                                        : reinterpret_cast<unsigned long long *>(ctx->wsacc);
    unsigned long long *sacc = reinterpret_cast<unsigned long long *>(sig);
    FCI_CUDA(cudaMemsetAsync(ctx->d_eG, 0, sizeof(int), s));
    k_global_exponent<<<grid_stride_blocks(n), 256, 0, s>>>(C, n, ctx->d_eG);
    FCI_CUDA(cudaGetLastError());
    const dim3 tb(32, 8);
    if (B.nsingle > 0) {
        k_transpose_u64<<<dim3(ceil_div(nsb, 32), ceil_div(nsa, 32)), tb, 0, s>>>(
            reinterpret_cast<const unsigned long long *>(C), acc, nsa, nsb);
        k_slice_global<<<ceil_div(n, 256), 256, 0, s>>>(reinterpret_cast<const double *>(acc), n, ctx->d_eG,
                                                        ctx->cs0123, ctx->cs45);
        FCI_CUDA(cudaGetLastError());
        prof_mark(ctx, rec, 0, s);
        FCI_CUDA(cudaMemsetAsync(sacc, 0, sizeof(long long) * (size_t)n, s));
        if (int rc = launch_wide<1>(ctx, B, nsa, sacc, s)) return rc;
        k_transpose_u64<<<dim3(ceil_div(nsa, 32), ceil_div(nsb, 32)), tb, 0, s>>>(sacc, acc, nsb, nsa);
        FCI_CUDA(cudaGetLastError());
        prof_mark(ctx, rec, 1, s);
    } else {
        FCI_CUDA(cudaMemsetAsync(acc, 0, sizeof(long long) * (size_t)n, s));
        prof_mark(ctx, rec, 0, s);
        prof_mark(ctx, rec, 1, s);
    }
    if (A.nsingle > 0) {
        k_slice_global<<<ceil_div(n, 256), 256, 0, s>>>(C, n, ctx->d_eG, ctx->cs0123, ctx->cs45);
        FCI_CUDA(cudaGetLastError());
        if (B.nsingle > 0)
            if (int rc = launch_wide<0>(ctx, A, nsb, acc, s)) return rc;
        prof_mark(ctx, rec, 2, s);
        if (int rc = launch_wide<1>(ctx, A, nsb, acc, s)) return rc;
        prof_mark(ctx, rec, 3, s);
    } else {
        prof_mark(ctx, rec, 2, s);
        prof_mark(ctx, rec, 3, s);
    }
    k_convert_acc<<<grid_stride_blocks(n), 256, 0, s>>>(reinterpret_cast<const long long *>(acc), sig, n, ctx->d_eG,
                                                         ctx->eC);
    FCI_CUDA(cudaGetLastError());
    prof_mark(ctx, rec, 4, s);
    return FCI_OK;
}

}  // namespace fci
