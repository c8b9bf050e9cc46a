// Host side of the tensor-core sigma kernels (sigma_tc_kernel.cuh): layout
// and epilogue selection, launches of sigma_3 and of the same-spin terms.
#include "sigma_tc_kernel.cuh"

namespace fci {

static int round_up(int x, int m) { return (x + m - 1) / m * m; }

void *tc_kernel_2s(int kpad, int epi);
void *tc_kernel_2t(int kpad, int epi);
void *tc_kernel_3s(int kpad, int epi);
void *tc_kernel_3t(int kpad, int epi);

static void *tc_kernel(int nsplit, int kpad, int epi, bool atm) {
    if (nsplit == 2) return atm ? tc_kernel_2t(kpad, epi) : tc_kernel_2s(kpad, epi);
    return atm ? tc_kernel_3t(kpad, epi) : tc_kernel_3s(kpad, epi);
}

// Tensor-memory columns: two accumulators, and with the A operand in tensor
// memory its stages of NS slices (KPAD/2 columns each); allocations are powers
// of two from 32 to 512.
static int tmem_columns(int npad, int kpad, int nsplit, int stages, bool atm) {
    const int need = 2 * npad + (atm ? stages * nsplit * (kpad / 2) : 0);
    int cols = 32;
    while (cols < need) cols <<= 1;
    return cols;
}

// Epilogue (2: sigma row in shared memory, 3: in global memory), A buffers and
// A placement that fit in `lim` bytes of shared memory and 512 tensor-memory
// columns; A in tensor memory and two A buffers preferred.
static bool pick_layout(int nsplit, int kpad, int npad, int64_t nsb, int nsa_single, int lim, int *epi, int *stages,
                        bool *atm, bool global_row = false) {
    // {epilogue, A buffers, A in tensor memory}
    static const int order[][3] = {{2, 2, 1}, {2, 2, 0}, {2, 1, 1}, {2, 1, 0},
                                   {3, 2, 1}, {3, 1, 1}, {3, 2, 0}, {3, 1, 0}};
    for (const auto &o : order)
        if ((o[0] == 3 || !global_row) && tmem_columns(npad, kpad, nsplit, o[1], o[2] != 0) <= 512 &&
            (int)tc::make_layout(nsplit, kpad, npad, nsb, nsa_single, o[0], o[1], o[2] != 0).total <= lim) {
            *epi = o[0];
            *stages = o[1];
            *atm = o[2] != 0;
            return true;
        }
    return false;
}

struct TcPlan {
    void *kern = nullptr;
    int npad = 0, stages = 0;
    uint32_t cols = 0, smem = 0;
};

static int tc_plan(const fci_ctx *ctx, int nsplit, TcPlan *P) {
    const int kpad = round_up(ctx->A.nsingle, 16), npad = round_up(ctx->npair, 16);
    if (npad > 256) return fail(FCI_ERR_ARG, "tensor-core sigma_3 supports at most 256 orbital pairs (norb <= 22)");
    if (kpad > 96) return fail(FCI_ERR_ARG, "tensor-core sigma_3 supports at most 96 alpha replacements per string");
    int lim = 0;
    FCI_CUDA(cudaDeviceGetAttribute(&lim, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
    if (!ctx->B.tsched) return fail(FCI_ERR_ARG, "tensor-core sigma_3: no tile schedule (more than 65408 beta strings)");
    int epi = 0, stages = 0;
    bool atm = false;
    if (!pick_layout(nsplit, kpad, npad, ctx->B.ns, ctx->A.nsingle, lim, &epi, &stages, &atm, ctx->opt.f32_row_global != 0))
        return fail(FCI_ERR_ARG, "tensor-core sigma_3: operands exceed shared or tensor memory");
    P->kern = tc_kernel(nsplit, kpad, epi, atm);
    P->npad = npad;
    P->stages = stages;
    P->smem = tc::make_layout(nsplit, kpad, npad, ctx->B.ns, ctx->A.nsingle, epi, stages, atm).total;
    const int cols = tmem_columns(npad, kpad, nsplit, stages, atm);
    P->cols = (uint32_t)cols;
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
    void *args[] = {(void *)&C,        (void *)&sig,        (void *)&ctx->A, (void *)&ctx->B,
                    (void *)&ctx->Wf,  (void *)&ctx->npair, (void *)&P.npad, (void *)&P.stages,
                    (void *)&P.cols,   (void *)&ctx->d_err, (void *)&active, (void *)&no_kf};
    FCI_CUDA(cudaLaunchKernel(P.kern, dim3((unsigned)grid), dim3(tc::kThreads2), args, P.smem, s));
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
    const int epi = 4;
    int stages = 0;
    bool atm = false;
    uint32_t smem = 0;
    static const int order[][2] = {{2, 1}, {2, 0}, {1, 1}, {1, 0}};  // {A buffers, A in tensor memory}
    for (const auto &o : order) {
        const uint32_t sm = tc::make_layout(nsplit, kpad, npad, cols.ns, R.nsingle, epi, o[0], o[1] != 0).total;
        if ((int)sm <= lim && tmem_columns(npad, kpad, nsplit, o[0], o[1] != 0) <= 512) {
            stages = o[0];
            atm = o[1] != 0;
            smem = sm;
            break;
        }
    }
    if (!stages) return fail(FCI_ERR_ARG, "same-spin tensor-core sigma: operands exceed shared or tensor memory");
    void *kern = tc_kernel(nsplit, kpad, epi, atm);
    const uint32_t tcols = (uint32_t)tmem_columns(npad, kpad, nsplit, stages, atm);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    FCI_CUDA(cudaStreamIsCapturing(s, &cap));
    if (cap == cudaStreamCaptureStatusNone) FCI_CUDA(opt_in_max_smem(kern, ctx->device));
    int64_t grid = nsm;
    if (grid > R.ns) grid = R.ns;
    const int *no_gate = nullptr;
    SpinTables Rt = R, Ct = cols;
    void *args[] = {(void *)&C,       (void *)&sig,        (void *)&Rt,     (void *)&Ct,
                    (void *)&ctx->Wf, (void *)&ctx->npair, (void *)&npad,   (void *)&stages,
                    (void *)&tcols,   (void *)&ctx->d_err, (void *)&no_gate, (void *)&ctx->kf};
    FCI_CUDA(cudaLaunchKernel(kern, dim3((unsigned)grid), dim3(tc::kThreads2), args, smem, s));
    return FCI_OK;
}

// One block waits, through the bounded wait of the tensor-core kernels, on a
// barrier that no thread arrives on; when the wait gives up it sets the error
// word, as those kernels do, and then completes the barrier's phase itself so
// that nothing is left pending.
__global__ void k_wait_timeout_probe(int *err) {
    __shared__ uint64_t bar;
    const uint32_t a = tc::smem_u32(&bar);
    if (threadIdx.x == 0) tc::mbar_init(a, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (!tc::mbar_wait_bounded(a, 0u)) atomicExch(err, 1);
        tc::mbar_arrive(a);
    }
}

int launch_wait_timeout_probe(fci_ctx *ctx) {
    k_wait_timeout_probe<<<1, 32, 0, ctx->stream>>>(ctx->d_err);
    FCI_CUDA(cudaGetLastError());
    return FCI_OK;
}

size_t sigma3_tc_smem(const fci_ctx *ctx, int nsplit) {
    if (ctx->A.nsingle == 0 || ctx->B.nsingle == 0 || !ctx->B.tsched) return 0;
    const int kpad = round_up(ctx->A.nsingle, 16), npad = round_up(ctx->npair, 16);
    int epi = 0, st = 0;
    bool atm = false;
    if (!pick_layout(nsplit, kpad, npad, ctx->B.ns, ctx->A.nsingle, 232448, &epi, &st, &atm)) return 0;
    return tc::make_layout(nsplit, kpad, npad, ctx->B.ns, ctx->A.nsingle, epi, st, atm).total;
}

}  // namespace fci
