// Spin-summed one-particle density gamma_pq = <c| E_pq |c> (Eq. 7), the
// density the paper builds in an extra CI pass after the Davidson iterations
// (Section 4, Table 2 "1e/2e Density Matrices").
//
// gamma = gamma_alpha + gamma_beta.  With the replacement list of string J
// (entry e: a+_k a_l |J> = s |T>),
//   alpha: sum_{J, e} s * <C(T, :), C(J, :)>      (dot of two rows)
//   beta:  sum_{J, e} s * <C(:, T), C(:, J)>      (dot of two columns)
// land in the bin of the unordered pair {k, l}; a bin with k != l receives
// gamma_kl + gamma_lk = 2 gamma_kl (real c).  Pass 1 writes one partial per
// (entry, string) into scratch, pass 2 sums each pair bin in a fixed order,
// so the result is bitwise reproducible.
#include "internal.cuh"

namespace fci {

template <typename T>
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x < 32) {
        r = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    }
    return r;  // valid in thread 0
}

// alpha partials: block (e, J) -> s * <C(T,:), C(J,:)>
template <typename T>
__global__ void __launch_bounds__(256) k_rdm_alpha(const T *__restrict__ C, SpinTables A, int64_t nsb,
                                                   double *__restrict__ part) {
    const int e = blockIdx.y;
    const int64_t j = blockIdx.x;
    const uint32_t ent = A.tab[(int64_t)e * A.ns + j];
    const int64_t t = ent_target(ent);
    double acc = 0.0;
    for (int64_t b = threadIdx.x; b < nsb; b += blockDim.x) acc += (double)C[t * nsb + b] * (double)C[j * nsb + b];
    acc = block_sum<T>(acc);
    if (threadIdx.x == 0) part[(int64_t)e * A.ns + j] = ent_negative(ent) ? -acc : acc;
}

// beta partials: thread (e, J) -> s * sum_Ia C(Ia, T) C(Ia, J)
template <typename T>
__global__ void __launch_bounds__(256) k_rdm_beta(const T *__restrict__ C, SpinTables B, int64_t nsa,
                                                  double *__restrict__ part) {
    const int e = blockIdx.y;
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= B.ns) return;
    const uint32_t ent = B.tab[(int64_t)e * B.ns + j];
    const int64_t t = ent_target(ent);
    double acc = 0.0;
    for (int64_t a = 0; a < nsa; ++a) acc += (double)C[a * B.ns + t] * (double)C[a * B.ns + j];
    part[(int64_t)e * B.ns + j] = ent_negative(ent) ? -acc : acc;
}

// pass 2: one block per pair bin, fixed-order sums over both partial arrays
__global__ void __launch_bounds__(256) k_rdm_bins(SpinTables A, SpinTables B, const double *__restrict__ pa,
                                                  const double *__restrict__ pb, int norb, double *__restrict__ gamma) {
    const int P = blockIdx.x;
    double acc = 0.0;
    const int64_t na = A.ns * A.nsingle, nb = B.ns * B.nsingle;
    for (int64_t i = threadIdx.x; i < na; i += blockDim.x)
        if ((int)ent_pair(A.tab[i]) == P) acc += pa[i];
    for (int64_t i = threadIdx.x; i < nb; i += blockDim.x)
        if ((int)ent_pair(B.tab[i]) == P) acc += pb[i];
    acc = block_sum<double>(acc);
    if (threadIdx.x == 0) {
        int k = 0;
        while ((k + 1) * (k + 2) / 2 <= P) ++k;
        int l = P - k * (k + 1) / 2;
        if (k == l) {
            gamma[k * norb + k] = acc;
        } else {
            gamma[k * norb + l] = 0.5 * acc;
            gamma[l * norb + k] = 0.5 * acc;
        }
    }
}

template <typename T>
static int rdm_impl(fci_ctx *ctx, const T *C, double *gamma_host) {
    const SpinTables &A = ctx->A, &B = ctx->B;
    const int n = ctx->norb;
    int rc = FCI_OK;
    const size_t na = (size_t)A.ns * A.nsingle, nb = (size_t)B.ns * B.nsingle;
    double *pa = (double *)dalloc(ctx, sizeof(double) * (na ? na : 1), &rc);
    double *pb = (double *)dalloc(ctx, sizeof(double) * (nb ? nb : 1), &rc);
    double *g = (double *)dalloc(ctx, sizeof(double) * n * n, &rc);
    cudaStream_t s = ctx->stream;
    cudaError_t e = cudaSuccess;
    if (rc == FCI_OK) {
        e = cudaMemsetAsync(g, 0, sizeof(double) * n * n, s);
        if (e == cudaSuccess && na) {
            k_rdm_alpha<T><<<dim3((unsigned)A.ns, A.nsingle), 256, 0, s>>>(C, A, B.ns, pa);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess && nb) {
            k_rdm_beta<T><<<dim3(ceil_div(B.ns, 256), B.nsingle), 256, 0, s>>>(C, B, A.ns, pb);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) {
            k_rdm_bins<<<ctx->npair, 256, 0, s>>>(A, B, pa, pb, n, g);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(gamma_host, g, sizeof(double) * n * n, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_fail(e, "rdm1");
    }
    dfree(ctx, pa, sizeof(double) * (na ? na : 1));
    dfree(ctx, pb, sizeof(double) * (nb ? nb : 1));
    dfree(ctx, g, sizeof(double) * n * n);
    return rc;
}

int run_rdm1(fci_ctx *ctx, const void *c, int dtype, double *gamma) {
    if (dtype == FCI_F64) return rdm_impl<double>(ctx, (const double *)c, gamma);
    return rdm_impl<float>(ctx, (const float *)c, gamma);
}

}  // namespace fci

// ---------------------------------------------------------------------------
// fci_rdm1_noalloc: the same density as fci_rdm1, with its scratch in a
// file-scope device array instead of per-call cudaMalloc/cudaFree.
//
// The array below is a host-side stand-in in host code: its device address
// is looked up with cudaGetSymbolAddress once per device (with that device
// current) and cached; kernels receive that address.  Every call shares the
// one array, so calls whose GPU work overlaps race on it.
// ---------------------------------------------------------------------------
#include <mutex>

static __device__ __align__(256) double g_rdm1_scratch[FCI_RDM1_NOALLOC_MAX_DOUBLES];

namespace fci {
namespace {
std::mutex g_scratch_mu;
constexpr int kMaxDevices = 64;
double *g_scratch_addr[kMaxDevices] = {};

// Device address of g_rdm1_scratch on the current device `dev`.
int scratch_address(int dev, double **out) {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (dev < 0 || dev >= kMaxDevices) return fail(FCI_ERR_ARG, "device ordinal out of range for the scratch cache");
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_rdm1_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(rdm1 scratch)");
        g_scratch_addr[dev] = (double *)p;
    }
    *out = g_scratch_addr[dev];
    return FCI_OK;
}

template <typename T>
int rdm_noalloc_impl(fci_ctx *ctx, const T *C, double *gamma_host, cudaStream_t s) {
    const SpinTables &A = ctx->A, &B = ctx->B;
    const int n = ctx->norb;
    const size_t na = (size_t)A.ns * A.nsingle, nb = (size_t)B.ns * B.nsingle, ng = (size_t)n * n;
    if (na + nb + ng > (size_t)FCI_RDM1_NOALLOC_MAX_DOUBLES) {
        char buf[200];
        snprintf(buf, sizeof(buf),
                 "fci_rdm1_noalloc needs %zu scratch doubles, above its fixed limit of %d "
                 "(FCI_RDM1_NOALLOC_MAX_DOUBLES); use fci_rdm1",
                 na + nb + ng, FCI_RDM1_NOALLOC_MAX_DOUBLES);
        return fail(FCI_ERR_ARG, buf);
    }
    double *base = nullptr;
    if (int rc = scratch_address(ctx->device, &base)) return rc;
    double *pa = base, *pb = base + na, *g = base + na + nb;
    // the density bins must start at zero; the partials are fully overwritten
    FCI_CUDA(cudaMemsetAsync(g, 0, sizeof(double) * ng, s));
    if (na) {
        k_rdm_alpha<T><<<dim3((unsigned)A.ns, A.nsingle), 256, 0, s>>>(C, A, B.ns, pa);
        FCI_CUDA(cudaGetLastError());
    }
    if (nb) {
        k_rdm_beta<T><<<dim3(ceil_div(B.ns, 256), B.nsingle), 256, 0, s>>>(C, B, A.ns, pb);
        FCI_CUDA(cudaGetLastError());
    }
    k_rdm_bins<<<ctx->npair, 256, 0, s>>>(A, B, pa, pb, n, g);
    FCI_CUDA(cudaGetLastError());
    FCI_CUDA(cudaMemcpyAsync(gamma_host, g, sizeof(double) * ng, cudaMemcpyDeviceToHost, s));
    FCI_CUDA(cudaStreamSynchronize(s));
    return FCI_OK;
}
}  // namespace
}  // namespace fci

extern "C" int fci_rdm1_noalloc(fci_ctx *ctx, const void *c, int dtype, double *gamma, void *stream) {
    using namespace fci;
    if (!ctx || !c || !gamma) return fail(FCI_ERR_ARG, "NULL argument");
    if (dtype != FCI_F64 && dtype != FCI_F32) return fail(FCI_ERR_ARG, "dtype must be FCI_F64 or FCI_F32");
    // the caller's current device is restored on every return path
    int prev = -1;
    FCI_CUDA(cudaGetDevice(&prev));
    FCI_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    const int rc = dtype == FCI_F64 ? rdm_noalloc_impl<double>(ctx, (const double *)c, gamma, s)
                                    : rdm_noalloc_impl<float>(ctx, (const float *)c, gamma, s);
    const cudaError_t e = cudaSetDevice(prev);
    if (rc == FCI_OK && e != cudaSuccess) return cuda_fail(e, "cudaSetDevice (restoring the caller's device)");
    return rc;
}
