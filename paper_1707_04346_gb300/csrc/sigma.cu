// sigma = H c as sigma_1 + sigma_2 + sigma_3 (Eq. 8), string driven (Section 3.3).
//
// Layout: C and sigma are row-major [N_alpha][N_beta] (Eq. 4).
//  sigma_2 (alpha-alpha, I_beta = J_beta): row gather
//      sigma(Ia, :) = sum_J G_a(Ia, J) C(J, :)
//    over the ELL row of the alpha same-spin Hamiltonian; every load of a C
//    row is coalesced along beta.
//  sigma_1 (beta-beta, I_alpha = J_alpha): gather inside one C row
//      sigma(Ia, Ib) += sum_J G_b(Ib, J) C(Ia, J)
//    with the C row staged in shared memory.
//  sigma_3 (alpha-beta): with W[(ij),(kl)] = (ij|kl) and the replacement
//    lists of both strings,
//      sigma(Ia, Ib) += sum_{a in E(Ia)} s_a sum_{b in E(Ib)} s_b W[p_a][p_b] C(J_a, J_b)
//    (the alpha-beta part of 1/2 sum (ij|kl) E_ij E_kl, where the alpha-beta
//    and beta-alpha halves coincide).  One CTA owns an output row; for each
//    alpha replacement a it stages C(J_a, :) and W[p_a, :] in shared memory
//    and accumulates the row of sigma in shared memory.
#include "internal.cuh"

namespace fci {

template <typename T>
__device__ __forceinline__ T gval_of(const SpinTables &S, int64_t idx);
template <>
__device__ __forceinline__ double gval_of<double>(const SpinTables &S, int64_t idx) {
    return S.gval[idx];
}
template <>
__device__ __forceinline__ float gval_of<float>(const SpinTables &S, int64_t idx) {
    return S.gvalf[idx];
}

// sigma(Ia, Ib) = sum_e G_a[e][Ia] * C(col_e, Ib)   (overwrites sigma)
template <typename T>
__global__ void __launch_bounds__(256) k_sigma2_rows(const T *__restrict__ C, T *__restrict__ sig, SpinTables A,
                                                     int64_t nsb) {
    extern __shared__ unsigned char smem_raw[];
    int32_t *col = reinterpret_cast<int32_t *>(smem_raw);
    T *val = reinterpret_cast<T *>(smem_raw + ((sizeof(int32_t) * A.nsame + 15) & ~size_t(15)));
    const int64_t ia = blockIdx.y;
    for (int e = threadIdx.x; e < A.nsame; e += blockDim.x) {
        col[e] = A.gcol[(int64_t)e * A.ns + ia];
        val[e] = gval_of<T>(A, (int64_t)e * A.ns + ia);
    }
    __syncthreads();
    const int64_t ib = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (ib >= nsb) return;
    T acc = 0;
    for (int e = 0; e < A.nsame; ++e) acc += val[e] * C[(int64_t)col[e] * nsb + ib];
    sig[ia * nsb + ib] = acc;
}

// sigma(Ia, Ib) += sum_e G_b[e][Ib] * C(Ia, col_e)
template <typename T>
__global__ void __launch_bounds__(512) k_sigma1_cols(const T *__restrict__ C, T *__restrict__ sig, SpinTables B) {
    extern __shared__ unsigned char smem_raw[];
    T *row = reinterpret_cast<T *>(smem_raw);
    const int64_t nsb = B.ns;
    const int64_t ia = blockIdx.x;
    for (int64_t j = threadIdx.x; j < nsb; j += blockDim.x) row[j] = C[ia * nsb + j];
    __syncthreads();
    for (int64_t ib = threadIdx.x; ib < nsb; ib += blockDim.x) {
        T acc = 0;
        for (int e = 0; e < B.nsame; ++e) {
            int64_t idx = (int64_t)e * nsb + ib;
            acc += gval_of<T>(B, idx) * row[B.gcol[idx]];
        }
        sig[ia * nsb + ib] += acc;
    }
}

template <typename T>
__device__ __forceinline__ T w_of(const double *W, const float *Wf, int64_t i);
template <>
__device__ __forceinline__ double w_of<double>(const double *W, const float *, int64_t i) {
    return W[i];
}
template <>
__device__ __forceinline__ float w_of<float>(const double *, const float *Wf, int64_t i) {
    return Wf[i];
}

__device__ __forceinline__ double flip_sign(double x, uint32_t signbit) {
    return __longlong_as_double(__double_as_longlong(x) ^ ((long long)signbit << 32));
}
__device__ __forceinline__ float flip_sign(float x, uint32_t signbit) {
    return __int_as_float(__float_as_int(x) ^ (int)signbit);
}

template <typename T>
__global__ void __launch_bounds__(512) k_sigma3_exact(const T *__restrict__ C, T *__restrict__ sig, SpinTables A,
                                                      SpinTables B, const double *__restrict__ W,
                                                      const float *__restrict__ Wf, int npair) {
    extern __shared__ unsigned char smem_raw[];
    const int64_t nsb = B.ns;
    T *crow = reinterpret_cast<T *>(smem_raw);
    T *acc = crow + nsb;
    T *wrow = acc + nsb;
    uint32_t *ea = reinterpret_cast<uint32_t *>(wrow + npair);
    const int64_t ia = blockIdx.x;
    for (int e = threadIdx.x; e < A.nsingle; e += blockDim.x) ea[e] = A.tab[(int64_t)e * A.ns + ia];
    for (int64_t j = threadIdx.x; j < nsb; j += blockDim.x) acc[j] = 0;
    for (int a = 0; a < A.nsingle; ++a) {
        __syncthreads();  // previous a finished with crow / wrow; ea visible
        const uint32_t enta = ea[a];
        const int64_t ja = ent_target(enta);
        const int pa = ent_pair(enta);
        for (int64_t j = threadIdx.x; j < nsb; j += blockDim.x) crow[j] = C[ja * nsb + j];
        for (int q = threadIdx.x; q < npair; q += blockDim.x) wrow[q] = w_of<T>(W, Wf, (int64_t)pa * npair + q);
        __syncthreads();
        const T sa = ent_negative(enta) ? T(-1) : T(1);
        for (int64_t ib = threadIdx.x; ib < nsb; ib += blockDim.x) {
            T v = 0;
            for (int b = 0; b < B.nsingle; ++b) {
                const uint32_t entb = B.tab[(int64_t)b * nsb + ib];
                // the beta sign goes in by flipping the sign bit (integer pipe), so
                // each replacement pair costs one fused multiply-add
                v = fma(flip_sign(wrow[ent_pair(entb)], entb & 0x80000000u), crow[ent_target(entb)], v);
            }
            acc[ib] += sa * v;
        }
    }
    __syncthreads();
    for (int64_t j = threadIdx.x; j < nsb; j += blockDim.x) sig[ia * nsb + j] += acc[j];
}

static size_t smem_limit() {
    static int lim = -1;
    if (lim < 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&lim, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    }
    return (size_t)lim;
}

template <typename T>
static int sigma_impl(fci_ctx *ctx, const T *C, T *sig, cudaStream_t s) {
    const SpinTables &A = ctx->A, &B = ctx->B;
    const int64_t nsa = A.ns, nsb = B.ns;
    const size_t lim = smem_limit();
    static const char *const names[3] = {"sigma2_rows", "sigma1_cols", sizeof(T) == 4 ? "sigma3_tc" : "sigma3_exact"};
    const int rec = prof_begin(ctx, s, 3, names);
    // sigma_2
    {
        size_t sm = ((sizeof(int32_t) * A.nsame + 15) & ~size_t(15)) + sizeof(T) * A.nsame;
        if (sm > lim) return fail(FCI_ERR_ARG, "same-spin row too wide for shared memory");
        if (sm > 48 * 1024) FCI_CUDA(cudaFuncSetAttribute(k_sigma2_rows<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        dim3 grid(ceil_div(nsb, 256), (unsigned)nsa);
        k_sigma2_rows<T><<<grid, 256, sm, s>>>(C, sig, A, nsb);
        FCI_CUDA(cudaGetLastError());
        prof_mark(ctx, rec, 0, s);
    }
    // sigma_1
    {
        size_t sm = sizeof(T) * nsb;
        if (sm > lim) return fail(FCI_ERR_ARG, "beta string count too large for the sigma_1 row kernel");
        if (sm > 48 * 1024) FCI_CUDA(cudaFuncSetAttribute(k_sigma1_cols<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        k_sigma1_cols<T><<<(unsigned)nsa, 512, sm, s>>>(C, sig, B);
        FCI_CUDA(cudaGetLastError());
        prof_mark(ctx, rec, 1, s);
    }
    // sigma_3
    if (A.nsingle > 0 && B.nsingle > 0 && sizeof(T) == 4) {
        if (int rc = launch_sigma3_tc(ctx, (const float *)C, (float *)sig, ctx->opt.f32_splits, s)) return rc;
    } else if (A.nsingle > 0 && B.nsingle > 0) {
        size_t sm = sizeof(T) * (2 * nsb + ctx->npair) + sizeof(uint32_t) * A.nsingle;
        if (sm > lim) return fail(FCI_ERR_ARG, "beta string count too large for the sigma_3 row kernel");
        if (sm > 48 * 1024) FCI_CUDA(cudaFuncSetAttribute(k_sigma3_exact<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        k_sigma3_exact<T><<<(unsigned)nsa, 512, sm, s>>>(C, sig, A, B, ctx->W, ctx->Wf, ctx->npair);
        FCI_CUDA(cudaGetLastError());
    }
    prof_mark(ctx, rec, 2, s);
    return FCI_OK;
}

int launch_sigma(fci_ctx *ctx, const void *c, void *sigma, int dtype, cudaStream_t s) {
    if (dtype == FCI_F64) return sigma_impl<double>(ctx, (const double *)c, (double *)sigma, s);
    if (dtype == FCI_F32) return sigma_impl<float>(ctx, (const float *)c, (float *)sigma, s);
    return fail(FCI_ERR_ARG, "dtype must be FCI_F64 or FCI_F32");
}

}  // namespace fci
