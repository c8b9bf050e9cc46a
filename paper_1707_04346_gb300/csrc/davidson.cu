// Device-resident Davidson eigensolver (Section 3.3).
//
// The paper lists the steps: (1) build and diagonalise an initial subspace
// matrix, which needs an initial sigma; (2) compute the preconditioner;
// (3) multiply by the inverse (diagonal) Hessian and orthogonalise against the
// previous vectors; (4) build the new sigma and diagonalise the enlarged
// projected matrix; repeat from (2) until converged.  The variant it uses
// ("modified inverted-Davidson") is not defined there; this driver reads it
// as block Davidson-Liu with
//   t_k = -(H_diag - E_k)^{-1} r_k,  r_k = H x_k - E_k x_k,
// denominators with |H_II - E| < 1e-8 replaced by +-1e-8, classical
// Gram-Schmidt applied twice, corrections with norm < 1e-10 dropped,
// convergence when every root has |dE| < tol and ||r|| < sqrt(tol), unit
// vectors on the lowest diagonal elements as the guess (ties: lower index),
// and a thick restart when the subspace is full: collapse onto the lowest
// min(8, max_subspace/2) Ritz vectors (at least nroots).
//
// Every vector operation, the projected matrix, its diagonalisation (cyclic
// Jacobi in one CTA, FP64) and the residual norms stay on the device.  The
// host reads back 2*nroots doubles per iteration for the convergence test.
//
// Mixed precision: every new correction gets an FP32 sigma (sigma_3 on the
// tensor cores); the basis, the projected matrix, orthogonalisation and the
// residuals stay FP64.  The FP32 error of sigma (about 1e-7 relative) puts a
// floor of about 1e-7 ||H|| under the residual, below sqrt(tol) for the
// tolerances used here, so FP64 work is only needed near the end: refinement
// points come when the residual is below sqrt(tol), when it has not halved in
// 15 iterations, or after 60 corrections.  There the FP64 sigma of each Ritz
// vector x = B v is built and the subspace sigma vectors are corrected along
// v, S <- S + (sigma64(x) - S v) v^T, together with the projected matrix; the
// Ritz values are then exact Rayleigh quotients and the residuals exact.
// Convergence is tested only at those points, which the iteration log marks
// with precision 0.
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.cuh"

namespace fci {

constexpr int kMaxSub = 32;   // subspace limit (vectors)
constexpr int kDotBlocks = 304;  // 2 x 152 SMs

// partial[b][i] = sum over this block's stripe of X_i . y
template <int MAXM>
__global__ void __launch_bounds__(256) k_multidot(const double *__restrict__ X, int m, const double *__restrict__ y,
                                                  int64_t n, double *__restrict__ partial) {
    double acc[MAXM];
#pragma unroll
    for (int i = 0; i < MAXM; ++i) acc[i] = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += stride) {
        const double yr = y[r];
#pragma unroll
        for (int i = 0; i < MAXM; ++i)
            if (i < m) acc[i] += X[(int64_t)i * n + r] * yr;
    }
    __shared__ double red[MAXM][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < MAXM; ++i) {
        double v = acc[i];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[i][warp] = v;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        double v = 0.0;
        for (int w = 0; w < 8; ++w) v += red[i][w];
        partial[(int64_t)blockIdx.x * MAXM + i] = v;
    }
}

// out[i] = sum_b partial[b][i] (fixed order), optionally written to a matrix slot.
template <int MAXM>
__global__ void k_reduce_partials(const double *__restrict__ partial, int nb, int m, double *__restrict__ out,
                                  int out_stride) {
    int i = threadIdx.x;
    if (i >= m) return;
    double v = 0.0;
    for (int b = 0; b < nb; ++b) v += partial[(int64_t)b * MAXM + i];
    out[(int64_t)i * out_stride] = v;
}

// y[r] = beta*y[r] + sum_i coef[i] X_i[r]
__global__ void k_lincomb(const double *__restrict__ X, int m, const double *__restrict__ coef, int coef_stride,
                          double beta, double *__restrict__ y, int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += stride) {
        double v = beta == 0.0 ? 0.0 : beta * y[r];
        for (int i = 0; i < m; ++i) v += coef[(int64_t)i * coef_stride] * X[(int64_t)i * n + r];
        y[r] = v;
    }
}

// y -= sum_i coef[i] X_i (Gram-Schmidt update with device coefficients)
__global__ void k_sub_proj(const double *__restrict__ X, int m, const double *__restrict__ coef,
                           double *__restrict__ y, int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += stride) {
        double v = y[r];
        for (int i = 0; i < m; ++i) v -= coef[i] * X[(int64_t)i * n + r];
        y[r] = v;
    }
}

// r = hx - e x; t = -r / (d - e) with the denominator floor; partial ||r||^2
__global__ void __launch_bounds__(256) k_residual_precond(const double *__restrict__ x, const double *__restrict__ hx,
                                                          const double *__restrict__ diag, const double *__restrict__ ev,
                                                          int k, double *__restrict__ t, int64_t n,
                                                          double *__restrict__ partial) {
    const double e = ev[k];
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
        double r = hx[i] - e * x[i];
        double d = diag[i] - e;
        if (fabs(d) < 1e-8) d = d < 0 ? -1e-8 : 1e-8;
        t[i] = -r / d;
        acc += r * r;
    }
    __shared__ double red[8];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = 0.0;
        for (int w = 0; w < 8; ++w) v += red[w];
        partial[blockIdx.x] = v;
    }
}

// S_j += V[j][k] * delta for j < m (rank-1 correction of the subspace sigma vectors)
__global__ void k_rank1_sigma(double *__restrict__ S, int m, const double *__restrict__ V, int k,
                              const double *__restrict__ delta, int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += stride) {
        const double d = delta[r];
        for (int j = 0; j < m; ++j) S[(int64_t)j * n + r] += V[j * m + k] * d;
    }
}

// A[i][j] += g[i] * V[j][k]  (projected matrix after the rank-1 correction)
__global__ void k_rank1_proj(double *__restrict__ A, int lda, int m, const double *__restrict__ g,
                             const double *__restrict__ V, int k) {
    for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
        const int i = t / m, j = t % m;
        A[i * lda + j] += g[i] * V[j * m + k];
    }
}

// delta = a - b
__global__ void k_sub(const double *__restrict__ a, const double *__restrict__ b, double *__restrict__ out, int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += stride) out[r] = a[r] - b[r];
}

__global__ void k_scale(double *__restrict__ y, const double *__restrict__ nrm2, double floor_norm,
                        int *__restrict__ keep, int64_t n) {
    const double nn = sqrt(*nrm2);
    const bool ok = nn >= floor_norm;
    if (blockIdx.x == 0 && threadIdx.x == 0) *keep = ok ? 1 : 0;
    if (!ok) return;
    const double s = 1.0 / nn;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) y[i] *= s;
}

// Cyclic Jacobi on the symmetric m x m matrix A (row-major, ld = lda); writes
// ascending eigenvalues to w and eigenvectors (columns) to V[m][m].
__global__ void k_jacobi(const double *__restrict__ A, int lda, int m, double *__restrict__ w, double *__restrict__ V) {
    __shared__ double a[kMaxSub][kMaxSub + 1];
    __shared__ double v[kMaxSub][kMaxSub + 1];
    __shared__ double cs[2];
    __shared__ int order[kMaxSub];
    const int tid = threadIdx.x;
    for (int t = tid; t < m * m; t += blockDim.x) {
        int i = t / m, j = t % m;
        a[i][j] = 0.5 * (A[i * lda + j] + A[j * lda + i]);
        v[i][j] = (i == j) ? 1.0 : 0.0;
    }
    __syncthreads();
    // a rotation is skipped when |a_pq| is negligible next to a_pp and a_qq;
    // the sweeps stop once a whole sweep skipped every pair (60 at most)
    __shared__ int rotated;
    for (int sweep = 0; sweep < 60; ++sweep) {
        if (tid == 0) rotated = 0;
        __syncthreads();
        for (int p = 0; p < m - 1; ++p)
            for (int q = p + 1; q < m; ++q) {
                if (tid == 0) {
                    double apq = a[p][q];
                    double c = 1.0, s = 0.0;
                    if (fabs(apq) > 1e-14 * (fabs(a[p][p]) + fabs(a[q][q]))) {
                        rotated = 1;
                        double theta = (a[q][q] - a[p][p]) / (2.0 * apq);
                        double tt = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                        c = 1.0 / sqrt(tt * tt + 1.0);
                        s = tt * c;
                    }
                    cs[0] = c;
                    cs[1] = s;
                }
                __syncthreads();
                const double c = cs[0], s = cs[1];
                if (s != 0.0) {
                    // rows/cols p and q of a = J^T a J ; v = v J
                    for (int k = tid; k < m; k += blockDim.x) {
                        double akp = a[k][p], akq = a[k][q];
                        a[k][p] = c * akp - s * akq;
                        a[k][q] = s * akp + c * akq;
                    }
                    __syncthreads();
                    for (int k = tid; k < m; k += blockDim.x) {
                        double apk = a[p][k], aqk = a[q][k];
                        a[p][k] = c * apk - s * aqk;
                        a[q][k] = s * apk + c * aqk;
                        double vkp = v[k][p], vkq = v[k][q];
                        v[k][p] = c * vkp - s * vkq;
                        v[k][q] = s * vkp + c * vkq;
                    }
                }
                __syncthreads();
            }
        __syncthreads();
        if (!rotated) break;
    }
    if (tid == 0) {
        for (int i = 0; i < m; ++i) order[i] = i;
        for (int i = 1; i < m; ++i) {  // insertion sort, stable
            int o = order[i];
            int j = i - 1;
            while (j >= 0 && a[order[j]][order[j]] > a[o][o]) {
                order[j + 1] = order[j];
                --j;
            }
            order[j + 1] = o;
        }
    }
    __syncthreads();
    for (int t = tid; t < m; t += blockDim.x) w[t] = a[order[t]][order[t]];
    for (int t = tid; t < m * m; t += blockDim.x) {
        int i = t / m, k = t % m;
        V[i * m + k] = v[i][order[k]];
    }
}

// k smallest diagonal entries, ties broken by index: one pass per root over
// the whole diagonal, excluding indices already chosen.
__global__ void __launch_bounds__(1024) k_argmin_excl(const double *__restrict__ d, int64_t n,
                                                       const int64_t *__restrict__ chosen, int nchosen,
                                                       int64_t *__restrict__ out) {
    double best = INFINITY;
    int64_t bi = INT64_MAX;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        bool skip = false;
        for (int c = 0; c < nchosen; ++c) skip |= (chosen[c] == i);
        if (skip) continue;
        double v = d[i];
        if (v < best || (v == best && i < bi)) { best = v; bi = i; }
    }
    __shared__ double sb[1024];
    __shared__ int64_t si[1024];
    sb[threadIdx.x] = best;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            double v = sb[threadIdx.x + s];
            int64_t j = si[threadIdx.x + s];
            if (v < sb[threadIdx.x] || (v == sb[threadIdx.x] && j < si[threadIdx.x])) {
                sb[threadIdx.x] = v;
                si[threadIdx.x] = j;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = si[0];
}

__global__ void k_set_unit(double *__restrict__ y, int64_t n, const int64_t *__restrict__ idx) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t at = *idx;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) y[i] = (i == at) ? 1.0 : 0.0;
}

__global__ void k_cvt_d2f(const double *__restrict__ a, float *__restrict__ b, int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) b[i] = (float)a[i];
}
__global__ void k_cvt_f2d(const float *__restrict__ a, double *__restrict__ b, int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) b[i] = (double)a[i];
}

// sign fix: make the element of largest magnitude positive
__global__ void __launch_bounds__(1024) k_absmax_sign(const double *__restrict__ x, int64_t n, double *__restrict__ sgn) {
    double best = -1.0, val = 0.0;
    int64_t bi = INT64_MAX;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        double a = fabs(x[i]);
        if (a > best || (a == best && i < bi)) { best = a; bi = i; val = x[i]; }
    }
    __shared__ double sb[1024], sv[1024];
    __shared__ int64_t si[1024];
    sb[threadIdx.x] = best;
    sv[threadIdx.x] = val;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            double v = sb[threadIdx.x + s];
            int64_t j = si[threadIdx.x + s];
            if (v > sb[threadIdx.x] || (v == sb[threadIdx.x] && j < si[threadIdx.x])) {
                sb[threadIdx.x] = v;
                si[threadIdx.x] = j;
                sv[threadIdx.x] = sv[threadIdx.x + s];
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *sgn = sv[0] < 0 ? -1.0 : 1.0;
}

__global__ void k_scale_by(double *__restrict__ y, const double *__restrict__ s, int64_t n) {
    const double f = *s;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) y[i] *= f;
}

namespace {

struct Work {
    fci_ctx *ctx = nullptr;
    cudaStream_t s = nullptr;
    int64_t n = 0;
    int maxsub = 0, nroots = 0;
    double *Bv = nullptr, *Sv = nullptr;   // [maxsub][n]
    double *X = nullptr, *HX = nullptr;     // [nroots][n]
    double *T = nullptr;                    // [nroots][n] corrections
    float *c32 = nullptr, *s32 = nullptr;   // [n] mixed-precision sigma buffers
    double *A = nullptr;                    // [kMaxSub][kMaxSub] projected matrix
    double *w = nullptr, *V = nullptr;      // eigenvalues, eigenvectors
    double *partial = nullptr;              // [kDotBlocks][32]
    double *scal = nullptr;                 // [64] scalars
    double *rn2 = nullptr;                  // [nroots] residual norms squared
    int *keep = nullptr;
    int64_t *idx = nullptr;                 // [nroots]
    int rc = FCI_OK;
    std::vector<void *> allocs;
    std::vector<size_t> sizes;

    template <typename P>
    P *get(size_t count) {
        P *p = (P *)dalloc(ctx, sizeof(P) * count, &rc);
        if (p) {
            allocs.push_back(p);
            sizes.push_back(sizeof(P) * count);
        }
        return p;
    }
    ~Work() {
        for (size_t i = 0; i < allocs.size(); ++i) dfree(ctx, allocs[i], sizes[i]);
    }
};

unsigned grid_for(int64_t n) {
    int64_t g = (n + 255) / 256;
    return (unsigned)(g < 4 * 152 ? (g < 1 ? 1 : g) : 4 * 152);
}

// out[i*stride] = X_i . y for i < m (m <= 32)
int dots(Work &W, const double *X, int m, const double *y, double *out, int stride) {
    if (m <= 0) return FCI_OK;
    if (m <= 8) {
        k_multidot<8><<<kDotBlocks, 256, 0, W.s>>>(X, m, y, W.n, W.partial);
        k_reduce_partials<8><<<1, 32, 0, W.s>>>(W.partial, kDotBlocks, m, out, stride);
    } else if (m <= 32) {
        k_multidot<32><<<kDotBlocks, 256, 0, W.s>>>(X, m, y, W.n, W.partial);
        k_reduce_partials<32><<<1, 32, 0, W.s>>>(W.partial, kDotBlocks, m, out, stride);
    } else {
        return fail(FCI_ERR_ARG, "subspace larger than 32 vectors");
    }
    FCI_CUDA(cudaGetLastError());
    return FCI_OK;
}

int sigma_of(Work &W, bool fp32, const double *x, double *hx) {
    fci_ctx *ctx = W.ctx;
    ctx->sigma_calls++;
    if (!fp32) return launch_sigma(ctx, x, hx, FCI_F64, W.s);
    k_cvt_d2f<<<grid_for(W.n), 256, 0, W.s>>>(x, W.c32, W.n);
    int rc = launch_sigma(ctx, W.c32, W.s32, FCI_F32, W.s);
    if (rc) return rc;
    k_cvt_f2d<<<grid_for(W.n), 256, 0, W.s>>>(W.s32, hx, W.n);
    FCI_CUDA(cudaGetLastError());
    return FCI_OK;
}

// Orthogonalise y against X_0..X_{m-1} twice, normalise; *kept = 1 if kept.
int orthonormalise(Work &W, const double *X, int m, double *y, int *kept) {
    for (int pass = 0; pass < 2; ++pass) {
        if (m > 0) {
            if (int rc = dots(W, X, m, y, W.scal, 1)) return rc;
            k_sub_proj<<<grid_for(W.n), 256, 0, W.s>>>(X, m, W.scal, y, W.n);
            FCI_CUDA(cudaGetLastError());
        }
    }
    if (int rc = dots(W, y, 1, y, W.scal + 40, 1)) return rc;
    k_scale<<<grid_for(W.n), 256, 0, W.s>>>(y, W.scal + 40, 1e-10, W.keep, W.n);
    FCI_CUDA(cudaGetLastError());
    int h = 0;
    FCI_CUDA(cudaMemcpyAsync(&h, W.keep, sizeof(int), cudaMemcpyDeviceToHost, W.s));
    FCI_CUDA(cudaStreamSynchronize(W.s));
    *kept = h;
    return FCI_OK;
}

}  // namespace

int run_davidson(fci_ctx *ctx, int nroots, double tol, double *energies, void *vecs, const void *guess) {
    using clk = std::chrono::steady_clock;
    const auto t0 = clk::now();
    FCI_CUDA(cudaDeviceSynchronize());  // caller's guess buffer is complete
    Work W;
    W.ctx = ctx;
    W.s = ctx->stream;
    W.n = ctx->ndet;
    W.nroots = nroots;
    int maxsub = ctx->opt.max_subspace;
    if (maxsub > 32) maxsub = 32;
    if (maxsub < 2 * nroots) maxsub = 2 * nroots;
    if (maxsub > W.n) maxsub = (int)W.n;
    W.maxsub = maxsub;
    const bool mixed = ctx->opt.precision == FCI_PREC_MIXED;
    W.Bv = W.get<double>((size_t)maxsub * W.n);
    W.Sv = W.get<double>((size_t)maxsub * W.n);
    // thick restart: a collapse keeps up to `keepn` Ritz vectors (at least nroots)
    const int keepn = std::max(nroots, std::min(8, maxsub / 2));
    W.X = W.get<double>((size_t)keepn * W.n);
    W.HX = W.get<double>((size_t)keepn * W.n);
    W.T = W.get<double>((size_t)nroots * W.n);
    if (mixed) {
        W.c32 = W.get<float>(W.n);
        W.s32 = W.get<float>(W.n);
    }
    W.A = W.get<double>(kMaxSub * kMaxSub);
    W.w = W.get<double>(kMaxSub);
    W.V = W.get<double>(kMaxSub * kMaxSub);
    W.partial = W.get<double>(kDotBlocks * 32);
    W.scal = W.get<double>(64);
    W.rn2 = W.get<double>(8);
    W.keep = W.get<int>(1);
    W.idx = W.get<int64_t>(8);
    if (W.rc) return W.rc;
    const int64_t n = W.n;
    cudaStream_t s = W.s;

    ctx->log.clear();
    ctx->log_width = nroots + 3;
    ctx->iterations = 0;
    ctx->sigma_calls = 0;

    // (1) initial subspace
    int m = 0;
    for (int k = 0; k < nroots; ++k) {
        double *b = W.Bv + (size_t)m * n;
        if (guess) {
            FCI_CUDA(cudaMemcpyAsync(b, (const double *)guess + (size_t)k * n, sizeof(double) * n,
                                     cudaMemcpyDeviceToDevice, s));
        } else {
            k_argmin_excl<<<1, 1024, 0, s>>>(ctx->hdiag, n, W.idx, k, W.idx + k);
            k_set_unit<<<grid_for(n), 256, 0, s>>>(b, n, W.idx + k);
            FCI_CUDA(cudaGetLastError());
        }
        int kept = 0;
        if (int rc = orthonormalise(W, W.Bv, m, b, &kept)) return rc;
        if (kept) ++m;
    }
    if (m == 0) return fail(FCI_ERR_ARG, "initial guess vectors are linearly dependent");
    for (int i = 0; i < m; ++i)
        if (int rc = sigma_of(W, mixed, W.Bv + (size_t)i * n, W.Sv + (size_t)i * n)) return rc;
    for (int j = 0; j < m; ++j)
        if (int rc = dots(W, W.Bv, m, W.Sv + (size_t)j * n, W.A + j, kMaxSub)) return rc;

    // exact: the subspace sigma vectors are FP64-exact along the current Ritz
    // vectors, so Ritz values and residuals are exact; convergence is only
    // tested there.  Always true in FP64 mode.
    bool exact = !mixed;
    std::vector<double> e_prev(nroots, INFINITY), ev(kMaxSub), rn(nroots);
    bool converged = false;
    int it = 0, inner = 0;
    double r_ref = INFINITY, r_win = INFINITY;
    std::vector<double> r_hist;
    (void)r_ref;

    for (it = 1; it <= ctx->opt.max_iter; ++it) {
        // (4) diagonalise the projected matrix
        k_jacobi<<<1, 64, 0, s>>>(W.A, kMaxSub, m, W.w, W.V);
        FCI_CUDA(cudaGetLastError());
        const int nr = nroots < m ? nroots : m;
        // Ritz vectors, their sigma, residuals and (2)-(3) preconditioned corrections
        for (int k = 0; k < nr; ++k) {
            k_lincomb<<<grid_for(n), 256, 0, s>>>(W.Bv, m, W.V + k, m, 0.0, W.X + (size_t)k * n, n);
            k_lincomb<<<grid_for(n), 256, 0, s>>>(W.Sv, m, W.V + k, m, 0.0, W.HX + (size_t)k * n, n);
            k_residual_precond<<<kDotBlocks, 256, 0, s>>>(W.X + (size_t)k * n, W.HX + (size_t)k * n, ctx->hdiag, W.w,
                                                          k, W.T + (size_t)k * n, n, W.partial);
            k_reduce_partials<1><<<1, 32, 0, s>>>(W.partial, kDotBlocks, 1, W.rn2 + k, 1);
            FCI_CUDA(cudaGetLastError());
        }
        FCI_CUDA(cudaMemcpyAsync(ev.data(), W.w, sizeof(double) * nr, cudaMemcpyDeviceToHost, s));
        FCI_CUDA(cudaMemcpyAsync(rn.data(), W.rn2, sizeof(double) * nr, cudaMemcpyDeviceToHost, s));
        int derr = 0;
        FCI_CUDA(cudaMemcpyAsync(&derr, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
        FCI_CUDA(cudaStreamSynchronize(s));
        if (derr) return fail(FCI_ERR_TIMEOUT, "a bounded device wait gave up inside sigma");
        double rmax = 0.0, demax = 0.0;
        for (int k = 0; k < nr; ++k) {
            rn[k] = std::sqrt(rn[k]);
            rmax = std::max(rmax, rn[k]);
            demax = std::max(demax, std::fabs(ev[k] - e_prev[k]));
        }
        {
            const double el = std::chrono::duration<double>(clk::now() - t0).count();
            ctx->log.push_back((double)it);
            ctx->log.push_back(exact ? 0.0 : 1.0);
            ctx->log.push_back(el);
            for (int k = 0; k < nroots; ++k) ctx->log.push_back(k < nr ? ev[k] : NAN);
        }
        // residual 15 iterations ago (stagnation test of the FP32 phase)
        r_hist.push_back(rmax);
        r_win = r_hist.size() > 15 ? r_hist[r_hist.size() - 16] : INFINITY;
        if (exact) {
            if (nr == nroots && demax < tol && rmax < std::sqrt(tol)) {
                converged = true;
                break;
            }
            for (int k = 0; k < nr; ++k) e_prev[k] = ev[k];
            r_ref = rmax;
            inner = 0;
        } else if (++inner >= 60 || rmax < std::sqrt(tol) || (inner >= 15 && rmax > 0.5 * r_win)) {
            // refinement: exact FP64 sigma of each Ritz vector; the difference to
            // the subspace estimate corrects every sigma vector along that Ritz
            // direction (S += delta v^T) and the projected matrix with it
            for (int k = 0; k < nr; ++k) {
                double *d = W.T + (size_t)k * n;
                if (int rc = sigma_of(W, false, W.X + (size_t)k * n, d)) return rc;
                k_sub<<<grid_for(n), 256, 0, s>>>(d, W.HX + (size_t)k * n, d, n);
                if (int rc = dots(W, W.Bv, m, d, W.scal, 1)) return rc;
                k_rank1_sigma<<<grid_for(n), 256, 0, s>>>(W.Sv, m, W.V, k, d, n);
                k_rank1_proj<<<1, 256, 0, s>>>(W.A, kMaxSub, m, W.scal, W.V, k);
                FCI_CUDA(cudaGetLastError());
            }
            exact = true;
            continue;
        }
        if (m + nr > maxsub) {
            // thick restart: collapse onto the lowest `keep` Ritz vectors (orthonormal
            // to rounding) and their sigma
            const int keep = std::min(keepn, m);
            for (int k = nr; k < keep; ++k) {
                k_lincomb<<<grid_for(n), 256, 0, s>>>(W.Bv, m, W.V + k, m, 0.0, W.X + (size_t)k * n, n);
                k_lincomb<<<grid_for(n), 256, 0, s>>>(W.Sv, m, W.V + k, m, 0.0, W.HX + (size_t)k * n, n);
            }
            FCI_CUDA(cudaGetLastError());
            FCI_CUDA(cudaMemcpyAsync(W.Bv, W.X, sizeof(double) * keep * n, cudaMemcpyDeviceToDevice, s));
            FCI_CUDA(cudaMemcpyAsync(W.Sv, W.HX, sizeof(double) * keep * n, cudaMemcpyDeviceToDevice, s));
            if (mixed && keep > nr) exact = false;  // the extra vectors carry FP32 sigma
            m = keep;
            FCI_CUDA(cudaMemsetAsync(W.A, 0, sizeof(double) * kMaxSub * kMaxSub, s));
            for (int j = 0; j < m; ++j)
                if (int rc = dots(W, W.Bv, m, W.Sv + (size_t)j * n, W.A + j, kMaxSub)) return rc;
        }
        int added = 0;
        for (int k = 0; k < nr && m < maxsub; ++k) {
            double *b = W.Bv + (size_t)m * n;
            FCI_CUDA(cudaMemcpyAsync(b, W.T + (size_t)k * n, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
            int kept = 0;
            if (int rc = orthonormalise(W, W.Bv, m, b, &kept)) return rc;
            if (!kept) continue;
            // (4) new sigma (FP32 in mixed mode), new row/column of the projected matrix
            if (int rc = sigma_of(W, mixed, b, W.Sv + (size_t)m * n)) return rc;
            ++m;
            if (int rc = dots(W, W.Bv, m, W.Sv + (size_t)(m - 1) * n, W.A + (m - 1), kMaxSub)) return rc;
            if (int rc = dots(W, W.Sv, m, W.Bv + (size_t)(m - 1) * n, W.A + (size_t)(m - 1) * kMaxSub, 1)) return rc;
            ++added;
        }
        if (added == 0) {
            if (!exact) {
                inner = 1 << 20;  // force a refinement on the next pass
                continue;
            }
            converged = rmax < std::sqrt(tol);
            break;
        }
        if (mixed) exact = false;
    }
    ctx->iterations = it > ctx->opt.max_iter ? ctx->opt.max_iter : it;
    for (int k = 0; k < nroots; ++k) energies[k] = ev[k];
    if (vecs) {
        for (int k = 0; k < nroots; ++k) {
            double *dst = (double *)vecs + (size_t)k * n;
            k_absmax_sign<<<1, 1024, 0, s>>>(W.X + (size_t)k * n, n, W.scal + 50);
            k_scale_by<<<grid_for(n), 256, 0, s>>>(W.X + (size_t)k * n, W.scal + 50, n);
            FCI_CUDA(cudaMemcpyAsync(dst, W.X + (size_t)k * n, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        }
    }
    FCI_CUDA(cudaStreamSynchronize(s));
    if (!converged) return fail(FCI_ERR_NOCONV, "Davidson did not converge within max_iter");
    return FCI_OK;
}

}  // namespace fci
