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
// Gram-Schmidt (a second pass when the first removed more than half of the
// squared norm), corrections with norm < 1e-10 dropped,
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
// with precision 0.  When a refinement point finds the FP32 sigma error along a
// Ritz vector above sqrt(tol)/2 and the residual has stopped halving between
// exact points (the FP32 phase cannot reach the required residual), the
// subspace collapses onto the Ritz vectors with fresh FP64 sigma and the
// remaining corrections get FP64 sigma.
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.cuh"

namespace fci {

constexpr int kMaxSub = 32;   // subspace limit (vectors)
constexpr int kDotBlocks = 304;  // 2 x 152 SMs

// partial[b][g*8 + j] = sum over stripe b of X_{g*8+j} . y, j < 8.  The
// vectors are split into groups of 8 (blockIdx.x % groups) so that each
// thread keeps 8 accumulators and many blocks fit on an SM; the groups of one
// stripe run side by side and share y through L2.  On GB300 these products are
// bound by the FP64 pipe (about 1.2 TFLOP/s against 2 FLOP per 8-byte element),
// so each element costs exactly one FMA (a single chain per accumulator).
// VEC = 4 reads 32-byte vectors (n % 4 == 0, 32-byte aligned rows).
template <int VEC>
__global__ void __launch_bounds__(256) k_multidot(const double *__restrict__ X, int m, const double *__restrict__ y,
                                                  int64_t n, int groups, double *__restrict__ partial) {
    const int g = blockIdx.x % groups;
    const int stripe = blockIdx.x / groups;
    const int nstripes = gridDim.x / groups;
    const int i0 = g * 8;
    const int mg = m - i0 < 8 ? m - i0 : 8;
    double acc[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j] = 0.0;
    const int64_t stride = (int64_t)nstripes * blockDim.x;
    if (VEC == 4) {
        const int64_t n4 = n / 4;
        const double4_32a *y4 = reinterpret_cast<const double4_32a *>(y);
        for (int64_t r = stripe * (int64_t)blockDim.x + threadIdx.x; r < n4; r += stride) {
            const double4_32a yr = y4[r];
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (j < mg) {
                    const double4_32a x = reinterpret_cast<const double4_32a *>(X + (int64_t)(i0 + j) * n)[r];
                    double a = acc[j];
                    a = fma(x.x, yr.x, a);
                    a = fma(x.y, yr.y, a);
                    a = fma(x.z, yr.z, a);
                    a = fma(x.w, yr.w, a);
                    acc[j] = a;
                }
        }
    } else {
        for (int64_t r = stripe * (int64_t)blockDim.x + threadIdx.x; r < n; r += stride) {
            const double yr = y[r];
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (j < mg) acc[j] = fma(X[(int64_t)(i0 + j) * n + r], yr, acc[j]);
        }
    }
    __shared__ double red[8][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        double v = acc[j];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[j][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < mg) {
        double v = 0.0;
        for (int w = 0; w < 8; ++w) v += red[threadIdx.x][w];
        partial[(int64_t)stripe * 32 + i0 + threadIdx.x] = v;
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

// y[r] = beta*y[r] + sum_i coef[i] X_i[r]; pairs of elements per thread
// (double2) when n is even and the rows are 16-byte aligned.
template <int VEC>
__global__ void k_lincomb(const double *__restrict__ X, int m, const double *__restrict__ coef, int coef_stride,
                          double beta, double *__restrict__ y, int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (VEC == 2) {
        const int64_t n2 = n / 2;
        for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n2; r += stride) {
            double2 v = make_double2(0.0, 0.0);
            if (beta != 0.0) {
                const double2 y0 = reinterpret_cast<const double2 *>(y)[r];
                v.x = beta * y0.x;
                v.y = beta * y0.y;
            }
#pragma unroll 8
            for (int i = 0; i < m; ++i) {
                const double c = coef[(int64_t)i * coef_stride];
                const double2 x = reinterpret_cast<const double2 *>(X + (int64_t)i * n)[r];
                v.x += c * x.x;
                v.y += c * x.y;
            }
            reinterpret_cast<double2 *>(y)[r] = v;
        }
    } else {
        for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += stride) {
            double v = beta == 0.0 ? 0.0 : beta * y[r];
#pragma unroll 8
            for (int i = 0; i < m; ++i) v += coef[(int64_t)i * coef_stride] * X[(int64_t)i * n + r];
            y[r] = v;
        }
    }
}

// y -= sum_i coef[i] X_i (Gram-Schmidt update with device coefficients);
// partial[block] = this block's share of ||y||^2 after the update.
template <int VEC>
__global__ void __launch_bounds__(256) k_sub_proj(const double *__restrict__ X, int m, const double *__restrict__ coef,
                                                  double *__restrict__ y, int64_t n, double *__restrict__ partial) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    double nrm = 0.0;
    if (VEC == 2) {
        const int64_t n2 = n / 2;
        for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n2; r += stride) {
            double2 v = reinterpret_cast<const double2 *>(y)[r];
#pragma unroll 8
            for (int i = 0; i < m; ++i) {
                const double c = coef[i];
                const double2 x = reinterpret_cast<const double2 *>(X + (int64_t)i * n)[r];
                v.x = fma(-c, x.x, v.x);
                v.y = fma(-c, x.y, v.y);
            }
            reinterpret_cast<double2 *>(y)[r] = v;
            nrm = fma(v.x, v.x, nrm);
            nrm = fma(v.y, v.y, nrm);
        }
    } else {
        for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += stride) {
            double v = y[r];
#pragma unroll 8
            for (int i = 0; i < m; ++i) v = fma(-coef[i], X[(int64_t)i * n + r], v);
            y[r] = v;
            nrm = fma(v, v, nrm);
        }
    }
    __shared__ double red[8];
    for (int o = 16; o > 0; o >>= 1) nrm += __shfl_down_sync(0xffffffffu, nrm, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = nrm;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = 0.0;
        for (int w = 0; w < 8; ++w) v += red[w];
        partial[blockIdx.x] = v;
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
    __shared__ int order[kMaxSub];
    const int tid = threadIdx.x;
    for (int t = tid; t < m * m; t += blockDim.x) {
        int i = t / m, j = t % m;
        a[i][j] = 0.5 * (A[i * lda + j] + A[j * lda + i]);
        v[i][j] = (i == j) ? 1.0 : 0.0;
    }
    __syncthreads();
    // Parallel cyclic Jacobi with round-robin pair ordering: each step rotates
    // m/2 disjoint pairs at once (rotations on disjoint index pairs commute).
    // A rotation is skipped when |a_pq| < 1e-14 (|a_pp| + |a_qq|); the sweeps
    // stop after a sweep without rotation (60 at most).
    __shared__ int rotated;
    __shared__ int pos[kMaxSub + 1];
    __shared__ int pp[kMaxSub / 2 + 1], pq[kMaxSub / 2 + 1];
    __shared__ double pc[kMaxSub / 2 + 1], psn[kMaxSub / 2 + 1];
    const int me = m + (m & 1);  // even number of players; index m is a dummy when m is odd
    const int half = me / 2;
    for (int t = tid; t < me; t += blockDim.x) pos[t] = t;
    __syncthreads();
    for (int sweep = 0; sweep < 60; ++sweep) {
        if (tid == 0) rotated = 0;
        __syncthreads();
        for (int step = 0; step < me - 1; ++step) {
            for (int k = tid; k < half; k += blockDim.x) {
                int p = pos[k], q = pos[me - 1 - k];
                if (p > q) { const int t2 = p; p = q; q = t2; }
                double c = 1.0, sn = 0.0;
                if (q < m) {
                    const double apq = a[p][q];
                    if (fabs(apq) > 1e-14 * (fabs(a[p][p]) + fabs(a[q][q]))) {
                        rotated = 1;
                        const double theta = (a[q][q] - a[p][p]) / (2.0 * apq);
                        const double tt = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                        c = 1.0 / sqrt(tt * tt + 1.0);
                        sn = tt * c;
                    }
                }
                pp[k] = p;
                pq[k] = q;
                pc[k] = c;
                psn[k] = sn;
            }
            __syncthreads();
            // columns: a <- a J
            for (int t = tid; t < half * m; t += blockDim.x) {
                const int k = t / m, r = t % m;
                if (psn[k] == 0.0) continue;
                const int p = pp[k], q = pq[k];
                const double c = pc[k], sn = psn[k];
                const double arp = a[r][p], arq = a[r][q];
                a[r][p] = c * arp - sn * arq;
                a[r][q] = sn * arp + c * arq;
            }
            __syncthreads();
            // rows: a <- J^T a ; eigenvectors v <- v J
            for (int t = tid; t < half * m; t += blockDim.x) {
                const int k = t / m, r = t % m;
                if (psn[k] == 0.0) continue;
                const int p = pp[k], q = pq[k];
                const double c = pc[k], sn = psn[k];
                const double apr = a[p][r], aqr = a[q][r];
                a[p][r] = c * apr - sn * aqr;
                a[q][r] = sn * apr + c * aqr;
                const double vrp = v[r][p], vrq = v[r][q];
                v[r][p] = c * vrp - sn * vrq;
                v[r][q] = sn * vrp + c * vrq;
            }
            __syncthreads();
            // next round-robin pairing: player 0 stays, the others rotate
            if (tid == 0) {
                const int last = pos[me - 1];
                for (int t = me - 1; t > 1; --t) pos[t] = pos[t - 1];
                pos[1] = last;
            }
            __syncthreads();
        }
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
// the whole diagonal, excluding indices already chosen.  Two stages: each
// block reduces a grid-strided share into (pv, pi)[block], then one block
// reduces those (the order of (value, index) is total, so the result does not
// depend on the split).
__device__ __forceinline__ bool less_vi(double v, int64_t i, double bv, int64_t bi) {
    return v < bv || (v == bv && i < bi);
}

template <int NT>
__device__ void block_min_vi(double &best, int64_t &bi, double *sb, int64_t *si) {
    sb[threadIdx.x] = best;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int s = NT / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s && less_vi(sb[threadIdx.x + s], si[threadIdx.x + s], sb[threadIdx.x], si[threadIdx.x])) {
            sb[threadIdx.x] = sb[threadIdx.x + s];
            si[threadIdx.x] = si[threadIdx.x + s];
        }
        __syncthreads();
    }
    best = sb[0];
    bi = si[0];
}

// par != 0 (spin parity, a square [ncols][ncols] vector) restricts the
// candidates to one determinant per pair (I_a, I_b), (I_b, I_a): I_a >= I_b, and
// I_a > I_b for par < 0 (the diagonal ones have no antisymmetric combination).
__global__ void __launch_bounds__(256) k_argmin_excl_part(const double *__restrict__ d, int64_t n,
                                                          const int64_t *__restrict__ chosen, int nchosen,
                                                          double *__restrict__ pv, int64_t *__restrict__ pi,
                                                          int64_t ncols, int par) {
    double best = INFINITY;
    int64_t bi = INT64_MAX;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
        if (par != 0) {
            const int64_t r = i / ncols, c = i % ncols;
            if (r < c || (par < 0 && r == c)) continue;
        }
        bool skip = false;
        for (int c = 0; c < nchosen; ++c) skip |= (chosen[c] == i);
        if (skip) continue;
        const double v = d[i];
        if (less_vi(v, i, best, bi)) {
            best = v;
            bi = i;
        }
    }
    __shared__ double sb[256];
    __shared__ int64_t si[256];
    block_min_vi<256>(best, bi, sb, si);
    if (threadIdx.x == 0) {
        pv[blockIdx.x] = best;
        pi[blockIdx.x] = bi;
    }
}

// out = index of the smallest (pv, pi) pair (one block of 256 threads)
__global__ void __launch_bounds__(256) k_argmin_final(const double *__restrict__ pv, const int64_t *__restrict__ pi,
                                                      int nb, int64_t *__restrict__ out) {
    double best = INFINITY;
    int64_t bi = INT64_MAX;
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
        if (less_vi(pv[b], pi[b], best, bi)) {
            best = pv[b];
            bi = pi[b];
        }
    __shared__ double sb[256];
    __shared__ int64_t si[256];
    block_min_vi<256>(best, bi, sb, si);
    if (threadIdx.x == 0) *out = bi;
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

// sign fix: make the element of largest magnitude positive (ties: lower index).
// Stage 1 per block (the key -|x_i| with index i, so the minimum is wanted);
// stage 2 takes the sign of the winner.
__global__ void __launch_bounds__(256) k_absmax_part(const double *__restrict__ x, int64_t n, double *__restrict__ pv,
                                                     int64_t *__restrict__ pi) {
    double best = INFINITY;
    int64_t bi = INT64_MAX;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
        const double v = -fabs(x[i]);
        if (less_vi(v, i, best, bi)) {
            best = v;
            bi = i;
        }
    }
    __shared__ double sb[256];
    __shared__ int64_t si[256];
    block_min_vi<256>(best, bi, sb, si);
    if (threadIdx.x == 0) {
        pv[blockIdx.x] = best;
        pi[blockIdx.x] = bi;
    }
}

__global__ void k_sign_of(const double *__restrict__ x, const int64_t *__restrict__ at, double *__restrict__ sgn) {
    *sgn = x[*at] < 0 ? -1.0 : 1.0;
}

// *q = *a / *b
__global__ void k_quotient(const double *__restrict__ a, const double *__restrict__ b, double *__restrict__ q) {
    *q = *a / *b;
}

__global__ void k_scale_by(double *__restrict__ y, const double *__restrict__ s, int64_t n) {
    const double f = *s;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) y[i] *= f;
}

// ---- FP32 basis (large spaces): the basis vectors and their sigma vectors
// are stored in FP32, the Ritz vectors and their sigma in FP64 ----

// a b added exactly to the double-float pair (sh, sl): error-free product by
// FMA, TwoSum of the leading parts (GB300 issues FP32 64 times faster than FP64)
__device__ __forceinline__ void df_acc(float a, float b, float &sh, float &sl) {
    const float p = a * b;
    const float e = fmaf(a, b, -p);
    const float t = sh + p;
    const float bp = t - sh;
    sl += ((sh - (t - bp)) + (p - bp)) + e;
    sh = t;
}

// partial[stripe][32] = this stripe's share of X_i . y for FP32 X [m][n] and
// y [n]: double-float sums per thread, FP64 across threads (layout as k_multidot)
__global__ void __launch_bounds__(256) k_multidot_f32(const float *__restrict__ X, int m, const float *__restrict__ y,
                                                      int64_t n, int groups, double *__restrict__ partial) {
    const int g = blockIdx.x % groups;
    const int stripe = blockIdx.x / groups;
    const int nstripes = gridDim.x / groups;
    const int i0 = g * 8;
    const int mg = m - i0 < 8 ? m - i0 : 8;
    float sh[8], sl[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) sh[j] = sl[j] = 0.f;
    const int64_t stride = (int64_t)nstripes * blockDim.x;
    for (int64_t r = stripe * (int64_t)blockDim.x + threadIdx.x; r < n; r += stride) {
        const float yr = y[r];
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (j < mg) df_acc(X[(int64_t)(i0 + j) * n + r], yr, sh[j], sl[j]);
    }
    __shared__ double red[8][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        double v = (double)sh[j] + (double)sl[j];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[j][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < mg) {
        double v = 0.0;
        for (int w = 0; w < 8; ++w) v += red[threadIdx.x][w];
        partial[(int64_t)stripe * 32 + i0 + threadIdx.x] = v;
    }
}

// y = sum_i coef[i coef_stride] X_i (FP32 X, FP64 y and sums)
__global__ void k_lincomb_f32(const float *__restrict__ X, int m, const double *__restrict__ coef, int coef_stride,
                              double *__restrict__ y, int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += stride) {
        double v = 0.0;
        for (int i = 0; i < m; ++i) v = fma(coef[(int64_t)i * coef_stride], (double)X[(int64_t)i * n + r], v);
        y[r] = v;
    }
}

// y -= sum_i coef[i] X_i in FP32 (Gram-Schmidt on the FP32 basis); partial[block]
// = the block's share of ||y||^2 after the update
__global__ void __launch_bounds__(256) k_sub_proj_f32(const float *__restrict__ X, int m, const double *__restrict__ coef,
                                                      float *__restrict__ y, int64_t n, double *__restrict__ partial) {
    __shared__ float c[32];
    if (threadIdx.x < m) c[threadIdx.x] = (float)coef[threadIdx.x];
    __syncthreads();
    float sh = 0.f, sl = 0.f;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += stride) {
        float v = y[r];
        for (int i = 0; i < m; ++i) v = fmaf(-c[i], X[(int64_t)i * n + r], v);
        y[r] = v;
        df_acc(v, v, sh, sl);
    }
    double acc = (double)sh + (double)sl;
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

__global__ void k_scale_f32(float *__restrict__ y, const double *__restrict__ nrm2, double floor_norm,
                            int *__restrict__ keep, int64_t n) {
    const double nn = sqrt(*nrm2);
    const bool ok = nn >= floor_norm;
    if (blockIdx.x == 0 && threadIdx.x == 0) *keep = ok ? 1 : 0;
    if (!ok) return;
    const float sc = (float)(1.0 / nn);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) y[i] *= sc;
}

// X_k <- sum_i V[i][k] X_i for k < keep, in place (every element's m values
// are read before any is written; m <= 32, keep <= 8)
__global__ void __launch_bounds__(256) k_collapse_f32(float *__restrict__ X, int m, const double *__restrict__ V,
                                                      int keep, int64_t n) {
    __shared__ float c[32][8];
    for (int t = threadIdx.x; t < 32 * 8; t += blockDim.x) {
        const int i = t / 8, k = t % 8;
        c[i][k] = (i < m && k < keep) ? (float)V[i * m + k] : 0.f;
    }
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += stride) {
        float b[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) b[i] = i < m ? X[(int64_t)i * n + r] : 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (k >= keep) break;
            float a = 0.f;
#pragma unroll
            for (int i = 0; i < 32; ++i) a = fmaf(c[i][k], b[i], a);
            X[(int64_t)k * n + r] = a;
        }
    }
}

__global__ void k_set_unit_f32(float *__restrict__ y, int64_t n, const int64_t *__restrict__ idx) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t at = *idx;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) y[i] = (i == at) ? 1.f : 0.f;
}

// partial[block] = share of ||hx - e x||^2 (e = ev[k])
__global__ void __launch_bounds__(256) k_resnorm(const double *__restrict__ x, const double *__restrict__ hx,
                                                 const double *__restrict__ ev, int k, int64_t n,
                                                 double *__restrict__ partial) {
    const double e = ev[k];
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
        const double r = hx[i] - e * x[i];
        acc = fma(r, r, acc);
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

// t = -(hx - e x) / (d - e) with the denominator floor, stored in FP32
__global__ void k_precond_f32(const double *__restrict__ x, const double *__restrict__ hx,
                              const double *__restrict__ diag, const double *__restrict__ ev, int k,
                              float *__restrict__ t, int64_t n) {
    const double e = ev[k];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
        double d = diag[i] - e;
        if (fabs(d) < 1e-8) d = d < 0 ? -1e-8 : 1e-8;
        t[i] = (float)(-(hx[i] - e * x[i]) / d);
    }
}

// delta = hx - sum_i V[i][k] S_i (the FP64 sigma of a Ritz vector less the
// subspace estimate), stored in FP32
__global__ void k_sigma_delta_f32(const double *__restrict__ hx, const float *__restrict__ S, int m,
                                  const double *__restrict__ V, int k, float *__restrict__ delta, int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += stride) {
        double v = hx[r];
        for (int i = 0; i < m; ++i) v = fma(-V[i * m + k], (double)S[(int64_t)i * n + r], v);
        delta[r] = (float)v;
    }
}

// S_j += V[j][k] delta for j < m (FP32 storage)
__global__ void k_rank1_sigma_f32(float *__restrict__ S, int m, const double *__restrict__ V, int k,
                                  const float *__restrict__ delta, int64_t n) {
    __shared__ float c[32];
    if (threadIdx.x < m) c[threadIdx.x] = (float)V[threadIdx.x * m + k];
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += stride) {
        const float d = delta[r];
        for (int j = 0; j < m; ++j) S[(int64_t)j * n + r] = fmaf(c[j], d, S[(int64_t)j * n + r]);
    }
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
    float *Bf = nullptr, *Sf = nullptr;     // FP32 basis: [maxsub][n] vectors and their sigma
    float *y32 = nullptr;                   // FP32 basis: [n] scratch
    double *A = nullptr;                    // [kMaxSub][kMaxSub] projected matrix
    double *w = nullptr, *V = nullptr;      // eigenvalues, eigenvectors
    double *partial = nullptr;              // [kDotBlocks][32]
    double *scal = nullptr;                 // [64] scalars
    double *rn2 = nullptr;                  // [nroots] residual norms squared
    int *keep = nullptr;
    int64_t *idx = nullptr;                 // [nroots]
    int64_t *pidx = nullptr;                // [kDotBlocks + 1] reduction scratch (indices)
    int parity = 0;                         // fci_options.spin_parity (C^T = parity C), 0 = none
    int rc = FCI_OK;
    std::vector<void *> allocs;
    std::vector<size_t> sizes;

    // The bookkeeping slots are made before the device allocation, so a host
    // allocation failure (bad_alloc) can never leave a device buffer unrecorded.
    template <typename P>
    P *get(size_t count) {
        allocs.push_back(nullptr);
        sizes.push_back(0);
        P *p = (P *)dalloc(ctx, sizeof(P) * count, &rc);
        allocs.back() = p;
        sizes.back() = p ? sizeof(P) * count : 0;
        return p;
    }
    ~Work() {
        for (size_t i = 0; i < allocs.size() && i < sizes.size(); ++i) dfree(ctx, allocs[i], sizes[i]);
    }
};

unsigned grid_for(int64_t n) {
    int64_t g = (n + 255) / 256;
    return (unsigned)(g < 4 * 152 ? (g < 1 ? 1 : g) : 4 * 152);
}

// W.idx[k] = index of the smallest diagonal entry not among W.idx[0..k)
void argmin_excl(Work &W, const double *d, int k) {
    k_argmin_excl_part<<<kDotBlocks, 256, 0, W.s>>>(d, W.n, W.idx, k, W.partial, W.pidx, W.ctx->B.ns, W.parity);
    k_argmin_final<<<1, 256, 0, W.s>>>(W.partial, W.pidx, kDotBlocks, W.idx + k);
}

// *sgn = the sign of the element of x of largest magnitude (lowest index on ties)
void sign_of_absmax(Work &W, const double *x, double *sgn) {
    k_absmax_part<<<kDotBlocks, 256, 0, W.s>>>(x, W.n, W.partial, W.pidx);
    k_argmin_final<<<1, 256, 0, W.s>>>(W.partial, W.pidx, kDotBlocks, W.pidx + kDotBlocks);
    k_sign_of<<<1, 1, 0, W.s>>>(x, W.pidx + kDotBlocks, sgn);
}

bool vec2(int64_t n, const void *a, const void *b) {
    return n % 2 == 0 && (uintptr_t)a % 16 == 0 && (uintptr_t)b % 16 == 0;
}

// y = beta*y + sum_i coef[i*coef_stride] X_i
void lincomb(cudaStream_t s, const double *X, int m, const double *coef, int coef_stride, double beta, double *y,
             int64_t n) {
    if (vec2(n, X, y))
        k_lincomb<2><<<grid_for(n / 2), 256, 0, s>>>(X, m, coef, coef_stride, beta, y, n);
    else
        k_lincomb<1><<<grid_for(n), 256, 0, s>>>(X, m, coef, coef_stride, beta, y, n);
}

// out[i*stride] = X_i . y for i < m (m <= 32)
int dots(Work &W, const double *X, int m, const double *y, double *out, int stride) {
    if (m <= 0) return FCI_OK;
    if (m > 32) return fail(FCI_ERR_ARG, "subspace larger than 32 vectors");
    const int groups = (m + 7) / 8;
    const bool vec = (W.n % 4 == 0) && ((uintptr_t)X % 32 == 0) && ((uintptr_t)y % 32 == 0);
    if (vec)
        k_multidot<4><<<kDotBlocks * groups, 256, 0, W.s>>>(X, m, y, W.n, groups, W.partial);
    else
        k_multidot<1><<<kDotBlocks * groups, 256, 0, W.s>>>(X, m, y, W.n, groups, W.partial);
    k_reduce_partials<32><<<1, 32, 0, W.s>>>(W.partial, kDotBlocks, m, out, stride);
    FCI_CUDA(cudaGetLastError());
    return FCI_OK;
}

// project y onto the spin parity (y <- (y + p y^T) / 2), if one is set
int project_parity(Work &W, void *y, int elem) {
    if (W.parity == 0) return FCI_OK;
    return sym_pairs(y, W.ctx->A.ns, elem, W.parity, 1, W.s);
}

int sigma_of(Work &W, bool fp32, const double *x, double *hx) {
    fci_ctx *ctx = W.ctx;
    ctx->sigma_calls++;
    if (!fp32) return launch_sigma(ctx, x, hx, FCI_F64, W.s, W.parity);
    k_cvt_d2f<<<grid_for(W.n), 256, 0, W.s>>>(x, W.c32, W.n);
    int rc = launch_sigma(ctx, W.c32, W.s32, FCI_F32, W.s, W.parity);
    if (rc) return rc;
    k_cvt_f2d<<<grid_for(W.n), 256, 0, W.s>>>(W.s32, hx, W.n);
    FCI_CUDA(cudaGetLastError());
    return FCI_OK;
}

// Orthogonalise y against X_0..X_{m-1} (a second pass when needed), normalise; *kept = 1 if kept.
int orthonormalise(Work &W, const double *X, int m, double *y, int *kept) {
    if (m > 0) {
        const bool v2 = vec2(W.n, X, y);
        const unsigned grid = v2 ? grid_for(W.n / 2) : grid_for(W.n);
        // classical Gram-Schmidt, repeated only when the first pass removed more
        // than half of ||y||^2 (DGKS criterion, ||y1|| < ||y0||/sqrt(2)); against
        // an orthonormal basis ||y0||^2 = ||y1||^2 + sum_i c_i^2
        for (int pass = 0; pass < 2; ++pass) {
            if (int rc = dots(W, X, m, y, W.scal, 1)) return rc;
            if (v2)
                k_sub_proj<2><<<grid, 256, 0, W.s>>>(X, m, W.scal, y, W.n, W.partial);
            else
                k_sub_proj<1><<<grid, 256, 0, W.s>>>(X, m, W.scal, y, W.n, W.partial);
            k_reduce_partials<1><<<1, 32, 0, W.s>>>(W.partial, (int)grid, 1, W.scal + 40, 1);
            FCI_CUDA(cudaGetLastError());
            if (pass == 0) {
                double h[41];
                FCI_CUDA(cudaMemcpyAsync(h, W.scal, sizeof(double) * 41, cudaMemcpyDeviceToHost, W.s));
                FCI_CUDA(cudaStreamSynchronize(W.s));
                double c2 = 0.0;
                for (int i = 0; i < m; ++i) c2 += h[i] * h[i];
                if (h[40] >= c2) break;  // ||y1||^2 >= ||y0||^2 / 2: one pass suffices
            }
        }
    } else if (int rc = dots(W, y, 1, y, W.scal + 40, 1)) {
        return rc;
    }
    k_scale<<<grid_for(W.n), 256, 0, W.s>>>(y, W.scal + 40, 1e-10, W.keep, W.n);
    FCI_CUDA(cudaGetLastError());
    int h = 0;
    FCI_CUDA(cudaMemcpyAsync(&h, W.keep, sizeof(int), cudaMemcpyDeviceToHost, W.s));
    FCI_CUDA(cudaStreamSynchronize(W.s));
    *kept = h;
    return FCI_OK;
}


// out[i*stride] = X_i . y for FP32 X [m][n] and y (m <= 32), double-float sums
int dots_f32(Work &W, const float *X, int m, const float *y, double *out, int stride) {
    if (m <= 0) return FCI_OK;
    if (m > 32) return fail(FCI_ERR_ARG, "subspace larger than 32 vectors");
    const int groups = (m + 7) / 8;
    k_multidot_f32<<<kDotBlocks * groups, 256, 0, W.s>>>(X, m, y, W.n, groups, W.partial);
    k_reduce_partials<32><<<1, 32, 0, W.s>>>(W.partial, kDotBlocks, m, out, stride);
    FCI_CUDA(cudaGetLastError());
    return FCI_OK;
}

// orthonormalise the FP32 vector y against the FP32 basis X_0..X_{m-1} (the
// same criterion for a second pass as orthonormalise), normalise; *kept = 1 if kept
int orthonormalise_f32(Work &W, const float *X, int m, float *y, int *kept) {
    const unsigned grid = grid_for(W.n);
    if (m > 0) {
        for (int pass = 0; pass < 2; ++pass) {
            if (int rc = dots_f32(W, X, m, y, W.scal, 1)) return rc;
            k_sub_proj_f32<<<grid, 256, 0, W.s>>>(X, m, W.scal, y, W.n, W.partial);
            k_reduce_partials<1><<<1, 32, 0, W.s>>>(W.partial, (int)grid, 1, W.scal + 40, 1);
            FCI_CUDA(cudaGetLastError());
            if (pass == 0) {
                double h[41];
                FCI_CUDA(cudaMemcpyAsync(h, W.scal, sizeof(double) * 41, cudaMemcpyDeviceToHost, W.s));
                FCI_CUDA(cudaStreamSynchronize(W.s));
                double c2 = 0.0;
                for (int i = 0; i < m; ++i) c2 += h[i] * h[i];
                if (h[40] >= c2) break;
            }
        }
    } else if (int rc = dots_f32(W, y, 1, y, W.scal + 40, 1)) {
        return rc;
    }
    k_scale_f32<<<grid, 256, 0, W.s>>>(y, W.scal + 40, 1e-10, W.keep, W.n);
    FCI_CUDA(cudaGetLastError());
    int h = 0;
    FCI_CUDA(cudaMemcpyAsync(&h, W.keep, sizeof(int), cudaMemcpyDeviceToHost, W.s));
    FCI_CUDA(cudaStreamSynchronize(W.s));
    *kept = h;
    return FCI_OK;
}

}  // namespace

// Mixed-precision Davidson with an FP32 basis, for spaces whose FP64 basis
// does not fit in device memory (CAS(18,18): one FP64 vector is 18.9 GB).
// The same iteration as the FP64-basis mixed mode: FP32 sigma for every new
// correction, refinement points where the FP64 sigma of each Ritz vector
// x = B v corrects the subspace sigma vectors along v (S <- S + (sigma64(x) -
// S v) v^T) and the projected matrix with them, convergence tested only there
// (exact Rayleigh quotients and residuals of the FP64 Ritz vectors).  The
// basis B and S are stored in FP32 (orthonormal to FP32 rounding, products
// summed in double-float), the Ritz vectors and their sigma in FP64.  The FP32
// storage of S puts a floor of about 1e-7 ||H|| under the residual, below
// sqrt(tol) for tol >= 1e-9; a thick restart collapses B and S in place onto
// the lowest Ritz directions (S v keeps the FP64 sigma of refined Ritz vectors).
static int run_davidson_f32basis(fci_ctx *ctx, int nroots, double tol, double *energies, void *vecs,
                                 const void *guess, int maxsub) {
    using clk = std::chrono::steady_clock;
    const auto t0 = clk::now();
    Work W;
    W.ctx = ctx;
    W.s = ctx->stream;
    W.n = ctx->ndet;
    W.nroots = nroots;
    W.maxsub = maxsub;
    W.parity = ctx->opt.spin_parity;
    const int64_t n = W.n;
    cudaStream_t s = W.s;
    W.Bf = W.get<float>((size_t)maxsub * n);
    W.Sf = W.get<float>((size_t)maxsub * n);
    W.y32 = W.get<float>(n);
    W.X = W.get<double>((size_t)nroots * n);
    W.HX = W.get<double>((size_t)nroots * n);
    W.A = W.get<double>(kMaxSub * kMaxSub);
    W.w = W.get<double>(kMaxSub);
    W.V = W.get<double>(kMaxSub * kMaxSub);
    W.partial = W.get<double>(kDotBlocks * 32);
    W.scal = W.get<double>(64);
    W.rn2 = W.get<double>(8);
    W.keep = W.get<int>(1);
    W.idx = W.get<int64_t>(8);
    W.pidx = W.get<int64_t>(kDotBlocks + 1);
    if (W.rc) return W.rc;
    ctx->log.clear();
    ctx->log_width = nroots + 3;
    ctx->iterations = 0;
    ctx->sigma_calls = 0;
    auto sigma32 = [&](int i) {
        ctx->sigma_calls++;
        return launch_sigma(ctx, W.Bf + (size_t)i * n, W.Sf + (size_t)i * n, FCI_F32, s, W.parity);
    };
    auto sigma64 = [&](int k) {
        ctx->sigma_calls++;
        return launch_sigma(ctx, W.X + (size_t)k * n, W.HX + (size_t)k * n, FCI_F64, s, W.parity);
    };
    auto project = [&](int m) -> int {  // A = B^T S (columns j < m)
        FCI_CUDA(cudaMemsetAsync(W.A, 0, sizeof(double) * kMaxSub * kMaxSub, s));
        for (int j = 0; j < m; ++j)
            if (int rc = dots_f32(W, W.Bf, m, W.Sf + (size_t)j * n, W.A + j, kMaxSub)) return rc;
        return FCI_OK;
    };

    // (1) initial subspace
    int m = 0;
    for (int k = 0; k < nroots; ++k) {
        float *b = W.Bf + (size_t)m * n;
        if (guess) {
            k_cvt_d2f<<<grid_for(n), 256, 0, s>>>((const double *)guess + (size_t)k * n, b, n);
        } else {
            argmin_excl(W, ctx->hdiag, k);
            k_set_unit_f32<<<grid_for(n), 256, 0, s>>>(b, n, W.idx + k);
        }
        FCI_CUDA(cudaGetLastError());
        if (int rc = project_parity(W, b, 4)) return rc;
        int kept = 0;
        if (int rc = orthonormalise_f32(W, W.Bf, m, b, &kept)) return rc;
        if (kept) ++m;
    }
    if (m == 0) return fail(FCI_ERR_ARG, "initial guess vectors are linearly dependent");
    for (int i = 0; i < m; ++i)
        if (int rc = sigma32(i)) return rc;
    if (int rc = project(m)) return rc;

    // Ritz values and residuals of the FP32 subspace guide the iteration; at a
    // refinement point the reported values are the exact Rayleigh quotients
    // x.sigma64(x) / x.x of the FP64 Ritz vectors and their exact residuals
    // (the FP32-stored basis and sigma vectors hold the projected matrix only
    // to about 1e-7 relative, so its eigenvalues are not the energies)
    std::vector<double> e_prev(nroots, INFINITY), ev(kMaxSub), rn(nroots);
    bool converged = false;
    int it = 0, inner = 0;
    std::vector<double> r_hist;
    auto read_back = [&](int nr, double *rmax, bool exact) -> int {
        FCI_CUDA(cudaMemcpyAsync(ev.data(), W.w, sizeof(double) * nr, cudaMemcpyDeviceToHost, s));
        FCI_CUDA(cudaMemcpyAsync(rn.data(), W.rn2, sizeof(double) * nr, cudaMemcpyDeviceToHost, s));
        int derr = 0;
        FCI_CUDA(cudaMemcpyAsync(&derr, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
        FCI_CUDA(cudaStreamSynchronize(s));
        if (derr & 1) return fail(FCI_ERR_TIMEOUT, "a bounded device wait gave up inside sigma");
        if (derr) return fail(FCI_ERR_RANGE, "a level sum of the FP64 tensor-core sigma left its exact range");
        *rmax = 0.0;
        for (int k = 0; k < nr; ++k) {
            rn[k] = std::sqrt(rn[k]);
            *rmax = std::max(*rmax, rn[k]);
        }
        const double el = std::chrono::duration<double>(clk::now() - t0).count();
        ctx->log.push_back((double)it);
        ctx->log.push_back(exact ? 0.0 : 1.0);
        ctx->log.push_back(el);
        for (int k = 0; k < nroots; ++k) ctx->log.push_back(k < nr ? ev[k] : NAN);
        for (int k = 0; k < nr; ++k)
            if (!std::isfinite(ev[k]) || !std::isfinite(rn[k]))
                return fail(FCI_ERR_NAN, "Davidson: a Ritz value or residual norm is not finite (non-finite guess?)");
        return FCI_OK;
    };
    auto residuals = [&](int nr) -> int {
        for (int k = 0; k < nr; ++k) {
            k_resnorm<<<kDotBlocks, 256, 0, s>>>(W.X + (size_t)k * n, W.HX + (size_t)k * n, W.w, k, n, W.partial);
            k_reduce_partials<1><<<1, 32, 0, s>>>(W.partial, kDotBlocks, 1, W.rn2 + k, 1);
        }
        FCI_CUDA(cudaGetLastError());
        return FCI_OK;
    };
    for (it = 1; it <= ctx->opt.max_iter; ++it) {
        k_jacobi<<<1, 256, 0, s>>>(W.A, kMaxSub, m, W.w, W.V);
        FCI_CUDA(cudaGetLastError());
        const int nr = nroots < m ? nroots : m;
        for (int k = 0; k < nr; ++k) {
            k_lincomb_f32<<<grid_for(n), 256, 0, s>>>(W.Bf, m, W.V + k, m, W.X + (size_t)k * n, n);
            k_lincomb_f32<<<grid_for(n), 256, 0, s>>>(W.Sf, m, W.V + k, m, W.HX + (size_t)k * n, n);
        }
        if (int rc = residuals(nr)) return rc;
        double rmax = 0.0;
        if (int rc = read_back(nr, &rmax, false)) return rc;
        r_hist.push_back(rmax);
        const double r_win = r_hist.size() > 15 ? r_hist[r_hist.size() - 16] : INFINITY;
        if (++inner >= 60 || rmax < std::sqrt(tol) || (inner >= 15 && rmax > 0.5 * r_win)) {
            // refinement point: FP64 sigma of each Ritz vector; its difference to
            // the subspace estimate corrects S along v (and the projected matrix),
            // and the exact Rayleigh quotient and residual replace the estimates
            for (int k = 0; k < nr; ++k) {
                double *x = W.X + (size_t)k * n, *hx = W.HX + (size_t)k * n;
                if (int rc = sigma64(k)) return rc;
                k_sigma_delta_f32<<<grid_for(n), 256, 0, s>>>(hx, W.Sf, m, W.V, k, W.y32, n);
                if (int rc = dots_f32(W, W.Bf, m, W.y32, W.scal, 1)) return rc;
                k_rank1_sigma_f32<<<grid_for(n), 256, 0, s>>>(W.Sf, m, W.V, k, W.y32, n);
                k_rank1_proj<<<1, 256, 0, s>>>(W.A, kMaxSub, m, W.scal, W.V, k);
                if (int rc = dots(W, x, 1, hx, W.scal + 52, 1)) return rc;
                if (int rc = dots(W, x, 1, x, W.scal + 53, 1)) return rc;
                k_quotient<<<1, 1, 0, s>>>(W.scal + 52, W.scal + 53, W.w + k);
                FCI_CUDA(cudaGetLastError());
            }
            if (int rc = residuals(nr)) return rc;
            if (int rc = read_back(nr, &rmax, true)) return rc;
            double demax = 0.0;
            for (int k = 0; k < nr; ++k) demax = std::max(demax, std::fabs(ev[k] - e_prev[k]));
            if (nr == nroots && demax < tol && rmax < std::sqrt(tol)) {
                converged = true;
                break;
            }
            for (int k = 0; k < nr; ++k) e_prev[k] = ev[k];
            inner = 0;
        }
        if (m + nr > maxsub) {
            // thick restart in place: B and S collapse onto the lowest `keep` Ritz
            // directions (B v_k, S v_k); along a refined Ritz vector S v_k is its
            // FP64 sigma (stored in FP32), so no FP32 sigma error enters along it
            const int keep = std::min(m, std::max(nr, std::min(4, maxsub / 2)));
            k_collapse_f32<<<grid_for(n), 256, 0, s>>>(W.Bf, m, W.V, keep, n);
            k_collapse_f32<<<grid_for(n), 256, 0, s>>>(W.Sf, m, W.V, keep, n);
            FCI_CUDA(cudaGetLastError());
            m = keep;
            if (int rc = project(m)) return rc;
        }
        int added = 0;
        for (int k = 0; k < nr && m < maxsub; ++k) {
            float *b = W.Bf + (size_t)m * n;
            k_precond_f32<<<grid_for(n), 256, 0, s>>>(W.X + (size_t)k * n, W.HX + (size_t)k * n, ctx->hdiag, W.w, k, b, n);
            FCI_CUDA(cudaGetLastError());
            if (int rc = project_parity(W, b, 4)) return rc;
            int kept = 0;
            if (int rc = orthonormalise_f32(W, W.Bf, m, b, &kept)) return rc;
            if (!kept) continue;
            if (int rc = sigma32(m)) return rc;
            ++m;
            if (int rc = dots_f32(W, W.Bf, m, W.Sf + (size_t)(m - 1) * n, W.A + (m - 1), kMaxSub)) return rc;
            if (int rc = dots_f32(W, W.Sf, m, W.Bf + (size_t)(m - 1) * n, W.A + (size_t)(m - 1) * kMaxSub, 1))
                return rc;
            ++added;
        }
        if (added == 0) {
            if (inner == 0) {  // an exact point that adds nothing: no further progress
                converged = rmax < std::sqrt(tol);
                break;
            }
            inner = 1 << 20;  // refine on the next pass
        }
    }
    ctx->iterations = it > ctx->opt.max_iter ? ctx->opt.max_iter : it;
    for (int k = 0; k < nroots; ++k) energies[k] = ev[k];
    if (vecs) {
        for (int k = 0; k < nroots; ++k) {
            double *x = W.X + (size_t)k * n;
            if (int rc = dots(W, x, 1, x, W.scal + 54, 1)) return rc;
            k_scale<<<grid_for(n), 256, 0, s>>>(x, W.scal + 54, 0.0, W.keep, n);
            sign_of_absmax(W, x, W.scal + 50);
            k_scale_by<<<grid_for(n), 256, 0, s>>>(x, W.scal + 50, n);
            FCI_CUDA(cudaMemcpyAsync((double *)vecs + (size_t)k * n, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        }
    }
    FCI_CUDA(cudaStreamSynchronize(s));
    if (!converged) return fail(FCI_ERR_NOCONV, "Davidson did not converge within max_iter");
    return FCI_OK;
}

// Device bytes of the FP64-basis workspace, and the largest FP32-basis
// subspace (<= want) that fits in `avail` bytes (0 when none does).
static size_t f64_basis_bytes(int64_t n, int maxsub, int keepn, int nroots, bool mixed) {
    return (size_t)n * 8 * (size_t)(2 * maxsub + 2 * keepn + nroots) + (mixed ? (size_t)n * 8 : 0);
}
static int f32_basis_fit(int64_t n, int nroots, int want, size_t avail) {
    for (int m = want; m >= 2 * nroots && m >= 2; --m)
        if ((size_t)n * 4 * (size_t)(2 * m + 1) + (size_t)n * 8 * 2 * nroots <= avail) return m;
    return 0;
}

int run_davidson(fci_ctx *ctx, int nroots, double tol, double *energies, void *vecs, const void *guess) {
    {  // basis storage: FP64, or FP32 (mixed precision) where asked for or where FP64 does not fit
        int maxsub = std::min(32, std::max(ctx->opt.max_subspace, 2 * nroots));
        if (maxsub > ctx->ndet) maxsub = (int)ctx->ndet;
        const int keepn = std::max(nroots, std::min(8, maxsub / 2));
        const bool mixed = ctx->opt.precision == FCI_PREC_MIXED;
        size_t fr = 0, tot = 0;
        FCI_CUDA(cudaMemGetInfo(&fr, &tot));
        size_t avail = fr > ((size_t)2 << 30) ? fr - ((size_t)2 << 30) : 0;  // 2 GiB left for the runtime
        if (ctx->opt.max_device_bytes > 0) {
            const double cap = ctx->opt.max_device_bytes - (double)ctx->bytes;
            avail = std::min(avail, cap > 0 ? (size_t)cap : (size_t)0);
        }
        const bool f32b = mixed && (ctx->opt.basis_f32 == 1 ||
                                    (ctx->opt.basis_f32 == 0 && f64_basis_bytes(ctx->ndet, maxsub, keepn, nroots, mixed) > avail));
        if (f32b) {
            FCI_CUDA(cudaDeviceSynchronize());  // caller's guess buffer is complete
            const int m = ctx->opt.basis_f32 == 1 ? maxsub : f32_basis_fit(ctx->ndet, nroots, std::min(maxsub, 8), avail);
            if (m == 0) return fail(FCI_ERR_OOM, "Davidson: not even an FP32 basis of 2 vectors per root fits");
            return run_davidson_f32basis(ctx, nroots, tol, energies, vecs, guess, m);
        }
    }
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
    W.parity = ctx->opt.spin_parity;
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
    W.pidx = W.get<int64_t>(kDotBlocks + 1);
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
            argmin_excl(W, ctx->hdiag, k);
            k_set_unit<<<grid_for(n), 256, 0, s>>>(b, n, W.idx + k);
            FCI_CUDA(cudaGetLastError());
        }
        if (int rc = project_parity(W, b, 8)) return rc;
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
    double r_win = INFINITY;
    std::vector<double> r_hist;
    // FP64 tail: a refinement point measures the FP32 sigma error along each
    // Ritz vector (||sigma64(x) - S v||).  When that error exceeds sqrt(tol)/2
    // and the residual at an exact point is not below half of the previous
    // exact point's, the FP32 phase has stopped making progress: the subspace
    // collapses onto the Ritz vectors (with fresh FP64 sigma) and every later
    // correction gets an FP64 sigma
    bool fp64_tail = false, want_tail = false;
    double r_exact_prev = INFINITY;

    for (it = 1; it <= ctx->opt.max_iter; ++it) {
        // (4) diagonalise the projected matrix
        k_jacobi<<<1, 256, 0, s>>>(W.A, kMaxSub, m, W.w, W.V);
        FCI_CUDA(cudaGetLastError());
        const int nr = nroots < m ? nroots : m;
        // Ritz vectors, their sigma, residuals and (2)-(3) preconditioned corrections
        for (int k = 0; k < nr; ++k) {
            lincomb(s, W.Bv, m, W.V + k, m, 0.0, W.X + (size_t)k * n, n);
            lincomb(s, W.Sv, m, W.V + k, m, 0.0, W.HX + (size_t)k * n, n);
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
        if (derr & 1) return fail(FCI_ERR_TIMEOUT, "a bounded device wait gave up inside sigma");
        if (derr) return fail(FCI_ERR_RANGE, "a level sum of the FP64 tensor-core sigma left its exact range");
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
        for (int k = 0; k < nr; ++k)
            if (!std::isfinite(ev[k]) || !std::isfinite(rn[k]))
                return fail(FCI_ERR_NAN, "Davidson: a Ritz value or residual norm is not finite (non-finite guess?)");
        // residual 15 iterations ago (stagnation test of the FP32 phase)
        r_hist.push_back(rmax);
        r_win = r_hist.size() > 15 ? r_hist[r_hist.size() - 16] : INFINITY;
        if (exact) {
            if (nr == nroots && demax < tol && rmax < std::sqrt(tol)) {
                converged = true;
                break;
            }
            for (int k = 0; k < nr; ++k) e_prev[k] = ev[k];
            inner = 0;
            if (mixed && !fp64_tail) {
                if (want_tail && rmax > 0.5 * r_exact_prev && nr == nroots) {
                    // collapse onto the Ritz vectors with fresh FP64 sigma
                    FCI_CUDA(cudaMemcpyAsync(W.Bv, W.X, sizeof(double) * nr * n, cudaMemcpyDeviceToDevice, s));
                    for (int k = 0; k < nr; ++k)
                        if (int rc = sigma_of(W, false, W.Bv + (size_t)k * n, W.Sv + (size_t)k * n)) return rc;
                    m = nr;
                    FCI_CUDA(cudaMemsetAsync(W.A, 0, sizeof(double) * kMaxSub * kMaxSub, s));
                    for (int j = 0; j < m; ++j)
                        if (int rc = dots(W, W.Bv, m, W.Sv + (size_t)j * n, W.A + j, kMaxSub)) return rc;
                    fp64_tail = true;
                }
                r_exact_prev = rmax;
            }
        } else if (++inner >= 60 || rmax < std::sqrt(tol) || (inner >= 15 && rmax > 0.5 * r_win)) {
            // refinement: exact FP64 sigma of each Ritz vector; the difference to
            // the subspace estimate corrects every sigma vector along that Ritz
            // direction (S += delta v^T) and the projected matrix with it
            for (int k = 0; k < nr; ++k) {
                double *d = W.T + (size_t)k * n;
                if (int rc = sigma_of(W, false, W.X + (size_t)k * n, d)) return rc;
                k_sub<<<grid_for(n), 256, 0, s>>>(d, W.HX + (size_t)k * n, d, n);
                if (int rc = dots(W, d, 1, d, W.scal + 48 + k, 1)) return rc;  // ||sigma error||^2
                if (int rc = dots(W, W.Bv, m, d, W.scal, 1)) return rc;
                k_rank1_sigma<<<grid_for(n), 256, 0, s>>>(W.Sv, m, W.V, k, d, n);
                k_rank1_proj<<<1, 256, 0, s>>>(W.A, kMaxSub, m, W.scal, W.V, k);
                FCI_CUDA(cudaGetLastError());
            }
            {
                std::vector<double> err2(nr);
                FCI_CUDA(cudaMemcpyAsync(err2.data(), W.scal + 48, sizeof(double) * nr, cudaMemcpyDeviceToHost, s));
                FCI_CUDA(cudaStreamSynchronize(s));
                for (int k = 0; k < nr; ++k)
                    if (std::sqrt(err2[k]) > 0.5 * std::sqrt(tol)) want_tail = true;
            }
            exact = true;
            continue;
        }
        if (m + nr > maxsub) {
            // thick restart: collapse onto the lowest `keep` Ritz vectors (orthonormal
            // to rounding) and their sigma
            const int keep = std::min(keepn, m);
            for (int k = nr; k < keep; ++k) {
                lincomb(s, W.Bv, m, W.V + k, m, 0.0, W.X + (size_t)k * n, n);
                lincomb(s, W.Sv, m, W.V + k, m, 0.0, W.HX + (size_t)k * n, n);
            }
            FCI_CUDA(cudaGetLastError());
            FCI_CUDA(cudaMemcpyAsync(W.Bv, W.X, sizeof(double) * keep * n, cudaMemcpyDeviceToDevice, s));
            FCI_CUDA(cudaMemcpyAsync(W.Sv, W.HX, sizeof(double) * keep * n, cudaMemcpyDeviceToDevice, s));
            if (mixed && !fp64_tail && keep > nr) exact = false;  // the extra vectors carry FP32 sigma
            m = keep;
            FCI_CUDA(cudaMemsetAsync(W.A, 0, sizeof(double) * kMaxSub * kMaxSub, s));
            for (int j = 0; j < m; ++j)
                if (int rc = dots(W, W.Bv, m, W.Sv + (size_t)j * n, W.A + j, kMaxSub)) return rc;
        }
        int added = 0;
        for (int k = 0; k < nr && m < maxsub; ++k) {
            double *b = W.Bv + (size_t)m * n;
            FCI_CUDA(cudaMemcpyAsync(b, W.T + (size_t)k * n, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
            if (int rc = project_parity(W, b, 8)) return rc;
            int kept = 0;
            if (int rc = orthonormalise(W, W.Bv, m, b, &kept)) return rc;
            if (!kept) continue;
            // (4) new sigma (FP32 in mixed mode), new row/column of the projected matrix
            if (int rc = sigma_of(W, mixed && !fp64_tail, b, W.Sv + (size_t)m * n)) return rc;
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
        if (mixed && !fp64_tail) exact = false;
    }
    ctx->iterations = it > ctx->opt.max_iter ? ctx->opt.max_iter : it;
    for (int k = 0; k < nroots; ++k) energies[k] = ev[k];
    if (vecs) {
        for (int k = 0; k < nroots; ++k) {
            double *dst = (double *)vecs + (size_t)k * n;
            sign_of_absmax(W, W.X + (size_t)k * n, W.scal + 50);
            k_scale_by<<<grid_for(n), 256, 0, s>>>(W.X + (size_t)k * n, W.scal + 50, n);
            FCI_CUDA(cudaMemcpyAsync(dst, W.X + (size_t)k * n, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        }
    }
    FCI_CUDA(cudaStreamSynchronize(s));
    if (!converged) return fail(FCI_ERR_NOCONV, "Davidson did not converge within max_iter");
    return FCI_OK;
}

}  // namespace fci
