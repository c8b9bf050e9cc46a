// C ABI entry points (include/fci.h): context lifetime, argument checks,
// error reporting, and dispatch to the kernels.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include <mutex>

#include "internal.cuh"

namespace fci {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

int fail(int code, const std::string &msg) {
    set_error(msg);
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    char buf[512];
    snprintf(buf, sizeof(buf), "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
    set_error(buf);
    return e == cudaErrorMemoryAllocation ? FCI_ERR_OOM : FCI_ERR_CUDA;
}

void *dalloc(fci_ctx *ctx, size_t bytes, int *rc) {
    if (*rc != FCI_OK || bytes == 0) return nullptr;
    if (ctx->opt.max_device_bytes > 0 && (double)ctx->bytes + (double)bytes > ctx->opt.max_device_bytes) {
        char buf[200];
        snprintf(buf, sizeof(buf), "allocation of %zu bytes would exceed fci_options.max_device_bytes (%.0f; %zu held)",
                 bytes, ctx->opt.max_device_bytes, ctx->bytes);
        set_error(buf);
        *rc = FCI_ERR_OOM;
        return nullptr;
    }
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        char buf[160];
        snprintf(buf, sizeof(buf), "cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
        set_error(buf);
        *rc = FCI_ERR_OOM;
        return nullptr;
    }
    ctx->bytes += bytes;
    return p;
}

void dfree(fci_ctx *ctx, void *p, size_t bytes) {
    if (!p) return;
    cudaFree(p);
    ctx->bytes -= bytes;
}

int unpack_table(fci_ctx *ctx, int spin, int32_t *tgt, int8_t *k, int8_t *l, int8_t *sg);

int prof_begin(fci_ctx *ctx, cudaStream_t s, int nkernels, const char *const *names) {
    if (!ctx->prof || ctx->prof_ev.empty()) return -1;
    if (ctx->prof_count > 0 && ctx->prof_nk != nkernels) {
        ctx->prof_count = 0;  // pipeline changed: drop old records
        ctx->prof_head = 0;
    }
    ctx->prof_nk = nkernels;
    ctx->prof_names.assign(names, names + nkernels);
    int slot = ctx->prof_head;
    ctx->prof_head = (ctx->prof_head + 1) % kProfRing;
    if (ctx->prof_count < kProfRing) ctx->prof_count++;
    int base = slot * (kProfMaxKernels + 1);
    cudaEventRecord(ctx->prof_ev[base], s);
    return base;
}

void prof_mark(fci_ctx *ctx, int rec, int i, cudaStream_t s) {
    if (rec < 0) return;
    cudaEventRecord(ctx->prof_ev[rec + 1 + i], s);
}

static int check_integrals(int n, const double *h1, const double *eri, double tol) {
    for (int i = 0; i < n * n; ++i)
        if (!std::isfinite(h1[i])) return fail(FCI_ERR_ARG, "h1 has a non-finite element");
    for (int p = 0; p < n; ++p)
        for (int q = 0; q < p; ++q)
            if (std::fabs(h1[p * n + q] - h1[q * n + p]) > tol) return fail(FCI_ERR_ARG, "h1 is not symmetric");
    const int64_t n2 = (int64_t)n * n;
    auto at = [&](int i, int j, int k, int l) { return eri[(i * n2 * n) + (int64_t)j * n2 + (int64_t)k * n + l]; };
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            for (int k = 0; k < n; ++k)
                for (int l = 0; l < n; ++l) {
                    double v = at(i, j, k, l);
                    if (!std::isfinite(v)) return fail(FCI_ERR_ARG, "eri has a non-finite element");
                    if (std::fabs(v - at(j, i, k, l)) > tol || std::fabs(v - at(i, j, l, k)) > tol ||
                        std::fabs(v - at(k, l, i, j)) > tol)
                        return fail(FCI_ERR_ARG, "eri lacks the 8-fold permutational symmetry of real orbitals");
                }
    return FCI_OK;
}

static int64_t binom64(int n, int k) {
    if (k < 0 || k > n) return 0;
    int64_t r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

}  // namespace fci

using namespace fci;

extern "C" {

void fci_default_options(fci_options *opt) {
    if (!opt) return;
    memset(opt, 0, sizeof(*opt));
    opt->struct_size = (int)sizeof(fci_options);
    opt->device = -1;
    opt->max_subspace = 24;
    opt->max_iter = 300;
    opt->precision = FCI_PREC_FP64;
    opt->mixed_switch = 1e-2;
    opt->symmetry_tol = 1e-12;
    opt->f32_splits = 3;
    opt->same_spin_tc = 0;
    opt->f64_kernels = FCI_F64_AUTO;
    opt->basis_f32 = 0;
}

const char *fci_last_error(void) { return g_last_error.c_str(); }

int fci_init(fci_ctx **out, int norb, int nalpha, int nbeta, const double *h1, const double *eri,
             const fci_options *opt) {
    set_error("");
    if (!out) return fail(FCI_ERR_ARG, "ctx pointer is NULL");
    *out = nullptr;
    if (!h1 || !eri) return fail(FCI_ERR_ARG, "h1 or eri is NULL");
    if (norb < 1 || norb > 30) return fail(FCI_ERR_ARG, "norb must be in 1..30");
    if (nalpha < 0 || nbeta < 0 || nalpha > norb || nbeta > norb)
        return fail(FCI_ERR_ARG, "electron counts must be in 0..norb");
    if (binom64(norb, nalpha) > kMaxStrings || binom64(norb, nbeta) > kMaxStrings)
        return fail(FCI_ERR_ARG, "too many strings of one spin (limit 2^21 - 1)");
    fci_options o;
    fci_default_options(&o);
    if (opt) {
        if (opt->struct_size != (int)sizeof(fci_options)) return fail(FCI_ERR_ARG, "fci_options.struct_size mismatch");
        o = *opt;
    }
    if (o.max_subspace < 2 || o.max_iter < 1) return fail(FCI_ERR_ARG, "max_subspace >= 2 and max_iter >= 1 required");
    if (o.precision != FCI_PREC_FP64 && o.precision != FCI_PREC_MIXED) return fail(FCI_ERR_ARG, "unknown precision");
    if (o.f32_splits != 2 && o.f32_splits != 3) return fail(FCI_ERR_ARG, "f32_splits must be 2 or 3");
    if (o.same_spin_tc != 0 && o.same_spin_tc != 1) return fail(FCI_ERR_ARG, "same_spin_tc must be 0 or 1");
    if (!(o.max_device_bytes >= 0)) return fail(FCI_ERR_ARG, "max_device_bytes must be >= 0");
    if (o.f32_row_global != 0 && o.f32_row_global != 1) return fail(FCI_ERR_ARG, "f32_row_global must be 0 or 1");
    if (o.basis_f32 < 0 || o.basis_f32 > 2) return fail(FCI_ERR_ARG, "basis_f32 must be 0, 1 or 2");
    if (o.spin_parity < -1 || o.spin_parity > 1) return fail(FCI_ERR_ARG, "spin_parity must be -1, 0 or 1");
    if (o.spin_parity != 0 && nalpha != nbeta)
        return fail(FCI_ERR_ARG, "spin_parity needs n_alpha = n_beta (Ms = 0)");
    if (!(o.rdm2_chunk_bytes >= 0)) return fail(FCI_ERR_ARG, "rdm2_chunk_bytes must be >= 0");
    if (o.f64_same_spin != FCI_SS_AUTO && o.f64_same_spin != FCI_SS_FAMILY)
        return fail(FCI_ERR_ARG, "f64_same_spin must be FCI_SS_AUTO or FCI_SS_FAMILY");
    if (o.f64_kernels < FCI_F64_AUTO || o.f64_kernels > FCI_F64_WIDE)
        return fail(FCI_ERR_ARG, "f64_kernels must be FCI_F64_AUTO, FCI_F64_FMA, FCI_F64_SLICED or FCI_F64_WIDE");
    if (int rc = check_integrals(norb, h1, eri, o.symmetry_tol)) return rc;

    fci_ctx *ctx = new (std::nothrow) fci_ctx();
    if (!ctx) return fail(FCI_ERR_OOM, "host allocation failed");
    ctx->opt = o;
    ctx->norb = norb;
    ctx->A.ne = nalpha;
    ctx->B.ne = nbeta;
    int dev = o.device;
    if (dev < 0) {
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) { delete ctx; return cuda_fail(e, "cudaGetDevice"); }
    }
    ctx->device = dev;
    cudaError_t e = cudaSetDevice(dev);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { delete ctx; return cuda_fail(e, "device setup"); }
    int rc = FCI_OK;
    try {
        rc = build_tables(ctx, h1, eri);
    } catch (const std::bad_alloc &) {  // host tables: no exception crosses the C ABI
        rc = fail(FCI_ERR_OOM, "host allocation failed while building the tables");
    }
    if (rc) {
        std::string msg = g_last_error;
        fci_free(ctx);
        set_error(msg);
        return rc;
    }
    *out = ctx;
    return FCI_OK;
}

int fci_free(fci_ctx *ctx) {
    if (!ctx) return FCI_OK;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    free_tables(ctx);
    for (auto &e : ctx->prof_ev) cudaEventDestroy(e);
    if (ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return FCI_OK;
}

namespace {
std::mutex g_default_mu;
fci_ctx *g_default_ctx = nullptr;
}  // namespace

int fci_init_default(int norb, int nalpha, int nbeta, const double *h1, const double *eri) {
    std::lock_guard<std::mutex> lock(g_default_mu);
    fci_free(g_default_ctx);
    g_default_ctx = nullptr;
    return fci_init(&g_default_ctx, norb, nalpha, nbeta, h1, eri, nullptr);
}

fci_ctx *fci_default_context(void) {
    std::lock_guard<std::mutex> lock(g_default_mu);
    return g_default_ctx;
}

int fci_free_default(void) {
    std::lock_guard<std::mutex> lock(g_default_mu);
    const int rc = fci_free(g_default_ctx);
    g_default_ctx = nullptr;
    return rc;
}

int fci_sigma(fci_ctx *ctx, const void *c, void *sigma, int dtype, void *stream) {
    if (!ctx) return fail(FCI_ERR_ARG, "ctx is NULL");
    if (!c || !sigma) return fail(FCI_ERR_ARG, "c or sigma is NULL");
    if (c == sigma) return fail(FCI_ERR_ARG, "c and sigma must not overlap");
    FCI_CUDA(cudaSetDevice(ctx->device));
    try {
        return launch_sigma(ctx, c, sigma, dtype, (cudaStream_t)stream);
    } catch (const std::bad_alloc &) {
        return fail(FCI_ERR_OOM, "host allocation failed");
    }
}

int fci_hdiag(fci_ctx *ctx, double *out, void *stream) {
    if (!ctx || !out) return fail(FCI_ERR_ARG, "NULL argument");
    FCI_CUDA(cudaSetDevice(ctx->device));
    FCI_CUDA(cudaMemcpyAsync(out, ctx->hdiag, sizeof(double) * ctx->ndet, cudaMemcpyDeviceToDevice,
                             (cudaStream_t)stream));
    return FCI_OK;
}

int fci_davidson(fci_ctx *ctx, int nroots, double tol, double *energies, void *vecs, const void *guess) {
    if (!ctx || !energies) return fail(FCI_ERR_ARG, "NULL argument");
    if (nroots < 1 || nroots > 8 || nroots > ctx->ndet) return fail(FCI_ERR_ARG, "nroots must be in 1..min(8, N)");
    if (!(tol > 0)) return fail(FCI_ERR_ARG, "tol must be positive");
    FCI_CUDA(cudaSetDevice(ctx->device));
    try {
        return run_davidson(ctx, nroots, tol, energies, vecs, guess);
    } catch (const std::bad_alloc &) {  // the workspace frees itself on unwinding
        return fail(FCI_ERR_OOM, "host allocation failed");
    }
}

int fci_davidson_log(fci_ctx *ctx, double *out, int cap, int *count) {
    if (!ctx) return fail(FCI_ERR_ARG, "ctx is NULL");
    int w = ctx->log_width;
    int nrec = w ? (int)(ctx->log.size() / w) : 0;
    if (count) *count = nrec;
    if (out && cap > 0 && w) {
        int m = nrec < cap ? nrec : cap;
        memcpy(out, ctx->log.data(), sizeof(double) * (size_t)m * w);
    }
    return FCI_OK;
}

int fci_rdm1(fci_ctx *ctx, const void *c, int dtype, double *gamma) {
    if (!ctx || !c || !gamma) return fail(FCI_ERR_ARG, "NULL argument");
    if (dtype != FCI_F64 && dtype != FCI_F32) return fail(FCI_ERR_ARG, "dtype must be FCI_F64 or FCI_F32");
    FCI_CUDA(cudaSetDevice(ctx->device));
    FCI_CUDA(cudaDeviceSynchronize());  // c may still be in flight on the caller's streams
    try {
        return run_rdm1(ctx, c, dtype, gamma);
    } catch (const std::bad_alloc &) {
        return fail(FCI_ERR_OOM, "host allocation failed");
    }
}

int fci_rdm2(fci_ctx *ctx, const void *c, int dtype, double *gamma1, double *gamma2) {
    if (!ctx || !c || !gamma2) return fail(FCI_ERR_ARG, "NULL argument");
    if (dtype != FCI_F64 && dtype != FCI_F32) return fail(FCI_ERR_ARG, "dtype must be FCI_F64 or FCI_F32");
    FCI_CUDA(cudaSetDevice(ctx->device));
    FCI_CUDA(cudaDeviceSynchronize());  // c may still be in flight on the caller's streams
    try {
        return run_rdm2(ctx, c, dtype, gamma1, gamma2);
    } catch (const std::bad_alloc &) {
        return fail(FCI_ERR_OOM, "host allocation failed");
    }
}

int fci_get_strings(fci_ctx *ctx, int spin, uint32_t *out) {
    if (!ctx || !out || (spin != 0 && spin != 1)) return fail(FCI_ERR_ARG, "bad argument");
    FCI_CUDA(cudaSetDevice(ctx->device));
    const SpinTables &T = spin ? ctx->B : ctx->A;
    FCI_CUDA(cudaMemcpyAsync(out, T.str, sizeof(uint32_t) * T.ns, cudaMemcpyDeviceToHost, ctx->stream));
    FCI_CUDA(cudaStreamSynchronize(ctx->stream));
    return FCI_OK;
}

int fci_get_single_table(fci_ctx *ctx, int spin, int32_t *tgt, int8_t *k, int8_t *l, int8_t *sign) {
    if (!ctx || (spin != 0 && spin != 1)) return fail(FCI_ERR_ARG, "bad argument");
    FCI_CUDA(cudaSetDevice(ctx->device));
    return unpack_table(ctx, spin, tgt, k, l, sign);
}

static int tile_schedule_api(int64_t ns, int nsingle, int npair, const int32_t *tgt, const int32_t *pair,
                             const int8_t *sign, uint32_t *sched, int64_t cap, int64_t *nsched, int32_t *toff);

int fci_tile_schedule(int64_t ns, int nsingle, int npair, const int32_t *tgt, const int32_t *pair,
                      const int8_t *sign, uint32_t *sched, int64_t cap, int64_t *nsched, int32_t *toff) {
    if (!tgt || !pair || !sign || !nsched) return fail(FCI_ERR_ARG, "fci_tile_schedule: NULL table or nsched");
    if (ns < 1 || ns > fci::kMaxScheduleStrings)
        return fail(FCI_ERR_ARG, "fci_tile_schedule: ns must be in [1, 65408]");
    if (nsingle < 1 || nsingle > 1024 || npair < 1 || npair > 256)
        return fail(FCI_ERR_ARG, "fci_tile_schedule: 1 <= nsingle <= 1024 and 1 <= npair <= 256 required");
    try {
        return tile_schedule_api(ns, nsingle, npair, tgt, pair, sign, sched, cap, nsched, toff);
    } catch (const std::bad_alloc &) {
        return fail(FCI_ERR_OOM, "fci_tile_schedule: host allocation failed");
    }
}

static int tile_schedule_api(int64_t ns, int nsingle, int npair, const int32_t *tgt, const int32_t *pair,
                             const int8_t *sign, uint32_t *sched, int64_t cap, int64_t *nsched, int32_t *toff) {
    // packed entry-major copy, the layout fci_init builds on the device
    std::vector<uint32_t> tab((size_t)ns * nsingle);
    for (int64_t x = 0; x < ns; ++x)
        for (int e = 0; e < nsingle; ++e) {
            const size_t i = (size_t)x * nsingle + e;
            if (tgt[i] < 0 || tgt[i] >= ns || pair[i] < 0 || pair[i] >= npair || (sign[i] != 1 && sign[i] != -1))
                return fail(FCI_ERR_ARG, "fci_tile_schedule: table entry out of range");
            tab[(size_t)e * ns + x] = (uint32_t)tgt[i] | ((uint32_t)pair[i] << fci::kPairShift) |
                                      (sign[i] < 0 ? 0x80000000u : 0u);
        }
    std::vector<uint32_t> out;
    std::vector<int32_t> off;
    if (!fci::tile_schedule_host(tab.data(), ns, nsingle, out, off))
        return fail(FCI_ERR_ARG, "fci_tile_schedule: schedule longer than 2^31 entries");
    *nsched = (int64_t)out.size();
    if (toff) std::memcpy(toff, off.data(), sizeof(int32_t) * off.size());
    if (sched && cap >= (int64_t)out.size()) std::memcpy(sched, out.data(), sizeof(uint32_t) * out.size());
    return FCI_OK;
}

int fci_profile_enable(fci_ctx *ctx, int on) {
    if (!ctx) return fail(FCI_ERR_ARG, "ctx is NULL");
    FCI_CUDA(cudaSetDevice(ctx->device));
    if (on && ctx->prof_ev.empty()) {
        ctx->prof_ev.resize((size_t)kProfRing * (kProfMaxKernels + 1));
        for (auto &e : ctx->prof_ev) FCI_CUDA(cudaEventCreate(&e));
    }
    ctx->prof = on != 0;
    ctx->prof_count = 0;
    ctx->prof_head = 0;
    return FCI_OK;
}

int fci_profile_read(fci_ctx *ctx, double *ms, int cap_records, int *nrecords, int *nkernels) {
    if (!ctx) return fail(FCI_ERR_ARG, "ctx is NULL");
    FCI_CUDA(cudaSetDevice(ctx->device));
    const int nk = ctx->prof_nk, cnt = ctx->prof_count;
    if (nkernels) *nkernels = nk;
    int m = cnt < cap_records ? cnt : cap_records;
    if (!ms) m = 0;
    const int first = (ctx->prof_head - cnt + kProfRing) % kProfRing;
    for (int r = 0; r < m; ++r) {
        int base = ((first + r) % kProfRing) * (kProfMaxKernels + 1);
        for (int i = 0; i < nk; ++i) {
            FCI_CUDA(cudaEventSynchronize(ctx->prof_ev[base + 1 + i]));
            float t = 0.f;
            FCI_CUDA(cudaEventElapsedTime(&t, ctx->prof_ev[base + i], ctx->prof_ev[base + 1 + i]));
            ms[(size_t)r * nk + i] = t;
        }
    }
    if (nrecords) *nrecords = ms ? m : cnt;
    if (ms) {
        ctx->prof_count = 0;
        ctx->prof_head = 0;
    }
    return FCI_OK;
}

const char *fci_profile_kernel_name(fci_ctx *ctx, int i) {
    if (!ctx || i < 0 || i >= (int)ctx->prof_names.size()) return nullptr;
    return ctx->prof_names[i];
}

int fci_check_wait_timeout(fci_ctx *ctx) {
    if (!ctx) return fail(FCI_ERR_ARG, "ctx is NULL");
    FCI_CUDA(cudaSetDevice(ctx->device));
    FCI_CUDA(cudaStreamSynchronize(ctx->stream));
    FCI_CUDA(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream));
    if (int rc = launch_wait_timeout_probe(ctx)) return rc;
    int h = 0;
    FCI_CUDA(cudaMemcpyAsync(&h, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    FCI_CUDA(cudaStreamSynchronize(ctx->stream));
    FCI_CUDA(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream));
    FCI_CUDA(cudaStreamSynchronize(ctx->stream));
    if (h) return fail(FCI_ERR_TIMEOUT, "a bounded device wait gave up (self-test: no thread arrives on its barrier)");
    return FCI_OK;
}

int64_t fci_query(fci_ctx *ctx, int what) {
    if (!ctx) return -1;
    switch (what) {
        case FCI_Q_NDET: return ctx->ndet;
        case FCI_Q_NSTR_ALPHA: return ctx->A.ns;
        case FCI_Q_NSTR_BETA: return ctx->B.ns;
        case FCI_Q_NSINGLE_ALPHA: return ctx->A.nsingle;
        case FCI_Q_NSINGLE_BETA: return ctx->B.nsingle;
        case FCI_Q_NPAIR: return ctx->npair;
        case FCI_Q_DEVICE_BYTES: return (int64_t)ctx->bytes;
        case FCI_Q_ITERATIONS: return ctx->iterations;
        case FCI_Q_SIGMA_CALLS: return ctx->sigma_calls;
        case FCI_Q_DEVICE_ERROR: {
            int h = 0;
            if (cudaSetDevice(ctx->device) != cudaSuccess) return -1;
            if (cudaDeviceSynchronize() != cudaSuccess) return -1;
            if (cudaMemcpy(&h, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
            if (h && cudaMemset(ctx->d_err, 0, sizeof(int)) != cudaSuccess) return -1;
            return h;
        }
        default: return -1;
    }
}

}  // extern "C"
