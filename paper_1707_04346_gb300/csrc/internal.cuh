// Internal declarations shared by the library's translation units.
// Not part of the public ABI (see include/fci.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "fci.h"

namespace fci {

// ---- error plumbing -------------------------------------------------------
void set_error(const std::string &msg);
int fail(int code, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);

#define FCI_CUDA(call)                                          \
    do {                                                        \
        cudaError_t _e = (call);                                \
        if (_e != cudaSuccess) return ::fci::cuda_fail(_e, #call); \
    } while (0)

// ---- packed single-replacement entry -------------------------------------
// bits 0..20  target string address (< 2^21)
// bits 21..30 packed orbital-pair index (k,l) -> max*(max+1)/2 + min (< 1024)
// bit  31     1 if the sign is negative
constexpr int kTargetBits = 21;
constexpr uint32_t kTargetMask = (1u << kTargetBits) - 1u;
constexpr int kPairShift = 21;
constexpr uint32_t kPairMask = 0x3FFu;
constexpr int kMaxStrings = (1 << kTargetBits) - 1;
constexpr uint32_t kNoEntry = 0xFFFFFFFFu;  // per-string pair table: no entry with that pair

__host__ __device__ inline uint32_t ent_target(uint32_t e) { return e & kTargetMask; }
__host__ __device__ inline uint32_t ent_pair(uint32_t e) { return (e >> kPairShift) & kPairMask; }
__host__ __device__ inline bool ent_negative(uint32_t e) { return (e >> 31) != 0u; }
__host__ __device__ inline int pair_index(int k, int l) {
    int hi = k > l ? k : l, lo = k > l ? l : k;
    return hi * (hi + 1) / 2 + lo;
}

constexpr int kTileStrings = 128;  // beta strings per tensor-core tile (the MMA's M)
constexpr int64_t kMaxScheduleStrings = 65536 - kTileStrings;  // targets and dummies fit 16 bits

// ---- per-spin string data on the device ------------------------------------
struct SpinTables {
    int ne = 0;
    int64_t ns = 0;        // number of strings
    int nsingle = 0;       // ne*(norb-ne)+ne entries per string
    int nsame = 0;         // same-spin Hamiltonian row width: 1 + singles + doubles
    uint32_t *str = nullptr;   // [ns] bitmasks, ascending
    uint32_t *tab = nullptr;   // [nsingle][ns] packed entries (entry-major)
    uint32_t *tabo = nullptr;  // [ne*(norb-ne)][ns] off-diagonal entries only (k != l), entry-major
    double *wdiag = nullptr;   // [npair][ns]: sum over occupied l of (p | ll)
    int32_t *gcol = nullptr;   // [nsame][ns] same-spin Hamiltonian columns (ELL)
    double *gval = nullptr;    // [nsame][ns]
    float *gvalf = nullptr;    // [nsame][ns] FP32 copy (the leading part of the double-float pair)
    float *gvall = nullptr;    // [nsame][ns] fl(gval - gvalf): the trailing part of the double-float pair
    // Tile schedule of the replacement lists for the tensor-core sigma_3
    // (strings in tiles of kTileStrings): the entries of tile t's strings,
    // grouped by target, each target's run dealt whole to one of kTileStrings
    // shares (longest runs first, to the least loaded share), packed as
    // target | local source string << 16 | pair << 23 | negative << 31 and
    // stored step-major, entry j of share k at tsched[toff[t] + j*kTileStrings + k].
    // Shares are padded to the tile's longest share (toff[t+1] - toff[t] = that
    // length * kTileStrings) with entries for the dummy target ns + k.  Null when
    // ns > 65536 - kTileStrings or there are more than 256 pairs.
    uint32_t *tsched = nullptr;
    int32_t *toff = nullptr;  // [ntiles + 1]
    int64_t nsched = 0;
    // Replacement lists by orbital pair for the FP64 sliced sigma_3 (beta spin
    // only): tabp[x][q] (npad pairs per string, padded) = target | negative << 15
    // of the entry of string x with pair q, or 0xFFFF.  Owned by the context
    // (freed with the sliced tables).
    uint16_t *tabp = nullptr;
    // The same with 32-bit packed entries (kNoEntry where none), for the wide
    // FP64 kernels (sigma_wide.cu; beta spin only, owned by the context).
    uint32_t *tabp32 = nullptr;
    bool owner = true;         // false when aliasing the alpha tables
};

}  // namespace fci

struct fci_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;  // internal stream (blocking calls, Davidson)
    fci_options opt{};
    int norb = 0;
    int npair = 0;
    int64_t ndet = 0;
    fci::SpinTables A, B;           // alpha, beta
    double *h1 = nullptr;           // [n][n]
    double *eri = nullptr;          // [n^4]
    double *W = nullptr;            // [npair][npair] packed (ij|kl)
    float *Wf = nullptr;
    float *kf = nullptr;            // [npair] k_kl = h_kl - 1/2 sum_j (kj|jl), FP32 (same-spin tensor-core path)
    float *ws32 = nullptr;          // [2][ndet] FP32 workspace of that path (allocated on first use)
    // FP64 sliced sigma_3 (sigma3_sliced.cu): fixed-point integrals, the
    // per-call row exponents of C and its six bf16 digit slices (slices 0-3
    // and 4-5 as two planes, 12 bytes per determinant)
    long long *XW = nullptr;        // [npair][npair] round(W 2^(47 - eW))
    int eW = 0;                     // |W| < 2^eW
    int *rowexp = nullptr;          // [N_alpha]
    uint2 *cs0123 = nullptr;        // [ndet]
    uint32_t *cs45 = nullptr;       // [ndet]
    // FP64 sigma for large spaces (sigma_wide.cu): the fixed-point integral
    // table, the exponent of the call's C, and the 64-bit accumulator
    // (aliases ws32 when the context has it)
    long long *XT = nullptr;        // [npair + 1][npair]: round((q|p) 2^(47 - eC)), round(k_p 2^(48 - eC - sh1))
    int eC = 0;
    int sh1 = 0;
    int *d_eG = nullptr;            // device: largest biased exponent of C
    long long *wsacc = nullptr;     // [ndet] when ws32 is absent
    // FP64 same-spin terms as dense sliced products (sigma_ss.cu): digit planes
    // of each spin's same-spin Hamiltonian G_s with per-row exponents (the
    // beta ones alias the alpha ones when both spins share one string space),
    // and the per-call planes of C by rows and by columns with their exponents
    unsigned char *ssG_a = nullptr, *ssG_b = nullptr;
    int *ssE_a = nullptr, *ssE_b = nullptr;
    unsigned char *ssCr = nullptr, *ssCc = nullptr;
    int *ssEr = nullptr, *ssEc = nullptr;
    double *hdiag = nullptr;        // [ndet]
    int *d_err = nullptr;           // device error word (bounded waits that gave up)
    size_t bytes = 0;
    // Davidson bookkeeping
    std::vector<double> log;        // records of (nroots + 3) doubles
    int log_width = 0;
    int iterations = 0;
    int sigma_calls = 0;
    // per-kernel timing ring (fci_profile_*)
    bool prof = false;
    std::vector<cudaEvent_t> prof_ev;    // kProfRing * (kProfMaxKernels + 1)
    int prof_head = 0, prof_count = 0, prof_nk = 0;
    std::vector<const char *> prof_names;
};

namespace fci {

constexpr int kProfRing = 1024;
constexpr int kProfMaxKernels = 8;

// Start a profiling record for one sigma call (no-op unless enabled); returns
// the record's first event index or -1.  prof_mark(ctx, rec, i, s) records
// the event that closes kernel slot i.
int prof_begin(fci_ctx *ctx, cudaStream_t s, int nkernels, const char *const *names);
void prof_mark(fci_ctx *ctx, int rec, int i, cudaStream_t s);

void *dalloc(fci_ctx *ctx, size_t bytes, int *rc);
void dfree(fci_ctx *ctx, void *p, size_t bytes);

// tables.cu
int build_tables(fci_ctx *ctx, const double *h1_host, const double *eri_host);
void free_tables(fci_ctx *ctx);
// tile schedule of a packed entry-major table tab[e * ns + x] (host only; see
// SpinTables::tsched); false when its length would not fit the int32 offsets
bool tile_schedule_host(const uint32_t *tab, int64_t ns, int K, std::vector<uint32_t> &out,
                        std::vector<int32_t> &off);

// sigma.cu
// parity != 0 (Davidson with fci_options.spin_parity, n_alpha = n_beta): c is
// known to satisfy C^T = parity * C, so sigma_1 = parity * sigma_2^T is formed
// from sigma_2 by one transpose-add instead of its own kernel
int launch_sigma(fci_ctx *ctx, const void *c, void *sigma, int dtype, cudaStream_t s, int parity = 0);
// y <- y + sgn * y^T (half = 0) or (y + sgn * y^T) / 2 (half = 1) in place for a
// square n x n matrix of floats (elem 4), doubles (elem 8) or 64-bit integers
// (elem -8; half must be 0)
int sym_pairs(void *y, int64_t n, int elem, int sgn, int half, cudaStream_t s);
bool f32_same_spin_tc(const fci_ctx *ctx);
int alloc_sigma_workspace(fci_ctx *ctx);  // at fci_init: ws32 when the FP32 same-spin tensor-core path is used

// FP64 sigma of one batched instance (sliced sigma_3, double-float same-spin
// terms), skipped on the device when *active == 0; opted in beforehand
bool sigma_f64_gated_ok(const fci_ctx *ctx);
int prepare_sigma_f64_gated(const fci_ctx *ctx);
int launch_sigma_f64_gated(fci_ctx *ctx, const double *C, double *sig, const int *active, cudaStream_t s);

// FP32 sigma of one batched instance, skipped on the device when *active == 0
bool sigma_f32_gated_ok(const fci_ctx *ctx);
int prepare_sigma_f32_gated(const fci_ctx *ctx);
int launch_sigma_f32_gated(fci_ctx *ctx, const float *C, float *sig, const int *active, cudaStream_t s);

// sigma_tc.cu (tensor-core sigma_3 for FP32 vectors; nsplit = 2 or 3 bf16
// slices; the kernel returns at once when active is non-null and *active == 0)
int launch_sigma3_tc(fci_ctx *ctx, const float *C, float *sig, int nsplit, cudaStream_t s,
                     const int *active = nullptr);
int prepare_sigma3_tc(const fci_ctx *ctx, int nsplit);
int launch_same_spin_tc(fci_ctx *ctx, const float *C, float *sig, const SpinTables &R, const SpinTables &cols,
                        cudaStream_t s);
size_t sigma3_tc_smem(const fci_ctx *ctx, int nsplit);
int launch_wait_timeout_probe(fci_ctx *ctx);  // fci_check_wait_timeout

// sigma3_sliced.cu (FP64-accurate sigma_3 on the tensor cores)
int build_sliced_tables(fci_ctx *ctx, const double *h1_host, const double *eri_host);
void free_sliced_tables(fci_ctx *ctx);
bool sigma3_sliced_ok(const fci_ctx *ctx);
int launch_sigma3_sliced(fci_ctx *ctx, const double *C, double *sig, cudaStream_t s, int rec, int prof_slot,
                         const int *active = nullptr, int add = 0);
int prepare_sigma3_sliced(const fci_ctx *ctx);

// sigma_wide.cu (FP64-accurate sigma for large spaces: all three terms on the
// tensor cores, one integer accumulator)
bool sigma_wide_fits(const fci_ctx *ctx);
bool sigma_wide_ok(const fci_ctx *ctx);
int build_wide_tables(fci_ctx *ctx, const double *h1_host, const double *eri_host);
void free_wide_tables(fci_ctx *ctx);
int launch_sigma_f64_wide(fci_ctx *ctx, const double *C, double *sig, cudaStream_t s, int parity = 0);

// sigma_ss.cu (FP64 sigma_1 / sigma_2 as dense sliced tensor-core products)
bool sigma_ss_ok(const fci_ctx *ctx);
int build_ss_tables(fci_ctx *ctx);
void free_ss_tables(fci_ctx *ctx);
// sigma += sigma_1 (which & 1) then sigma_2 (which & 2); profiling slots slot, slot + 1
int launch_sigma_ss(fci_ctx *ctx, const double *C, double *sig, int which, cudaStream_t s, int rec, int slot);

// davidson.cu
int run_davidson(fci_ctx *ctx, int nroots, double tol, double *energies, void *vecs, const void *guess);

// rdm.cu
int run_rdm1(fci_ctx *ctx, const void *c, int dtype, double *gamma);
// rdm2.cu
int run_rdm2(fci_ctx *ctx, const void *c, int dtype, double *gamma1, double *gamma2);

inline unsigned ceil_div(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

// Opt a kernel in to the device's largest dynamic shared memory (the opt-in
// maximum less the kernel's static shared memory).  The attribute is only an
// upper bound, and one value serves every launch of the kernel, including
// launches captured in graphs while other contexts use the same kernel.
inline cudaError_t opt_in_max_smem(const void *kern, int device) {
    int lim = 0;
    cudaError_t e = cudaDeviceGetAttribute(&lim, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, kern)) != cudaSuccess) return e;
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, lim - (int)fa.sharedSizeBytes);
}

}  // namespace fci
