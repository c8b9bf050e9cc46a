/*
 * fci.h -- C ABI of the GB300 determinant-CI sigma library.
 *
 * The library computes, on one CUDA device, the sigma vector of direct
 * determinant CI, sigma = H c (arXiv 1707.04346, Section 2.1, Eq. 4-5), with
 * the spin-free Hamiltonian of Eq. 6 over Slater determinants factorised into
 * alpha and beta strings (Eq. 2), and the Davidson eigensolver around it
 * (Section 3.3).  All compute runs in the library's own CUDA kernels; there is
 * no CPU fallback.  Every call returns an int status (FCI_OK on success).  On
 * failure fci_last_error() returns a message for the calling thread.
 *
 * Conventions shared by every call:
 *  - Orbitals are real; h1 is norb x norb row-major, symmetric; eri is the
 *    chemist-notation tensor (ij|kl) as norb^4 row-major doubles with the
 *    8-fold permutational symmetry.  Eq. 6 has no core energy and neither do
 *    the energies returned here.
 *  - Strings of one spin are listed in ascending bitmask order (bit p =
 *    orbital p); the address of a string p0 < p1 < ... is sum_m C(p_m, m+1).
 *  - A determinant is alpha(Ia) beta(Ib)|vac> with alpha creators to the left
 *    (Eq. 2); CI vectors are row-major N_alpha x N_beta matrices (Eq. 4):
 *    element Ia * N_beta + Ib.
 *  - Vectors passed as `const void*` / `void*` are DEVICE pointers owned by
 *    the caller, unless the parameter says "host".
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Stream-ordered calls return before the work has finished.
 */
#ifndef FCI_GB300_H
#define FCI_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define FCI_OK 0
#define FCI_ERR_ARG 1     /* invalid argument (sizes, symmetry, null pointer) */
#define FCI_ERR_OOM 2     /* device allocation failed */
#define FCI_ERR_CUDA 3    /* a CUDA call or kernel launch failed */
#define FCI_ERR_NOCONV 4  /* Davidson reached max_iter; best energies filled */
#define FCI_ERR_TIMEOUT 5 /* a bounded device wait gave up */
#define FCI_ERR_STATE 6   /* call not valid in the context's current state */
#define FCI_ERR_NAN 7     /* non-finite value detected in an input or result */
#define FCI_ERR_RANGE 8   /* a level sum of the wide FP64 tensor-core sigma left the range in
                             which it is exact (needs C and integral digits aligned across
                             more than 73 replacements; detected, never silent) */

/* ---- element types of CI vectors --------------------------------------- */
#define FCI_F64 0
#define FCI_F32 1

/* ---- precision modes for the Davidson driver --------------------------- */
#define FCI_PREC_FP64 0  /* every sigma in FP64 */
#define FCI_PREC_MIXED 1 /* FP32 sigma for new vectors, FP64 sigma only at refinement points */

/* ---- fci_query selectors ------------------------------------------------ */
#define FCI_Q_NDET 1          /* N_alpha * N_beta */
#define FCI_Q_NSTR_ALPHA 2
#define FCI_Q_NSTR_BETA 3
#define FCI_Q_NSINGLE_ALPHA 4 /* replacement-list entries per alpha string */
#define FCI_Q_NSINGLE_BETA 5
#define FCI_Q_NPAIR 6         /* norb (norb + 1) / 2 */
#define FCI_Q_DEVICE_BYTES 7  /* device memory held by the context */
#define FCI_Q_ITERATIONS 8    /* iterations of the last fci_davidson call */
#define FCI_Q_SIGMA_CALLS 9   /* sigma builds done inside the last fci_davidson */
#define FCI_Q_DEVICE_ERROR 10 /* device error word (blocking read; the word is then cleared):
                                 bit 0 = a bounded wait inside a kernel gave up, bit 1 = a
                                 level sum of the wide FP64 sigma left its exact range */

typedef struct fci_ctx fci_ctx;

typedef struct fci_options {
    int struct_size;     /* set to sizeof(fci_options) */
    int device;          /* CUDA device ordinal; -1 = the current device */
    int max_subspace;    /* Davidson subspace limit in vectors (default 24) */
    int max_iter;        /* Davidson iteration limit (default 300) */
    int precision;       /* FCI_PREC_FP64 (default) or FCI_PREC_MIXED */
    double mixed_switch; /* MIXED: residual reduction between FP64 refinements (default 1e-2) */
    double symmetry_tol; /* absolute tolerance of the h1/eri symmetry check (default 1e-12) */
    int f32_splits;      /* FCI_F32 sigma_3 on the tensor cores: FP32 operands split into 2
                            (split-BF16x3, ~1e-5 relative) or 3 (split-BF16x6, ~FP32) bf16
                            slices; default 3 */
    int same_spin_tc;    /* FCI_F32 sigma_1 and sigma_2 through intermediate strings on the
                            tensor cores (Eq. 8's E_ij E_kl as a pair-matrix contraction):
                            0 = only when the staged same-spin kernels do not fit in shared
                            memory (default), 1 = always */
    int f64_kernels;     /* FCI_F64 sigma kernels: FCI_F64_AUTO (default), FCI_F64_FMA,
                            FCI_F64_SLICED or FCI_F64_WIDE, below */
    double max_device_bytes; /* cap on the device memory one context (with its Davidson
                            workspace) may hold; an allocation beyond it fails with
                            FCI_ERR_OOM before cudaMalloc is called.  0 = no cap (default).
                            (Resource control; no counterpart in the paper.) */
    int f32_row_global;  /* FCI_F32 tensor-core sigma_3: 1 = keep the sigma row in global
                            memory (the epilogue large spaces such as CAS(18,18) need) even
                            where it fits in shared memory, so that small spaces exercise
                            it; 0 = shared memory where it fits (default) */
    int basis_f32;       /* FCI_PREC_MIXED Davidson: store the subspace basis and its sigma
                            vectors in FP32 (Ritz vectors and refinement sigma stay FP64).
                            0 = only when the FP64 basis does not fit in free device memory
                            (default; then at most 8 vectors, fewer if memory asks), 1 =
                            always (max_subspace vectors), 2 = never */
    int spin_parity;     /* Davidson on the Ms = 0 combinations of one spin parity
                            (n_alpha = n_beta): +1 = C^T = C (S even: singlets,
                            quintets, ...), -1 = C^T = -C (S odd: triplets, ...), 0 = all
                            states (default).  The guess and every correction are
                            projected onto the parity, and sigma_1 = parity sigma_2^T is
                            formed from sigma_2 by a transpose-add (Section 3.1's Ms = 0
                            combinations); fci_sigma itself is unaffected */
    int f64_same_spin;   /* FCI_F64 sigma_1 and sigma_2 with the tensor-core sigma_3:
                            FCI_SS_AUTO (default) as dense sliced products on the tensor cores
                            (below) when both string spaces hold at most 16384 strings,
                            FCI_SS_FAMILY the same-spin kernels of the f64_kernels family
                            (double-float next to the per-row sigma_3, intermediate strings
                            next to the wide kernels) */
    double rdm2_chunk_bytes; /* fci_rdm2: device memory for the digit planes of one chunk of
                            determinants (about 192 (norb^2 + 1) bytes per 16 determinants
                            per chunk); 0 = 1 GiB (default).  (Resource control; no
                            counterpart in the paper.) */
} fci_options;

/* fci_options.f64_same_spin.  FCI_SS_AUTO computes sigma_1 = C G_b^T and
 * sigma_2 = G_a C with the dense same-spin Hamiltonians G_s (the one-spin part
 * of Eq. 6 between the strings of one spin, zeros included) on the bf16
 * tensor cores: every row of G_s and every row or column of C in 46-bit fixed
 * point relative to its own largest power of two, six 8-bit digits, exact
 * 64-bit integer sums; the diagonal of G_s in FP64.  Costs 12 bytes per
 * element of each G_s (141 MB at CAS(14,14), 2 GB at CAS(16,16)) at fci_init
 * and the same for two copies of C.  The results are bit-reproducible. */
#define FCI_SS_AUTO 0
#define FCI_SS_FAMILY 1

/* fci_options.f64_kernels: how the FCI_F64 sigma is computed.  All modes meet
 * the FP64 accuracy of Eq. 4-8's direct sum (the tests hold each to the same
 * 1e-12 bars).
 *  FCI_F64_FMA     FP64 fused multiply-adds throughout (GB300's FP64 pipe).
 *  FCI_F64_AUTO    sigma_3 on the bf16 tensor cores from 8-bit slices where the
 *                  space fits the per-row sliced kernel (CAS(14,14)), else,
 *                  when both spins have electrons, through the wide kernels
 *                  (CAS(16,16), CAS(18,18)); sigma_1 and sigma_2 next to either
 *                  as dense sliced products on the tensor cores where each
 *                  string space holds at most 16384 strings (fci_options.
 *                  f64_same_spin), else with the family's own kernels:
 *                  double-float FP32 arithmetic next to the per-row sigma_3
 *                  (each FP64 value as two FP32 parts, 48 significant bits;
 *                  error-free products and sums to within a few units of
 *                  2^-48), intermediate strings next to the wide sigma_3;
 *                  where neither tensor-core sigma_3 applies, FP64 FMAs.
 *  FCI_F64_SLICED  as AUTO, but fci_init fails with FCI_ERR_ARG where neither
 *                  tensor-core FP64 path fits.
 *  FCI_F64_WIDE    the wide kernels on every space they cover (FCI_ERR_ARG
 *                  elsewhere); lets small spaces exercise the large-space path.
 * The sliced kernels write C and the integrals as 47-bit fixed point, cut
 * into six balanced 8-bit digits that bf16 holds exactly, and accumulate the
 * 21 digit products of weight <= 5 per weight in FP32 (exact for weights
 * 0-2); their adds into sigma are 64-bit integers, so the result does not
 * depend on the order of the adds.  The per-row kernel takes C relative to
 * one power of two per alpha row and holds the sigma row in shared memory:
 * at most 128 orbital pairs (norb <= 15), 85 alpha replacements, and the
 * sigma row (8 N_beta bytes) plus 12 (128 + npair) K bytes of operands in
 * shared memory.  The wide kernels take C relative to one power of two for
 * the whole vector (errors are relative to max|C|), cut the pair columns into
 * parts of at most 64, and accumulate in global memory; the same-spin terms
 * go through intermediate strings (1/2 sum (ij|kl) E_ij E_kl with the
 * identity resolved over single replacements, plus the one-body operator
 * k_kl = h_kl - 1/2 sum_j (kj|jl)).  Limits: at most 96 replacements per
 * string and 255 orbital pairs (norb <= 21); 20 bytes per determinant of
 * workspace (12 of digit planes, 8 of accumulator, shared with the FCI_F32
 * same-spin workspace). */
#define FCI_F64_AUTO 0
#define FCI_F64_FMA 1
#define FCI_F64_SLICED 2
#define FCI_F64_WIDE 3

/* Fill *opt with the defaults listed above. */
void fci_default_options(fci_options *opt);

/*
 * Create a context for CAS(n_alpha + n_beta electrons, norb orbitals).
 *
 * Builds on the device, once: the alpha and beta string lists (Eq. 2), the
 * single-replacement lists E_kl with signs (Eq. 7), the same-spin string
 * Hamiltonians used by sigma_1 / sigma_2 (Eq. 8), the packed pair matrix of
 * two-electron integrals used by sigma_3, and the determinant diagonal.
 *
 *  ctx      out: new context (free with fci_free)
 *  norb     1..30
 *  nalpha,nbeta  0..norb; the string counts must stay below 2^21
 *  h1, eri  HOST pointers, copied in; the caller keeps ownership
 *  opt      may be NULL (defaults)
 * Errors: FCI_ERR_ARG (sizes, NULL pointers, or h1/eri not symmetric within
 * opt->symmetry_tol, or non-finite values), FCI_ERR_OOM, FCI_ERR_CUDA.
 * Blocking.
 */
int fci_init(fci_ctx **ctx, int norb, int nalpha, int nbeta, const double *h1, const double *eri,
             const fci_options *opt);

/* Release every device buffer of the context.  NULL is accepted.  (Resource
 * management; no counterpart in the paper.) */
int fci_free(fci_ctx *ctx);

/*
 * The short form fci_init(norb, nalpha, nbeta, h1, eri): one context held by
 * the library, built with the default options (fci_default_options) on the
 * current device.  fci_init_default builds it, first freeing any earlier
 * default context; fci_default_context returns it (NULL when none), for use
 * with every other call; fci_free_default frees it (also when none exists).
 * Arguments and errors as fci_init; on an error no default context remains.
 * The three calls are serialised by a lock; calls that use the default
 * context while another thread replaces or frees it are the caller's race.
 * (Interface convenience; no counterpart in the paper.)
 */
int fci_init_default(int norb, int nalpha, int nbeta, const double *h1, const double *eri);
fci_ctx *fci_default_context(void);
int fci_free_default(void);

/*
 * sigma = H c (Eq. 4-5), computed as sigma_1 + sigma_2 + sigma_3 (Eq. 8):
 * beta-beta, alpha-alpha and alpha-beta parts.
 *
 *  c, sigma  device vectors of N = N_alpha * N_beta elements of type dtype
 *            (FCI_F64 or FCI_F32); must not overlap.  sigma is overwritten.
 *  dtype     FCI_F64: FP64 vectors and FP64 accuracy (fci_options.f64_kernels
 *            and f64_same_spin say which kernels: tensor-core contractions of
 *            8-bit digit slices with exact integer sums, double-float FP32
 *            arithmetic, or FP64 FMAs).  FCI_F32: FP32 vectors;
 *            sigma_1/sigma_2 in FP32, sigma_3 on the tensor cores with bf16
 *            slices of the FP32 operands and FP32 accumulation (see
 *            fci_options.f32_splits); the low-precision phase of the mixed
 *            Davidson.  For large string spaces (or with
 *            fci_options.same_spin_tc = 1) sigma_1/sigma_2 also run on the
 *            tensor cores, through intermediate strings (Eq. 7 operators
 *            E_ij E_kl); their adds are atomic, so FP32 results may differ in
 *            the last bits between calls.  FCI_F32 needs the replacement lists
 *            of both spins to have at most 96 entries (norb 18 at half
 *            filling) and at most 65408 strings per spin; FCI_F64 covers
 *            every space with at most 96 replacements per string and 255
 *            orbital pairs on the tensor cores (CAS(18,18) included), beyond
 *            that the FMA kernels, which need one beta row of C and sigma
 *            (2 N_beta doubles) in shared memory.
 *  stream    cudaStream_t or NULL.  Asynchronous; allocates nothing (the
 *            workspaces of the large-space FP32 path, 8N bytes, of the sliced
 *            FP64 sigma_3, 12N bytes, and of the dense same-spin products,
 *            24N bytes, are made at fci_init), so it can be captured in a
 *            CUDA graph.  The context's workspaces are shared
 *            by its calls: fci_sigma calls on one context must not overlap in
 *            time (issue them on one stream, or order the streams).
 * Errors: FCI_ERR_ARG (including the size limits above, reported on the host
 * before any launch), FCI_ERR_OOM, FCI_ERR_CUDA (launch failure).
 */
int fci_sigma(fci_ctx *ctx, const void *c, void *sigma, int dtype, void *stream);

/* Copy the FP64 determinant diagonal H_II of Eq. 6 (N elements) to device
 * memory `out`: the diagonal preconditioner of Section 3.3 step (2).
 * Stream-ordered.  Errors: FCI_ERR_ARG, FCI_ERR_CUDA. */
int fci_hdiag(fci_ctx *ctx, double *out, void *stream);

/*
 * Davidson eigensolver (Section 3.3) for the lowest nroots eigenpairs.
 *
 *  nroots    1..8
 *  tol       energy convergence threshold (Eh); also ||r|| < sqrt(tol)
 *  energies  HOST array [nroots], ascending, filled on return (also on
 *            FCI_ERR_NOCONV, with the last Ritz values)
 *  vecs      NULL, or DEVICE FP64 [nroots][N]: normalised eigenvectors
 *  guess     NULL (unit vectors on the lowest diagonal elements), or DEVICE
 *            FP64 [nroots][N] starting vectors
 * Uses the options given at fci_init (max_subspace, max_iter, precision,
 * basis_f32, spin_parity: with a parity the guess and every correction are
 * projected onto it and the energies are those of that parity's states).
 * In FCI_PREC_MIXED with an FP32 basis (large spaces: the FP64
 * basis of CAS(18,18) would need 300 GB) the device workspace is
 * 8 (2 m + 1) / 2 + 16 nroots bytes per determinant for m basis vectors.
 * Blocking; runs on the context's internal stream.
 * Errors: FCI_ERR_ARG (also when no guess vector survives orthonormalisation,
 * e.g. all-NaN guesses), FCI_ERR_OOM, FCI_ERR_CUDA, FCI_ERR_TIMEOUT,
 * FCI_ERR_NAN (a Ritz value or residual norm became non-finite, e.g. from an
 * infinite guess entry; checked every iteration, energies not filled),
 * FCI_ERR_NOCONV.
 */
int fci_davidson(fci_ctx *ctx, int nroots, double tol, double *energies, void *vecs, const void *guess);

/*
 * Per-iteration log of the last fci_davidson call (one record per pass through
 * steps (2)-(4) of Section 3.3).  Writes up to `cap` records of (nroots + 3)
 * doubles each into HOST `out`: iteration, precision (0: every subspace sigma
 * FP64-exact, 1: FP32 sigma present), elapsed seconds since the call started,
 * then the nroots Ritz values.  Returns the number of records available via
 * *count.
 */
int fci_davidson_log(fci_ctx *ctx, double *out, int cap, int *count);

/*
 * Spin-summed one-particle density gamma_pq = <c|E_pq|c> (Eq. 7 operator),
 * the density built after the Davidson iterations (Section 4).
 *
 *  c      device vector (dtype FCI_F64 or FCI_F32) of N elements; the call
 *         first waits for all work on the device, so c may come from any stream
 *  gamma  HOST array norb x norb, row-major, filled on return (blocking)
 */
int fci_rdm1(fci_ctx *ctx, const void *c, int dtype, double *gamma);

/*
 * Spin-summed two-particle density Gamma_pqrs = <c| E_pq E_rs |c> (the
 * density of the two-electron term of Eq. 6; E_pq of Eq. 7), the second half
 * of the density step after the Davidson iterations (Section 4, Table 2's
 * "1e/2e Density Matrices").  With gamma = fci_rdm1's density,
 *   <c|H|c> = sum h_pq gamma_pq + 1/2 sum (pq|rs) (Gamma_pqrs - delta_qr gamma_ps).
 * Gamma_pqrs = sum_K <K|E_qp|c> <K|E_rs|c> over the determinants K, computed
 * as one Gram matrix on the tensor cores with FP64 accuracy (c in 45-bit fixed
 * point relative to its largest element, six 8-bit digits, exact 64-bit
 * integer accumulation): about 1e-14 of ||c||^2, bit-reproducible.  c need
 * not be normalised (both densities scale with ||c||^2).
 *
 *  c       device vector (dtype FCI_F64 or FCI_F32) of N elements; the call
 *          first waits for all work on the device
 *  gamma1  HOST array norb x norb (gamma_pq, from the same pass), or NULL
 *  gamma2  HOST array norb^4, row-major [p][q][r][s], filled on return
 * Allocates its scratch (the digit planes of one chunk of determinants, see
 * fci_options.rdm2_chunk_bytes, and (norb^2 + 1)^2 64-bit integers) per call.
 * A non-finite c gives NaN densities.  Blocking.  FCI_ERR_TIMEOUT when a
 * bounded wait inside the tensor-core kernel gave up, FCI_ERR_RANGE if an
 * exact accumulator left its range (neither is expected).
 */
int fci_rdm2(fci_ctx *ctx, const void *c, int dtype, double *gamma1, double *gamma2);

/*
 * fci_rdm1_noalloc -- the density of fci_rdm1, computed without allocating
 * any device memory.  The paper has no counterpart: this is an interface
 * convenience.
 *
 * fci_rdm1 allocates its scratch (one partial sum per replacement-list entry)
 * with cudaMalloc and releases it with cudaFree on every call.  Some callers
 * cannot do that: an application whose device memory is handed out entirely
 * by its own pool or by a framework's caching allocator, or one that keeps
 * other streams busy and cannot accept the device-wide synchronisation that
 * cudaFree implies.  This entry point serves them: it uses a fixed array in
 * the library's device memory and runs on the caller's stream.
 *
 *  c       device vector (dtype FCI_F64 or FCI_F32), ordered on `stream`
 *  gamma   HOST array norb x norb, row-major, filled on return
 *  stream  cudaStream_t or NULL; the call waits for this stream only
 *
 * Limit: N_alpha * n_single_alpha + N_beta * n_single_beta + norb^2 must not
 * exceed FCI_RDM1_NOALLOC_MAX_DOUBLES (2^21 doubles, 16 MiB: enough for
 * CAS(16,16)); larger spaces get FCI_ERR_ARG and must use fci_rdm1.
 * The array lives in every GPU that loads the library until the process
 * exits.  The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current.  The call is blocking: it
 * copies gamma to pageable host memory and synchronises `stream`, so it can
 * never be issued on a capturing stream; the one-time address lookup should
 * also come before any capture that other threads run in global capture mode.
 * The call makes ctx's device current while it runs and restores the caller's
 * current device before returning.  All calls share the one array, which keeps
 * the last call's contents: calls whose GPU work overlaps (other streams,
 * threads or contexts on the same device) race on it and corrupt each other's
 * results, so serialise them.
 */
#define FCI_RDM1_NOALLOC_MAX_DOUBLES (1 << 21)
int fci_rdm1_noalloc(fci_ctx *ctx, const void *c, int dtype, double *gamma, void *stream);

/*
 * Copy tables to the host (for checking): the string list of one spin
 * (spin 0 = alpha, 1 = beta; the strings of Eq. 2) as uint32 bitmasks
 * [N_spin], and its single-replacement lists (the E_kl of Eq. 7)
 * [N_spin][n_single]: for string X and each
 * (k, l) with l occupied and k empty or k == l, in the order l ascending
 * then k ascending, a+_k a_l |X> = sign |target>.  Any of tgt/k/l/sign may
 * be NULL.  Blocking.
 */
int fci_get_strings(fci_ctx *ctx, int spin, uint32_t *out);
int fci_get_single_table(fci_ctx *ctx, int spin, int32_t *tgt, int8_t *k, int8_t *l, int8_t *sign);

/*
 * Host only, no CUDA call: the tile schedule that the tensor-core sigma_3
 * epilogue uses for the beta-side scatter of Eq. 8 (sigma_3(I_a, I_b) gets
 * sign * G(J_b) for every I_b = E_kl J_b), built by the routine fci_init runs
 * on the beta table, from a single-replacement table in host memory.
 *  ns, nsingle  strings and entries per string (1 <= ns <= 65408,
 *               1 <= nsingle <= 1024)
 *  npair        number of packed orbital pairs (1..256); pair index of (k, l)
 *               is max*(max+1)/2 + min
 *  tgt, pair, sign  row-major [ns][nsingle] (tgt in [0, ns), pair in
 *               [0, npair), sign +1 or -1), the layout fci_get_single_table
 *               returns; entry order within a row does not matter
 *  sched, cap   output records, uint32: target | (source string - 128 t) << 16
 *               | pair << 23 | (sign < 0) << 31.  Strings form tiles of 128
 *               (t = x / 128); each tile's entries are grouped by target and
 *               every target's entries go whole to one of 128 shares, so no
 *               two shares of a tile write the same target; entry j of share k
 *               of tile t is sched[toff[t] + 128 j + k], and shorter shares
 *               are padded with the dummy target ns + k.  Written only when
 *               sched != NULL and cap >= *nsched.
 *  nsched       out: schedule length (call once with sched = NULL to size it)
 *  toff         out (nullable): [ceil(ns/128) + 1] offsets of the tiles
 * Returns FCI_ERR_ARG for NULL inputs, sizes out of range, an entry out of
 * range or a schedule longer than 2^31 records (degenerate tables with very
 * long rows), FCI_ERR_OOM when host memory runs out; nothing is written then.  fci_init builds no schedule in that
 * case, and the tensor-core sigma_3 refuses the space.
 */
int fci_tile_schedule(int64_t ns, int nsingle, int npair, const int32_t *tgt, const int32_t *pair,
                      const int8_t *sign, uint32_t *sched, int64_t cap, int64_t *nsched, int32_t *toff);

/*
 * Per-kernel timing (tracing; no counterpart in the paper, whose tables give
 * per-step wall times).  While enabled, every fci_sigma call records
 * CUDA events on the caller's stream around each kernel it launches (no
 * synchronisation; the events go into a ring of 1024 records).
 * fci_profile_read waits for the recorded events and returns, per record,
 * the elapsed milliseconds of each kernel, row-major [nrecords][nkernels],
 * oldest first (at most cap_records), then empties the ring.
 * fci_profile_kernel_name names kernel slot i of the current sigma pipeline
 * (NULL if out of range).  Enabling allocates the events (FCI_ERR_CUDA on
 * failure); disabling keeps them for reuse.
 */
int fci_profile_enable(fci_ctx *ctx, int on);
int fci_profile_read(fci_ctx *ctx, double *ms, int cap_records, int *nrecords, int *nkernels);
const char *fci_profile_kernel_name(fci_ctx *ctx, int i);

/* ---- batched CASCI ------------------------------------------------------
 *
 * Many independent CASCI problems solved together, the single-GPU analogue
 * of the paper's many TTSS batches distributed over processors (Section 3.1):
 * all instances advance through the Davidson iterations of Section 3.3 in
 * lock-step, every vector operation is one launch over all instances, and the
 * sigma vectors of all instances come from one persistent kernel that pulls
 * (instance, alpha-row group) work items, largest instances first, from a
 * device queue.  The per-iteration kernel sequences are captured in CUDA
 * graphs.  Threads per alpha row are chosen per (norb, precision) by timing
 * the candidates {32, 64, 128, 256} on the first instance of each size at
 * fci_batch_init (the tuning table is readable with fci_batch_tuning).
 */
typedef struct fci_instance {
    int norb, nalpha, nbeta;  /* as in fci_init (norb <= 16 here) */
    const double *h1;         /* HOST, norb x norb */
    const double *eri;        /* HOST, norb^4 */
} fci_instance;

typedef struct fci_batch fci_batch;

/*
 * Build the tables of every instance and tune the sigma kernel.
 *  opt: precision FCI_PREC_FP64 (FP64 sigma) or FCI_PREC_MIXED (FP32 sigma for
 *       new vectors, FP64 refinement as in fci_davidson); max_subspace,
 *       max_iter and mixed_switch as for fci_davidson.
 * Errors: FCI_ERR_ARG (ninst < 1, a bad instance, norb > 16), FCI_ERR_OOM,
 * FCI_ERR_CUDA.  Blocking.
 */
int fci_batch_init(fci_batch **batch, int ninst, const fci_instance *inst, const fci_options *opt);

/*
 * Lowest nroots eigenvalues of every instance by the Davidson steps of
 * Section 3.3, all instances in lock-step; energies is HOST
 * [ninst][nroots].  Returns FCI_ERR_NOCONV if any instance did not converge
 * within max_iter (all energies are still filled).  Blocking.
 */
int fci_batch_davidson(fci_batch *batch, int nroots, double tol, double *energies);

/*
 * sigma (Eq. 4, split as Eq. 8) for every instance at once: c and sigma are
 * DEVICE vectors holding
 * the instances' CI vectors back to back (instance i at offset
 * fci_batch_offset(batch, i)), dtype FCI_F64 or FCI_F32.  Stream-ordered.
 */
int fci_batch_sigma(fci_batch *batch, const void *c, void *sigma, int dtype, void *stream);

/* Offset of instance i in a batch vector; i == ninst gives the total length.
 * (The following batch queries are bookkeeping with no counterpart in the
 * paper.) */
int64_t fci_batch_offset(fci_batch *batch, int i);

/* Tuning table: for each distinct (norb, dtype) writes norb, dtype and the
 * chosen threads per row into HOST `out` (3 ints per entry, up to cap
 * entries); *count receives the number of entries. */
int fci_batch_tuning(fci_batch *batch, int *out, int cap, int *count);

/* Iterations and sigma launches of the last fci_batch_davidson: what = 0
 * iterations (of the slowest instance), 1 batched sigma launches issued
 * (instances masked off skip them on the device), 2 graph launches (one per
 * chunk of up to 8 iterations), 3 host synchronisations (one per chunk: the
 * convergence, refinement and expansion decisions are made on the device). */
int64_t fci_batch_stats(fci_batch *batch, int what);

int fci_batch_free(fci_batch *batch);

/*
 * Self-test of the failure path of the bounded device waits (no counterpart in
 * the paper).  Every mbarrier wait inside the tensor-core sigma kernels gives
 * up after a fixed number of polls, sets the context's device error word and
 * lets the kernel drain and exit, so that a stalled pipeline is reported
 * instead of hanging the GPU.  This call runs one block that waits, through the
 * same bounded-wait routine, on a barrier no thread arrives on; the wait gives
 * up (well under a second on GB300), and the call reads and clears the error
 * word and returns FCI_ERR_TIMEOUT, as fci_davidson does after a sigma whose
 * wait gave up.  The context stays usable.  Blocking; runs on the context's
 * internal stream.  Returns FCI_OK only if the wait did not give up (which
 * would mean the routine is broken).
 */
int fci_check_wait_timeout(fci_ctx *ctx);

/* Sizes and counters (FCI_Q_*); returns -1 for an unknown selector.  (No
 * counterpart in the paper.) */
int64_t fci_query(fci_ctx *ctx, int what);

/* Message of the last failed call on this thread ("" if none).  (Error
 * reporting; no counterpart in the paper.) */
const char *fci_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FCI_GB300_H */
