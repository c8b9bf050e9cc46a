/*
 * FP64 CPU oracle for determinant CI (arXiv 1707.04346, Section 2.1).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path may call,
 * link or load this file; it exists so that tests, the smoke check and the
 * benchmark's CPU-baseline leg can compare the CUDA path against a plain,
 * slow, obviously correct implementation.  It shares no code with the CUDA
 * sources.
 *
 * Conventions (the paper leaves them open; the readings are stated here):
 *  - A determinant is alpha(I_a) beta(I_b)|vac> (Eq. 2): all alpha creators
 *    stand to the left of all beta creators, and inside a string creators are
 *    in ascending orbital order.  In this file a determinant is a 64-bit
 *    spin-orbital mask: bit p (p < norb) is alpha orbital p, bit norb + p is
 *    beta orbital p, and the canonical creator order is ascending bit index.
 *  - Strings of one spin are listed in ascending bitmask order; a string's
 *    address is its position in that list (found here by binary search).
 *  - Determinant index = I_a * N_b + I_b (C stored as a row-major matrix,
 *    Eq. 4).
 *  - The Hamiltonian is Eq. 6 with real orbitals and chemist-notation
 *    integrals (ij|kl); no core energy.
 *
 * Functions:
 *  oracle_strings        string list (Eq. 2 strings), ascending bitmask order
 *  oracle_single_table   E_kl single-replacement lists with signs (Eq. 7)
 *  oracle_h_slater       explicit H by the Slater-Condon rules (Eq. 6)
 *  oracle_h_operator     explicit H by applying Eq. 6 literally to bitstrings
 *  oracle_sigma_rows     sigma(I) = sum_J H_IJ c_J for chosen I (Eq. 4/5)
 *  oracle_sigma_rows_gen the same with c_J = 2 u_J - 1 regenerated per index
 *  oracle_sigma          the same for every I (OpenMP over I)
 *  oracle_hdiag          H_II
 *  oracle_rdm1           spin-summed one-particle density <c|E_pq|c>
 *  oracle_rdm2           spin-summed two-particle density <c|E_pq E_rs|c>
 *  oracle_s2             <c|S^2|c> / <c|c> (total spin of an expansion)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef uint64_t det_t;

static int popc64(uint64_t x) { return __builtin_popcountll(x); }

int64_t oracle_binom(int n, int k) {
    if (k < 0 || k > n) return 0;
    int64_t r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

/* All ne-subsets of norb orbitals, ascending as integers.  Returns count. */
int64_t oracle_strings(int norb, int ne, uint32_t *out) {
    if (norb < 0 || norb > 30 || ne < 0 || ne > norb) return -1;
    int64_t cnt = 0;
    uint64_t lim = (uint64_t)1 << norb;
    for (uint64_t m = 0; m < lim; ++m)
        if (popc64(m) == ne) {
            if (out) out[cnt] = (uint32_t)m;
            ++cnt;
        }
    return cnt;
}

/* Address of mask in the ascending list (binary search); -1 if absent. */
static int64_t address_of(const uint32_t *list, int64_t ns, uint32_t mask) {
    int64_t lo = 0, hi = ns - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        if (list[mid] == mask) return mid;
        if (list[mid] < mask) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* ---- creation / annihilation on a spin-orbital mask -------------------- */
/* a_p |m>: returns 0 if p is empty, else sign (+1/-1), writes result. */
static int op_annihilate(det_t m, int p, det_t *out) {
    if (!((m >> p) & 1ULL)) return 0;
    int s = (popc64(m & (((det_t)1 << p) - 1)) & 1) ? -1 : 1;
    *out = m & ~((det_t)1 << p);
    return s;
}
static int op_create(det_t m, int p, det_t *out) {
    if ((m >> p) & 1ULL) return 0;
    int s = (popc64(m & (((det_t)1 << p) - 1)) & 1) ? -1 : 1;
    *out = m | ((det_t)1 << p);
    return s;
}
/* a+_p a_q |m> */
static int op_excite(det_t m, int p, int q, det_t *out) {
    det_t t;
    int s1 = op_annihilate(m, q, &t);
    if (!s1) return 0;
    int s2 = op_create(t, p, out);
    return s1 * s2;
}

/* ---- Single-replacement table ------------------------------------------ *
 * For string X and each (k, l) with l in X and (k not in X or k == l), in the
 * order: l ascending over occupied orbitals, then k ascending over 0..norb-1:
 *   target = address(X - l + k), sign from a+_k a_l applied to the string.
 * Per string there are ne*(norb-ne) + ne entries.  Returns entries/string.  */
int oracle_single_table(int norb, int ne, int32_t *tgt, int8_t *kk, int8_t *ll, int8_t *sg) {
    int64_t ns = oracle_binom(norb, ne);
    uint32_t *list = (uint32_t *)malloc(sizeof(uint32_t) * (ns ? ns : 1));
    oracle_strings(norb, ne, list);
    int per = ne * (norb - ne) + ne;
    for (int64_t x = 0; x < ns; ++x) {
        int e = 0;
        for (int l = 0; l < norb; ++l) {
            if (!((list[x] >> l) & 1u)) continue;
            for (int k = 0; k < norb; ++k) {
                if (k != l && ((list[x] >> k) & 1u)) continue;
                det_t y;
                int s = op_excite(list[x], k, l, &y);
                int64_t at = x * per + e;
                tgt[at] = (int32_t)address_of(list, ns, (uint32_t)y);
                kk[at] = (int8_t)k;
                ll[at] = (int8_t)l;
                sg[at] = (int8_t)s;
                ++e;
            }
        }
    }
    free(list);
    return per;
}

/* ---- Slater-Condon matrix elements ------------------------------------- */
typedef struct {
    int norb;
    const double *h;   /* [n][n] */
    const double *eri; /* [n][n][n][n] chemist (ij|kl) */
} ham_t;

static inline double H1(const ham_t *H, int p, int q) { return H->h[p * H->norb + q]; }
static inline double ERI(const ham_t *H, int i, int j, int k, int l) {
    int n = H->norb;
    return H->eri[((i * n + j) * n + k) * n + l];
}
/* spin-orbital -> spatial orbital and spin */
static inline int sp(const ham_t *H, int p) { return p % H->norb; }
static inline int spin(const ham_t *H, int p) { return p / H->norb; }

/* physicist <pq|rs> over spin orbitals = (pr|qs) delta(sp,sr) delta(sq,ss) */
static double phys(const ham_t *H, int p, int q, int r, int s) {
    if (spin(H, p) != spin(H, r) || spin(H, q) != spin(H, s)) return 0.0;
    return ERI(H, sp(H, p), sp(H, r), sp(H, q), sp(H, s));
}

static double sc_diag(const ham_t *H, det_t m) {
    int occ[64], no = 0;
    for (int p = 0; p < 2 * H->norb; ++p)
        if ((m >> p) & 1ULL) occ[no++] = p;
    double e = 0.0;
    for (int a = 0; a < no; ++a) e += H1(H, sp(H, occ[a]), sp(H, occ[a]));
    for (int a = 0; a < no; ++a)
        for (int b = 0; b < no; ++b)
            e += 0.5 * (phys(H, occ[a], occ[b], occ[a], occ[b]) - phys(H, occ[a], occ[b], occ[b], occ[a]));
    return e;
}

/* <I|H|J> for two determinants of the same particle numbers. */
static double sc_element(const ham_t *H, det_t I, det_t J) {
    if (I == J) return sc_diag(H, I);
    det_t out = J & ~I; /* occupied in J, empty in I: annihilated */
    det_t in = I & ~J;  /* created */
    int nd = popc64(out);
    if (nd != popc64(in) || nd > 2) return 0.0;
    int n2 = 2 * H->norb;
    if (nd == 1) {
        int i = __builtin_ctzll(out), a = __builtin_ctzll(in);
        if (spin(H, i) != spin(H, a)) return 0.0;
        det_t t;
        int ph = op_excite(J, a, i, &t);
        double v = H1(H, sp(H, a), sp(H, i));
        for (int k = 0; k < n2; ++k) {
            if (!((J >> k) & 1ULL) || k == i) continue;
            v += phys(H, a, k, i, k) - phys(H, a, k, k, i);
        }
        return ph * v;
    }
    /* double: i<j annihilated, a<b created; pair i->a and j->b */
    int i = __builtin_ctzll(out);
    int j = 63 - __builtin_clzll(out);
    int a = __builtin_ctzll(in);
    int b = 63 - __builtin_clzll(in);
    det_t t1, t2;
    int ph1 = op_excite(J, b, j, &t1);
    int ph2 = op_excite(t1, a, i, &t2);
    if (!ph1 || !ph2 || t2 != I) return 0.0;
    return ph1 * ph2 * (phys(H, a, b, i, j) - phys(H, a, b, j, i));
}

static det_t make_det(int norb, uint32_t a, uint32_t b) { return (det_t)a | ((det_t)b << norb); }

typedef struct {
    int norb, na, nb;
    int64_t nsa, nsb;
    uint32_t *la, *lb;
} space_t;

static int space_init(space_t *S, int norb, int na, int nb) {
    if (norb < 1 || norb > 30 || na < 0 || nb < 0 || na > norb || nb > norb) return -1;
    S->norb = norb; S->na = na; S->nb = nb;
    S->nsa = oracle_binom(norb, na);
    S->nsb = oracle_binom(norb, nb);
    S->la = (uint32_t *)malloc(sizeof(uint32_t) * S->nsa);
    S->lb = (uint32_t *)malloc(sizeof(uint32_t) * S->nsb);
    oracle_strings(norb, na, S->la);
    oracle_strings(norb, nb, S->lb);
    return 0;
}
static void space_free(space_t *S) { free(S->la); free(S->lb); }

/* Explicit H (N x N, row-major) by the Slater-Condon rules. */
int oracle_h_slater(int norb, int na, int nb, const double *h, const double *eri, double *Hout) {
    space_t S;
    if (space_init(&S, norb, na, nb)) return -1;
    ham_t H = {norb, h, eri};
    int64_t N = S.nsa * S.nsb;
#pragma omp parallel for schedule(dynamic)
    for (int64_t I = 0; I < N; ++I) {
        det_t dI = make_det(norb, S.la[I / S.nsb], S.lb[I % S.nsb]);
        for (int64_t J = 0; J < N; ++J) {
            det_t dJ = make_det(norb, S.la[J / S.nsb], S.lb[J % S.nsb]);
            Hout[I * N + J] = sc_element(&H, dI, dJ);
        }
    }
    space_free(&S);
    return 0;
}

/* Explicit H by applying Eq. 6 term by term to every basis determinant:
 *   H = sum_kl h_kl E_kl + 1/2 sum_ijkl (ij|kl) (E_ij E_kl - delta_jk E_il),
 *   E_kl = a+_{k alpha} a_{l alpha} + a+_{k beta} a_{l beta}   (Eq. 7).
 * Column J of H is H|J>.                                                   */
static int64_t det_index(const space_t *S, det_t m) {
    uint32_t mask = (1u << S->norb) - 1u;
    uint32_t a = (uint32_t)(m & mask), b = (uint32_t)((m >> S->norb) & mask);
    int64_t ia = address_of(S->la, S->nsa, a), ib = address_of(S->lb, S->nsb, b);
    if (ia < 0 || ib < 0) return -1;
    return ia * S->nsb + ib;
}
/* E_kl |m>: up to two determinants (alpha part, beta part). */
static int apply_E(int norb, int k, int l, det_t m, det_t out[2], int sgn[2]) {
    int c = 0;
    for (int s = 0; s < 2; ++s) {
        det_t t;
        int ph = op_excite(m, k + s * norb, l + s * norb, &t);
        if (ph) { out[c] = t; sgn[c] = ph; ++c; }
    }
    return c;
}

int oracle_h_operator(int norb, int na, int nb, const double *h, const double *eri, double *Hout) {
    space_t S;
    if (space_init(&S, norb, na, nb)) return -1;
    int n = norb;
    int64_t N = S.nsa * S.nsb;
    memset(Hout, 0, sizeof(double) * N * N);
#pragma omp parallel for schedule(dynamic)
    for (int64_t J = 0; J < N; ++J) {
        det_t dJ = make_det(n, S.la[J / S.nsb], S.lb[J % S.nsb]);
        det_t o1[2], o2[2];
        int s1[2], s2[2];
        for (int k = 0; k < n; ++k)
            for (int l = 0; l < n; ++l) {
                int c1 = apply_E(n, k, l, dJ, o1, s1);
                for (int u = 0; u < c1; ++u) {
                    int64_t I = det_index(&S, o1[u]);
                    Hout[I * N + J] += h[k * n + l] * s1[u];
                }
            }
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j)
                for (int k = 0; k < n; ++k)
                    for (int l = 0; l < n; ++l) {
                        double g = eri[((i * n + j) * n + k) * n + l];
                        if (g == 0.0) continue;
                        int c1 = apply_E(n, k, l, dJ, o1, s1);
                        for (int u = 0; u < c1; ++u) {
                            int c2 = apply_E(n, i, j, o1[u], o2, s2);
                            for (int v = 0; v < c2; ++v) {
                                int64_t I = det_index(&S, o2[v]);
                                Hout[I * N + J] += 0.5 * g * s1[u] * s2[v];
                            }
                        }
                        if (j == k) {
                            c1 = apply_E(n, i, l, dJ, o1, s1);
                            for (int u = 0; u < c1; ++u) {
                                int64_t I = det_index(&S, o1[u]);
                                Hout[I * N + J] -= 0.5 * g * s1[u];
                            }
                        }
                    }
    }
    space_free(&S);
    return 0;
}

/* ---- Direct sigma (Eq. 4/5): sigma_I = sum_J H_IJ c_J ------------------- *
 * For each output determinant I, every determinant J that differs from it by
 * at most two spin-orbital replacements inside the same (n_alpha, n_beta)
 * sector is generated, and H_IJ is taken from the Slater-Condon rules.      */
static double sigma_one(const space_t *S, const ham_t *H, const double *c, int64_t I) {
    int n = S->norb;
    int n2 = 2 * n;
    det_t dI = make_det(n, S->la[I / S->nsb], S->lb[I % S->nsb]);
    double acc = sc_diag(H, dI) * c[I];
    int occ[64], vir[64], no = 0, nv = 0;
    for (int p = 0; p < n2; ++p) {
        if ((dI >> p) & 1ULL) occ[no++] = p; else vir[nv++] = p;
    }
    /* singles */
    for (int x = 0; x < no; ++x)
        for (int y = 0; y < nv; ++y) {
            if (spin(H, occ[x]) != spin(H, vir[y])) continue;
            det_t dJ = (dI & ~((det_t)1 << occ[x])) | ((det_t)1 << vir[y]);
            int64_t J = det_index(S, dJ);
            acc += sc_element(H, dI, dJ) * c[J];
        }
    /* doubles: occupied pair x1<x2 leaves I, virtual pair y1<y2 enters */
    for (int x1 = 0; x1 < no; ++x1)
        for (int x2 = x1 + 1; x2 < no; ++x2)
            for (int y1 = 0; y1 < nv; ++y1)
                for (int y2 = y1 + 1; y2 < nv; ++y2) {
                    det_t dJ = dI & ~((det_t)1 << occ[x1]) & ~((det_t)1 << occ[x2]);
                    dJ |= ((det_t)1 << vir[y1]) | ((det_t)1 << vir[y2]);
                    /* det_index is -1 unless the alpha and beta counts are kept */
                    int64_t J = det_index(S, dJ);
                    if (J < 0) continue;
                    acc += sc_element(H, dI, dJ) * c[J];
                }
    return acc;
}

int oracle_sigma_rows(int norb, int na, int nb, const double *h, const double *eri, const double *c,
                      const int64_t *rows, int64_t nrows, double *out) {
    space_t S;
    if (space_init(&S, norb, na, nb)) return -1;
    ham_t H = {norb, h, eri};
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t r = 0; r < nrows; ++r) out[r] = sigma_one(&S, &H, c, rows[r]);
    space_free(&S);
    return 0;
}

/* ---- Sampled rows with a regenerated trial vector --------------------------- *
 * For spaces whose vectors do not fit in host memory, c_J = 2 u_J - 1 with
 * u_J from the input module's counter-based SplitMix64 (Steele, Lea & Flood,
 * OOPSLA 2014): u_J = top 53 bits of mix64(key + (J + 1) * GAMMA) * 2^-53,
 * key = mix64(mix64(seed) ^ stream * 0xD1B54A32D192ED03).  Same direct sum as
 * sigma_one, with c_J evaluated where it is needed.                        */
static uint64_t sm_mix64(uint64_t z) {
    z ^= z >> 30;
    z *= 0xBF58476D1CE4E5B9ULL;
    z ^= z >> 27;
    z *= 0x94D049BB133111EBULL;
    z ^= z >> 31;
    return z;
}

static double gen_c(uint64_t key, int64_t J) {
    uint64_t w = sm_mix64(key + (uint64_t)(J + 1) * 0x9E3779B97F4A7C15ULL);
    return 2.0 * ((double)(w >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
}

static double sigma_one_gen(const space_t *S, const ham_t *H, uint64_t key, int64_t I) {
    int n = S->norb;
    int n2 = 2 * n;
    det_t dI = make_det(n, S->la[I / S->nsb], S->lb[I % S->nsb]);
    double acc = sc_diag(H, dI) * gen_c(key, I);
    int occ[64], vir[64], no = 0, nv = 0;
    for (int p = 0; p < n2; ++p) {
        if ((dI >> p) & 1ULL) occ[no++] = p; else vir[nv++] = p;
    }
    for (int x = 0; x < no; ++x)
        for (int y = 0; y < nv; ++y) {
            if (spin(H, occ[x]) != spin(H, vir[y])) continue;
            det_t dJ = (dI & ~((det_t)1 << occ[x])) | ((det_t)1 << vir[y]);
            acc += sc_element(H, dI, dJ) * gen_c(key, det_index(S, dJ));
        }
    for (int x1 = 0; x1 < no; ++x1)
        for (int x2 = x1 + 1; x2 < no; ++x2)
            for (int y1 = 0; y1 < nv; ++y1)
                for (int y2 = y1 + 1; y2 < nv; ++y2) {
                    det_t dJ = dI & ~((det_t)1 << occ[x1]) & ~((det_t)1 << occ[x2]);
                    dJ |= ((det_t)1 << vir[y1]) | ((det_t)1 << vir[y2]);
                    int64_t J = det_index(S, dJ);
                    if (J < 0) continue;
                    acc += sc_element(H, dI, dJ) * gen_c(key, J);
                }
    return acc;
}

int oracle_sigma_rows_gen(int norb, int na, int nb, const double *h, const double *eri, uint64_t seed,
                          uint64_t stream, const int64_t *rows, int64_t nrows, double *out) {
    space_t S;
    if (space_init(&S, norb, na, nb)) return -1;
    ham_t H = {norb, h, eri};
    uint64_t key = sm_mix64(sm_mix64(seed) ^ (stream * 0xD1B54A32D192ED03ULL));
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t r = 0; r < nrows; ++r) out[r] = sigma_one_gen(&S, &H, key, rows[r]);
    space_free(&S);
    return 0;
}

int oracle_sigma(int norb, int na, int nb, const double *h, const double *eri, const double *c, double *sigma) {
    space_t S;
    if (space_init(&S, norb, na, nb)) return -1;
    ham_t H = {norb, h, eri};
    int64_t N = S.nsa * S.nsb;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t I = 0; I < N; ++I) sigma[I] = sigma_one(&S, &H, c, I);
    space_free(&S);
    return 0;
}

int oracle_hdiag(int norb, int na, int nb, const double *h, const double *eri, double *out) {
    space_t S;
    if (space_init(&S, norb, na, nb)) return -1;
    ham_t H = {norb, h, eri};
    int64_t N = S.nsa * S.nsb;
#pragma omp parallel for schedule(static)
    for (int64_t I = 0; I < N; ++I) out[I] = sc_diag(&H, make_det(norb, S.la[I / S.nsb], S.lb[I % S.nsb]));
    space_free(&S);
    return 0;
}

/* gamma_pq = sum_sigma <c| a+_{p sigma} a_{q sigma} |c>, spin summed (n x n). */
int oracle_rdm1(int norb, int na, int nb, const double *c, double *gamma) {
    space_t S;
    if (space_init(&S, norb, na, nb)) return -1;
    int n = norb;
    int64_t N = S.nsa * S.nsb;
    memset(gamma, 0, sizeof(double) * n * n);
    for (int64_t J = 0; J < N; ++J) {
        if (c[J] == 0.0) continue;
        det_t dJ = make_det(n, S.la[J / S.nsb], S.lb[J % S.nsb]);
        for (int p = 0; p < n; ++p)
            for (int q = 0; q < n; ++q)
                for (int s = 0; s < 2; ++s) {
                    det_t dI;
                    int ph = op_excite(dJ, p + s * n, q + s * n, &dI);
                    if (!ph) continue;
                    int64_t I = det_index(&S, dI);
                    gamma[p * n + q] += ph * c[I] * c[J];
                }
    }
    space_free(&S);
    return 0;
}

/* Spin-summed two-particle density Gamma_pqrs = <c| E_pq E_rs |c>, the
 * density of the two-electron term of Eq. 6, with which
 *   <c|H|c> = sum h_pq gamma_pq + 1/2 sum (pq|rs) (Gamma_pqrs - delta_qr gamma_ps).
 * Straight from the definition: E_rs (both spins) takes J to K, E_pq (both
 * spins) takes K to I, and c_I * phase * c_J lands in Gamma[p][q][r][s].
 * OpenMP over p; each thread owns the slab Gamma[p][.][.][.]. */
int oracle_rdm2(int norb, int na, int nb, const double *c, double *gamma2) {
    space_t S;
    if (space_init(&S, norb, na, nb)) return -1;
    const int n = norb;
    const int64_t N = S.nsa * S.nsb;
    const int64_t n2 = (int64_t)n * n;
    memset(gamma2, 0, sizeof(double) * n2 * n2);
#pragma omp parallel for schedule(dynamic, 1)
    for (int p = 0; p < n; ++p) {
        double *slab = gamma2 + p * n2 * n;
        for (int64_t J = 0; J < N; ++J) {
            if (c[J] == 0.0) continue;
            det_t dJ = make_det(n, S.la[J / S.nsb], S.lb[J % S.nsb]);
            for (int r = 0; r < n; ++r)
                for (int s = 0; s < n; ++s)
                    for (int t = 0; t < 2; ++t) {
                        det_t dK;
                        int ph1 = op_excite(dJ, r + t * n, s + t * n, &dK);
                        if (!ph1) continue;
                        for (int q = 0; q < n; ++q)
                            for (int u = 0; u < 2; ++u) {
                                det_t dI;
                                int ph2 = op_excite(dK, p + u * n, q + u * n, &dI);
                                if (!ph2) continue;
                                int64_t I = det_index(&S, dI);
                                slab[(q * n + r) * n + s] += (double)(ph1 * ph2) * c[I] * c[J];
                            }
                    }
        }
    }
    space_free(&S);
    return 0;
}

/* Total spin of an expansion c in the (n_alpha, n_beta) sector:
 *   <S^2> = (||S+ c||^2 + (Sz^2 + Sz) ||c||^2) / ||c||^2,
 * from S^2 = S- S+ + Sz^2 + Sz with S+ = sum_p a+_{p alpha} a_{p beta} and
 * Sz = (n_alpha - n_beta) / 2.  S+ c is formed explicitly in the
 * (n_alpha + 1, n_beta - 1) sector (zero when that sector is empty).  NAN for
 * a bad space or c = 0. */
double oracle_s2(int norb, int na, int nb, const double *c) {
    space_t S;
    if (space_init(&S, norb, na, nb)) return NAN;
    const int64_t N = S.nsa * S.nsb;
    double nrm = 0.0;
    for (int64_t I = 0; I < N; ++I) nrm += c[I] * c[I];
    double plus = 0.0;
    if (nb >= 1 && na + 1 <= norb) {
        space_t T;
        space_init(&T, norb, na + 1, nb - 1);
        const int64_t M = T.nsa * T.nsb;
        double *v = (double *)calloc((size_t)M, sizeof(double));
        for (int64_t J = 0; J < N; ++J) {
            if (c[J] == 0.0) continue;
            det_t dJ = make_det(norb, S.la[J / S.nsb], S.lb[J % S.nsb]);
            for (int p = 0; p < norb; ++p) {
                det_t dI;
                int ph = op_excite(dJ, p, norb + p, &dI); /* a+_{p alpha} a_{p beta} */
                if (ph) v[det_index(&T, dI)] += ph * c[J];
            }
        }
        for (int64_t I = 0; I < M; ++I) plus += v[I] * v[I];
        free(v);
        space_free(&T);
    }
    space_free(&S);
    if (nrm == 0.0) return NAN;
    const double sz = 0.5 * (na - nb);
    return (plus + (sz * sz + sz) * nrm) / nrm;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
