// Device-resident tables built once per context (fci_init):
//  - string lists in ascending bitmask order and their addresses (Eq. 2),
//  - single-replacement lists E_kl with signs (Eq. 7),
//  - the same-spin string Hamiltonians (the alpha-alpha and beta-beta parts of
//    Eq. 6 that sigma_2 and sigma_1 of Eq. 8 apply), stored ELL-style,
//  - the packed pair matrix W[(ij),(kl)] = (ij|kl) used by sigma_3,
//  - the determinant diagonal H_II (the preconditioner of Section 3.3).
#include <cmath>
#include <cstring>

#include <algorithm>
#include <utility>
#include <vector>

#include "internal.cuh"

namespace fci {

__constant__ uint32_t c_binom[33][33];  // C(n, k), n, k <= 32 (C(32,16) < 2^31)

__device__ __forceinline__ uint32_t binom(int n, int k) { return (k < 0 || k > n) ? 0u : c_binom[n][k]; }

// Address of a string: sum over occupied orbitals p_0 < p_1 < ... of C(p_m, m+1).
__device__ __forceinline__ uint32_t string_address(uint32_t mask) {
    uint32_t a = 0;
    int m = 0;
    while (mask) {
        int p = __ffs(mask) - 1;
        a += binom(p, m + 1);
        ++m;
        mask &= mask - 1u;
    }
    return a;
}

__device__ __forceinline__ uint32_t between_mask(int k, int l) {
    int lo = k < l ? k : l, hi = k < l ? l : k;
    if (hi - lo < 2) return 0u;
    return ((1u << hi) - 1u) & ~((1u << (lo + 1)) - 1u);
}

// Invert the address: the largest p with C(p, m) <= r fixes the m-th orbital.
__global__ void k_unrank(uint32_t *out, int64_t ns, int norb, int ne) {
    int64_t r0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r0 >= ns) return;
    uint32_t r = (uint32_t)r0, mask = 0;
    int p = norb - 1;
    for (int m = ne; m >= 1; --m) {
        while (binom(p, m) > r) --p;
        mask |= 1u << p;
        r -= binom(p, m);
        --p;
    }
    out[r0] = mask;
}

// Entry e of string x: l = (e / (norb-ne+1))-th occupied orbital; k runs over
// {l} and the empty orbitals in ascending order.
__global__ void k_single_table(const uint32_t *str, int64_t ns, int norb, int ne, int nsingle, uint32_t *tab) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= ns * nsingle) return;
    int64_t x = t % ns;
    int e = (int)(t / ns);
    uint32_t X = str[x];
    int width = norb - ne + 1;
    int lslot = e / width, kslot = e % width;
    uint32_t m = X;
    for (int i = 0; i < lslot; ++i) m &= m - 1u;
    int l = __ffs(m) - 1;
    int k = -1, cnt = 0;
    for (int q = 0; q < norb; ++q) {
        if (q != l && ((X >> q) & 1u)) continue;
        if (cnt == kslot) { k = q; break; }
        ++cnt;
    }
    uint32_t Y = (X & ~(1u << l)) | (1u << k);
    bool neg = (__popc(X & between_mask(k, l)) & 1) != 0;
    uint32_t ent = string_address(Y) | ((uint32_t)pair_index(k, l) << kPairShift) | (neg ? 0x80000000u : 0u);
    tab[(int64_t)e * ns + x] = ent;
}

__global__ void k_unpack_table(const uint32_t *tab, const uint32_t *str, int64_t ns, int norb, int nsingle,
                               int32_t *tgt, int8_t *kk, int8_t *ll, int8_t *sg) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= ns * nsingle) return;
    int64_t x = t / nsingle;
    int e = (int)(t % nsingle);
    uint32_t ent = tab[(int64_t)e * ns + x];
    uint32_t X = str[x];
    int width = norb - __popc(X) + 1;
    int lslot = e / width;
    uint32_t m = X;
    for (int i = 0; i < lslot; ++i) m &= m - 1u;
    int l = __ffs(m) - 1;
    // k from the pair index and l
    int p = (int)ent_pair(ent);
    int hi = 0;
    while ((hi + 1) * (hi + 2) / 2 <= p) ++hi;
    int lo = p - hi * (hi + 1) / 2;
    int k = (hi == l) ? lo : hi;
    if (tgt) tgt[t] = (int32_t)ent_target(ent);
    if (kk) kk[t] = (int8_t)k;
    if (ll) ll[t] = (int8_t)l;
    if (sg) sg[t] = ent_negative(ent) ? (int8_t)-1 : (int8_t)1;
}

// Off-diagonal entries (k != l) of each string's list, in list order.
__global__ void k_offdiag_table(const uint32_t *tab, const uint32_t *str, int64_t ns, int nsingle, int noff,
                                uint32_t *tabo) {
    int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (x >= ns) return;
    int o = 0;
    for (int e = 0; e < nsingle; ++e) {
        const uint32_t v = tab[(int64_t)e * ns + x];
        if ((int64_t)ent_target(v) == x) continue;  // only E_kk maps a string onto itself
        tabo[(int64_t)o * ns + x] = v;
        ++o;
    }
}

// wdiag[p][x] = sum over orbitals l occupied in string x of W[p][(ll)]
__global__ void k_wdiag(const double *W, int npair, const uint32_t *str, int64_t ns, double *wd) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)npair * ns) return;
    const int p = (int)(t / ns);
    const int64_t x = t % ns;
    double a = 0.0;
    for (uint32_t m = str[x]; m; m &= m - 1u) {
        const int l = __ffs(m) - 1;
        a += W[(int64_t)p * npair + l * (l + 1) / 2 + l];
    }
    wd[t] = a;
}

__device__ __forceinline__ double eri4(const double *eri, int n, int p, int q, int r, int s) {
    return eri[((p * n + q) * n + r) * n + s];
}

// Row X of the same-spin Hamiltonian h_kl a+_k a_l + 1/2 sum (ij|kl) a+_i a+_k a_l a_j
// restricted to one spin (the one-spin part of Eq. 6), by the Slater-Condon
// rules.  Row layout: [0] diagonal; then single replacements i -> a (i occupied
// ascending, a empty ascending); then double replacements (i<j) -> (a<b).
__global__ void k_same_spin_rows(const uint32_t *str, int64_t ns, int norb, int ne, int nsame, const double *h,
                                 const double *eri, int32_t *gcol, double *gval) {
    int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (x >= ns) return;
    const int n = norb;
    uint32_t X = str[x];
    int occ[32], vir[32], no = 0, nv = 0;
    for (int p = 0; p < n; ++p) {
        if ((X >> p) & 1u) occ[no++] = p; else vir[nv++] = p;
    }
    int64_t e = 0;
    // diagonal
    double d = 0.0;
    for (int a = 0; a < no; ++a) {
        int k = occ[a];
        d += h[k * n + k];
        for (int b = 0; b < no; ++b) {
            int l = occ[b];
            d += 0.5 * (eri4(eri, n, k, k, l, l) - eri4(eri, n, k, l, l, k));
        }
    }
    gcol[e * ns + x] = (int32_t)x;
    gval[e * ns + x] = d;
    ++e;
    // singles i -> a
    for (int u = 0; u < no; ++u)
        for (int w = 0; w < nv; ++w) {
            int i = occ[u], a = vir[w];
            uint32_t Y = (X & ~(1u << i)) | (1u << a);
            double v = h[a * n + i];
            for (int q = 0; q < no; ++q) {
                int k = occ[q];
                if (k == i) continue;
                v += eri4(eri, n, a, i, k, k) - eri4(eri, n, a, k, k, i);
            }
            if (__popc(X & between_mask(i, a)) & 1) v = -v;
            gcol[e * ns + x] = (int32_t)string_address(Y);
            gval[e * ns + x] = v;
            ++e;
        }
    // doubles (i<j) -> (a<b): apply j->b, then i->a
    for (int u1 = 0; u1 < no; ++u1)
        for (int u2 = u1 + 1; u2 < no; ++u2)
            for (int w1 = 0; w1 < nv; ++w1)
                for (int w2 = w1 + 1; w2 < nv; ++w2) {
                    int i = occ[u1], j = occ[u2], a = vir[w1], b = vir[w2];
                    uint32_t X1 = (X & ~(1u << j)) | (1u << b);
                    int par = __popc(X & between_mask(j, b)) + __popc(X1 & between_mask(i, a));
                    uint32_t Y = (X1 & ~(1u << i)) | (1u << a);
                    double v = eri4(eri, n, a, i, b, j) - eri4(eri, n, a, j, b, i);
                    if (par & 1) v = -v;
                    gcol[e * ns + x] = (int32_t)string_address(Y);
                    gval[e * ns + x] = v;
                    ++e;
                }
}

__global__ void k_pack_pairs(const double *eri, int n, int npair, double *W, float *Wf) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= npair * npair) return;
    int P = t / npair, Q = t % npair;
    int i = 0;
    while ((i + 1) * (i + 2) / 2 <= P) ++i;
    int j = P - i * (i + 1) / 2;
    int k = 0;
    while ((k + 1) * (k + 2) / 2 <= Q) ++k;
    int l = Q - k * (k + 1) / 2;
    double v = eri4(eri, n, i, j, k, l);
    W[t] = v;
    Wf[t] = (float)v;
}

// H_II = G_alpha(Ia,Ia) + G_beta(Ib,Ib) + sum_{p in Ia, q in Ib} (pp|qq)
__global__ void k_hdiag(const double *ga, const double *gb, const uint32_t *sa, const uint32_t *sb, int64_t nsa,
                        int64_t nsb, int norb, const double *eri, double *out) {
    __shared__ double J[32 * 32];
    for (int t = threadIdx.x; t < norb * norb; t += blockDim.x) {
        int p = t / norb, q = t % norb;
        J[t] = eri4(eri, norb, p, p, q, q);
    }
    __syncthreads();
    int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (d >= nsa * nsb) return;
    int64_t ia = d / nsb, ib = d % nsb;
    uint32_t A = sa[ia], Bm = sb[ib];
    double c = 0.0;
    for (uint32_t m = A; m; m &= m - 1u) {
        int p = __ffs(m) - 1;
        for (uint32_t r = Bm; r; r &= r - 1u) c += J[p * norb + (__ffs(r) - 1)];
    }
    out[d] = ga[ia] + gb[ib] + c;
}

__global__ void k_f64_to_f32(const double *a, float *b, int64_t n) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < n) b[t] = (float)a[t];
}

// Trailing FP32 part of the double-float pair of each value: fl(a - fl(a)).
__global__ void k_f64_lo(const double *a, float *lo, int64_t n) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < n) lo[t] = (float)(a[t] - (double)(float)a[t]);
}

static int64_t host_binom(int n, int k) {
    if (k < 0 || k > n) return 0;
    int64_t r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

// Tile schedule for the gather epilogue of the tensor-core sigma_3 (see
// SpinTables::tsched): built on the host from the entry-major table.
bool tile_schedule_host(const uint32_t *tab, int64_t ns, int K, std::vector<uint32_t> &out,
                        std::vector<int32_t> &off) {
    const int R = kTileStrings;
    const int64_t ntiles = (ns + R - 1) / R;
    out.clear();
    off.assign((size_t)ntiles + 1, 0);
    std::vector<std::pair<uint64_t, uint32_t>> keyed;
    keyed.reserve((size_t)R * K);
    size_t pos = 0;
    for (int64_t t = 0; t < ntiles; ++t) {
        keyed.clear();
        for (int jl = 0; jl < R && t * R + jl < ns; ++jl)
            for (int e = 0; e < K; ++e) {
                const uint32_t v = tab[(size_t)e * ns + t * R + jl];
                const uint32_t tg = ent_target(v), p = ent_pair(v);
                const uint32_t rec = tg | ((uint32_t)jl << 16) | (p << 23) | (ent_negative(v) ? 0x80000000u : 0u);
                keyed.push_back({((uint64_t)tg << 16) | ((uint64_t)jl << 8) | p, rec});
            }
        std::sort(keyed.begin(), keyed.end());
        const size_t cnt = keyed.size();
        // runs of one target, dealt to the least loaded share (longest runs
        // first, ties by target and share index) so that shares stay even
        std::vector<std::pair<size_t, size_t>> runs;  // [begin, end)
        for (size_t i = 0; i < cnt;) {
            size_t j = i + 1;
            while (j < cnt && (keyed[j].second & 0xFFFFu) == (keyed[i].second & 0xFFFFu)) ++j;
            runs.push_back({i, j});
            i = j;
        }
        std::vector<size_t> order(runs.size());
        for (size_t r = 0; r < runs.size(); ++r) order[r] = r;
        std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) {
            return runs[x].second - runs[x].first > runs[y].second - runs[y].first;
        });
        std::vector<size_t> load(R, 0);
        std::vector<std::vector<size_t>> share(R);
        for (size_t r : order) {
            int best = 0;
            for (int k = 1; k < R; ++k)
                if (load[k] < load[best]) best = k;
            load[best] += runs[r].second - runs[r].first;
            share[best].push_back(r);
        }
        size_t kmax = 0;
        for (int k = 0; k < R; ++k) {
            std::sort(share[k].begin(), share[k].end());  // runs in target order
            kmax = std::max(kmax, load[k]);
        }
        // stored step-major: entry j of share k at [j][k]; share k is padded
        // with entries for the dummy target ns + k (pair 0, source 0, sign +)
        if (pos + kmax * R > (size_t)INT32_MAX) return false;  // offsets are int32
        off[t] = (int32_t)pos;
        out.resize(pos + kmax * R);
        for (int k = 0; k < R; ++k) {
            size_t j = 0;
            for (size_t r : share[k])
                for (size_t i = runs[r].first; i < runs[r].second; ++i, ++j) out[pos + j * R + k] = keyed[i].second;
            for (; j < kmax; ++j) out[pos + j * R + k] = (uint32_t)(ns + k);
        }
        pos += kmax * R;
    }
    off[ntiles] = (int32_t)pos;
    return true;
}

static int build_tile_schedule(fci_ctx *ctx, SpinTables &T) {
    if (T.nsingle == 0 || T.ns > kMaxScheduleStrings || ctx->npair > 256) return FCI_OK;
    std::vector<uint32_t> tab((size_t)T.ns * T.nsingle);
    FCI_CUDA(cudaMemcpyAsync(tab.data(), T.tab, sizeof(uint32_t) * tab.size(), cudaMemcpyDeviceToHost, ctx->stream));
    FCI_CUDA(cudaStreamSynchronize(ctx->stream));
    std::vector<uint32_t> out;
    std::vector<int32_t> off;
    if (!tile_schedule_host(tab.data(), T.ns, T.nsingle, out, off)) return FCI_OK;  // no schedule
    int rc = FCI_OK;
    T.nsched = (int64_t)out.size();
    T.tsched = (uint32_t *)dalloc(ctx, sizeof(uint32_t) * out.size(), &rc);
    T.toff = (int32_t *)dalloc(ctx, sizeof(int32_t) * off.size(), &rc);
    if (rc) return rc;
    FCI_CUDA(cudaMemcpyAsync(T.tsched, out.data(), sizeof(uint32_t) * out.size(), cudaMemcpyHostToDevice, ctx->stream));
    FCI_CUDA(cudaMemcpyAsync(T.toff, off.data(), sizeof(int32_t) * off.size(), cudaMemcpyHostToDevice, ctx->stream));
    FCI_CUDA(cudaStreamSynchronize(ctx->stream));
    return FCI_OK;
}

static int build_spin(fci_ctx *ctx, SpinTables &T, int ne) {
    const int n = ctx->norb;
    int rc = FCI_OK;
    T.ne = ne;
    T.ns = host_binom(n, ne);
    T.nsingle = ne * (n - ne) + ne;
    T.nsame = 1 + ne * (n - ne) + (int)(host_binom(ne, 2) * host_binom(n - ne, 2));
    T.owner = true;
    const int64_t ns = T.ns;
    T.str = (uint32_t *)dalloc(ctx, sizeof(uint32_t) * ns, &rc);
    T.tab = (uint32_t *)dalloc(ctx, sizeof(uint32_t) * ns * T.nsingle, &rc);
    const int noff = ne * (n - ne);
    T.tabo = (uint32_t *)dalloc(ctx, sizeof(uint32_t) * ns * (noff > 0 ? noff : 1), &rc);
    T.wdiag = (double *)dalloc(ctx, sizeof(double) * ns * ctx->npair, &rc);
    T.gcol = (int32_t *)dalloc(ctx, sizeof(int32_t) * ns * T.nsame, &rc);
    T.gval = (double *)dalloc(ctx, sizeof(double) * ns * T.nsame, &rc);
    T.gvalf = (float *)dalloc(ctx, sizeof(float) * ns * T.nsame, &rc);
    T.gvall = (float *)dalloc(ctx, sizeof(float) * ns * T.nsame, &rc);
    if (rc) return rc;
    cudaStream_t s = ctx->stream;
    k_unrank<<<ceil_div(ns, 256), 256, 0, s>>>(T.str, ns, n, ne);
    FCI_CUDA(cudaGetLastError());
    if (T.nsingle > 0) {
        k_single_table<<<ceil_div(ns * T.nsingle, 256), 256, 0, s>>>(T.str, ns, n, ne, T.nsingle, T.tab);
        FCI_CUDA(cudaGetLastError());
        k_offdiag_table<<<ceil_div(ns, 128), 128, 0, s>>>(T.tab, T.str, ns, T.nsingle, noff, T.tabo);
        FCI_CUDA(cudaGetLastError());
    }
    k_wdiag<<<ceil_div(ns * ctx->npair, 256), 256, 0, s>>>(ctx->W, ctx->npair, T.str, ns, T.wdiag);
    k_same_spin_rows<<<ceil_div(ns, 64), 64, 0, s>>>(T.str, ns, n, ne, T.nsame, ctx->h1, ctx->eri, T.gcol, T.gval);
    FCI_CUDA(cudaGetLastError());
    k_f64_to_f32<<<ceil_div(ns * T.nsame, 256), 256, 0, s>>>(T.gval, T.gvalf, ns * T.nsame);
    FCI_CUDA(cudaGetLastError());
    k_f64_lo<<<ceil_div(ns * T.nsame, 256), 256, 0, s>>>(T.gval, T.gvall, ns * T.nsame);
    FCI_CUDA(cudaGetLastError());
    return build_tile_schedule(ctx, T);
}

int build_tables(fci_ctx *ctx, const double *h1_host, const double *eri_host) {
    const int n = ctx->norb;
    int rc = FCI_OK;
    uint32_t hb[33][33];
    for (int a = 0; a <= 32; ++a)
        for (int b = 0; b <= 32; ++b) hb[a][b] = (uint32_t)(b <= a ? host_binom(a, b) : 0);
    FCI_CUDA(cudaMemcpyToSymbol(c_binom, hb, sizeof(hb)));

    const int64_t n4 = (int64_t)n * n * n * n;
    ctx->h1 = (double *)dalloc(ctx, sizeof(double) * n * n, &rc);
    ctx->eri = (double *)dalloc(ctx, sizeof(double) * n4, &rc);
    ctx->npair = n * (n + 1) / 2;
    ctx->W = (double *)dalloc(ctx, sizeof(double) * ctx->npair * ctx->npair, &rc);
    ctx->Wf = (float *)dalloc(ctx, sizeof(float) * ctx->npair * ctx->npair, &rc);
    if (rc) return rc;
    FCI_CUDA(cudaMemcpyAsync(ctx->h1, h1_host, sizeof(double) * n * n, cudaMemcpyHostToDevice, ctx->stream));
    FCI_CUDA(cudaMemcpyAsync(ctx->eri, eri_host, sizeof(double) * n4, cudaMemcpyHostToDevice, ctx->stream));
    k_pack_pairs<<<ceil_div((int64_t)ctx->npair * ctx->npair, 256), 256, 0, ctx->stream>>>(ctx->eri, n, ctx->npair,
                                                                                          ctx->W, ctx->Wf);
    FCI_CUDA(cudaGetLastError());
    {  // one-body part of H written as sum k_kl E_kl + 1/2 sum (ij|kl) E_ij E_kl
        std::vector<float> kh((size_t)ctx->npair);
        for (int k = 0; k < n; ++k)
            for (int l = 0; l <= k; ++l) {
                double v = h1_host[k * n + l];
                for (int j = 0; j < n; ++j) v -= 0.5 * eri_host[(((int64_t)k * n + j) * n + j) * n + l];
                kh[pair_index(k, l)] = (float)v;
            }
        ctx->kf = (float *)dalloc(ctx, sizeof(float) * ctx->npair, &rc);
        if (rc) return rc;
        FCI_CUDA(cudaMemcpyAsync(ctx->kf, kh.data(), sizeof(float) * ctx->npair, cudaMemcpyHostToDevice, ctx->stream));
        FCI_CUDA(cudaStreamSynchronize(ctx->stream));
    }

    if ((rc = build_spin(ctx, ctx->A, ctx->A.ne))) return rc;
    if (ctx->B.ne == ctx->A.ne) {
        ctx->B = ctx->A;
        ctx->B.owner = false;
    } else if ((rc = build_spin(ctx, ctx->B, ctx->B.ne))) {
        return rc;
    }
    ctx->ndet = ctx->A.ns * ctx->B.ns;
    if ((rc = build_sliced_tables(ctx, h1_host, eri_host))) return rc;
    if ((sigma3_sliced_ok(ctx) || sigma_wide_ok(ctx)) && (rc = build_ss_tables(ctx))) return rc;
    if ((rc = alloc_sigma_workspace(ctx))) return rc;
    ctx->hdiag = (double *)dalloc(ctx, sizeof(double) * ctx->ndet, &rc);
    ctx->d_err = (int *)dalloc(ctx, sizeof(int), &rc);
    if (rc) return rc;
    FCI_CUDA(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream));
    // the diagonal same-spin entries sit in ELL slot 0
    k_hdiag<<<ceil_div(ctx->ndet, 256), 256, 0, ctx->stream>>>(ctx->A.gval, ctx->B.gval, ctx->A.str, ctx->B.str,
                                                              ctx->A.ns, ctx->B.ns, n, ctx->eri, ctx->hdiag);
    FCI_CUDA(cudaGetLastError());
    FCI_CUDA(cudaStreamSynchronize(ctx->stream));
    return FCI_OK;
}

static void free_spin(fci_ctx *ctx, SpinTables &T) {
    if (!T.owner) return;
    dfree(ctx, T.str, sizeof(uint32_t) * T.ns);
    dfree(ctx, T.tab, sizeof(uint32_t) * T.ns * T.nsingle);
    const int noff = T.ne * (ctx->norb - T.ne);
    dfree(ctx, T.tabo, sizeof(uint32_t) * T.ns * (noff > 0 ? noff : 1));
    dfree(ctx, T.wdiag, sizeof(double) * T.ns * ctx->npair);
    dfree(ctx, T.gcol, sizeof(int32_t) * T.ns * T.nsame);
    dfree(ctx, T.gval, sizeof(double) * T.ns * T.nsame);
    dfree(ctx, T.gvalf, sizeof(float) * T.ns * T.nsame);
    dfree(ctx, T.gvall, sizeof(float) * T.ns * T.nsame);
    if (T.tsched) {
        dfree(ctx, T.tsched, sizeof(uint32_t) * T.nsched);
        dfree(ctx, T.toff, sizeof(int32_t) * ((T.ns + kTileStrings - 1) / kTileStrings + 1));
    }
    T = SpinTables{};
}

void free_tables(fci_ctx *ctx) {
    const int n = ctx->norb;
    free_wide_tables(ctx);
    free_ss_tables(ctx);
    free_sliced_tables(ctx);
    free_spin(ctx, ctx->B);
    free_spin(ctx, ctx->A);
    dfree(ctx, ctx->h1, sizeof(double) * n * n);
    dfree(ctx, ctx->eri, sizeof(double) * (int64_t)n * n * n * n);
    dfree(ctx, ctx->W, sizeof(double) * ctx->npair * ctx->npair);
    dfree(ctx, ctx->Wf, sizeof(float) * ctx->npair * ctx->npair);
    dfree(ctx, ctx->kf, sizeof(float) * ctx->npair);
    dfree(ctx, ctx->ws32, sizeof(float) * 2 * ctx->ndet);
    ctx->kf = nullptr;
    ctx->ws32 = nullptr;
    dfree(ctx, ctx->hdiag, sizeof(double) * ctx->ndet);
    dfree(ctx, ctx->d_err, sizeof(int));
    ctx->d_err = nullptr;
    ctx->h1 = ctx->eri = ctx->W = ctx->hdiag = nullptr;
    ctx->Wf = nullptr;
}

int unpack_table(fci_ctx *ctx, int spin, int32_t *tgt, int8_t *k, int8_t *l, int8_t *sg) {
    SpinTables &T = spin ? ctx->B : ctx->A;
    const int64_t cnt = T.ns * T.nsingle;
    if (cnt == 0) return FCI_OK;
    int rc = FCI_OK;
    int32_t *dt = (int32_t *)dalloc(ctx, sizeof(int32_t) * cnt, &rc);
    int8_t *dk = (int8_t *)dalloc(ctx, cnt, &rc);
    int8_t *dl = (int8_t *)dalloc(ctx, cnt, &rc);
    int8_t *ds = (int8_t *)dalloc(ctx, cnt, &rc);
    if (rc == FCI_OK) {
        k_unpack_table<<<ceil_div(cnt, 256), 256, 0, ctx->stream>>>(T.tab, T.str, T.ns, ctx->norb, T.nsingle, dt, dk,
                                                                     dl, ds);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess && tgt) e = cudaMemcpyAsync(tgt, dt, sizeof(int32_t) * cnt, cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess && k) e = cudaMemcpyAsync(k, dk, cnt, cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess && l) e = cudaMemcpyAsync(l, dl, cnt, cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess && sg) e = cudaMemcpyAsync(sg, ds, cnt, cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) rc = cuda_fail(e, "unpack_table");
    }
    dfree(ctx, dt, sizeof(int32_t) * cnt);
    dfree(ctx, dk, cnt);
    dfree(ctx, dl, cnt);
    dfree(ctx, ds, cnt);
    return rc;
}

}  // namespace fci
