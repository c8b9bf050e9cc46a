"""GPU parity of the large-space FP64 sigma (fci_options.f64_kernels =
FCI_F64_WIDE forces it on any space; FCI_F64_AUTO takes it where the per-row
sliced kernel does not fit, CAS(16,16) and CAS(18,18)) against the CPU oracle:
sigma_3 and both same-spin terms (through intermediate strings) from six 8-bit
slices on the bf16 tensor cores, all added as 64-bit integers in one scale.
Bars as for the other FP64 kernels:
* per element on small spaces: |d sigma_I| <= 1e-12 * sum_J |H_IJ||c_J|;
* normwise elsewhere: max|d sigma| <= 1e-12 * max|sigma|;
and the result is bit-reproducible (integer adds in any order).
"""
import numpy as np
import pytest

import fci_inputs as fi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
FMA, WIDE = 1, 3


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_1707_04346_gb300 as p

    return p


def ctx_for(pkg, norb, na, nb, mode, rank=40, seed=1707):
    h1, eri = fi.make_integrals(norb, rank, seed)
    # the wide family's own same-spin kernels (intermediate strings), not the dense products
    return pkg.fci_init(norb, na, nb, h1, eri, pkg.default_options(f64_kernels=mode, f64_same_spin=1)), h1, eri


def sigma(pkg, ctx, c):
    c_d = torch.as_tensor(c).to(DEV, torch.float64)
    s_d = torch.full_like(c_d, float("nan"))  # sigma is overwritten
    pkg.fci_sigma(ctx, c_d, s_d)
    torch.cuda.synchronize()
    return s_d.cpu().numpy()


# ragged tiles and parts, n_alpha != n_beta, one-string spins, spins without
# electrons (only the same-spin term of the other spin), full strings
SPACES = [(2, 1, 1), (3, 1, 2), (4, 2, 2), (5, 2, 3), (6, 3, 3), (6, 4, 2), (7, 3, 4), (8, 4, 4), (8, 5, 3),
          (9, 4, 5), (5, 5, 5), (6, 5, 1), (10, 1, 9), (4, 0, 2), (5, 3, 0), (11, 2, 2)]


@pytest.mark.parametrize("norb,na,nb", SPACES)
def test_wide_elementwise_small(pkg, oracle_mod, norb, na, nb):
    ctx, h1, eri = ctx_for(pkg, norb, na, nb, WIDE)
    H = oracle_mod.hamiltonian(norb, na, nb, h1, eri)
    for kind in ("random", "uniform"):
        c = fi.make_vector(H.shape[0], kind=kind)
        got = sigma(pkg, ctx, c)
        ref = H @ c
        bound = 1e-12 * (np.abs(H) @ np.abs(c)) + 1e-300
        assert np.all(np.abs(got - ref) <= bound), float(np.max(np.abs(got - ref) / bound))
    pkg.fci_free(ctx)


@pytest.mark.parametrize("norb,na,nb", [(10, 5, 5), (11, 6, 5), (10, 4, 6), (12, 6, 6), (13, 5, 4)])
def test_wide_full_vectors(pkg, oracle_mod, norb, na, nb):
    ctx, h1, eri = ctx_for(pkg, norb, na, nb, WIDE, rank=100)
    c = fi.make_vector(ctx.ndet)
    got = sigma(pkg, ctx, c)
    ref = oracle_mod.sigma(norb, na, nb, h1, eri, c)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    pkg.fci_free(ctx)


def test_wide_reproducible_and_equal_to_fma(pkg):
    norb, na, nb = 12, 6, 6
    cw, _, _ = ctx_for(pkg, norb, na, nb, WIDE, rank=100)
    cf, _, _ = ctx_for(pkg, norb, na, nb, FMA, rank=100)
    c = fi.make_vector(cw.ndet)
    a = sigma(pkg, cw, c)
    b = sigma(pkg, cw, c)
    e = sigma(pkg, cf, c)
    assert np.array_equal(a, b)
    assert np.abs(a - e).max() <= 1e-12 * np.abs(e).max()
    pkg.fci_free(cw)
    pkg.fci_free(cf)


def test_wide_large_one_body(pkg, oracle_mod):
    """One-body integrals 40x larger than the two-electron ones: the one-body
    column of the same-spin contraction has its own, coarser scale, so the
    two-electron part keeps its bits and the bar still holds."""
    norb, na, nb = 8, 4, 4
    h1, eri = fi.make_integrals(norb, 40, 1707)
    h1 = 40.0 * h1
    ctx = pkg.fci_init(norb, na, nb, h1, eri, pkg.default_options(f64_kernels=WIDE, f64_same_spin=1))
    H = oracle_mod.hamiltonian(norb, na, nb, h1, eri)
    c = fi.make_vector(ctx.ndet)
    got = sigma(pkg, ctx, c)
    ref = H @ c
    bound = 1e-12 * (np.abs(H) @ np.abs(c))
    assert np.all(np.abs(got - ref) <= bound), float(np.max(np.abs(got - ref) / bound))
    pkg.fci_free(ctx)


def test_wide_dynamic_range(pkg, oracle_mod):
    """A CI-like vector: one dominant coefficient, the rest over ten orders of
    magnitude.  One fixed-point scale for all of C: errors are relative to
    max|C|, so the normwise bar holds."""
    norb, na, nb = 10, 5, 5
    ctx, h1, eri = ctx_for(pkg, norb, na, nb, WIDE, rank=100)
    rng = np.random.default_rng(3)
    c = rng.standard_normal(ctx.ndet) * 10.0 ** rng.uniform(-10, -1, ctx.ndet)
    c[0] = 0.97
    got = sigma(pkg, ctx, c)
    ref = oracle_mod.sigma(norb, na, nb, h1, eri, c)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    pkg.fci_free(ctx)


def test_wide_nonfinite_input(pkg):
    """A non-finite C value makes the whole result NaN (one scale for all of
    C), never a silently finite sigma."""
    ctx, _, _ = ctx_for(pkg, 8, 4, 4, WIDE)
    c = fi.make_vector(ctx.ndet)
    c[77] = np.inf
    got = sigma(pkg, ctx, c)
    assert np.isnan(got).all()
    pkg.fci_free(ctx)


def test_wide_zero_vector(pkg):
    ctx, _, _ = ctx_for(pkg, 8, 4, 4, WIDE)
    got = sigma(pkg, ctx, np.zeros(ctx.ndet))
    assert np.array_equal(got, np.zeros(ctx.ndet))
    pkg.fci_free(ctx)


def test_wide_cas14_sampled_rows(pkg, oracle_mod):
    norb, na, nb = 14, 7, 7
    ctx, h1, eri = ctx_for(pkg, norb, na, nb, WIDE, rank=100)
    c = fi.make_vector(ctx.ndet)
    got = sigma(pkg, ctx, c)
    rows = np.random.default_rng(4).choice(ctx.ndet, 300, replace=False)
    ref = oracle_mod.sigma_rows(norb, na, nb, h1, eri, c, rows)
    assert np.abs(got[rows] - ref).max() <= 1e-12 * np.abs(got).max()
    pkg.fci_free(ctx)


def test_auto_cas16_takes_wide_path(pkg, oracle_mod):
    """CAS(16,16) under the default options: the per-row kernel does not fit,
    so the FP64 sigma runs the wide sigma_3 and the dense same-spin products
    (profiled names), on sampled rows
    against the oracle, with the trial vector filled on the device."""
    from fci_inputs import gpu

    norb, ne = 16, 8
    h1, eri = fi.make_integrals(norb, 100)
    ctx = pkg.fci_init(norb, ne, ne, h1, eri)
    N = ctx.ndet
    c = torch.empty(N, dtype=torch.float64, device=DEV)
    gpu.fill_pm1(c)
    s = torch.empty_like(c)
    pkg.fci_profile_enable(ctx, True)
    pkg.fci_sigma(ctx, c, s)
    torch.cuda.synchronize()
    names, _ = pkg.fci_profile_read(ctx)
    assert "sigma3_wide" in names and "sigma1_ss" in names and "sigma2_ss" in names
    rows = np.unique(np.concatenate([[0, 1, 12870, N // 2, N - 1],
                                     np.random.default_rng(16).integers(0, N, 195)]))
    got = s[torch.from_numpy(rows).to(DEV)].cpu().numpy()
    ref = oracle_mod.sigma_rows_generated(norb, ne, ne, h1, eri, rows, fi.DEFAULT_VECTOR_SEED, fi.STREAM_C_PM1)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    pkg.fci_free(ctx)
