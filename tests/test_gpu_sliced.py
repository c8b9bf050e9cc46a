"""GPU parity of the FP64 sigma kernels against the CPU oracle, in both
kernel families (fci_options.f64_kernels):
* FCI_F64_SLICED: sigma_3 from six 8-bit slices of C and of the integrals on
  the bf16 tensor cores (an integer scatter), sigma_1 and sigma_2 as dense
  sliced products with the same-spin Hamiltonians on the tensor cores (or, with
  fci_options.f64_same_spin = FCI_SS_FAMILY, in double-float FP32
  arithmetic);
* FCI_F64_FMA: FP64 fused multiply-adds throughout.
Both are held to the same bars:
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
FMA, SLICED = 1, 2


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
    return pkg.fci_init(norb, na, nb, h1, eri, pkg.default_options(f64_kernels=mode)), h1, eri


def sigma(pkg, ctx, c):
    c_d = torch.as_tensor(c).to(DEV, torch.float64)
    s_d = torch.full_like(c_d, float("nan"))  # sigma is overwritten
    pkg.fci_sigma(ctx, c_d, s_d)
    torch.cuda.synchronize()
    return s_d.cpu().numpy()


# both spins with electrons (sigma_3 runs): ragged tiles, n_alpha != n_beta,
# one-string spins, full and near-full strings
SPACES = [(2, 1, 1), (3, 1, 2), (4, 2, 2), (5, 2, 3), (6, 3, 3), (6, 4, 2), (7, 3, 4), (8, 4, 4), (8, 5, 3),
          (9, 4, 5), (5, 5, 5), (6, 5, 1), (10, 1, 9)]


@pytest.mark.parametrize("mode", [SLICED, FMA])
@pytest.mark.parametrize("norb,na,nb", SPACES)
def test_sliced_elementwise_small(pkg, oracle_mod, norb, na, nb, mode):
    ctx, h1, eri = ctx_for(pkg, norb, na, nb, mode)
    H = oracle_mod.hamiltonian(norb, na, nb, h1, eri)
    for kind in ("random", "uniform"):
        c = fi.make_vector(H.shape[0], kind=kind)
        got = sigma(pkg, ctx, c)
        ref = H @ c
        bound = 1e-12 * (np.abs(H) @ np.abs(c)) + 1e-300
        assert np.all(np.abs(got - ref) <= bound), float(np.max(np.abs(got - ref) / bound))
    pkg.fci_free(ctx)


@pytest.mark.parametrize("norb,na,nb", [(10, 5, 5), (11, 6, 5), (10, 4, 6), (12, 6, 6)])
def test_sliced_full_vectors(pkg, oracle_mod, norb, na, nb):
    ctx, h1, eri = ctx_for(pkg, norb, na, nb, SLICED, rank=100)
    c = fi.make_vector(ctx.ndet)
    got = sigma(pkg, ctx, c)
    ref = oracle_mod.sigma(norb, na, nb, h1, eri, c)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    pkg.fci_free(ctx)


def test_sliced_equals_fma_kernels_and_is_reproducible(pkg):
    """The two FP64 kernel families on the same vector agree to the FP64 bar,
    and two calls of the sliced family give identical bits (the double-float
    same-spin kernels sum in a fixed order; the sliced scatter adds integers)."""
    norb, na, nb = 12, 6, 6
    c_s, _, _ = ctx_for(pkg, norb, na, nb, SLICED, rank=100)
    c_e, _, _ = ctx_for(pkg, norb, na, nb, FMA, rank=100)
    c = fi.make_vector(c_s.ndet)
    a = sigma(pkg, c_s, c)
    b = sigma(pkg, c_s, c)
    e = sigma(pkg, c_e, c)
    assert np.array_equal(a, b)
    assert np.abs(a - e).max() <= 1e-12 * np.abs(e).max()
    pkg.fci_free(c_s)
    pkg.fci_free(c_e)


def test_sliced_large_dynamic_range(pkg, oracle_mod):
    """A CI-like vector: one dominant coefficient, the rest spread over ten
    orders of magnitude.  The fixed point is relative to each alpha row's
    largest gathered |C|; the normwise bar still holds."""
    norb, na, nb = 10, 5, 5
    ctx, h1, eri = ctx_for(pkg, norb, na, nb, SLICED, rank=100)
    rng = np.random.default_rng(3)
    c = rng.standard_normal(ctx.ndet) * 10.0 ** rng.uniform(-10, -1, ctx.ndet)
    c[0] = 0.97
    got = sigma(pkg, ctx, c)
    ref = oracle_mod.sigma(norb, na, nb, h1, eri, c)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    pkg.fci_free(ctx)


def test_sliced_cas14_sampled_rows(pkg, oracle_mod):
    norb, na, nb = 14, 7, 7
    ctx, h1, eri = ctx_for(pkg, norb, na, nb, SLICED, rank=100)
    c = fi.make_vector(ctx.ndet)
    got = sigma(pkg, ctx, c)
    rows = np.random.default_rng(4).choice(ctx.ndet, 300, replace=False)
    ref = oracle_mod.sigma_rows(norb, na, nb, h1, eri, c, rows)
    assert np.abs(got[rows] - ref).max() <= 1e-12 * np.abs(got).max()
    pkg.fci_free(ctx)


def test_sliced_nan_input_propagates(pkg):
    """A non-finite C value reaches sigma as NaN or infinity (the rows whose
    sigma_3 gathers it), as with the FMA kernels."""
    norb, na, nb = 8, 4, 4
    ctx, _, _ = ctx_for(pkg, norb, na, nb, SLICED)
    c = fi.make_vector(ctx.ndet)
    c[123] = np.inf
    got = sigma(pkg, ctx, c)
    assert np.isnan(got).any() or np.isinf(got).any()
    assert np.isfinite(got).sum() > 0
    pkg.fci_free(ctx)


def test_sliced_refused_where_it_does_not_fit(pkg):
    """Beyond both tensor-core FP64 paths (100 beta replacements per string,
    more than 96): FCI_F64_SLICED and FCI_F64_WIDE refuse at fci_init."""
    h1, eri = fi.make_integrals(19, 10)
    for mode in (SLICED, 3):
        with pytest.raises(pkg.FciError) as ei:
            pkg.fci_init(19, 1, 10, h1, eri, pkg.default_options(f64_kernels=mode))
        assert ei.value.code == pkg.fci.FCI_ERR_ARG


@pytest.mark.parametrize("norb,na,nb", [(6, 3, 3), (7, 3, 4), (9, 4, 5), (8, 5, 3), (10, 1, 9)])
def test_same_spin_dense_and_double_float(pkg, oracle_mod, norb, na, nb):
    """sigma_1 and sigma_2 both ways (dense sliced products on the tensor cores,
    the default; double-float kernels): each per element within the FP64 bar of
    H c, the dense result bit-identical on a repeat, and the profile names show
    which kernels ran."""
    h1, eri = fi.make_integrals(norb, 40)
    H = oracle_mod.hamiltonian(norb, na, nb, h1, eri)
    c = fi.make_vector(H.shape[0])
    ref = H @ c
    bound = 1e-12 * (np.abs(H) @ np.abs(c)) + 1e-300
    got = {}
    for ss in (pkg.fci.FCI_SS_AUTO, pkg.fci.FCI_SS_FAMILY):
        ctx = pkg.fci_init(norb, na, nb, h1, eri, pkg.default_options(f64_same_spin=ss))
        pkg.fci_profile_enable(ctx, True)
        got[ss] = sigma(pkg, ctx, c)
        names, _ = pkg.fci_profile_read(ctx)
        assert ("sigma1_ss" in names and "sigma2_ss" in names) == (ss == pkg.fci.FCI_SS_AUTO), names
        assert np.all(np.abs(got[ss] - ref) <= bound), float(np.max(np.abs(got[ss] - ref) / bound))
        if ss == pkg.fci.FCI_SS_AUTO:
            assert np.array_equal(sigma(pkg, ctx, c), got[ss])
        pkg.fci_free(ctx)
