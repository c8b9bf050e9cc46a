"""More GPU checks: the CAS(16,16) workload at full size (sampled parity, FP64
and the tensor-core path's large-space layout), Davidson restart from a
guess, the non-convergence path, the iteration log, per-kernel timing, and
the density of an eigenvector (trace, bounds, oracle)."""
import numpy as np
import pytest

import fci_inputs as fi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_1707_04346_gb300 as p

    return p


def test_cas16_sigma_sampled(pkg, oracle_mod):
    """CAS(16e,16o), 165,636,900 determinants: FP64 sigma to 1e-12 and FP32
    (tcgen05, split-BF16x6) sigma to 2e-6 on sampled rows."""
    h1, eri = fi.make_integrals(16, 100)
    ctx = pkg.fci_init(16, 8, 8, h1, eri)
    N = ctx.ndet
    assert N == 165636900
    c = fi.make_vector(N)
    c_d = torch.from_numpy(c).to(DEV)
    s_d = torch.empty_like(c_d)
    pkg.fci_sigma(ctx, c_d, s_d)
    rng = np.random.default_rng(16)
    rows = np.unique(np.concatenate([[0, N // 2, N - 1], rng.integers(0, N, 600)]))
    got = s_d[torch.from_numpy(rows).to(DEV)].cpu().numpy()
    ref = oracle_mod.sigma_rows(16, 8, 8, h1, eri, c, rows)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    del s_d
    c32 = c_d.float()
    del c_d
    s32 = torch.empty_like(c32)
    pkg.fci_sigma(ctx, c32, s32)
    got32 = s32[torch.from_numpy(rows).to(DEV)].double().cpu().numpy()
    ref32 = oracle_mod.sigma_rows(16, 8, 8, h1, eri, c.astype(np.float32).astype(np.float64), rows)
    assert np.abs(got32 - ref32).max() <= 2e-6 * np.abs(ref32).max()
    assert pkg.fci_query(ctx, 10) == 0
    pkg.fci_free(ctx)


def test_davidson_restart_from_guess_and_log(pkg):
    h1, eri = fi.make_integrals(10, 60)
    ctx = pkg.fci_init(10, 5, 5, h1, eri)
    vec = torch.empty((2, ctx.ndet), dtype=torch.float64, device=DEV)
    e = pkg.fci_davidson(ctx, 2, 1e-10, vecs=vec)
    it_first = pkg.fci_query(ctx, 8)
    e2 = pkg.fci_davidson(ctx, 2, 1e-10, guess=vec)
    assert np.abs(e2 - e).max() < 1e-9
    assert pkg.fci_query(ctx, 8) < it_first
    log = pkg.fci_davidson_log(ctx, 2)
    assert log.shape[1] == 5 and np.all(np.diff(log[:, 0]) == 1) and np.all(np.diff(log[:, 2]) >= 0)
    pkg.fci_free(ctx)


def test_davidson_not_converged_reports_energies(pkg):
    h1, eri = fi.make_integrals(10, 60)
    ctx = pkg.fci_init(10, 5, 5, h1, eri, pkg.default_options(max_iter=3))
    with pytest.raises(pkg.FciError) as ei:
        pkg.fci_davidson(ctx, 1, 1e-12)
    assert ei.value.code == 4
    pkg.fci_free(ctx)


@pytest.mark.parametrize("mode,ss,expect", [
    (0, 0, ["slice_c", "sigma3_sliced", "sigma1_ss", "sigma2_ss"]),  # FCI_F64_AUTO
    (0, 1, ["slice_c", "sigma3_sliced", "sigma1_rows", "sigma2_cols"]),  # FCI_SS_FAMILY: double-float
    (1, 0, ["sigma1_rows", "sigma2_cols", "sigma3_exact"]),  # FCI_F64_FMA
])
def test_profile_api(pkg, mode, ss, expect):
    h1, eri = fi.make_integrals(10, 60)
    ctx = pkg.fci_init(10, 5, 5, h1, eri, pkg.default_options(f64_kernels=mode, f64_same_spin=ss))
    c = torch.from_numpy(fi.make_vector(ctx.ndet)).to(DEV)
    s = torch.empty_like(c)
    pkg.fci_profile_enable(ctx, True)
    for _ in range(3):
        pkg.fci_sigma(ctx, c, s)
    names, ms = pkg.fci_profile_read(ctx)
    assert names == expect
    assert ms.shape == (3, len(expect)) and np.all(ms > 0)
    pkg.fci_profile_enable(ctx, False)
    pkg.fci_free(ctx)


def test_rdm1_of_eigenvector(pkg, oracle_mod):
    norb, na, nb = 8, 4, 4
    h1, eri = fi.make_integrals(norb, 40)
    ctx = pkg.fci_init(norb, na, nb, h1, eri)
    vec = torch.empty((1, ctx.ndet), dtype=torch.float64, device=DEV)
    pkg.fci_davidson(ctx, 1, 1e-11, vecs=vec)
    g = pkg.fci_rdm1(ctx, vec[0])
    assert abs(np.trace(g) - (na + nb)) < 1e-10
    occ = np.linalg.eigvalsh(g)
    assert occ.min() > -1e-10 and occ.max() < 2 + 1e-10
    x = vec[0].cpu().numpy()
    # the density of the returned vector itself, element by element
    assert np.abs(g - oracle_mod.rdm1(norb, na, nb, x)).max() < 1e-12
    # against the exact ground state: gamma_pq(x) - gamma_pq(y) = <x-y|E_pq|x> + <y|E_pq|x-y>
    # and ||E_pq|| <= 2, so the difference is at most 4 ||x - y|| for unit vectors
    w, v = np.linalg.eigh(oracle_mod.hamiltonian(norb, na, nb, h1, eri))
    y = v[:, 0] * np.sign(v[:, 0] @ x)
    dx = np.linalg.norm(x - y)
    assert dx < 1e-4
    assert np.abs(g - oracle_mod.rdm1(norb, na, nb, y)).max() <= 4 * dx + 1e-12
    pkg.fci_free(ctx)


def test_mixed_davidson_fp64_tail(pkg):
    """With split-BF16x3 sigma (about 1e-5 relative error) and tol 1e-12 the
    FP32 error floor lies far above sqrt(tol): the solver must notice that its
    refinement points stop reducing the residual, switch to FP64 sigma and
    still reach the FP64 energies."""
    h1, eri = fi.make_integrals(10, 60)
    ref_ctx = pkg.fci_init(10, 5, 5, h1, eri)
    ref = pkg.fci_davidson(ref_ctx, 2, 1e-12)
    ctx = pkg.fci_init(10, 5, 5, h1, eri, pkg.default_options(precision=pkg.FCI_PREC_MIXED, f32_splits=2,
                                                               max_iter=400))
    e = pkg.fci_davidson(ctx, 2, 1e-12)
    assert np.abs(e - ref).max() < 1e-10
    log = pkg.fci_davidson_log(ctx, 2)
    assert (log[:, 1] == 1).sum() > 0 and log[-1, 1] == 0  # FP32 phase first, exact at the end
    pkg.fci_free(ctx)
    pkg.fci_free(ref_ctx)


def test_default_context_short_form(pkg, oracle_mod):
    """fci_init(norb, nalpha, nbeta, h1, eri) over the library's default context:
    the same sigma as an explicit context, replaced by a second init, freed."""
    h1, eri = fi.make_integrals(6, 20)
    ctx = pkg.fci_init_default(6, 3, 2, h1, eri)
    c = fi.make_vector(ctx.ndet)
    cd = torch.from_numpy(c).to(DEV)
    s = torch.empty_like(cd)
    pkg.fci_sigma(ctx, cd, s)
    torch.cuda.synchronize()
    assert np.abs(s.cpu().numpy() - oracle_mod.sigma(6, 3, 2, h1, eri, c)).max() <= 1e-12 * np.abs(s.cpu().numpy()).max()
    ctx2 = pkg.fci_init_default(5, 2, 2, *fi.make_integrals(5, 20))  # replaces the first
    assert ctx2.ndet == 100
    del ctx  # a view: dropping it frees nothing
    assert ctx2.ndet == 100
    pkg.fci_free_default()
    pkg.fci_free_default()  # nothing left: still fine
