"""Mixed-precision Davidson with the subspace basis and its sigma vectors in
FP32 (fci_options.basis_f32 = 1 forces it; by default it is taken where the
FP64 basis does not fit, CAS(18,18)), against LAPACK on the oracle's explicit
H and against one full oracle sigma of the returned vector.  The reported
energies are exact Rayleigh quotients of the FP64 Ritz vectors (FP64 sigma at
the refinement points), so they carry FP64 accuracy although the basis is FP32.
"""
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


def make_ctx(pkg, norb, na, nb, rank=40, **opt):
    h1, eri = fi.make_integrals(norb, rank)
    o = pkg.default_options(precision=pkg.FCI_PREC_MIXED, basis_f32=1, **opt)
    return pkg.fci_init(norb, na, nb, h1, eri, o), h1, eri


@pytest.mark.parametrize("norb,na,nb,nroots,maxsub", [(6, 3, 3, 1, 8), (8, 4, 4, 1, 6), (8, 4, 4, 3, 8),
                                                      (7, 4, 3, 2, 16), (9, 5, 4, 1, 4)])
def test_f32basis_matches_lapack(pkg, oracle_mod, norb, na, nb, nroots, maxsub):
    ctx, h1, eri = make_ctx(pkg, norb, na, nb, max_subspace=maxsub)
    H = oracle_mod.hamiltonian(norb, na, nb, h1, eri)
    w = np.linalg.eigvalsh(H)
    vecs = torch.empty((nroots, ctx.ndet), dtype=torch.float64, device=DEV)
    e = pkg.fci_davidson(ctx, nroots, 1e-10, vecs=vecs)
    assert np.abs(e - w[:nroots]).max() < 1e-8, (e, w[:nroots])
    X = vecs.cpu().numpy()
    for k in range(nroots):
        assert abs(np.linalg.norm(X[k]) - 1) < 1e-10
        assert np.linalg.norm(H @ X[k] - w[k] * X[k]) < 1e-4
        assert X[k][np.argmax(np.abs(X[k]))] > 0
    log = pkg.fci_davidson_log(ctx, nroots)
    assert log[:, 1].max() == 1.0 and log[-1, 1] == 0.0  # FP32 phase, ends at an exact point
    pkg.fci_free(ctx)


def test_f32basis_cas12_energy_tied_to_oracle(pkg, oracle_mod):
    """CAS(12,12) at tol 1e-8 (the large-space target): the energy equals the
    oracle Rayleigh quotient of the returned vector within 1e-9 Eh, and the
    oracle residual is below sqrt(tol).  (The FP32-stored sigma vectors hold
    the projected matrix to about 1e-7 relative, which puts a floor near 1e-5
    under the residual: tolerances much below 1e-9 need the FP64 basis.)"""
    norb, ne = 12, 6
    ctx, h1, eri = make_ctx(pkg, norb, ne, ne, rank=100, max_subspace=8)
    vec = torch.empty((1, ctx.ndet), dtype=torch.float64, device=DEV)
    e = pkg.fci_davidson(ctx, 1, 1e-8, vecs=vec)[0]
    x = vec[0].cpu().numpy()
    hx = oracle_mod.sigma(norb, ne, ne, h1, eri, x)
    rq = float(x @ hx / (x @ x))
    r = np.linalg.norm(hx - rq * x) / np.linalg.norm(x)
    assert abs(e - rq) < 1e-9, (e, rq)
    assert r < 1e-4, r
    pkg.fci_free(ctx)


def test_f32basis_equals_f64basis_mixed(pkg):
    """CAS(10,10), 2 roots: the FP32-basis solve and the FP64-basis mixed solve
    agree to the tolerance."""
    norb, ne = 10, 5
    h1, eri = fi.make_integrals(norb, 100)
    e = []
    for b in (1, 2):
        ctx = pkg.fci_init(norb, ne, ne, h1, eri,
                           pkg.default_options(precision=pkg.FCI_PREC_MIXED, basis_f32=b, max_subspace=8))
        e.append(pkg.fci_davidson(ctx, 2, 1e-9))
        pkg.fci_free(ctx)
    assert np.abs(e[0] - e[1]).max() < 1e-8


def test_f32basis_nan_guess(pkg):
    ctx, _, _ = make_ctx(pkg, 6, 3, 3)
    g = torch.zeros((1, ctx.ndet), dtype=torch.float64, device=DEV)
    g[0, 0] = 1.0
    g[0, 3] = float("inf")
    with pytest.raises(pkg.FciError) as ei:
        pkg.fci_davidson(ctx, 1, 1e-8, guess=g)
    assert ei.value.code in (pkg.fci.FCI_ERR_NAN, pkg.fci.FCI_ERR_ARG)
    pkg.fci_free(ctx)
