"""Davidson on the Ms = 0 combinations of one spin parity
(fci_options.spin_parity): C^T = +C (singlets and other even-S states) or
C^T = -C (triplets ...), with sigma_1 formed as parity * sigma_2^T inside the
solver.  Energies against LAPACK on the oracle's H restricted to the parity
subspace, in every sigma path that has a parity shortcut: the per-row sliced
FP64 kernels, the wide FP64 kernels, the large-space FP32 kernels (same-spin
terms through intermediate strings) and the FP32-basis solver."""
import numpy as np
import pytest

import fci_inputs as fi
from test_oracle_spin_parity_cpu import parity_basis

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


def restricted_eigs(oracle_mod, norb, ne, h1, eri, par):
    H = oracle_mod.hamiltonian(norb, ne, ne, h1, eri)
    ns = int(round(np.sqrt(H.shape[0])))
    Q = parity_basis(ns, par)
    return np.linalg.eigvalsh(Q.T @ H @ Q), H, ns


CASES = [  # (label, options)
    ("fp64", dict()),
    ("mixed", dict(precision=1)),
    ("fp64_wide", dict(f64_kernels=3)),
    ("fp64_wide_family", dict(f64_kernels=3, f64_same_spin=1)),
    ("mixed_tc_same_spin", dict(precision=1, same_spin_tc=1)),
    ("mixed_f32basis", dict(precision=1, basis_f32=1, max_subspace=8)),
]


@pytest.mark.parametrize("label,opts", CASES)
@pytest.mark.parametrize("par", [1, -1])
def test_parity_energies_match_lapack(pkg, oracle_mod, label, opts, par):
    norb, ne, nroots = 8, 4, 2
    h1, eri = fi.make_integrals(norb, 40, 77)
    w, H, ns = restricted_eigs(oracle_mod, norb, ne, h1, eri, par)
    ctx = pkg.fci_init(norb, ne, ne, h1, eri, pkg.default_options(spin_parity=par, **opts))
    vecs = torch.empty((nroots, ctx.ndet), dtype=torch.float64, device=DEV)
    tol = 1e-11 if opts.get("precision", 0) == 0 else 1e-9
    e = pkg.fci_davidson(ctx, nroots, tol, vecs=vecs)
    assert np.abs(e - w[:nroots]).max() < (1e-9 if tol < 1e-10 else 1e-8), (e, w[:nroots])
    X = vecs.cpu().numpy()
    for k in range(nroots):
        c = X[k].reshape(ns, ns)
        assert np.abs(c - par * c.T).max() < 1e-12  # stays in the parity subspace
        assert np.linalg.norm(H @ X[k] - e[k] * X[k]) < 1e-4
    pkg.fci_free(ctx)


def test_parity_union_is_full_spectrum_cas14(pkg):
    """CAS(14,14): the lowest root of the full space is the lower of the two
    parities' lowest roots (FP64, within 1e-10 Eh)."""
    norb, ne = 14, 7
    h1, eri = fi.make_integrals(norb, 100)
    e = {}
    for par in (0, 1, -1):
        ctx = pkg.fci_init(norb, ne, ne, h1, eri, pkg.default_options(spin_parity=par))
        e[par] = pkg.fci_davidson(ctx, 1, 1e-12)[0]
        pkg.fci_free(ctx)
    assert abs(min(e[1], e[-1]) - e[0]) < 1e-10, e
    assert e[1] != e[-1]


def test_parity_needs_one_string_space(pkg):
    h1, eri = fi.make_integrals(6, 20)
    with pytest.raises(pkg.FciError) as ei:
        pkg.fci_init(6, 3, 2, h1, eri, pkg.default_options(spin_parity=1))
    assert ei.value.code == pkg.fci.FCI_ERR_ARG
