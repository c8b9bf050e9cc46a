"""Pins for the oracle's Davidson solver (Section 3.3) and 1-RDM (Table 2's
density step): LAPACK eigenvalues, the variational bound, Hellmann-Feynman,
trace and N-representability bounds, and a second construction of E_pq."""
import numpy as np
import pytest

import fci_inputs as fi


@pytest.mark.parametrize("norb,na,nb,nroots", [(6, 3, 3, 1), (6, 3, 3, 3), (8, 4, 4, 1), (8, 4, 4, 2), (7, 4, 3, 2)])
def test_davidson_matches_lapack(oracle_mod, norb, na, nb, nroots):
    h, eri = fi.make_integrals(norb, 40)
    H = oracle_mod.hamiltonian(norb, na, nb, h, eri)
    ref = np.linalg.eigvalsh(H)[:nroots]
    res = oracle_mod.davidson(lambda x: oracle_mod.sigma(norb, na, nb, h, eri, x),
                              oracle_mod.hdiag(norb, na, nb, h, eri), nroots=nroots, tol=1e-11, max_subspace=12)
    assert res["converged"]
    assert np.abs(res["energies"] - ref).max() < 1e-9
    assert np.all(res["energies"] >= ref - 1e-12)  # Ritz values bound from above
    for k in range(nroots):
        x = res["vectors"][k]
        assert abs(np.linalg.norm(x) - 1) < 1e-10
        assert np.linalg.norm(H @ x - ref[k] * x) < 1e-4


def test_davidson_collapse_path(oracle_mod):
    """A tiny subspace limit forces restarts; the answer must not change."""
    h, eri = fi.make_integrals(6, 40)
    H = oracle_mod.hamiltonian(6, 3, 3, h, eri)
    res = oracle_mod.davidson(lambda x: H @ x, np.diag(H), nroots=2, tol=1e-10, max_subspace=4, max_iter=500)
    assert res["converged"]
    assert np.abs(res["energies"] - np.linalg.eigvalsh(H)[:2]).max() < 1e-8


def ground_state(oracle_mod, norb, na, nb, h, eri):
    w, v = np.linalg.eigh(oracle_mod.hamiltonian(norb, na, nb, h, eri))
    return w[0], v[:, 0]


@pytest.mark.parametrize("norb,na,nb", [(4, 2, 2), (6, 3, 3), (5, 3, 2)])
def test_rdm1_hellmann_feynman(oracle_mod, norb, na, nb):
    h, eri = fi.make_integrals(norb, 20)
    _, c = ground_state(oracle_mod, norb, na, nb, h, eri)
    g = oracle_mod.rdm1(norb, na, nb, c)
    assert np.abs(g - g.T).max() < 1e-12
    assert abs(np.trace(g) - (na + nb)) < 1e-12
    occ = np.linalg.eigvalsh(g)
    assert occ.min() > -1e-12 and occ.max() < 2 + 1e-12
    d = 1e-5
    for p, q in [(0, 0), (0, 1), (1, norb - 1), (norb - 1, norb - 1)]:
        V = np.zeros((norb, norb))
        V[p, q] += 1.0
        V[q, p] += 1.0 if p != q else 0.0
        ep, _ = ground_state(oracle_mod, norb, na, nb, h + d * V, eri)
        em, _ = ground_state(oracle_mod, norb, na, nb, h - d * V, eri)
        dE = (ep - em) / (2 * d)
        assert abs(dE - np.sum(V * g)) < 1e-6


def test_rdm1_equals_expectation_of_e_pq(oracle_mod):
    """gamma_pq = c^T E_pq c, with E_pq the matrix of Eq. 6 for h = e_pq, eri = 0."""
    norb, na, nb = 5, 2, 3
    rng = np.random.default_rng(4)
    n = oracle_mod.ndet(norb, na, nb)
    c = rng.standard_normal(n)
    g = oracle_mod.rdm1(norb, na, nb, c)
    z = np.zeros((norb,) * 4)
    for p in range(norb):
        for q in range(norb):
            e = np.zeros((norb, norb))
            e[p, q] = 1.0
            Epq = oracle_mod.hamiltonian(norb, na, nb, e, z, "operator")
            assert abs(c @ Epq @ c - g[p, q]) < 1e-12
