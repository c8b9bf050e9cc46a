"""Pins for the oracle's Hamiltonian and sigma (Eq. 2, 4-8).

Each check ties the oracle to something other than itself: a second
construction of H (Eq. 6 applied literally), closed forms (2-site Hubbard,
minimal-basis H2, free fermions, eri = 0), exact symmetries ([H, S^2] = 0,
alpha/beta transpose, orbital-rotation invariance) and linear algebra.
"""
import itertools
import math

import numpy as np
import pytest

import fci_inputs as fi


def random_eri(n, rng):
    """Random real integrals with 8-fold symmetry (not PSD, not low-rank)."""
    g = rng.standard_normal((n, n, n, n))
    g = g + g.transpose(1, 0, 2, 3)
    g = g + g.transpose(0, 1, 3, 2)
    g = g + g.transpose(2, 3, 0, 1)
    return g / 8.0


def random_h(n, rng):
    a = rng.standard_normal((n, n))
    return 0.5 * (a + a.T)


SPACES = [(2, 1, 1), (3, 2, 1), (4, 2, 2), (5, 3, 2), (6, 3, 3), (6, 4, 2)]


@pytest.mark.parametrize("norb,na,nb", SPACES)
def test_two_constructions_agree(oracle_mod, norb, na, nb):
    rng = np.random.default_rng(norb * 100 + na * 10 + nb)
    h, eri = random_h(norb, rng), random_eri(norb, rng)
    H1 = oracle_mod.hamiltonian(norb, na, nb, h, eri, "slater")
    H2 = oracle_mod.hamiltonian(norb, na, nb, h, eri, "operator")
    assert np.abs(H1 - H2).max() < 1e-12 * max(1.0, np.abs(H1).max())
    assert np.abs(H1 - H1.T).max() < 1e-13


def test_two_constructions_agree_cas8(oracle_mod):
    h, eri = fi.make_integrals(8, 40)
    H1 = oracle_mod.hamiltonian(8, 4, 4, h, eri, "slater")
    H2 = oracle_mod.hamiltonian(8, 4, 4, h, eri, "operator")
    assert np.abs(H1 - H2).max() < 1e-12


def _spin_orbital_basis(oracle_mod, norb, na, nb):
    la = oracle_mod.strings(norb, na).tolist()
    lb = oracle_mod.strings(norb, nb).tolist()
    dets = [a | (b << norb) for a in la for b in lb]
    return dets, {d: i for i, d in enumerate(dets)}


def _op(mask, p, create):
    """Creation/annihilation of spin orbital p on a mask; creators ascending."""
    occ = (mask >> p) & 1
    if create == bool(occ):
        return None, 0
    sign = (-1) ** bin(mask & ((1 << p) - 1)).count("1")
    return (mask | (1 << p)) if create else (mask & ~(1 << p)), sign


def splus_matrix(oracle_mod, norb, na, nb):
    """S+ = sum_p a+_{p alpha} a_{p beta}: sector (na, nb) -> (na+1, nb-1)."""
    src, _ = _spin_orbital_basis(oracle_mod, norb, na, nb)
    dst, dindex = _spin_orbital_basis(oracle_mod, norb, na + 1, nb - 1)
    M = np.zeros((len(dst), len(src)))
    for j, d in enumerate(src):
        for p in range(norb):
            t, s1 = _op(d, norb + p, False)
            if t is None:
                continue
            u, s2 = _op(t, p, True)
            if u is None:
                continue
            M[dindex[u], j] += s1 * s2
    return M


@pytest.mark.parametrize("norb,na,nb", [(4, 2, 2), (5, 3, 2), (6, 3, 3)])
def test_commutes_with_total_spin(oracle_mod, norb, na, nb):
    rng = np.random.default_rng(7)
    h, eri = random_h(norb, rng), random_eri(norb, rng)
    H = oracle_mod.hamiltonian(norb, na, nb, h, eri)
    Sp = splus_matrix(oracle_mod, norb, na, nb)
    sz = 0.5 * (na - nb)
    S2 = Sp.T @ Sp + (sz * sz + sz) * np.eye(H.shape[0])
    assert np.abs(H @ S2 - S2 @ H).max() < 1e-11
    # and S^2 itself has eigenvalues S(S+1)
    ev = np.linalg.eigvalsh(S2)
    S = (-1 + np.sqrt(1 + 4 * ev)) / 2
    assert np.allclose(S * 2, np.round(S * 2), atol=1e-9)


@pytest.mark.parametrize("norb,na,nb", [(4, 2, 2), (5, 2, 3), (6, 3, 3)])
def test_no_two_electron_integrals_gives_orbital_energy_sums(oracle_mod, norb, na, nb):
    rng = np.random.default_rng(11)
    h = random_h(norb, rng)
    H = oracle_mod.hamiltonian(norb, na, nb, h, np.zeros((norb,) * 4))
    eps = np.linalg.eigvalsh(h)
    sums = sorted(
        sum(eps[list(a)]) + sum(eps[list(b)])
        for a in itertools.combinations(range(norb), na)
        for b in itertools.combinations(range(norb), nb)
    )
    assert np.allclose(np.linalg.eigvalsh(H), sums, atol=1e-12)
    assert abs(np.linalg.eigvalsh(H)[0] - (eps[:na].sum() + eps[:nb].sum())) < 1e-12


@pytest.mark.parametrize("t,U", [(1.0, 4.0), (0.7, 0.0), (1.3, 8.5), (0.0, 3.0)])
def test_two_site_hubbard(oracle_mod, t, U):
    h = np.array([[0.0, -t], [-t, 0.0]])
    eri = np.zeros((2, 2, 2, 2))
    eri[0, 0, 0, 0] = eri[1, 1, 1, 1] = U
    ev = np.linalg.eigvalsh(oracle_mod.hamiltonian(2, 1, 1, h, eri))
    r = math.sqrt(U * U + 16 * t * t)
    ref = sorted([(U - r) / 2, 0.0, U, (U + r) / 2])
    assert np.allclose(ev, ref, atol=1e-13)


def test_h2_minimal_basis(oracle_mod):
    """Two orbitals of opposite inversion parity: h12 = 0 and (11|12) = (22|12) = 0."""
    h0, e0 = fi.make_integrals(2, 3, seed=99)
    h = np.diag(np.diag(h0))
    eri = np.zeros((2, 2, 2, 2))
    for idx in itertools.product(range(2), repeat=4):
        if sum(idx) % 2 == 0:  # even number of index-1 (odd-parity) orbitals
            eri[idx] = e0[idx]
    H = oracle_mod.hamiltonian(2, 1, 1, h, eri)
    E1 = 2 * h[0, 0] + eri[0, 0, 0, 0]
    E2 = 2 * h[1, 1] + eri[1, 1, 1, 1]
    K = eri[0, 1, 0, 1]
    J = eri[0, 0, 1, 1]
    gs = 0.5 * (E1 + E2) - math.sqrt(0.25 * (E1 - E2) ** 2 + K * K)
    ex = 0.5 * (E1 + E2) + math.sqrt(0.25 * (E1 - E2) ** 2 + K * K)
    open_t = h[0, 0] + h[1, 1] + J - K
    open_s = h[0, 0] + h[1, 1] + J + K
    assert np.allclose(np.linalg.eigvalsh(H), sorted([gs, ex, open_t, open_s]), atol=1e-13)


def test_hubbard_ring_free_fermions(oracle_mod):
    n, t = 6, 1.0
    h = np.zeros((n, n))
    for i in range(n):
        h[i, (i + 1) % n] = h[(i + 1) % n, i] = -t
    H = oracle_mod.hamiltonian(n, 3, 3, h, np.zeros((n,) * 4))
    eps = sorted(-2 * t * math.cos(2 * math.pi * k / n) for k in range(n))
    assert abs(np.linalg.eigvalsh(H)[0] - 2 * sum(eps[:3])) < 1e-12


def test_atomic_limit_hubbard(oracle_mod):
    """t = 0: H is diagonal, U times the number of doubly occupied sites."""
    n, U = 4, 2.5
    eri = np.zeros((n,) * 4)
    for i in range(n):
        eri[i, i, i, i] = U
    H = oracle_mod.hamiltonian(n, 2, 2, np.zeros((n, n)), eri)
    assert np.abs(H - np.diag(np.diag(H))).max() == 0
    la = oracle_mod.strings(n, 2)
    ref = [U * bin(int(a) & int(b)).count("1") for a in la for b in la]
    assert np.allclose(np.diag(H), ref)


def _rotate(h, eri, U):
    h2 = U.T @ h @ U
    e2 = np.einsum("pqrs,pi,qj,rk,sl->ijkl", eri, U, U, U, U, optimize=True)
    return h2, e2


@pytest.mark.parametrize("norb,na,nb", [(4, 2, 2), (5, 3, 2), (6, 3, 3)])
def test_orbital_rotation_invariance(oracle_mod, norb, na, nb):
    h, eri = fi.make_integrals(norb, 20, seed=5)
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.standard_normal((norb, norb)))
    h2, e2 = _rotate(h, eri, Q)
    ev1 = np.linalg.eigvalsh(oracle_mod.hamiltonian(norb, na, nb, h, eri))
    ev2 = np.linalg.eigvalsh(oracle_mod.hamiltonian(norb, na, nb, h2, e2))
    assert np.abs(ev1 - ev2).max() < 1e-11


@pytest.mark.parametrize("norb,na,nb", [(4, 2, 2), (6, 3, 3), (6, 2, 4), (7, 3, 3), (8, 4, 4)])
def test_direct_sigma_equals_explicit_h(oracle_mod, norb, na, nb):
    h, eri = fi.make_integrals(norb, 40)
    H = oracle_mod.hamiltonian(norb, na, nb, h, eri)
    c = fi.make_vector(H.shape[0])
    s = oracle_mod.sigma(norb, na, nb, h, eri, c)
    assert np.abs(s - H @ c).max() < 1e-13 * np.abs(H).sum(axis=1).max()
    rows = np.array([0, H.shape[0] // 3, H.shape[0] - 1])
    assert np.allclose(oracle_mod.sigma_rows(norb, na, nb, h, eri, c, rows), s[rows], rtol=0, atol=1e-14)
    assert np.allclose(oracle_mod.hdiag(norb, na, nb, h, eri), np.diag(H), rtol=0, atol=1e-14)


def test_direct_sigma_random_symmetric_integrals(oracle_mod):
    rng = np.random.default_rng(21)
    h, eri = random_h(6, rng), random_eri(6, rng)
    H = oracle_mod.hamiltonian(6, 4, 2, h, eri, "operator")
    c = rng.standard_normal(H.shape[0])
    assert np.abs(oracle_mod.sigma(6, 4, 2, h, eri, c) - H @ c).max() < 1e-12


def test_sigma_linear_and_transpose_symmetric(oracle_mod):
    n, ne = 8, 4
    h, eri = fi.make_integrals(n, 40)
    ns = oracle_mod.binom(n, ne)
    rng = np.random.default_rng(1)
    a, b = rng.standard_normal(ns * ns), rng.standard_normal(ns * ns)
    sa = oracle_mod.sigma(n, ne, ne, h, eri, a)
    sb = oracle_mod.sigma(n, ne, ne, h, eri, b)
    sab = oracle_mod.sigma(n, ne, ne, h, eri, 2.0 * a - 3.0 * b)
    assert np.abs(sab - (2 * sa - 3 * sb)).max() < 1e-12
    # n_alpha == n_beta: swapping the spins transposes C and sigma
    at = a.reshape(ns, ns).T.reshape(-1)
    sat = oracle_mod.sigma(n, ne, ne, h, eri, at)
    assert np.abs(sat.reshape(ns, ns).T.reshape(-1) - sa).max() < 1e-12
    # c^T sigma = <c|H|c> with H from the other construction
    H = oracle_mod.hamiltonian(n, ne, ne, h, eri, "operator")
    assert abs(a @ sa - a @ H @ a) < 1e-10 * abs(a @ sa)


@pytest.mark.parametrize("norb,na,nb", [(8, 4, 4), (7, 4, 3)])
def test_sigma_rows_generated_matches_full_vector(oracle_mod, norb, na, nb):
    """The oracle's per-index generator (for spaces too large for host memory)
    gives the same rows as the full vector from the input module."""
    h1, eri = fi.make_integrals(norb, 40)
    N = oracle_mod.ndet(norb, na, nb)
    c = fi.vector_pm1(0, N)
    rows = np.array([0, 1, N // 3, N // 2, N - 1])
    a = oracle_mod.sigma_rows(norb, na, nb, h1, eri, c, rows)
    b = oracle_mod.sigma_rows_generated(norb, na, nb, h1, eri, rows, fi.DEFAULT_VECTOR_SEED, fi.STREAM_C_PM1)
    assert np.array_equal(a, b)


def test_vector_pm1_counter_based():
    """Any slice of the regenerated vector equals the same slice of a longer run."""
    whole = fi.vector_pm1(0, 1000)
    assert np.array_equal(fi.vector_pm1(400, 100), whole[400:500])
    assert whole.min() >= -1.0 and whole.max() < 1.0
