"""Pins for the oracle's spin-summed 2-RDM Gamma_pqrs = <c| E_pq E_rs |c>, the
density of the two-electron term of Eq. 6 that the paper forms after the
Davidson iterations (Table 2, "1e/2e Density Matrices").

Each pin reaches Gamma from outside the function: the Slater-Condon
Hamiltonian (energy of any vector), the Eq. 6 operator construction of E_pq
as explicit matrices, the closed form for one determinant, the commutator
[E_pq, E_rs] = delta_qr E_ps - delta_ps E_rq, the number operator in the
partial traces, and Hellmann-Feynman for the two-electron integrals."""
import numpy as np
import pytest

import fci_inputs as fi


def _energy(h, eri, g1, g2):
    """<c|H|c> from the densities (Eq. 6 with E_pq E_rs - delta_qr E_ps)."""
    e2 = np.einsum("pqrs,pqrs->", eri, g2) - np.einsum("pqqs,ps->", eri, g1)
    return float(np.sum(h * g1) + 0.5 * e2)


@pytest.mark.parametrize("norb,na,nb", [(4, 2, 2), (5, 3, 2), (6, 3, 3), (5, 1, 0), (4, 4, 1)])
def test_energy_of_any_vector(oracle_mod, norb, na, nb):
    """c^T H c (Slater-Condon H) equals the energy formed from gamma and Gamma,
    for a random, unnormalised c."""
    h, eri = fi.make_integrals(norb, 31)
    H = oracle_mod.hamiltonian(norb, na, nb, h, eri, "slater")
    rng = np.random.default_rng(norb * 100 + na * 10 + nb)
    c = rng.standard_normal(H.shape[0])
    g1 = oracle_mod.rdm1(norb, na, nb, c)
    g2 = oracle_mod.rdm2(norb, na, nb, c)
    ref = float(c @ H @ c)
    assert abs(_energy(h, eri, g1, g2) - ref) < 1e-10 * max(1.0, abs(ref))


def test_equals_product_of_explicit_e_matrices(oracle_mod):
    """Gamma_pqrs = c^T E_pq E_rs c, with E_pq the matrix that the Eq. 6
    operator construction gives for h = e_pq and no two-electron integrals."""
    norb, na, nb = 4, 2, 1
    n = oracle_mod.ndet(norb, na, nb)
    rng = np.random.default_rng(12)
    c = rng.standard_normal(n)
    z = np.zeros((norb,) * 4)
    E = {}
    for p in range(norb):
        for q in range(norb):
            e = np.zeros((norb, norb))
            e[p, q] = 1.0
            E[p, q] = oracle_mod.hamiltonian(norb, na, nb, e, z, "operator")
    g2 = oracle_mod.rdm2(norb, na, nb, c)
    for p in range(norb):
        for q in range(norb):
            left = c @ E[p, q]
            for r in range(norb):
                for s in range(norb):
                    assert abs(left @ (E[r, s] @ c) - g2[p, q, r, s]) < 1e-12


@pytest.mark.parametrize("norb,na,nb,amask,bmask", [(4, 2, 2, 0b0011, 0b0101), (5, 3, 1, 0b10110, 0b01000),
                                                   (4, 2, 2, 0b1001, 0b1001)])
def test_single_determinant_closed_form(oracle_mod, norb, na, nb, amask, bmask):
    """For one determinant with spin-orbital occupations n_p,sigma:
    Gamma_pqrs = delta_pq delta_rs o_p o_r
               + delta_ps delta_qr (1 - delta_pq) sum_sigma n_p,sigma (1 - n_q,sigma),
    o_p = n_p,alpha + n_p,beta (the exchange term moves an electron to an
    empty orbital of the same spin and back)."""
    sa = list(oracle_mod.strings(norb, na))
    sb = list(oracle_mod.strings(norb, nb))
    c = np.zeros(len(sa) * len(sb))
    c[sa.index(amask) * len(sb) + sb.index(bmask)] = 1.0
    na_ = np.array([(amask >> p) & 1 for p in range(norb)], dtype=float)
    nb_ = np.array([(bmask >> p) & 1 for p in range(norb)], dtype=float)
    o = na_ + nb_
    ref = np.zeros((norb,) * 4)
    for p in range(norb):
        for r in range(norb):
            ref[p, p, r, r] += o[p] * o[r]
    for p in range(norb):
        for q in range(norb):
            if p != q:
                ref[p, q, q, p] += na_[p] * (1 - na_[q]) + nb_[p] * (1 - nb_[q])
    assert np.array_equal(oracle_mod.rdm2(norb, na, nb, c), ref)


@pytest.mark.parametrize("norb,na,nb", [(5, 2, 3), (6, 3, 2)])
def test_commutator_and_traces(oracle_mod, norb, na, nb):
    """[E_pq, E_rs] = delta_qr E_ps - delta_ps E_rq gives
    Gamma_pqrs - Gamma_rspq = delta_qr gamma_ps - delta_ps gamma_rq;
    sum_r E_rr = N (commutes with every E_pq) gives
    sum_r Gamma_pqrr = sum_r Gamma_rrpq = N gamma_pq; and for real c the
    adjoint gives Gamma_pqrs = Gamma_srqp."""
    n = oracle_mod.ndet(norb, na, nb)
    rng = np.random.default_rng(77)
    c = rng.standard_normal(n)
    g1 = oracle_mod.rdm1(norb, na, nb, c)
    g2 = oracle_mod.rdm2(norb, na, nb, c)
    d = np.eye(norb)
    lhs = g2 - g2.transpose(2, 3, 0, 1)
    rhs = np.einsum("qr,ps->pqrs", d, g1) - np.einsum("ps,rq->pqrs", d, g1)
    assert np.abs(lhs - rhs).max() < 1e-12
    N = na + nb
    assert np.abs(np.einsum("pqrr->pq", g2) - N * g1).max() < 1e-11
    assert np.abs(np.einsum("rrpq->pq", g2) - N * g1).max() < 1e-11
    assert abs(np.einsum("pprr->", g2) - N * N * (c @ c)) < 1e-10
    assert np.abs(g2 - g2.transpose(3, 2, 1, 0)).max() < 1e-12


def test_two_electron_hellmann_feynman(oracle_mod):
    """dE0/dlambda for eri + lambda V (V with the 8-fold symmetry of real
    orbitals) equals 1/2 sum V_pqrs (Gamma_pqrs - delta_qr gamma_ps) of the
    normalised ground state, by central differences of the Slater-Condon H."""
    norb, na, nb = 4, 2, 2
    h, eri = fi.make_integrals(norb, 8)

    def ground(e2):
        w, v = np.linalg.eigh(oracle_mod.hamiltonian(norb, na, nb, h, e2))
        return w[0], v[:, 0]

    _, c = ground(eri)
    g1 = oracle_mod.rdm1(norb, na, nb, c)
    g2 = oracle_mod.rdm2(norb, na, nb, c)
    d = 1e-5
    for (p, q, r, s) in [(0, 0, 0, 0), (0, 1, 2, 3), (1, 1, 2, 2), (0, 2, 0, 2), (3, 1, 0, 0)]:
        V = np.zeros((norb,) * 4)
        for (a, b, x, y) in [(p, q, r, s), (q, p, r, s), (p, q, s, r), (q, p, s, r),
                             (r, s, p, q), (s, r, p, q), (r, s, q, p), (s, r, q, p)]:
            V[a, b, x, y] = 1.0
        ep, _ = ground(eri + d * V)
        em, _ = ground(eri - d * V)
        dE = (ep - em) / (2 * d)
        ref = 0.5 * (np.sum(V * g2) - np.einsum("pqqs,ps->", V, g1))
        assert abs(dE - ref) < 1e-6


def test_rejects_bad_inputs(oracle_mod):
    with pytest.raises(ValueError):
        oracle_mod.rdm2(4, 2, 2, np.zeros(5))
