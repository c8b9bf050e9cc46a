"""Pins for the oracle's total-spin diagnostic <S^2> (the Ms = 0 roots of
random integrals may have any S, so the roots are characterised by it).

Closed forms: a closed-shell determinant is a singlet; a determinant whose beta
orbitals all lie in its alpha orbitals has S = Sz; the two Ms = 0 combinations of
one alpha and one beta electron in two orbitals are a singlet and a triplet, and
either determinant alone has <S^2> = 1; the two-site Hubbard ground state is a
singlet.  Invariants: non-degenerate eigenvectors of H are spin eigenstates
(S^2 commutes with H), and the value agrees with S^2 = S- S+ + Sz^2 + Sz built
as a matrix in the test from its own creation/annihilation operators.
"""
import math

import numpy as np
import pytest

import fci_inputs as fi
import test_oracle_hamiltonian as th


def unit(n, i):
    v = np.zeros(n)
    v[i] = 1.0
    return v


def det_index(oracle_mod, norb, na, nb, amask, bmask):
    la, lb = oracle_mod.strings(norb, na).tolist(), oracle_mod.strings(norb, nb).tolist()
    return la.index(amask) * len(lb) + lb.index(bmask)


@pytest.mark.parametrize("norb,ne,amask", [(2, 1, 0b01), (4, 2, 0b0110), (6, 3, 0b101010)])
def test_closed_shell_is_singlet(oracle_mod, norb, ne, amask):
    n = oracle_mod.ndet(norb, ne, ne)
    c = unit(n, det_index(oracle_mod, norb, ne, ne, amask, amask))
    assert abs(oracle_mod.s_squared(norb, ne, ne, c)) < 1e-14


@pytest.mark.parametrize("norb,na,nb,amask,bmask", [
    (4, 3, 1, 0b0111, 0b0010),  # S = 1
    (4, 2, 0, 0b1001, 0b0000),  # S = 1
    (5, 3, 0, 0b10101, 0b00000),  # S = 3/2
    (6, 4, 2, 0b111100, 0b001100),  # S = 1
])
def test_high_spin_determinant(oracle_mod, norb, na, nb, amask, bmask):
    n = oracle_mod.ndet(norb, na, nb)
    c = unit(n, det_index(oracle_mod, norb, na, nb, amask, bmask))
    S = 0.5 * (na - nb)
    assert abs(oracle_mod.s_squared(norb, na, nb, c) - S * (S + 1)) < 1e-14


def test_two_electron_open_shell(oracle_mod):
    """alpha(p) beta(q) and alpha(q) beta(p): one combination is the singlet
    (S^2 = 0), the other the Ms = 0 triplet (S^2 = 2); each alone gives 1."""
    n = oracle_mod.ndet(2, 1, 1)
    d1 = unit(n, det_index(oracle_mod, 2, 1, 1, 0b01, 0b10))
    d2 = unit(n, det_index(oracle_mod, 2, 1, 1, 0b10, 0b01))
    vals = sorted(oracle_mod.s_squared(2, 1, 1, v) for v in ((d1 + d2) / math.sqrt(2), (d1 - d2) / math.sqrt(2)))
    assert abs(vals[0]) < 1e-14 and abs(vals[1] - 2) < 1e-14
    assert abs(oracle_mod.s_squared(2, 1, 1, d1) - 1) < 1e-14
    assert abs(oracle_mod.s_squared(2, 1, 1, 3 * d2) - 1) < 1e-14  # normalisation is divided out


def test_two_site_hubbard_ground_state_is_singlet(oracle_mod):
    h = np.array([[0.0, -1.0], [-1.0, 0.0]])
    eri = np.zeros((2,) * 4)
    eri[0, 0, 0, 0] = eri[1, 1, 1, 1] = 4.0
    w, v = np.linalg.eigh(oracle_mod.hamiltonian(2, 1, 1, h, eri))
    assert abs(oracle_mod.s_squared(2, 1, 1, v[:, 0])) < 1e-12


@pytest.mark.parametrize("norb,na,nb", [(6, 3, 3), (5, 3, 2), (6, 4, 2)])
def test_eigenvectors_are_spin_eigenstates(oracle_mod, norb, na, nb):
    h, eri = fi.make_integrals(norb, 20)
    w, v = np.linalg.eigh(oracle_mod.hamiltonian(norb, na, nb, h, eri))
    checked = 0
    for k in range(min(12, len(w))):
        gap = min(abs(w[k] - w[k - 1]) if k else np.inf, abs(w[k + 1] - w[k]) if k + 1 < len(w) else np.inf)
        if gap < 1e-6:
            continue  # degenerate: any mixture of the multiplet is an eigenvector
        s2 = oracle_mod.s_squared(norb, na, nb, v[:, k])
        S = (-1 + math.sqrt(1 + 4 * s2)) / 2
        assert abs(2 * S - round(2 * S)) < 1e-8
        assert round(2 * S) % 2 == (na - nb) % 2  # S - Sz is an integer
        assert S >= 0.5 * abs(na - nb) - 1e-8
        checked += 1
    assert checked >= 3


@pytest.mark.parametrize("norb,na,nb", [(4, 2, 2), (5, 3, 2), (6, 3, 3)])
def test_matches_explicit_s2_matrix(oracle_mod, norb, na, nb):
    Sp = th.splus_matrix(oracle_mod, norb, na, nb)
    sz = 0.5 * (na - nb)
    S2 = Sp.T @ Sp + (sz * sz + sz) * np.eye(Sp.shape[1])
    c = np.random.default_rng(norb + na).standard_normal(Sp.shape[1])
    assert abs(oracle_mod.s_squared(norb, na, nb, c) - c @ S2 @ c / (c @ c)) < 1e-12


def test_bad_input(oracle_mod):
    with pytest.raises(ValueError):
        oracle_mod.s_squared(4, 2, 2, np.zeros(36))
    with pytest.raises(ValueError):
        oracle_mod.s_squared(4, 2, 2, np.ones(5))
