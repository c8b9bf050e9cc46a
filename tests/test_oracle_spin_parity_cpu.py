"""Pins of the Ms = 0 spin-parity decomposition the GPU solver uses (Section
3.1's Ms = 0 combinations): with n_alpha = n_beta the oracle's H commutes with
the transposition C -> C^T of the [N_alpha][N_beta] coefficient array, its
spectrum is the union of the spectra on C^T = C and C^T = -C, and in this
storage convention the states with C^T = C have even total spin (singlets)
and those with C^T = -C odd spin (triplets), by the oracle's <S^2>."""
import numpy as np
import pytest

import fci_inputs as fi


def parity_basis(ns, par):
    cols = []
    for i in range(ns):
        for j in range(i + 1):
            v = np.zeros((ns, ns))
            if i == j:
                if par < 0:
                    continue
                v[i, i] = 1.0
            else:
                v[i, j] = 1.0
                v[j, i] = float(par)
                v /= np.sqrt(2.0)
            cols.append(v.ravel())
    return np.array(cols).T


@pytest.mark.parametrize("norb,ne", [(4, 2), (5, 2), (6, 3), (7, 3)])
def test_transposition_commutes_and_splits_the_spectrum(oracle_mod, norb, ne):
    h1, eri = fi.make_integrals(norb, 20, 5)
    H = oracle_mod.hamiltonian(norb, ne, ne, h1, eri)
    ns = int(round(np.sqrt(H.shape[0])))
    perm = np.arange(ns * ns).reshape(ns, ns).T.ravel()  # index of C^T's element
    assert np.abs(H[np.ix_(perm, perm)] - H).max() <= 1e-12 * np.abs(H).max()
    w = np.linalg.eigvalsh(H)
    ws = []
    for par in (1, -1):
        Q = parity_basis(ns, par)
        assert np.abs(Q.T @ Q - np.eye(Q.shape[1])).max() < 1e-13
        ws.append(np.linalg.eigvalsh(Q.T @ H @ Q))
    assert np.abs(np.sort(np.concatenate(ws)) - w).max() <= 1e-10 * np.abs(w).max()


@pytest.mark.parametrize("norb,ne", [(4, 2), (6, 3), (6, 2)])
def test_parity_is_spin_even_or_odd(oracle_mod, norb, ne):
    h1, eri = fi.make_integrals(norb, 20, 9)
    H = oracle_mod.hamiltonian(norb, ne, ne, h1, eri)
    ns = int(round(np.sqrt(H.shape[0])))
    for par in (1, -1):
        Q = parity_basis(ns, par)
        w, v = np.linalg.eigh(Q.T @ H @ Q)
        for k in range(3):
            x = Q @ v[:, k]
            s2 = oracle_mod.s_squared(norb, ne, ne, x)
            S = (-1 + np.sqrt(1 + 4 * s2)) / 2
            assert abs(S - round(S)) < 1e-8
            assert int(round(S)) % 2 == (0 if par > 0 else 1), (par, s2)
