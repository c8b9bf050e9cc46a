"""Randomised cross-checks of the oracle on spaces drawn at random (empty,
full and single-string sectors included) with random 8-fold-symmetric
integrals (not positive semidefinite, not low-rank):

* the Slater-Condon H equals Eq. 6 applied term by term;
* the direct sigma equals H c, and its diagonal equals the diagonal of H;
* the 1-RDM of c equals c^T E_pq c with E_pq built by Eq. 6 (h = e_pq, eri = 0)
  and has trace (n_alpha + n_beta) |c|^2;
* <S^2> of c equals the explicit S- S+ + Sz^2 + Sz (Sz terms exact).
"""
import numpy as np
import pytest

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")
from hypothesis import given, settings  # noqa: E402

import test_oracle_hamiltonian as th  # noqa: E402


@st.composite
def spaces(draw):
    norb = draw(st.integers(1, 5))
    na = draw(st.integers(0, norb))
    nb = draw(st.integers(0, norb))
    seed = draw(st.integers(0, 2**31 - 1))
    return norb, na, nb, seed


@settings(max_examples=60, deadline=None)
@given(spaces())
def test_random_spaces(oracle_mod, space):
    norb, na, nb, seed = space
    rng = np.random.default_rng(seed)
    h, eri = th.random_h(norb, rng), th.random_eri(norb, rng)
    H = oracle_mod.hamiltonian(norb, na, nb, h, eri, "slater")
    H2 = oracle_mod.hamiltonian(norb, na, nb, h, eri, "operator")
    scale = max(1.0, np.abs(H).max())
    assert np.abs(H - H2).max() <= 1e-12 * scale
    assert np.abs(H - H.T).max() <= 1e-12 * scale
    c = rng.standard_normal(H.shape[0])
    assert np.abs(oracle_mod.sigma(norb, na, nb, h, eri, c) - H @ c).max() <= 1e-12 * scale * max(1, np.abs(c).sum())
    assert np.abs(oracle_mod.hdiag(norb, na, nb, h, eri) - np.diag(H)).max() <= 1e-12 * scale
    g = oracle_mod.rdm1(norb, na, nb, c)
    assert abs(np.trace(g) - (na + nb) * (c @ c)) <= 1e-10 * max(1.0, c @ c)
    z = np.zeros((norb,) * 4)
    for p in range(norb):
        for q in range(norb):
            e = np.zeros((norb, norb))
            e[p, q] = 1.0
            Epq = oracle_mod.hamiltonian(norb, na, nb, e, z, "operator")
            assert abs(c @ Epq @ c - g[p, q]) <= 1e-10 * max(1.0, c @ c)
    if H.shape[0] and np.any(c):
        s2 = oracle_mod.s_squared(norb, na, nb, c)
        sz = 0.5 * (na - nb)
        if nb >= 1 and na + 1 <= norb:
            Sp = th.splus_matrix(oracle_mod, norb, na, nb)
            ref = (np.linalg.norm(Sp @ c) ** 2 + (sz * sz + sz) * (c @ c)) / (c @ c)
        else:
            ref = sz * sz + sz  # S+ c = 0: every state of the sector has S = Sz
        assert abs(s2 - ref) <= 1e-12 * max(1.0, abs(ref))
