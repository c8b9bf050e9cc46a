"""Evidence for a design claim about work not yet built: an FP64-accurate
sigma_3 contraction on bf16 tensor cores (Ozaki-style slicing).

G[J_b][q] = sum_a D[J_b][a] B[q][a] with D[J_b][a] = C(J_a, J_b) and
B[q][a] = s_a (q|p_a) (one output alpha row) is emulated as a tensor core
would run it:
  * every row of D and of B gets a power-of-two scale and is cut into S signed
    8-bit integer slices, which bf16 represents exactly;
  * slice products i x j with i + j = L share the scale 2^(-8(L+2)); each level
    is an integer matrix product (what FP32 accumulation computes exactly while
    the sums stay below 2^24);
  * the levels are combined in FP64 and scattered into sigma_3 with the beta
    replacement signs (Eq. 8).
The normwise error against the FP64 contraction must fall below the 1e-12 bar
with 6 slices (21 products) and reach the FP64 rounding level with 7, on the
CAS(10,10) workload of the synthetic integrals.
"""
import numpy as np
import pytest

import fci_inputs as fi


def _slices(M, S, bits=8):
    amax = np.abs(M).max(axis=1, keepdims=True)
    e = np.where(amax > 0, np.ceil(np.log2(np.where(amax > 0, amax, 1.0))), 0.0)
    R = M / 2.0**e
    out = []
    for _ in range(S):
        R = R * 2.0**bits
        d = np.trunc(R)
        out.append(d.astype(np.int64))
        R = R - d
    return out, e


@pytest.fixture(scope="module")
def case(oracle_mod):
    norb, ne = 10, 5
    h1, eri = fi.make_integrals(norb, 100)
    pk, pl = np.tril_indices(norb)
    W = eri[pk, pl][:, pk, pl]
    tgt, kk, ll, sg = oracle_mod.single_table(norb, ne)
    hi = np.maximum(kk, ll).astype(int)
    lo = np.minimum(kk, ll).astype(int)
    pair = hi * (hi + 1) // 2 + lo
    ns = tgt.shape[0]
    C = fi.make_vector(ns * ns).reshape(ns, ns)
    rows = np.random.default_rng(0).choice(ns, 12, replace=False)
    return tgt, pair, sg.astype(float), W, C, rows


def _sigma3_rows(case, S=None):
    tgt, pair, sg, W, C, rows = case
    ns = tgt.shape[0]
    out = []
    for Ia in rows:
        D = C[tgt[Ia], :].T
        B = sg[Ia][None, :] * W[:, pair[Ia]]
        if S is None:
            G = D @ B.T
        else:
            dS, eD = _slices(D, S)
            bS, eB = _slices(B, S)
            G = np.zeros((D.shape[0], B.shape[0]))
            for lev in range(S):
                P = sum(dS[i] @ bS[lev - i].T for i in range(lev + 1))
                if lev <= 3:
                    assert np.abs(P).max() < 2**24  # exact in FP32 accumulation
                G += P.astype(float) * 2.0 ** (-8 * (lev + 2))
            G *= 2.0**eD * 2.0**eB.T
        s = np.zeros(ns)
        for x in range(ns):
            np.add.at(s, tgt[x], sg[x] * G[x, pair[x]])
        out.append(s)
    return np.array(out)


def test_six_slices_meet_the_fp64_bar(case):
    ref = _sigma3_rows(case)
    scale = np.abs(ref).max()
    err = {S: np.abs(_sigma3_rows(case, S) - ref).max() / scale for S in (5, 6, 7)}
    assert err[5] > 1e-12  # five slices are not enough
    assert err[6] < 1e-12  # six slices (21 products) meet the 1e-12 normwise bar
    assert err[7] < 1e-14  # seven reach the FP64 rounding level
