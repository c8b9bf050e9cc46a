"""Pins for the oracle's string lists and single-replacement tables (Eq. 2, Eq. 7).

Brute force in this file is written independently of oracle.c: strings from
itertools, signs by counting occupied orbitals to the left of each operator.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_counts.json")


def colex_rank(mask):
    """addr(p0<p1<...) = sum_m C(p_m, m+1)."""
    occ = [p for p in range(32) if (mask >> p) & 1]
    return sum(math.comb(p, m + 1) for m, p in enumerate(occ))


@pytest.mark.parametrize("norb,ne", [(1, 0), (1, 1), (4, 2), (6, 3), (7, 2), (8, 4), (10, 5), (12, 6), (5, 5)])
def test_strings_are_all_subsets_in_ascending_order(oracle_mod, norb, ne):
    s = oracle_mod.strings(norb, ne)
    ref = sorted(sum(1 << p for p in c) for c in itertools.combinations(range(norb), ne))
    assert s.tolist() == ref
    assert len(s) == math.comb(norb, ne)


@pytest.mark.parametrize("norb,ne", [(6, 3), (8, 4), (9, 4), (12, 6)])
def test_colex_rank_is_position(oracle_mod, norb, ne):
    s = oracle_mod.strings(norb, ne)
    assert [colex_rank(int(m)) for m in s] == list(range(len(s)))


def _excite_brute(mask, k, l):
    """a+_k a_l on a single-spin string, signs counted operator by operator."""
    if not (mask >> l) & 1:
        return None, 0
    s1 = (-1) ** bin(mask & ((1 << l) - 1)).count("1")
    m = mask & ~(1 << l)
    if (m >> k) & 1:
        return None, 0
    s2 = (-1) ** bin(m & ((1 << k) - 1)).count("1")
    return m | (1 << k), s1 * s2


@pytest.mark.parametrize("norb,ne", [(4, 2), (6, 3), (7, 3), (8, 4), (5, 1), (5, 4)])
def test_single_table_brute_force(oracle_mod, norb, ne):
    strs = oracle_mod.strings(norb, ne).tolist()
    index = {m: i for i, m in enumerate(strs)}
    tgt, kk, ll, sg = oracle_mod.single_table(norb, ne)
    per = ne * (norb - ne) + ne
    assert tgt.shape == (len(strs), per)
    for x, m in enumerate(strs):
        e = 0
        for l in range(norb):
            if not (m >> l) & 1:
                continue
            for k in range(norb):
                if k != l and (m >> k) & 1:
                    continue
                y, s = _excite_brute(m, k, l)
                assert (tgt[x, e], kk[x, e], ll[x, e], sg[x, e]) == (index[y], k, l, s)
                # sign = (-1)^(occupied strictly between k and l)
                lo, hi = min(k, l), max(k, l)
                between = bin(m & ((1 << hi) - 1) & ~((1 << (lo + 1)) - 1)).count("1") if hi > lo else 0
                assert s == (-1) ** between
                e += 1
        assert e == per


def test_paper_printed_counts(oracle_mod):
    g = json.load(open(GOLDEN))
    for key in ("cas22_sd_count", "cas24_sd_count"):
        d = g[key]
        assert oracle_mod.binom(d["norb"], d["nalpha"]) * oracle_mod.binom(d["norb"], d["nbeta"]) == d["value"]


def test_paper_d2h_counts(oracle_mod):
    """CAS(20,20) in D2h, 1Ag: count strings by irrep (D2h as Z2^3, products by XOR)."""
    g = json.load(open(GOLDEN))
    d = g["cas20_d2h_ag_sd_count"]
    label = {"ag": 0, "b1g": 1, "b2g": 2, "b3g": 3, "au": 4, "b1u": 5, "b2u": 6, "b3u": 7}
    orbs = []
    for k, cnt in d["orbital_irreps"].items():
        orbs += [label[k]] * cnt
    assert len(orbs) == d["norb"]
    ne = d["nalpha"]
    dp = {(0, 0): 1}
    for gi in orbs:
        nd = dict(dp)
        for (e, G), v in dp.items():
            if e < ne:
                nd[(e + 1, G ^ gi)] = nd.get((e + 1, G ^ gi), 0) + v
        dp = nd
    per_irrep = [dp.get((ne, G), 0) for G in range(8)]
    assert sum(per_irrep) == oracle_mod.binom(20, 10)
    n_ag = sum(x * x for x in per_irrep)  # Ag needs Gamma_alpha == Gamma_beta
    assert n_ag == d["value"]
    # Ms=0 combinations: pairs {I, I^T} plus the diagonal I_a == I_b
    assert (n_ag + oracle_mod.binom(20, 10)) // 2 == g["cas20_d2h_ag_combination_count"]["value"]


def test_gas_loop_counts():
    g = json.load(open(GOLDEN))["gas_loop_counts"]
    assert 6 ** 4 == g["six_gas"] and 8 ** 4 == g["eight_gas"]


def test_paper_linear_scaling_reading():
    """Section 5 extrapolates the CAS(20,20) time linearly in the number of
    determinants to CAS(22,22): the printed D2h 1Ag counts reproduce the printed
    4110 s and the "about 30x" ratio (a check of how the counts were read)."""
    g = json.load(open(GOLDEN))
    ratio = g["cas22_d2h_ag_sd_count"]["value"] / g["cas20_d2h_ag_sd_count"]["value"]
    t = g["linear_scaling_times"]
    assert abs(ratio - 30) < 1.0
    assert abs(t["cas20_s_per_ci_iteration_2048"] * ratio - t["cas22_extrapolated_s_2048"]) < 2.0
