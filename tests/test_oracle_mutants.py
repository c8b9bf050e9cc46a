"""Planted mistakes: the oracle's pins must catch a plausible error anywhere.

Each mutant below is one small, plausible mistake in the oracle (a dropped
term, a lost fermionic phase, a swapped index, a wrong factor, an off-by-one),
planted in a temporary copy of ``oracle/csrc/oracle.c`` or
``oracle/davidson.py``; the committed oracle is never modified.  The copy is
built and exercised in a child process (so a mutant that crashes cannot take
the test run down), against the pins of ``test_oracle_strings.py``,
``test_oracle_hamiltonian.py``, ``test_oracle_davidson_rdm.py`` and
``test_oracle_spin.py`` and ``test_oracle_rdm2.py``.  A mutant
counts as caught when at least one pin fails (or a signal kills the child).  The
unmodified copy, built the same way, must pass every pin, so the harness itself
is checked too.

Run directly (``python tests/test_oracle_mutants.py SPEC.json``) this file is
the child: it builds the copy named in SPEC and prints the names of the pins
that failed as one JSON line.
"""
import concurrent.futures
import ctypes
import json
import os
import subprocess
import sys
import types

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
ORACLE_C = os.path.join(ROOT, "oracle", "csrc", "oracle.c")
ORACLE_DAV = os.path.join(ROOT, "oracle", "davidson.py")

# (name, file, text in the oracle, replacement); the text must occur exactly once.
C_MUTANTS = [
    # Slater-Condon single replacement: phase dropped (Eq. 6, E_kl with sign)
    ("single_phase_dropped", "c", "        return ph * v;\n", "        return v;\n"),
    # single replacement: exchange with the spectator electrons dropped
    ("single_exchange_dropped", "c",
     "v += phys(H, a, k, i, k) - phys(H, a, k, k, i);", "v += phys(H, a, k, i, k);"),
    # diagonal: the 1/2 of the pair sum dropped
    ("diag_half_dropped", "c",
     "e += 0.5 * (phys(H, occ[a], occ[b], occ[a], occ[b]) - phys(H, occ[a], occ[b], occ[b], occ[a]));",
     "e += (phys(H, occ[a], occ[b], occ[a], occ[b]) - phys(H, occ[a], occ[b], occ[b], occ[a]));"),
    # diagonal: same-spin exchange dropped
    ("diag_exchange_dropped", "c",
     "e += 0.5 * (phys(H, occ[a], occ[b], occ[a], occ[b]) - phys(H, occ[a], occ[b], occ[b], occ[a]));",
     "e += 0.5 * phys(H, occ[a], occ[b], occ[a], occ[b]);"),
    # double replacement: exchange integral dropped
    ("double_exchange_dropped", "c",
     "return ph1 * ph2 * (phys(H, a, b, i, j) - phys(H, a, b, j, i));",
     "return ph1 * ph2 * phys(H, a, b, i, j);"),
    # double replacement: phase of the second replacement dropped
    ("double_phase_dropped", "c",
     "return ph1 * ph2 * (phys(H, a, b, i, j) - phys(H, a, b, j, i));",
     "return ph1 * (phys(H, a, b, i, j) - phys(H, a, b, j, i));"),
    # physicist <pq|rs> read as chemist (pq|rs): transposed operand
    ("physicist_chemist_swap", "c",
     "return ERI(H, sp(H, p), sp(H, r), sp(H, q), sp(H, s));",
     "return ERI(H, sp(H, p), sp(H, q), sp(H, r), sp(H, s));"),
    # no spin selection in <pq|rs>: exchange between opposite spins let through
    ("spin_rule_dropped", "c",
     "if (spin(H, p) != spin(H, r) || spin(H, q) != spin(H, s)) return 0.0;", "(void)0;"),
    # creation operator without its phase
    ("creation_phase_dropped", "c",
     "    int s = (popc64(m & (((det_t)1 << p) - 1)) & 1) ? -1 : 1;\n    *out = m | ((det_t)1 << p);",
     "    int s = 1;\n    *out = m | ((det_t)1 << p);"),
    # direct sigma: diagonal term dropped
    ("sigma_diagonal_dropped", "c", "double acc = sc_diag(H, dI) * c[I];", "double acc = 0.0;"),
    # direct sigma: some double replacements skipped (wrong loop start)
    ("sigma_doubles_skipped", "c",
     "for (int y2 = y1 + 1; y2 < nv; ++y2) {\n"
     "                    det_t dJ = dI & ~((det_t)1 << occ[x1]) & ~((det_t)1 << occ[x2]);\n"
     "                    dJ |= ((det_t)1 << vir[y1]) | ((det_t)1 << vir[y2]);\n"
     "                    /* det_index",
     "for (int y2 = y1 + 2; y2 < nv; ++y2) {\n"
     "                    det_t dJ = dI & ~((det_t)1 << occ[x1]) & ~((det_t)1 << occ[x2]);\n"
     "                    dJ |= ((det_t)1 << vir[y1]) | ((det_t)1 << vir[y2]);\n"
     "                    /* det_index"),
    # Eq. 6 applied literally: the delta_jk E_il term dropped
    ("operator_delta_term_dropped", "c", "if (j == k) {", "if (0) {"),
    # Eq. 6 applied literally: the 1/2 of the two-body sum dropped
    ("operator_half_dropped", "c",
     "Hout[I * N + J] += 0.5 * g * s1[u] * s2[v];", "Hout[I * N + J] += g * s1[u] * s2[v];"),
    # 1-RDM: beta electrons forgotten
    ("rdm1_one_spin", "c",
     "for (int s = 0; s < 2; ++s) {\n                    det_t dI;",
     "for (int s = 0; s < 1; ++s) {\n                    det_t dI;"),
    # 1-RDM: ket coefficient used twice
    ("rdm1_wrong_coefficient", "c",
     "gamma[p * n + q] += ph * c[I] * c[J];", "gamma[p * n + q] += ph * c[J] * c[J];"),
    # 2-RDM: the second operator acts on alpha electrons only
    ("rdm2_one_spin", "c",
     "for (int u = 0; u < 2; ++u) {", "for (int u = 0; u < 1; ++u) {"),
    # 2-RDM: phase of the first replacement dropped
    ("rdm2_phase_dropped", "c", "(double)(ph1 * ph2) * c[I] * c[J]", "(double)ph2 * c[I] * c[J]"),
    # 2-RDM: second and third indices swapped on store
    ("rdm2_index_swapped", "c", "slab[(q * n + r) * n + s]", "slab[(r * n + q) * n + s]"),
    # 2-RDM: operators applied in the other order (Gamma_rspq)
    ("rdm2_operator_order", "c",
     "int ph1 = op_excite(dJ, r + t * n, s + t * n, &dK);", "int ph1 = op_excite(dJ, s + t * n, r + t * n, &dK);"),
    # single-replacement list: sign not stored
    ("table_sign_dropped", "c", "sg[at] = (int8_t)s;", "sg[at] = (int8_t)1;"),
    # single-replacement list: operator indices swapped (a+_l a_k)
    ("table_indices_swapped", "c",
     "int s = op_excite(list[x], k, l, &y);", "int s = op_excite(list[x], l, k, &y);"),
    # string list: the empty string missed (loop starts at 1)
    ("strings_start_at_one", "c",
     "for (uint64_t m = 0; m < lim; ++m)", "for (uint64_t m = 1; m < lim; ++m)"),
    # <S^2>: the Sz term of S^2 = S- S+ + Sz^2 + Sz dropped
    ("s2_sz_term_dropped", "c",
     "return (plus + (sz * sz + sz) * nrm) / nrm;", "return (plus + sz * sz * nrm) / nrm;"),
    # <S^2>: phase of a+_{p alpha} a_{p beta} dropped
    ("s2_phase_dropped", "c",
     "if (ph) v[det_index(&T, dI)] += ph * c[J];", "if (ph) v[det_index(&T, dI)] += c[J];"),
    # regenerated trial vector: counter off by one
    ("generator_counter_off_by_one", "c",
     "sm_mix64(key + (uint64_t)(J + 1) * 0x9E3779B97F4A7C15ULL)",
     "sm_mix64(key + (uint64_t)J * 0x9E3779B97F4A7C15ULL)"),
]

PY_MUTANTS = [
    # residual with the wrong sign: r = Hx + Ex
    ("davidson_residual_sign", "py", "R = HX - w[:, None] * X", "R = HX + w[:, None] * X"),
    # highest instead of lowest Ritz pairs
    ("davidson_highest_roots", "py", "w, v = w[:nroots], v[:, :nroots]", "w, v = w[-nroots:], v[:, -nroots:]"),
    # new corrections not orthogonalised against each other
    ("davidson_block_not_orthogonal", "py", "t = t - q * (q @ t)", "t = t"),
    # collapse keeps the old subspace's sigma vectors with the new basis
    ("davidson_collapse_stale_sigma", "py", "B, S = X.copy(), HX.copy()", "B, S = X.copy(), S[: X.shape[0]].copy()"),
]


def _pins():
    """The pins run against each mutant, each on one small case."""
    sys.path.insert(0, HERE)
    import test_oracle_davidson_rdm as td
    import test_oracle_hamiltonian as th
    import test_oracle_rdm2 as tr2
    import test_oracle_spin as tsp
    import test_oracle_strings as ts

    return [
        ("strings_subsets", lambda o: [ts.test_strings_are_all_subsets_in_ascending_order(o, n, e)
                                       for n, e in [(1, 0), (4, 2), (6, 3)]]),
        ("colex_rank", lambda o: ts.test_colex_rank_is_position(o, 6, 3)),
        ("single_table_brute_force", lambda o: [ts.test_single_table_brute_force(o, n, e)
                                                for n, e in [(4, 2), (5, 1), (6, 3)]]),
        ("paper_counts", ts.test_paper_printed_counts),
        ("two_constructions", lambda o: [th.test_two_constructions_agree(o, n, a, b)
                                         for n, a, b in [(2, 1, 1), (3, 2, 1), (4, 2, 2)]]),
        ("spin_commutes", lambda o: th.test_commutes_with_total_spin(o, 4, 2, 2)),
        ("eri_zero_orbital_sums", lambda o: th.test_no_two_electron_integrals_gives_orbital_energy_sums(o, 4, 2, 2)),
        ("hubbard_two_site", lambda o: th.test_two_site_hubbard(o, 1.0, 4.0)),
        ("h2_minimal_basis", th.test_h2_minimal_basis),
        ("hubbard_ring_free", th.test_hubbard_ring_free_fermions),
        ("hubbard_atomic_limit", th.test_atomic_limit_hubbard),
        ("rotation_invariance", lambda o: th.test_orbital_rotation_invariance(o, 4, 2, 2)),
        ("direct_sigma_vs_h", lambda o: th.test_direct_sigma_equals_explicit_h(o, 6, 3, 3)),
        ("sigma_linear_transpose", th.test_sigma_linear_and_transpose_symmetric),
        ("sigma_rows_generated", lambda o: th.test_sigma_rows_generated_matches_full_vector(o, 7, 4, 3)),
        ("davidson_lapack", lambda o: [td.test_davidson_matches_lapack(o, 6, 3, 3, r) for r in (1, 3)]),
        ("davidson_collapse", td.test_davidson_collapse_path),
        ("rdm1_hellmann_feynman", lambda o: td.test_rdm1_hellmann_feynman(o, 4, 2, 2)),
        ("rdm1_e_pq", td.test_rdm1_equals_expectation_of_e_pq),
        ("rdm2_energy", lambda o: tr2.test_energy_of_any_vector(o, 5, 3, 2)),
        ("rdm2_e_matrices", tr2.test_equals_product_of_explicit_e_matrices),
        ("rdm2_single_det", lambda o: tr2.test_single_determinant_closed_form(o, 4, 2, 2, 0b0011, 0b0101)),
        ("rdm2_commutator", lambda o: tr2.test_commutator_and_traces(o, 5, 2, 3)),
        ("s2_closed_shell", lambda o: tsp.test_closed_shell_is_singlet(o, 4, 2, 0b0110)),
        ("s2_high_spin", lambda o: tsp.test_high_spin_determinant(o, 4, 3, 1, 0b0111, 0b0010)),
        ("s2_open_shell", tsp.test_two_electron_open_shell),
        ("s2_hubbard_singlet", tsp.test_two_site_hubbard_ground_state_is_singlet),
        ("s2_eigenvectors", lambda o: tsp.test_eigenvectors_are_spin_eigenstates(o, 5, 3, 2)),
        ("s2_explicit_matrix", lambda o: tsp.test_matches_explicit_s2_matrix(o, 5, 3, 2)),
    ]


def _plant(path, old, new):
    text = open(path).read()
    assert text.count(old) == 1, f"mutation site not unique in {os.path.basename(path)}: {old[:60]!r}"
    return text.replace(old, new)


def _child(spec):
    """Build the (possibly mutated) oracle copy and run every pin against it."""
    sys.path.insert(0, ROOT)
    import oracle

    work = spec["dir"]
    csrc = open(ORACLE_C).read() if spec["file"] != "c" else _plant(ORACLE_C, spec["old"], spec["new"])
    cpath = os.path.join(work, "oracle.c")
    so = os.path.join(work, "liboracle.so")
    with open(cpath, "w") as f:
        f.write(csrc)
    subprocess.run(["gcc", "-O1", "-std=c11", "-fopenmp", "-fPIC", "-shared", cpath, "-o", so, "-lm"], check=True)
    oracle._lib = oracle._bind(ctypes.CDLL(so))
    if spec["file"] == "py":
        mod = types.ModuleType("oracle_davidson_mutant")
        exec(compile(_plant(ORACLE_DAV, spec["old"], spec["new"]), "davidson_mutant.py", "exec"), mod.__dict__)
        oracle.davidson = mod.davidson
    failed = []
    for name, pin in _pins():
        try:
            pin(oracle)
        except Exception:  # an assertion, or an error raised by the mutant
            failed.append(name)
    print(json.dumps({"failed": failed}))


def _run(name, file, old, new, tmp):
    if file != "none":
        _plant(ORACLE_C if file == "c" else ORACLE_DAV, old, new)  # the site must exist, once
    work = os.path.join(tmp, name)
    os.makedirs(work, exist_ok=True)
    spec = os.path.join(work, "spec.json")
    with open(spec, "w") as f:
        json.dump({"file": file, "old": old, "new": new, "dir": work}, f)
    env = dict(os.environ, OMP_NUM_THREADS="2")
    p = subprocess.run([sys.executable, os.path.abspath(__file__), spec], capture_output=True, text=True,
                       timeout=600, env=env, cwd=ROOT)
    if p.returncode != 0:
        return name, None, p.returncode, p.stderr[-2000:]
    return name, json.loads(p.stdout.strip().splitlines()[-1])["failed"], 0, ""


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    tmp = str(tmp_path_factory.mktemp("oracle_mutants"))
    jobs = [("unmodified", "none", "", "")] + C_MUTANTS + PY_MUTANTS
    with concurrent.futures.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        futs = [ex.submit(_run, n, f, o, w, tmp) for n, f, o, w in jobs]
        return {r[0]: r[1:] for r in (fu.result() for fu in futs)}


def test_unmodified_copy_passes_every_pin(outcomes):
    failed, rc, err = outcomes["unmodified"]
    assert rc == 0 and failed == [], (failed, err)


@pytest.mark.parametrize("name", [m[0] for m in C_MUTANTS + PY_MUTANTS])
def test_planted_mistake_is_caught(outcomes, name):
    failed, rc, err = outcomes[name]
    if rc < 0:
        return  # the mutant crashed its process (killed by a signal): caught
    assert rc == 0, f"mutant {name}: child failed to run\n{err}"
    assert len(failed) >= 1, f"mutant {name} passes every pin"


if __name__ == "__main__":
    with open(sys.argv[1]) as f:
        _child(json.load(f))
