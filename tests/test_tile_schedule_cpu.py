"""Host-side check of the tile schedule behind the tensor-core sigma_3 epilogue.

The epilogue adds s_b G[J_b][p] into sigma(I_a, E_kl J_b) (Eq. 8, the beta
scatter of sigma_3) with plain loads and stores, no atomics.  That is race-free
only if the schedule keeps these properties:
  * every (string, replacement) entry of a tile appears exactly once, with its
    target, pair and sign;
  * within a tile each target belongs to one share (one thread);
  * within a share each target forms one contiguous run (a batch of 8 entries
    issues all its loads before any store, so a target may be stored once per
    run only);
  * a share is padded at its end only, with its own dummy target ns + k;
  * every tile has at least one step (the kernel clamps its loads to
    steps - 1) and whole steps of 128;
  * the shares stay balanced (least-loaded dealing: the longest share is at
    most the mean plus the longest run).
The tables are built here from the definition (Eq. 7: a+_k a_l on ascending
bitstrings), independently of the library and of the oracle, for the
benchmark's active spaces and for adversarial random tables.  No CUDA call.
"""
import itertools

import numpy as np
import pytest

R = 128


@pytest.fixture(scope="module")
def pkg():
    from paper_1707_04346_gb300 import build_ext

    build_ext.build()
    import paper_1707_04346_gb300 as p

    return p


def parity(v):
    """Parity of the number of set bits of each (non-negative) int64."""
    v = v.copy()
    for sh in (32, 16, 8, 4, 2, 1):
        v ^= v >> sh
    return v & 1


def replacement_table(norb, ne):
    """[ns][ne*(norb-ne)+ne] targets, packed pairs and signs of a+_k a_l."""
    strings = np.array(sorted(sum(1 << p for p in c) for c in itertools.combinations(range(norb), ne)),
                       dtype=np.int64)
    ns = len(strings)
    cols_t, cols_p, cols_s = [], [], []
    for l in range(norb):
        for k in range(norb):
            occ_l = (strings >> l) & 1
            empty_k = ((strings >> k) & 1) == 0
            ok = (occ_l == 1) & (empty_k | (k == l))
            lo, hi = min(k, l), max(k, l)
            between = ((1 << hi) - 1) ^ ((1 << (lo + 1)) - 1) if hi > lo else 0
            y = (strings & ~(1 << l)) | (1 << k)
            tgt = np.searchsorted(strings, y)
            par = parity(strings & between)
            cols_t.append(np.where(ok, tgt, -1))
            cols_p.append(np.full(ns, hi * (hi + 1) // 2 + lo))
            cols_s.append(np.where(par == 1, -1, 1))
    T, P, S = np.stack(cols_t, 1), np.stack(cols_p, 1), np.stack(cols_s, 1)
    keep = T >= 0
    per = ne * (norb - ne) + ne
    assert (keep.sum(1) == per).all()
    tgt = T[keep].reshape(ns, per)
    pair = P[keep].reshape(ns, per)
    sign = S[keep].reshape(ns, per)
    assert (strings[tgt] >= 0).all()
    return tgt.astype(np.int32), pair.astype(np.int32), sign.astype(np.int8)


def check_schedule(tgt, pair, sign, sched, toff):
    ns, per = tgt.shape
    ntiles = (ns + R - 1) // R
    assert toff.shape == (ntiles + 1,)
    assert toff[0] == 0 and toff[-1] == len(sched)
    lens = np.diff(toff.astype(np.int64))
    assert (lens % R == 0).all() and (lens >= R).all()  # whole steps, at least one per tile
    steps = lens // R
    # coordinates of every record: tile, step, share
    tile = np.repeat(np.arange(ntiles), lens)
    local = np.arange(len(sched)) - np.repeat(toff[:-1].astype(np.int64), lens)
    step, share = local // R, local % R
    target = (sched & 0xFFFF).astype(np.int64)
    jl = ((sched >> 16) & 127).astype(np.int64)
    pr = ((sched >> 23) & 255).astype(np.int64)
    neg = (sched >> 31).astype(np.int64)
    real = target < ns
    # padding: the dummy target of share k is ns + k, only after the real entries
    assert (target[~real] == ns + share[~real]).all()
    assert (jl[~real] == 0).all() and (pr[~real] == 0).all() and (neg[~real] == 0).all()
    key_ts = tile * R + share
    last_real = np.full(ntiles * R, -1)
    np.maximum.at(last_real, key_ts[real], step[real])
    first_pad = np.full(ntiles * R, np.iinfo(np.int64).max)
    np.minimum.at(first_pad, key_ts[~real], step[~real])
    assert (last_real < first_pad).all()
    # coverage: the real records are exactly the table's entries, each once
    x = np.repeat(np.arange(ns), per)
    want = np.sort(((((x // R) * R + x % R) * 65536 + tgt.ravel().astype(np.int64)) * 512
                    + pair.ravel().astype(np.int64) * 2 + (sign.ravel() < 0)))
    got = np.sort((((tile[real] * R + jl[real]) * 65536 + target[real]) * 512 + pr[real] * 2 + neg[real]))
    assert np.array_equal(want, got)
    assert (tile[real] * R + jl[real] < ns).all()
    # one owner per (tile, target), and one contiguous run within that share
    kt = tile[real] * 65536 + target[real]
    o = np.lexsort((step[real], kt))
    kt_s, sh_s, st_s = kt[o], share[real][o], step[real][o]
    same = kt_s[1:] == kt_s[:-1]
    assert (sh_s[1:][same] == sh_s[:-1][same]).all(), "a target has two owners in one tile"
    assert (st_s[1:][same] == st_s[:-1][same] + 1).all(), "a target's entries are not one run"
    # balance: the longest share is at most the mean share plus the longest run
    counts = np.bincount(tile[real], minlength=ntiles)
    _, run_len = np.unique(kt, return_counts=True)
    run_tile = np.unique(kt) // 65536
    max_run = np.zeros(ntiles, dtype=np.int64)
    np.maximum.at(max_run, run_tile, run_len)
    assert (steps <= np.ceil(counts / R) + max_run).all()
    return steps


@pytest.mark.parametrize("norb,ne", [(4, 2), (6, 3), (8, 4), (9, 2), (10, 5), (11, 8), (12, 6), (7, 7), (13, 1)])
def test_schedule_of_replacement_tables(pkg, norb, ne):
    tgt, pair, sign = replacement_table(norb, ne)
    sched, toff = pkg.fci_tile_schedule(tgt, pair, sign, norb * (norb + 1) // 2)
    check_schedule(tgt, pair, sign, sched, toff)


@pytest.mark.parametrize("norb", [14, 16, 18])
def test_schedule_of_benchmark_spaces(pkg, norb):
    """CAS(14,14), CAS(16,16) and CAS(18,18): the beta tables the sigma_3
    kernels use in the benchmark (3432, 12870 and 48620 strings)."""
    tgt, pair, sign = replacement_table(norb, norb // 2)
    sched, toff = pkg.fci_tile_schedule(tgt, pair, sign, norb * (norb + 1) // 2)
    steps = check_schedule(tgt, pair, sign, sched, toff)
    # near-perfect balance on these tables: about nsingle steps per tile
    assert steps.max() <= tgt.shape[1] + 8


@pytest.mark.parametrize("seed,ntarget", [(0, 1), (1, 3), (2, 50), (3, 5000)])
def test_schedule_of_adversarial_tables(pkg, seed, ntarget):
    """Random tables with few distinct targets (long runs, one target owning a
    whole tile) and a ragged last tile."""
    rng = np.random.default_rng(seed)
    ns, per, npair = 1000 + seed * 77, 37, 200
    tgt = rng.integers(0, min(ntarget, ns), (ns, per)).astype(np.int32)
    pair = rng.integers(0, npair, (ns, per)).astype(np.int32)
    sign = np.where(rng.random((ns, per)) < 0.5, -1, 1).astype(np.int8)
    sched, toff = pkg.fci_tile_schedule(tgt, pair, sign, npair)
    check_schedule(tgt, pair, sign, sched, toff)


def test_schedule_rejects_bad_tables(pkg):
    tgt, pair, sign = replacement_table(6, 3)
    for bad in ({"tgt": tgt + 100}, {"pair": pair + 300}, {"sign": sign * 0}):
        args = {"tgt": tgt, "pair": pair, "sign": sign}
        args.update(bad)
        with pytest.raises(pkg.FciError):
            pkg.fci_tile_schedule(args["tgt"], args["pair"], args["sign"], 21)
    with pytest.raises(pkg.FciError):
        pkg.fci_tile_schedule(tgt, pair, sign, 300)  # more than 256 pairs
    wide = np.zeros((4, 1025), dtype=np.int32)
    with pytest.raises(pkg.FciError):
        pkg.fci_tile_schedule(wide, wide, np.ones((4, 1025), dtype=np.int8), 1)  # nsingle > 1024
    big = np.zeros((65409, 1), dtype=np.int32)
    with pytest.raises(pkg.FciError):
        pkg.fci_tile_schedule(big, big, np.ones((65409, 1), dtype=np.int8), 1)


def test_checker_rejects_broken_schedules(pkg):
    """The checks above have teeth: a target split over two shares, a run
    broken inside a share and a dropped entry are each rejected."""
    tgt, pair, sign = replacement_table(10, 5)  # several runs per share
    sched, toff = pkg.fci_tile_schedule(tgt, pair, sign, 55)
    check_schedule(tgt, pair, sign, sched, toff)
    ns = tgt.shape[0]
    blk = sched[toff[0]:toff[1]].reshape(-1, R)  # tile 0, [step][share]

    def find_run_end(col, followed=False):
        """Step of the last entry of a run of length >= 2 in share col (one
        followed by another real entry if asked), or None."""
        t = blk[:, col] & 0xFFFF
        for j in range(1, len(t)):
            end = j + 1 == len(t) or t[j + 1] != t[j]
            nxt_real = j + 1 < len(t) and t[j + 1] < ns
            if t[j] == t[j - 1] and end and t[j] < ns and (nxt_real or not followed):
                return j
        return None

    # (a) the last entry of a run moved to the padding of another share
    bad = sched.copy()
    b = bad[toff[0]:toff[1]].reshape(-1, R)
    col = next(k for k in range(R) if any((blk[:, k] & 0xFFFF) >= ns))  # a share with padding
    src, j = next((k, find_run_end(k)) for k in range(R) if k != col and find_run_end(k) is not None)
    pad_j = int(np.argmax((b[:, col] & 0xFFFF) >= ns))
    b[pad_j, col], b[j, src] = b[j, src], ns + src
    with pytest.raises(AssertionError):
        check_schedule(tgt, pair, sign, bad, toff)
    # (b) a run broken inside its share: swap its last entry with the next run's first
    bad = sched.copy()
    b = bad[toff[0]:toff[1]].reshape(-1, R)
    k, j = next((k, find_run_end(k, True)) for k in range(R) if find_run_end(k, True) is not None)
    b[j, k], b[j + 1, k] = b[j + 1, k], b[j, k]
    with pytest.raises(AssertionError):
        check_schedule(tgt, pair, sign, bad, toff)
    # (c) an entry dropped (replaced by its share's dummy)
    bad = sched.copy()
    bad[toff[0] + 0 * R + 5] = ns + 5
    with pytest.raises(AssertionError):
        check_schedule(tgt, pair, sign, bad, toff)
