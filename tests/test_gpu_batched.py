"""Batched CASCI (many independent instances in lock-step) against the
single-instance path and the oracle."""
import numpy as np
import pytest

import fci_inputs as fi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_1707_04346_gb300 as p

    return p


def instances(spec, base_seed=1707):
    out = []
    for i, (n, na, nb) in enumerate(spec):
        rank = min(40, n * (n + 1) // 2)
        h1, eri = fi.make_integrals(n, rank, seed=base_seed + i)
        out.append((n, na, nb, h1, eri))
    return out


SPEC = [(6, 3, 3), (8, 4, 4), (10, 5, 5), (7, 4, 3), (6, 3, 3), (9, 4, 5), (4, 2, 2)]


@pytest.mark.parametrize("dtype,rtol,prec", [(torch.float64, 1e-12, 0), (torch.float32, 2e-5, 0),
                                             (torch.float32, 2e-5, 1)])
def test_batch_sigma_matches_single_instance(pkg, dtype, rtol, prec):
    """prec 1 (mixed) turns on the FP32 path that stages every off-diagonal
    alpha row of an output row at once (instances up to CAS(12,12) here)."""
    insts = instances(SPEC + ([(12, 6, 6)] if prec else []))
    batch = pkg.fci_batch_init(insts, pkg.default_options(precision=prec))
    total = batch.offset(batch.ninst)
    c = torch.from_numpy(fi.make_vector(total, seed=9)).to(DEV, dtype)
    s = torch.empty_like(c)
    pkg.fci_batch_sigma(batch, c, s)
    torch.cuda.synchronize()
    for i, (n, na, nb, h1, eri) in enumerate(insts):
        ctx = pkg.fci_init(n, na, nb, h1, eri)
        lo, hi = batch.offset(i), batch.offset(i + 1)
        ci = c[lo:hi].contiguous().double()
        si = torch.empty_like(ci)
        pkg.fci_sigma(ctx, ci, si)
        torch.cuda.synchronize()
        ref = si.cpu().numpy()
        got = s[lo:hi].double().cpu().numpy()
        assert np.abs(got - ref).max() <= rtol * np.abs(ref).max(), i
        pkg.fci_free(ctx)


def test_batch_davidson_fp64_matches_lapack(pkg, oracle_mod):
    spec = [(6, 3, 3), (8, 4, 4), (7, 4, 3), (6, 3, 3), (5, 3, 2), (8, 4, 4)]
    insts = instances(spec, base_seed=11)
    batch = pkg.fci_batch_init(insts, pkg.default_options(max_subspace=16))
    e = pkg.fci_batch_davidson(batch, 2, 1e-11)
    for i, (n, na, nb, h1, eri) in enumerate(insts):
        ref = np.linalg.eigvalsh(oracle_mod.hamiltonian(n, na, nb, h1, eri))[:2]
        assert np.abs(e[i] - ref).max() < 1e-9, (i, e[i], ref)
    st = pkg.fci_batch_stats(batch)
    assert st["iterations"] > 0 and st["graph_launches"] > 0 and st["sigma_launches"] > 0
    # device-driven iterations: one graph and one host synchronisation per chunk of up to 8
    assert st["graph_launches"] == st["host_syncs"] and st["graph_launches"] <= st["iterations"] / 2 + 1


def test_batch_davidson_mixed_matches_single_fp64(pkg):
    spec = [(10, 5, 5), (8, 4, 4), (6, 3, 3), (10, 5, 5), (9, 5, 4), (12, 6, 6)]
    insts = instances(spec, base_seed=31)
    batch = pkg.fci_batch_init(insts, pkg.default_options(precision=pkg.FCI_PREC_MIXED))
    e = pkg.fci_batch_davidson(batch, 2, 1e-10)
    for i, (n, na, nb, h1, eri) in enumerate(insts):
        ctx = pkg.fci_init(n, na, nb, h1, eri)
        ref = pkg.fci_davidson(ctx, 2, 1e-10)
        assert np.abs(e[i] - ref).max() < 1e-8, (i, e[i], ref)
        pkg.fci_free(ctx)


def test_batch_tuning_table(pkg):
    insts = instances([(6, 3, 3), (8, 4, 4), (6, 3, 3)])
    batch = pkg.fci_batch_init(insts)
    table = pkg.fci_batch_tuning(batch)
    assert sorted((n, d) for n, d, _ in table) == [(6, 0), (6, 1), (8, 0), (8, 1)]
    assert all(t in (32, 64, 128, 256) for _, _, t in table)


def test_batch_mixed_large_instance_first(pkg):
    """Instances large enough for the single-instance FP32 kernels (gated by
    their active flags inside the captured graphs), the largest first, so that
    a smaller instance is prepared after it."""
    spec = [(12, 6, 6), (10, 5, 5), (8, 4, 4), (6, 3, 3), (10, 5, 5)]
    insts = instances(spec, base_seed=57)
    batch = pkg.fci_batch_init(insts, pkg.default_options(precision=pkg.FCI_PREC_MIXED))
    e = pkg.fci_batch_davidson(batch, 2, 1e-10)
    for i, (n, na, nb, h1, eri) in enumerate(insts):
        ctx = pkg.fci_init(n, na, nb, h1, eri)
        ref = pkg.fci_davidson(ctx, 2, 1e-10)
        assert np.abs(e[i] - ref).max() < 1e-8, (i, e[i], ref)
        pkg.fci_free(ctx)


def test_interleaved_contexts_fp32_sigma_reproducible(pkg):
    """FP32 sigma of a large and a small context called alternately gives the
    same bits each time (one shared-memory opt-in serves both)."""
    big = instances([(12, 6, 6)], base_seed=5)[0]
    small = instances([(8, 4, 4)], base_seed=6)[0]
    cb, cs = pkg.fci_init(*big), pkg.fci_init(*small)
    xb = torch.from_numpy(fi.make_vector(cb.ndet, seed=1)).to(DEV, torch.float32)
    xs = torch.from_numpy(fi.make_vector(cs.ndet, seed=2)).to(DEV, torch.float32)
    outs = []
    for _ in range(2):
        sb, ss = torch.empty_like(xb), torch.empty_like(xs)
        pkg.fci_sigma(cb, xb, sb)
        pkg.fci_sigma(cs, xs, ss)
        torch.cuda.synchronize()
        outs.append((sb.cpu().numpy(), ss.cpu().numpy()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    pkg.fci_free(cb)
    pkg.fci_free(cs)


SPEC_ORACLE = [(6, 3, 3), (8, 4, 4), (10, 5, 5), (7, 4, 3), (9, 4, 5), (4, 2, 2), (8, 5, 3)]


@pytest.mark.parametrize("dtype,prec", [(torch.float64, 0), (torch.float32, 0), (torch.float32, 1)])
def test_batch_sigma_matches_oracle(pkg, oracle_mod, dtype, prec):
    """Every instance's slice of the batched sigma against the CPU oracle:
    full vectors up to CAS(10,10), 200 sampled rows of a CAS(12,12) instance.
    FP64: 1e-12 normwise; FP32 (the input rounded to FP32 on both sides):
    2e-6 normwise, as for the single-instance FP32 sigma.  prec 1 (mixed) turns
    on the FP32 kernel that stages all off-diagonal alpha rows at once."""
    insts = instances(SPEC_ORACLE + [(12, 6, 6)], base_seed=71)
    batch = pkg.fci_batch_init(insts, pkg.default_options(precision=prec))
    total = batch.offset(batch.ninst)
    v = fi.make_vector(total, seed=13)
    if dtype == torch.float32:
        v = v.astype(np.float32).astype(np.float64)
    c = torch.from_numpy(v).to(DEV, dtype)
    s = torch.empty_like(c)
    pkg.fci_batch_sigma(batch, c, s)
    torch.cuda.synchronize()
    got_all = s.double().cpu().numpy()
    rtol = 1e-12 if dtype == torch.float64 else 2e-6
    for i, (n, na, nb, h1, eri) in enumerate(insts):
        lo, hi = batch.offset(i), batch.offset(i + 1)
        ci, got = v[lo:hi], got_all[lo:hi]
        if n <= 10:
            ref = oracle_mod.sigma(n, na, nb, h1, eri, ci)
            assert np.abs(got - ref).max() <= rtol * np.abs(ref).max(), i
        else:
            rows = np.random.default_rng(i).choice(hi - lo, 200, replace=False)
            ref = oracle_mod.sigma_rows(n, na, nb, h1, eri, ci, rows)
            assert np.abs(got[rows] - ref).max() <= rtol * np.abs(got).max(), i


def test_batch_davidson_mixed_matches_lapack(pkg, oracle_mod):
    """Mixed-precision batched energies (FP32 sigma, FP64 refinement) against
    LAPACK on the oracle's Hamiltonian, within the 1e-8 Eh target."""
    spec = [(6, 3, 3), (8, 4, 4), (7, 4, 3), (6, 3, 3), (5, 3, 2), (8, 4, 4), (8, 5, 3)]
    insts = instances(spec, base_seed=23)
    batch = pkg.fci_batch_init(insts, pkg.default_options(precision=pkg.FCI_PREC_MIXED, max_subspace=16))
    e = pkg.fci_batch_davidson(batch, 2, 1e-10)
    for i, (n, na, nb, h1, eri) in enumerate(insts):
        ref = np.linalg.eigvalsh(oracle_mod.hamiltonian(n, na, nb, h1, eri))[:2]
        assert np.abs(e[i] - ref).max() < 1e-8, (i, e[i], ref)
