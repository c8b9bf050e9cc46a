"""GPU parity of the two-particle density Gamma_pqrs = <c|E_pq E_rs|c> (and the
gamma_pq of the same pass) against the CPU oracle.

fci_rdm2 forms Gamma = sum_K D_qp(K) D_rs(K) as one Gram matrix on the bf16
tensor cores from six 8-bit digits of c in 45-bit fixed point, accumulated
exactly in 64-bit integers.  Bar: every element within 1e-12 ||c||^2 of the
oracle (the arithmetic leaves about 1e-14 ||c||^2: c's fixed-point rounding at
2^-46 of max|c| enters each product once, the digit products left out are
below 2^-46 of the leading one, and the integer unit is 2^-59 ||c||^2).
Because the integer adds are exact, the result does not depend on the order
of the adds: it is bitwise the same for every chunking of the determinants
and on every run.  Sizes span one and two 128-row tiles, ragged 48-row column
tiles and ragged 16-determinant steps; full size (CAS(14,14)) is checked
through the energy, the traces and the commutator relation.
"""
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


def rdm2(pkg, ctx, c, dtype=torch.float64):
    return pkg.fci_rdm2(ctx, torch.as_tensor(c).to(DEV, dtype))


# one and two row tiles (norb^2 + 1 = 17 .. 145 rows), spins without
# electrons, full strings, n_alpha != n_beta, N not a multiple of 16
SPACES = [(2, 1, 1), (4, 2, 2), (5, 3, 1), (5, 0, 2), (4, 4, 1), (6, 3, 3), (7, 4, 2), (8, 4, 4), (11, 2, 1),
          (12, 2, 2)]


@pytest.mark.parametrize("norb,na,nb", SPACES)
def test_rdm2_matches_oracle(pkg, oracle_mod, norb, na, nb):
    h1, eri = fi.make_integrals(norb, 30)
    ctx = pkg.fci_init(norb, na, nb, h1, eri)
    n = oracle_mod.ndet(norb, na, nb)
    for kind in ("random", "uniform"):
        c = fi.make_vector(n, kind=kind)
        c = c / np.linalg.norm(c)
        g1, g2 = rdm2(pkg, ctx, c)
        r2 = oracle_mod.rdm2(norb, na, nb, c)
        r1 = oracle_mod.rdm1(norb, na, nb, c)
        assert np.abs(g2 - r2).max() <= 1e-12, (kind, np.abs(g2 - r2).max())
        assert np.abs(g1 - r1).max() <= 1e-12
    pkg.fci_free(ctx)


def test_rdm2_fp32_input(pkg, oracle_mod):
    norb, na, nb = 8, 4, 3
    h1, eri = fi.make_integrals(norb, 30)
    ctx = pkg.fci_init(norb, na, nb, h1, eri)
    c = fi.make_vector(oracle_mod.ndet(norb, na, nb))
    c32 = (c / np.linalg.norm(c)).astype(np.float32)
    g1, g2 = rdm2(pkg, ctx, c32, torch.float32)
    c64 = c32.astype(np.float64)
    assert np.abs(g2 - oracle_mod.rdm2(norb, na, nb, c64)).max() <= 1e-12 * (c64 @ c64)
    assert np.abs(g1 - oracle_mod.rdm1(norb, na, nb, c64)).max() <= 1e-12 * (c64 @ c64)
    pkg.fci_free(ctx)


def test_rdm2_unnormalised_scales_with_norm(pkg, oracle_mod):
    """Any scale of c (the integer unit follows ||c||^2), including a vector
    whose weight sits on one determinant and tiny elsewhere."""
    norb, na, nb = 6, 3, 2
    h1, eri = fi.make_integrals(norb, 30)
    ctx = pkg.fci_init(norb, na, nb, h1, eri)
    n = oracle_mod.ndet(norb, na, nb)
    c = fi.make_vector(n)
    for scale in (1e-150, 3e-5, 1.0, 7e40):
        g1, g2 = rdm2(pkg, ctx, c * scale)
        ref = oracle_mod.rdm2(norb, na, nb, c * scale)
        assert np.abs(g2 - ref).max() <= 1e-12 * scale * scale * (c @ c)
    peaked = 1e-9 * fi.make_vector(n, seed=5)
    peaked[17] = 1.0
    _, g2 = rdm2(pkg, ctx, peaked)
    assert np.abs(g2 - oracle_mod.rdm2(norb, na, nb, peaked)).max() <= 1e-12 * (peaked @ peaked)
    pkg.fci_free(ctx)


def test_rdm2_bitwise_reproducible_over_chunks(pkg, oracle_mod):
    """Integer accumulation: the same bits for every chunking and every run."""
    norb, na, nb = 10, 5, 4
    h1, eri = fi.make_integrals(norb, 30)
    n = oracle_mod.ndet(norb, na, nb)  # 252 * 210 = 52920 determinants, 3308 steps of 16
    c = fi.make_vector(n)
    c /= np.linalg.norm(c)
    step = 6 * 104 * 32  # bytes of one 16-determinant step (104 rows)
    ref = None
    for chunk in (0.0, 1000.0 * step, 77.0 * step, 1.0 * step):
        ctx = pkg.fci_init(norb, na, nb, h1, eri, pkg.default_options(rdm2_chunk_bytes=chunk))
        for _ in range(2):
            g1, g2 = rdm2(pkg, ctx, c)
            if ref is None:
                ref = (g1, g2)
            assert np.array_equal(g1, ref[0]) and np.array_equal(g2, ref[1]), chunk
        pkg.fci_free(ctx)


def test_rdm2_single_determinant_exact(pkg, oracle_mod):
    norb, na, nb = 7, 3, 3
    h1, eri = fi.make_integrals(norb, 30)
    ctx = pkg.fci_init(norb, na, nb, h1, eri)
    n = oracle_mod.ndet(norb, na, nb)
    for idx in (0, 100, n - 1):
        c = np.zeros(n)
        c[idx] = -1.0
        g1, g2 = rdm2(pkg, ctx, c)
        assert np.array_equal(g2, oracle_mod.rdm2(norb, na, nb, c))
        assert np.array_equal(g1, oracle_mod.rdm1(norb, na, nb, c))
    pkg.fci_free(ctx)


def test_rdm2_zero_and_nonfinite(pkg):
    norb, na, nb = 5, 2, 2
    h1, eri = fi.make_integrals(norb, 30)
    ctx = pkg.fci_init(norb, na, nb, h1, eri)
    n = 100
    g1, g2 = rdm2(pkg, ctx, np.zeros(n))
    assert not g1.any() and not g2.any()
    c = fi.make_vector(n)
    c[3] = np.nan
    g1, g2 = rdm2(pkg, ctx, c)
    assert np.isnan(g2).all() and np.isnan(g1).all()
    c[3] = np.inf
    _, g2 = rdm2(pkg, ctx, c.astype(np.float32), torch.float32)
    assert np.isnan(g2).all()
    pkg.fci_free(ctx)


def test_rdm2_cas14_energy_traces_commutator(pkg):
    """CAS(14e,14o), 11.8 million determinants: the energy from the densities
    equals c^T sigma (FP64 sigma), gamma matches fci_rdm1, the partial traces
    give N gamma and the commutator [E_pq, E_rs] holds."""
    from fci_inputs import gpu

    norb, ne = 14, 7
    h1, eri = fi.make_integrals(norb, 100)
    ctx = pkg.fci_init(norb, ne, ne, h1, eri)
    N = ctx.ndet
    c = torch.empty(N, dtype=torch.float64, device=DEV)
    gpu.fill_pm1(c)
    c /= torch.linalg.vector_norm(c)
    s = torch.empty_like(c)
    pkg.fci_sigma(ctx, c, s)
    e_sigma = float(torch.dot(c, s))
    g1, g2 = pkg.fci_rdm2(ctx, c)
    e_dens = float(np.sum(h1 * g1) + 0.5 * (np.einsum("pqrs,pqrs->", eri, g2) - np.einsum("pqqs,ps->", eri, g1)))
    assert abs(e_dens - e_sigma) <= 1e-11 * max(1.0, abs(e_sigma))
    r1 = pkg.fci_rdm1(ctx, c)
    assert np.abs(g1 - r1).max() <= 1e-12
    assert np.abs(np.einsum("pqrr->pq", g2) - 2 * ne * g1).max() <= 1e-11
    d = np.eye(norb)
    lhs = g2 - g2.transpose(2, 3, 0, 1)
    rhs = np.einsum("qr,ps->pqrs", d, g1) - np.einsum("ps,rq->pqrs", d, g1)
    assert np.abs(lhs - rhs).max() <= 1e-12
    assert np.array_equal(g2, g2.transpose(3, 2, 1, 0))  # read from one integer per pair
    pkg.fci_free(ctx)


def test_rdm2_cas16_energy_and_traces(pkg):
    """CAS(16e,16o), 165.6 million determinants: 257 rows of D (three 128-row
    tiles, 11 Gram tiles), digit planes in about 490 chunks of 1 GiB; the
    energy from the densities equals c^T sigma (FP64 sigma of the large-space
    kernels), gamma matches fci_rdm1 and the partial traces give N gamma."""
    from fci_inputs import gpu

    norb, ne = 16, 8
    h1, eri = fi.make_integrals(norb, 100)
    ctx = pkg.fci_init(norb, ne, ne, h1, eri)
    c = torch.empty(ctx.ndet, dtype=torch.float64, device=DEV)
    gpu.fill_pm1(c)
    c /= torch.linalg.vector_norm(c)
    s = torch.empty_like(c)
    pkg.fci_sigma(ctx, c, s)
    e_sigma = float(torch.dot(c, s))
    del s
    g1, g2 = pkg.fci_rdm2(ctx, c)
    e_dens = float(np.sum(h1 * g1) + 0.5 * (np.einsum("pqrs,pqrs->", eri, g2) - np.einsum("pqqs,ps->", eri, g1)))
    assert abs(e_dens - e_sigma) <= 1e-11 * max(1.0, abs(e_sigma))
    assert np.abs(g1 - pkg.fci_rdm1(ctx, c)).max() <= 1e-12
    assert np.abs(np.einsum("pqrr->pq", g2) - 2 * ne * g1).max() <= 1e-11
    d = np.eye(norb)
    lhs = g2 - g2.transpose(2, 3, 0, 1)
    rhs = np.einsum("qr,ps->pqrs", d, g1) - np.einsum("ps,rq->pqrs", d, g1)
    assert np.abs(lhs - rhs).max() <= 1e-12
    pkg.fci_free(ctx)
