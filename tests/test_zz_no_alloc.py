"""The allocation-free 1-RDM entry point (fci_rdm1_noalloc).

It exists for callers that cannot allocate device memory on this path (their
memory is owned by their own pool or a framework allocator, or they cannot
accept the device-wide synchronisation of cudaFree).  The test calls it
through the C ABI and checks it against fci_rdm1, which allocates its
scratch, and against the CPU oracle's density, on two calls in a row with
different vectors: the shared scratch array keeps the previous call's
contents, and the second result must not depend on them.  This file is
collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import fci_inputs as fi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_1707_04346_gb300 as p

    return p


def call_noalloc(lib, ctx, c, norb):
    gamma = np.full((norb, norb), np.nan)
    code = 0 if c.dtype == torch.float64 else 1
    stream = torch.cuda.current_stream()
    rc = lib.fci_rdm1_noalloc(ctx.handle, ctypes.c_void_p(c.data_ptr()), code,
                              gamma.ctypes.data_as(ctypes.c_void_p), ctypes.c_void_p(stream.cuda_stream))
    return rc, gamma


@pytest.mark.parametrize("norb,na,nb", [(8, 4, 4), (9, 5, 3)])
def test_noalloc_matches_rdm1_on_two_calls(pkg, oracle_mod, norb, na, nb):
    lib = pkg.load()
    h1, eri = fi.make_integrals(norb, 40)
    ctx = pkg.fci_init(norb, na, nb, h1, eri)
    v1, v2 = fi.make_vector(ctx.ndet, seed=11), fi.make_vector(ctx.ndet, seed=12)
    c1 = torch.from_numpy(v1).cuda()
    c2 = torch.from_numpy(v2).cuda()
    torch.cuda.synchronize()
    ref1 = pkg.fci_rdm1(ctx, c1)
    ref2 = pkg.fci_rdm1(ctx, c2)
    dev_before = torch.cuda.current_device()
    rc, g1 = call_noalloc(lib, ctx, c1, norb)
    assert rc == 0, lib.fci_last_error()
    rc, g2 = call_noalloc(lib, ctx, c2, norb)
    assert rc == 0, lib.fci_last_error()
    assert torch.cuda.current_device() == dev_before
    assert np.abs(g1 - ref1).max() < 1e-13
    assert np.abs(g2 - ref2).max() < 1e-13
    # and against the CPU oracle's density directly
    assert np.abs(g1 - oracle_mod.rdm1(norb, na, nb, v1)).max() < 1e-13
    assert np.abs(g2 - oracle_mod.rdm1(norb, na, nb, v2)).max() < 1e-13
    assert abs(np.trace(g2) - (na + nb)) < 1e-12
    pkg.fci_free(ctx)


def test_noalloc_rejects_spaces_beyond_its_limit(pkg):
    lib = pkg.load()
    # C(18,9) alpha strings x 90 entries > 2^21 scratch doubles, with only 48620
    # determinants (no beta electrons)
    norb, na, nb = 18, 9, 0
    h1, eri = fi.make_integrals(norb, 10)
    ctx = pkg.fci_init(norb, na, nb, h1, eri)
    c = torch.zeros(ctx.ndet, dtype=torch.float32, device="cuda")
    rc, _ = call_noalloc(lib, ctx, c, norb)
    assert rc == pkg.fci.FCI_ERR_ARG
    assert b"limit" in lib.fci_last_error()
    pkg.fci_free(ctx)
