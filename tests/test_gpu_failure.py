"""Failure paths on the GPU, made without faulting or hanging it.

* A bounded device wait that runs out: the library's self-test waits, through
  the same bounded-wait routine as the tensor-core sigma kernels, on a barrier
  that no thread arrives on.  The call must return FCI_ERR_TIMEOUT, clear the
  error word, and leave the context usable.
* A non-finite starting vector: the Davidson driver must stop with
  FCI_ERR_NAN instead of iterating to max_iter.
* Running out of device memory, simulated by the per-context cap
  (fci_options.max_device_bytes): fci_init and fci_davidson must return
  FCI_ERR_OOM, and a context that failed to get its Davidson workspace must
  still compute sigma.
"""
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


def test_bounded_wait_timeout_is_reported_and_context_stays_usable(pkg, oracle_mod):
    F = pkg.fci
    lib = pkg.load()
    norb, na, nb = 6, 3, 3
    h1, eri = fi.make_integrals(norb, 21)
    ctx = pkg.fci_init(norb, na, nb, h1, eri)
    assert lib.fci_check_wait_timeout(ctx.handle) == F.FCI_ERR_TIMEOUT
    assert b"bounded device wait" in lib.fci_last_error()
    assert pkg.fci_query(ctx, F.FCI_Q_DEVICE_ERROR) == 0  # the word was cleared
    # the tensor-core FP32 sigma still runs and is right
    c = fi.make_vector(ctx.ndet)
    c32 = torch.from_numpy(c).cuda().float()
    s32 = torch.empty_like(c32)
    pkg.fci_sigma(ctx, c32, s32)
    torch.cuda.synchronize()
    ref = oracle_mod.sigma(norb, na, nb, h1, eri, c.astype(np.float32).astype(np.float64))
    assert np.abs(s32.double().cpu().numpy() - ref).max() <= 2e-6 * np.abs(ref).max()
    assert pkg.fci_query(ctx, F.FCI_Q_DEVICE_ERROR) == 0
    pkg.fci_free(ctx)


@pytest.mark.parametrize("precision", [0, 1])
def test_infinite_guess_entry_returns_nan_error(pkg, precision):
    F = pkg.fci
    norb, na, nb = 6, 3, 3
    h1, eri = fi.make_integrals(norb, 21)
    ctx = pkg.fci_init(norb, na, nb, h1, eri, pkg.default_options(precision=precision))
    g = torch.zeros(ctx.ndet, dtype=torch.float64, device="cuda")
    g[0] = 1.0
    g[5] = float("inf")
    with pytest.raises(pkg.FciError) as ei:
        pkg.fci_davidson(ctx, 1, 1e-8, guess=g)
    assert ei.value.code == F.FCI_ERR_NAN
    # the context is still usable
    e = pkg.fci_davidson(ctx, 1, 1e-8)
    assert np.isfinite(e).all()
    pkg.fci_free(ctx)


def test_device_memory_cap_gives_oom_and_leaves_context_usable(pkg, oracle_mod):
    F = pkg.fci
    norb, na, nb = 8, 4, 4
    h1, eri = fi.make_integrals(norb, 40)
    with pytest.raises(pkg.FciError) as ei:
        pkg.fci_init(norb, na, nb, h1, eri, pkg.default_options(max_device_bytes=1e4))
    assert ei.value.code == F.FCI_ERR_OOM
    # room for the tables, not for the Davidson workspace
    free_ctx = pkg.fci_init(norb, na, nb, h1, eri)
    need = pkg.fci_query(free_ctx, F.FCI_Q_DEVICE_BYTES)
    pkg.fci_free(free_ctx)
    ctx = pkg.fci_init(norb, na, nb, h1, eri, pkg.default_options(max_device_bytes=float(need + 4096)))
    with pytest.raises(pkg.FciError) as ei:
        pkg.fci_davidson(ctx, 1, 1e-8)
    assert ei.value.code == F.FCI_ERR_OOM
    assert pkg.fci_query(ctx, F.FCI_Q_DEVICE_BYTES) == need  # the failed workspace was released
    c = fi.make_vector(ctx.ndet)
    c_d = torch.from_numpy(c).cuda()
    s_d = torch.empty_like(c_d)
    pkg.fci_sigma(ctx, c_d, s_d)
    torch.cuda.synchronize()
    ref = oracle_mod.sigma(norb, na, nb, h1, eri, c)
    assert np.abs(s_d.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()
    pkg.fci_free(ctx)
