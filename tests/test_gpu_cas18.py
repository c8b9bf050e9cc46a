"""CAS(18e,18o): 48620 x 48620 = 2.36e9 determinants, FP32 sigma streamed
through HBM (same-spin terms through intermediate strings and sigma_3 with the
gather epilogue into a global sigma row, both on the tensor cores) and the FP64
sigma (the wide sliced kernels), checked on sampled rows against the oracle,
which regenerates the trial vector per index."""
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


def test_device_fill_matches_host(pkg):
    from fci_inputs import gpu

    for start in (0, 123456789, 2363904400 - 1000):
        x = torch.empty(1000, dtype=torch.float64, device=DEV)
        gpu.fill_pm1(x, start=start)
        assert np.array_equal(x.cpu().numpy(), fi.vector_pm1(start, 1000))
        y = torch.empty(1000, dtype=torch.float32, device=DEV)
        gpu.fill_pm1(y, start=start)
        assert np.array_equal(y.cpu().numpy(), fi.vector_pm1(start, 1000).astype(np.float32))


def test_cas18_fp32_sigma_sampled(pkg, oracle_mod):
    from fci_inputs import gpu

    norb, ne = 18, 9
    h1, eri = fi.make_integrals(norb, 100)
    ctx = pkg.fci_init(norb, ne, ne, h1, eri)
    N = ctx.ndet
    assert N == 48620 * 48620
    c = torch.empty(N, dtype=torch.float32, device=DEV)
    gpu.fill_pm1(c)
    s = torch.empty_like(c)
    pkg.fci_sigma(ctx, c, s)
    torch.cuda.synchronize()
    rng = np.random.default_rng(18)
    rows = np.unique(np.concatenate([[0, 1, 48620, N // 2, N - 1], rng.integers(0, N, 43)]))
    got = s[torch.from_numpy(rows).to(DEV)].double().cpu().numpy()
    ref = oracle_mod.sigma_rows_generated(norb, ne, ne, h1, eri, rows, fi.DEFAULT_VECTOR_SEED, fi.STREAM_C_PM1)
    # FP32: the input rounding (2^-24 relative) and FP32 accumulation of about 1e4
    # terms per element (sqrt(1e4) * 2^-24 relative to the largest term) stay below 1e-5
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()
    # split-BF16x3 (2 bf16 slices): about 1e-5 relative per product on top
    ctx3 = pkg.fci_init(norb, ne, ne, h1, eri, pkg.default_options(f32_splits=2))
    pkg.fci_sigma(ctx3, c, s)
    torch.cuda.synchronize()
    got3 = s[torch.from_numpy(rows).to(DEV)].double().cpu().numpy()
    pkg.fci_free(ctx3)
    assert np.abs(got3 - ref).max() <= 1e-4 * np.abs(ref).max()
    del c, s
    # FP64: all three terms through the wide tensor-core kernels (six 8-bit
    # slices, 64-bit integer accumulation), at the FP64 bar
    c64 = torch.empty(N, dtype=torch.float64, device=DEV)
    gpu.fill_pm1(c64)
    s64 = torch.empty_like(c64)
    pkg.fci_sigma(ctx, c64, s64)
    torch.cuda.synchronize()
    got64 = s64[torch.from_numpy(rows).to(DEV)].cpu().numpy()
    assert np.abs(got64 - ref).max() <= 1e-12 * np.abs(ref).max()
    del c64, s64
    pkg.fci_free(ctx)
