"""The FP32 tensor-core sigma_3 epilogue that keeps the sigma row in global
memory (used by spaces whose row does not fit in shared memory, e.g.
CAS(18,18)), forced on small spaces (fci_options.f32_row_global = 1) so that
whole vectors can be compared with the CPU oracle element by element, with
ragged beta tiles, n_alpha != n_beta, both slice counts, and together with
the same-spin terms through intermediate strings (same_spin_tc = 1, whose
adds go to global memory with red.global)."""
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


SPACES = [(4, 2, 2), (6, 3, 3), (7, 3, 4), (8, 4, 4), (8, 5, 3), (9, 4, 5), (10, 5, 5), (11, 6, 5)]


@pytest.mark.parametrize("splits,rtol", [(3, 2e-6), (2, 1e-4)])
@pytest.mark.parametrize("same_tc", [0, 1])
@pytest.mark.parametrize("norb,na,nb", SPACES)
def test_global_row_epilogue_matches_oracle(pkg, oracle_mod, norb, na, nb, same_tc, splits, rtol):
    h1, eri = fi.make_integrals(norb, 40)
    o = pkg.default_options(f32_row_global=1, same_spin_tc=same_tc, f32_splits=splits)
    ctx = pkg.fci_init(norb, na, nb, h1, eri, o)
    c = fi.make_vector(ctx.ndet).astype(np.float32).astype(np.float64)
    c_d = torch.from_numpy(c).to(DEV, torch.float32)
    s_d = torch.empty_like(c_d)
    pkg.fci_sigma(ctx, c_d, s_d)
    torch.cuda.synchronize()
    got = s_d.double().cpu().numpy()
    ref = oracle_mod.sigma(norb, na, nb, h1, eri, c)
    assert np.abs(got - ref).max() <= rtol * np.abs(ref).max()
    pkg.fci_free(ctx)
