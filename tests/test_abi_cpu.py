"""Host-side checks of the C ABI: the library builds for sm_103a, loads, and
exports every function include/fci.h declares; argument checks that run
before any CUDA call return FCI_ERR_ARG.  No kernel runs here."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1707_04346_gb300 import build_ext, fci

    build_ext.build()
    return fci.load()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "fci.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fci_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_abi():
    names = declared_functions()
    for must in ("fci_init", "fci_sigma", "fci_davidson", "fci_rdm1", "fci_free", "fci_last_error"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1707_04346_gb300 import fci

    names = declared_functions()
    for n in names:
        assert hasattr(lib, n), f"{n} not exported"
    assert sorted(fci.EXPORTED) == names


def test_binary_targets_sm103a():
    from paper_1707_04346_gb300 import build_ext

    assert "arch=compute_103a,code=sm_103a" in " ".join(build_ext.ARCH)


def test_default_options(lib):
    from paper_1707_04346_gb300 import fci

    o = fci.default_options()
    assert o.struct_size == ctypes.sizeof(fci.fci_options)
    assert o.max_subspace == 24 and o.max_iter == 300 and o.precision == fci.FCI_PREC_FP64
    assert o.device == -1 and o.symmetry_tol == 1e-12 and o.f32_splits == 3


def _init(lib, norb, na, nb, h1, eri, opt=None):
    from paper_1707_04346_gb300 import fci

    h = ctypes.c_void_p()
    h1 = np.ascontiguousarray(h1, dtype=np.float64)
    eri = np.ascontiguousarray(eri, dtype=np.float64)
    o = opt if opt is not None else fci.default_options()
    rc = lib.fci_init(ctypes.byref(h), norb, na, nb, h1.ctypes.data_as(ctypes.c_void_p),
                      eri.ctypes.data_as(ctypes.c_void_p), ctypes.byref(o))
    return rc, lib.fci_last_error().decode()


def test_bad_arguments_are_rejected_before_any_cuda_call(lib):
    from paper_1707_04346_gb300 import fci

    import fci_inputs as fi

    h1, eri = fi.make_integrals(4, 10)
    assert _init(lib, 0, 0, 0, h1, eri)[0] == fci.FCI_ERR_ARG
    assert _init(lib, 31, 1, 1, np.zeros((31, 31)), np.zeros(1))[0] == fci.FCI_ERR_ARG
    assert _init(lib, 4, 5, 2, h1, eri)[0] == fci.FCI_ERR_ARG
    bad = h1.copy()
    bad[0, 1] += 1e-6
    rc, msg = _init(lib, 4, 2, 2, bad, eri)
    assert rc == fci.FCI_ERR_ARG and "symmetric" in msg
    bad_eri = eri.copy()
    bad_eri[0, 1, 2, 3] += 1e-3
    rc, msg = _init(lib, 4, 2, 2, h1, bad_eri)
    assert rc == fci.FCI_ERR_ARG and "8-fold" in msg
    nan_h = h1.copy()
    nan_h[2, 2] = np.nan
    assert _init(lib, 4, 2, 2, nan_h, eri)[0] == fci.FCI_ERR_ARG
    o = fci.default_options()
    o.struct_size = 3
    assert _init(lib, 4, 2, 2, h1, eri, o)[0] == fci.FCI_ERR_ARG
    # 2^21 string limit: C(24, 12) = 2,704,156
    rc, msg = _init(lib, 24, 12, 12, np.zeros((24, 24)), np.zeros(24 ** 4))
    assert rc == fci.FCI_ERR_ARG and "strings" in msg
    # NULL context pointers on the other calls
    assert lib.fci_sigma(None, None, None, 0, None) == fci.FCI_ERR_ARG
    assert lib.fci_query(None, 1) == -1
    assert lib.fci_rdm2(None, None, 0, None, None) == fci.FCI_ERR_ARG
    # the short form: argument errors leave no default context behind
    assert lib.fci_init_default(0, 0, 0, None, None) == fci.FCI_ERR_ARG
    assert lib.fci_default_context() is None
    assert lib.fci_free_default() == fci.FCI_OK
    assert lib.fci_free(None) == fci.FCI_OK


def test_missing_library_fails_loudly(tmp_path):
    from paper_1707_04346_gb300 import fci

    with pytest.raises(RuntimeError, match="not built"):
        fci.load.__wrapped__(str(tmp_path / "nope.so")) if hasattr(fci.load, "__wrapped__") else _load_missing(fci, tmp_path)


def _load_missing(fci, tmp_path):
    saved = fci._lib
    fci._lib = None
    try:
        fci.load(str(tmp_path / "nope.so"))
    finally:
        fci._lib = saved


def test_option_validation_on_host(lib):
    from paper_1707_04346_gb300 import fci

    import fci_inputs as fi

    h1, eri = fi.make_integrals(4, 10)
    for field, bad in (("f32_splits", 4), ("precision", 7), ("max_subspace", 1), ("max_iter", 0),
                       ("same_spin_tc", 2), ("f64_kernels", 4), ("basis_f32", 3), ("spin_parity", 2),
                       ("spin_parity", -2), ("f32_row_global", 2), ("rdm2_chunk_bytes", -1.0),
                       ("f64_same_spin", 2), ("f64_same_spin", -1)):
        o = fci.default_options()
        setattr(o, field, bad)
        assert _init(lib, 4, 2, 2, h1, eri, o)[0] == fci.FCI_ERR_ARG, field
    # a spin parity needs Ms = 0 (one string space for both spins)
    o = fci.default_options(spin_parity=1)
    rc, msg = _init(lib, 4, 2, 1, h1, eri, o)
    assert rc == fci.FCI_ERR_ARG and "spin_parity" in msg


def test_default_options_match_header(lib):
    """The binding's struct has the header's layout (struct_size filled by the library)."""
    from paper_1707_04346_gb300 import fci

    o = fci.default_options()
    assert o.struct_size == ctypes.sizeof(fci.fci_options)
    assert (o.max_subspace, o.max_iter, o.f32_splits, o.same_spin_tc) == (24, 300, 3, 0)
    assert (o.f64_kernels, o.basis_f32, o.spin_parity, o.f32_row_global) == (0, 0, 0, 0)
    assert o.rdm2_chunk_bytes == 0.0 and o.f64_same_spin == 0


def test_batch_rejects_bad_instances_on_host(lib):
    from paper_1707_04346_gb300 import fci

    h = ctypes.c_void_p()
    z = np.zeros(17 ** 4)
    inst = (fci.fci_instance * 1)(fci.fci_instance(17, 8, 8, z.ctypes.data, z.ctypes.data))
    assert lib.fci_batch_init(ctypes.byref(h), 1, inst, None) == fci.FCI_ERR_ARG
    assert lib.fci_batch_init(ctypes.byref(h), 0, inst, None) == fci.FCI_ERR_ARG
    assert lib.fci_batch_free(None) == fci.FCI_OK
