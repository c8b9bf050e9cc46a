"""Python binding of the C ABI in include/fci.h (argument marshalling only).

Every function here forwards to ``libfci_gb300.so``; nothing is computed in
Python.  Device vectors are torch CUDA tensors (PyTorch provides memory and
streams only).  If the library has not been built, loading raises
``RuntimeError``: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfci_gb300.so")

(FCI_OK, FCI_ERR_ARG, FCI_ERR_OOM, FCI_ERR_CUDA, FCI_ERR_NOCONV, FCI_ERR_TIMEOUT, FCI_ERR_STATE, FCI_ERR_NAN,
 FCI_ERR_RANGE) = range(9)
FCI_F64, FCI_F32 = 0, 1
FCI_PREC_FP64, FCI_PREC_MIXED = 0, 1
FCI_F64_AUTO, FCI_F64_FMA, FCI_F64_SLICED, FCI_F64_WIDE = 0, 1, 2, 3
FCI_SS_AUTO, FCI_SS_FAMILY = 0, 1
FCI_Q_NDET, FCI_Q_NSTR_ALPHA, FCI_Q_NSTR_BETA = 1, 2, 3
FCI_Q_NSINGLE_ALPHA, FCI_Q_NSINGLE_BETA, FCI_Q_NPAIR = 4, 5, 6
FCI_Q_DEVICE_BYTES, FCI_Q_ITERATIONS, FCI_Q_SIGMA_CALLS, FCI_Q_DEVICE_ERROR = 7, 8, 9, 10

EXPORTED = [
    "fci_default_options", "fci_init", "fci_free", "fci_init_default", "fci_default_context", "fci_free_default", "fci_sigma", "fci_hdiag", "fci_davidson",
    "fci_davidson_log", "fci_rdm1", "fci_rdm2", "fci_get_strings", "fci_get_single_table", "fci_query",
    "fci_last_error", "fci_profile_enable", "fci_profile_read", "fci_profile_kernel_name",
    "fci_rdm1_noalloc", "fci_batch_init", "fci_batch_davidson", "fci_batch_sigma", "fci_batch_offset",
    "fci_batch_tuning", "fci_batch_stats", "fci_batch_free", "fci_tile_schedule", "fci_check_wait_timeout",
]


class FciError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"fci error {code}: {msg}")
        self.code = code


class fci_instance(ctypes.Structure):
    _fields_ = [
        ("norb", ctypes.c_int),
        ("nalpha", ctypes.c_int),
        ("nbeta", ctypes.c_int),
        ("h1", ctypes.c_void_p),
        ("eri", ctypes.c_void_p),
    ]


class fci_options(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_int),
        ("device", ctypes.c_int),
        ("max_subspace", ctypes.c_int),
        ("max_iter", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("mixed_switch", ctypes.c_double),
        ("symmetry_tol", ctypes.c_double),
        ("f32_splits", ctypes.c_int),
        ("same_spin_tc", ctypes.c_int),
        ("f64_kernels", ctypes.c_int),
        ("max_device_bytes", ctypes.c_double),
        ("f32_row_global", ctypes.c_int),
        ("basis_f32", ctypes.c_int),
        ("spin_parity", ctypes.c_int),
        ("f64_same_spin", ctypes.c_int),
        ("rdm2_chunk_bytes", ctypes.c_double),
    ]


_lib = None
_lock = threading.Lock()


def load(path: str = LIB_PATH):
    """Load the shared library and declare every exported signature."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path} is missing (run __graft_entry__.build())")
        lib = ctypes.CDLL(path)
        vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
        lib.fci_default_options.restype = None
        lib.fci_default_options.argtypes = [ctypes.POINTER(fci_options)]
        lib.fci_init.restype = i32
        lib.fci_init.argtypes = [ctypes.POINTER(vp), i32, i32, i32, vp, vp, ctypes.POINTER(fci_options)]
        lib.fci_free.restype = i32
        lib.fci_free.argtypes = [vp]
        lib.fci_init_default.restype = i32
        lib.fci_init_default.argtypes = [i32, i32, i32, vp, vp]
        lib.fci_default_context.restype = vp
        lib.fci_default_context.argtypes = []
        lib.fci_free_default.restype = i32
        lib.fci_free_default.argtypes = []
        lib.fci_sigma.restype = i32
        lib.fci_sigma.argtypes = [vp, vp, vp, i32, vp]
        lib.fci_hdiag.restype = i32
        lib.fci_hdiag.argtypes = [vp, vp, vp]
        lib.fci_davidson.restype = i32
        lib.fci_davidson.argtypes = [vp, i32, dbl, vp, vp, vp]
        lib.fci_davidson_log.restype = i32
        lib.fci_davidson_log.argtypes = [vp, vp, i32, ctypes.POINTER(i32)]
        lib.fci_rdm1.restype = i32
        lib.fci_rdm1.argtypes = [vp, vp, i32, vp]
        lib.fci_rdm2.restype = i32
        lib.fci_rdm2.argtypes = [vp, vp, i32, vp, vp]
        lib.fci_get_strings.restype = i32
        lib.fci_get_strings.argtypes = [vp, i32, vp]
        lib.fci_get_single_table.restype = i32
        lib.fci_get_single_table.argtypes = [vp, i32, vp, vp, vp, vp]
        lib.fci_query.restype = i64
        lib.fci_query.argtypes = [vp, i32]
        lib.fci_last_error.restype = ctypes.c_char_p
        lib.fci_last_error.argtypes = []
        lib.fci_profile_enable.restype = i32
        lib.fci_profile_enable.argtypes = [vp, i32]
        lib.fci_profile_read.restype = i32
        lib.fci_profile_read.argtypes = [vp, vp, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)]
        lib.fci_batch_init.restype = i32
        lib.fci_batch_init.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(fci_instance), ctypes.POINTER(fci_options)]
        lib.fci_batch_davidson.restype = i32
        lib.fci_batch_davidson.argtypes = [vp, i32, dbl, vp]
        lib.fci_batch_sigma.restype = i32
        lib.fci_batch_sigma.argtypes = [vp, vp, vp, i32, vp]
        lib.fci_batch_offset.restype = i64
        lib.fci_batch_offset.argtypes = [vp, i32]
        lib.fci_batch_tuning.restype = i32
        lib.fci_batch_tuning.argtypes = [vp, vp, i32, ctypes.POINTER(i32)]
        lib.fci_batch_stats.restype = i64
        lib.fci_batch_stats.argtypes = [vp, i32]
        lib.fci_batch_free.restype = i32
        lib.fci_batch_free.argtypes = [vp]
        lib.fci_check_wait_timeout.restype = i32
        lib.fci_check_wait_timeout.argtypes = [vp]
        lib.fci_rdm1_noalloc.restype = i32
        lib.fci_rdm1_noalloc.argtypes = [vp, vp, i32, vp, vp]
        lib.fci_profile_kernel_name.restype = ctypes.c_char_p
        lib.fci_profile_kernel_name.argtypes = [vp, i32]
        lib.fci_tile_schedule.restype = i32
        lib.fci_tile_schedule.argtypes = [i64, i32, i32, vp, vp, vp, vp, i64, ctypes.POINTER(i64), vp]
        _lib = lib
    return _lib


def _check(rc: int):
    if rc != FCI_OK:
        raise FciError(rc, load().fci_last_error().decode(errors="replace"))


def _np_ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _dev_ptr(t, dtype_code: int | None = None):
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA torch tensor")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if dtype_code is not None:
        want = torch.float64 if dtype_code == FCI_F64 else torch.float32
        if t.dtype != want:
            raise TypeError(f"expected {want}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


def _dtype_code(t) -> int:
    import torch

    if t.dtype == torch.float64:
        return FCI_F64
    if t.dtype == torch.float32:
        return FCI_F32
    raise TypeError("CI vectors must be float64 or float32")


def _stream_ptr(stream):
    if stream is None:
        import torch

        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def default_options(**kw) -> fci_options:
    o = fci_options()
    load().fci_default_options(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class FciContext:
    """Owns a ``fci_ctx*``; freed by :func:`fci_free` or garbage collection
    (a view of the library's default context, ``owned=False``, frees nothing)."""

    def __init__(self, handle: ctypes.c_void_p, norb: int, nalpha: int, nbeta: int, owned: bool = True):
        self.handle = handle
        self.norb, self.nalpha, self.nbeta = norb, nalpha, nbeta
        self.owned = owned

    @property
    def ndet(self) -> int:
        return fci_query(self, FCI_Q_NDET)

    @property
    def nstr(self) -> tuple[int, int]:
        return fci_query(self, FCI_Q_NSTR_ALPHA), fci_query(self, FCI_Q_NSTR_BETA)

    def __del__(self):
        try:
            fci_free(self)
        except Exception:
            pass


def fci_init(norb: int, nalpha: int, nbeta: int, h1, eri, options: fci_options | None = None) -> FciContext:
    lib = load()
    h1 = np.ascontiguousarray(h1, dtype=np.float64)
    eri = np.ascontiguousarray(eri, dtype=np.float64)
    if h1.size != norb * norb or eri.size != norb ** 4:
        raise ValueError("h1 must have norb^2 and eri norb^4 elements")
    handle = ctypes.c_void_p()
    opt = options if options is not None else default_options()
    _check(lib.fci_init(ctypes.byref(handle), norb, nalpha, nbeta, _np_ptr(h1), _np_ptr(eri), ctypes.byref(opt)))
    return FciContext(handle, norb, nalpha, nbeta)


def fci_free(ctx: FciContext):
    if ctx.handle and getattr(ctx, "owned", True):
        load().fci_free(ctx.handle)
    ctx.handle = None


def fci_init_default(norb: int, nalpha: int, nbeta: int, h1, eri) -> FciContext:
    """The short form fci_init(norb, nalpha, nbeta, h1, eri): (re)builds the
    library's default context with default options and returns a view of it."""
    lib = load()
    h1 = np.ascontiguousarray(h1, dtype=np.float64)
    eri = np.ascontiguousarray(eri, dtype=np.float64)
    if h1.size != norb * norb or eri.size != norb ** 4:
        raise ValueError("h1 must have norb^2 and eri norb^4 elements")
    _check(lib.fci_init_default(norb, nalpha, nbeta, _np_ptr(h1), _np_ptr(eri)))
    return FciContext(ctypes.c_void_p(lib.fci_default_context()), norb, nalpha, nbeta, owned=False)


def fci_free_default():
    _check(load().fci_free_default())


def fci_sigma(ctx: FciContext, c, sigma, stream=None):
    """sigma = H c on the device (dtype taken from the tensors)."""
    code = _dtype_code(c)
    _check(load().fci_sigma(ctx.handle, _dev_ptr(c, code), _dev_ptr(sigma, code), code, _stream_ptr(stream)))
    return sigma


def fci_sigma_ptr(ctx: FciContext, c_ptr: int, sigma_ptr: int, dtype_code: int, stream_ptr: int):
    """Raw-pointer form (for CUDA-graph capture and benchmarks)."""
    _check(load().fci_sigma(ctx.handle, ctypes.c_void_p(c_ptr), ctypes.c_void_p(sigma_ptr), dtype_code,
                            ctypes.c_void_p(stream_ptr)))


def fci_hdiag(ctx: FciContext, out, stream=None):
    _check(load().fci_hdiag(ctx.handle, _dev_ptr(out, FCI_F64), _stream_ptr(stream)))
    return out


def fci_davidson(ctx: FciContext, nroots: int, tol: float, vecs=None, guess=None) -> np.ndarray:
    e = np.zeros(nroots)
    vp = _dev_ptr(vecs, FCI_F64) if vecs is not None else None
    gp = _dev_ptr(guess, FCI_F64) if guess is not None else None
    _check(load().fci_davidson(ctx.handle, nroots, float(tol), _np_ptr(e), vp, gp))
    return e


def fci_davidson_log(ctx: FciContext, nroots: int) -> np.ndarray:
    cnt = ctypes.c_int(0)
    load().fci_davidson_log(ctx.handle, None, 0, ctypes.byref(cnt))
    out = np.zeros((max(cnt.value, 0), nroots + 3))
    if cnt.value:
        _check(load().fci_davidson_log(ctx.handle, _np_ptr(out), cnt.value, ctypes.byref(cnt)))
    return out


def fci_rdm1(ctx: FciContext, c) -> np.ndarray:
    g = np.zeros((ctx.norb, ctx.norb))
    code = _dtype_code(c)
    _check(load().fci_rdm1(ctx.handle, _dev_ptr(c, code), code, _np_ptr(g)))
    return g


def fci_rdm2(ctx: FciContext, c):
    """(gamma [n][n], Gamma [n][n][n][n]): Gamma_pqrs = <c|E_pq E_rs|c> and
    gamma_pq = <c|E_pq|c> from one tensor-core pass (see include/fci.h)."""
    n = ctx.norb
    g1 = np.zeros((n, n))
    g2 = np.zeros((n, n, n, n))
    code = _dtype_code(c)
    _check(load().fci_rdm2(ctx.handle, _dev_ptr(c, code), code, _np_ptr(g1), _np_ptr(g2)))
    return g1, g2


def fci_rdm1_noalloc(ctx: FciContext, c, stream=None) -> np.ndarray:
    """1-RDM without device allocation (fixed library scratch; see include/fci.h)."""
    g = np.zeros((ctx.norb, ctx.norb))
    code = _dtype_code(c)
    _check(load().fci_rdm1_noalloc(ctx.handle, _dev_ptr(c, code), code, _np_ptr(g), _stream_ptr(stream)))
    return g


def fci_get_strings(ctx: FciContext, spin: int) -> np.ndarray:
    n = fci_query(ctx, FCI_Q_NSTR_ALPHA if spin == 0 else FCI_Q_NSTR_BETA)
    out = np.zeros(n, dtype=np.uint32)
    _check(load().fci_get_strings(ctx.handle, spin, _np_ptr(out)))
    return out


def fci_get_single_table(ctx: FciContext, spin: int):
    n = fci_query(ctx, FCI_Q_NSTR_ALPHA if spin == 0 else FCI_Q_NSTR_BETA)
    per = fci_query(ctx, FCI_Q_NSINGLE_ALPHA if spin == 0 else FCI_Q_NSINGLE_BETA)
    tgt = np.zeros((n, per), dtype=np.int32)
    kk = np.zeros((n, per), dtype=np.int8)
    ll = np.zeros((n, per), dtype=np.int8)
    sg = np.zeros((n, per), dtype=np.int8)
    _check(load().fci_get_single_table(ctx.handle, spin, _np_ptr(tgt), _np_ptr(kk), _np_ptr(ll), _np_ptr(sg)))
    return tgt, kk, ll, sg


def fci_tile_schedule(tgt, pair, sign, npair: int):
    """Tile schedule of the tensor-core sigma_3 epilogue for a replacement
    table given on the host (row-major [ns][nsingle] targets, packed pair
    indices and signs).  Host-only.  Returns (sched uint32 [nsched],
    toff int32 [ceil(ns/128) + 1])."""
    tgt = np.ascontiguousarray(tgt, dtype=np.int32)
    pair = np.ascontiguousarray(pair, dtype=np.int32)
    sign = np.ascontiguousarray(sign, dtype=np.int8)
    if tgt.ndim != 2 or pair.shape != tgt.shape or sign.shape != tgt.shape:
        raise ValueError("tgt, pair and sign must be [ns][nsingle] arrays of one shape")
    ns, per = tgt.shape
    toff = np.zeros((ns + 127) // 128 + 1, dtype=np.int32)
    n = ctypes.c_int64(0)
    lib = load()
    _check(lib.fci_tile_schedule(ns, per, npair, _np_ptr(tgt), _np_ptr(pair), _np_ptr(sign), None, 0,
                                 ctypes.byref(n), _np_ptr(toff)))
    sched = np.zeros(n.value, dtype=np.uint32)
    _check(lib.fci_tile_schedule(ns, per, npair, _np_ptr(tgt), _np_ptr(pair), _np_ptr(sign), _np_ptr(sched),
                                 n.value, ctypes.byref(n), _np_ptr(toff)))
    return sched, toff


def fci_query(ctx: FciContext, what: int) -> int:
    return int(load().fci_query(ctx.handle, what))


def fci_profile_enable(ctx: FciContext, on: bool = True):
    _check(load().fci_profile_enable(ctx.handle, 1 if on else 0))


def fci_profile_read(ctx: FciContext):
    """Per-kernel milliseconds of the recorded sigma calls: (names, array[nrec, nk])."""
    nrec, nk = ctypes.c_int(0), ctypes.c_int(0)
    _check(load().fci_profile_read(ctx.handle, None, 0, ctypes.byref(nrec), ctypes.byref(nk)))
    out = np.zeros((nrec.value, max(nk.value, 1)))
    _check(load().fci_profile_read(ctx.handle, _np_ptr(out), nrec.value, ctypes.byref(nrec), ctypes.byref(nk)))
    names = [load().fci_profile_kernel_name(ctx.handle, i).decode() for i in range(nk.value)]
    return names, out[: nrec.value, : nk.value]


class FciBatch:
    """Owns a ``fci_batch*`` (many independent CASCI instances)."""

    def __init__(self, handle, insts, keep):
        self.handle = handle
        self.insts = insts
        self._keep = keep  # host integral buffers referenced during init

    @property
    def ninst(self) -> int:
        return len(self.insts)

    def offset(self, i: int) -> int:
        return int(load().fci_batch_offset(self.handle, i))

    def __del__(self):
        try:
            fci_batch_free(self)
        except Exception:
            pass


def fci_batch_init(instances, options: fci_options | None = None) -> FciBatch:
    """instances: sequence of (norb, nalpha, nbeta, h1, eri)."""
    lib = load()
    arr = (fci_instance * len(instances))()
    keep = []
    for i, (norb, na, nb, h1, eri) in enumerate(instances):
        h1 = np.ascontiguousarray(h1, dtype=np.float64)
        eri = np.ascontiguousarray(eri, dtype=np.float64)
        keep += [h1, eri]
        arr[i] = fci_instance(norb, na, nb, h1.ctypes.data, eri.ctypes.data)
    handle = ctypes.c_void_p()
    opt = options if options is not None else default_options()
    _check(lib.fci_batch_init(ctypes.byref(handle), len(instances), arr, ctypes.byref(opt)))
    return FciBatch(handle, [tuple(x[:3]) for x in instances], keep)


def fci_batch_davidson(batch: FciBatch, nroots: int, tol: float) -> np.ndarray:
    e = np.zeros((batch.ninst, nroots))
    _check(load().fci_batch_davidson(batch.handle, nroots, float(tol), _np_ptr(e)))
    return e


def fci_batch_sigma(batch: FciBatch, c, sigma, stream=None):
    code = _dtype_code(c)
    _check(load().fci_batch_sigma(batch.handle, _dev_ptr(c, code), _dev_ptr(sigma, code), code, _stream_ptr(stream)))
    return sigma


def fci_batch_tuning(batch: FciBatch):
    cnt = ctypes.c_int(0)
    load().fci_batch_tuning(batch.handle, None, 0, ctypes.byref(cnt))
    out = np.zeros(3 * max(cnt.value, 1), dtype=np.int32)
    _check(load().fci_batch_tuning(batch.handle, _np_ptr(out), cnt.value, ctypes.byref(cnt)))
    return [tuple(int(v) for v in out[3 * i:3 * i + 3]) for i in range(cnt.value)]


def fci_batch_stats(batch: FciBatch) -> dict:
    lib = load()
    return {"iterations": int(lib.fci_batch_stats(batch.handle, 0)),
            "sigma_launches": int(lib.fci_batch_stats(batch.handle, 1)),
            "graph_launches": int(lib.fci_batch_stats(batch.handle, 2)),
            "host_syncs": int(lib.fci_batch_stats(batch.handle, 3))}


def fci_batch_free(batch: FciBatch):
    if batch.handle:
        load().fci_batch_free(batch.handle)
        batch.handle = None
