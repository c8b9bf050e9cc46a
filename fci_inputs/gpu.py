"""Device fill of the input module's trial vector ``c_J = 2 u_J - 1`` (see
``fci_inputs.vector_pm1``), for spaces whose vectors do not fit in host memory.

The CUDA source (``csrc/fill.cu``) holds the same counter-based generator and
nothing else; :func:`build` compiles it with nvcc into ``_build/libfill.so``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

from . import DEFAULT_VECTOR_SEED, STREAM_C_PM1

_DIR = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_DIR, "csrc", "fill.cu")
_BUILD = os.path.join(_DIR, "_build")
_SO = os.path.join(_BUILD, "libfill.so")
_lib = None


def build(force: bool = False) -> str:
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-Xcompiler", "-fPIC",
                        "-shared", _SRC, "-o", tmp], check=True)
        os.replace(tmp, _SO)
    return _SO


def fill_pm1(x, start: int = 0, seed: int = DEFAULT_VECTOR_SEED, stream=None) -> None:
    """x[i] = c_{start+i} for a contiguous CUDA tensor x (float32 or float64)."""
    global _lib
    import torch

    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.fci_inputs_fill_pm1.restype = ctypes.c_int
        _lib.fci_inputs_fill_pm1.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                             ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p]
    if not (x.is_cuda and x.is_contiguous() and x.dtype in (torch.float32, torch.float64)):
        raise ValueError("x must be a contiguous CUDA float32/float64 tensor")
    st = (stream or torch.cuda.current_stream(x.device)).cuda_stream
    rc = _lib.fci_inputs_fill_pm1(ctypes.c_void_p(x.data_ptr()), start, x.numel(), int(x.dtype == torch.float32),
                                  seed & 0xFFFFFFFFFFFFFFFF, STREAM_C_PM1, ctypes.c_void_p(st))
    if rc:
        raise RuntimeError(f"fill kernel failed (CUDA error {rc})")
