"""FP64 CPU oracle for determinant CI (arXiv 1707.04346, Sections 2.1 and 3.3).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The library under
``paper_1707_04346_gb300`` never imports it, and this package never imports the
library: the two share no code.  Inputs come from ``fci_inputs`` (random
numbers and the integral recipe only).

What lives here:

* ``oracle/csrc/oracle.c`` -- plain C, FP64: string lists, the E_kl
  single-replacement lists (Eq. 7), the Hamiltonian of Eq. 6 built two
  independent ways (Slater-Condon rules, and Eq. 6 applied term by term to
  bitstrings), direct sigma = H c (Eq. 4/5), H diagonal, the spin-summed
  one- and two-particle densities and the total spin <S^2> of an expansion.
* ``oracle.davidson`` -- a plain NumPy Davidson eigensolver following the
  steps of Section 3.3 (reading of the unspecified parts in its docstring).

Every function is pinned by ``tests/test_oracle_*.py`` against closed forms,
brute force, invariants and the determinant counts the paper prints.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csrc", "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (-O2 -fopenmp) into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def _bind(lib):
    """Declare the argument and result types of the oracle's C entry points."""
    i64, i32, dp = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
    u64 = ctypes.c_uint64
    lib.oracle_binom.restype = i64
    lib.oracle_binom.argtypes = [i32, i32]
    lib.oracle_strings.restype = i64
    lib.oracle_strings.argtypes = [i32, i32, dp]
    lib.oracle_single_table.restype = i32
    lib.oracle_single_table.argtypes = [i32, i32, dp, dp, dp, dp]
    for name in ("oracle_h_slater", "oracle_h_operator"):
        f = getattr(lib, name)
        f.restype = i32
        f.argtypes = [i32, i32, i32, dp, dp, dp]
    lib.oracle_sigma.restype = i32
    lib.oracle_sigma.argtypes = [i32, i32, i32, dp, dp, dp, dp]
    lib.oracle_sigma_rows.restype = i32
    lib.oracle_sigma_rows.argtypes = [i32, i32, i32, dp, dp, dp, dp, i64, dp]
    lib.oracle_sigma_rows_gen.restype = i32
    lib.oracle_sigma_rows_gen.argtypes = [i32, i32, i32, dp, dp, u64, u64, dp, i64, dp]
    lib.oracle_hdiag.restype = i32
    lib.oracle_hdiag.argtypes = [i32, i32, i32, dp, dp, dp]
    lib.oracle_rdm1.restype = i32
    lib.oracle_rdm1.argtypes = [i32, i32, i32, dp, dp]
    lib.oracle_rdm2.restype = i32
    lib.oracle_rdm2.argtypes = [i32, i32, i32, dp, dp]
    lib.oracle_s2.restype = ctypes.c_double
    lib.oracle_s2.argtypes = [i32, i32, i32, dp]
    lib.oracle_num_threads.restype = i32
    lib.oracle_num_threads.argtypes = []
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _bind(ctypes.CDLL(_SO))
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def binom(n: int, k: int) -> int:
    return int(_load().oracle_binom(n, k))


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def strings(norb: int, ne: int) -> np.ndarray:
    """All ne-electron strings of norb orbitals as uint32 bitmasks, ascending (Eq. 2)."""
    lib = _load()
    ns = lib.oracle_strings(norb, ne, None)
    out = np.zeros(max(ns, 0), dtype=np.uint32)
    lib.oracle_strings(norb, ne, _ptr(out))
    return out


def single_table(norb: int, ne: int):
    """Single-replacement lists (Eq. 7).

    Returns (target, k, l, sign), each shaped [Ns, ne*(norb-ne)+ne]: for
    string X and each (k, l) with l occupied and k empty or k == l (l
    ascending, then k ascending), ``a+_k a_l |X> = sign |target>``.
    """
    ns = binom(norb, ne)
    per = ne * (norb - ne) + ne
    tgt = np.zeros((ns, per), dtype=np.int32)
    kk = np.zeros((ns, per), dtype=np.int8)
    ll = np.zeros((ns, per), dtype=np.int8)
    sg = np.zeros((ns, per), dtype=np.int8)
    _load().oracle_single_table(norb, ne, _ptr(tgt), _ptr(kk), _ptr(ll), _ptr(sg))
    return tgt, kk, ll, sg


def ndet(norb: int, na: int, nb: int) -> int:
    return binom(norb, na) * binom(norb, nb)


def hamiltonian(norb: int, na: int, nb: int, h1, eri, method: str = "slater") -> np.ndarray:
    """Explicit H in the determinant basis (tiny spaces only).

    method="slater": Slater-Condon rules; method="operator": Eq. 6 applied
    term by term to every basis determinant.
    """
    n = ndet(norb, na, nb)
    H = np.zeros((n, n))
    f = _load().oracle_h_slater if method == "slater" else _load().oracle_h_operator
    h1 = _f64(h1)
    eri = _f64(eri)
    rc = f(norb, na, nb, _ptr(h1), _ptr(eri), _ptr(H))
    if rc:
        raise ValueError("bad space")
    return H


def sigma(norb: int, na: int, nb: int, h1, eri, c) -> np.ndarray:
    """sigma = H c by the direct (determinant-driven) Slater-Condon sum."""
    h1, eri, c = _f64(h1), _f64(eri), _f64(c)
    out = np.zeros(ndet(norb, na, nb))
    rc = _load().oracle_sigma(norb, na, nb, _ptr(h1), _ptr(eri), _ptr(c), _ptr(out))
    if rc:
        raise ValueError("bad space")
    return out


def sigma_rows(norb: int, na: int, nb: int, h1, eri, c, rows) -> np.ndarray:
    """sigma(I) for the given determinant indices I only."""
    h1, eri, c = _f64(h1), _f64(eri), _f64(c)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    out = np.zeros(len(rows))
    rc = _load().oracle_sigma_rows(norb, na, nb, _ptr(h1), _ptr(eri), _ptr(c), _ptr(rows), len(rows), _ptr(out))
    if rc:
        raise ValueError("bad space")
    return out


def sigma_rows_generated(norb: int, na: int, nb: int, h1, eri, rows, seed: int, stream: int) -> np.ndarray:
    """sigma(I) for chosen I with c_J = 2 u_J - 1 from the counter-based
    generator (seed, stream), evaluated per index (no full vector)."""
    h1, eri = _f64(h1), _f64(eri)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    out = np.zeros(len(rows))
    rc = _load().oracle_sigma_rows_gen(norb, na, nb, _ptr(h1), _ptr(eri), ctypes.c_uint64(seed),
                                       ctypes.c_uint64(stream), _ptr(rows), len(rows), _ptr(out))
    if rc:
        raise ValueError("bad space")
    return out


def hdiag(norb: int, na: int, nb: int, h1, eri) -> np.ndarray:
    h1, eri = _f64(h1), _f64(eri)
    out = np.zeros(ndet(norb, na, nb))
    _load().oracle_hdiag(norb, na, nb, _ptr(h1), _ptr(eri), _ptr(out))
    return out


def rdm1(norb: int, na: int, nb: int, c) -> np.ndarray:
    """gamma_pq = <c| E_pq |c> (spin summed, Eq. 7 operator)."""
    c = _f64(c)
    g = np.zeros((norb, norb))
    _load().oracle_rdm1(norb, na, nb, _ptr(c), _ptr(g))
    return g


def rdm2(norb: int, na: int, nb: int, c) -> np.ndarray:
    """Gamma_pqrs = <c| E_pq E_rs |c> (spin summed), shaped [norb]*4.

    With gamma = rdm1(c), <c|H|c> = sum h_pq gamma_pq
    + 1/2 sum (pq|rs) (Gamma_pqrs - delta_qr gamma_ps) (Eq. 6)."""
    c = _f64(c)
    if c.size != ndet(norb, na, nb):
        raise ValueError("vector length does not match the space")
    g = np.zeros((norb,) * 4)
    if _load().oracle_rdm2(norb, na, nb, _ptr(c), _ptr(g)):
        raise ValueError("bad space")
    return g


def s_squared(norb: int, na: int, nb: int, c) -> float:
    """<c|S^2|c> / <c|c>: total spin of an expansion in the (na, nb) sector
    (a diagnostic for the roots; Ms = 0 roots of random integrals can have any S)."""
    c = _f64(c)
    if c.size != ndet(norb, na, nb):
        raise ValueError("vector length does not match the space")
    v = float(_load().oracle_s2(norb, na, nb, _ptr(c)))
    if v != v:
        raise ValueError("bad space or zero vector")
    return v


from .davidson import davidson  # noqa: E402  (pure NumPy, no library import)

__all__ = [
    "build", "binom", "strings", "single_table", "ndet", "hamiltonian", "sigma",
    "sigma_rows", "sigma_rows_generated", "hdiag", "rdm1", "rdm2", "s_squared", "davidson", "num_threads",
]
