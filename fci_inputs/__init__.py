"""Seeded synthetic inputs for determinant CI: integrals and trial vectors.

This module is shared by the CPU oracle, the tests and the benchmark.  It holds
only the random-number generator and the recipe that turns random numbers into
integrals and vectors; none of the CI arithmetic (strings, Hamiltonian, sigma)
lives here.

Random numbers come from a counter-based SplitMix64 (Steele, Lea & Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014): the i-th 64-bit
word of a stream is ``mix64(key + (i + 1) * GAMMA)``.  Uniforms take the top 53
bits; normals use the Box-Muller transform (Box & Muller 1958) on two
consecutive uniforms.  Every value therefore depends only on (seed, stream,
index), so any element can be regenerated on its own.

Integral recipe (the stand-in for molecular integrals, which the paper's
workloads use but which are not available here):

* one-electron ``h``: ``g_ij ~ N(0,1)`` for ``i <= j``, mirrored;
  ``A_ij = g_ij * exp(-|i-j|/3)``; orbital energies ``eps_i ~ U(-2, 1)``,
  sorted ascending; ``h = A + diag(eps)``.
* two-electron ``(ij|kl) = sum_P L^P_ij L^P_kl`` with
  ``L^P_ij ~ N(0, 0.3^2) / (1 + P)`` for ``i <= j`` (mirrored), ``P < rank``.
  This is 8-fold symmetric and positive semidefinite as a pair matrix.
* trial vector ``c``: i.i.d. ``N(0,1)``, normalised in FP64; or the uniform
  vector ``1/sqrt(N)`` that the paper uses for its single-iteration timings
  (Section 5); or, for spaces too large for host memory, the unnormalised
  ``c_J = 2 u_J - 1`` that both sides regenerate per index.
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_STREAM_MUL = np.uint64(0xD1B54A32D192ED03)

# stream ids (arbitrary, fixed)
STREAM_H = 1
STREAM_EPS = 2
STREAM_L = 3
STREAM_C = 4
STREAM_SIZES = 5
STREAM_C_PM1 = 6  # trial vectors too large for the host: c_J = 2 u_J - 1, regenerated per index

DEFAULT_INTEGRAL_SEED = 1707
DEFAULT_VECTOR_SEED = 4346


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def stream_key(seed: int, stream: int) -> np.uint64:
    s = _mix64(np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))
    s ^= np.array([stream], dtype=np.uint64) * _STREAM_MUL
    return _mix64(s)[0]


def u64(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """64-bit words ``start .. start+count-1`` of stream (seed, stream)."""
    key = stream_key(seed, stream)
    idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    return _mix64(key + idx * GAMMA)


def uniforms(seed: int, stream: int, count: int, start: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of each word."""
    w = u64(seed, stream, start, count)
    return (w >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normals(seed: int, stream: int, count: int, start: int = 0) -> np.ndarray:
    """Standard normals; normal ``i`` uses uniforms ``2i`` and ``2i+1``."""
    u = uniforms(seed, stream, 2 * count, start=2 * start)
    u1 = u[0::2]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log1p(-u1))
    return r * np.cos(2.0 * math.pi * u2)


def _sym_from_upper(vals: np.ndarray, n: int) -> np.ndarray:
    """Fill an n x n symmetric matrix from values listed for i <= j (row-major)."""
    m = np.zeros((n, n))
    iu = np.triu_indices(n)
    m[iu] = vals
    m = m + m.T - np.diag(np.diag(m))
    return m


def make_h1(norb: int, seed: int = DEFAULT_INTEGRAL_SEED) -> np.ndarray:
    npair = norb * (norb + 1) // 2
    g = _sym_from_upper(normals(seed, STREAM_H, npair), norb)
    i = np.arange(norb)
    decay = np.exp(-np.abs(i[:, None] - i[None, :]) / 3.0)
    eps = np.sort(-2.0 + 3.0 * uniforms(seed, STREAM_EPS, norb))
    return g * decay + np.diag(eps)


def make_cholesky_factors(norb: int, rank: int, seed: int = DEFAULT_INTEGRAL_SEED) -> np.ndarray:
    """L[P, i, j], symmetric in (i, j)."""
    npair = norb * (norb + 1) // 2
    raw = normals(seed, STREAM_L, rank * npair).reshape(rank, npair) * 0.3
    raw /= (1.0 + np.arange(rank))[:, None]
    L = np.zeros((rank, norb, norb))
    for p in range(rank):
        L[p] = _sym_from_upper(raw[p], norb)
    return L


def make_eri(norb: int, rank: int, seed: int = DEFAULT_INTEGRAL_SEED) -> np.ndarray:
    """Chemist-notation (ij|kl) as a dense [n, n, n, n] array."""
    L = make_cholesky_factors(norb, rank, seed)
    flat = L.reshape(rank, norb * norb)
    return (flat.T @ flat).reshape(norb, norb, norb, norb)


def make_integrals(norb: int, rank: int, seed: int = DEFAULT_INTEGRAL_SEED):
    return make_h1(norb, seed), make_eri(norb, rank, seed)


def make_vector(ndet: int, seed: int = DEFAULT_VECTOR_SEED, kind: str = "random") -> np.ndarray:
    """Normalised trial vector of length ``ndet`` (FP64)."""
    if kind == "uniform":
        return np.full(ndet, 1.0 / math.sqrt(ndet)) if ndet else np.zeros(0)
    c = normals(seed, STREAM_C, ndet)
    nrm = np.linalg.norm(c)
    return c / nrm if nrm > 0 else c


def vector_pm1(start: int, count: int, seed: int = DEFAULT_VECTOR_SEED) -> np.ndarray:
    """Elements ``start .. start+count-1`` of the unnormalised trial vector
    ``c_J = 2 u_J - 1`` (u from stream STREAM_C_PM1).  Integer mixing and an
    exact conversion only, so a device implementation of the same definition
    (``fci_inputs.gpu``) produces the same bits; used for spaces whose
    vectors do not fit in host memory (CAS(18,18): 2.36e9 elements)."""
    return 2.0 * uniforms(seed, STREAM_C_PM1, count, start=start) - 1.0


def batched_sizes(ninst: int, seed: int = DEFAULT_INTEGRAL_SEED, choices=(6, 8, 10, 12)) -> list[int]:
    """Active-space sizes drawn uniformly from ``choices`` (even n, Ms=0 at half filling)."""
    u = uniforms(seed, STREAM_SIZES, ninst)
    return [int(choices[min(int(x * len(choices)), len(choices) - 1)]) for x in u]


# Named workloads: (norb, nalpha, nbeta, rank)
WORKLOADS = {
    "cas8": (8, 4, 4, 40),
    "cas14": (14, 7, 7, 100),
    "cas16": (16, 8, 8, 100),
    "cas18": (18, 9, 9, 100),
}
