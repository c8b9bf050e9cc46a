"""The seeded input generators (fci_inputs): the counter-based SplitMix64
against its published definition, and the structure of the integral recipe.

SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) started from state 0 emits
0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, ...: the k-th word
is mix64(k * GAMMA).  The stream words here are mix64(key + (i + 1) * GAMMA), so
with key = 0 they must be exactly that sequence.
"""
import numpy as np

import fci_inputs as fi


def test_splitmix64_published_sequence():
    k = np.arange(1, 4, dtype=np.uint64)
    got = fi._mix64(k * fi.GAMMA)
    assert [int(x) for x in got] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_words_depend_only_on_their_index():
    a = fi.u64(1707, 3, 0, 40)
    b = fi.u64(1707, 3, 17, 10)
    assert np.array_equal(a[17:27], b)
    assert not np.array_equal(fi.u64(1707, 3, 0, 40), fi.u64(1707, 4, 0, 40))
    assert not np.array_equal(fi.u64(1707, 3, 0, 40), fi.u64(1708, 3, 0, 40))


def test_uniforms_and_normals():
    u = fi.uniforms(11, 2, 200000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert np.all(u * 2.0**53 == np.floor(u * 2.0**53))  # 53-bit grid
    assert abs(u.mean() - 0.5) < 4 * np.sqrt(1 / 12 / u.size)
    z = fi.normals(11, 2, 200000)
    assert abs(z.mean()) < 4 / np.sqrt(z.size)
    assert abs(z.var() - 1) < 4 * np.sqrt(2 / z.size)
    assert np.array_equal(fi.normals(11, 2, 10, start=5), z[5:15])  # counter access


def test_pm1_vector_range_and_slices():
    v = fi.vector_pm1(0, 1000)
    assert v.min() >= -1.0 and v.max() < 1.0
    assert np.array_equal(fi.vector_pm1(300, 50), v[300:350])


def test_one_electron_integrals():
    for n in (4, 8, 14):
        h = fi.make_h1(n)
        assert h.shape == (n, n) and np.array_equal(h, h.T)
        # far from the diagonal the couplings decay as exp(-|i-j|/3)
        assert np.abs(h[0, n - 1]) < 6 * np.exp(-(n - 1) / 3.0) + 1e-300


def test_two_electron_integrals_symmetry_rank_psd():
    for n, rank in ((4, 3), (6, 40), (8, 40), (8, 10)):
        g = fi.make_eri(n, rank)
        for perm in ((1, 0, 2, 3), (0, 1, 3, 2), (2, 3, 0, 1)):
            # 8-fold symmetry up to the rounding of the BLAS product (its summation
            # order may differ between mirrored elements)
            assert np.abs(g - g.transpose(perm)).max() <= 1e-15 * np.abs(g).max()
        iu = np.triu_indices(n)
        npair = len(iu[0])
        G = g[iu[0], iu[1]][:, iu[0], iu[1]]  # pair matrix (ij|kl), i <= j, k <= l
        w = np.linalg.eigvalsh(G)
        assert w.min() > -1e-12 * w.max()  # positive semidefinite
        assert np.linalg.matrix_rank(G, tol=1e-10 * w.max()) == min(rank, npair)


def test_batched_sizes_of_the_benchmark():
    s = fi.batched_sizes(64)
    assert set(s) <= {6, 8, 10, 12}
    assert s == fi.batched_sizes(64)
    assert {n: s.count(n) for n in (6, 8, 10, 12)} == {6: 20, 8: 14, 10: 13, 12: 17}


def test_trial_vectors():
    c = fi.make_vector(1000)
    assert abs(np.linalg.norm(c) - 1) < 1e-14
    u = fi.make_vector(16, kind="uniform")
    assert np.allclose(u, 0.25)
    assert fi.make_vector(0).size == 0


def test_device_fill_library_builds_for_sm103a_and_exports_its_entry_point():
    """The device fill (same generator, used for vectors too large for the host)
    cross-compiles here and exports its C entry point; running it needs a GPU
    (tests/test_gpu_cas18.py checks it bit-exactly against vector_pm1)."""
    import ctypes

    from fci_inputs import gpu

    lib = ctypes.CDLL(gpu.build())
    assert hasattr(lib, "fci_inputs_fill_pm1")
