"""Host-side pieces of bench.py: the time-to-tolerance reading of a Davidson
log, the workload strings shared by both arms, and the guard that reports ncu
DRAM traffic only for the kernel source it was measured on."""
import os

import numpy as np

import bench


def test_time_to_tol_needs_every_root_at_an_exact_point():
    log = np.array([
        [1, 1, 0.1, -1.0, -0.5],          # FP32 point: never counts
        [2, 0, 0.2, -1.0, -0.5 + 2e-8],   # root 1 not yet within 1e-8
        [3, 0, 0.3, -1.0 + 5e-9, -0.5],   # all roots within 1e-8
    ])
    assert bench.time_to_tol(log, [-1.0, -0.5]) == 0.3
    assert bench.time_to_tol(log[:2], [-1.0, -0.5]) is None
    assert bench.time_to_tol(log, -1.0) == 0.2  # one root


def test_both_arms_describe_the_same_workload():
    for w in bench.WORKLOADS:
        assert bench.workload_desc(w) == bench.workload_desc(w)
        assert ("FP32" in bench.metric_name(w)) == (w in bench.LARGE)
    assert "11778624 determinants (3432x3432)" in bench.workload_desc("cas14")
    assert "2363904400 determinants (48620x48620)" in bench.workload_desc("cas18")


def test_kernel_digest_tracks_the_kernel_source(tmp_path, monkeypatch):
    src = "void other() {\n}\n__global__ void k_x(int a) {\n  a += 1;\n}\nvoid tail() {\n}\n"
    (tmp_path / "k.cu").write_text(src)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    d0 = bench.kernel_digest("k.cu", "k_x(")
    (tmp_path / "k.cu").write_text(src.replace("void tail() {\n}\n", "void tail() { int q; }\n"))
    assert bench.kernel_digest("k.cu", "k_x(") == d0  # other code changed: same digest
    (tmp_path / "k.cu").write_text(src.replace("a += 1", "a += 2"))
    assert bench.kernel_digest("k.cu", "k_x(") != d0  # the kernel changed
    monkeypatch.setattr(bench, "NCU_TRAFFIC", {"k_x": ("k.cu", "k_x(", d0, 123.0)})
    assert bench.ncu_traffic("k_x", "cas14") is None
    monkeypatch.setattr(bench, "NCU_TRAFFIC", {"k_x": ("k.cu", "k_x(", bench.kernel_digest("k.cu", "k_x("), 123.0)})
    assert bench.ncu_traffic("k_x", "cas14") == 123.0
    assert bench.ncu_traffic("k_x", "cas12") is None  # measured on CAS(14,14) only


def test_committed_traffic_entries_name_existing_kernels():
    for name, (path, marker, digest, nbytes) in bench.NCU_TRAFFIC.items():
        assert os.path.exists(os.path.join(bench.ROOT, path)), name
        assert len(digest) == 16 and nbytes > 0


def test_every_profiled_kernel_of_the_default_pipelines_has_a_roofline():
    """The profile slot names that fci_sigma's FP64 and FP32 pipelines record (the
    names are string literals in the library's sources) all have an algorithmic
    work entry, so the bench's roofline table covers each of them; the launch
    counts per FP64 pipeline are at least one per slot."""
    import re

    peaks = {"bf16_tflops": 1937.6, "hbm_gbs": 6779.0}
    src = ""
    for f in ("sigma.cu", "sigma_wide.cu", "sigma3_sliced.cu"):
        src += open(os.path.join(bench.ROOT, "paper_1707_04346_gb300", "csrc", f)).read()
    names = set(re.findall(r'"(sigma[0-9a-z_]+|slice_c|transpose_slice|convert)"', src))
    assert {"sigma1_ss", "sigma2_ss", "sigma3_sliced", "sigma3_wide", "slice_c"} <= names
    uncovered = {"sigma1_sym"}  # the parity transpose-add: a copy, no algorithmic work entry
    for n in sorted(names - uncovered):
        w = bench.kernel_work(n, 14, 7, 7, 3432 * 3432, 56, 56, 3432, 3432, peaks)
        assert w is not None, n
        bound, amount, unit, peak, _, _ = w
        assert bound in ("tensor", "hbm", "alu") and amount > 0 and peak > 0, n
    for slots, launches in bench.LAUNCHES_PER_SIGMA.items():
        assert launches >= len(slots)
