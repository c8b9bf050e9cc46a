"""Benchmark: sigma = H c throughput (determinants/s) on CAS(14e,14o), Ms=0.

One step = one full sigma build (sigma_1 + sigma_2 + sigma_3 of Eq. 8) over
the 11,778,624-determinant CI vector, with the tables and integrals resident
on the device.  The reported value is whole-job throughput in Gdet/s.

Timing: W untimed warm-up steps, then K steps bracketed by a barrier and
cuda synchronize, timed with CUDA events on the launching stream, max over
ranks.  The inputs rotate through a ring of vectors whose total size exceeds
the 129 MB L2, so no step reads its input from L2.

Extra keys: per-kernel roofline of the dominant kernel, the oracle on the host
cores (cpu_baseline), end-to-end throughput with host buffers (e2e), the FP32
sigma rate, and Davidson time-to-1e-8 Eh (FP64 and mixed).

``--impl reference`` times the CPU oracle instead (the only reference this
work has: a plain FP64 CPU implementation written from the paper).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import fci_inputs as fi  # noqa: E402

WORKLOADS = {"cas14": (14, 7, 7, 100), "cas16": (16, 8, 8, 100), "cas12": (12, 6, 6, 100), "cas8": (8, 4, 4, 40),
             "cas18": (18, 9, 9, 100)}
LARGE = {"cas18"}  # vectors too large for the host: trial vector regenerated on the device
F64_KERNELS = {"auto": 0, "fma": 1, "sliced": 2, "wide": 3}  # fci_options.f64_kernels of the main context
FP64_NOMINAL_TFLOPS = 1.25  # GB300 FP64 (vector and tensor), nominal
GB300_SMS = 152
FP32_LANES_PER_SM = 128  # FP32 operations issued per SM per clock

# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one
# ncu capture of the CAS(14e,14o) workload (the summaries under profiles/ give the
# command), keyed to a digest of the kernel's source at capture time: reported
# only while that source is unchanged.
NCU_TRAFFIC = {
    "sigma3_exact": ("paper_1707_04346_gb300/csrc/sigma.cu", "k_sigma3_exact(", "d3fba1cadf6cd31c", 610262016.0),
    "sigma3_tc": ("paper_1707_04346_gb300/csrc/sigma_tc_kernel.cuh", "k_sigma3_tc(", "878aabf229629b81", 124323328.0),
    "sigma3_sliced": ("paper_1707_04346_gb300/csrc/sigma3_sliced_kernel.cuh", "k_sigma3_sliced(", "2f62dcb8acf96f61",
                      978847232.0),
    # sigma_1 as a dense sliced product (k_ss_tc; sigma_2 runs the same kernel with the operands swapped)
    "sigma1_ss": ("paper_1707_04346_gb300/csrc/sigma_ss.cu", "k_ss_tc(", "9c370e9bb4171175", 2206744880.0),
    # the wide kernels at CAS(14,14) (bench.py --f64-kernels wide)
    "sigma3_wide": ("paper_1707_04346_gb300/csrc/sigma_wide_kernel.cuh", "k_sigma_wide(", "3b63c3cbe309e741", 1016815808.0),
    "sigma1_wide": ("paper_1707_04346_gb300/csrc/sigma_wide_kernel.cuh", "k_sigma_wide(", "3b63c3cbe309e741", 2433141328.0),
    "sigma2_wide": ("paper_1707_04346_gb300/csrc/sigma_wide_kernel.cuh", "k_sigma_wide(", "3b63c3cbe309e741", 2452579616.0),
}


# The 2-RDM's Gram kernel, captured on CAS(12e,12o) (the CAS(14,14) launch holds 28 GB of digit
# planes, above the capture size rule): DRAM bytes per byte of digit planes read once, scaled to
# the workload's planes while the kernel's source is unchanged.
RDM2_TC_TRAFFIC = ("paper_1707_04346_gb300/csrc/rdm2.cu", "k_rdm2_tc(", "dbb9c2a6acd29160",
                   (2413767000.0 + 3238656.0) / (53361 * 6 * 152 * 32))


# Kernels one sigma call launches, by its profiled slots (the slots group kernels: "slice_c"
# is the row-exponent and slicing pair, each dense same-spin product its exponent or plane
# pass, the product and, once per call, the FP64 diagonal), counted from the ncu launch
# lists under profiles/.  Pipelines not listed launch one kernel per slot.
LAUNCHES_PER_SIGMA = {
    ("slice_c", "sigma3_sliced", "sigma1_ss", "sigma2_ss"): 9,
    ("slice_c", "sigma3_sliced", "sigma1_rows", "sigma2_cols"): 5,
}


def kernel_digest(path: str, marker: str) -> str:
    """sha256 (16 hex digits) of a kernel's source, from its name to its closing brace."""
    with open(os.path.join(ROOT, path)) as f:
        src = f.read()
    i = src.index(marker)
    return hashlib.sha256(src[i:src.index("\n}\n", i)].encode()).hexdigest()[:16]


def ncu_traffic(kernel: str, workload: str):
    if workload != "cas14" or kernel not in NCU_TRAFFIC:
        return None
    path, marker, digest, nbytes = NCU_TRAFFIC[kernel]
    try:
        return nbytes if kernel_digest(path, marker) == digest else None
    except (OSError, ValueError):
        return None


def metric_name(workload: str) -> str:
    return "sigma=Hc throughput (FP32)" if workload in LARGE else "sigma=Hc throughput (FP64)"


def workload_desc(workload: str) -> str:
    """The workload string of the JSON line, the same for both arms."""
    norb, na, nb, rank_eri = WORKLOADS[workload]
    nsa, nsb = math.comb(norb, na), math.comb(norb, nb)
    if workload in LARGE:
        return (f"CAS({na + nb}e,{norb}o) Ms=0 FP32 sigma, {nsa * nsb} determinants ({nsa}x{nsb}), "
                f"Cholesky-factored integrals rank {rank_eri}, c_J = 2u_J - 1 generated per index")
    return (f"CAS({na + nb}e,{norb}o) Ms=0 sigma, {nsa * nsb} determinants ({nsa}x{nsb}), "
            f"Cholesky-factored integrals rank {rank_eri}, seeds 1707/4346")


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "_fallback": True}


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "100"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.samples.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


from paper_1707_04346_gb300 import replicas  # noqa: E402  (pure Python; no library load)


def dist_setup(n_gpus):
    return replicas.setup()


barrier = replicas.barrier
max_over_ranks = replicas.max_over_ranks


def cpu_baseline(norb, na, nb, h1, eri, c, target_s=15.0, seed=0):
    """The oracle as it stands, on a bounded random sample of sigma rows."""
    import oracle

    N = c.size
    rng = np.random.default_rng(seed)
    pilot = rng.integers(0, N, 256)
    t = time.perf_counter()
    oracle.sigma_rows(norb, na, nb, h1, eri, c, pilot)
    dt = max(time.perf_counter() - t, 1e-3)
    nrows = int(min(N, max(256, 256 * target_s / dt)))
    rows = rng.integers(0, N, nrows)
    t = time.perf_counter()
    oracle.sigma_rows(norb, na, nb, h1, eri, c, rows)
    dt = time.perf_counter() - t
    return {"value": nrows / dt / 1e9, "unit": "Gdet/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{nrows} random sigma rows of CAS({na + nb}e,{norb}o), direct Slater-Condon sum, FP64, "
                      f"{dt:.1f} s"}


def kernel_work(name, norb, na, nb, N, sa, sb, nsa, nsb, peaks, f32_splits=3):
    """(bound, amount per launch, unit, peak, peak source, description) of one
    sigma kernel: the algorithmic work each kernel's roofline is taken on."""
    nsame = 1 + na * (norb - na) + (na * (na - 1) // 2) * ((norb - na) * (norb - na - 1) // 2)
    npair = norb * (norb + 1) // 2
    kpad = -(-sa // 16) * 16
    npad = -(-npair // 16) * 16
    npad1 = -(-(npair + 1) // 16) * 16
    tiles = nsa * (-(-nsb // 128))
    fp32_pipe = FP32_LANES_PER_SM * GB300_SMS * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12  # Tops/s
    bf16 = (peaks["bf16_tflops"], "MEASURED_PEAKS.json bf16_tflops (burst; the kernel is timed in short bursts)")
    fp32src = "FP32 pipe: 128 lanes x 152 SMs x max SM clock"
    prods32 = f32_splits * (f32_splits + 1) // 2
    if name == "sigma3_exact":  # diagonal replacements merged
        f = 2.0 * (sb + (sa - na) * (sb - nb + 1))
        return ("alu", f * N, "TFLOP/s", FP64_NOMINAL_TFLOPS,
                "GB300 FP64 nominal 1.25 TFLOP/s (no FP64 entry in MEASURED_PEAKS.json)", f"FP64 FLOP, {f:.0f} per determinant")
    if name == "sigma3_sliced":
        return ("tensor", 21 * 2.0 * 128 * npad * kpad * tiles, "TFLOP/s", *bf16,
                f"bf16 MMA FLOP: 21 slice products x 2 x 128 x {npad} x {kpad} x {tiles} tiles")
    if name in ("sigma1_rows", "sigma2_cols"):  # FP64 path: double-float, 12 FP32 operations per term
        return ("alu", 12.0 * nsame * N, "Tops/s", fp32_pipe, fp32src,
                f"FP32 operations: 12 per term x {nsame} terms per determinant")
    if name in ("sigma1_ss", "sigma2_ss"):  # FP64 same-spin terms as dense sliced products
        # one GEMM of (strings of the summed spin) x (other spin) x (summed spin), 21 digit
        # products, tiles of 128 x 48 rows (the plane rows padded to 384) and the FP64 diagonal
        ns_sum = nsb if name == "sigma1_ss" else nsa
        mt, nt = -(-nsb // 128), -(-nsa // 48)  # output tiles: beta strings x alpha strings
        f = 21 * 2.0 * 128 * 48 * (-(-ns_sum // 16) * 16) * mt * nt
        return ("tensor", f, "TFLOP/s", *bf16,
                f"bf16 MMA FLOP: 21 digit products x 2 x 128 x 48 x {-(-ns_sum // 16) * 16} x {mt * nt} tiles")
    if name == "sigma12_f32":  # FP32 sigma_1 + sigma_2: one FMA per term
        return ("alu", 2.0 * nsame * N, "Tops/s", fp32_pipe, fp32src,
                f"FP32 FMAs: {nsame} terms per determinant, two spins")
    if name == "sigma3_tc":
        return ("tensor", prods32 * 2.0 * 128 * npad * kpad * tiles, "TFLOP/s", *bf16,
                f"bf16 MMA FLOP: {prods32} slice products x 2 x 128 x {npad} x {kpad} x {tiles} tiles")
    if name in ("sigma2_tc", "sigma1_tc"):  # same-spin terms through intermediate strings
        return ("tensor", prods32 * 2.0 * 128 * npad1 * kpad * tiles, "TFLOP/s", *bf16,
                f"bf16 MMA FLOP: {prods32} slice products x 2 x 128 x {npad1} x {kpad} x {tiles} tiles")
    if name in ("sigma3_wide", "sigma1_wide", "sigma2_wide"):  # wide FP64 kernels: 21 products per tile and part
        if name == "sigma3_wide":
            kp, npd, t = kpad, npad, tiles
        elif name == "sigma2_wide":
            kp, npd, t = kpad, npad1, tiles
        else:  # beta strings as rows, over C transposed
            kp, npd, t = -(-sb // 16) * 16, npad1, nsb * (-(-nsa // 128))
        return ("tensor", 21 * 2.0 * 128 * npd * kp * t, "TFLOP/s", *bf16,
                f"bf16 MMA FLOP: 21 slice products x 2 x 128 x {npd} x {kp} x {t} tiles")
    if name == "transpose_slice":  # C transposed (read 8, write 8) and sliced (read 8, write 12)
        return ("hbm", 36.0 * N, "GB/s", peaks["hbm_gbs"], "MEASURED_PEAKS.json hbm_gbs",
                "bytes: transpose of C (8 + 8 per determinant) and its digit slices (8 + 12)")
    if name == "convert":  # 64-bit integers in, FP64 out
        return ("hbm", 16.0 * N, "GB/s", peaks["hbm_gbs"], "MEASURED_PEAKS.json hbm_gbs",
                "bytes: 8 read and 8 written per determinant")
    if name == "slice_c":  # row exponents (one read of C) and the digit slices (a read, 12 bytes written)
        return ("hbm", 28.0 * N, "GB/s", peaks["hbm_gbs"], "MEASURED_PEAKS.json hbm_gbs",
                "bytes: two reads of C (8 + 8 per determinant) and 12 written")
    return None


def roofline_table(names, kmean, kshare, norb, na, nb, N, sa, sb, nsa, nsb, peaks, workload):
    """Roofline of every kernel of one sigma pipeline; the dominant one first."""
    def one(i):
        w = kernel_work(names[i], norb, na, nb, N, sa, sb, nsa, nsb, peaks)
        if w is None:
            return {"kernel": names[i], "ms": float(kmean[i] * 1e3)}
        bound, amount, unit, peak, src, what = w
        ach = amount / kmean[i] / (1e9 if unit == "GB/s" else 1e12)
        return {"kernel": names[i], "bound": bound, "achieved": ach, "peak": peak, "unit": unit, "frac": ach / peak,
                "traffic": ncu_traffic(names[i], workload), "peak_source": src,
                "work_per_launch": f"{amount:.4g} ({what})"}
    top = int(np.argmax(kmean))
    roof = one(top)
    roof["kernels"] = {n: {"ms": float(kmean[i] * 1e3), "share": float(kshare[i]),
                           **({"frac": one(i)["frac"], "unit": one(i)["unit"]} if "frac" in one(i) else {})}
                       for i, n in enumerate(names)}
    return roof


def sigma_leg(pkg, workload, steps, warmup, stream, world, cpu_seconds, dtypes=("f64", "f32")):
    """sigma = H c throughput of one more configuration (the device fills the
    trial vector c_J = 2 u_J - 1 from the input module's generator; one vector
    is larger than L2), per precision: Gdet/s, per-kernel times and rooflines,
    and the oracle on sampled rows of the same vector on the host cores."""
    import torch
    from fci_inputs import gpu as fgpu

    norb, na, nb, rank_eri = WORKLOADS[workload]
    h1, eri = fi.make_integrals(norb, rank_eri)
    t0 = time.perf_counter()
    ctx = pkg.fci_init(norb, na, nb, h1, eri)
    out = {"workload": workload_desc(workload).replace("seeds 1707/4346", "c_J = 2u_J - 1 generated per index"),
           "init_s": time.perf_counter() - t0}
    N = ctx.ndet
    nsa, nsb = ctx.nstr
    sa, sb = pkg.fci_query(ctx, 4), pkg.fci_query(ctx, 5)
    peaks = load_peaks()
    for dt in dtypes:
        tdt = torch.float64 if dt == "f64" else torch.float32
        c = torch.empty(N, dtype=tdt, device=stream.device)
        fgpu.fill_pm1(c)
        sgm = torch.empty_like(c)
        pkg.fci_profile_enable(ctx, True)
        t = time_sigma_ring(pkg, ctx, [c], [sgm], steps, warmup, stream, world)
        names, prof = pkg.fci_profile_read(ctx)
        pkg.fci_profile_enable(ctx, False)
        t = max_over_ranks(t, world)
        prof = prof[-steps:]
        kmean = prof.mean(axis=0) / 1e3
        kshare = prof.sum(axis=0) / prof.sum()
        out[dt] = {"value": world * N * steps / t / 1e9, "unit": "Gdet/s", "ms_per_step": t / steps * 1e3,
                   "steps": steps, "warmup": warmup,
                   "roofline": roofline_table(names, kmean, kshare, norb, na, nb, N, sa, sb, nsa, nsb, peaks, workload)}
        del c, sgm
    pkg.fci_free(ctx)
    if cpu_seconds > 0:
        import oracle

        rows = np.random.default_rng(7).integers(0, N, 16)
        oracle.sigma_rows_generated(norb, na, nb, h1, eri, rows[:2], fi.DEFAULT_VECTOR_SEED, fi.STREAM_C_PM1)
        t0, nrows = time.perf_counter(), 0
        while time.perf_counter() - t0 < cpu_seconds:
            oracle.sigma_rows_generated(norb, na, nb, h1, eri, rows, fi.DEFAULT_VECTOR_SEED, fi.STREAM_C_PM1)
            nrows += len(rows)
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": nrows / dt / 1e9, "unit": "Gdet/s", "cores": oracle.num_threads(),
                               "kind": "oracle", "sample": f"{nrows} sampled sigma rows of CAS({na + nb}e,{norb}o), "
                                                          f"direct Slater-Condon sum, FP64, {dt:.1f} s"}
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    norb, na, nb, rank_eri = WORKLOADS[args.workload]
    h1, eri = fi.make_integrals(norb, rank_eri)
    import oracle

    N = oracle.ndet(norb, na, nb)
    rng = np.random.default_rng(1)
    if args.workload in LARGE:  # the vector is regenerated per index (no 19 GB host copy)
        rows_per_step = 64

        def rows_sigma(rows):
            return oracle.sigma_rows_generated(norb, na, nb, h1, eri, rows, fi.DEFAULT_VECTOR_SEED, fi.STREAM_C_PM1)
    else:
        rows_per_step = 2000
        c = fi.make_vector(N)

        def rows_sigma(rows):
            return oracle.sigma_rows(norb, na, nb, h1, eri, c, rows)
    for _ in range(args.warmup):
        rows_sigma(rng.integers(0, N, 8))
    t = time.perf_counter()
    for _ in range(args.steps):
        rows_sigma(rng.integers(0, N, rows_per_step))
    dt = time.perf_counter() - t
    value = rows_per_step * args.steps / dt / 1e9
    out = {"impl": "reference", "metric": metric_name(args.workload), "value": value, "unit": "Gdet/s",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": workload_desc(args.workload),
                      "step": f"{rows_per_step} sigma rows per step (bounded sample, FP64 oracle)",
                      "device": "host cores of rank 0 (the oracle uses no GPU)"},
           "cpu_baseline": {"value": value, "unit": "Gdet/s", "cores": oracle.num_threads(), "kind": "oracle",
                            "sample": f"{rows_per_step} random rows per step, {args.steps} steps"},
           "e2e": {"value": value, "unit": "Gdet/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def time_sigma_ring(pkg, ctx, vecs, outs, steps, warmup, stream, world):
    import torch

    for i in range(warmup):
        pkg.fci_sigma(ctx, vecs[i % len(vecs)], outs[i % len(outs)], stream=stream)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(steps):
        pkg.fci_sigma(ctx, vecs[i % len(vecs)], outs[i % len(outs)], stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    return e0.elapsed_time(e1) / 1e3


def time_to_tol(log, e_ref, tol=1e-8):
    """Elapsed seconds at the first iteration whose energies are exact (every
    sigma in the subspace FP64, log flag 0) and all within tol of e_ref."""
    e_ref = np.atleast_1d(e_ref)
    for row in log:
        if row[1] == 0 and np.all(np.abs(row[3:3 + len(e_ref)] - e_ref) <= tol):
            return float(row[2])
    return None


def run_batched(pkg, ninst, nroots=2, tol=1e-8):
    """Batched CASCI: ninst instances, active spaces drawn uniformly from
    CAS(6,6)..CAS(12,12) (even, Ms=0), own seeded integrals (rank min(40, npair)),
    nroots roots each.  Times one batched solve (mixed and FP64) against the
    same instances solved one after another with the single-instance FP64
    path; all to the same convergence threshold."""
    import torch

    sizes = fi.batched_sizes(ninst)
    insts = []
    for i, n in enumerate(sizes):
        h1, eri = fi.make_integrals(n, min(40, n * (n + 1) // 2), seed=1707 + i)
        insts.append((n, n // 2, n // 2, h1, eri))
    out = {"instances": ninst, "roots": nroots, "tol": tol,
           "sizes": {str(n): sizes.count(n) for n in sorted(set(sizes))}}
    # sequential single-instance FP64 solves
    ctxs = [pkg.fci_init(*x) for x in insts]
    torch.cuda.synchronize()
    t = time.perf_counter()
    e_seq, noconv = [], 0
    for c in ctxs:
        try:
            e_seq.append(pkg.fci_davidson(c, nroots, tol))
        except pkg.FciError:
            noconv += 1
            e_seq.append(np.full(nroots, np.nan))
    e_seq = np.array(e_seq)
    torch.cuda.synchronize()
    out["sequential_fp64_s"] = time.perf_counter() - t
    out["sequential_fp64_not_converged"] = noconv
    for c in ctxs:
        pkg.fci_free(c)
    for name, prec in (("batched_mixed", pkg.FCI_PREC_MIXED), ("batched_fp64", pkg.FCI_PREC_FP64)):
        t0 = time.perf_counter()
        b = pkg.fci_batch_init(insts, pkg.default_options(precision=prec))
        t_init = time.perf_counter() - t0
        torch.cuda.synchronize()
        t = time.perf_counter()
        try:
            e = pkg.fci_batch_davidson(b, nroots, tol)
            out[name + "_converged"] = True
        except pkg.FciError:
            e = np.full((ninst, nroots), np.nan)
            out[name + "_converged"] = False
        torch.cuda.synchronize()
        out[name + "_s"] = time.perf_counter() - t
        out[name + "_init_s"] = t_init
        out[name + "_max_abs_dE_vs_sequential"] = float(np.nanmax(np.abs(e - e_seq)))
        out[name + "_stats"] = pkg.fci_batch_stats(b)
        if prec == pkg.FCI_PREC_MIXED:
            out["tuning"] = [{"norb": n, "dtype": "f64" if d == 0 else "f32", "threads_per_row": tpr}
                             for n, d, tpr in pkg.fci_batch_tuning(b)]
            out["determinants_total"] = int(b.offset(b.ninst))
        pkg.fci_batch_free(b)
    out["speedup_mixed_vs_sequential"] = out["sequential_fp64_s"] / out["batched_mixed_s"]
    return out


def run_large(args):
    """FP32 sigma of a space whose vectors do not fit in host memory
    (CAS(18e,18o): 2.36e9 determinants, 9.4 GB per FP32 vector): the trial
    vector c_J = 2 u_J - 1 is generated on the device from the input module's
    counter-based generator; the CPU baseline is the oracle's direct sum on
    sampled rows with c_J regenerated per index."""
    import torch

    rank, world, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_1707_04346_gb300 as pkg
    from fci_inputs import gpu as fgpu

    norb, na, nb, rank_eri = WORKLOADS[args.workload]
    h1, eri = fi.make_integrals(norb, rank_eri)
    ctx = pkg.fci_init(norb, na, nb, h1, eri)
    N = ctx.ndet
    nsa, nsb = ctx.nstr
    c = torch.empty(N, dtype=torch.float32, device=dev)
    fgpu.fill_pm1(c)
    s = torch.empty_like(c)
    stream = torch.cuda.current_stream(dev)
    pkg.fci_profile_enable(ctx, True)
    clocks = ClockSampler(local)
    clocks.start()
    t = time_sigma_ring(pkg, ctx, [c], [s], args.steps, args.warmup, stream, world)
    clk = clocks.stop()
    names, prof = pkg.fci_profile_read(ctx)
    pkg.fci_profile_enable(ctx, False)
    t = max_over_ranks(t, world)
    kmean = prof[-args.steps:].mean(axis=0) / 1e3
    value = world * N * args.steps / t / 1e9
    sa = pkg.fci_query(ctx, 4)
    kpad = -(-sa // 16) * 16
    npad = -(-(norb * (norb + 1) // 2) // 16) * 16
    nsplit = pkg.default_options().f32_splits
    products = nsplit * (nsplit + 1) // 2
    tiles = nsa * (-(-nsb // 128))
    mma_flops = products * 2.0 * 128 * npad * kpad * tiles
    itc = names.index("sigma3_tc")
    peaks = load_peaks()
    roof = {"kernel": "sigma3_tc", "bound": "tensor", "achieved": mma_flops / kmean[itc] / 1e12,
            "peak": peaks["bf16_tflops"], "unit": "TFLOP/s", "frac": mma_flops / kmean[itc] / 1e12 / peaks["bf16_tflops"],
            "traffic": None,
            "work_per_launch": f"{mma_flops:.4g} bf16 MMA FLOP ({products} slice products x 2 x 128 x {npad} x "
                               f"{kpad} x {tiles} tiles)",
            "kernels": {n: {"ms": float(kmean[i] * 1e3), "share": float(kmean[i] / kmean.sum())}
                        for i, n in enumerate(names)}}
    # end to end: host vector in, host sigma out, every step (a few steps: 9.4 GB each way)
    e2e_steps = min(args.steps, 3)
    hc = c.cpu().pin_memory()
    hs = torch.empty_like(hc).pin_memory()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        c.copy_(hc, non_blocking=True)
        pkg.fci_sigma(ctx, c, s, stream=stream)
        hs.copy_(s, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e = world * N * e2e_steps / (e0.elapsed_time(e1) / 1e3) / 1e9
    pkg.fci_free(ctx)
    # split-BF16x3 (2 bf16 slices, 3 products; about 1e-5 relative) on the same vectors
    ctx3 = pkg.fci_init(norb, na, nb, h1, eri, pkg.default_options(f32_splits=2))
    pkg.fci_profile_enable(ctx3, True)
    t3 = time_sigma_ring(pkg, ctx3, [c], [s], args.steps, args.warmup, stream, world)
    names3, prof3 = pkg.fci_profile_read(ctx3)
    t3 = max_over_ranks(t3, world)
    bf16x3 = {"value": world * N * args.steps / t3 / 1e9, "unit": "Gdet/s",
              "kernels": {n: {"ms": float(prof3[-args.steps:, i].mean())} for i, n in enumerate(names3)}}
    pkg.fci_free(ctx3)
    result = {
        "metric": metric_name(args.workload), "value": value, "unit": "Gdet/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_desc(args.workload),
                   "l2": f"one input vector of {N * 4 / 1e9:.1f} GB > 129 MB L2", "parallelism": "single GPU"},
        "roofline": roof, "clocks": clk, "gpu_launches": int(args.steps * 5),  # sigma_2, transpose, sigma_1, transpose-add, sigma_3
        "e2e": {"value": e2e, "unit": "Gdet/s", "h2d_bytes_per_step": N * 4, "d2h_bytes_per_step": N * 4},
        "bf16x3_sigma": bf16x3,
    }
    if args.davidson and rank == 0:
        # the mixed-precision solve of this space: FP32 basis of at most 8
        # vectors (the FP64 basis does not fit), FP32 sigma for the
        # corrections, FP64 sigma at refinement points, to 1e-8 Eh
        del hc, hs, c, s
        torch.cuda.empty_cache()
        ctxm = pkg.fci_init(norb, na, nb, h1, eri,
                            pkg.default_options(precision=pkg.FCI_PREC_MIXED, max_iter=args.max_iter,
                                                spin_parity=args.spin_parity))
        t0 = time.perf_counter()
        try:
            em = pkg.fci_davidson(ctxm, args.roots, 1e-8)
            conv = True
        except pkg.FciError as ex:
            if ex.code != pkg.fci.FCI_ERR_NOCONV:
                raise
            em, conv = None, False
        wall = time.perf_counter() - t0
        log = pkg.fci_davidson_log(ctxm, args.roots)
        exact = log[log[:, 1] == 0]
        last32 = log[log[:, 1] == 1]
        result["davidson"] = {
            "roots": args.roots, "tol": 1e-8, "converged": conv, "wall_s": wall,
            "E_exact": [float(x) for x in (exact[-1, 3:] if len(exact) else [])],
            "E_fp32_subspace_last": [float(x) for x in (last32[-1, 3:] if len(last32) else [])],
            "abs_diff_fp32_subspace_vs_exact": (float(np.abs(last32[-1, 3:] - exact[-1, 3:]).max())
                                                if len(exact) and len(last32) else None),
            "iterations": int(pkg.fci_query(ctxm, 8)), "sigma_calls": int(pkg.fci_query(ctxm, 9)),
            "refinement_points": int(len(exact)),
            "exact_energies": [[float(r[0]), float(r[2]), float(r[3])] for r in exact],
            "basis": "FP32 (fci_options.basis_f32 = 0 chose it: the FP64 basis does not fit)",
            "spin_parity": args.spin_parity,
        }
        pkg.fci_free(ctxm)
    if args.cpu_baseline and rank == 0 and world == 1:
        import oracle

        rng = np.random.default_rng(7)
        rows = rng.integers(0, N, 64)
        oracle.sigma_rows_generated(norb, na, nb, h1, eri, rows[:4], fi.DEFAULT_VECTOR_SEED, fi.STREAM_C_PM1)
        t0 = time.perf_counter()
        nrows = 0
        while time.perf_counter() - t0 < args.cpu_seconds:
            oracle.sigma_rows_generated(norb, na, nb, h1, eri, rows, fi.DEFAULT_VECTOR_SEED, fi.STREAM_C_PM1)
            nrows += len(rows)
        dt = time.perf_counter() - t0
        result["cpu_baseline"] = {"value": nrows / dt / 1e9, "unit": "Gdet/s", "cores": oracle.num_threads(),
                                  "kind": "oracle", "sample": f"{nrows} sampled sigma rows of CAS({na + nb}e,{norb}o), "
                                                              f"direct Slater-Condon sum, FP64, {dt:.1f} s"}
    if rank == 0:
        print(json.dumps(result))
    return 0


def density_leg(pkg, norb, na, nb, h1, eri, c_dev, sigma_ms, peaks):
    """The density step after the Davidson iterations (Table 2's "1e/2e
    Density Matrices"): gamma (fci_rdm1) and Gamma with gamma (fci_rdm2) of one
    vector, blocking calls timed whole (median of three), and the kernels of a
    one-chunk fci_rdm2 from the library's CUDA-event profile."""
    import time

    ctx = pkg.fci_init(norb, na, nb, h1, eri)
    t1, t2 = [], []
    for _ in range(3):
        t = time.perf_counter()
        pkg.fci_rdm1(ctx, c_dev)
        t1.append(time.perf_counter() - t)
        t = time.perf_counter()
        pkg.fci_rdm2(ctx, c_dev)
        t2.append(time.perf_counter() - t)
    pkg.fci_free(ctx)
    n = norb
    R = n * n + 1
    Rd = (R + 7) // 8 * 8
    nks = (c_dev.numel() + 15) // 16
    ctx1 = pkg.fci_init(norb, na, nb, h1, eri, pkg.default_options(rdm2_chunk_bytes=float(6 * Rd * 32 * nks + 1)))
    pkg.fci_profile_enable(ctx1, True)
    for _ in range(3):
        pkg.fci_rdm2(ctx1, c_dev)
    names, prof = pkg.fci_profile_read(ctx1)
    pkg.fci_profile_enable(ctx1, False)
    pkg.fci_free(ctx1)
    km = np.median(prof[-2:], axis=0)  # ms per kernel
    bn = 48  # B rows per tile of the Gram kernel
    nrb, ncb = (Rd + 127) // 128, (Rd + bn - 1) // bn
    ntile = sum(ncb - (-(-(rb * 128 - (bn - 1)) // bn) if rb * 128 > bn - 1 else 0) for rb in range(nrb))
    executed = 2.0 * 128 * bn * 16 * 21 * ntile * nks  # MMA FLOP: 21 digit products per tile and K-step
    useful = float(R) * R * 16 * nks  # one triangle of the FP64 Gram matrix, 2 FLOP per product
    itc = list(names).index("rdm2_tc")
    tc_s = km[itc] / 1e3
    peak = peaks.get("bf16_tflops")
    planes = 6.0 * Rd * 32 * nks  # digit-plane bytes, read once
    path, marker, digest, ratio = RDM2_TC_TRAFFIC
    try:
        traffic = planes * ratio if kernel_digest(path, marker) == digest else None
    except (OSError, ValueError):
        traffic = None
    return {
        "workload": f"CAS({na + nb}e,{norb}o), N = {c_dev.numel()}",
        "rdm1_ms": 1e3 * float(np.median(t1)), "rdm2_ms": 1e3 * float(np.median(t2)),
        "rdm2_over_sigma": float(np.median(t2)) * 1e3 / sigma_ms,
        "rdm2_one_chunk_kernels_ms": {nm: float(km[i]) for i, nm in enumerate(names)},
        "rdm2_tc_roofline": {"bound": "tensor", "achieved": executed / tc_s / 1e12, "peak": peak,
                             "unit": "TFLOP/s", "frac": (executed / tc_s / 1e12 / peak) if peak else None,
                             "executed_flop": executed, "fp64_equivalent_tflops": useful / tc_s / 1e12,
                             "traffic": traffic, "digit_plane_bytes": planes,
                             "traffic_note": "DRAM bytes per digit-plane byte of a CAS(12e,12o) ncu capture "
                                             "(profiles/rdm2_tc_cas12.md), scaled to this workload's planes",
                             "note": "executed bf16 MMA FLOP (6 digits, 21 products, 128 x 48 tiles) per launch / "
                                     "CUDA-event time; peak = measured burst bf16"},
        "timing": "whole blocking calls (allocation, statistics round trip, host copies included), median of 3",
    }


def run_densities(args):
    """Only the density step on the chosen workload (profiling the 2-RDM kernels):
    one JSON line with the density leg and the FP64 sigma time it is compared with."""
    import torch

    import paper_1707_04346_gb300 as pkg

    norb, na, nb, rank_eri = WORKLOADS[args.workload]
    h1, eri = fi.make_integrals(norb, rank_eri)
    ctx = pkg.fci_init(norb, na, nb, h1, eri)
    c = fi.make_vector(ctx.ndet)
    cd = torch.from_numpy(c / np.linalg.norm(c)).cuda()
    sd = torch.empty_like(cd)
    for _ in range(args.warmup):
        pkg.fci_sigma(ctx, cd, sd)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        pkg.fci_sigma(ctx, cd, sd)
    e1.record()
    torch.cuda.synchronize()
    sigma_ms = e0.elapsed_time(e1) / args.steps
    pkg.fci_free(ctx)
    print(json.dumps({"workload": workload_desc(args.workload), "sigma_ms": sigma_ms,
                      "densities": density_leg(pkg, norb, na, nb, h1, eri, cd, sigma_ms, load_peaks())}))
    return 0


def run_ours(args):
    import torch

    rank, world, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_1707_04346_gb300 as pkg

    norb, na, nb, rank_eri = WORKLOADS[args.workload]
    h1, eri = fi.make_integrals(norb, rank_eri)
    ctx = pkg.fci_init(norb, na, nb, h1, eri, pkg.default_options(f64_kernels=F64_KERNELS[args.f64_kernels],
                                                                  same_spin_tc=args.same_spin_tc))
    N = ctx.ndet
    nsa, nsb = ctx.nstr
    c_host = fi.make_vector(N)
    stream = torch.cuda.current_stream(dev)
    # ring of inputs/outputs larger than L2
    ring = max(2, int(np.ceil(4 * 129e6 / (N * 8))))
    c0 = torch.from_numpy(c_host).to(dev)
    vecs = [c0 * (1.0 + 0.01 * k) for k in range(ring)]
    outs = [torch.empty_like(c0) for _ in range(ring)]

    # FP64 sigma: the headline
    pkg.fci_profile_enable(ctx, True)
    clocks = ClockSampler(local)
    clocks.start()
    t = time_sigma_ring(pkg, ctx, vecs, outs, args.steps, args.warmup, stream, world)
    clk = clocks.stop()
    names, prof = pkg.fci_profile_read(ctx)
    pkg.fci_profile_enable(ctx, False)
    prof = prof[-args.steps:]
    t = max_over_ranks(t, world)
    value = replicas.job_throughput(N * args.steps, t, world) / 1e9
    kmean = prof.mean(axis=0) / 1e3  # seconds per launch
    kshare = prof.sum(axis=0) / prof.sum()
    top = int(np.argmax(kmean))
    sa = pkg.fci_query(ctx, 4)
    sb = pkg.fci_query(ctx, 5)

    peaks = load_peaks()
    roof = roofline_table(names, kmean, kshare, norb, na, nb, N, sa, sb, nsa, nsb, peaks, args.workload)
    if "sigma3_sliced" in names:
        i3 = names.index("sigma3_sliced")
        exact_sparse = 2.0 * sa * sb * N  # 2 s^2 FLOP per determinant (the method's exact-sparse count)
        roof["sigma3_sliced_exact_sparse_equivalent_tflops"] = exact_sparse / kmean[i3] / 1e12

    # FP32 sigma (sigma_3 on the tensor cores, split-BF16x6 by default)
    v32 = [v.float() for v in vecs]
    o32 = [torch.empty_like(v) for v in v32]
    pkg.fci_profile_enable(ctx, True)
    t32 = time_sigma_ring(pkg, ctx, v32, o32, args.steps, args.warmup, stream, world)
    names32, prof32 = pkg.fci_profile_read(ctx)
    pkg.fci_profile_enable(ctx, False)
    t32 = max_over_ranks(t32, world)
    fp32_value = world * N * args.steps / t32 / 1e9
    del v32, o32
    p32 = prof32[-args.steps:]
    roof_tc = roofline_table(names32, p32.mean(axis=0) / 1e3, p32.sum(axis=0) / p32.sum(), norb, na, nb, N, sa, sb,
                             nsa, nsb, peaks, args.workload)
    if roof_tc["kernel"] != "sigma3_tc":  # report the tensor-core kernel's own roofline next to the top one
        k = list(names32).index("sigma3_tc")
        roof_tc["sigma3_tc"] = roofline_table(names32[k:k + 1], p32.mean(axis=0)[k:k + 1] / 1e3, np.ones(1), norb, na,
                                              nb, N, sa, sb, nsa, nsb, peaks, args.workload)

    # split-BF16x3 sigma_3 (2 bf16 slices, 3 products; about 1e-5 relative)
    ctx3 = pkg.fci_init(norb, na, nb, h1, eri, pkg.default_options(f32_splits=2))
    v32 = [v.float() for v in vecs]
    o32 = [torch.empty_like(v) for v in v32]
    pkg.fci_profile_enable(ctx3, True)
    t3 = time_sigma_ring(pkg, ctx3, v32, o32, args.steps, args.warmup, stream, world)
    names3, prof3 = pkg.fci_profile_read(ctx3)
    t3 = max_over_ranks(t3, world)
    bf16x3 = {"value": world * N * args.steps / t3 / 1e9, "unit": "Gdet/s",
              "kernels": {n: {"ms": float(prof3[-args.steps:, i].mean())} for i, n in enumerate(names3)}}
    del v32, o32
    pkg.fci_free(ctx3)

    # end to end through the C ABI with host buffers: every step copies its input from pinned
    # host memory and reads its sigma back; two buffer sets and separate copy streams let the
    # copies of one step run under the sigma of the next (the copies stay inside the timed region)
    hc = torch.from_numpy(c_host).pin_memory()
    hs = [torch.empty(N, dtype=torch.float64).pin_memory() for _ in range(2)]
    dc = [torch.empty(N, dtype=torch.float64, device=dev) for _ in range(2)]
    ds = [torch.empty_like(dc[0]) for _ in range(2)]
    s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_sig = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]

    def e2e_step(k):
        b = k % 2
        if k >= 2:
            s_in.wait_event(ev_sig[b])  # the sigma that read dc[b] two steps ago is done
        with torch.cuda.stream(s_in):
            dc[b].copy_(hc, non_blocking=True)
            ev_in[b].record(s_in)
        stream.wait_event(ev_in[b])
        if k >= 2:
            stream.wait_event(ev_out[b])  # ds[b] of two steps ago has been read back
        pkg.fci_sigma(ctx, dc[b], ds[b], stream=stream)
        ev_sig[b].record(stream)
        s_out.wait_event(ev_sig[b])
        with torch.cuda.stream(s_out):
            hs[b].copy_(ds[b], non_blocking=True)
            ev_out[b].record(s_out)

    for k in range(args.warmup):
        e2e_step(k)
    torch.cuda.synchronize()
    barrier(world)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s_in)
    for k in range(args.steps):
        e2e_step(k)
    s_out.wait_event(ev_sig[(args.steps - 1) % 2])
    e1.record(s_out)
    torch.cuda.synchronize()
    te = max_over_ranks(e0.elapsed_time(e1) / 1e3, world)
    e2e = {"value": world * N * args.steps / te / 1e9, "unit": "Gdet/s", "h2d_bytes_per_step": N * 8,
           "d2h_bytes_per_step": N * 8,
           "pipelining": "two buffer sets; host-to-device and device-to-host copies on their own streams, "
                         "overlapping the neighbouring steps' sigma"}
    del vecs, outs

    result = None
    if rank == 0:
        result = {
            "metric": metric_name(args.workload), "value": value, "unit": "Gdet/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_desc(args.workload),
                       "l2": f"input/output ring of {ring} vectors x {N * 8 / 1e6:.0f} MB > 129 MB L2",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": roof, "clocks": clk,
            "gpu_launches": LAUNCHES_PER_SIGMA.get(tuple(names), len(names)) * args.steps, "e2e": e2e,
            "fp32_sigma": {"value": fp32_value, "unit": "Gdet/s", "roofline": roof_tc},
            "bf16x3_sigma": bf16x3,
        }
    if args.davidson and rank == 0:
        import torch as _t

        nr = args.roots
        ref_converged = True
        if args.ref_from_mixed:
            # mixed solve first; the FP64 reference then starts from its vectors
            # (an FP64 solve from scratch is not timed on this path)
            ctxm = pkg.fci_init(norb, na, nb, h1, eri,
                                pkg.default_options(precision=pkg.FCI_PREC_MIXED, max_iter=600))
            xm = _t.empty((nr, N), dtype=_t.float64, device=dev)
            em = pkg.fci_davidson(ctxm, nr, 1e-8, vecs=xm)  # the target accuracy (1e-8 Eh)
            logm = pkg.fci_davidson_log(ctxm, nr)
            pkg.fci_free(ctxm)
            ctxm = None
            ref_ctx = pkg.fci_init(norb, na, nb, h1, eri, pkg.default_options(max_iter=30))
            try:
                e_ref = pkg.fci_davidson(ref_ctx, nr, 1e-10, guess=xm)
                ref_converged = True
            except pkg.FciError:  # bounded: report the last FP64 iterate
                ref_converged = False
                e_ref = pkg.fci_davidson_log(ref_ctx, nr)[-1, 3:3 + nr]
            log64 = pkg.fci_davidson_log(ref_ctx, nr)
            pkg.fci_free(ref_ctx)
            del xm
        else:
            # the FP64 solve from scratch (on a context with room for many
            # iterations: a 3-root CAS(16,16) solve needs several hundred)
            ctx64 = pkg.fci_init(norb, na, nb, h1, eri, pkg.default_options(max_iter=args.max_iter))
            e_ref = pkg.fci_davidson(ctx64, nr, 1e-10 if args.workload == "cas14" else 1e-9)
            log64 = pkg.fci_davidson_log(ctx64, nr)
            pkg.fci_free(ctx64)
            ctxm = pkg.fci_init(norb, na, nb, h1, eri,
                                pkg.default_options(precision=pkg.FCI_PREC_MIXED, max_iter=args.max_iter))
            em = pkg.fci_davidson(ctxm, nr, 1e-10 if args.workload == "cas14" else 1e-9)
            logm = pkg.fci_davidson_log(ctxm, nr)
        result["davidson"] = {
            "roots": nr, "E_fp64": [float(x) for x in e_ref], "E_mixed": [float(x) for x in em],
            "abs_diff": float(np.abs(em - e_ref).max()),
            "abs_diff_per_root": [float(x) for x in np.abs(em - e_ref)],
            "fp64_reference": (("FP64 solve to 1e-10 from the mixed vectors (mixed solve to 1e-8)"
                                + ("" if ref_converged else ", not converged in 30 iterations: last iterate"))
                               if args.ref_from_mixed else
                               "FP64 solve from scratch to " + ("1e-10" if args.workload == "cas14" else "1e-9")),
            "fp64_time_to_1e-8_s": None if args.ref_from_mixed else time_to_tol(log64, e_ref),
            "mixed_time_to_1e-8_s": time_to_tol(logm, e_ref),
            "fp64_iterations": int(len(log64)), "mixed_iterations": int(len(logm)),
            "mixed_fp32_iterations": int((logm[:, 1] == 1).sum()),
        }
        if ctxm is not None:
            pkg.fci_free(ctxm)
        if na == nb and nr == 1 and not args.ref_from_mixed:
            # the same solves on the singlet combinations (spin_parity = +1: the
            # ground state here is a singlet), with sigma_1 formed from sigma_2
            sp = {}
            for label, prec in (("fp64", pkg.FCI_PREC_FP64), ("mixed", pkg.FCI_PREC_MIXED)):
                cs = pkg.fci_init(norb, na, nb, h1, eri, pkg.default_options(precision=prec, spin_parity=1))
                if label == "fp64":
                    pkg.fci_profile_enable(cs, True)  # the solver's sigma calls (sigma_1 from sigma_2)
                es = pkg.fci_davidson(cs, 1, 1e-10)
                ls = pkg.fci_davidson_log(cs, 1)
                sp[label] = {"E": float(es[0]), "abs_diff_vs_full_space_fp64": float(abs(es[0] - e_ref[0])),
                             "time_to_1e-8_s": time_to_tol(ls, e_ref), "iterations": int(len(ls))}
                if label == "fp64":
                    names_s, prof_s = pkg.fci_profile_read(cs)
                    km = prof_s[2:].mean(axis=0)
                    sp[label]["sigma_ms"] = float(km.sum())
                    sp[label]["sigma_kernels_ms"] = {n: float(km[i]) for i, n in enumerate(names_s)}
                    pkg.fci_profile_enable(cs, False)
                pkg.fci_free(cs)
            result["davidson"]["singlet"] = sp
    if args.batched and rank == 0:
        result["batched"] = run_batched(pkg, args.batch_instances)
    if args.extra and args.workload == "cas14":
        # the other sigma configurations: CAS(16,16) and CAS(18,18), both
        # precisions (an FP64 sigma at CAS(18,18) takes about 10 s: two steps)
        legs = {}
        legs["cas16_sigma"] = sigma_leg(pkg, "cas16", max(3, args.steps // 4), 3, stream, world,
                                        args.cpu_seconds / 3 if (args.cpu_baseline and world == 1) else 0)
        legs["cas18_sigma"] = sigma_leg(pkg, "cas18", 2, 2, stream, world,
                                        args.cpu_seconds / 3 if (args.cpu_baseline and world == 1) else 0)
        if rank == 0:
            cd = torch.from_numpy(c_host / np.linalg.norm(c_host)).to(dev)
            legs["densities"] = density_leg(pkg, norb, na, nb, h1, eri, cd, t / args.steps * 1e3, peaks)
            del cd
        if rank == 0:
            result.update(legs)
    if args.cpu_baseline and rank == 0 and world == 1:
        result["cpu_baseline"] = cpu_baseline(norb, na, nb, h1, eri, c_host, target_s=args.cpu_seconds)
    if rank == 0:
        print(json.dumps(result))
    pkg.fci_free(ctx)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cas14", choices=sorted(WORKLOADS))
    ap.add_argument("--no-davidson", dest="davidson", action="store_false")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-batched", dest="batched", action="store_false")
    ap.add_argument("--batch-instances", type=int, default=64)
    ap.add_argument("--no-extra", dest="extra", action="store_false",
                    help="skip the CAS(16,16) and CAS(18,18) sigma legs")
    ap.add_argument("--roots", type=int, default=1, help="Davidson roots (CAS(16,16) configuration: 3)")
    ap.add_argument("--max-iter", type=int, default=600,
                    help="Davidson iteration limit of the large solves (CAS(16,16) roots, CAS(18,18))")
    ap.add_argument("--f64-kernels", default="auto", choices=sorted(F64_KERNELS),
                    help="FP64 sigma kernels of the timed context (profiling a kernel family on a small space)")
    ap.add_argument("--spin-parity", type=int, default=0, choices=(-1, 0, 1),
                    help="CAS(18,18) solve on the Ms = 0 combinations of one spin parity (1: singlets)")
    ap.add_argument("--same-spin-tc", type=int, default=0, choices=(0, 1),
                    help="FP32 same-spin terms through intermediate strings on the tensor cores in the timed context")
    ap.add_argument("--densities-only", action="store_true",
                    help="run only the density step (fci_rdm1, fci_rdm2) on the workload and print its leg")
    ap.add_argument("--ref-from-mixed", action="store_true",
                    help="FP64 reference energies from an FP64 solve started at the mixed solution")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.densities_only and args.workload not in LARGE:
        return run_densities(args)
    if args.workload in LARGE:
        return run_large(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
