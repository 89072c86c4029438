#!/usr/bin/env python3
"""Benchmark: GSE-SpMV GB/s and % of the HBM roofline per precision level k,
and stepped-CG time-to-1e-10 against FP64 CSR CG on the same GPU.

Workload (one "step"): GSE-SpMV at k = 1, 2, 3 on the 3D 7-point Laplacian
128^3 (n = 2,097,152, nnz = 14,581,760) and on the random power-law matrix
(n = 1,000,000, mean row length 16, max 2048, values +-10^U(-3,3)); x ~ U[-1,1],
seeded.  L2 is flushed (a 256 MiB write) before every timed SpMV; each SpMV is
timed with CUDA events on the launching stream.  After the timed steps, the
FP64/FP32 CSR baselines of the same matrices and the solver comparison (config
"3D 7-point Laplacian 192^3 + 1e-3 shift, CG to 1e-10") are measured once and
reported beside the headline.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun (N > 1) every rank runs the same workload on its own GPU
(replicas: the single-matrix SpMV does not shard) and rank 0 prints one line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "GSE-SpMV GB/s & % HBM roofline per k; stepped-CG time-to-1e-10 vs FP64 CSR CG"


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


PEAKS_FILE = os.path.join(ROOT, "profiles", "peaks_gb300.json")


def machine_peaks():
    """The FP64 FMA rate and the random-gather rate that `bench.py --peaks`
    measured on this GPU pool (profiles/peaks_gb300.json, written by that mode
    with the command that made it)."""
    d = json.load(open(PEAKS_FILE))
    return float(d["dfma_per_s"]), float(d["gather_per_s_8MB"])


def run_peaks(args):
    """Measures the machine floors the SpMV is held against: the FP64 FMA rate
    (full occupancy, and with a given number of dependent chains per SM), the
    DFMA latency, and random 8-byte gathers from tables of 8 MB to 1 GB through
    L1 and L2 only.  Prints one JSON line; with --peaks-out also writes it."""
    import torch
    import paper_2411_04686_gb300 as gse
    torch.cuda.set_device(0)
    res = {"gpu": torch.cuda.get_device_name(0), "sms": torch.cuda.get_device_properties(0).multi_processor_count}
    with Clocks(0) as clk:
        res["dfma_per_s"] = max(gse.probe(gse.PROBE_DFMA_RATE)[0] for _ in range(3))
        res["dfma_latency_cycles"] = gse.probe(gse.PROBE_DFMA_LATENCY)[0]
        res["dfma_per_s_by_warps_per_sm"] = {str(w): gse.probe(gse.PROBE_DFMA_CHAINS, w)[0]
                                             for w in (4, 8, 16, 24, 32, 48, 64)}
        for mb in (8, 32, 128, 1024):
            words = mb * 2**20 // 8
            t = torch.rand(words, dtype=torch.float64, device="cuda")
            res[f"gather_per_s_{mb}MB"] = max(gse.probe(gse.PROBE_GATHER_L1, words, t)[0] for _ in range(3))
            res[f"gather_l2only_per_s_{mb}MB"] = max(gse.probe(gse.PROBE_GATHER_L2, words, t)[0] for _ in range(3))
            del t
        torch.cuda.synchronize()
    res["clocks"] = clk.summary()
    res["command"] = "python bench.py --peaks --peaks-out profiles/peaks_gb300.json"
    line = json.dumps(res)
    print(line)
    if args.peaks_out:
        with open(args.peaks_out, "w") as f:
            f.write(json.dumps(res, indent=1) + "\n")


def algorithmic_bytes(nnz, n_rows, n_cols, k, seg=(16, 16, 20), G=32):
    """col 4 B + live segments + group exponent per nonzero, row_ptr, x once, y once.
    G = 0: the global-table format (no per-group exponents; the index rides in col)."""
    return nnz * (4 + sum(seg[:k]) / 8.0 + (2.0 / G if G else 0.0)) + 4 * (n_rows + 1) + 8 * n_cols + 8 * n_rows


def csr_bytes(nnz, n_rows, n_cols, vbytes):
    return nnz * (4 + vbytes) + 4 * (n_rows + 1) + 8 * n_cols + 8 * n_rows


def spmv_kernels_per_call(schedule, nnz, rows_schedule=8):
    """Kernels one gse_spmv call launches at a GSE level: one for the row
    schedule; for the nonzero split (schedule = units of 8 nonzeros per lane,
    256 * schedule nonzeros per chunk) a second, the split-row pass, whenever
    the matrix spans more than one chunk."""
    if schedule == rows_schedule:
        return 1
    return 2 if nnz > 256 * schedule else 1


SPMV_SOURCES = ("gse_internal.cuh", "spmv_core.cuh", "spmv_lanerow.cuh", "spmv_pipe.cuh", "spmv.cu")


def src_hash():
    """Hash of the sources the standalone SpMV kernels are built from: the
    stored DRAM counters are reported only while it still matches."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2411_04686_gb300", "csrc")
    for f in SPMV_SOURCES:
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi during a region.

    The GPU is named by the UUID of the CUDA device (nvidia-smi numbers GPUs
    its own way on a shared node).  If the full query is refused, a smaller
    set of fields is tried; nvidia-smi's error text is kept for the summary."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    Q_OLD = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_throttle_reasons.active,"
             "clocks_throttle_reasons.hw_slowdown,clocks_throttle_reasons.hw_thermal_slowdown,"
             "clocks_throttle_reasons.sw_thermal_slowdown,clocks_throttle_reasons.sw_power_cap")
    Q_MIN = "index,clocks.sm,clocks.max.sm,power.draw"

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.err = ""
        self.lines = []

    def _gpu_id(self):
        try:
            import torch
            u = str(torch.cuda.get_device_properties(self.gpu).uuid)
            return u if u.startswith("GPU-") else "GPU-" + u
        except Exception:                   # noqa: BLE001 -- older torch: fall back to the index
            return str(self.gpu)

    def _start(self, q):
        p = subprocess.Popen(["nvidia-smi", f"--id={self._gpu_id()}", f"--query-gpu={q}",
                              "--format=csv,noheader,nounits", "-lms", "50"],
                             stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)
        first = p.stdout.readline()         # the sampler is running before the region starts
        if first.strip() and "," in first:
            return p, first
        try:
            _, err = p.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            p.kill()
            _, err = p.communicate()
        self.err = (first + " " + (err or "")).strip()[:200]
        return None, ""

    def __enter__(self):
        for q in (self.Q, self.Q_OLD, self.Q_MIN):
            try:
                self.proc, first = self._start(q)
            except (OSError, FileNotFoundError) as e:
                self.err = str(e)[:200]
                self.proc = None
                break
            if self.proc:
                self.first = first
                break
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in (self.first + out).splitlines() if l.strip()]

    def summary(self):
        return clock_summary(self.lines, self.err)


def clock_summary(lines, err=""):
    """Median SM clock, maximum clock and the throttle reasons seen in
    nvidia-smi CSV lines (index, clocks.sm, clocks.max.sm, power.draw and,
    when queried, the active mask and four reason flags)."""
    sm, mx, reasons = [], 0.0, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for l in lines:
        f = [x.strip() for x in l.split(",")]
        if len(f) < 4:
            continue
        try:
            sm.append(float(f[1]))
            mx = max(mx, float(f[2]))
        except ValueError:
            continue
        for nm, v in zip(names, f[5:9]):
            if v.lower().startswith("active"):
                reasons.add(nm)
    if not sm:
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        if err:
            out["error"] = err
        return out
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def build_workload():
    A = synth.laplace3d(128)
    B = synth.powerlaw_random(1_000_000, 16.0, 2048, seed=0)
    return [("laplace3d_128", A), ("powerlaw_1m", B)]


def host_cores():
    """Host threads this process may run on (its CPU affinity)."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def step_sample(mats, frac):
    """A bounded sample of the step for the CPU legs: for each matrix, the block
    of rows in its middle holding `frac` of its rows, swept at k = 1, 2, 3.
    Returns (A, x, encoding, r0, r1, algorithmic bytes of the sampled part)
    per matrix; the bytes are the step's per-level bytes scaled by the sampled
    share of nonzeros, so the GB/s compare with the GPU's."""
    import oracle
    work = []
    for name, A in mats:
        n = A.n_rows
        m = max(1, int(n * frac))
        r0 = (n - m) // 2
        r1 = r0 + m
        share = (int(A.row_ptr[r1]) - int(A.row_ptr[r0])) / max(A.nnz, 1)
        nb = sum(algorithmic_bytes(A.nnz, A.n_rows, A.n_cols, k) for k in (1, 2, 3)) * share
        work.append((name, A, synth.uniform_x(A.n_cols, seed=0), oracle.encode(A.val), r0, r1, nb))
    return work


def sweep_sample(work, threads):
    import oracle
    for name, A, x, enc, r0, r1, nb in work:
        y = np.zeros(A.n_rows)
        for k in (1, 2, 3):
            oracle.gse_spmv_rows(A.row_ptr, A.col, enc, k, x, r0, r1, threads=threads, y=y)


REF_SAMPLE = 1.0 / 16.0   # share of each matrix's rows in one reference-arm step


def run_reference(args):
    """The oracle (plain single-thread C) on the host cores, same metric and
    unit: each step is the whole step's workload (both matrices, k = 1, 2, 3)
    on a bounded row sample (the middle sixteenth of each matrix's rows)."""
    import oracle
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    oracle.build()
    work = step_sample(build_workload(), REF_SAMPLE)
    per_step_bytes = sum(w[6] for w in work)
    for _ in range(args.warmup):
        sweep_sample(work, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sweep_sample(work, 1)
    dt = time.perf_counter() - t0
    v = per_step_bytes * args.steps / dt / 1e9
    sample = ("GSE-SpMV k=1,2,3 on laplace3d_128 and powerlaw_1m (the whole step's workload), each step on the "
              "middle 1/16 of each matrix's rows; one host thread")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": "gse_spmv_sweep_laplace3d128_powerlaw1m", "sample": sample,
                                        "sample_rows_fraction": REF_SAMPLE},
        "cpu_baseline": {"kind": "oracle", "value": round(v, 3), "unit": "GB/s", "cores": 1, "sample": sample},
        "e2e": {"value": round(v, 3), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def cpu_baseline(mats, min_seconds=10.0):
    """The oracle (plain single-thread C) on a bounded sample of the same step:
    GSE-SpMV at k = 1, 2, 3 over both matrices, whole passes repeated until at
    least min_seconds have passed."""
    import oracle
    oracle.build()
    work = []
    for name, A in mats:
        work.append((A, synth.uniform_x(A.n_cols, seed=0), oracle.encode(A.val)))
    passes, nbytes = 0, 0.0
    t0 = time.perf_counter()
    while True:
        for A, x, enc in work:
            for k in (1, 2, 3):
                oracle.gse_spmv(A.row_ptr, A.col, enc, k, x)
                nbytes += algorithmic_bytes(A.nnz, A.n_rows, A.n_cols, k)
        passes += 1
        dt = time.perf_counter() - t0
        if dt >= min_seconds:
            break
    names = " and ".join(name for name, _ in mats)
    return {"value": round(nbytes / dt / 1e9, 3), "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": f"{passes} whole passes of the step (GSE-SpMV k=1,2,3 on {names}), {dt:.1f} s on one host thread"}


def cpu_baseline_all_cores(mats, min_seconds=5.0):
    """The oracle's SpMV with its rows shared among all host cores (OpenMP;
    every row summed as the single-thread oracle sums it): whole passes of the
    step repeated for at least min_seconds."""
    import oracle
    oracle.build()
    work = step_sample(mats, 1.0)
    cores = host_cores()
    sweep_sample(work, cores)                      # warm (thread pool, pages)
    passes, nbytes = 0, 0.0
    t0 = time.perf_counter()
    while True:
        sweep_sample(work, cores)
        nbytes += sum(w[6] for w in work)
        passes += 1
        dt = time.perf_counter() - t0
        if dt >= min_seconds:
            break
    names = " and ".join(name for name, _ in mats)
    return {"value": round(nbytes / dt / 1e9, 3), "unit": "GB/s", "cores": cores, "kind": "oracle (OpenMP rows)",
            "sample": f"{passes} whole passes of the step (GSE-SpMV k=1,2,3 on {names}), {dt:.1f} s on {cores} host threads"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gse")
    ap.add_argument("--no-solve", action="store_true", help="skip every solver section")
    ap.add_argument("--no-gmres", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-table", action="store_true", help="skip the global-table format section")
    ap.add_argument("--batch-systems", type=int, default=512)
    ap.add_argument("--profile-spmv", nargs=2, metavar=("MATRIX", "K"), default=None,
                    help="no timing: encode MATRIX (laplace3d_128 | powerlaw_1m), run gse_spmv at level K "
                         "(1, 2, 3, 64 = FP64 CSR) three times and exit; the target for ncu captures")
    ap.add_argument("--profile-cg", type=int, metavar="N", default=None,
                    help="no timing: FP64 and stepped CG once each on the N^3 Laplacian with shift 1e-3 "
                         "and exit; the target for ncu captures of the engine kernels")
    ap.add_argument("--profile-gmres", type=int, nargs=2, metavar=("N", "ITERS"), default=None,
                    help="no timing: FP64 GMRES(30) for ITERS iterations on the N^2 convection-diffusion "
                         "operator and exit; the target for ncu captures of the GMRES kernels")
    ap.add_argument("--serve-requests", type=int, default=10000)
    ap.add_argument("--serve-rates", default="0.5,1,2",
                    help="arrival rates as fractions of the measured saturated batch throughput")
    ap.add_argument("--peaks", action="store_true",
                    help="measure the FP64 FMA and random-gather rates (machine probes) and exit")
    ap.add_argument("--peaks-out", default=None, help="with --peaks: also write the JSON to this file")
    args = ap.parse_args()
    if args.peaks:
        run_peaks(args)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import paper_2411_04686_gb300 as gse
    if args.profile_spmv:
        name, k = args.profile_spmv[0], int(args.profile_spmv[1])
        A = dict(build_workload())[name]
        M = gse.GseMatrix.from_csr(A, attach=(64, 32))      # schedule from row statistics
        x = torch.from_numpy(synth.uniform_x(A.n_cols, seed=0)).cuda()
        y = torch.empty(A.n_rows, dtype=torch.float64, device="cuda")
        for _ in range(3):
            M.spmv(k, x, y)
        torch.cuda.synchronize()
        print(json.dumps({"profiled": name, "k": k, "schedule": M.info().schedule, "nnz": A.nnz}))
        return

    if args.profile_gmres:
        N, iters = args.profile_gmres
        A = synth.convdiff2d(N)
        M = gse.GseMatrix.from_csr(A, attach=(64,))
        b = torch.from_numpy(synth.rhs_ones(A)).cuda()
        x = torch.zeros(A.n_rows, dtype=torch.float64, device="cuda")
        pol = gse.Policy(**{**gse.fp64_policy(gse.SCALED_GMRES).__dict__, "max_iter": iters})
        t0 = time.perf_counter()
        info = M.gmres(b, x, tol=1e-10, policy=pol)
        torch.cuda.synchronize()
        print(json.dumps({"profiled_gmres": N, "iters": info["iters"], "status": info["status"],
                          "us_per_iter": round((time.perf_counter() - t0) / max(info["iters"], 1) * 1e6, 1)}))
        return

    if args.profile_cg:
        A = synth.laplace3d(args.profile_cg, shift=1e-3)
        M = gse.GseMatrix.from_csr(A, attach=(64,))
        b = torch.from_numpy(synth.rhs_ones(A)).cuda()
        out = {}
        for name, pol in (("fp64", gse.fp64_policy(gse.SCALED_CG)), ("gse", gse.SCALED_CG)):
            x = torch.zeros(A.n_rows, dtype=torch.float64, device="cuda")
            info = M.cg(b, x, tol=1e-10, policy=pol)
            out[name] = {"iters": info["iters"], "status": info["status"], "switch_iter": info["switch_iter"]}
        torch.cuda.synchronize()
        print(json.dumps({"profiled_cg": args.profile_cg, **out}))
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    hbm_peak, peak_kind = load_peaks()
    stream = torch.cuda.current_stream()

    mats = build_workload()
    handles = []
    for name, A in mats:
        M = gse.GseMatrix.from_csr(A, attach=(64, 32, gse.LEVEL_FP16, gse.LEVEL_BF16))  # schedule from row statistics
        x = torch.from_numpy(synth.uniform_x(A.n_cols, seed=0)).cuda()
        y = torch.empty(A.n_rows, dtype=torch.float64, device="cuda")
        handles.append((name, A, M, x, y))
    kernels_per_call = [spmv_kernels_per_call(h[2].info().schedule, h[1].nnz, gse.SCHEDULE_ROWS) for h in handles]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    flush_sink = torch.empty(1, dtype=torch.float32, device="cuda")

    def flush_l2(v):
        # write a buffer larger than L2, then read it back so that the dirty
        # lines are written out before the timed kernel starts
        flush.fill_(float(v))
        flush_sink.copy_(flush.sum())
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(6)]
    launches = [(hi, k) for hi in range(len(handles)) for k in (1, 2, 3)]

    def step(record):
        times = []
        for li, (hi, k) in enumerate(launches):
            name, A, M, x, y = handles[hi]
            flush_l2(li)
            e0, e1 = ev[li]
            e0.record(stream)
            M.spmv(k, x, y)
            e1.record(stream)
        if record:
            torch.cuda.synchronize()
            times = [ev[i][0].elapsed_time(ev[i][1]) for i in range(len(launches))]
        return times

    for _ in range(args.warmup):
        step(False)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    per_launch = [[] for _ in launches]
    with Clocks(local) as clk:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ts = step(True)
            for i, t in enumerate(ts):
                per_launch[i].append(t)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        wall = time.perf_counter() - t0
    clocks = clk.summary()
    kernel_ms = [sum(v) / len(v) for v in per_launch]
    ms_step = sum(kernel_ms)
    if dist:
        t = torch.tensor([ms_step], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_step = float(t.item())
    bytes_step = sum(algorithmic_bytes(handles[hi][1].nnz, handles[hi][1].n_rows, handles[hi][1].n_cols, k)
                     for hi, k in launches)
    value = bytes_step * world / (ms_step * 1e-3) / 1e9

    # per-k table and the dominant kernel's roofline
    DFMA_PEAK_PER_S, GATHER_PEAK_PER_S = machine_peaks()
    per_k = {}
    for i, (hi, k) in enumerate(launches):
        name, A = handles[hi][0], handles[hi][1]
        nb = algorithmic_bytes(A.nnz, A.n_rows, A.n_cols, k)
        gbs = nb / (kernel_ms[i] * 1e-3) / 1e9
        dfma_bound_gbs = nb / (A.nnz / DFMA_PEAK_PER_S) / 1e9
        per_k[f"{name}_k{k}"] = {"us": round(kernel_ms[i] * 1e3, 2), "GB_s": round(gbs, 1),
                                 "frac_hbm_measured": round(gbs / hbm_peak, 3),
                                 "frac_hbm_nominal_8TBs": round(gbs / 8000.0, 3),
                                 "algorithmic_MB": round(nb / 1e6, 1),
                                 "fp64_fma_bound_GB_s": round(dfma_bound_gbs, 1),
                                 "bound": "hbm" if dfma_bound_gbs >= hbm_peak else "alu(fp64 fma)"}
    dom = max(range(len(launches)), key=lambda i: kernel_ms[i])
    hi, k = launches[dom]
    dA = handles[hi][1]
    dbytes = algorithmic_bytes(dA.nnz, dA.n_rows, dA.n_cols, k)
    achieved = dbytes / (kernel_ms[dom] * 1e-3) / 1e9
    traffic = None
    tp = os.path.join(ROOT, "profiles", "spmv_traffic.json")
    if os.path.exists(tp):
        t = json.load(open(tp))
        key = f"{handles[hi][0]}_k{k}"
        if t.get("src_hash") == src_hash() and key in t.get("traffic_bytes", {}):
            traffic = t["traffic_bytes"][key]
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm_peak, "unit": "GB/s",
                "frac": round(achieved / hbm_peak, 3), "traffic": traffic,
                "kernel": f"gse_spmv k={k} on {handles[hi][0]} ({kernels_per_call[hi]} kernel(s) per call, timed together)",
                "peak_kind": peak_kind,
                "algorithmic_bytes": int(dbytes)}
    if handles[hi][0].startswith("powerlaw"):
        # the random-column matrix is bound by its x gathers, not by HBM: one
        # 8-byte gather per nonzero at the random-gather rate of an L2-resident
        # 8 MB vector that `bench.py --peaks` measured (profiles/peaks_gb300.json)
        floor_us = dA.nnz / GATHER_PEAK_PER_S * 1e6
        roofline["gather_floor_us"] = round(floor_us, 1)
        roofline["frac_of_gather_floor"] = round(floor_us / (kernel_ms[dom] * 1e3), 3)

    # baselines (not part of the step)
    baselines = {}
    for name, A, M, x, y in handles:
        for lv, vb in ((gse.LEVEL_FP64, 8), (gse.LEVEL_FP32, 4), (gse.LEVEL_FP16, 2), (gse.LEVEL_BF16, 2)):
            ts = []
            for _ in range(10):
                flush_l2(1)
                e0, e1 = ev[0]
                e0.record(stream)
                M.spmv(lv, x, y)
                e1.record(stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            ms = statistics.median(ts)
            nb = csr_bytes(A.nnz, A.n_rows, A.n_cols, vb)
            tag = {gse.LEVEL_FP64: "fp64", gse.LEVEL_FP32: "fp32", gse.LEVEL_FP16: "fp16", gse.LEVEL_BF16: "bf16"}[lv]
            baselines[f"{name}_{tag}"] = {"us": round(ms * 1e3, 2), "GB_s": round(nb / (ms * 1e-3) / 1e9, 1),
                                          "frac_hbm_measured": round(nb / (ms * 1e-3) / 1e9 / hbm_peak, 3)}
        gse_k1 = per_k[f"{name}_k1"]["us"]
        baselines[f"{name}_speedup_k1_vs_fp64"] = round(baselines[f"{name}_fp64"]["us"] / gse_k1, 3)
        baselines[f"{name}_fp16_overflow_values"] = int(M.info().overflow16)

    # the paper's default format: one global table of numExp shared exponents
    # (Sec. III-B), the index in the column word (Sec. III-C); per-level times
    # at numExp = 8 and the numExp sweep of Sec. IV-B (time and max |y - y_FP64|);
    # then numExp = 8 with the index kept in the head (Sec. III-C's layout for
    # columns without spare bits) and with the sampled extraction (Sec. III-B,
    # one row per 64-row block), with the encode's wall time beside the exact one
    table = None
    if not args.no_table:
        table = {}
        for name, A, M, x, y in handles:
            y64 = M.spmv(gse.LEVEL_FP64, x).clone()

            def measure(T, levels, row):
                for k in levels:
                    ts = []
                    for r in range(10):
                        flush_l2(r)
                        e0, e1 = ev[0]
                        e0.record(stream)
                        T.spmv(k, x, y)
                        e1.record(stream)
                        torch.cuda.synchronize()
                        ts.append(e0.elapsed_time(e1))
                    ms = statistics.median(ts)
                    nb = algorithmic_bytes(A.nnz, A.n_rows, A.n_cols, k, G=0)
                    row[f"k{k}_us"] = round(ms * 1e3, 2)
                    row[f"k{k}_GB_s"] = round(nb / (ms * 1e-3) / 1e9, 1)
                    row[f"k{k}_max_abs_err_vs_fp64"] = float((T.spmv(k, x) - y64).abs().max().item())
                return row

            sweep = {}
            for ne in (2, 4, 8, 16, 32, 64):
                T = gse.GseMatrix.from_csr(A, num_exp=ne)
                sweep[f"num_exp_{ne}"] = measure(T, (1, 2, 3) if ne == 8 else (1,), {"entries": T.info().num_exp})
                T.free()
            T = gse.GseMatrix.from_csr(A, num_exp=8, index_place=gse.INDEX_VALUE)
            sweep["num_exp_8_index_in_head"] = measure(T, (1, 2, 3), {"entries": T.info().num_exp,
                                                                      "index_in_head": T.info().index_in_head})
            T.free()
            # encode wall time from a device-resident CSR: exact vs sampled counts
            dA = [torch.from_numpy(a).cuda() for a in (A.row_ptr, A.col, A.val)]
            srows = synth.sample_rows(A.n_rows, 64, seed=0)
            enc_ms = {}
            for tag, kw in (("exact", {}), ("sampled_64", {"sample_block_rows": 64, "sample_rows": srows})):
                ts = []
                for r in range(4):
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    T = gse.GseMatrix(*dA, n_cols=A.n_cols, num_exp=8, **kw)
                    torch.cuda.synchronize()
                    ts.append((time.perf_counter() - t0) * 1e3)
                    if r < 3:
                        T.free()
                enc_ms[tag] = round(statistics.median(ts[1:]), 2)
            full_table = gse.GseMatrix(*dA, n_cols=A.n_cols, num_exp=8)
            row = {"entries": T.info().num_exp, "block_rows": 64,
                   "same_table_as_exact": T.export_table()[0].tolist() == full_table.export_table()[0].tolist(),
                   "encode_ms": enc_ms["sampled_64"], "encode_ms_exact": enc_ms["exact"]}
            full_table.free()
            sweep["num_exp_8_sampled_64"] = measure(T, (1,), row)
            T.free()
            del dA
            table[name] = sweep

    # e2e: through the C ABI with host buffers, copies inside the timed region.
    # Each step uploads every x from pinned memory and reads every y_k back;
    # the copies run on two copy streams ordered by events, so the upload of
    # the next matrix's x and the read-back of y_k overlap the SpMVs (one
    # result buffer per level), and the step ends with a full synchronise.
    pinned_x = [torch.from_numpy(synth.uniform_x(h[1].n_cols, seed=0)).pin_memory() for h in handles]
    pinned_y = [[torch.empty(h[1].n_rows, dtype=torch.float64).pin_memory() for _ in range(3)] for h in handles]
    ybuf = [[torch.empty(h[1].n_rows, dtype=torch.float64, device="cuda") for _ in range(3)] for h in handles]
    h2d = sum(p.numel() * 8 for p in pinned_x)
    d2h = sum(p.numel() * 8 for ps in pinned_y for p in ps)
    s_up, s_down = torch.cuda.Stream(), torch.cuda.Stream()
    comp = torch.cuda.current_stream()

    def e2e_step():
        ev_x = []
        with torch.cuda.stream(s_up):
            for hi, h in enumerate(handles):
                h[3].copy_(pinned_x[hi], non_blocking=True)
                ev_x.append(torch.cuda.Event())
                ev_x[-1].record(s_up)
        for hi, (name, A, M, x, y) in enumerate(handles):
            comp.wait_event(ev_x[hi])
            for ki, k in enumerate((1, 2, 3)):
                M.spmv(k, x, ybuf[hi][ki])
                ev = torch.cuda.Event()
                ev.record(comp)
                s_down.wait_event(ev)
                with torch.cuda.stream(s_down):
                    pinned_y[hi][ki].copy_(ybuf[hi][ki], non_blocking=True)
        torch.cuda.synchronize()

    e2e_step()                           # warm
    t0 = time.perf_counter()
    E = max(3, args.steps // 2)
    for _ in range(E):
        e2e_step()
    e2e_s = (time.perf_counter() - t0) / E
    for hi, (name, A, M, x, y) in enumerate(handles):    # the read-back is the SpMV result
        assert torch.equal(pinned_y[hi][2], M.spmv(3, x).cpu())
    e2e = {"value": round(bytes_step * world / e2e_s / 1e9, 2), "unit": "GB/s",
           "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

    solve = gmres = batched = served = None
    if not args.no_solve:
        solve = solver_comparison(gse, torch)
        if not args.no_gmres:
            gmres = gmres_comparison(gse, torch)
        if not args.no_batch:
            batched = batched_comparison(gse, torch, args.batch_systems, rank, world)
        if not args.no_serve:
            rate = batched["gse_stepped_batched"]["solves_per_s"] if batched else 400.0
            factors = tuple(float(f) for f in args.serve_rates.split(","))
            served = served_benchmark(gse, torch, args.serve_requests, rate, rank, world, factors)

    cpu = cpu_all = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline(mats)
        cpu_all = cpu_baseline_all_cores(mats)

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_step, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded; stand-ins for the paper's SuiteSparse sets)",
            "config": {"workload": "gse_spmv_sweep_laplace3d128_powerlaw1m", "levels": [1, 2, 3],
                       "group_size": 32, "seg_bits": [16, 16, 20], "l2": "flushed before each SpMV (256 MiB write, then a 256 MiB read so no dirty line is written back inside the timed kernel)",
                       "parallelism": "replicas" if world > 1 else "single_gpu",
                       "wall_s_timed_region": round(wall, 3)},
            "roofline": roofline, "per_k": per_k, "baselines": baselines, "table_format": table,
            "solve": solve, "gmres": gmres,
            "batched": batched, "served": served,
            "e2e": e2e, "gpu_launches": sum(kernels_per_call[hi] for hi, _ in launches) * args.steps, "clocks": clocks,
            "cpu_baseline": cpu,
            "cpu_baseline_all_cores": cpu_all,
        }
        print(json.dumps(line))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def iters_per_level(info):
    """Iterations run at each level k, from the switch iterations (the
    iteration at which level k started; -1: never reached)."""
    sw = list(info["switch_iter"]) + [info["iters"]]
    out = {}
    for k in range(len(sw) - 1):
        if sw[k] < 0:
            break
        nxt = next((v for v in sw[k + 1:] if v >= 0), info["iters"])
        out[f"k{k + 1}"] = nxt - sw[k]
    return out


def solver_comparison(gse, torch):
    """Time-to-1e-10: stepped GSE-CG vs FP64 CSR CG (same fused engine), on the
    3D 7-point Laplacian 192^3 with diagonal shift 1e-3; b = A*1, x0 = 0."""
    A = synth.laplace3d(192, shift=1e-3)
    M = gse.GseMatrix.from_csr(A, attach=(64,))
    b = torch.from_numpy(synth.rhs_ones(A)).cuda()
    out = {"workload": "laplace3d_192_shift1e-3_cg_tol1e-10", "n": A.n_rows, "nnz": A.nnz}
    variants = [("fp64_csr_cg", "SCALED_CG at FP64", gse.fp64_policy(gse.SCALED_CG)),
                ("gse_stepped_cg_paper_policy", "SCALED_CG", gse.SCALED_CG),
                ("gse_stepped_cg_floor_policy", "SCALED_CG + floor rule",
                 gse.Policy(**{**gse.SCALED_CG.__dict__, "flags": gse.POLICY_FLOOR})),
                ("gse_stepped_cg_paper_cg_preset", "PAPER_CG (first check at iteration l = 3000)", gse.PAPER_CG)]
    for name, pname, pol in variants:
        x = torch.zeros(A.n_rows, dtype=torch.float64, device="cuda")
        M.cg(b, x, tol=1e-10, policy=pol)     # warm (workspace, floor coefficients)
        x.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info = M.cg(b, x, tol=1e-10, policy=pol)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        err = float((x - 1.0).abs().max().item())
        out[name] = {"policy": pname, "seconds": round(dt, 4), "iters": info["iters"], "status": info["status"],
                     "k_final": info["k_final"], "switch_iter": info["switch_iter"],
                     "iters_per_level": iters_per_level(info),
                     "us_per_iter": round(dt / max(info["iters"], 1) * 1e6, 1),
                     "rel_res_true": info["rel_res_true"], "max_abs_err_vs_ones": err}
    M.free()
    # the same solve on the global-table format (numExp = 8, the paper's setting)
    T = gse.GseMatrix.from_csr(A, num_exp=8)
    x = torch.zeros(A.n_rows, dtype=torch.float64, device="cuda")
    T.cg(b, x, tol=1e-10, policy=gse.SCALED_CG)
    x.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    info = T.cg(b, x, tol=1e-10, policy=gse.SCALED_CG)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    out["gse_stepped_cg_table8"] = {"seconds": round(dt, 4), "iters": info["iters"], "status": info["status"],
                                    "k_final": info["k_final"], "switch_iter": info["switch_iter"],
                                    "rel_res_true": info["rel_res_true"],
                                    "max_abs_err_vs_ones": float((x - 1.0).abs().max().item())}
    T.free()
    # the paper's comparison (Sec. IV-D, tol 1e-6): FP64, FP16, BF16 storage and
    # stepped GSE; every residual also measured against the FP64 matrix
    P = gse.GseMatrix.from_csr(A, attach=(64, gse.LEVEL_FP16, gse.LEVEL_BF16))
    nb = float(b.norm().item())
    tol6 = {}
    for name, pol in (("fp64", gse.fp64_policy(gse.SCALED_CG)),
                      ("fp16", gse.fp64_policy(gse.SCALED_CG, gse.LEVEL_FP16)),
                      ("bf16", gse.fp64_policy(gse.SCALED_CG, gse.LEVEL_BF16)),
                      ("gse_stepped", gse.SCALED_CG)):
        x = torch.zeros(A.n_rows, dtype=torch.float64, device="cuda")
        P.cg(b, x, tol=1e-6, policy=pol)
        x.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info = P.cg(b, x, tol=1e-6, policy=pol)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        r = b - P.spmv(gse.LEVEL_FP64, x)
        tol6[name] = {"seconds": round(dt, 4), "iters": info["iters"], "status": info["status"],
                      "switch_iter": info["switch_iter"],
                      "rel_res_fp64_matrix": float(r.norm().item()) / nb}
    for name in ("fp16", "bf16", "gse_stepped"):
        tol6[name]["speedup_vs_fp64"] = round(tol6["fp64"]["seconds"] / tol6[name]["seconds"], 3)
    out["paper_tolerance_1e-6"] = tol6
    P.free()
    f = out["fp64_csr_cg"]["seconds"]
    for name in ("gse_stepped_cg_paper_policy", "gse_stepped_cg_floor_policy", "gse_stepped_cg_paper_cg_preset",
                 "gse_stepped_cg_table8"):
        out[name]["speedup_vs_fp64"] = round(f / out[name]["seconds"], 3)
    return out


def gmres_comparison(gse, torch):
    """Stepped GSE-GMRES(30) vs FP64 CSR GMRES(30) on the 2D convection-diffusion
    operator (Peclet 10, upwind), at most 15000 iterations:
      - 256^2 to tol 1e-10, which both reach (the oracle takes 2190 iterations);
      - 1024^2 to tol 1e-10, which neither reaches within the cap (the record
        of where they stall), and then to a residual both reach: 1.2 times the
        larger of the two final residuals (time to a common residual)."""
    pol = gse.Policy(**{**gse.SCALED_GMRES.__dict__, "max_iter": 15000})

    def run(M, b, n, tol, p):
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info = M.gmres(b, x, tol=tol, policy=p)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        return {"seconds": round(dt, 4), "iters": info["iters"], "status": info["status"],
                "k_final": info["k_final"], "switch_iter": info["switch_iter"],
                "rel_res_true": info["rel_res_true"], "max_abs_err_vs_ones": float((x - 1.0).abs().max().item())}

    def pair(N, tol):
        A = synth.convdiff2d(N, 10.0)
        M = gse.GseMatrix.from_csr(A, attach=(64,))
        b = torch.from_numpy(synth.rhs_ones(A)).cuda()
        r = {"fp64_csr_gmres": run(M, b, A.n_rows, tol, gse.fp64_policy(pol)),
             "gse_stepped_gmres_paper_policy": run(M, b, A.n_rows, tol, pol)}
        r["gse_stepped_gmres_paper_policy"]["speedup_vs_fp64"] = round(
            r["fp64_csr_gmres"]["seconds"] / r["gse_stepped_gmres_paper_policy"]["seconds"], 3)
        M.free()
        return r, A

    out = {"max_iter": 15000}
    r256, A = pair(256, 1e-10)
    out["converged_256"] = {"workload": "convdiff2d_256_pe10_gmres30_tol1e-10", "n": A.n_rows, "nnz": A.nnz, **r256}
    r1024, A = pair(1024, 1e-10)
    out["workload"] = "convdiff2d_1024_pe10_gmres30_tol1e-10"
    out["n"], out["nnz"] = A.n_rows, A.nnz
    out.update(r1024)
    common = 1.2 * max(r1024["fp64_csr_gmres"]["rel_res_true"], r1024["gse_stepped_gmres_paper_policy"]["rel_res_true"])
    rc, _ = pair(1024, common)
    out["common_residual_1024"] = {"tol": common, **rc}
    return out


def batched_comparison(gse, torch, nsys, rank, world):
    """nsys SPD systems of uneven size (n log-uniform 1e3..2.56e5, 2D/3D
    anisotropic Laplacians with a diagonal shift) solved to 1e-10 in one
    continuous batch: stepped GSE-CG under the scaled policy, the same with the
    perturbation-floor trigger added, FP64 CSR in the same batched engine, and
    FP64 CSR CG one system at a time (a sample of 32 systems, scaled)."""
    specs = synth.shard_specs(synth.batch_specs(nsys, seed=0), rank, world) if world > 1 else synth.batch_specs(nsys, seed=0)
    t0 = time.perf_counter()
    As = [sp.build() for sp in specs]
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    mats = [gse.GseMatrix.from_csr(A, attach=(64,)) for A in As]
    torch.cuda.synchronize()
    t_enc = time.perf_counter() - t0
    bs = [torch.from_numpy(synth.rhs_ones(A)).cuda() for A in As]
    out = {"workload": f"{len(As)} SPD Laplacians, n log-uniform 1e3..2.56e5, tol 1e-10",
           "systems": len(As), "total_rows": int(sum(A.n_rows for A in As)),
           "total_nnz": int(sum(A.nnz for A in As)), "host_generate_s": round(t_gen, 2),
           "encode_s": round(t_enc, 3)}
    floor = gse.Policy(**{**gse.SCALED_CG.__dict__, "flags": gse.POLICY_FLOOR})
    for name, pol in (("gse_stepped_batched", gse.SCALED_CG), ("gse_stepped_batched_floor", floor),
                      ("fp64_csr_batched", gse.fp64_policy(gse.SCALED_CG))):
        xs = [torch.zeros(A.n_rows, dtype=torch.float64, device="cuda") for A in As]
        gse.batch_cg(mats, bs, xs, tol=1e-10, policy=pol)     # warm (workspaces, floor coefficients)
        for x in xs:
            x.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, infos = gse.batch_cg(mats, bs, xs, tol=1e-10, policy=pol)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        nsolved = len(As)
        if world > 1:                    # whole job: all ranks' systems over the slowest rank's time
            import torch.distributed as tdist
            tm = torch.tensor([dt], device="cuda", dtype=torch.float64)
            tn = torch.tensor([float(len(As))], device="cuda", dtype=torch.float64)
            tdist.all_reduce(tm, op=tdist.ReduceOp.MAX)
            tdist.all_reduce(tn, op=tdist.ReduceOp.SUM)
            dt, nsolved = float(tm.item()), int(tn.item())
        out[name] = {"seconds": round(dt, 4), "solves_per_s": round(nsolved / dt, 2), "status": rc,
                     "all_converged": all(i["status"] == gse.OK for i in infos),
                     "max_iters": max(i["iters"] for i in infos),
                     # sum over systems of rows x iterations: the work the batch does
                     "row_iters": int(sum(A.n_rows * i["iters"] for A, i in zip(As, infos))),
                     "max_rel_res_true": max(i["rel_res_true"] for i in infos)}
    idx = list(range(0, len(As), max(1, len(As) // 32)))[:32]
    t_single = 0.0
    for i in idx:
        x = torch.zeros(As[i].n_rows, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mats[i].cg(bs[i], x, tol=1e-10, policy=gse.fp64_policy(gse.SCALED_CG))
        torch.cuda.synchronize()
        t_single += time.perf_counter() - t0
    est = t_single / len(idx) * len(As)
    out["fp64_csr_one_at_a_time"] = {"seconds_estimated": round(est, 3), "sampled_systems": len(idx),
                                     "solves_per_s": round(len(As) / est, 2)}
    out["speedup_batched_gse_vs_one_at_a_time_fp64"] = round(est / out["gse_stepped_batched"]["seconds"], 2)
    for name in ("gse_stepped_batched", "gse_stepped_batched_floor"):
        g, f = out[name], out["fp64_csr_batched"]
        g["speedup_vs_fp64_batched"] = round(f["seconds"] / g["seconds"], 3)
        g["row_iters_vs_fp64"] = round(g["row_iters"] / f["row_iters"], 3)
    for M in mats:
        M.free()
    return out


def served_benchmark(gse, torch, nreq, rate, rank, world, rate_factors=(0.5,)):
    """Poisson arrivals of nreq solve requests drawn from the batched
    distribution (a pool of 64 systems), admitted by HBM footprint into a
    continuous batch; p50/p99 latency from arrival to completion.  One run per
    arrival rate factor (times the saturated batch throughput `rate`); the
    first factor's run is reported at the top level, all of them in `sweep`,
    and the 1x stream once more under SCALED_CG + the floor rule."""
    from paper_2411_04686_gb300 import serve
    specs = synth.batch_specs(64, seed=1)
    pool = []
    for sp in specs:
        A = sp.build()
        pool.append((A, synth.rhs_ones(A)))
    sweep = []
    for f in rate_factors:
        sweep.append(_served_run(gse, serve, pool, nreq, rate * f, rank, world))
        sweep[-1]["rate_factor"] = f
    out = dict(sweep[0])
    out["sweep"] = sweep
    # the same arrival stream at 1x under SCALED_CG + the floor rule, which does
    # less work per system (row-iterations 1.13x FP64's instead of 1.69x)
    floor = gse.Policy(**{**gse.SCALED_CG.__dict__, "flags": gse.POLICY_FLOOR})
    out["floor_policy_1x"] = _served_run(gse, serve, pool, nreq, rate, rank, world, policy=floor)
    # one-at-a-time FP64 CSR CG throughput on the same pool (8 systems)
    t_single = 0.0
    for A, b in pool[:8]:
        M = gse.GseMatrix.from_csr(A, attach=(64,))
        bd = torch.from_numpy(b).cuda()
        x = torch.zeros(A.n_rows, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        M.cg(bd, x, tol=1e-10, policy=gse.fp64_policy(gse.SCALED_CG))
        torch.cuda.synchronize()
        t_single += time.perf_counter() - t1
        M.free()
    out["fp64_one_at_a_time_solves_per_s"] = round(8 / t_single, 2)
    return out


def _served_run(gse, serve, pool, nreq, rate, rank, world, policy=None):
    arrivals = serve.poisson_arrivals(nreq, rate, seed=2)
    rng = np.random.default_rng(3)
    picks = rng.integers(0, len(pool), nreq)
    reqs = [serve.Request(i, float(arrivals[i]), pool[picks[i]][0].n_rows, pool[picks[i]][0].nnz, int(picks[i]))
            for i in range(nreq)]
    if world > 1:
        reqs = serve.shard(reqs, rank, world)
    srv = serve.Server(lambda i: pool[i], capacity=64, slots_per_step=16, backlog_slots_per_step=32, policy=policy)
    t0 = time.perf_counter()
    srv.clock = lambda: time.perf_counter() - t0
    k = 0
    while k < len(reqs) or srv.queue or srv.active:
        now = srv.clock()
        while k < len(reqs) and reqs[k].arrival <= now:
            srv.submit(reqs[k])
            k += 1
        if not srv.queue and not srv.active and k < len(reqs):
            time.sleep(max(0.0, min(0.01, reqs[k].arrival - now)))
            continue
        srv.step()
    wall = srv.clock()
    srv.close()
    st = serve.latency_stats(srv.done)
    ok = all(c.info["status"] == gse.OK for c in srv.done)
    return {"requests": len(reqs), "arrival_rate_per_s": round(rate, 2), "wall_s": round(wall, 3),
            "solves_per_s": round(len(srv.done) / wall, 2), "p50_latency_s": round(st.get("p50_s", 0), 4),
            "p99_latency_s": round(st.get("p99_s", 0), 4), "all_converged": ok}


if __name__ == "__main__":
    main()
