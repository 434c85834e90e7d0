"""Benchmark: SMASH H^2 build + matvec throughput (points/s) on one GB300.

A step is one pass of the whole path over one point cloud: the adaptive
tree, the interaction lists, the per-level compression (basis + strong RRQR
/ ID) and one H^2 matvec with nrhs right-hand sides.  The default workload is
the 3D 1/|x-y| problem at N = 2^20 uniform points in the unit cube, leaf
<= 128, 4 interpolation points per axis, RRQR tol 1e-8, 16 RHS, FP64.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs its own independent replica of the
workload (the path has no exchange step), timings are max-reduced and rank 0
prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import smash_inputs as si  # noqa: E402

METRIC = "build+matvec points/s, 3D 1/r N=2^20 at <=1e-8 rel err"
UNIT = "points/s"
CPU_SAMPLE_N = 32768      # oracle sample for cpu_baseline (same recipe, ~10-30 s of CPU work)
REF_SAMPLE_N = 16384      # oracle sample per step of the reference arm
NUM_SMS = 152
# nominal unit counts per SM and clock (the derived ALU peaks): FP32 pipe one
# FMA per lane per clock on 128 lanes, FP64 about 1.25 TFLOP/s per GPU, i.e.
# 2 DFMA per clock per SM at 2.07 GHz
FP32_FLOPS_PER_CLK_SM = 2 * 128
FP64_FLOPS_PER_CLK_SM = 4
# algorithmic work of one kernel entry of the coupling (3.19) and the near
# field (3.20): the squared distance and kernel (about 10 flops and one
# special function) plus one multiply-add per right-hand side
ENTRY_FLOPS = 10
# DRAM bytes of one digit-split coupling launch (3D 1/r, N = 2^18, 16 RHS,
# 6.099e9 entries), read and write, from an ncu capture of that launch;
# scaled to other sizes by the entries of the launch
OZ_COUPLING_TRAFFIC = (72.571648e6 + 20.937216e6, 6099084090)
DD_COUPLING_TRAFFIC = (53.189376e6 + 13.053952e6, 6099084090)
OZ5_COUPLING_TRAFFIC = (73.001728e6 + 18.445568e6, 6099084090)   # the tcgen05 form, same launch
COUPLING_NAMES = {0: "digit split, warp MMAs", 1: "double-float on the FP32 pipe", 2: "digit split, tcgen05.mma"}
HEADLINE_ORACLE_LEAVES = 64   # leaves of the headline compared with the oracle's H^2 matvec
DENSE_ROWS = 1024             # rows compared with the dense product (O1)
SWEEP_N = 65536               # order sweep: the 3D 1/r configuration's small size
SWEEP_ORDERS = (2, 3, 4, 5, 6, 7, 8)
HSS_N = 1 << 16               # HSS block: points of the serving configuration's recipe


def nvtx_range(start: bool, name: str = "smash_timed_steps") -> None:
    """Open or close the NVTX range around the timed steps (a no-op where
    PyTorch was built without NVTX)."""
    try:
        import torch

        if start:
            torch.cuda.nvtx.range_push(name)
        else:
            torch.cuda.nvtx.range_pop()
    except Exception:  # pragma: no cover
        pass

def _coupling_choice(sm, nrhs, pinned="auto"):
    """Which double-float coupling ran: the pinned variant, else the tuner's
    record (0 digit split by warp MMAs, 1 all on the FP32 pipe, 2 digit split
    by tcgen05.mma), else the untuned default (the digit split from 8 columns
    per pass)."""
    if pinned != "auto":
        return {"warp": 0, "fp32": 1, "tcgen05": 2}[pinned]
    import json
    import tempfile
    with tempfile.NamedTemporaryFile(suffix=".json") as f:
        sm.smash_autotune_save(f.name)  # raises on failure
        with open(f.name) as fh:
            entries = json.load(fh).get("entries", {})
    vals = [v for k, v in entries.items() if k.startswith("coupling_dd/")]
    if vals:
        return vals[0]
    ldq = 1 << max(0, (nrhs - 1).bit_length()) if nrhs <= 32 else 32 * ((nrhs + 31) // 32)
    return 0 if ldq >= 8 else 1


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


def replica_value(local_total_ms: float, n_per_rank: int, steps: int, dist=None, device=None):
    """Whole-job throughput of independent replicas (one per rank): all ranks'
    points over the slowest rank's time.  Returns (value, max total ms)."""
    import torch
    tot = float(local_total_ms)
    ws = 1
    if dist is not None:
        ws = dist.get_world_size()
        t = torch.tensor([tot], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot = float(t.item())
    return ws * n_per_rank * steps / (tot / 1e3), tot


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def cpu_info() -> dict:
    """Host cores and CPU model of this machine."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"nproc": os.cpu_count(), "model": model}


def run_cpu_oracle(n: int, w: dict) -> dict:
    import oracle
    x = si.uniform_cube(n, w["d"], w["index"] * 1000 + 7)
    q = si.rhs(n, w["nrhs"], w["index"] * 1000 + 8)
    t0 = time.perf_counter()
    h = oracle.H2(x, w["kernel"], w["leaf"], w["order"], w["tol"])
    h.matvec(q)
    dt = time.perf_counter() - t0
    return {"value": n / dt, "seconds": dt}


_CPU_CHILD = r"""
import json, os, sys, time
sys.path.insert(0, sys.argv[1])
import oracle, smash_inputs as si
n, d, kid, leaf, order, tol, nrhs, index = json.loads(sys.argv[2])
x = si.uniform_cube(n, d, index * 1000 + 7)
q = si.rhs(n, nrhs, index * 1000 + 8)
t0 = time.perf_counter()
h = oracle.H2(x, kid, leaf, order, tol)
h.matvec(q)
print(json.dumps({"seconds": time.perf_counter() - t0, "openmp": oracle.openmp()}))
"""


def run_cpu_oracle_threads(n: int, w: dict, threads: int) -> dict:
    """The oracle's -fopenmp build (same bits as the serial one: node and row
    loops on `threads` host threads) on the same sample, in a child process."""
    env = dict(os.environ, ORACLE_OPENMP="1", OMP_NUM_THREADS=str(threads))
    spec = json.dumps([n, w["d"], w["kernel"], w["leaf"], w["order"], w["tol"], w["nrhs"], w["index"]])
    out = subprocess.run([sys.executable, "-c", _CPU_CHILD, ROOT, spec], env=env, capture_output=True, text=True,
                         check=True, timeout=900).stdout
    r = json.loads(out.strip().splitlines()[-1])
    assert r["openmp"]
    return {"value": n / r["seconds"], "seconds": r["seconds"], "threads": threads}


# ---------------------------------------------------------------- oracle jobs
# Run in spawned worker processes while the GPU is measured: each rebuilds its
# inputs from the seeded generators and returns only the oracle's numbers.

def _job_init(threads: int):
    """Worker set-up: the oracle's -fopenmp build on `threads` host threads
    (it computes the same bits as the serial build)."""
    os.environ["ORACLE_OPENMP"] = "1"
    os.environ["OMP_NUM_THREADS"] = str(threads)


def _leaf_rows(e, leaves):
    return np.concatenate([e["permx"][e["rs"][g]:e["rs"][g] + e["rc"][g]] for g in leaves])


def job_oracle_rows(name: str, nleaves: int, ndense: int, seed: int, min_rows: int = 0) -> dict:
    """The oracle's H^2 matvec and its row scales (sums of |terms|) on the
    rows of at least `nleaves` random leaves (more until they hold `min_rows`
    points), and the dense product (O1) on `ndense` sampled rows, for a named
    workload."""
    import oracle
    w = si.make_workload(name)
    x, q = w["x"], w["q"]
    t0 = time.perf_counter()
    ho = oracle.H2(x, w["kernel"], w["leaf"], w["order"], w["tol"])
    e = ho.export()
    leaves = np.flatnonzero(e["leaf"])
    order = np.random.default_rng(seed).permutation(leaves)
    cnt = np.cumsum(e["rc"][order])
    take = max(min(nleaves, len(order)), int(np.searchsorted(cnt, min_rows)) + 1 if min_rows else 0)
    pick = np.sort(order[:min(take, len(order))]).astype(np.int32)
    rows = _leaf_rows(e, pick)
    out = {"rows": rows, "zo": ho.matvec_leaves(q, pick)[rows], "sc": ho.matvec_abs(q, pick)[rows],
           "leaves": len(pick)}
    if ndense:
        drows = si.sample_rows(len(x), ndense, seed + 1)
        out["drows"] = drows
        out["zd"] = oracle.dense_rows(x, w["kernel"], q, rows=drows)
    out["seconds"] = time.perf_counter() - t0
    return out


def job_sweep_dense(n: int, nrhs: int, nrows: int, seed: int) -> dict:
    """Dense rows (O1) of the order sweep's 3D 1/r problem."""
    import oracle
    x = si.uniform_cube(n, 3, seed)
    q = si.rhs(n, nrhs, seed + 1)
    rows = si.sample_rows(n, nrows, seed + 2)
    return {"rows": rows, "zd": oracle.dense_rows(x, si.KERNEL_INVR, q, rows=rows)}


def entry_errors(z_rows: np.ndarray, zo: np.ndarray, sc: np.ndarray) -> dict:
    """Worst |z - z_o| / (sum of |terms|) over the entries, and the relative
    2-norm, of GPU rows against the oracle's rows."""
    d = np.abs(z_rows - zo)
    ratio = np.where(sc > 0, d / np.where(sc > 0, sc, 1.0), np.where(d == 0, 0.0, np.inf))
    return {"worst_entry_vs_sum_abs_terms": float(ratio.max()),
            "rel_2norm": float(np.linalg.norm(z_rows - zo) / np.linalg.norm(zo)), "rows": int(len(zo))}


def build_flops(ranks: dict, r: int, d: int) -> float:
    """Algorithmic FP64 work of the compression: per node with a working set
    of m points and rank k, the basis m r (d + 1), the QR with column
    pivoting 4 r m k - 2 k^2 (r + m) + 4 k^3 / 3 and the ID k^2 (m - k)."""
    m = ranks["m"].astype(np.float64)
    k = ranks["k"].astype(np.float64)
    sel = m > 0
    m, k = m[sel], k[sel]
    qr = 4 * r * m * k - 2 * k * k * (r + m) + 4 * k ** 3 / 3
    return float(np.sum(m * r * (d + 1) + np.maximum(qr, 0) + k * k * (m - k)))


def pass_bytes(ranks: dict, ldq: int) -> float:
    """HBM bytes of one upward (or downward) pass: G ((m - k) k doubles) and
    the vectors (m in, k out, ldq doubles each) of every node."""
    m = ranks["m"].astype(np.float64)
    k = ranks["k"].astype(np.float64)
    return float(np.sum(8.0 * (m - k) * k + 8.0 * ldq * (m + k)))


def rooflines(info, ranks, prof, nrhs, ldq, peaks, prec, sm) -> dict:
    """Achieved work rate of each kernel phase against its bound, in the
    algorithmic units of the method (not implementation instructions)."""
    fp32, fp64, hbm = peaks["fp32_tflops"], peaks["fp64_tflops"], peaks["hbm_gbs"]
    entry = ENTRY_FLOPS + 2 * nrhs
    ksum_peak, ksum_src = (fp64, "fp64") if prec == sm.SMASH_PREC_F64 else (fp32, "fp32")
    out = {}

    def alu(name, work, ms, peak, src, what):
        a = work / (ms / 1e3) / 1e12
        out[name] = {"bound": "alu", "achieved": a, "peak": peak, "unit": "TFLOP/s", "frac": a / peak,
                     "peak_kind": src, "work_per_launch": work, "ms": ms, "work_definition": what}

    alu("coupling", info["coupling_pairs"] * entry, prof["coupling"], ksum_peak, ksum_src,
        f"sum over L of k_i k_j kernel entries x ({ENTRY_FLOPS} + 2 nrhs) flops")
    alu("near_field", info["near_pairs"] * entry, prof["near"], ksum_peak, ksum_src,
        f"sum over L^- of |i| |j| kernel entries x ({ENTRY_FLOPS} + 2 nrhs) flops")
    alu("compression", build_flops(ranks, info["r"], info["dim"]), prof["compression"], fp64, "fp64",
        "basis m r (d+1) + QRCP 4rmk - 2k^2(r+m) + 4k^3/3 + ID k^2(m-k) FP64 flops per node")
    for name in ("upward", "downward"):
        b = pass_bytes(ranks, ldq)
        a = b / (prof[name] / 1e3) / 1e9
        out[name] = {"bound": "hbm", "achieved": a, "peak": hbm, "unit": "GB/s", "frac": a / hbm,
                     "work_per_launch": b, "ms": prof[name],
                     "work_definition": "8 (m-k) k bytes of G + 8 ldq (m + k) bytes of vectors per node"}
    return out


def run_serving(sm, torch, requests: int, rate: float, seed: int, precision: int,
                budgets_gib=(2, 8, 32), slots: int = 16) -> dict:
    """Poisson stream of construct-and-apply requests shaped like the serving
    configuration (1D Cauchy-like kernel 1/(x_i - y_j), x ~ U[0,1],
    y = x + 1e-3 U, N log-uniform in [2^12, 2^20], leaf 64, order 16,
    tol 1e-10, 1..64 right-hand sides), served by the library's request
    server at several device-memory budgets (the budget, not the slot count,
    decides how many requests overlap: `slots` worker streams are always
    there) and, for comparison, one request at a time by the plain path with
    the same arrival times.  Inputs are prefixes of pinned host pools."""
    g = np.random.default_rng(seed)
    nmax = 1 << 20
    xp = torch.from_numpy(g.random((nmax, 1))).pin_memory()
    yp = (xp + 1e-3 * torch.from_numpy(g.random((nmax, 1)))).pin_memory()
    Xp = torch.from_numpy(g.standard_normal(nmax * 64)).pin_memory()
    arrivals = np.cumsum(g.exponential(1.0 / rate, size=requests))
    sizes = np.floor(2.0 ** g.uniform(12, 20, size=requests)).astype(int)
    nrhs = g.integers(1, 65, size=requests)
    Xs = [Xp[: int(n) * int(k)].view(int(n), int(k)) for n, k in zip(sizes, nrhs)]
    leaf, order, tol, kid = 64, 16, 1e-10, sm.SMASH_K_CAUCHY1D
    # outputs: a pool of pinned buffers, taken at submission and returned when
    # the request has completed; when all are taken the client waits, and the
    # latency below runs from the scheduled arrival, so that wait counts
    import queue
    pool = queue.Queue()
    nbuf = min(requests, 2 * slots)
    for _ in range(nbuf):
        pool.put(torch.empty(nmax * 64, dtype=torch.float64).pin_memory())
    predicted = [sm.smash_predict_footprint(int(n), 1, leaf, order, int(k)) for n, k in zip(sizes, nrhs)]

    def served(budget_bytes):
        srv = sm.SmashServer(max_inflight=slots, mem_budget_bytes=budget_bytes, precision=precision)
        # warm the kernels and the pools once
        srv.wait(srv.submit(xp[:4096], kid, leaf, order, tol, Xs[0][:0].new_empty((4096, 1)).fill_(1.0),
                            y=yp[:4096]))
        lat, done_at = [None] * requests, [None] * requests
        tickets = [None] * requests
        held = [None] * requests
        t0 = time.perf_counter()

        def waiter():
            for i in range(requests):
                while tickets[i] is None:
                    time.sleep(0.0002)
                srv.wait(tickets[i])
                done_at[i] = time.perf_counter() - t0
                lat[i] = (done_at[i] - arrivals[i]) * 1e3
                pool.put(held[i])
                held[i] = None

        th = threading.Thread(target=waiter)
        th.start()
        for i in range(requests):
            dt = arrivals[i] - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            n, k = int(sizes[i]), int(nrhs[i])
            held[i] = pool.get()
            tickets[i] = srv.submit(xp[:n], kid, leaf, order, tol, Xs[i], y=yp[:n],
                                    Y=held[i][: n * k].view(n, k))
        th.join()
        seen = srv.max_inflight_seen()
        srv.close()
        return {"budget_gib": budget_bytes / 2 ** 30, "p50_ms": float(np.percentile(lat, 50)),
                "p99_ms": float(np.percentile(lat, 99)), "points_per_s": float(sizes.sum()) / max(done_at),
                "max_inflight_seen": seen, "slots": slots}

    runs = [served(int(b * 2 ** 30)) for b in budgets_gib]
    Yplain = pool.get()
    # one request at a time, same arrival times
    plain_lat = []
    t0 = time.perf_counter()
    for i in range(requests):
        now = time.perf_counter() - t0
        if arrivals[i] > now:
            time.sleep(arrivals[i] - now)
        n = int(sizes[i])
        h = sm.smash_build_xy(xp[:n], yp[:n], kid, leaf, order, tol)
        sm.smash_matvec_ex(h, Xs[i], Yplain[: n * int(nrhs[i])].view(n, int(nrhs[i])), precision)
        sm.smash_free(h)
        plain_lat.append((time.perf_counter() - t0 - arrivals[i]) * 1e3)
    plain_makespan = time.perf_counter() - t0
    pts = float(sizes.sum())
    return {
        "workload": f"{requests} requests, Poisson {rate:.0f}/s, 1D Cauchy-like, N log-uniform 2^12..2^20, "
                    "leaf 64, order 16, tol 1e-10, 1-64 RHS",
        "predicted_footprint_gib": {"median": float(np.median(predicted)) / 2 ** 30,
                                    "max": float(np.max(predicted)) / 2 ** 30},
        "served": runs,
        "latency": "completion minus scheduled arrival",
        "plain_one_at_a_time": {"p50_ms": float(np.percentile(plain_lat, 50)),
                                "p99_ms": float(np.percentile(plain_lat, 99)),
                                "points_per_s": pts / plain_makespan},
    }


def run_batched(sm, torch, dev, steps: int = 3, warmup: int = 1, reps: int = 10) -> dict:
    """The batched-trees workload: 512 independent problems (2D log and 3D
    1/r, uniform or Gaussian-mixture clouds), one batch representation per
    dimension built concurrently on two streams, then the FP32 matvec with 8
    RHS of each.  A step is both builds plus both matvecs; points/s counts
    every point of every problem.  Also times repeated applies of the built
    batches through smash_matvec_ex and through the CUDA-graph replay."""
    import threading
    wl = si.make_workload("batched_512")
    groups = wl["groups"]
    ds = sorted(groups)
    xs = {d: torch.from_numpy(groups[d][0]).to(dev) for d in ds}
    qs = {d: torch.from_numpy(wl["q"][d]).to(dev) for d in ds}
    zs = {d: torch.empty_like(qs[d]) for d in ds}
    streams = {d: torch.cuda.Stream(dev) for d in ds}
    handles = {}
    errors = []

    def one(d):
        try:
            x, off, kid, _ = groups[d]
            h = sm.smash_build_batch(xs[d], off, kid, wl["leaf"], wl["order"], wl["tol"], stream=streams[d])
            sm.smash_matvec_ex(h, qs[d], zs[d], sm.SMASH_PREC_F32, stream=streams[d])
            handles[d] = h
        except Exception as e:  # reported by the caller
            errors.append(e)

    main = torch.cuda.Stream(dev)

    def step():
        """Both builds and matvecs; device time from an event on `main` that
        both streams wait for to the later of their end events."""
        e0 = torch.cuda.Event(enable_timing=True)
        ends = {d: torch.cuda.Event(enable_timing=True) for d in ds}
        e0.record(main)
        for d in ds:
            streams[d].wait_event(e0)
        ts = [threading.Thread(target=one, args=(d,)) for d in ds]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
        for d in ds:
            ends[d].record(streams[d])
        torch.cuda.synchronize()
        if errors:
            raise errors[0]
        return max(e0.elapsed_time(ends[d]) for d in ds)

    times = []
    phases = {}
    sm.smash_set_profiling(True)
    for i in range(warmup + steps):
        if i >= warmup:
            sm.smash_set_autotune(False)
        for h in handles.values():
            sm.smash_free(h)
        handles.clear()
        torch.cuda.synchronize()
        ms = step()
        if i >= warmup:
            times.append(ms / 1e3)
            for d in ds:
                prof = sm.smash_last_profile(handles[d])
                for k, v in prof.items():
                    phases.setdefault(str(d), {}).setdefault(k, []).append(v)
    sm.smash_set_profiling(False)
    n = wl["n"]
    info = {d: sm.smash_info(handles[d]) for d in ds}
    # repeated applies of the resident batches
    s = streams[ds[0]]
    plain, graph = [], []
    for mode, out in (("plain", plain), ("graph", graph)):
        for d in ds:
            fn = sm.smash_matvec_ex if mode == "plain" else sm.smash_matvec_graph
            fn(handles[d], qs[d], zs[d], sm.SMASH_PREC_F32, stream=s)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(reps):
            for d in ds:
                fn = sm.smash_matvec_ex if mode == "plain" else sm.smash_matvec_graph
                fn(handles[d], qs[d], zs[d], sm.SMASH_PREC_F32, stream=s)
        e1.record(s)
        e1.synchronize()
        out.append(e0.elapsed_time(e1) / reps)
    for h in handles.values():
        sm.smash_free(h)
    med = statistics.median(times)
    return {
        "workload": "batched_512: 512 problems, N log-uniform in [1024, 32768], 2D log|x-y| / 3D 1/|x-y|, "
                    "uniform cube or 4-component Gaussian mixture (sigma 0.1), leaf 64, order 4, tol 1e-8, "
                    "FP64 build, FP32 matvec with 8 RHS",
        "problems": int(sum(info[d]["nproblems"] for d in ds)), "points": int(n),
        "value": n / med, "unit": "points/s (build + FP32 matvec of all problems)",
        "ms_per_step": 1e3 * med, "steps": steps,
        "timing": "CUDA events: from an event both build streams wait for to the later stream's end event",
        "phases_ms": {d: {k: statistics.median(v) for k, v in ph.items()} for d, ph in phases.items()},
        "per_dimension": {str(d): {"problems": info[d]["nproblems"], "points": info[d]["nx"],
                                   "levels": info[d]["levels"], "nodes": info[d]["nnodes"]} for d in ds},
        "resident_apply_ms": {"smash_matvec_ex": plain[0], "smash_matvec_graph": graph[0],
                              "note": "both batches, FP32, 8 RHS, mean of %d applies" % reps},
    }


def run_mixed(sm, torch, dev, orc=None, reps: int = 2) -> dict:
    """The sphere configuration (2^20 points on S^2 with 8 caps, Yukawa, leaf
    128, order 5, 32 RHS): the FP64 build, then the matvec in every precision
    on the same representation.  Errors: relative 2-norms against the FP64
    matvec of the same build on all rows, and, with `orc` (the oracle's rows,
    job_oracle_rows), against the FP64 oracle's H^2 matvec on the rows of
    its sampled leaves: worst entry over its sum of |terms| and 2-norm."""
    w = si.make_workload("sphere_yukawa_1m")
    x = torch.from_numpy(w["x"]).to(dev)
    q = torch.from_numpy(w["q"]).to(dev)
    z = torch.empty_like(q)
    st = torch.cuda.Stream(dev)

    def timed(fn, keep_last=True):
        """Best of `reps` runs of fn on stream st; for builds (keep_last) the
        handles of all runs but the last are freed."""
        best, out = None, None
        for i in range(reps):
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            out = fn()
            e1.record(st)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None or ms < best else best
            if keep_last and i < reps - 1:
                sm.smash_free(out)
        return best, out

    sm.smash_set_profiling(True)
    build_ms, h = timed(lambda: sm.smash_build_xy(x, None, w["kernel"], w["leaf"], w["order"], w["tol"],
                                                  stream=st))
    names = {"f64": sm.SMASH_PREC_F64, "f32": sm.SMASH_PREC_F32, "tf32": sm.SMASH_PREC_TF32,
             "bf16": sm.SMASH_PREC_BF16, "tf32x3": sm.SMASH_PREC_TF32X3}
    res = {}
    z64 = None
    for name, p in names.items():
        ms, _ = timed(lambda: sm.smash_matvec_ex(h, q, z, p, stream=st), keep_last=False)
        prof = sm.smash_last_profile(h)
        if p == sm.SMASH_PREC_F64:
            z64 = z.clone()
            err = 0.0
        else:
            err = float(torch.linalg.norm(z - z64) / torch.linalg.norm(z64))
        res[name] = {"matvec_ms": ms, "coupling_ms": prof["coupling"], "near_ms": prof["near"],
                     "rel_err_vs_fp64": err,
                     "build_plus_matvec_points_per_s": w["n"] / ((build_ms + ms) / 1e3)}
        if orc is not None:
            rows_t = torch.from_numpy(orc["rows"]).to(dev)
            res[name]["vs_fp64_oracle"] = entry_errors(z.index_select(0, rows_t).cpu().numpy(), orc["zo"],
                                                       orc["sc"])
    sm.smash_set_profiling(False)
    info = sm.smash_info(h)
    sm.smash_free(h)
    return {"workload": "sphere_yukawa_1m: 2^20 points on S^2 (90% uniform, 10% in 8 caps, sigma 0.02), "
                        "exp(-r)/r, leaf 128, order 5, tol 1e-8, 32 RHS",
            "build_ms": build_ms, "coupling_entries": info["coupling_pairs"], "near_entries": info["near_pairs"],
            "precisions": res,
            "oracle_rows": None if orc is None else {"rows": int(len(orc["rows"])), "leaves": orc["leaves"],
                                                     "seconds": orc["seconds"]},
            "note": "tf32/bf16/tf32x3: coupling products on the tensor cores (warp MMAs), near field FP32 "
                    "with compensated sums; errors against the FP64 matvec of the same build (all rows) and "
                    "against the FP64 oracle on the rows of sampled leaves"}


TABLE_6_1 = {1600: (6.69e-13, 0.52, 0.02), 6400: (2.00e-12, 1.97, 0.07), 25600: (3.65e-12, 9.53, 0.30),
             102400: (4.87e-12, 39.47, 1.18)}   # n: (relative error, t_constr s, t_matvec s), MATLAB, Section 6.2


def job_taylor_dense(sizes, nrows: int, seed: int) -> dict:
    """Dense rows of kappa (2.1) on C (d_x = 1) times u ~ U[0,1] on the m x m
    grids of Section 6.2 (the oracle's O1)."""
    import oracle
    out = {}
    for n in sizes:
        m = int(round(n ** 0.5))
        x = si.grid_2d(m)
        u = si.uniform_01(n, 1, seed).astype(np.complex128)
        rows = si.sample_rows(n, nrows, seed + 1)
        out[n] = {"rows": rows, "zd": oracle.dense_rows_taylor(x, u, rows=rows)}
    return out


def run_taylor(sm, torch, dev, dense: dict, seed: int, reps: int = 3) -> dict:
    """The workload of Table 6.1 (Section 6.2): kappa (2.1) on C with d_x = 1
    on an m x m grid in [0,1]^2, leaves of at most 50 points, the Taylor
    basis (2.4) with r = 22 terms, tau = 0.65, one vector u ~ U[0,1]: GPU
    build and matvec times (CUDA events, best of `reps`), the error against
    the dense product on sampled rows, and the paper's MATLAB times beside."""
    st = torch.cuda.Stream(dev)
    res = []
    for n, (p_err, p_c, p_m) in TABLE_6_1.items():
        m = int(round(n ** 0.5))
        x = torch.from_numpy(si.grid_2d(m)).to(dev)
        u = torch.from_numpy(si.uniform_01(n, 1, seed).astype(np.complex128)).to(dev)
        y = torch.empty_like(u)
        tb, tm = [], []
        for _ in range(reps):
            torch.cuda.synchronize()
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(st)
            h = sm.smash_build_taylor(x, 50, 22, tau=0.65, tol=1e-14, dx=1.0)
            e1.record(st)
            sm.smash_matvec_complex(h, u, y, stream=st)
            e2.record(st)
            e2.synchronize()
            tb.append(e0.elapsed_time(e1))
            tm.append(e1.elapsed_time(e2))
            info = sm.smash_info(h)
            sm.smash_free(h)
        d = dense[n]
        zr = y.cpu().numpy()[d["rows"]]
        err = float(np.linalg.norm(zr - d["zd"]) / np.linalg.norm(d["zd"]))
        res.append({"n": n, "build_ms": min(tb), "matvec_ms": min(tm), "rel_err_vs_dense": err,
                    "levels": info["levels"], "skeleton_points": info["skel_row"],
                    "paper": {"rel_err": p_err, "t_constr_s": p_c, "t_matvec_s": p_m}})
    return {"workload": "Section 6.2 / Table 6.1: 1/(x-y) on C, d_x = 1, m x m grid in [0,1]^2, leaf <= 50, "
                        "Taylor basis r = 22, tau = 0.65, u ~ U[0,1]; FP64 complex",
            "timing": "CUDA events on the build stream (the build is synchronous, so build_ms includes its host "
                      "orchestration); best of %d" % reps,
            "paper_hardware": "MATLAB R2014b, MacBook Air 1.6 GHz, 8 GB (context only)",
            "sizes": res}


def job_hss_dense(n: int, nrhs: int, nrows: int, seed: int) -> dict:
    """Dense rows (O1) of the Cauchy kernel on the HSS block's points."""
    import oracle
    x, y = si.cauchy_1d(n, seed)
    q = si.rhs(n, nrhs, seed + 1)
    rows = si.sample_rows(n, nrows, seed + 2)
    return {"rows": rows, "zd": oracle.dense_rows(x, si.KERNEL_CAUCHY, q, rows=rows, y=y)}


def run_hss(sm, torch, dev, dense: dict, n: int, seed: int, reps: int = 2) -> dict:
    """HSS construction (Section 3.3.1) for the serving configuration's points
    (x ~ U[0,1], y = x + 1e-3 U(0,1), kernel 1/(x - y)), leaf 32, order 16,
    tol 1e-12, eps_svd 1e-10, tau 0.6, 4 right-hand sides: build and FP64
    matvec times and the error against the dense product on sampled rows."""
    x, y = si.cauchy_1d(n, seed)
    q = si.rhs(n, 4, seed + 1)
    xd, yd, qd = (torch.from_numpy(a).to(dev) for a in (x, y, q))
    z = torch.empty_like(qd)
    st = torch.cuda.Stream(dev)
    tb, tm = [], []
    for _ in range(reps):
        torch.cuda.synchronize()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(st)
        h = sm.smash_build_hss(xd, yd, sm.SMASH_K_CAUCHY1D, 32, 16, 1e-12, 1e-10, tau=0.6, stream=st)
        e1.record(st)
        sm.smash_matvec_ex(h, qd, z, sm.SMASH_PREC_F64, stream=st)
        e2.record(st)
        e2.synchronize()
        tb.append(e0.elapsed_time(e1))
        tm.append(e1.elapsed_time(e2))
        info = sm.smash_info(h)
        svd = sm.smash_export_hss(h)
        sm.smash_free(h)
    zr = z.cpu().numpy()[dense["rows"]]
    err = float(np.linalg.norm(zr - dense["zd"]) / np.linalg.norm(dense["zd"]))
    return {"workload": f"HSS, 1/(x-y), N={n}, x ~ U[0,1], y = x + 1e-3 U(0,1), leaf 32, order 16, tol 1e-12, "
                        "eps_svd 1e-10, tau 0.6, 4 RHS, FP64",
            "build_ms": min(tb), "matvec_ms": min(tm), "points_per_s": n / ((min(tb) + min(tm)) / 1e3),
            "rel_err_vs_dense": err, "levels": info["levels"], "ranks_row": info["skel_row"],
            "max_singular_vectors": int(max(svd["svd_row"].max(), svd["svd_col"].max())),
            "max_nearfield_nodes": int(np.diff(svd["nf_ptr"]).max())}


def run_order_sweep(sm, torch, dev, dense: dict, tol: float = 1e-8) -> dict:
    """Error against the dense product (O1 rows) as the interpolation order
    rises, 3D 1/r on SWEEP_N uniform points, leaf 128: the smallest order
    whose FP64 H^2 matvec is within 1e-8 of dense on the sampled rows.  The
    library allows order^3 <= 512, i.e. orders up to 8 in 3D."""
    x = torch.from_numpy(si.uniform_cube(SWEEP_N, 3, 9100)).to(dev)
    q = torch.from_numpy(si.rhs(SWEEP_N, 4, 9101)).to(dev)
    z = torch.empty_like(q)
    rows_t = torch.from_numpy(dense["rows"]).to(dev)
    out = []
    for p in SWEEP_ORDERS:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = sm.smash_build_xy(x, None, sm.SMASH_K_INVR, 128, p, tol)
        sm.smash_matvec_ex(h, q, z, sm.SMASH_PREC_F64)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        info = sm.smash_info(h)
        zr = z.index_select(0, rows_t).cpu().numpy()
        err = float(np.linalg.norm(zr - dense["zd"]) / np.linalg.norm(dense["zd"]))
        out.append({"order": p, "r": p ** 3, "rel_err_vs_dense": err, "skeleton_points": info["skel_row"],
                    "coupling_entries": info["coupling_pairs"], "build_plus_matvec_s": dt})
        sm.smash_free(h)
    hit = [o["order"] for o in out if o["rel_err_vs_dense"] <= 1e-8]
    return {"workload": f"3D 1/|x-y|, N={SWEEP_N} uniform cube, leaf 128, tol {tol:g}, 4 RHS, FP64; "
                        f"{len(dense['rows'])} sampled rows against the dense product",
            "orders": out, "smallest_order_at_1e-8": hit[0] if hit else None}


def bench_reference(args, w):
    ws, rank = _dist()
    if rank != 0:
        return
    import oracle
    oracle.build()
    for _ in range(args.warmup):
        run_cpu_oracle(REF_SAMPLE_N, w)
    t = []
    for _ in range(args.steps):
        t.append(run_cpu_oracle(REF_SAMPLE_N, w)["seconds"])
    total = sum(t)
    val = REF_SAMPLE_N * args.steps / total
    host = cpu_info()
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"3d_invr uniform cube, N={REF_SAMPLE_N} sample of the N=2^20 recipe",
                   "leaf": w["leaf"], "order": w["order"], "tol": w["tol"], "nrhs": w["nrhs"]},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"N={REF_SAMPLE_N} points per step, build + one {w['nrhs']}-RHS matvec",
                         "nproc": host["nproc"], "cpu_model": host["model"]},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


PREC_NAMES = {"f32x2": 1, "f64": 0, "f32": 2, "tf32": 3, "bf16": 4, "tf32x3": 5}
PREC_TEXT = {
    0: "fp64",
    1: "double-float kernel sums and transfers; coupling and near-field products as exact 8-bit digit products "
       "on the tensor cores",
    2: "fp32 kernel sums, fp64 transfers",
    3: "tf32 coupling products, fp32 near field",
    4: "bf16 coupling products, fp32 near field",
    5: "split-tf32 coupling products, fp32 near field",
}
DTYPE = {0: "f64", 1: "f32x2", 2: "f32", 3: "tf32", 4: "bf16", 5: "tf32x3"}


def bench_ours(args, w):
    ws, rank = _dist()
    # oracle work for the error columns runs in spawned processes (started
    # before any CUDA call) while the GPU is measured
    pool, jobs = None, {}
    if rank == 0 and args.oracle_checks:
        import multiprocessing as mp
        pool = mp.get_context("spawn").Pool(3, initializer=_job_init, initargs=(4,))
        if args.workload == "3d_invr_1m" and w["n"] == 1 << 20:
            jobs["headline"] = pool.apply_async(job_oracle_rows, ("3d_invr_1m", HEADLINE_ORACLE_LEAVES,
                                                                  DENSE_ROWS, 9000))
        if args.mixed:
            jobs["sphere"] = pool.apply_async(job_oracle_rows, ("sphere_yukawa_1m", 64, 0, 9200, 4096))
        if args.sweep:
            jobs["sweep"] = pool.apply_async(job_sweep_dense, (SWEEP_N, 4, 256, 9100))
        if args.taylor:
            jobs["taylor"] = pool.apply_async(job_taylor_dense, (tuple(TABLE_6_1), 512, 9300))
        if args.hss:
            jobs["hss"] = pool.apply_async(job_hss_dense, (HSS_N, 4, 512, 9400))

    import torch
    import paper_1705_05443_gb300 as sm

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    sm.load_library()
    n = w["n"]
    wl = si.make_workload(args.workload, rep=rank, n=n)
    x_np, q_np = wl["x"], wl["q"]
    x = torch.from_numpy(x_np).to(dev)
    q = torch.from_numpy(q_np).to(dev)
    z = torch.empty_like(q)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    # a dedicated stream: the library runs build and matvec on it and the
    # timing events are recorded on it (the default stream's handle is NULL,
    # which the C ABI reads as "the handle's own stream")
    stream = torch.cuda.Stream(dev)
    torch.cuda.synchronize()
    prec = PREC_NAMES[args.precision]
    nrhs = w["nrhs"]
    ldq = 1 << max(0, (nrhs - 1).bit_length()) if nrhs <= 32 else 32 * ((nrhs + 31) // 32)

    def step(host=False, precision=prec, out=None):
        if host:
            h = sm.smash_build_xy(xh, None, w["kernel"], w["leaf"], w["order"], w["tol"], stream=stream)
            sm.smash_matvec_ex(h, qh, zh, precision, stream=stream)
        else:
            h = sm.smash_build_xy(x, None, w["kernel"], w["leaf"], w["order"], w["tol"], stream=stream)
            sm.smash_matvec_ex(h, q, z if out is None else out, precision, stream=stream)
        return h

    def timed_steps(k, precision, out=None):
        """k device-timed steps; returns (per-step ms, profile and info of the first)."""
        ms, first = [], None
        for _ in range(k):
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h = step(precision=precision, out=out)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            if first is None:
                first = (sm.smash_last_profile(h), sm.smash_info(h), sm.smash_node_ranks(h))
            sm.smash_free(h)
        return ms, first

    if args.coupling != "auto":
        sm.smash_autotune_force("coupling_dd/", {"warp": 0, "fp32": 1, "tcgen05": 2}[args.coupling])
    sm.smash_set_profiling(True)
    # the first warm-up step times the candidate launch shapes of every tuned
    # site (autotuner); later steps use the recorded choices
    sm.smash_set_autotune(args.autotune)
    for _ in range(args.warmup):
        sm.smash_free(step())
        sm.smash_set_autotune(False)
    torch.cuda.synchronize()
    tune_entries = sm.smash_autotune_entries()
    sampler = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = sm.smash_launch_count()
    sampler.start()
    wall0 = time.perf_counter()
    nvtx_range(True)  # lets a profiler keep only the timed steps' launches
    step_ms, (phases, info, ranks) = timed_steps(args.steps, prec)
    torch.cuda.synchronize()
    nvtx_range(False)
    wall = time.perf_counter() - wall0
    clocks = sampler.stop()
    launches = sm.smash_launch_count() - launches0
    if dist:
        dist.barrier()
    value, tot_ms = replica_value(sum(step_ms), n, args.steps, dist, dev)
    z_head = z.clone()

    # end to end through the same C ABI with pinned host buffers
    xh = torch.from_numpy(x_np).pin_memory()
    qh = torch.from_numpy(q_np).pin_memory()
    zh = torch.empty(q_np.shape, dtype=torch.float64).pin_memory()

    def e2e(precision, reps):
        sm.smash_free(step(host=True, precision=precision))
        torch.cuda.synchronize()
        t = []
        for _ in range(reps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            hh = sm.smash_build_xy(xh, None, w["kernel"], w["leaf"], w["order"], w["tol"], stream=stream)
            sm.smash_matvec_ex(hh, qh, zh, precision, stream=stream)
            torch.cuda.synchronize()
            t.append(time.perf_counter() - t0)
            sm.smash_free(hh)
        return ws * n / statistics.median(t)

    e2e_val = e2e(prec, max(1, min(args.steps, 3)))

    # the same step with the FP64 matvec (the paper's arithmetic), timed the same way
    fp64 = None
    z64 = None
    if prec != sm.SMASH_PREC_F64 and args.fp64:
        sm.smash_free(step(precision=sm.SMASH_PREC_F64))
        k64 = max(1, min(args.steps, 3))
        z64 = torch.empty_like(q)
        ms64, (ph64, info64, ranks64) = timed_steps(k64, sm.SMASH_PREC_F64, out=z64)
        fp64 = {"ms_per_step": statistics.mean(ms64), "steps": k64,
                "value": ws * n / (statistics.mean(ms64) / 1e3), "unit": UNIT, "dtype": "f64",
                "phases_ms": ph64,
                "e2e": {"value": e2e(sm.SMASH_PREC_F64, 1), "unit": UNIT,
                        "h2d_bytes_per_step": int(x_np.nbytes + q_np.nbytes),
                        "d2h_bytes_per_step": int(q_np.nbytes)}}
    elif prec == sm.SMASH_PREC_F64:
        z64 = z_head
    sm.smash_set_profiling(False)
    parity = None if z64 is None or prec == sm.SMASH_PREC_F64 else \
        float(torch.linalg.norm(z_head - z64) / torch.linalg.norm(z64))

    # peaks: nominal unit counts at the sampled clock (the roofline
    # denominators) and the library's FMA-chain probe of this device
    peaks_file, peak_src = _peaks()
    sm_mhz = clocks.get("sm_mhz") or peaks_file.get("sm_max_mhz", 2070.0)
    peaks = {"fp32_tflops": NUM_SMS * FP32_FLOPS_PER_CLK_SM * sm_mhz * 1e6 / 1e12,
             "fp64_tflops": NUM_SMS * FP64_FLOPS_PER_CLK_SM * sm_mhz * 1e6 / 1e12,
             "hbm_gbs": float(peaks_file["hbm_gbs"]),
             "fp32_tflops_probe": sm.smash_measure_fma_peak(False),
             "fp64_tflops_probe": sm.smash_measure_fma_peak(True),
             "source": f"FP32 {FP32_FLOPS_PER_CLK_SM} and FP64 {FP64_FLOPS_PER_CLK_SM} flop/clk/SM x {NUM_SMS} "
                       f"SMs x {sm_mhz:.0f} MHz (sampled clock); HBM from MEASURED_PEAKS.json ({peak_src}); "
                       "probes: smash_measure_fma_peak in this run"}
    roofs = rooflines(info, ranks, phases, nrhs, ldq, peaks, prec, sm)
    if fp64 is not None:
        fp64["rooflines"] = rooflines(info64, ranks64, ph64, nrhs, ldq, peaks, sm.SMASH_PREC_F64, sm)
    cpl = dict(roofs["coupling"])
    traffic = None
    if prec == sm.SMASH_PREC_F32X2 and args.workload == "3d_invr_1m":
        choice = _coupling_choice(sm, nrhs, args.coupling)
        tr = {0: OZ_COUPLING_TRAFFIC, 1: DD_COUPLING_TRAFFIC, 2: OZ5_COUPLING_TRAFFIC}[choice]
        traffic = tr[0] * info["coupling_pairs"] / tr[1]
        cpl["variant"] = COUPLING_NAMES[choice]
    roofline = {"bound": "alu", "kernel": "coupling over L (3.19)" + (f", {cpl['variant']}" if "variant" in cpl else ""),
                "achieved": cpl["achieved"],
                "peak": cpl["peak"], "unit": "TFLOP/s", "frac": cpl["frac"], "traffic": traffic,
                "traffic_source": None if traffic is None else
                "ncu dram__bytes_read+write of the N=2^18 launch, scaled by kernel entries",
                "peak_source": peaks["source"], "work_definition": cpl["work_definition"],
                "work_per_launch": cpl["work_per_launch"], "ms_per_launch": cpl["ms"]}

    # the other configurations, the ones with oracle columns last so that the
    # spawned oracle work overlaps the GPU work before them
    sweep = None
    if args.sweep and "sweep" in jobs:
        sweep = run_order_sweep(sm, torch, dev, jobs["sweep"].get())
    batched = None
    if args.batched:
        sm.smash_set_autotune(args.autotune)
        batched = run_batched(sm, torch, dev)
        sm.smash_set_autotune(False)
    serving = None
    if args.serve_requests > 0:
        serving = run_serving(sm, torch, args.serve_requests, 200.0, 4000, prec)
    taylor = run_taylor(sm, torch, dev, jobs["taylor"].get(), 9300) if "taylor" in jobs else None
    hss = run_hss(sm, torch, dev, jobs["hss"].get(), HSS_N, 9400) if "hss" in jobs else None
    mixed = None
    if args.mixed:
        orc = jobs["sphere"].get() if "sphere" in jobs else None
        mixed = run_mixed(sm, torch, dev, orc)

    # errors of the headline (and FP64) step against the oracle and dense
    errors = None
    if "headline" in jobs:
        o = jobs["headline"].get()
        rows_t = torch.from_numpy(o["rows"]).to(dev)
        drows_t = torch.from_numpy(o["drows"]).to(dev)
        errors = {"oracle_rows": {"rows": int(len(o["rows"])), "leaves": o["leaves"], "seconds": o["seconds"]},
                  "dense_rows": int(len(o["drows"]))}
        for tag, zz in (("headline", z_head), ("fp64", z64)):
            if zz is None:
                continue
            zr = zz.index_select(0, rows_t).cpu().numpy()
            zd = zz.index_select(0, drows_t).cpu().numpy()
            errors[tag] = {"vs_oracle": entry_errors(zr, o["zo"], o["sc"]),
                           "rel_err_vs_dense": float(np.linalg.norm(zd - o["zd"]) / np.linalg.norm(o["zd"]))}
    if pool is not None:
        pool.close()
        pool.join()

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    host = cpu_info()
    cpu = run_cpu_oracle(CPU_SAMPLE_N, w) if not args.no_cpu_baseline else None
    cpu_mt = None
    if cpu and args.openmp_baseline:
        cpu_mt = run_cpu_oracle_threads(CPU_SAMPLE_N, w, host["nproc"] or 1)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE[prec],
        "data": "synthetic",
        "config": {"workload": (args.workload if args.workload != "3d_invr_1m" else "3d_invr uniform cube N=2^20")
                   + ("" if n == 1 << 20 else f" at N={n}"),
                   "n": n, "dim": w["d"], "kernel": {0: "log|x-y|", 1: "1/|x-y|", 2: "exp(-|x-y|)/|x-y|",
                                                     3: "1/(x-y)"}[w["kernel"]],
                   "leaf": w["leaf"], "order": w["order"], "tol": w["tol"], "nrhs": nrhs, "tau": 0.7,
                   "precision": "build fp64; matvec " + PREC_TEXT[prec],
                   "coupling": args.coupling,
                   "l2": "flushed (256 MiB write) before every timed step",
                   "parallelism": f"replicas{ws}"},
        "roofline": roofline,
        "rooflines": roofs,
        "peaks": peaks,
        "fp64": fp64,
        "errors": errors,
        "rel_diff_vs_fp64_matvec": parity,
        "phases_ms": phases,
        "structure": {k: info[k] for k in ("levels", "nnodes", "nadm", "nnear", "skel_row", "g_row",
                                           "coupling_pairs", "near_pairs", "swaps")},
        "e2e": {"value": e2e_val, "unit": UNIT,
                "h2d_bytes_per_step": int(x_np.nbytes + q_np.nbytes), "d2h_bytes_per_step": int(q_np.nbytes)},
        "gpu_launches": int(launches),  # library kernels launched in the timed region (all K steps)
        "gpu_launches_per_step": int(launches / args.steps),
        "order_sweep": sweep,
        "taylor_table_6_1": taylor,
        "hss": hss,
        "serving": serving,
        "batched": batched,
        "mixed_precision": mixed,
        "autotune": {"enabled": bool(args.autotune), "entries_after_warmup": tune_entries,
                     "entries": sm.smash_autotune_entries()},
        "clocks": clocks,
        "wall_s": wall,
        "peaks_file": peak_src,
    }
    if cpu:
        line["cpu_baseline"] = {"value": cpu["value"], "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"N={CPU_SAMPLE_N} points of the same recipe, build + one "
                                          f"{nrhs}-RHS matvec, serial C oracle",
                                "nproc": host["nproc"], "cpu_model": host["model"],
                                "openmp": None if cpu_mt is None else
                                {"value": cpu_mt["value"], "threads": cpu_mt["threads"],
                                 "sample": "the same sample, the oracle built with -fopenmp (node and row loops "
                                           "on all host threads; same bits as the serial build)"}}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="3d_invr_1m")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n", type=int, default=None, help="point count (same recipe); for profiling cases")
    ap.add_argument("--serve-requests", type=int, default=400,
                    help="requests of the serving measurement (0 = skip)")
    ap.add_argument("--precision", default="f32x2", choices=list(PREC_NAMES),
                    help="matvec arithmetic: double-float kernel sums (FP64-accurate), plain FP64, or "
                         "mixed precision FP32")
    ap.add_argument("--no-batched", dest="batched", action="store_false",
                    help="skip the batched-trees measurement")
    ap.add_argument("--no-mixed", dest="mixed", action="store_false",
                    help="skip the sphere mixed-precision measurement")
    ap.add_argument("--no-fp64", dest="fp64", action="store_false",
                    help="skip the FP64 step beside the headline")
    ap.add_argument("--no-sweep", dest="sweep", action="store_false", help="skip the order sweep")
    ap.add_argument("--no-taylor", dest="taylor", action="store_false",
                    help="skip the Taylor-basis (Table 6.1) measurement")
    ap.add_argument("--no-hss", dest="hss", action="store_false", help="skip the HSS measurement")
    ap.add_argument("--no-oracle-checks", dest="oracle_checks", action="store_false",
                    help="skip the oracle and dense error columns (spawned CPU processes)")
    ap.add_argument("--no-openmp-baseline", dest="openmp_baseline", action="store_false",
                    help="skip the multi-threaded oracle run of the CPU baseline")
    ap.add_argument("--coupling", default="auto", choices=["auto", "warp", "tcgen05", "fp32"],
                    help="pin the double-float coupling: digit products by warp MMAs or by tcgen05.mma, "
                         "or every operation on the FP32 pipe (default: the tuner's choice)")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="use the default launch shapes instead of tuning them in the first warm-up step")
    args = ap.parse_args()
    w = dict(si.WORKLOADS[args.workload])
    if args.n:
        w["n"] = args.n
    if args.impl == "reference":
        bench_reference(args, w)
    else:
        bench_ours(args, w)


if __name__ == "__main__":
    main()
