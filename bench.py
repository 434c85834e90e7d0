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
FP64_FLOPS_PER_CLK_SM = 4  # 1.25 TFLOP/s nominal FP64 / (152 SMs x 2.07 GHz) ~= 4 (2 DFMA per clock)
FP32_OPS_PER_CLK_SM = 128  # FP32 pipe lanes per SM: one arithmetic instruction per lane per clock
NUM_SMS = 152
PAIR_EVAL_FLOPS = 9        # FP64: squared distance (8) + reciprocal square root (1) per kernel entry
DD_EVAL_OPS = 54           # double-float: FP32 instructions of one 1/|x-y| entry (difference, square, rsqrt + Newton)
DD_MAC_OPS = 12            # double-float: FP32 instructions of one error-free multiply-accumulate
# DRAM bytes of one double-float coupling launch (3D 1/r, N = 2^18, 16 RHS,
# 6.099e9 entries) from ncu (profiles/ksum_dd_coupling_3d_invr_262144.md);
# scaled to other sizes by the entries of the launch
DD_COUPLING_TRAFFIC = (53.189376e6 + 13.053952e6, 6099084090)
F32_EVAL_OPS = 14          # FP32: two-float difference (9), squared distance (3), rsqrt + select (2)
# digit-split coupling: FP32-pipe instructions per entry -- the double-float
# 1/|x-y| of an admissible pair (43) and its split into six digits with their
# packing to bf16 (23); the 21 digit products per entry and column run on the
# tensor cores (mma.sync m16n8k16) and are not counted
OZ_EVAL_OPS = 43 + 23
OZ_PRODUCTS = 21
# DRAM bytes of one digit-split coupling launch (3D 1/r, N = 2^18, 16 RHS,
# 6.099e9 entries) from ncu (profiles/ksum_oz_coupling_3d_invr_262144.md)
OZ_COUPLING_TRAFFIC = (73.693184e6 + 20.957184e6, 6099084090)


def _coupling_choice(sm, nrhs):
    """Which double-float coupling ran: the tuner's record (0 digit split on
    the tensor cores, 1 all on the FP32 pipe), else the untuned default (the
    digit split from 8 columns per pass)."""
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


def run_cpu_oracle(n: int, w: dict) -> dict:
    import oracle
    x = si.uniform_cube(n, w["d"], w["index"] * 1000 + 7)
    q = si.rhs(n, w["nrhs"], w["index"] * 1000 + 8)
    t0 = time.perf_counter()
    h = oracle.H2(x, w["kernel"], w["leaf"], w["order"], w["tol"])
    h.matvec(q)
    dt = time.perf_counter() - t0
    return {"value": n / dt, "seconds": dt}


def run_serving(sm, torch, requests: int, rate: float, seed: int, precision: int, max_inflight: int = 4) -> dict:
    """Poisson stream of construct-and-apply requests shaped like the serving
    configuration (1D Cauchy-like kernel 1/(x_i - y_j), x ~ U[0,1],
    y = x + 1e-3 U, N log-uniform in [2^12, 2^20], leaf 64, order 16,
    tol 1e-10, 1..64 right-hand sides), served by the library's request
    server and, for comparison, one request at a time by the plain path with
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
    nbuf = min(requests, 4 * max_inflight)
    for _ in range(nbuf):
        pool.put(torch.empty(nmax * 64, dtype=torch.float64).pin_memory())

    # warm the kernels and the pools once
    srv = sm.SmashServer(max_inflight=max_inflight, precision=precision)
    srv.wait(srv.submit(xp[:4096], kid, leaf, order, tol, Xs[0][:0].new_empty((4096, 1)).fill_(1.0),
                        y=yp[:4096]))

    lat, done_at = [None] * requests, [None] * requests
    t0 = time.perf_counter()
    tickets = [None] * requests
    held = [None] * requests

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
        tickets[i] = srv.submit(xp[:n], kid, leaf, order, tol, Xs[i], y=yp[:n], Y=held[i][: n * k].view(n, k))
    th.join()
    makespan = max(done_at)
    seen = srv.max_inflight_seen()
    srv.close()
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
        "served": {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                   "points_per_s": pts / makespan, "max_inflight": max_inflight, "max_inflight_seen": seen,
                   "latency": "completion minus scheduled arrival"},
        "plain_one_at_a_time": {"p50_ms": float(np.percentile(plain_lat, 50)),
                                "p99_ms": float(np.percentile(plain_lat, 99)),
                                "points_per_s": pts / plain_makespan},
    }


def run_batched(sm, torch, dev, steps: int = 2, warmup: int = 1, reps: int = 10) -> dict:
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

    def step():
        ts = [threading.Thread(target=one, args=(d,)) for d in ds]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
        torch.cuda.synchronize()
        if errors:
            raise errors[0]

    times = []
    for i in range(warmup + steps):
        if i >= warmup:
            sm.smash_set_autotune(False)
        for h in handles.values():
            sm.smash_free(h)
        handles.clear()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step()
        if i >= warmup:
            times.append(time.perf_counter() - t0)
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
        "ms_per_step": 1e3 * med, "steps": steps, "timing": "host wall clock around the synchronous builds",
        "per_dimension": {str(d): {"problems": info[d]["nproblems"], "points": info[d]["nx"],
                                   "levels": info[d]["levels"], "nodes": info[d]["nnodes"]} for d in ds},
        "resident_apply_ms": {"smash_matvec_ex": plain[0], "smash_matvec_graph": graph[0],
                              "note": "both batches, FP32, 8 RHS, mean of %d applies" % reps},
    }


def run_mixed(sm, torch, dev, reps: int = 2) -> dict:
    """The sphere configuration (2^20 points on S^2 with 8 caps, Yukawa, leaf
    128, order 5, 32 RHS): the FP64 build, then the matvec in every precision
    on the same representation.  Errors are relative 2-norms against the
    FP64 matvec of the same build (which agrees with the oracle's H^2 matvec
    to <= 1e-11)."""
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
    sm.smash_set_profiling(False)
    info = sm.smash_info(h)
    sm.smash_free(h)
    return {"workload": "sphere_yukawa_1m: 2^20 points on S^2 (90% uniform, 10% in 8 caps, sigma 0.02), "
                        "exp(-r)/r, leaf 128, order 5, tol 1e-8, 32 RHS",
            "build_ms": build_ms, "coupling_entries": info["coupling_pairs"], "near_entries": info["near_pairs"],
            "precisions": res,
            "note": "tf32/bf16/tf32x3: coupling products on the tensor cores (warp MMAs), near field FP32 "
                    "with compensated sums; errors against the FP64 matvec of the same build"}


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
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"3d_invr uniform cube, N={REF_SAMPLE_N} sample of the N=2^20 recipe",
                   "leaf": w["leaf"], "order": w["order"], "tol": w["tol"], "nrhs": w["nrhs"]},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"N={REF_SAMPLE_N} points per step, build + one {w['nrhs']}-RHS matvec"},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def bench_ours(args, w):
    import torch
    import paper_1705_05443_gb300 as sm

    ws, rank = _dist()
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

    prec = {"f32x2": sm.SMASH_PREC_F32X2, "f64": sm.SMASH_PREC_F64, "f32": sm.SMASH_PREC_F32,
            "tf32": sm.SMASH_PREC_TF32, "bf16": sm.SMASH_PREC_BF16, "tf32x3": sm.SMASH_PREC_TF32X3}[args.precision]

    def step(host=False, precision=prec):
        if host:
            h = sm.smash_build_xy(xh, None, w["kernel"], w["leaf"], w["order"], w["tol"], stream=stream)
            sm.smash_matvec_ex(h, qh, zh, precision, stream=stream)
        else:
            h = sm.smash_build_xy(x, None, w["kernel"], w["leaf"], w["order"], w["tol"], stream=stream)
            sm.smash_matvec_ex(h, q, z, precision, stream=stream)
        return h

    sm.smash_set_profiling(True)
    # the first warm-up step times the candidate launch shapes of every tuned
    # site (autotuner); later steps use the recorded choices
    sm.smash_set_autotune(args.autotune)
    for _ in range(args.warmup):
        sm.smash_free(step())
        sm.smash_set_autotune(False)
    torch.cuda.synchronize()
    tune_entries = sm.smash_autotune_entries()
    info = None
    coupling_ms, step_ms = [], []
    sampler = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = sm.smash_launch_count()
    sampler.start()
    wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h = step()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        prof = sm.smash_last_profile(h)
        coupling_ms.append(prof["coupling"])
        if info is None:
            info = sm.smash_info(h)
            phases = prof
        sm.smash_free(h)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    clocks = sampler.stop()
    launches = sm.smash_launch_count() - launches0
    if dist:
        dist.barrier()
    value, tot_ms = replica_value(sum(step_ms), n, args.steps, dist, dev)

    # end to end through the same C ABI with pinned host buffers
    xh = torch.from_numpy(x_np).pin_memory()
    qh = torch.from_numpy(q_np).pin_memory()
    zh = torch.empty(q_np.shape, dtype=torch.float64).pin_memory()
    sm.smash_free(step(host=True))
    torch.cuda.synchronize()
    e2e_t = []
    for _ in range(max(1, min(args.steps, 3))):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = step(host=True)
        torch.cuda.synchronize()
        e2e_t.append(time.perf_counter() - t0)
        sm.smash_free(h)
    e2e_val = ws * n / statistics.median(e2e_t)

    # context: the same step with the FP64 matvec, and the agreement of the two
    fp64_ms = None
    parity = None
    if prec != sm.SMASH_PREC_F64:
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h = step(precision=sm.SMASH_PREC_F64)
        e1.record(stream)
        e1.synchronize()
        fp64_ms = e0.elapsed_time(e1)
        z64 = z.clone()
        sm.smash_matvec_ex(h, q, z, prec, stream=stream)
        torch.cuda.synchronize()
        parity = float(torch.linalg.norm(z - z64) / torch.linalg.norm(z64))
        sm.smash_free(h)
    sm.smash_set_profiling(False)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    peaks, peak_src = _peaks()
    sm_mhz = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    nrhs = w["nrhs"]
    cpl_ms = statistics.mean(coupling_ms)
    if prec == sm.SMASH_PREC_F64:
        peak = NUM_SMS * FP64_FLOPS_PER_CLK_SM * sm_mhz * 1e6 / 1e12
        cpl_work = info["coupling_pairs"] * (2 * nrhs + PAIR_EVAL_FLOPS)
        kname = "coupling (ksum_f64_kernel over L)"
        psrc = (f"FP64 {FP64_FLOPS_PER_CLK_SM} flop/clk/SM x {NUM_SMS} SMs x {sm_mhz:.0f} MHz "
                "(nominal unit count, sampled clock; an FMA probe measured 1.19 TFLOP/s)")
        wdef = f"per kernel entry 2*nrhs + {PAIR_EVAL_FLOPS} FP64 flops"
    elif prec in (sm.SMASH_PREC_TF32, sm.SMASH_PREC_BF16, sm.SMASH_PREC_TF32X3):
        # the products run on the tensor pipe; the FP32 pipe evaluates the entries
        cvt = {sm.SMASH_PREC_TF32: 1, sm.SMASH_PREC_BF16: 1, sm.SMASH_PREC_TF32X3: 3}[prec]
        peak = NUM_SMS * FP32_OPS_PER_CLK_SM * sm_mhz * 1e6 / 1e12
        cpl_work = info["coupling_pairs"] * (F32_EVAL_OPS + cvt)
        kname = "coupling (ksum_tc_kernel over L, entries on the FP32 pipe, products on the tensor cores)"
        psrc = (f"FP32 pipe {FP32_OPS_PER_CLK_SM} instructions/clk/SM x {NUM_SMS} SMs x {sm_mhz:.0f} MHz "
                "(the entry evaluation bounds this kernel; ncu: tensor pipe < 10 % active)")
        wdef = (f"per kernel entry {F32_EVAL_OPS} FP32 instructions of the entry + {cvt} rounding to the "
                "product format; the MMA products are not counted")
    elif prec == sm.SMASH_PREC_F32:
        peak = NUM_SMS * FP32_OPS_PER_CLK_SM * sm_mhz * 1e6 / 1e12
        cpl_work = info["coupling_pairs"] * (nrhs + F32_EVAL_OPS)
        kname = "coupling (ksum_f32_kernel over L)"
        psrc = (f"FP32 pipe {FP32_OPS_PER_CLK_SM} instructions/clk/SM x {NUM_SMS} SMs x {sm_mhz:.0f} MHz "
                "(one FMA = one operation)")
        wdef = f"per kernel entry nrhs FMAs + {F32_EVAL_OPS} FP32 instructions (difference, distance, kernel)"
    elif _coupling_choice(sm, nrhs) == 0 and nrhs <= 16 and info["levels"] <= 10:
        peak = NUM_SMS * FP32_OPS_PER_CLK_SM * sm_mhz * 1e6 / 1e12
        cpl_work = info["coupling_pairs"] * OZ_EVAL_OPS
        kname = ("coupling (ksum_oz_kernel over L: double-float entries split into 8-bit digits on the FP32 "
                 "pipe, exact digit products on the tensor cores)")
        psrc = (f"FP32 pipe {FP32_OPS_PER_CLK_SM} instructions/clk/SM x {NUM_SMS} SMs x {sm_mhz:.0f} MHz "
                "(one FMA = one operation)")
        wdef = (f"per kernel entry {OZ_EVAL_OPS} FP32-pipe instructions (double-float 1/|x-y| and its six-digit "
                f"split); the {OZ_PRODUCTS}*nrhs digit products per entry run as mma.sync and are not counted")
    else:
        peak = NUM_SMS * FP32_OPS_PER_CLK_SM * sm_mhz * 1e6 / 1e12
        cpl_work = info["coupling_pairs"] * (DD_MAC_OPS * nrhs + DD_EVAL_OPS)
        kname = "coupling (ksum_dd_kernel over L, double-float on the FP32 pipe)"
        psrc = (f"FP32 pipe {FP32_OPS_PER_CLK_SM} instructions/clk/SM x {NUM_SMS} SMs x {sm_mhz:.0f} MHz "
                "(one FMA = one operation)")
        wdef = (f"per kernel entry {DD_MAC_OPS}*nrhs + {DD_EVAL_OPS} FP32 instructions of the "
                "double-float algorithm (error-free products and sums)")
    achieved = cpl_work / (cpl_ms / 1e3) / 1e12
    traffic = None
    if prec == sm.SMASH_PREC_F32X2 and args.workload == "3d_invr_1m":
        tr = DD_COUPLING_TRAFFIC if kname.startswith("coupling (ksum_dd") else OZ_COUPLING_TRAFFIC
        traffic = tr[0] * info["coupling_pairs"] / tr[1]
    mixed = run_mixed(sm, torch, dev) if args.mixed else None
    batched = None
    if args.batched:
        sm.smash_set_autotune(args.autotune)
        batched = run_batched(sm, torch, dev)
        sm.smash_set_autotune(False)
    serving = None
    if args.serve_requests > 0:
        serving = run_serving(sm, torch, args.serve_requests, 200.0, 4000, prec)
    cpu = run_cpu_oracle(CPU_SAMPLE_N, w) if not args.no_cpu_baseline else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {sm.SMASH_PREC_F32X2: "f32x2", sm.SMASH_PREC_F64: "f64", sm.SMASH_PREC_F32: "f32",
                  sm.SMASH_PREC_TF32: "tf32", sm.SMASH_PREC_BF16: "bf16", sm.SMASH_PREC_TF32X3: "tf32x3"}[prec],
        "data": "synthetic",
        "config": {"workload": (args.workload if args.workload != "3d_invr_1m" else "3d_invr uniform cube N=2^20")
                   + ("" if n == 1 << 20 else f" at N={n}"),
                   "n": n, "dim": w["d"], "kernel": {0: "log|x-y|", 1: "1/|x-y|", 2: "exp(-|x-y|)/|x-y|",
                                                     3: "1/(x-y)"}[w["kernel"]],
                   "leaf": w["leaf"], "order": w["order"], "tol": w["tol"], "nrhs": nrhs, "tau": 0.7,
                   "precision": "build fp64; matvec " + {sm.SMASH_PREC_F64: "fp64",
                                                          sm.SMASH_PREC_F32X2: "double-float kernel sums and transfers; coupling and near-field products as exact 8-bit digit products on the tensor cores",
                                                          sm.SMASH_PREC_F32: "fp32 kernel sums, fp64 transfers",
                                                          sm.SMASH_PREC_TF32: "tf32 coupling products, fp32 near field",
                                                          sm.SMASH_PREC_BF16: "bf16 coupling products, fp32 near field",
                                                          sm.SMASH_PREC_TF32X3: "split-tf32 coupling products, "
                                                                                "fp32 near field"}[prec],
                   "l2": "flushed (256 MiB write) before every timed step",
                   "parallelism": f"replicas{ws}"},
        "roofline": {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "traffic_source": None if traffic is None else
                     "ncu dram__bytes_read+write of the N=2^18 launch, scaled by kernel entries",
                     "peak_source": psrc, "work_definition": wdef,
                     "work_per_launch": cpl_work, "ms_per_launch": cpl_ms},
        "fp64_matvec_step": None if fp64_ms is None else {"ms_per_step": fp64_ms, "value": ws * n / (fp64_ms / 1e3)},
        "rel_diff_vs_fp64_matvec": parity,
        "phases_ms": phases,
        "structure": {k: info[k] for k in ("levels", "nnodes", "nadm", "nnear", "skel_row", "g_row",
                                           "coupling_pairs", "near_pairs", "swaps")},
        "e2e": {"value": e2e_val, "unit": UNIT,
                "h2d_bytes_per_step": int(x_np.nbytes + q_np.nbytes), "d2h_bytes_per_step": int(q_np.nbytes)},
        "gpu_launches": int(launches / args.steps),
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
                                          f"{nrhs}-RHS matvec, serial C oracle"}
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
    ap.add_argument("--serve-requests", type=int, default=200,
                    help="requests of the serving measurement (0 = skip)")
    ap.add_argument("--precision", default="f32x2", choices=["f32x2", "f64", "f32", "tf32", "bf16", "tf32x3"],
                    help="matvec arithmetic: double-float kernel sums (FP64-accurate), plain FP64, or "
                         "mixed precision FP32")
    ap.add_argument("--no-batched", dest="batched", action="store_false",
                    help="skip the batched-trees measurement")
    ap.add_argument("--no-mixed", dest="mixed", action="store_false",
                    help="skip the sphere mixed-precision measurement")
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
