#!/usr/bin/env python3
"""Benchmark: Trotter site-steps/s of the second-order Trotter-Suzuki step.

Workload (one "step" of this benchmark): the 8192 x 8192 FP32 roofline grid
(32 seed-placed Gaussians in V, one seed-random packet), run through the
whole hot path: table preparation from V (FP64 -> rounded FP32 tables),
200 second-order Trotter steps on the fused temporally blocked kernel, and
the FP64-compensated observables.  Inputs (8 B/site state + 8 B/site V) live
in HBM when the timed region starts; the 1.6 GB working set is larger than
L2, so no flush is needed between steps.

``value`` = grid sites x Trotter steps x ranks / wall time of the timed steps
(CUDA events, max over ranks).  ``e2e`` = the same through the C ABI with
pinned host buffers (host->device of state and V, device->host of the result
state and observables inside the timed region).

``--impl reference`` times the FP64 CPU oracle on this host's cores on a
bounded sample of the same workload.  Multi-GPU runs are independent
replicas (no collective in the data path; the method needs none on one GPU).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Trotter site-steps/s"
UNIT = "site-steps/s"
TROTTER_STEPS = 200
BYTES_PER_SITE_LAUNCH = 24      # read re, im, gamma_V, s_V; write re, im (FP32)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=8192, help="grid side")
    ap.add_argument("--K", type=int, default=0, help="fused depth (0 = library default)")
    ap.add_argument("--trotter-steps", type=int, default=TROTTER_STEPS)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-serve", action="store_true", help="skip the serving workload")
    ap.add_argument("--no-precision", action="store_true",
                    help="skip the FP32 / FP64 path comparison")
    ap.add_argument("--no-k-sweep", action="store_true",
                    help="skip the depth sweep (K = 1..8 at 8192^2 and 16384^2, plain paths)")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the accuracy block (FP64 oracle on the host: ~1-2 minutes)")
    ap.add_argument("--no-adjoint", action="store_true",
                    help="skip the adjoint timing (1024^2 x 500 and 4096^2 x 200 steps)")
    ap.add_argument("--serve-requests", type=int, default=512)
    ap.add_argument("--n3", type=int, default=512, help="side of the 3-D lattice in --variants")
    ap.add_argument("--only", choices=["order4", "drive", "3d"], default=None,
                    help="with --variants: run one variant (default depth) only")
    ap.add_argument("--variants", action="store_true",
                    help="time fourth-order steps and a time-dependent potential instead "
                         "(prints its own JSON line)")
    ap.add_argument("--adjoint", action="store_true",
                    help="time only the adjoint on one --adj-n^2 grid (--adj-steps, --adj-ckpt; "
                         "backward depth --K, 0 = depths 1..4; --steps runs each)")
    ap.add_argument("--traffic", action="store_true",
                    help="launch the fused kernel once per depth 1..8 on each --traffic-n side "
                         "(after one warm-up launch each), for an ncu DRAM-traffic capture")
    ap.add_argument("--traffic-n", type=int, nargs="+", default=[8192, 16384])
    ap.add_argument("--adj-n", type=int, default=1024)
    ap.add_argument("--adj-steps", type=int, default=500)
    ap.add_argument("--adj-ckpt", type=int, default=50)
    ap.add_argument("--paper", action="store_true",
                    help="time the paper's single-node sizes instead (L = 24576 FP32, "
                         "17472 FP64, flat V, ten iterations)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (replicas only)
# ---------------------------------------------------------------------------
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Dist:
    def __init__(self, world, local, backend):
        self.world = world
        self.pg = None
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group(backend=backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, v: float) -> float:
        if not self.pg:
            return v
        import torch
        dev = "cuda" if torch.cuda.is_available() else "cpu"
        t = torch.tensor([v], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


def replica_throughput(dist: "Dist", site_steps_per_rank: float, elapsed_s: float) -> float:
    """Whole-job throughput of independent replicas: every rank did the same
    amount of work; the job took as long as the slowest rank."""
    return site_steps_per_rank * dist.world / dist.max(elapsed_s)


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for n, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------
def oracle_sample(n: int, seed: int, budget_s: float = 12.0, max_steps: int = 10):
    """Time the FP64 oracle on the n x n workload with all host cores: one
    step to calibrate, then as many steps (<= 10, the paper's ten
    iterations) as fit the budget.  Returns (site-steps/s, cores, sample)."""
    import oracle
    from paper_1208_2407_gb300 import workloads as wl
    cores = os.cpu_count() or 1
    c = wl.roofline_grid(n=n, seed=seed, steps=1)
    re, im, V = c["re"], c["im"], c["V"]
    t0 = time.perf_counter()
    re, im = oracle.evolve(re, im, V, c["dt"], c["theta"], 1, nthreads=cores)
    t1 = time.perf_counter() - t0
    steps = int(max(1, min(max_steps, budget_s / max(t1, 1e-9))))
    t0 = time.perf_counter()
    oracle.evolve(re, im, V, c["dt"], c["theta"], steps, nthreads=cores)
    dt = time.perf_counter() - t0
    rate = n * n * steps / dt
    return rate, cores, "%dx%d FP64 oracle, %d Trotter steps (of the %d per step), %d threads" % (
        n, n, steps, TROTTER_STEPS, cores)


def workload_config(n: int, T: int) -> dict:
    """The workload both arms report: the n x n roofline grid, T steps per bench step."""
    return {"workload": "roofline grid %dx%d, 32-Gaussian V, seed-random packet, %d Trotter "
                        "steps per step" % (n, n, T),
            "n": n, "trotter_steps_per_step": T}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    from paper_1208_2407_gb300 import workloads as wl
    cores = os.cpu_count() or 1
    n = args.n
    c = wl.roofline_grid(n=n, seed=args.seed, steps=1)
    re, im, V = c["re"], c["im"], c["V"]
    # bounded sample per step: the oracle's Trotter steps that fit ~10 s / K steps
    t0 = time.perf_counter()
    oracle.evolve(re, im, V, c["dt"], c["theta"], 1, nthreads=cores)
    t1 = time.perf_counter() - t0
    per = int(max(1, min(10, (60.0 / max(1, args.steps + args.warmup)) / max(t1, 1e-9))))
    for _ in range(args.warmup):
        oracle.evolve(re, im, V, c["dt"], c["theta"], 1, nthreads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.norm(*oracle.evolve(re, im, V, c["dt"], c["theta"], per, nthreads=cores))
    el = time.perf_counter() - t0
    value = n * n * per * args.steps / el
    sample = "%dx%d FP64 oracle, %d Trotter steps per step (bounded sample of %d), %d threads" % (
        n, n, per, args.trotter_steps, cores)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": el * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(workload_config(n, args.trotter_steps), parallelism="host threads",
                       sample_steps_per_step=per),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# DRAM traffic of the fused kernel from the committed ncu record
# ---------------------------------------------------------------------------
def kernel_source_hash() -> str:
    """Hash of the fused kernel's sources with comments and whitespace runs
    removed, so that only a change to the code itself invalidates the
    recorded DRAM traffic."""
    import hashlib
    import re
    h = hashlib.sha256()
    for name in ("fused.cu", "common.cuh", "ffloat.cuh", "internal.h", "mbar.cuh"):
        with open(os.path.join(ROOT, "paper_1208_2407_gb300", "csrc", name)) as f:
            text = f.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)   # block comments
        text = re.sub(r"//[^\n]*", " ", text)                   # line comments
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def recorded_traffic(n: int, K: int):
    """dram__bytes_read.sum + dram__bytes_write.sum per launch of
    fused_kernel<K> on an n x n grid, from profiles/fused_kernel_traffic.json,
    or None if there is no record for this case or the kernel source changed
    since it was taken."""
    try:
        with open(os.path.join(ROOT, "profiles", "fused_kernel_traffic.json")) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    h = kernel_source_hash()
    for e in rec.get("captures", []):
        if e.get("n") == n and e.get("K") == K and e.get("source_hash") == h:
            return e.get("dram_bytes_per_launch")
    return None


# ---------------------------------------------------------------------------
# serving: Poisson arrivals of mixed grids, continuous batching vs one at a time
# ---------------------------------------------------------------------------
def serve_bench(n_requests: int, seed: int, budget_gb: float = 120.0):
    """512 requests (mean gap 2 ms), each side from {128, ..., 4096}, steps
    uniform in [10, 2000], FP32, admission by a 120 GB budget.  Inputs: one
    seeded potential and packet per (nx, ny) shape, in pinned host memory,
    shared by the requests of that shape (content does not change the cost).
    Runs the same arrival sequence twice: continuous batching (up to 128
    admitted requests) and one request at a time."""
    import torch
    from paper_1208_2407_gb300 import trotter
    from paper_1208_2407_gb300 import workloads as wl
    reqs = wl.serving_requests(count=n_requests, mean_gap_s=2e-3, seed=seed)
    bank = {}
    for r in reqs:
        key = (r.nx, r.ny)
        if key in bank:
            continue
        re, im, V = wl.Request(rid=-1, arrival_s=0.0, nx=r.nx, ny=r.ny, steps=0,
                               seed=seed * 7919 + r.nx * 13 + r.ny).inputs()
        bank[key] = (torch.from_numpy(V).pin_memory(),
                     torch.from_numpy(re.astype(np.float32)).pin_memory(),
                     torch.from_numpy(im.astype(np.float32)).pin_memory())
    total = float(sum(r.nx * r.ny * r.steps for r in reqs))

    def run(max_slots):
        srv = trotter.Server(hbm_budget_bytes=int(budget_gb * (1 << 30)), max_slots=max_slots,
                             K=4, max_epoch_steps=32)
        t0 = time.perf_counter()
        tickets = []
        for r in reqs:
            delay = t0 + r.arrival_s - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            V, re, im = bank[(r.nx, r.ny)]
            tickets.append(srv.submit(r.nx, r.ny, r.steps, r.dt, r.theta, V, re, im))
        lat = []
        for t in tickets:
            res = srv.wait(t, -1)
            lat.append(res.latency_ns * 1e-6)
            srv.release(t)
        wall = time.perf_counter() - t0
        st = srv.stats()
        srv.close()
        lat = np.array(lat)
        return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(lat.mean()), "site_steps_per_s": total / wall, "wall_s": wall,
                "epochs": int(st["epochs"]), "graph_launches": int(st["graph_launches"]),
                "peak_gb": st["peak_bytes"] / 1e9}

    batched = run(128)
    sequential = run(1)
    return {"workload": "%d requests, Poisson mean gap 2 ms, sides {128..4096}^2, steps "
                        "U[10,2000], FP32, budget %.0f GB" % (n_requests, budget_gb),
            "total_site_steps": total, "continuous_batching": batched,
            "one_at_a_time": sequential}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def e2e_bench(c, n, T, K, steps, warmup, dist, log=None, nbuf=2):
    """End to end through the C ABI with pinned host buffers.  Each step
    uploads psi (FP32) and V (FP64) from pinned host memory, runs the step and
    reads the state and the observables back.  Two grids on two streams make
    a double buffer, driven by one host thread in a fixed order: while one
    grid's kernels run, the other grid's result is read back and its next
    inputs are uploaded.  Each grid's evolution waits (an event, on the
    device) for the other grid's previous evolution, so the kernels of the two
    grids alternate whole steps instead of sharing the SMs.  `log`, if a
    list, receives (grid, step, start, get_state + observe of the previous
    step, set_state, set_potential, evolve) host times."""
    import torch
    from paper_1208_2407_gb300 import trotter
    grids = [trotter.Grid(n, n, "f32") for _ in range(nbuf)]
    streams = [torch.cuda.Stream() for _ in range(nbuf)]
    h_re = torch.from_numpy(c["re"].astype(np.float32)).pin_memory()
    h_im = torch.from_numpy(c["im"].astype(np.float32)).pin_memory()
    h_V = torch.from_numpy(c["V"]).pin_memory()
    outs = [(torch.empty((n, n), dtype=torch.float32).pin_memory(),
             torch.empty((n, n), dtype=torch.float32).pin_memory()) for _ in range(nbuf)]
    hp = lambda t: trotter._VP(t.data_ptr())
    # the host link's speed on this machine (pinned, one 256 MiB copy each way)
    probe = torch.empty(n * n, dtype=torch.float32, device="cuda")
    link = {}
    for name, dst, src in (("h2d_gbs", probe, h_re.view(-1)), ("d2h_gbs", outs[0][0].view(-1), probe)):
        dst.copy_(src, non_blocking=True)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        dst.copy_(src, non_blocking=True)
        b.record()
        torch.cuda.synchronize()
        link[name] = round(4.0 * n * n / (a.elapsed_time(b) / 1e3) / 1e9, 1)
    del probe
    sps = [trotter._VP(st.cuda_stream) for st in streams]
    evolved = [torch.cuda.Event() for _ in range(nbuf)]   # after each grid's last evolve

    def read_back(i):
        o_re, o_im = outs[i]
        trotter.ts_get_state(grids[i].handle, hp(o_re), hp(o_im), trotter.TS_F32,
                             trotter.TS_HOST, sps[i])
        trotter.ts_observe(grids[i].handle, sps[i])

    def run_e2e(count, t_origin):
        started = [False] * nbuf
        last = None                       # the grid whose evolution was enqueued last
        for k in range(count):
            for i in range(nbuf):
                t = [time.perf_counter()]
                if started[i]:
                    read_back(i)          # step k - 1 of grid i
                t.append(time.perf_counter())
                gh = grids[i].handle
                trotter.ts_set_state(gh, hp(h_re), hp(h_im), trotter.TS_F32, trotter.TS_HOST,
                                     sps[i])
                t.append(time.perf_counter())
                trotter.ts_set_potential(gh, hp(h_V), trotter.TS_HOST, c["dt"], c["theta"],
                                         sps[i])
                t.append(time.perf_counter())
                if last is not None:
                    streams[i].wait_event(evolved[last])
                trotter.ts_evolve(gh, T, K, sps[i])
                evolved[i].record(streams[i])
                last, started[i] = i, True
                t.append(time.perf_counter())
                if log is not None:
                    log.append((i, k, t[0] - t_origin) + tuple(t[m + 1] - t[m] for m in range(4)))
        for i in range(nbuf):
            j = (last + 1 + i) % nbuf     # the oldest evolution first
            if started[j]:
                read_back(j)

    run_e2e(max(1, warmup // nbuf), time.perf_counter())
    torch.cuda.synchronize()
    dist.barrier()
    # at least 8 steps: the pipeline's fill (the first uploads) and drain (the
    # last download) are inside the timed region and are amortised over them
    per = max((8 + nbuf - 1) // nbuf, (steps + nbuf - 1) // nbuf)
    if log is not None:
        log.clear()
    t0 = time.perf_counter()
    run_e2e(per, t0)
    torch.cuda.synchronize()
    e2e_value = replica_throughput(dist, float(n) * n * T * per * nbuf, time.perf_counter() - t0)
    for gg in grids:
        gg.close()
    return {"value": e2e_value, "unit": UNIT,
            "h2d_bytes_per_step": int(n * n * (4 + 4 + 8)),
            "d2h_bytes_per_step": int(n * n * (4 + 4) + 7 * 8),
            "pipeline": "%d grids on %d streams, one host thread; a grid's read-back and next "
                        "uploads overlap the other grid's kernels, whose steps alternate"
                        % (nbuf, nbuf),
            "steps": per * nbuf, "link": link}


def precision_paths(c, n, fused_rate, reps=3, steps=10):
    """FP32 vs FP64 on the same workload, inputs resident in HBM: Trotter
    site-steps/s of ts_evolve and of the plain one-sweep-per-kernel path
    (ts_evolve_plain, nine launches per step) for each precision, median of
    `reps` runs of `steps` steps timed with CUDA events.  FP64 grids run one
    sweep per launch under ts_evolve too, with the sweeps merged where steps
    meet (6 n + 2 sweeps) in lifting form."""
    import torch
    from paper_1208_2407_gb300 import trotter
    out = {"steps": steps, "fp32_fused": fused_rate}
    for dtype in ("f32", "f64"):
        tdt = torch.float32 if dtype == "f32" else torch.float64
        g = trotter.Grid(n, n, dtype)
        try:
            g.set_state(torch.from_numpy(c["re"]).to(tdt).cuda(),
                        torch.from_numpy(c["im"]).to(tdt).cuda())
            g.set_potential(torch.from_numpy(c["V"]).cuda(), c["dt"], c["theta"])
            runs = [("plain", g.evolve_plain)] + ([("default", g.evolve)] if dtype == "f64" else [])
            for name, fn in runs:
                fn(1)
                rates = []
                for _ in range(reps):
                    torch.cuda.synchronize()
                    a = torch.cuda.Event(enable_timing=True)
                    b = torch.cuda.Event(enable_timing=True)
                    a.record()
                    fn(steps)
                    b.record()
                    torch.cuda.synchronize()
                    rates.append(float(n) * n * steps / (a.elapsed_time(b) / 1e3))
                out["%s_%s" % ("fp32" if dtype == "f32" else "fp64", name)] = \
                    sorted(rates)[len(rates) // 2]
        finally:
            g.close()
    out["fp32_fused_over_fp64_plain"] = fused_rate / out["fp64_plain"]
    out["fp32_fused_over_fp64_default"] = fused_rate / out["fp64_default"]
    return out


# algorithmic bytes per site-step of the paths k_sweep times (state 8 B/site FP32,
# 16 B FP64; the table gamma_V, s_V as wide as the state)
PLAIN_BYTES = {"f32": 8 * 16 + 24, "f64": 16 * 16 + 48}   # 8 sweeps + the phase


def fp64_merged_bytes(T: int) -> float:
    """ts_evolve on an FP64 grid: 6 T + 2 sweeps (32 B/site each) and T phases
    (48 B/site) for T steps, per site-step."""
    return ((6 * T + 2) * 32 + T * 48) / T


def k_sweep(args, hbm_peak, sizes=(8192, 16384), depths=range(1, 9), reps=3):
    """The roofline sweep: for each grid side, 200 Trotter steps of the fused
    kernel at every depth K = 1..8 (median of `reps` runs, CUDA events), then
    the plain one-sweep-per-kernel FP32 and FP64 paths and FP64 ts_evolve (one
    run each, 200 steps).  A fused launch moves 24 B per site whatever its
    depth, so T steps at depth K move 24 B x sites x ceil(T / K)."""
    import torch
    from paper_1208_2407_gb300 import trotter
    from paper_1208_2407_gb300 import workloads as wl
    T = args.trotter_steps
    rows = []

    def timed(fn, count):
        fn(1)
        ms = []
        for _ in range(count):
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn(T)
            b.record()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return sorted(ms)[len(ms) // 2]

    for n in sizes:
        c = wl.roofline_grid(n=n, seed=args.seed, steps=T)
        sites = float(n) * n
        for dtype in ("f32", "f64"):
            tdt = torch.float32 if dtype == "f32" else torch.float64
            g = trotter.Grid(n, n, dtype)
            try:
                g.set_state(torch.from_numpy(c["re"]).to(tdt).cuda(),
                            torch.from_numpy(c["im"]).to(tdt).cuda())
                g.set_potential(torch.from_numpy(c["V"]).cuda(), c["dt"], c["theta"])
                paths = []
                if dtype == "f32":
                    for K in depths:
                        launches = -(-T // K)
                        paths.append(("fused", K, lambda m, K=K: g.evolve(m, K), reps,
                                      24.0 * launches / T))
                    paths.append(("plain", None, g.evolve_plain, 1, PLAIN_BYTES["f32"]))
                else:
                    paths.append(("plain", None, g.evolve_plain, 1, PLAIN_BYTES["f64"]))
                    paths.append(("evolve", None, g.evolve, 1, fp64_merged_bytes(T)))
                for path, K, fn, count, bps in paths:
                    ms = timed(fn, count)
                    rate = sites * T / (ms / 1e3)
                    gbs = rate * bps / 1e9
                    row = {"n": n, "dtype": dtype, "path": path, "K": K, "steps": T, "ms": ms,
                           "site_steps_per_s": rate, "bytes_per_site_step": bps,
                           "achieved_gbs": gbs, "frac": gbs / hbm_peak}
                    if path == "fused":
                        row["traffic_per_launch"] = recorded_traffic(n, K)
                    rows.append(row)
            finally:
                g.close()
        del c
        torch.cuda.empty_cache()
    return {"peak_gbs": hbm_peak, "rows": rows,
            "note": "inputs resident in HBM; fused rows: median of %d runs; others: one run" % reps}


def adjoint_bytes(n_sites: int, steps: int, ckpt: int, K: int, K_fwd: int):
    """Algorithmic bytes of one adjoint forward and one backward pass on an
    FP32 grid (per site: a state 8 B, the table 8 B, G 16 B as double-float
    re, im).  Forward: target conversion (16), per segment ts_evolve at depth
    K_fwd (24 per launch) and a checkpoint copy (16), the overlap
    <phi|psi_T> (16).  Backward: costate set-up (16), G cleared (16), per
    segment a checkpoint copy (16) and launches of K backward steps on psi
    and lambda together (72 per launch: both states read and written 32, the
    table 8, G read and written 32), then the gradient (G 16 in, 4 out)."""
    fwd, bwd = 16 + 16, 16 + 16 + 20
    for s0 in range(0, steps, ckpt):
        ns = min(ckpt, steps - s0)
        fwd += 16 + 24 * -(-ns // K_fwd)
        bwd += 16 + 72 * -(-ns // K)
    return fwd * n_sites, bwd * n_sites


def adjoint_bench(args, hbm_peak, cases=((1024, 500, 50), (4096, 200, 50)), depths=(1, 2, 3, 4),
                  reps=3):
    """The adjoint workload (config 5: 1024^2, 500 steps, checkpoints every
    50) and a 4096^2 grid: CUDA-event time of ts_adjoint_forward and of
    ts_adjoint_backward_depth at each depth (median of `reps`), with the
    algorithmic bytes of each pass and its fraction of measured HBM."""
    import torch
    from paper_1208_2407_gb300 import trotter
    from paper_1208_2407_gb300 import workloads as wl
    out = []
    K_fwd = trotter.ts_fused_default_depth()
    for n, steps, ckpt in cases:
        c = wl.adjoint_pair(n=n, steps=steps, seed=args.seed)
        g = trotter.Grid(n, n, "f32")
        try:
            re0 = torch.from_numpy(c["re"].astype(np.float32)).cuda()
            im0 = torch.from_numpy(c["im"].astype(np.float32)).cuda()
            tre = torch.from_numpy(c["target_re"].astype(np.float32)).cuda()
            tim = torch.from_numpy(c["target_im"].astype(np.float32)).cuda()
            g.set_potential(torch.from_numpy(c["V"]).cuda(), c["dt"], c["theta"])
            nbytes = trotter.ts_adjoint_workspace(g.handle, steps, ckpt)
            ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
            grad = torch.empty((n, n), dtype=torch.float32, device="cuda")
            sp = trotter.current_stream_ptr()
            wsp, gp = trotter._VP(ws.data_ptr()), trotter._VP(grad.data_ptr())

            def ev_time(fn):
                torch.cuda.synchronize()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                r = fn()
                b.record()
                torch.cuda.synchronize()
                return a.elapsed_time(b), r

            def forward():
                return trotter.ts_adjoint_forward(
                    g.handle, trotter._VP(tre.data_ptr()), trotter._VP(tim.data_ptr()),
                    trotter.TS_F32, trotter.TS_DEVICE, steps, ckpt, wsp, nbytes, sp)[0]

            row = {"n": n, "steps": steps, "ckpt": ckpt, "K_forward": K_fwd, "backward": []}
            fw_ms = []
            for K in depths:
                bw_ms = []
                for rep in range(reps + 1):
                    g.set_state(re0, im0)
                    ms, F = ev_time(forward)
                    if rep:
                        fw_ms.append(ms)
                    ms, _ = ev_time(lambda: trotter.ts_adjoint_backward_depth(
                        g.handle, wsp, nbytes, K, gp, sp))
                    if rep:
                        bw_ms.append(ms)
                t = sorted(bw_ms)[len(bw_ms) // 2]
                fb, bb = adjoint_bytes(n * n, steps, ckpt, K, K_fwd)
                row["backward"].append({
                    "K": K, "ms": t, "bytes": bb, "bytes_per_site_step": bb / (n * n * steps),
                    "achieved_gbs": bb / (t / 1e3) / 1e9,
                    "frac": bb / (t / 1e3) / 1e9 / hbm_peak})
            tf = sorted(fw_ms)[len(fw_ms) // 2]
            fb, _ = adjoint_bytes(n * n, steps, ckpt, 1, K_fwd)
            row.update({"forward_ms": tf, "forward_bytes": fb,
                        "forward_bytes_per_site_step": fb / (n * n * steps),
                        "forward_achieved_gbs": fb / (tf / 1e3) / 1e9,
                        "forward_frac": fb / (tf / 1e3) / 1e9 / hbm_peak, "fidelity": F})
            best = min(row["backward"], key=lambda r: r["ms"])
            row["best_backward_K"] = best["K"]
            row["backward_over_forward"] = best["ms"] / tf
            out.append(row)
            del ws, grad
        finally:
            g.close()
        torch.cuda.empty_cache()
    return {"peak_gbs": hbm_peak, "cases": out,
            "note": "inputs resident in HBM; median of %d runs per depth" % reps}


def accuracy_block(args):
    """The accuracy workloads against the FP64 oracle on this host's cores:
    the 256^2 FP64 plain workload (100 steps); the 2048^2 FP32 harmonic
    workload for seeds 0-4 (1000 steps: relative L2 error, norm drift, energy
    drift beside the oracle's own drift, and the oracle's time), and seed 0 on
    the FP64 path; the 1024^2 adjoint (500 steps, checkpoints every 50):
    fidelity and gradient against central differences in FP64 on 64 sites
    and against the oracle adjoint."""
    import oracle
    import torch
    from paper_1208_2407_gb300 import trotter
    from paper_1208_2407_gb300 import workloads as wl
    cores = os.cpu_count() or 1
    out = {"host_cores": cores}

    def rel(are, aim, bre, bim):
        return float(np.sqrt(np.sum((are - bre) ** 2 + (aim - bim) ** 2) /
                             np.sum(bre ** 2 + bim ** 2)))

    def gpu_run(c, dtype, plain=False):
        g = trotter.Grid(c["nx"], c["ny"], dtype)
        try:
            g.set_state(c["re"], c["im"])
            g.set_potential(c["V"], c["dt"], c["theta"])
            o0 = g.observe()
            (g.evolve_plain if plain else g.evolve)(c["steps"])
            o1 = g.observe()
            re, im = g.get_state(np.float64)
        finally:
            g.close()
        return re, im, o0, o1

    c = wl.plain_fp64_256()
    gre, gim, _, o1 = gpu_run(c, "f64", plain=True)
    t0 = time.perf_counter()
    ore, oim = oracle.evolve(c["re"], c["im"], c["V"], c["dt"], c["theta"], c["steps"])
    t_or = time.perf_counter() - t0
    m = oracle.moments(ore, oim)
    out["c1_plain_fp64_256"] = {
        "rel_l2": rel(gre, gim, ore, oim), "norm_minus_1": o1["norm"] - 1.0,
        "x_err": abs(o1["x"] - m[1] / m[0]), "y_err": abs(o1["y"] - m[2] / m[0]),
        "oracle_site_steps_per_s_1thread": 256 * 256 * c["steps"] / t_or}

    seeds = []
    for seed in range(5):
        c = wl.harmonic_2048(seed=seed)
        gre, gim, o0, o1 = gpu_run(c, "f32")
        t0 = time.perf_counter()
        ore, oim = oracle.evolve(c["re"], c["im"], c["V"], c["dt"], c["theta"], c["steps"],
                                 nthreads=cores)
        t_or = time.perf_counter() - t0
        e0 = sum(oracle.energy(c["re"], c["im"], c["V"]))
        eo = sum(oracle.energy(ore, oim, c["V"]))
        scale = max(1e-12, abs(e0))
        row = {"seed": seed, "rel_l2": rel(gre, gim, ore, oim),
               "norm_drift": abs(o1["norm"] - o0["norm"]),
               "energy_drift_rel": (o1["e_kin"] + o1["e_pot"] - o0["e_kin"] - o0["e_pot"]) / scale,
               "oracle_energy_drift_rel": (eo - e0) / scale,
               "oracle_site_steps_per_s": float(c["nx"]) * c["ny"] * c["steps"] / t_or}
        if seed == 0:
            fre, fim, _, _ = gpu_run(c, "f64")
            row["fp64_evolve_rel_l2"] = rel(fre, fim, ore, oim)
        seeds.append(row)
    out["c2_harmonic_2048_fp32"] = seeds

    c = wl.adjoint_pair(n=1024, steps=500, seed=0)
    g = trotter.Grid(c["nx"], c["ny"], "f32")
    try:
        g.set_state(c["re"], c["im"])
        g.set_potential(c["V"], c["dt"], c["theta"])
        F, grad = trotter.adjoint_fidelity_grad(g, c["target_re"], c["target_im"], c["steps"], 50)
        grad = grad.double().cpu().numpy()
    finally:
        g.close()
    rng = np.random.default_rng(123)
    weight = c["re"] ** 2 + c["im"] ** 2 + c["target_re"] ** 2 + c["target_im"] ** 2
    sites = rng.choice(np.flatnonzero(weight.ravel() > 1e-3 * weight.max()), 64, replace=False)
    g64 = trotter.Grid(c["nx"], c["ny"], "f64")
    fd = np.zeros(len(sites))
    h = 1e-3
    try:
        for i, j in enumerate(sites):
            vals = []
            for sgn in (1.0, -1.0):
                V = c["V"].copy()
                V.flat[j] += sgn * h
                g64.set_state(c["re"], c["im"])
                g64.set_potential(V, c["dt"], c["theta"])
                g64.evolve_plain(c["steps"])
                re, im = g64.get_state(np.float64)
                vals.append(abs(np.vdot(c["target_re"] + 1j * c["target_im"], re + 1j * im)) ** 2)
            fd[i] = (vals[0] - vals[1]) / (2 * h)
    finally:
        g64.close()
    t0 = time.perf_counter()
    og, oF, _ = oracle.adjoint_grad(c["re"], c["im"], c["target_re"], c["target_im"], c["V"],
                                    c["dt"], c["theta"], c["steps"], nthreads=cores)
    t_or = time.perf_counter() - t0
    gs = grad.ravel()[sites]
    out["c5_adjoint_1024"] = {
        "fidelity": F, "oracle_fidelity": oF,
        "grad_vs_fd_rel_l2": float(np.linalg.norm(gs - fd) / np.linalg.norm(fd)),
        "grad_vs_oracle_rel_l2": float(np.linalg.norm(grad - og) / np.linalg.norm(og)),
        "fd_sites": 64, "fd_h": h, "oracle_adjoint_s": t_or}
    return out


def run_ours(args):
    import torch
    from paper_1208_2407_gb300 import trotter
    from paper_1208_2407_gb300 import workloads as wl

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dist = Dist(world, local, "nccl")
    trotter.load()
    n, T = args.n, args.trotter_steps
    K = args.K
    c = wl.roofline_grid(n=n, seed=args.seed + rank, steps=T)

    # inputs resident in HBM
    re0 = torch.from_numpy(c["re"].astype(np.float32)).cuda()
    im0 = torch.from_numpy(c["im"].astype(np.float32)).cuda()
    Vd = torch.from_numpy(c["V"]).cuda()
    g = trotter.Grid(n, n, "f32")
    stream = torch.cuda.current_stream()
    sp = trotter.current_stream_ptr()

    ev_pairs = []

    def one_step(record):
        g.set_state(re0, im0, stream=sp)
        g.set_potential(Vd, c["dt"], c["theta"], stream=sp)
        if record:
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            g.evolve(T, K, stream=sp)
            b.record(stream)
            ev_pairs.append((a, b))
        else:
            g.evolve(T, K, stream=sp)
        return g.observe(stream=sp)

    for _ in range(args.warmup):
        obs = one_step(False)
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    dist.barrier()
    torch.cuda.synchronize()
    trotter.ts_launch_count(reset=True)
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for _ in range(args.steps):
        obs = one_step(True)
    end.record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    clocks = sampler.stop()
    launches = trotter.ts_launch_count()
    el_ms = start.elapsed_time(end)
    value = replica_throughput(dist, float(n) * n * T * args.steps, el_ms / 1e3)
    el_ms = dist.max(el_ms)
    evolve_ms = sum(a.elapsed_time(b) for a, b in ev_pairs)
    k_eff = K if K > 0 else trotter.ts_fused_default_depth()
    fused_launches_per_step = (T + k_eff - 1) // k_eff
    avg_launch_ms = evolve_ms / (fused_launches_per_step * args.steps)

    site_steps = float(n) * n * T

    # ---- end to end through the C ABI with pinned host buffers ----
    e2e = None
    if not args.no_e2e:
        g.close()
        g = None
        e2e = e2e_bench(c, n, T, K, args.steps, args.warmup, dist)

    # ---- roofline of the dominant kernel (the fused K-step kernel) ----
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except (OSError, ValueError):
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    achieved_gbs = BYTES_PER_SITE_LAUNCH * float(n) * n / (avg_launch_ms / 1e3) / 1e9
    traffic = recorded_traffic(n, k_eff)
    roofline = {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved_gbs / hbm_peak, "traffic": traffic, "peak_source": peak_src,
                "kernel": "fused_kernel<%d>" % k_eff,
                "avg_launch_ms": avg_launch_ms,
                "algorithmic_bytes_per_launch": BYTES_PER_SITE_LAUNCH * n * n}

    precision = None
    if rank == 0 and not args.no_precision:
        if g is not None:
            g.close()
            g = None
        precision = precision_paths(c, n, site_steps * args.steps / (evolve_ms / 1e3))

    ksweep = None
    if rank == 0 and world == 1 and not args.no_k_sweep:
        if g is not None:
            g.close()
            g = None
        ksweep = k_sweep(args, hbm_peak)

    adjoint = None
    if rank == 0 and world == 1 and not args.no_adjoint:
        if g is not None:
            g.close()
            g = None
        adjoint = adjoint_bench(args, hbm_peak)

    accuracy = None
    if rank == 0 and world == 1 and not args.no_accuracy:
        if g is not None:
            g.close()
            g = None
        accuracy = accuracy_block(args)

    serve = None
    if rank == 0 and not args.no_serve:
        if g is not None:
            g.close()
            g = None
        serve = serve_bench(args.serve_requests, args.seed)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, cores, sample = oracle_sample(n, args.seed)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": dict(workload_config(n, T), K=k_eff,
                           l2="inputs larger than L2 (%.1f GB working set)" % (n * n * 28 / 1e9),
                           parallelism="replicas" if world > 1 else "single"),
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clocks,
            "obs_last": {"norm": obs["norm"], "energy": obs["e_kin"] + obs["e_pot"]},
            "precision": precision,
            "k_sweep": ksweep,
            "adjoint": adjoint,
            "accuracy": accuracy,
            "serve": serve,
        }
        print(json.dumps(line), flush=True)
    if g is not None:
        g.close()
    dist.close()
    return 0


# ---------------------------------------------------------------------------
# the paper's single-node workloads on one GB300
# ---------------------------------------------------------------------------
def paper_sizes(args):
    """Ten iterations of the main loop on the sizes that filled one 2012 node
    (L = 24576 single precision, 17472 double precision; flat potential).
    Inputs are built on the device: a Gaussian packet (separable, so an outer
    product of two 1-D packets) and V = 0.3 everywhere."""
    import torch
    from paper_1208_2407_gb300 import trotter
    torch.cuda.set_device(0)
    trotter.load()
    out = []
    for L, dtype, path in ((24576, "f32", "fused"), (24576, "f32", "plain"),
                           (17472, "f64", "evolve"), (17472, "f64", "plain")):
        tdt = torch.float32 if dtype == "f32" else torch.float64
        x = torch.arange(L, device="cuda", dtype=torch.float64)
        sigma, k = L / 16.0, 0.5
        env = torch.exp(-((x - L / 2) ** 2) / (4 * sigma * sigma))
        fr, fi = env * torch.cos(k * x), env * torch.sin(k * x)
        nrm = torch.sqrt(torch.sum(env * env) ** 2)
        re = (torch.outer(env, fr) / nrm).to(tdt).contiguous()
        im = (torch.outer(env, fi) / nrm).to(tdt).contiguous()
        V = torch.full((L, L), 0.3, dtype=torch.float64, device="cuda")
        g = trotter.Grid(L, L, dtype)
        g.set_state(re, im)
        g.set_potential(V, 0.05, 0.025)
        del re, im, V
        torch.cuda.empty_cache()
        # "evolve": ts_evolve on an FP64 grid (one sweep per launch, merged)
        run = (lambda n: g.evolve_plain(n)) if path == "plain" else (lambda n: g.evolve(n))
        run(1)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        run(10)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        nrm_after = g.norm()
        g.close()
        out.append({"L": L, "dtype": dtype, "path": path, "iterations": 10, "ms": ms,
                    "site_steps_per_s": L * L * 10 / (ms / 1e3), "norm": nrm_after})
    print(json.dumps({"metric": "paper single-node sizes, 10 iterations", "runs": out}), flush=True)
    return 0


def method_variants(args):
    """The method's variants on the n x n random-Gaussian workload, inputs
    resident in HBM: second order (the default depth), fourth-order steps U4
    (five second-order substeps; counted per U4 step) at a few depths, a
    time-dependent potential V0 + a(t) V1 (a field along x oscillating in
    time; the drive phase is computed per site and step on the device), and
    an n3^3 lattice (harmonic V, a Gaussian packet) on the fast and the plain
    3-D paths."""
    import torch
    from paper_1208_2407_gb300 import trotter
    from paper_1208_2407_gb300 import workloads as wl
    torch.cuda.set_device(0)
    trotter.load()
    n = args.n
    T = args.trotter_steps
    T4 = max(1, T // 5)
    c = wl.roofline_grid(n=n, seed=args.seed, steps=T)
    re0 = torch.from_numpy(c["re"].astype(np.float32)).cuda()
    im0 = torch.from_numpy(c["im"].astype(np.float32)).cuda()
    Vd = torch.from_numpy(c["V"]).cuda()
    V1 = torch.arange(n, dtype=torch.float64, device="cuda").sub_(n / 2.0).expand(n, n).contiguous()
    amp = 1e-3 * np.cos(0.05 * (np.arange(T) + 0.5) * c["dt"])
    g = trotter.Grid(n, n, "f32")
    runs = []
    cases = (("order 2", 2, 0, T, False), ("order 4", 4, 0, T4, False), ("order 4", 4, 3, T4, False),
             ("drive", 2, 0, T, True), ("drive", 2, 4, T, True))
    only = args.only
    for name, order, K, steps, drive in cases:
        if only and not (only == "order4" and order == 4 and K == 0 or
                         only == "drive" and drive and K == 0):
            continue
        ms = []
        for rep in range(max(1, args.steps) + 1):
            g.set_state(re0, im0)
            g.set_potential(Vd, c["dt"], c["theta"], order=order)
            if drive:
                g.set_drive(V1, amp[:steps])
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            trotter.ts_launch_count(reset=True)
            a.record()
            g.evolve(steps, K)
            b.record()
            torch.cuda.synchronize()
            if rep > 0:                  # the first run is a warm-up
                ms.append(a.elapsed_time(b))
        t = float(np.median(ms))
        substeps = steps * (5 if order == 4 else 1)
        runs.append({"variant": name, "order": order, "K": K, "steps": steps, "ms": t,
                     "launches": trotter.ts_launch_count(),
                     "site_steps_per_s": float(n) * n * steps / (t / 1e3),
                     "site_substeps_per_s": float(n) * n * substeps / (t / 1e3),
                     "norm": g.norm()})
    g.close()
    del re0, im0, Vd, V1
    torch.cuda.empty_cache()
    if only and only != "3d":
        print(json.dumps({"metric": "site-steps/s of the method's variants", "n": n, "runs": runs,
                          "data": "synthetic", "inputs": "resident in HBM"}), flush=True)
        return 0
    # a 3-D lattice: n3^3 sites, separable packet and harmonic V built on the device
    n3 = args.n3
    t = torch.arange(n3, dtype=torch.float64, device="cuda")
    env = torch.exp(-((t - n3 / 2.0) ** 2) / (4.0 * (n3 / 16.0) ** 2))
    g1 = env * torch.exp(0.5j * t)
    g1 = g1 / torch.sqrt(torch.sum(torch.abs(g1) ** 2))
    psi = torch.einsum("z,y,x->zyx", g1, g1, g1)
    re3 = psi.real.float().contiguous()
    im3 = psi.imag.float().contiguous()
    del psi
    r2 = (t - n3 / 2.0) ** 2
    V3 = (0.5e-4 * (r2[None, None, :] + r2[None, :, None] + r2[:, None, None])).contiguous()
    g3 = trotter.Grid(n3, n3, "f32", nz=n3)
    T3 = max(1, T // 4)
    for path in ("fused",) if only else ("fused", "plain"):
        steps = T3 if path == "fused" else max(1, T3 // 10)
        ms = []
        for rep in range(max(1, args.steps) + 1):
            g3.set_state(re3, im3)
            g3.set_potential(V3, c["dt"], c["theta"])
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            trotter.ts_launch_count(reset=True)
            a.record()
            if path == "fused":
                g3.evolve(steps)
            else:
                g3.evolve_plain(steps)
            b.record()
            torch.cuda.synchronize()
            if rep > 0:
                ms.append(a.elapsed_time(b))
        tm = float(np.median(ms))
        runs.append({"variant": "3-D %d^3 %s" % (n3, path), "order": 2, "K": 1, "steps": steps,
                     "ms": tm, "launches": trotter.ts_launch_count(),
                     "site_steps_per_s": float(n3) ** 3 * steps / (tm / 1e3),
                     "site_substeps_per_s": float(n3) ** 3 * steps / (tm / 1e3),
                     "norm": g3.norm()})
    g3.close()
    print(json.dumps({"metric": "site-steps/s of the method's variants", "n": n, "runs": runs,
                      "data": "synthetic", "inputs": "resident in HBM"}), flush=True)
    return 0


def traffic_launches(args):
    """For an ncu capture of DRAM traffic (one pass, gpu__time_duration and
    dram__bytes_{read,write}): on each grid side of the depth sweep, one
    warm-up launch and then exactly one launch of the fused kernel at every
    depth K = 1..8 (ts_evolve of K steps at depth K).  The kernel of launch
    2i + 1 on side n is fused_kernel<i + 1>."""
    import torch
    from paper_1208_2407_gb300 import trotter
    from paper_1208_2407_gb300 import workloads as wl
    torch.cuda.set_device(0)
    trotter.load()
    for n in args.traffic_n:
        c = wl.roofline_grid(n=n, seed=args.seed, steps=1)
        g = trotter.Grid(n, n, "f32")
        try:
            g.set_state(torch.from_numpy(c["re"].astype(np.float32)).cuda(),
                        torch.from_numpy(c["im"].astype(np.float32)).cuda())
            g.set_potential(torch.from_numpy(c["V"]).cuda(), c["dt"], c["theta"])
            for K in range(1, 9):
                g.evolve(K, K)
                g.evolve(K, K)
            torch.cuda.synchronize()
        finally:
            g.close()
        del c
    print(json.dumps({"traffic_launches": list(args.traffic_n),
                      "kernel_source_hash": kernel_source_hash()}), flush=True)
    return 0


def adjoint_only(args):
    import torch
    from paper_1208_2407_gb300 import trotter
    torch.cuda.set_device(0)
    trotter.load()
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except (OSError, ValueError):
        pass
    depths = (args.K,) if args.K > 0 else (1, 2, 3, 4)
    r = adjoint_bench(args, float(peaks.get("hbm_gbs", 6800.0)),
                      cases=((args.adj_n, args.adj_steps, args.adj_ckpt),), depths=depths,
                      reps=max(1, args.steps))
    print(json.dumps({"metric": "adjoint forward and backward", "adjoint": r}), flush=True)
    return 0


def main():
    args = parse()
    if args.adjoint:
        return adjoint_only(args)
    if args.traffic:
        return traffic_launches(args)
    if args.paper:
        return paper_sizes(args)
    if args.variants:
        return method_variants(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
