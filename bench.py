"""Benchmark of the barrier-free AL contact step through the C ABI, on one or
more GPUs (one independent replica per rank, weak scaling).

Headline: the contact-rich compression scene (five spiky balls, 2,299,164
tets, 432,048 vertices, mixed precision) with the plate schedule of the
workload: down at 0.5 m/s to 30 % of its starting height (reached at step
52), then back up (the schedule ends at step 105).  The first steps advance
untimed up to a window centred on peak compression; W warm-up steps follow,
then K timed steps (each with CUDA events on the library's stream; the
working set, about 1.1 GB, is larger than L2).  The window is then replayed
from a checkpoint twice: with per-kernel timers (roofline of the PCG and the
per-phase split of the paper's Tab. 1 columns) and end to end through
bf_step_host with pinned host buffers.  The rest of the schedule (the
release) runs after the window.

A "step" is one time step of Alg. 1 (inertia target, mu, Newton solves with
PCG, line search, multiplier update, active-set update, CCD, blending).

Extras in the same line: the eight-cube scene (196,608 tets; L2 flushed
before each timed step) with its own roofline, the oracle timed on the same
contact steps, and the error against the FP64 oracle; batched scenes against
the plain FP64 path; a served request stream; material and friction
variants.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
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

METRIC = "time steps/s & PCG HBM GB/s vs peak; p50/p99 step latency, batched vs plain FP64"
LARGE_WORKLOAD = ("spiky_balls: 5 spiky balls (radius 0.1 m, 64 spikes of 0.02-0.05 m, grid Kuhn mesher at "
                  "3.9 mm: 2,299,164 tets, 432,048 vertices) in a 0.66 m open box, compressed by a plate moving "
                  "at 0.5 m/s to 30 % of its starting height, then released; SNH E=5e4 nu=0.45 rho=1000, "
                  "h=1/60 s, delta=1e-3, CG tol 1e-6, mixed precision (FP32 Hessian/SpMV/preconditioner, "
                  "FP64 CCD/TOI/multipliers/dots)")
EIGHT_WORKLOAD = ("eight_cubes: 8 cubes x 16^3 cells (196,608 tets, 39,304 verts) with seeded yaw/offsets "
                  "dropped into a static open box; SNH E=1e5 nu=0.4 rho=1000, h=0.01, delta=1e-3, CG tol 1e-6, "
                  "mixed precision (FP32 Hessian/SpMV/preconditioner, FP64 CCD/TOI/multipliers/dots)")
GOLDEN = os.path.join(ROOT, "tests", "golden", "eight_cubes_oracle.npz")


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ["clocks.sm", "clocks.max.sm", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap"]
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, index=0):
        self.index = index
        self.samples = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == len(self.FIELDS):
                self.samples.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        reasons = set()
        for s in self.samples:
            for name, val in zip(self.NAMES, s[2:]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


# ---------------------------------------------------------------------------
# algorithmic bytes per launch of the timed kernels
# ---------------------------------------------------------------------------
def pcg_iteration_bytes(nnzb, nv, nc, w):
    """algorithmic bytes of one block-Jacobi PCG iteration: one symmetric
    upper-BSR SpMV (values + column index per block; row pointer, x, y per
    vertex), the matrix-free contact rank-1 terms (FP64 gradient, weight,
    ids, mask per pair), the 3x3 block preconditioner and ~7 vector passes
    (read p, q, r, x, z; write x, r/p) of 3 values per vertex"""
    spmv = nnzb * (9 * w + 4) + nv * (4 + 3 * w + 3 * w)
    contacts = nc * (12 * 8 + 8 + 16 + 1)
    return spmv + contacts + nv * 9 * w + 7 * 3 * nv * w


def algorithmic_bytes(kernel, info, nv, nt, nc, mixed, cg_per_launch=None):
    w = 4 if mixed else 8
    nnzb = info["nnzb"]
    if kernel == "pcg_persistent":
        return pcg_iteration_bytes(nnzb, nv, nc, w) * cg_per_launch if cg_per_launch else None
    if kernel == "spmv_bsr_contact":
        # values + column index per block, row pointer + x + y per vertex,
        # contact pairs (12 gradient entries, weight, 4 ids, mask)
        return nnzb * (9 * w + 4) + nv * (4 + 3 * w + 3 * w) + nc * (12 * 8 + 8 + 16 + 1)
    if kernel == "pcg_update":
        # read x(8) p(w) q(w) r(8) P^-1(9w); write x(8) r(8) z(w), per DoF / vertex
        return nv * (3 * (8 + w + w + 8 + 8 + 8 + w) + 9 * w)
    if kernel == "pcg_direction":
        return nv * 3 * (3 * w + w)  # read z, p; write p, q
    if kernel == "elastic_grad_hess":
        # per tet: ids, 4 gathered positions, Dm^-1, V, mu, lam, block map;
        # outputs: block values once, gradient
        return nt * (16 + 96 + 72 + 24 + 40) + nnzb * 9 * w + nv * 24
    if kernel == "energy":
        return nt * (16 + 96 + 72 + 24) + nv * (8 + 1 + 48) + nc * (16 + 96 + 32)
    return None


def traffic_for(kernel):
    """DRAM traffic from a committed ncu summary, if it was taken on the
    current kernel source (else None): per launch, or per iteration for a
    persistent solver"""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    ent = d.get(kernel)
    if not ent:
        return None
    src = os.path.join(ROOT, "paper_2512_12151_b300", "csrc", ent["source"])
    if not os.path.exists(src):
        return None
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    if h != ent.get("source_sha256_16"):
        return None
    # a persistent solve's traffic is scaled by its iterations
    if "iterations_per_launch" in ent:
        return ent["bytes_per_launch"] / ent["iterations_per_launch"]
    return ent["bytes_per_launch"]


# ---------------------------------------------------------------------------
def dist_init(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return ws, rank, local


def _reduce_device():
    """CUDA for NCCL process groups, host memory for gloo"""
    import torch.distributed as dist
    return "cuda" if dist.get_backend() == "nccl" else "cpu"


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(ws, v):
    if ws <= 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=_reduce_device())
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allsum(ws, v):
    if ws <= 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=_reduce_device())
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ---------------------------------------------------------------------------
# the plate schedule of the spiky-ball scene
# ---------------------------------------------------------------------------
def schedule(s, scenes):
    """(peak step, number of steps): the 0-based step at whose end the plate
    is lowest, and the steps until it is back at its starting height"""
    z0 = s.meta["plate_z0"]
    zs, i = [], 0
    while True:
        zs.append(scenes.plate_schedule_z(s, i))
        if i > 0 and zs[-1] >= z0:
            break
        i += 1
    return int(np.argmin(zs)), len(zs)


# ---------------------------------------------------------------------------
# the oracle on the host cores: the CPU baseline and the reference values of
# the error against FP64 (the only part of this file that runs oracle/)
# ---------------------------------------------------------------------------
def _oracle_batch_scene(arg):
    """one batched scene (a seed, or the (seed, t_lo, t_hi) of a served
    request), 10 steps, in a worker process of the all-core leg"""
    import oracle as O
    from paper_2512_12151_b300 import scenes
    s = scenes.batch_scene(arg) if isinstance(arg, int) else scenes.batch_scene(*arg)
    o = O.Oracle(s)
    t0 = time.perf_counter()
    status, _ = o.step(10)
    return 10, time.perf_counter() - t0, status


def oracle_leg(prefix, seconds, batch_scenes=0):
    """Child process, started before any CUDA call.  (0) The two-cube scene
    in FP64, all 20 steps, positions after each saved.  (1) The eight-cube
    scene from the oracle's own stored state after 16 steps (in contact):
    two steps timed, positions saved.  (2) The spiky-ball scene from rest:
    whole steps with the plate schedule until `seconds` have elapsed (at
    least one), the positions after the first step saved.  (3) Once the
    file prefix_go exists (the GPU runs are over): the first `batch_scenes`
    batched scenes, 10 steps each, one scene per host core (spawned
    workers).  Prints one JSON line after each part."""
    import oracle as O
    from paper_2512_12151_b300 import scenes
    out = {}
    s = scenes.two_cubes(0)
    o = O.Oracle(s)
    xs = []
    t0 = time.perf_counter()
    for _ in range(s.n_steps):
        status, _st = o.step(1)
        xs.append(o.get_state()[0])
    el = time.perf_counter() - t0
    np.save(prefix + "_two.npy", np.array(xs))
    out["two"] = {"value": s.n_steps / el, "seconds": el, "steps": s.n_steps, "status": status}
    print(json.dumps(out), flush=True)
    g = np.load(GOLDEN)
    s = scenes.eight_cubes(0)
    o = O.Oracle(s)
    o.set_state(g["x16"], g["v16"])
    o.active_set(g["keys16"], g["lam16"], g["gam16"])
    xs, stats = [], []
    t0 = time.perf_counter()
    for _ in range(2):
        status, st = o.step(1)
        xs.append(o.get_state()[0])
        stats.append(st[0])
    el = time.perf_counter() - t0
    np.savez(prefix + "_eight.npz", x17=xs[0], x18=xs[1])
    out["eight"] = {"value": 2 / el, "seconds": el, "steps": "16..17 (in contact)", "status": status,
                    "outer_iters": [x["outer_iters"] for x in stats], "contacts": [x["n_contacts"] for x in stats]}
    print(json.dumps(out), flush=True)
    s = scenes.spiky_balls(precision=1)
    o = O.Oracle(s)
    n, stats = 0, []
    t0 = time.perf_counter()
    while True:
        ts = time.perf_counter()
        o.set_dirichlet_targets(scenes.plate_targets_schedule(s, n))
        status, st = o.step(1)
        stats.append(st[0])
        n += 1
        if n == 1:
            np.save(prefix + "_large_x1.npy", o.get_state()[0])
        el = time.perf_counter() - t0
        if status != 0 or el + (time.perf_counter() - ts) > seconds:
            break
    out["large"] = {"value": n / el, "seconds": el, "steps": n, "status": status,
                    "outer_iters": [x["outer_iters"] for x in stats], "contacts": [x["n_contacts"] for x in stats]}
    print(json.dumps(out), flush=True)
    # the all-core part waits until the GPU runs are over (their host threads
    # would otherwise compete with it for the cores)
    deadline = time.monotonic() + 1800
    while batch_scenes > 0 and not os.path.exists(prefix + "_go") and time.monotonic() < deadline:
        time.sleep(0.5)
    if batch_scenes > 0:
        import multiprocessing as mp
        cores = os.cpu_count() or 1
        t0 = time.perf_counter()
        with mp.get_context("spawn").Pool(cores) as pool:
            res = pool.map(_oracle_batch_scene, range(batch_scenes), chunksize=1)
        el = time.perf_counter() - t0
        out["batched"] = {"value": sum(r[0] for r in res) / el, "seconds": el, "scenes": batch_scenes,
                          "cores": cores, "failed": sum(1 for r in res if r[2] != 0)}
        print(json.dumps(out), flush=True)
        # the served stream's first requests (the same list as the GPU's
        # served line, rank 0's seed), one per core
        from paper_2512_12151_b300 import serving
        reqs = serving.poisson_requests(cores, 200.0, seed=1000)
        t0 = time.perf_counter()
        with mp.get_context("spawn").Pool(cores) as pool:
            res = pool.map(_oracle_batch_scene, [(r[1], r[2], r[3]) for r in reqs], chunksize=1)
        el = time.perf_counter() - t0
        out["served"] = {"value": sum(r[0] for r in res) / el, "seconds": el, "requests": len(reqs),
                         "cores": cores, "failed": sum(1 for r in res if r[2] != 0)}
        print(json.dumps(out), flush=True)
    return 0


def start_oracle_leg(seconds, batch_scenes):
    """the oracle leg in a child process (fork + exec: no CUDA state is shared)"""
    import tempfile
    prefix = os.path.join(tempfile.mkdtemp(prefix="bf_oracle_"), "leg")
    proc = subprocess.Popen([sys.executable, os.path.abspath(__file__), "--oracle-leg", prefix,
                             "--cpu-seconds", str(seconds), "--cpu-batch-scenes", str(batch_scenes)],
                            stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
    return proc, prefix


def finish_oracle_leg(proc, timeout):
    """the leg's last JSON line (whatever it finished within the timeout)"""
    try:
        out, _ = proc.communicate(timeout=timeout)
    except subprocess.TimeoutExpired:
        proc.kill()
        out, _ = proc.communicate()
    res = None
    for line in (out or "").splitlines():
        if line.startswith("{"):
            res = json.loads(line)
    return res or {}


def run_reference(args):
    """The reference arm: the FP64 oracle (no implementation of the paper
    exists; its single-threaded C restatement is the reference) on the
    headline workload, whole time steps from rest with the plate schedule,
    bounded in time (BF_REF_SECONDS, at least one step)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle as O
    from paper_2512_12151_b300 import scenes
    budget = float(os.environ.get("BF_REF_SECONDS", "240"))
    s = scenes.spiky_balls(precision=1)
    o = O.Oracle(s)
    n, stats = 0, []
    t0 = time.perf_counter()
    while n < max(1, args.steps):
        ts = time.perf_counter()
        o.set_dirichlet_targets(scenes.plate_targets_schedule(s, n))
        status, st = o.step(1)
        stats.append(st[0])
        n += 1
        now = time.perf_counter()
        if status != 0 or now - t0 + (now - ts) > budget:  # the next step would not end within the budget
            break
    el = time.perf_counter() - t0
    value = n / el
    sample = (f"first {n} time step(s) of the spiky-ball scene from rest (plate schedule; steps 0-1 are free of "
              f"contact), {el:.1f} s, single-threaded FP64 C oracle")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": ws,
            "steps": n, "warmup": 0, "ms_per_step": 1000.0 * el / n, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": LARGE_WORKLOAD.split(", mixed precision")[0] + ", FP64 oracle",
                       "sample": sample, "outer_iters": [x["outer_iters"] for x in stats]},
            "cpu_baseline": {"value": value, "unit": "steps/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def _progress(msg):
    sys.stderr.write(f"[bench {time.strftime('%H:%M:%S')}] {msg}\n")
    sys.stderr.flush()


def _pcts(ms):
    srt = sorted(ms)
    return srt[len(srt) // 2], srt[min(len(srt) - 1, int(round(0.99 * (len(srt) - 1))))]


def kernel_table(timers, info, nv, nt, nc, mixed, cg_iters):
    kernels = {}
    for name, (n, ms) in timers.items():
        if n == 0:
            continue
        avg_ms = ms / n
        ab = algorithmic_bytes(name, info, nv, nt, nc, mixed, cg_iters / n)
        kernels[name] = {"launches": n, "total_ms": round(ms, 3), "avg_us": round(1000 * avg_ms, 3),
                         "alg_bytes": ab, "gbs": (ab / (avg_ms / 1000.0) / 1e9) if ab else None}
    return kernels


def pcg_roofline(kernels, info, nv, nc, mixed, cg_iters, peak, peak_kind, cfg, traffic_key):
    """roofline of the persistent PCG: algorithmic bytes per launch over the
    average launch time (CUDA events on the library's stream)"""
    k = kernels.get("pcg_persistent")
    if not k:
        return None
    per_it = pcg_iteration_bytes(info["nnzb"], nv, nc, 4 if mixed else 8)
    achieved = k["gbs"]
    tr = traffic_for(traffic_key)
    top = {n: v for n, v in kernels.items() if not n.startswith("pcg_phase_")}
    return {"bound": "hbm", "kernel": "pcg_persistent", "achieved": round(achieved, 1), "peak": peak,
            "unit": "GB/s", "frac": round(achieved / peak, 4),
            "traffic": None if tr is None else round(tr * cg_iters / k["launches"]),
            "alg_bytes_per_launch": k["alg_bytes"], "alg_bytes_per_iteration": per_it,
            "iterations_per_launch": round(cg_iters / k["launches"], 1),
            "us_per_iteration": round(1000 * k["total_ms"] / max(1, cg_iters), 3),
            "share_of_kernel_time": round(k["total_ms"] / sum(v["total_ms"] for v in top.values()), 3),
            "pcg_config": cfg, "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_kind}, burst copy)",
            "traffic_note": "DRAM bytes per launch: per-iteration dram__bytes_read+write of the committed ncu "
                            "capture of this kernel source times the iterations per launch (null when the source "
                            "changed since)"}


PHASES = {"PCG": ("pcg_persistent", "spmv_bsr_contact", "pcg_update", "pcg_direction"),
          "Hess": ("elastic_grad_hess", "contact_assemble"),
          "CCD broad": ("lbvh_build", "ccd_broad_query"), "CCD narrow": ("ccd_narrow_accd",),
          "LS": ("energy",)}


def phase_split(timers, total_ms, steps):
    """ms per step by phase (the paper's Tab. 1 columns: Hess, PCG, CCD, LS,
    misc) from the per-kernel timers"""
    out, used = {}, 0.0
    for ph, names in PHASES.items():
        ms = sum(timers.get(n, (0, 0.0))[1] for n in names)
        out[ph] = round(ms / steps, 2)
        used += ms
    out["misc"] = round(max(0.0, total_ms - used) / steps, 2)
    return out


# ---------------------------------------------------------------------------
# the headline: spiky-ball compression around peak compression
# ---------------------------------------------------------------------------
def run_large(args, torch, B, scenes, stream, ws, peak, peak_kind):
    s = scenes.spiky_balls(precision=1)
    s.params.ccd_reuse = args.large_reuse
    P, N = schedule(s, scenes)
    K, W = args.steps, args.warmup
    S0 = args.large_start if args.large_start >= 0 else max(0, P - W - K // 2)
    lo, hi = S0 + W, S0 + W + K  # timed steps [lo, hi)
    assert hi <= N, "the timed window runs past the end of the plate schedule"
    sim = B.Sim(s, stream=stream.cuda_stream)
    info = sim.info()
    sched = {}

    def step(i, record=True):
        B.bf_set_obstacle_targets(sim.h, scenes.plate_targets_schedule(s, i))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        _, st = sim.step(1)
        b.record(stream)
        b.synchronize()
        if record:
            sched[i] = dict(st[0], ms=a.elapsed_time(b))
        return st[0]

    x_first = None
    t_setup = time.perf_counter()
    for i in range(lo):  # approach, then W warm-up steps
        step(i)
        if i == 0:
            x_first, _ = sim.state()
    _progress(f"large: steps 0..{lo - 1} done ({time.perf_counter() - t_setup:.0f} s)")
    if args.pcg_mode >= 0:
        tuned_mode, tuned_us = args.pcg_mode, {}
        B.bf_set_pcg_mode(sim.h, tuned_mode)
    else:
        tuned_mode, tuned_us = B.bf_autotune_pcg(sim.h, 64)
    ckpt = B.bf_save(sim.h)
    # ---- pass 1: the timed window, device-resident ----------------------
    torch.cuda.synchronize()
    barrier(ws)
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    n0 = B.bf_get_launch_count(sim.h)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    stats = []
    torch.cuda.synchronize()
    barrier(ws)
    torch.cuda.nvtx.range_push("timed_window")  # lets a profiler capture exactly these launches
    t_wall0 = time.perf_counter()
    for k, i in enumerate(range(lo, hi)):
        B.bf_set_obstacle_targets(sim.h, scenes.plate_targets_schedule(s, i))
        ev[k][0].record(stream)
        _, st = sim.step(1)
        ev[k][1].record(stream)
        stats.append(st[0])
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    torch.cuda.nvtx.range_pop()
    barrier(ws)
    clk = clocks.stop()
    launches = B.bf_get_launch_count(sim.h) - n0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    for k, i in enumerate(range(lo, hi)):
        sched[i] = dict(stats[k], ms=step_ms[k])
    total_ms = allmax(ws, sum(step_ms))
    value = allsum(ws, K) / (total_ms / 1000.0)
    p50, p99 = _pcts(step_ms)
    _progress(f"large pass 1: {value:.3f} steps/s")
    # ---- pass 2: the same window with per-kernel timers -------------------
    B.bf_load(sim.h, ckpt)
    B.bf_enable_timers(sim.h, True)
    cg2, ms2 = 0, 0.0
    for i in range(lo, hi):
        B.bf_set_obstacle_targets(sim.h, scenes.plate_targets_schedule(s, i))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        _, st = sim.step(1)
        b.record(stream)
        b.synchronize()
        cg2 += st[0]["cg_iters"]
        ms2 += a.elapsed_time(b)
    timers = B.bf_get_timers(sim.h)
    B.bf_enable_timers(sim.h, False)
    cfg = B.bf_get_pcg_config(sim.h)
    nc = statistics.mean(x["n_contacts"] for x in stats)
    kernels = kernel_table(timers, info, s.nv, s.nt, nc, True, cg2)
    roof = pcg_roofline(kernels, info, s.nv, nc, True, cg2, peak, peak_kind, cfg,
                        "pcg_persistent_sym" if cfg["resident"] == 3 else "pcg_persistent_global")
    phases = phase_split(timers, ms2, K)
    _progress("large pass 2 (per-kernel timers) done")
    # ---- pass 3: the same window end to end through bf_step_host ----------
    e2e = None
    if not args.no_e2e:
        B.bf_load(sim.h, ckpt)
        x0, v0 = sim.state()
        xin = torch.empty((s.nv, 3), dtype=torch.float64, pin_memory=True).numpy()
        vin = torch.empty((s.nv, 3), dtype=torch.float64, pin_memory=True).numpy()
        xin[:], vin[:] = x0, v0
        tg = scenes.plate_targets_schedule(s, lo)
        torch.cuda.synchronize()
        barrier(ws)
        e2e_s = 0.0
        st3 = []
        for i in range(lo, hi):
            tg = scenes.plate_targets_schedule(s, i)
            t0 = time.perf_counter()
            B.bf_set_obstacle_targets(sim.h, tg)
            st3.append(B.bf_step_host(sim.h, xin, vin, xin, vin))
            e2e_s += time.perf_counter() - t0
        e2e_s = allmax(ws, e2e_s)
        nbytes = 2 * s.nv * 3 * 8
        e2e = {"value": allsum(ws, K) / e2e_s, "unit": "steps/s", "h2d_bytes_per_step": nbytes + tg.nbytes,
               "d2h_bytes_per_step": nbytes,
               "mean_outer_iters": statistics.mean(x["outer_iters"] for x in st3),
               "mean_cg_iters_per_step": statistics.mean(x["cg_iters"] for x in st3),
               "note": "the same window replayed from a checkpoint; contact decisions may differ from pass 1 in "
                       "the last bits of FP32 vector reductions, so the iteration counts are given"}
        _progress(f"large pass 3 (end to end): {e2e['value']:.3f} steps/s")
    # ---- the release: the rest of the schedule ----------------------------
    for i in range(hi, N):
        step(i)
    sim.close()
    allms = [sched[i]["ms"] for i in sorted(sched)]
    sp50, sp99 = _pcts(allms)
    first = [sched[i]["ms"] for i in range(min(20, N)) if i in sched]
    f50, f99 = _pcts(first)
    whole = {"steps": len(allms), "steps_per_s": len(allms) / (sum(allms) / 1e3), "p50_step_ms": round(sp50, 3),
             "p99_step_ms": round(sp99, 3), "max_contacts": max(sched[i]["n_contacts"] for i in sched),
             "mean_outer_iters": round(statistics.mean(sched[i]["outer_iters"] for i in sched), 2),
             "mean_cg_iters_per_step": round(statistics.mean(sched[i]["cg_iters"] for i in sched), 1),
             "failed_steps": sum(1 for i in sched if sched[i]["status"] != 0),
             "first_20_steps": {"steps_per_s": len(first) / (sum(first) / 1e3), "p50_step_ms": round(f50, 3),
                                "p99_step_ms": round(f99, 3),
                                "max_contacts": max(sched[i]["n_contacts"] for i in range(len(first)))},
             "per_step": [[i, round(sched[i]["ms"], 1), sched[i]["outer_iters"], sched[i]["cg_iters"],
                           sched[i]["n_contacts"], round(scenes.plate_schedule_z(s, i), 4)] for i in sorted(sched)],
             "per_step_columns": ["step", "ms", "outer_iters", "cg_iters", "contacts", "plate_z_m"]}
    return {"value": value, "total_ms": total_ms, "p50": p50, "p99": p99, "stats": stats, "clocks": clk,
            "launches": launches, "t_wall": t_wall, "roofline": roof, "kernels": kernels, "phases_ms_per_step": phases,
            "e2e": e2e, "schedule": whole, "window": (lo, hi), "peak_step": P, "n_sched": N, "S0": S0,
            "tuned": (tuned_mode, tuned_us), "x_first": x_first, "diag": s.bbox_diag(), "nv": s.nv, "nt": s.nt,
            "nnzb": info["nnzb"]}


def run_large_window(args, torch, B, scenes, stream, ws, **params):
    """The headline scene with modified parameters (the CCD-reuse option, or
    the paper's CG tolerance): the same window around peak compression, the
    steps before it untimed with the same parameters, each timed step with
    CUDA events; no replays and no release."""
    s = scenes.spiky_balls(precision=1)
    for k, v in params.items():
        setattr(s.params, k, v)
    P, N = schedule(s, scenes)
    K, W = args.steps, args.warmup
    S0 = args.large_start if args.large_start >= 0 else max(0, P - W - K // 2)
    lo, hi = S0 + W, S0 + W + K
    sim = B.Sim(s, stream=stream.cuda_stream)
    for i in range(lo):
        B.bf_set_obstacle_targets(sim.h, scenes.plate_targets_schedule(s, i))
        sim.step(1)
    if args.pcg_mode >= 0:
        B.bf_set_pcg_mode(sim.h, args.pcg_mode)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    stats = []
    for k, i in enumerate(range(lo, hi)):
        B.bf_set_obstacle_targets(sim.h, scenes.plate_targets_schedule(s, i))
        ev[k][0].record(stream)
        _, st = sim.step(1)
        ev[k][1].record(stream)
        stats.append(st[0])
    torch.cuda.synchronize()
    sim.close()
    ms = [a.elapsed_time(b) for a, b in ev]
    p50, p99 = _pcts(ms)
    return {"steps": K, "timed_steps": f"{lo}..{hi - 1}",
            "steps_per_s": allsum(ws, K) / (allmax(ws, sum(ms)) / 1e3), "unit": "steps/s",
            "p50_step_ms": round(p50, 3), "p99_step_ms": round(p99, 3),
            "mean_outer_iters": statistics.mean(x["outer_iters"] for x in stats),
            "mean_cg_iters_per_step": statistics.mean(x["cg_iters"] for x in stats),
            "mean_contacts": statistics.mean(x["n_contacts"] for x in stats)}


# ---------------------------------------------------------------------------
# batched scenes over the ranks
# ---------------------------------------------------------------------------
def batched_leg(ws, rank, n_scenes, n_workers, scenes, serving, B, n_steps=10):
    """One fixed list of n_scenes seeded scenes, split over the ranks by size
    (serving.shard): each rank advances its share in mixed precision through
    the batch runner, then the same scenes in FP64 one at a time; the
    deviation of each mixed end state from the FP64 one is reported relative
    to the scene's bounding-box diagonal.  Throughputs are whole-job: steps
    summed over the ranks over the slowest rank's time."""
    sizes = [scenes.batch_scene_size(i) for i in range(n_scenes)]
    mine = serving.shard(sizes, ws)[rank]
    mix = [scenes.batch_scene(i, precision=1) for i in mine]
    batched, hs = serving.run_batched(mix, n_steps=n_steps, n_workers=n_workers)
    xm = [B.bf_get_state(h, s.nv)[0] for (h, _), s in zip(hs, mix)]
    serving.destroy(hs)
    fp64 = [scenes.batch_scene(i, precision=0) for i in mine]
    plain, hs = serving.run_sequential(fp64, n_steps=n_steps)
    dev = [float(np.abs(B.bf_get_state(h, s.nv)[0] - x).max() / s.bbox_diag()) for (h, _), s, x in zip(hs, fp64, xm)]
    serving.destroy(hs)
    batched["steps_per_s"] = allsum(ws, batched["steps"]) / allmax(ws, batched["seconds"])
    plain["steps_per_s"] = allsum(ws, plain["steps"]) / allmax(ws, plain["seconds"])
    batched["max_deviation_from_fp64"] = allmax(ws, max(dev) if dev else 0.0)
    batched["median_deviation_from_fp64_rank0"] = float(np.median(dev)) if dev else None
    batched["scenes_per_rank"] = [len(p) for p in serving.shard(sizes, ws)]
    batched["scaling"] = "strong (one fixed scene list split over the ranks)"
    batched["_mine"] = mine
    return batched, plain


def accuracy_study(mine, n, scenes, serving, B, n_steps=10):
    """Equal accuracy of the mixed batched path and the plain FP64 path on
    the first n scenes of this rank's share: (1) per step, teacher-forced:
    from each state of the FP64 trajectory one mixed step and one FP64 step,
    max |dx| / diagonal (the mixed-precision tolerance is per step, 1e-4);
    (2) free-running end states of both paths at the configured CG
    tolerance against a converged FP64 reference (CG tolerance 1e-10)."""
    tf, dm, d64 = 0.0, [], []
    for i in mine[:n]:
        s64, s32 = scenes.batch_scene(i, precision=0), scenes.batch_scene(i, precision=1)
        sref = scenes.batch_scene(i, precision=0)
        sref.params.cg_tol = 1e-10
        (h64, _k1), (h32, _k2), (hr, _k3) = serving.create(s64), serving.create(s32), serving.create(sref)
        try:
            B.bf_step(hr, n_steps, ok=tuple(B.STATUS))
            xr = B.bf_get_state(hr, sref.nv)[0]
            for _ in range(n_steps):
                x, v = B.bf_get_state(h64, s64.nv)
                keys, lam, gam = B.bf_get_active_set(h64)
                B.bf_set_state(h32, x, v)
                B.bf_set_active_set(h32, keys, lam, gam)
                B.bf_step(h64, 1, ok=tuple(B.STATUS))
                B.bf_step(h32, 1, ok=tuple(B.STATUS))
                tf = max(tf, float(np.abs(B.bf_get_state(h32, s32.nv)[0] - B.bf_get_state(h64, s64.nv)[0]).max()
                                   / s64.bbox_diag()))
            x64 = B.bf_get_state(h64, s64.nv)[0]
        finally:
            for h in (h64, h32, hr):
                B.bf_scene_destroy(h)
        # the free-running mixed end state: a fresh mixed run (as in the batch)
        hm, _k4 = serving.create(s32)
        B.bf_step(hm, n_steps, ok=tuple(B.STATUS))
        xm = B.bf_get_state(hm, s32.nv)[0]
        B.bf_scene_destroy(hm)
        dm.append(float(np.abs(xm - xr).max() / s64.bbox_diag()))
        d64.append(float(np.abs(x64 - xr).max() / s64.bbox_diag()))

    def stats(d):
        d = np.asarray(d)
        return {"median": float(np.median(d)), "p90": float(np.percentile(d, 90)), "max": float(d.max()),
                "scenes_above_1e-4": int((d > 1e-4).sum())}
    return {"scenes": len(dm), "teacher_forced_per_step_max_mixed_vs_fp64": tf,
            "free_running_vs_converged_fp64": {"mixed": stats(dm), "fp64": stats(d64)},
            "note": "per step: one mixed and one FP64 step from each state of the FP64 trajectory, max |dx| / "
                    "bbox diagonal over the scenes and 10 steps; free running: 10 steps from rest at CG tolerance "
                    "1e-6 against FP64 at 1e-10, per scene max |dx| / bbox diagonal (stacked cubes whose contact "
                    "decisions flip spread most, in either precision)"}


# ---------------------------------------------------------------------------
# the eight-cube scene (L2-resident system)
# ---------------------------------------------------------------------------
def run_eight(args, torch, B, scenes, stream, flush, ws, peak, peak_kind, seed):
    W, K = args.warmup, args.steps

    def make(precision=1):
        s = scenes.eight_cubes(seed, precision=precision)
        return s, B.Sim(s, stream=stream.cuda_stream)

    s, sim = make()
    info = sim.info()
    for _ in range(W):
        sim.step(1)
    tuned_mode, tuned_us = ((args.pcg_mode, {}) if args.pcg_mode >= 0 else B.bf_autotune_pcg(sim.h, 64))
    B.bf_set_pcg_mode(sim.h, tuned_mode)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    stats = []
    torch.cuda.synchronize()
    barrier(ws)
    torch.cuda.nvtx.range_push("eight_cubes_window")
    for i in range(K):
        with torch.cuda.stream(stream):
            flush.zero_()
        ev[i][0].record(stream)
        _, st = sim.step(1)
        ev[i][1].record(stream)
        stats.append(st[0])
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    sim.close()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = allmax(ws, sum(step_ms))
    value = allsum(ws, K) / (total_ms / 1000.0)
    p50, p99 = _pcts(step_ms)
    # pass 2: per-kernel timers
    s2, sim2 = make()
    B.bf_set_pcg_mode(sim2.h, tuned_mode)
    for _ in range(W):
        sim2.step(1)
    B.bf_enable_timers(sim2.h, True)
    cg2 = 0
    for i in range(K):
        with torch.cuda.stream(stream):
            flush.zero_()
        _, st2 = sim2.step(1)
        cg2 += st2[0]["cg_iters"]
    timers = B.bf_get_timers(sim2.h)
    cfg = B.bf_get_pcg_config(sim2.h)
    sim2.close()
    nc = statistics.mean(x["n_contacts"] for x in stats)
    kernels = kernel_table(timers, info, s.nv, s.nt, nc, True, cg2)
    roof = pcg_roofline(kernels, info, s.nv, nc, True, cg2, peak, peak_kind, cfg, "pcg_persistent")
    if roof:
        roof["note"] = ("the matrix stays in shared memory for the whole solve, so per-iteration DRAM traffic is "
                        "far below the algorithmic bytes; latency bounds it: the grid-wide reductions (one per "
                        "iteration in the single-reduction form, variant 4; two in the two-reduction form, "
                        "variant 1) and the L2 round trips of the window stage")
    # pass 3: end to end with host buffers; the positions after each step
    # give the free-running error curve against the stored oracle trajectory
    g = np.load(GOLDEN)
    ids, traj = g["sample_ids"], g["traj"]
    s3, sim3 = make()
    B.bf_set_pcg_mode(sim3.h, tuned_mode)
    xin = torch.empty((s3.nv, 3), dtype=torch.float64, pin_memory=True).numpy()
    vin = torch.empty((s3.nv, 3), dtype=torch.float64, pin_memory=True).numpy()
    xin[:], vin[:] = s3.x0, s3.v0
    curve = []
    e2e_s = 0.0
    for i in range(W + K):
        if i >= W:
            with torch.cuda.stream(stream):
                flush.zero_()
            torch.cuda.synchronize()
        t0 = time.perf_counter()
        B.bf_step_host(sim3.h, xin, vin, xin, vin)
        if i >= W:
            e2e_s += time.perf_counter() - t0
        if seed == 0 and i < len(traj):
            curve.append(float(np.abs(xin[ids] - traj[i]).max() / s3.bbox_diag()))
    sim3.close()
    e2e_s = allmax(ws, e2e_s)
    nbytes = 2 * s3.nv * 3 * 8
    e2e = {"value": allsum(ws, K) / e2e_s, "unit": "steps/s", "h2d_bytes_per_step": nbytes,
           "d2h_bytes_per_step": nbytes}
    # teacher-forced: two steps from the oracle's stored state after 16 steps
    s4, sim4 = make()
    B.bf_set_state(sim4.h, g["x16"], g["v16"])
    B.bf_set_active_set(sim4.h, g["keys16"], g["lam16"], g["gam16"])
    tf = []
    for _ in range(2):
        sim4.step(1)
        tf.append(sim4.state()[0])
    sim4.close()
    return {"value": value, "total_ms": total_ms, "p50": p50, "p99": p99, "stats": stats, "roofline": roof,
            "kernels": kernels, "e2e": e2e, "curve": curve, "teacher_forced_x": tf, "diag": s.bbox_diag(),
            "tuned": (tuned_mode, tuned_us)}


def run_two(torch, B, scenes, stream, flush, ws):
    """The small plain-FP64 configuration: two cubes (4^3 cells, 384 tets
    each), all 20 steps from rest, each timed with CUDA events after the L2
    flush; the positions after each step for the comparison with the
    oracle's run of the same steps."""
    s = scenes.two_cubes(0)
    sim = B.Sim(s, stream=stream.cuda_stream)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(s.n_steps)]
    xs, stats = [], []
    for i in range(s.n_steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        ev[i][0].record(stream)
        _, st = sim.step(1)
        ev[i][1].record(stream)
        stats.append(st[0])
        xs.append(sim.state()[0])
    torch.cuda.synchronize()
    sim.close()
    ms = [a.elapsed_time(b) for a, b in ev]
    p50, p99 = _pcts(ms)
    return {"workload": "two_cubes: 2 cubes x 4^3 cells (768 tets, 250 verts), the upper 1 mm above the lower, "
                        "falling onto a static ground quad; SNH E=1e5 nu=0.4 rho=1000, h=0.01, delta=1e-3, CG tol "
                        "1e-6, FP64 throughout; all 20 steps from rest, L2 flushed before each",
            "steps": s.n_steps, "steps_per_s": allsum(ws, s.n_steps) / (allmax(ws, sum(ms)) / 1e3), "unit": "steps/s",
            "p50_step_ms": round(p50, 3), "p99_step_ms": round(p99, 3),
            "mean_outer_iters": statistics.mean(x["outer_iters"] for x in stats),
            "max_contacts": max(x["n_contacts"] for x in stats), "_x": np.array(xs), "_diag": s.bbox_diag()}


def run_variant(args, seed, ws, B, scenes, stream, flush, workload, K, W, **params):
    """The eight-cube scene with modified parameters (friction, material),
    mixed precision: W warm-up steps, then each step timed with CUDA events
    after the L2 flush, like the main line."""
    import torch
    s = scenes.eight_cubes(seed, precision=args.precision)
    for k, v in params.items():
        setattr(s.params, k, v)
    sim = B.Sim(s, stream=stream.cuda_stream)
    for _ in range(W):
        sim.step(1)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    stats = []
    for i in range(K):
        with torch.cuda.stream(stream):
            flush.zero_()
        ev[i][0].record(stream)
        _, st = sim.step(1)
        ev[i][1].record(stream)
        stats.append(st[0])
    torch.cuda.synchronize()
    sim.close()
    ms = sorted(a.elapsed_time(b) for a, b in ev)
    total = allmax(ws, sum(ms))
    return {"workload": f"{workload}, steps {W}..{W + K - 1} from rest, mixed precision",
            "steps": K, "steps_per_s": allsum(ws, K) / (total / 1000.0), "unit": "steps/s",
            "p50_step_ms": round(ms[len(ms) // 2], 3), "p99_step_ms": round(ms[-1], 3),
            "mean_outer_iters": statistics.mean(x["outer_iters"] for x in stats),
            "mean_cg_iters_per_step": statistics.mean(x["cg_iters"] for x in stats),
            "mean_contacts": statistics.mean(x["n_contacts"] for x in stats)}


def main():
    import faulthandler
    import signal
    faulthandler.register(signal.SIGUSR1, all_threads=True)  # `kill -USR1` prints every thread's stack
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=30.0,
                    help="oracle budget on the spiky-ball scene (at least one whole step is always timed)")
    ap.add_argument("--cpu-batch-scenes", type=int, default=64,
                    help="batched scenes the oracle runs one per host core for the batched line's CPU baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--precision", type=int, default=1)
    ap.add_argument("--large-start", type=int, default=-1,
                    help="first warm-up step of the spiky-ball window (default: the window centred on peak "
                         "compression)")
    ap.add_argument("--large-reuse", type=int, default=0, help="headline with the CCD-reuse option")
    ap.add_argument("--large-reuse-line", type=int, default=1,
                    help="the headline window again with the CCD-reuse option, as an extra line (0: skip)")
    ap.add_argument("--large-tol-line", type=int, default=1,
                    help="the headline window again at the paper's CG tolerance 1e-4, as an extra line (0: skip)")
    ap.add_argument("--eight-cubes", type=int, default=1, help="the eight-cube line (0: skip)")
    ap.add_argument("--two-cubes", type=int, default=1, help="the two-cube FP64 line (0: skip)")
    ap.add_argument("--batched-scenes", type=int, default=256,
                    help="independent scenes of 1k-20k tets for the batched line, split over the ranks (0: skip)")
    ap.add_argument("--batch-workers", type=int, default=16)
    ap.add_argument("--accuracy-scenes", type=int, default=32,
                    help="batched scenes of the equal-accuracy study (mixed vs FP64 vs converged FP64; 0: skip)")
    ap.add_argument("--serve-requests", type=int, default=200, help="requests of the served stream (0: skip)")
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-workers", type=int, default=32)
    ap.add_argument("--serve-sweep-requests", type=int, default=100,
                    help="requests per arrival rate of the sustainable-rate sweep")
    ap.add_argument("--variant-steps", type=int, default=20,
                    help="timed steps of each eight-cube variant: friction, COR, NH, CCD reuse, CG tol 1e-4 "
                         "(0: skip)")
    ap.add_argument("--pcg-mode", type=int, default=-1,
                    help="fixed PCG execution configuration (bf_set_pcg_mode) instead of the autotuner's choice; "
                         "for runs under a profiler, whose serialised launches distort the tuner's timings")
    ap.add_argument("--oracle-leg", default=None, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.oracle_leg:
        return oracle_leg(args.oracle_leg, args.cpu_seconds, args.cpu_batch_scenes)
    if args.impl == "reference":
        return run_reference(args)
    args.warmup = max(args.warmup, 3)
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    leg = None
    if rank == 0 and ws == 1 and args.cpu_seconds > 0:  # before any CUDA call
        leg = start_oracle_leg(args.cpu_seconds, args.cpu_batch_scenes)

    ws, rank, local = dist_init(args)
    import torch
    from paper_2512_12151_b300 import binding as B
    from paper_2512_12151_b300 import build as build_mod
    from paper_2512_12151_b300 import scenes
    if not os.path.exists(B.LIB_PATH):
        build_mod.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    peak, peak_kind = load_peaks()
    K, W = args.steps, args.warmup

    # ---- headline: the spiky-ball compression ------------------------------
    L = run_large(args, torch, B, scenes, stream, ws, peak, peak_kind)
    lo, hi = L["window"]
    _progress(f"large: {L['value']:.3f} steps/s over steps {lo}..{hi - 1}; whole schedule "
              f"{L['schedule']['steps_per_s']:.3f} steps/s")

    # ---- the headline scene with the CCD-reuse option ------------------------
    LR = None
    if args.large_reuse_line:
        LR = run_large_window(args, torch, B, scenes, stream, ws, ccd_reuse=1)
        LR["workload"] = ("the spiky-ball compression with the CCD-reuse option (one CCD per outer iteration serves "
                          "UpdateActiveSet and MaxStepSize), the same window, mixed precision")
        _progress(f"large with CCD reuse: {LR['steps_per_s']:.3f} steps/s")
    LT = None
    if args.large_tol_line:
        LT = run_large_window(args, torch, B, scenes, stream, ws, cg_tol=1e-4)
        LT["workload"] = ("the spiky-ball compression at the paper's CG relative tolerance 1e-4 (the headline uses "
                          "1e-6), every step up to the window at that tolerance, the same window, mixed precision")
        _progress(f"large at CG tolerance 1e-4: {LT['steps_per_s']:.3f} steps/s")

    # ---- the two-cube scene, FP64 (the small configuration) --------------------
    T = run_two(torch, B, scenes, stream, flush, ws) if args.two_cubes else None

    # ---- the eight-cube scene ------------------------------------------------
    E = run_eight(args, torch, B, scenes, stream, flush, ws, peak, peak_kind, rank) if args.eight_cubes else None
    if E:
        _progress(f"eight cubes: {E['value']:.1f} steps/s")

    # ---- batched scenes (one fixed list split over the ranks), the plain FP64
    # path one scene at a time on the same scenes, and their deviation ------
    batched = plain = None
    if args.batched_scenes > 0:
        from paper_2512_12151_b300 import serving
        batched, plain = batched_leg(ws, rank, args.batched_scenes, args.batch_workers, scenes, serving, B)
        if args.accuracy_scenes > 0:
            batched["equal_accuracy"] = accuracy_study(batched["_mine"], args.accuracy_scenes, scenes, serving, B)
        del batched["_mine"]
        _progress(f"batched: {batched['steps_per_s']:.1f} steps/s, plain FP64 {plain['steps_per_s']:.1f}; "
                  f"max deviation {batched['max_deviation_from_fp64']:.2e} x diagonal")

    # ---- served request stream and its FP64 one-at-a-time baseline --------
    served = None
    if args.serve_requests > 0:
        from paper_2512_12151_b300 import serving
        reqs = serving.poisson_requests(args.serve_requests, args.serve_rate, seed=1000 + rank)
        served = serving.serve(reqs, n_steps=10, n_workers=args.serve_workers)
        served["steps_per_s"] = allsum(ws, served["steps"]) / allmax(ws, served["seconds"])
        base = [scenes.batch_scene(r[1], r[2], r[3], precision=0) for r in reqs]
        pl, hs = serving.run_sequential(base, n_steps=10)
        serving.destroy(hs)
        served["plain_fp64_same_requests"] = dict(
            pl, steps_per_s=allsum(ws, pl["steps"]) / allmax(ws, pl["seconds"]),
            workload="the same request list in FP64, one scene at a time on one stream (no arrival waits)")
        cap = served["steps_per_s"] / 10.0  # requests/s the served run completed
        sweep = serving.rate_sweep([round(f * cap, 1) for f in (0.5, 0.75, 1.0, 1.5)], args.serve_sweep_requests,
                                   n_steps=10, n_workers=args.serve_workers, seed=2000 + rank)
        served["sustainable_rate_per_s"] = sweep["sustainable_rate_per_s"]
        served["rate_sweep"] = sweep
        _progress(f"served: {served['steps_per_s']:.1f} steps/s (FP64 one at a time "
                  f"{served['plain_fp64_same_requests']['steps_per_s']:.1f})")

    variants = {}
    if args.variant_steps > 0:
        Wv = max(args.warmup, 15)  # from step 15 on the cubes are in contact
        for key, text, prm in (
                ("friction", "the eight-cube scene (196,608 tets) with the friction of appendix A: mu_f = 0.5, "
                             "eps_v = 1e-3 m/s, K_min = 6", dict(mu_f=0.5, eps_v=1e-3, k_min=6)),
                ("cor", "the eight-cube scene (196,608 tets) with the corotated material (COR)", dict(model=1)),
                ("nh", "the eight-cube scene (196,608 tets) with the Neo-Hookean material (NH) and the inversion "
                       "bound of MaxStepSize", dict(model=2)),
                ("ccd_reuse", "the eight-cube scene (196,608 tets) with the CCD-reuse option (one CCD per outer "
                              "iteration serves UpdateActiveSet and MaxStepSize)", dict(ccd_reuse=1)),
                ("cg_tol_1e-4", "the eight-cube scene (196,608 tets) at the paper's CG relative tolerance 1e-4 "
                                "(the configured workload uses 1e-6)", dict(cg_tol=1e-4))):
            variants[key] = run_variant(args, rank, ws, B, scenes, stream, flush, text, args.variant_steps, Wv,
                                        **prm)
            _progress(f"{key}: {variants[key]['steps_per_s']:.1f} steps/s")

    # ---- the oracle leg: CPU baseline and errors against FP64 --------------
    leg_res = {}
    if leg is not None:
        proc, prefix = leg
        open(prefix + "_go", "w").close()
        leg_res = finish_oracle_leg(proc, timeout=900)
    cpu = large_err = None
    eight_cpu = eight_err = None
    if "large" in leg_res:
        r = leg_res["large"]
        cpu = {"value": r["value"], "unit": "steps/s", "cores": 1, "kind": "oracle",
               "sample": f"first {r['steps']} time step(s) of the spiky-ball scene from rest with the plate "
                         f"schedule ({r['seconds']:.1f} s, single-threaded FP64 C oracle, concurrent with the GPU "
                         "runs; these steps have no contacts, so the sample overstates its rate in the timed "
                         "window)", "outer_iters": r["outer_iters"]}
        try:
            xo = np.load(prefix + "_large_x1.npy")
            large_err = float(np.abs(L["x_first"] - xo).max() / L["diag"])
        except OSError:
            pass
    if T:
        T["cpu_baseline"] = None
        if "two" in leg_res:
            r = leg_res["two"]
            T["cpu_baseline"] = {"value": r["value"], "unit": "steps/s", "cores": 1, "kind": "oracle",
                                 "sample": f"the same 20 steps from rest ({r['seconds']:.2f} s, single-threaded FP64 "
                                           "C oracle)"}
            try:
                xo = np.load(prefix + "_two.npy")
                err = [float(np.abs(T["_x"][i] - xo[i]).max() / T["_diag"]) for i in range(len(xo))]
                T["error_vs_fp64_oracle"] = {"free_running_per_step": [float("%.3g" % e) for e in err],
                                             "max": max(err), "bound": 1e-6,
                                             "note": "max |x_gpu - x_oracle| / bbox diagonal after each step, "
                                                     "both from rest"}
            except OSError:
                pass
        del T["_x"], T["_diag"]
    if "eight" in leg_res and E:
        r = leg_res["eight"]
        eight_cpu = {"value": r["value"], "unit": "steps/s", "cores": 1, "kind": "oracle",
                     "sample": f"steps {r['steps']} of the eight-cube scene from the oracle's own stored state "
                               f"(contact: {r['contacts']} pairs; {r['seconds']:.1f} s, single-threaded FP64 C "
                               "oracle); inside the GPU line's timed window"}
        try:
            g = np.load(prefix + "_eight.npz")
            eight_err = [float(np.abs(E["teacher_forced_x"][k] - g[n]).max() / E["diag"])
                         for k, n in ((0, "x17"), (1, "x18"))]
        except OSError:
            pass

    if leg is not None:  # the leg's files are read: remove its temporary directory
        import shutil
        shutil.rmtree(os.path.dirname(leg[1]), ignore_errors=True)
    if rank == 0:
        stats = L["stats"]
        line = {"metric": METRIC, "value": L["value"], "unit": "steps/s", "n_gpus": ws, "steps": K, "warmup": W,
                "ms_per_step": L["total_ms"] / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32+f64 (mixed)", "data": "synthetic",
                "config": {"workload": LARGE_WORKLOAD,
                           "timed_steps": f"{lo}..{hi - 1} (steps 0..{L['S0'] - 1} advance untimed to the window, "
                                          f"{L['S0']}..{lo - 1} are the warm-up; the plate is lowest, at 30 % of "
                                          f"its starting height, at the end of step {L['peak_step']})",
                           "l2": "not flushed: the scene's device working set (about 1.1 GB) is larger than L2",
                           "parallelism": f"{ws} independent replica(s), one per GPU",
                           "tets": L["nt"], "vertices": L["nv"], "upper_blocks": L["nnzb"],
                           "p50_step_ms": round(L["p50"], 3), "p99_step_ms": round(L["p99"], 3),
                           "wall_s": round(L["t_wall"], 3),
                           "mean_outer_iters": statistics.mean(x["outer_iters"] for x in stats),
                           "mean_cg_iters_per_step": statistics.mean(x["cg_iters"] for x in stats),
                           "mean_contacts": statistics.mean(x["n_contacts"] for x in stats),
                           "max_contacts": max(x["n_contacts"] for x in stats),
                           "phases_ms_per_step": L["phases_ms_per_step"],
                           "pcg_autotune": {"best_mode": L["tuned"][0],
                                            "us_per_iteration_by_mode": {str(k): round(v, 3)
                                                                         for k, v in L["tuned"][1].items()}}},
                "roofline": L["roofline"], "kernels": L["kernels"], "cpu_baseline": cpu, "e2e": L["e2e"],
                "error_vs_fp64_oracle": {"first_step_max_vertex_error_over_bbox_diag": large_err,
                                         "note": "GPU mixed precision vs the FP64 oracle after step 0 of the "
                                                 "spiky-ball scene from the same start"},
                "large_whole_schedule": dict(L["schedule"], workload="the same scene, every step of the plate "
                                             "schedule (approach, the window of pass 1, the release), each timed "
                                             "with CUDA events"),
                "gpu_launches": int(L["launches"]), "clocks": L["clocks"]}
        if E:
            st = E["stats"]
            line["eight_cubes"] = {
                "workload": EIGHT_WORKLOAD, "value": E["value"], "unit": "steps/s",
                "timed_steps": f"{W}..{W + K - 1}", "l2": "flushed (512 MiB write) before each timed step",
                "ms_per_step": E["total_ms"] / K, "p50_step_ms": round(E["p50"], 3), "p99_step_ms": round(E["p99"], 3),
                "mean_outer_iters": statistics.mean(x["outer_iters"] for x in st),
                "mean_cg_iters_per_step": statistics.mean(x["cg_iters"] for x in st),
                "mean_contacts": statistics.mean(x["n_contacts"] for x in st),
                "roofline": E["roofline"], "kernels": E["kernels"], "e2e": E["e2e"], "cpu_baseline": eight_cpu,
                "error_vs_fp64_oracle": {
                    "free_running_per_step": [float("%.3g" % e) for e in E["curve"]],
                    "free_running_note": "max over 1,024 sampled vertices of |x_gpu - x_oracle| / bbox diagonal "
                                         "after each step from rest (steps 0..%d; the oracle's trajectory is "
                                         "stored in tests/golden/eight_cubes_oracle.npz)" % (len(E["curve"]) - 1),
                    "teacher_forced_steps_16_17": eight_err,
                    "teacher_forced_note": "max over all vertices of |x_gpu - x_oracle| / bbox diagonal after one "
                                           "and two steps from the oracle's stored state after 16 steps (in "
                                           "contact); the bound is 1e-4"},
                "pcg_autotune": {"best_mode": E["tuned"][0],
                                 "us_per_iteration_by_mode": {str(k): round(v, 3) for k, v in E["tuned"][1].items()}}}
        if LR:
            line["large_ccd_reuse"] = LR
        if LT:
            line["large_cg_tol_1e-4"] = LT
        if T:
            line["two_cubes_fp64"] = T
        if batched:
            if "batched" in leg_res:
                r = leg_res["batched"]
                batched["cpu_baseline"] = {
                    "value": r["value"], "unit": "steps/s", "cores": r["cores"], "kind": "oracle",
                    "sample": f"the first {r['scenes']} scenes of the list, 10 steps each, one scene per host core "
                              f"({r['seconds']:.1f} s; spawned single-threaded FP64 C oracle processes, run after the "
                              "GPU lines)"}
            line["batched"] = dict(
                batched, workload=f"{args.batched_scenes} independent scenes (seeded; split over the ranks by size): "
                "1k-20k tets log-uniform, one cube or a stack of two on a ground quad, E log-uniform 1e4-1e6 Pa, "
                "nu U(0.3, 0.45), h = 0.01 s, 10 steps each, mixed precision, "
                f"{args.batch_workers} streams per GPU (native batch runner); deviation = max |x_mixed - x_fp64| "
                "/ bbox diagonal of each scene's end state against the same scene in FP64", unit="steps/s")
            line["plain_fp64_one_at_a_time"] = dict(plain, workload="the same scenes in FP64, one scene at a time "
                                                    "on one stream", unit="steps/s")
            line["batched_vs_plain_fp64"] = batched["steps_per_s"] / plain["steps_per_s"]
        if served:
            if "served" in leg_res:
                r = leg_res["served"]
                served["cpu_baseline"] = {
                    "value": r["value"], "unit": "steps/s", "cores": r["cores"], "kind": "oracle",
                    "sample": f"the first {r['requests']} requests of the list, 10 steps each, one scene per host "
                              f"core ({r['seconds']:.1f} s, until the largest finished; spawned single-threaded "
                              "FP64 C oracle processes, run after the GPU lines, no arrival waits)"}
            line["serving"] = dict(
                served, workload=f"{args.serve_requests} requests per GPU, Poisson arrivals at {args.serve_rate:g}/s, "
                "scenes 2k-200k tets log-uniform (same generator), 10 steps each, mixed precision, HBM budget "
                "150 GB, scenes generated and created inside the served loop by 8 host threads", unit="steps/s")
        line.update(variants)
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
