"""Many independent scenes through the native batch runner (bf_batch_*):
batched runs, a served request stream, the one-scene-at-a-time baseline,
and the size-balanced split of scenes across GPUs.

Host orchestration only: every time step runs in the library (the batch
runner's worker threads call the same step as bf_step, on their own CUDA
streams).  Scenes are created without the torch allocator, so their memory
comes from the device's stream-ordered pool and they can move between
streams.
"""
from __future__ import annotations

import math
import threading
import time

import numpy as np

from . import binding as B
from . import scenes


def create(scene, params=None):
    """(handle, keep-alive) of a scene on the default stream, pool memory"""
    return B.bf_scene_create(scene, params if params is not None else scene.params, None, None)


def shard(sizes, world):
    """Size-balanced split of scene indices over `world` ranks: largest
    first, each to the currently least-loaded rank (ties: lower rank)."""
    order = sorted(range(len(sizes)), key=lambda i: (-sizes[i], i))
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += sizes[i]
    return [sorted(p) for p in parts]


def _latencies(res):
    """per-step latencies of one finished ticket: step completion minus the
    previous step's completion (the first: minus admission)"""
    t = res["t_steps"]
    prev = np.concatenate([[res["t_admit"]], t[:-1]])
    return t - prev


def _summary(lat, steps, elapsed):
    lat = np.asarray(lat)
    return {"steps": int(steps), "seconds": elapsed, "steps_per_s": steps / elapsed if elapsed > 0 else None,
            "p50_step_ms": float(np.percentile(lat, 50) * 1e3) if len(lat) else None,
            "p99_step_ms": float(np.percentile(lat, 99) * 1e3) if len(lat) else None}


def _wait(b, t, deadline):
    """waits for a ticket, raising once the monotonic deadline has passed"""
    while not B.bf_batch_wait(b, t, 1000):
        if time.monotonic() > deadline:
            raise TimeoutError(f"batch ticket {t} did not finish in time")


def run_batched(scene_list, n_steps=None, n_workers=16, budget_bytes=150 << 30, timeout_s=900.0, autotune=False):
    """Creates every scene (untimed), then admits them all at once to a batch
    and runs them to completion.  Returns throughput and per-step latency
    (from the admission of all scenes); with `autotune`, the batch tunes the
    PCG configuration per size bucket and the result lists the choices."""
    handles = [create(s) for s in scene_list]
    b = B.bf_batch_create(n_workers, budget_bytes)
    if autotune:
        B.bf_batch_set_autotune(b, True)
    try:
        t0 = B.bf_batch_now(b)
        tickets = []
        for (h, _), s in zip(handles, scene_list):
            t = B.bf_batch_admit(b, h, n_steps or s.n_steps)
            if t is None:
                raise RuntimeError("batch admission refused by the HBM budget")
            tickets.append(t)
        deadline = time.monotonic() + timeout_s
        for t in tickets:
            _wait(b, t, deadline)
        lat, steps, t_end, bad = [], 0, t0, 0
        for t, s in zip(tickets, scene_list):
            r = B.bf_batch_result(b, t, n_steps or s.n_steps)
            bad += r["status"] != 0
            lat.extend(_latencies(r))
            steps += r["steps_done"]
            t_end = max(t_end, float(r["t_steps"][-1]) if len(r["t_steps"]) else t_end)
            B.bf_batch_release(b, t)
        out = _summary(lat, steps, t_end - t0)
        out.update({"workers": n_workers, "scenes": len(scene_list), "failed": bad})
        if autotune:
            out["pcg_mode_by_size_bucket"] = {str(k): v for k, v in B.bf_batch_tuned(b).items()}
        return out, handles
    finally:
        B.bf_batch_destroy(b)


def run_sequential(scene_list, n_steps=None):
    """The baseline: one scene at a time, every step on the default stream."""
    handles = [create(s) for s in scene_list]
    lat, steps, bad = [], 0, 0
    t0 = time.perf_counter()
    for (h, _), s in zip(handles, scene_list):
        for _ in range(n_steps or s.n_steps):
            a = time.perf_counter()
            st, _ = B.bf_step(h, 1, ok=tuple(B.STATUS))
            lat.append(time.perf_counter() - a)
            steps += 1
            if st != 0:
                bad += 1
                break
    out = _summary(lat, steps, time.perf_counter() - t0)
    out.update({"scenes": len(scene_list), "failed": bad})
    return out, handles


def evict(h):
    """Checkpoint of a scene (bf_save) whose device memory is then freed;
    the scene must not be running in a batch."""
    blob = B.bf_save(h)
    B.bf_scene_destroy(h)
    return blob


def restore(scene, blob, params=None):
    """(handle, keep-alive) of a scene re-created from its mesh and resumed
    from a checkpoint made by evict"""
    h, keep = create(scene, params)
    try:
        B.bf_load(h, blob)
    except Exception:
        B.bf_scene_destroy(h)
        raise
    return h, keep


def destroy(handles):
    for h, _ in handles:
        B.bf_scene_destroy(h)


def poisson_requests(n, rate, seed=0, t_lo=2e3, t_hi=2e5, precision=1):
    """n requests: seeded exponential inter-arrival gaps (mean 1/rate s), each
    a batch_scene drawn log-uniformly in [t_lo, t_hi] tets"""
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n))
    return [(float(a), int(rng.integers(1 << 30)), t_lo, t_hi, precision) for a in arrivals]


def waits_bounded(w):
    """Whether admission waits (in arrival order) stay bounded over a run:
    below a saturated server they grow with every request, so the mean wait
    of the last third of the requests exceeds twice that of the first third
    (plus 50 ms for the jitter of scene creation)."""
    n = len(w) // 3
    if n == 0:
        return True
    return bool(np.mean(w[-n:]) <= 2.0 * np.mean(w[:n]) + 0.05)


def rate_sweep(rates, n_requests, n_steps=10, n_workers=16, seed=0, **kw):
    """Serves `n_requests` requests at each arrival rate; per rate the
    throughput, admission waits and whether they stay bounded, and the
    highest rate at which they do (the sustainable rate, None if none)"""
    runs = []
    for r in rates:
        res = serve(poisson_requests(n_requests, r, seed=seed), n_steps=n_steps, n_workers=n_workers, **kw)
        runs.append({"rate_per_s": r, "steps_per_s": res["steps_per_s"],
                     "p50_step_ms": res["p50_step_ms"], "p99_step_ms": res["p99_step_ms"],
                     "admission_wait_p50_ms": res["admission_wait_p50_ms"],
                     "admission_wait_p99_ms": res["admission_wait_p99_ms"],
                     "bounded": res["admission_wait_bounded"], "failed": res["failed"]})
    ok = [x["rate_per_s"] for x in runs if x["bounded"] and x["failed"] == 0]
    return {"sustainable_rate_per_s": max(ok) if ok else None, "runs": runs, "requests_per_rate": n_requests}


def serve(requests, n_steps=10, n_workers=16, budget_bytes=150 << 30, poll_s=0.002, timeout_s=900.0,
          n_creators=8, blocking_sync=False, keep_states=()):
    """Serves a request stream: at each arrival time the request is handed
    to one of `n_creators` host threads, which generates and creates its
    scene and admits it to the running batch (waiting while the HBM budget
    refuses it); finished scenes are released and destroyed as they
    complete.  Returns aggregate steps/s (first arrival to last completion),
    per-step latency p50/p99 (completion of a step minus completion of the
    scene's previous step, or its admission) and the admission wait
    (admission minus arrival, scene creation included) p50/p99.  With
    `blocking_sync` the batch's worker threads sleep in their waits
    (bf_batch_set_blocking_sync): shorter step latency, longer admission.
    For the request indices in `keep_states` the result also holds the end
    positions (`states`) and how many other scenes were in the batch when
    each was admitted (`live_at_admission`)."""
    from concurrent.futures import ThreadPoolExecutor
    b = B.bf_batch_create(n_workers, budget_bytes)
    if blocking_sync:  # worker threads sleep in their waits, leaving host cores to the creators
        B.bf_batch_set_blocking_sync(b, True)
    deadline = time.monotonic() + timeout_s
    live = {}  # ticket -> (handle, keep, request index, vertices)
    lat, waits, steps, bad, statuses = [], [], 0, 0, []
    states, live_at = {}, {}
    t_gen, t_create = [], []  # host seconds per request: mesh generation, bf_scene_create
    keep_states = set(keep_states)
    lock = threading.Lock()
    t0 = B.bf_batch_now(b)

    def admit(idx, req):
        arrival, seed, t_lo, t_hi, prec = req
        c0 = time.perf_counter()
        s = scenes.batch_scene(seed, t_lo, t_hi, precision=prec)
        c1 = time.perf_counter()
        h, keep = create(s)
        c2 = time.perf_counter()
        with lock:
            t_gen.append(c1 - c0)
            t_create.append(c2 - c1)
        while True:
            with lock:
                n_live = len(live)
                t = B.bf_batch_admit(b, h, n_steps)
                if t is not None:
                    waits.append((arrival, B.bf_batch_now(b) - t0 - arrival))
                    live[t] = (h, keep, idx, s.nv)
                    if idx in keep_states:
                        live_at[idx] = n_live
                    break
            if time.monotonic() > deadline:
                B.bf_scene_destroy(h)
                raise TimeoutError("admission kept being refused by the HBM budget")
            time.sleep(poll_s)

    def reap(block=False):
        nonlocal steps, bad
        with lock:
            tickets = list(live)
        for t in tickets:
            if block:
                _wait(b, t, deadline)
            elif not B.bf_batch_wait(b, t, 0):
                continue
            r = B.bf_batch_result(b, t, n_steps)
            with lock:
                h, _keep, idx, nv = live.pop(t)
            if idx in keep_states:
                states[idx] = B.bf_get_state(h, nv)[0]
            with lock:
                lat.extend(_latencies(r))
                steps += r["steps_done"]
                bad += r["status"] != 0
                if r["status"] != 0:
                    statuses.append(int(r["status"]))
            B.bf_batch_release(b, t)
            B.bf_scene_destroy(h)

    pool = ThreadPoolExecutor(max_workers=n_creators)
    try:
        futures = []
        for idx, req in enumerate(requests):
            while B.bf_batch_now(b) - t0 < req[0]:
                reap()
                time.sleep(min(poll_s, max(0.0, req[0] - (B.bf_batch_now(b) - t0))))
            futures.append(pool.submit(admit, idx, req))
        for f in futures:
            f.result(timeout=max(1.0, deadline - time.monotonic()))
        with lock:
            tickets = list(live)
        for t in tickets:
            _wait(b, t, deadline)
        last_done = B.bf_batch_now(b)
        reap(block=True)
        out = _summary(lat, steps, last_done - t0 - requests[0][0] if requests else 0.0)
        w = np.asarray([x[1] for x in sorted(waits)])  # in arrival order
        out.update({"admission_wait_bounded": waits_bounded(w),"requests": len(requests), "failed": bad, "failed_status": statuses, "workers": n_workers,
                    "creators": n_creators,
                    "admission_wait_p50_ms": float(np.percentile(w, 50) * 1e3) if len(w) else None,
                    "admission_wait_p99_ms": float(np.percentile(w, 99) * 1e3) if len(w) else None,
                    "offered_rate_per_s": len(requests) / requests[-1][0] if requests else None,
                    "host_generate_ms_mean": float(np.mean(t_gen) * 1e3) if t_gen else None,
                    "host_create_ms_mean": float(np.mean(t_create) * 1e3) if t_create else None,
                    "host_create_ms_p99": float(np.percentile(t_create, 99) * 1e3) if t_create else None})
        if keep_states:
            out["states"] = states
            out["live_at_admission"] = live_at
        return out
    finally:
        pool.shutdown(wait=True)
        B.bf_batch_destroy(b)  # stops the workers after their current step
        for h, *_rest in list(live.values()):
            B.bf_scene_destroy(h)
