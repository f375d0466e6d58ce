"""Autotuner for the launch shape and the checkpoint interval.

Two choices, made per mesh shape:

* the patch decomposition: elements per patch and consumer threads per CTA
  (so elements per thread), picked by timing a short rollout + adjoint of the
  actual mesh for each candidate through the library;
* the checkpoint interval K of the rollout.  The paper's adjoint of an
  explicit method keeps every step's state (App. B); storing a checkpoint
  every K steps and recomputing in between is this library's way of fitting
  long rollouts of large meshes in memory, at the price of recomputation.  A
  segment of n steps costs n - 1 recomputed forward steps, so the recompute
  work falls as K shrinks, while the stored states, 1 + ceil(S/K) checkpoints
  and K + 1 segment buffers (S + 2 states when K = 1, which stores every
  state and recomputes nothing), fall as K grows towards sqrt(S).  The tuner
  takes the smallest K whose states fit the memory budget.

Results are cached in a JSON file keyed by device, mesh kind and sizes.
All timing runs the CUDA library; nothing here computes physics.
"""
from __future__ import annotations

import json
import math
import os
import time

STATE_BYTES = 48  # one stored state per node: (u, w), (v, plane offset) and the element force as float4

# (elements per patch, consumer threads per CTA)
# (patch elements, forward consumer threads[, adjoint consumer threads])
DEFAULT_CANDIDATES = ((256, 128), (320, 160, 128), (128, 128), (256, 256), (384, 128), (512, 256), (128, 64),
                      (64, 64))


def state_buffers(S: int, K: int) -> int:
    """State buffers a rollout of S steps with checkpoint interval K holds."""
    S = max(int(S), 0)
    if K == 1:
        return S + 2
    n_ck = max(1, -(-S // K))
    return 1 + n_ck + K + 1


def choose_K(n_nodes: int, S: int, budget_bytes: int) -> int:
    """Smallest checkpoint interval whose state buffers fit `budget_bytes`
    (the least recomputation); if none fits, the interval that needs the
    fewest buffers."""
    if S <= 1:
        return 1
    per_state = int(n_nodes) * STATE_BYTES
    k_max = max(2, math.isqrt(S - 1) + 1)  # past ~sqrt(S) the buffers grow again
    cands = [1] + list(range(2, k_max + 1))
    for K in cands:
        if state_buffers(S, K) * per_state <= budget_bytes:
            return K
    return min(cands, key=lambda K: (state_buffers(S, K), K))


def default_budget(fraction: float = 0.5) -> int:
    """A fraction of the device memory that is free now."""
    import torch
    free, _ = torch.cuda.mem_get_info()
    return int(free * fraction)


def _cache_path(path: str | None) -> str:
    if path:
        return path
    env = os.environ.get("GRADSIM_TUNE_CACHE")
    if env:
        return env
    return os.path.join(os.path.expanduser("~"), ".cache", "gradsim_autotune.json")


def cache_key(problem, steps: int, device_name: str) -> str:
    n_h = int(problem.hinges.shape[0]) if getattr(problem, "hinges", None) is not None else 0
    return f"{device_name}|kind={problem.kind}|E={problem.n_elems}|N={problem.n_nodes}|B={n_h}|S={steps}"


def load_cache(path: str | None = None) -> dict:
    p = _cache_path(path)
    try:
        with open(p) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def store_cache(entries: dict, path: str | None = None) -> None:
    p = _cache_path(path)
    os.makedirs(os.path.dirname(p) or ".", exist_ok=True)
    tmp = p + ".tmp"
    with open(tmp, "w") as f:
        json.dump(entries, f, indent=1, sort_keys=True)
    os.replace(tmp, p)


def _time_candidate(ctx, problem, patch_elems, block_threads, steps, K, reps, block_threads_adj=0):
    import torch
    from . import gradsim as gs
    dev = torch.device("cuda", ctx.device)
    try:
        m = gs.Mesh(ctx, problem, patch_elems=patch_elems, block_threads=block_threads,
                    block_threads_adj=block_threads_adj)
    except gs.GradsimError:
        return None  # e.g. the patch does not fit in shared memory
    try:
        E, N = problem.n_elems, problem.n_nodes
        f64 = dict(dtype=torch.float64, device=dev)
        grads = {"d_mu": torch.zeros(E, **f64), "d_lambda": torch.zeros(E, **f64)}
        target = torch.tensor(problem.X, dtype=torch.float32, device=dev)
        loss = torch.zeros(1, **f64)
        times = []
        for r in range(reps + 1):
            m.reset()
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            m.rollout(problem.dt, steps, K, target, loss)
            m.adjoint(grads)
            b.record()
            b.synchronize()
            if r:  # the first run builds graphs
                times.append(a.elapsed_time(b))
        times.sort()
        return times[len(times) // 2]
    finally:
        m.close()


def tune(ctx, problem, steps: int | None = None, horizon: int | None = None, candidates=DEFAULT_CANDIDATES,
         budget_bytes: int | None = None, reps: int = 2, cache: str | None = None, use_cache: bool = True) -> dict:
    """Pick (patch_elems, block_threads, block_threads_adj) by timing
    `steps` rollout + adjoint steps of `problem` per candidate (a candidate
    without a third entry runs the adjoint with block_threads), and K for a
    rollout of `horizon` steps (default problem.steps) under `budget_bytes`
    (default: half the free device memory).  Returns {"patch_elems",
    "block_threads", "block_threads_adj", "elems_per_thread", "K", "ms",
    "timings"}."""
    import torch
    horizon = int(problem.steps if horizon is None else horizon)
    steps = int(min(horizon, 20) if steps is None else steps)
    budget = default_budget() if budget_bytes is None else int(budget_bytes)
    K = choose_K(problem.n_nodes, horizon, budget)
    name = torch.cuda.get_device_name(ctx.device)
    key = cache_key(problem, steps, name)
    entries = load_cache(cache) if use_cache else {}
    hit = entries.get(key)
    if hit and all(k in hit for k in ("patch_elems", "block_threads", "ms")):
        out = dict(hit)
        out.setdefault("block_threads_adj", 0)
        out["K"] = K
        out["cached"] = True
        return out
    timings = []
    t0 = time.perf_counter()
    for cand in candidates:
        pe, bt = cand[0], cand[1]
        bta = cand[2] if len(cand) > 2 else 0
        ms = _time_candidate(ctx, problem, pe, bt, steps, min(K, max(steps, 1)), reps, bta)
        timings.append({"patch_elems": pe, "block_threads": bt, "block_threads_adj": bta, "ms": ms})
    ok = [t for t in timings if t["ms"] is not None]
    if not ok:
        raise RuntimeError("autotune: no candidate launch shape could be built for this mesh")
    best = min(ok, key=lambda t: t["ms"])
    out = {"patch_elems": best["patch_elems"], "block_threads": best["block_threads"],
           "block_threads_adj": best["block_threads_adj"],
           "elems_per_thread": best["patch_elems"] / best["block_threads"], "ms": best["ms"],
           "steps_timed": steps, "timings": timings, "tune_s": time.perf_counter() - t0}
    if use_cache:
        entries[key] = out
        try:
            store_cache(entries, cache)
        except OSError:
            pass
    out = dict(out)
    out["K"] = K
    out["cached"] = False
    return out
