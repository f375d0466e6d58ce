#!/usr/bin/env python3
"""Benchmark of the differentiable explicit FEM step and its adjoint on GB300.

One benchmark step = one whole pass of the hot path on the 1.3M-tet block:
set the initial state, a 200-step forward rollout with checkpoints and the
position loss, then the discrete adjoint through the rollout (segment
recompute + reverse steps) producing d/dmu, d/dlambda, d/drho and d/dv0.

Metric: forward+adjoint element-steps per second = tets x rollout steps /
time of (rollout + adjoint incl. recompute), summed over ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU runs are independent replicas (weak scaling, one mesh per rank, no
collective on the data path).  --impl reference times the FP64 CPU oracle on
the host cores on a bounded sample of the same workload.
"""
import argparse
import hashlib
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# Algorithmic bytes per element-step (reads + writes the method must do):
# forward: element stream 64 B (4 node ids, Dm^-1, V, mu, lambda) + node
# traffic 52 B per node (x, v, w read; x, v written) x N/E; adjoint: 64 B +
# 88 B per node (x, v read; x_bar, v_hat read + written; FP64 w_bar r/w) x N/E.
FWD_NODE_B, ADJ_NODE_B, ELEM_B = 52.0, 88.0, 64.0


def alg_bytes(kind_fwd, n_elems, n_nodes):
    node = FWD_NODE_B if kind_fwd else ADJ_NODE_B
    return ELEM_B * n_elems + node * n_nodes


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cells", type=int, default=64, help="block of cells^3 hex cells x 5 tets")
    ap.add_argument("--rollout", type=int, default=200, help="time steps per rollout")
    ap.add_argument("--K", type=int, default=0, help="checkpoint interval (0 = library choice)")
    ap.add_argument("--patch", type=int, default=0, help="elements per patch (0 = tuned/default)")
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--threads-adj", type=int, default=0, help="adjoint consumer threads (0 = --threads)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="block: library defaults instead of the autotuner's patch shape and K")
    ap.add_argument("--cpu-steps", type=int, default=4,
                    help="oracle steps in the one-thread CPU sample (the all-core sample runs 4x as many)")
    ap.add_argument("--no-extras", action="store_true",
                    help="block: skip the batched and served comparisons added to the default line")
    ap.add_argument("--extra-queries", type=int, default=300, help="block: queries per rate of the served comparison")
    ap.add_argument("--workload", default="block", choices=["block", "bar", "cloth", "batch", "serve", "control", "cloth_air", "render", "rigid", "recompute"],
                    help="block: the 1.3M-tet solid (default line); the others measure the remaining workloads")
    ap.add_argument("--meshes", type=int, default=512, help="batch: number of meshes")
    ap.add_argument("--rates", default="10,20,50,100,200,500", help="serve: arrival rates (req/s)")
    ap.add_argument("--queries", type=int, default=2000, help="serve: queries per rate")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.path = tempfile.mktemp(prefix="clocks", suffix=".csv")
        self.p = None

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:  # noqa: BLE001 - no nvidia-smi: clocks stay unknown
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        time.sleep(0.25)
        self.p.terminate()
        self.p.wait()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _shape_key(t):
    """'patch/threads' or 'patch/threads/adjoint threads' of an autotune timing."""
    k = f'{t["patch_elems"]}/{t["block_threads"]}'
    return k + (f'/{t["block_threads_adj"]}' if t.get("block_threads_adj") else "")


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("gs_kernels.cu", "gs_math.cuh"):
        with open(os.path.join(ROOT, "paper_2104_02646_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel, n_elems):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it
    was taken on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    k = d.get("kernels", {}).get(kernel)
    if not k or d.get("source_hash") != kernel_source_hash():
        return None
    return float(k["dram_bytes_per_elem"]) * n_elems


def cpu_sample(problem, steps, threads=0):
    """The FP64 oracle as it stands on a bounded sample: `steps` forward steps
    of the same mesh plus their adjoint, on `threads` host threads (0: every
    core; the results do not depend on it).  Returns (elem-steps/s, seconds,
    threads used)."""
    from oracle import oracle as O
    used = O.set_threads(threads)
    m = O.Model(problem)
    xS, _ = m.rollout(problem.x0, problem.v0, problem.dt, steps)
    target = xS + 1e-3
    t0 = time.perf_counter()
    m.loss_grad(problem.x0, problem.v0, problem.dt, steps, target)
    t = time.perf_counter() - t0
    O.set_threads(0)
    return problem.n_elems * steps / t, t, used


def cpu_baseline(problem, steps_one, steps_all, label):
    """The oracle on every host core (the reported value) and on one thread."""
    v1, t1, _ = cpu_sample(problem, steps_one, 1)
    va, ta, cores = cpu_sample(problem, steps_all, 0)
    return {"value": va, "unit": "element-steps/s", "cores": cores, "kind": "oracle",
            "sample": f"{label}: {steps_all} forward steps + their adjoint on {cores} threads ({ta:.1f} s); "
                      f"{steps_one} steps on 1 thread ({t1:.1f} s)",
            "single_thread": {"value": v1, "cores": 1}}


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_2104_02646_gb300 import inputs as I
    p = I.block(n=args.cells, steps=args.rollout)
    times = []
    for i in range(args.warmup + args.steps):
        _, t, cores = cpu_sample(p, args.cpu_steps, 0)
        if i >= args.warmup:
            times.append(t)
    value = p.n_elems * args.cpu_steps * len(times) / sum(times)
    sample = (f"block{args.cells} ({p.n_elems} tets): {args.cpu_steps} forward step(s) + their adjoint per "
              f"benchmark step, FP64 oracle, {cores} threads")
    line = {
        "impl": "reference", "metric": "fwd+adjoint element-steps/s", "value": value,
        "unit": "element-steps/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"block{args.cells}: {args.cells}^3 hex cells x 5 tets, "
                               f"{args.rollout}-step rollout at dt 5e-5 (sampled on the CPU)"},
        "cpu_baseline": {"value": value, "unit": "element-steps/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "element-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def max_over_ranks(value, dist=None, device=None):
    """Max of a per-rank scalar over all ranks (the job's wall time)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def throughput(n_ranks, n_elems, steps_per_rollout, bench_steps, total_ms):
    """Whole-job fwd+adjoint element-steps/s of independent replicas."""
    return n_ranks * n_elems * steps_per_rollout * bench_steps / (total_ms / 1e3)


def launches_per_step(S, K, have_bnd):
    """Kernels of ours launched by one benchmark step (reset + rollout +
    adjoint of a tet mesh), counted from the library's launch sequence."""
    K = mesh_K(K, S)
    n_ck = max(1, -(-S // K))
    per_step = 2 if have_bnd else 1
    n = 1                           # reset
    n += 1 + per_step * S + 2       # checkpoint copy, steps, loss + finalize
    if K == 1:
        n += 1                      # final state back to buffer 0
    n += 1 + 1 + 2                  # seed, zero w_bar, zero the mu and lambda accumulators
    if K == 1:
        n += per_step * S           # reverse steps over the stored states
    else:
        n += n_ck + per_step * S + per_step * S  # per segment: copy, n recomputed, n reverse
    n += 2                          # node and element gradient kernels
    return n


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload != "block":
        WORKLOADS[args.workload](args)
        return
    import numpy as np
    import torch

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    from paper_2104_02646_gb300 import gradsim as gs
    from paper_2104_02646_gb300 import inputs as I

    gs.load()
    p = I.block(n=args.cells, steps=args.rollout, seed=rank)
    E, N, S = p.n_elems, p.n_nodes, args.rollout
    ctx = gs.Context(local)
    # the autotuner's launch shape and checkpoint interval (untimed)
    tuned = None
    if not args.no_autotune:
        from paper_2104_02646_gb300 import autotune
        tuned = autotune.tune(ctx, p, steps=10, horizon=S, use_cache=False)
        if args.patch == 0 and args.threads == 0:
            args.patch, args.threads = tuned["patch_elems"], tuned["block_threads"]
            args.threads_adj = tuned["block_threads_adj"]
        if args.K == 0:
            args.K = tuned["K"]
    mesh = gs.Mesh(ctx, p, patch_elems=args.patch, block_threads=args.threads, block_threads_adj=args.threads_adj)
    dev = torch.device("cuda", local)
    x0 = torch.tensor(p.x0, dtype=torch.float32, device=dev)
    v0 = torch.tensor(p.v0, dtype=torch.float32, device=dev)
    # target: the library's own forward with 10 % stiffer materials + 1 mm noise
    mesh.set_params(mu=torch.tensor(p.mu * 1.1, dtype=torch.float32, device=dev),
                    lam=torch.tensor(p.lam * 1.1, dtype=torch.float32, device=dev))
    mesh.reset()
    mesh.step(p.dt, S)
    target = torch.empty(N, 3, device=dev)
    mesh.get_state(target)
    target += torch.tensor(I.position_noise(N, seed=rank), dtype=torch.float32, device=dev)
    mesh.set_params(mu=torch.tensor(p.mu, dtype=torch.float32, device=dev),
                    lam=torch.tensor(p.lam, dtype=torch.float32, device=dev))
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    grads = {k: torch.zeros(E, dtype=torch.float64, device=dev) for k in ("d_mu", "d_lambda", "d_density")}
    grads["d_v0"] = torch.zeros(N, 3, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def one_step():
        mesh.reset()
        mesh.rollout(p.dt, S, args.K, target, loss)
        mesh.adjoint(grads)

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    if mesh.check_finite() != 0:
        raise RuntimeError("non-finite state in the benchmark rollout")

    # ---- timed region: K steps, L2 flushed between them (not timed) ----------
    clocks = Clocks(local)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier()
    clocks.start()
    t_wall = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(float(k))
        starts[k].record()
        one_step()
        ends[k].record()
    barrier()
    t_wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    total_ms = max_over_ranks(sum(ms), dist, dev)
    value = throughput(ws, E, S, args.steps, total_ms)

    # ---- per-kernel launch durations (CUDA events per launch) ---------------
    check = gs.check
    L = gs.load()
    check(L.gs_profile(ctx.h, 1))
    torch.cuda.synchronize()
    flush.fill_(1.0)
    one_step()
    torch.cuda.synchronize()
    arr = (gs.gs_kernel_time * 16)()
    n_out = gs.C.c_int(0)
    check(L.gs_profile_read(ctx.h, arr, 16, gs.C.byref(n_out)))
    check(L.gs_profile(ctx.h, 0))
    kt = {arr[i].name.decode(): (arr[i].launches, arr[i].total_ms) for i in range(n_out.value)}
    dom = max(kt, key=lambda k: kt[k][1])
    launches, kms = kt[dom]
    avg_s = kms / launches / 1e3
    abytes = alg_bytes(dom.startswith("tet_fwd") or dom.startswith("cloth_fwd"), E, N)
    peak, peak_kind = measured_peaks()
    achieved = abytes / avg_s / 1e9
    traffic = ncu_traffic(dom, E)
    # the same kernel's share of the profiled step applied to the timed step:
    # the event nodes of the profiled step end the programmatic overlap
    # between neighbouring kernels, so the per-launch times above add up to
    # more than the timed step; scaled by their shares they add up to it
    prof_ms = sum(x[1] for x in kt.values())
    avg_s_timed = (kms / prof_ms) * (total_ms / args.steps) / launches / 1e3
    achieved_timed = abytes / avg_s_timed / 1e9
    # the whole timed step against the roofline of its algorithmic bytes
    step_bytes = S * (alg_bytes(True, E, N) + alg_bytes(False, E, N))
    step_achieved = step_bytes / (total_ms / args.steps / 1e3) / 1e9

    # ---- end to end through the C ABI with pinned host buffers ---------------
    e2e = None
    if not args.no_e2e:
        hx0 = x0.cpu().pin_memory()
        hv0 = v0.cpu().pin_memory()
        ht = target.cpu().pin_memory()
        hloss = torch.zeros(1, dtype=torch.float64).pin_memory()
        hg = {k: torch.zeros_like(t, device="cpu").pin_memory() for k, t in grads.items()}
        h2d = hx0.numel() * 4 + hv0.numel() * 4 + ht.numel() * 4
        d2h = 8 + sum(t.numel() * t.element_size() for t in hg.values())

        def e2e_step():
            mesh.set_state(hx0, hv0, host=True)
            mesh.rollout(p.dt, S, args.K, ht, hloss, host=True)
            mesh.adjoint(hg, host=True)

        e2e_step()
        torch.cuda.synchronize()
        barrier()
        e2e_s = 0.0
        for _ in range(args.steps):
            flush.fill_(2.0)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            e2e_step()
            torch.cuda.synchronize()
            e2e_s += time.perf_counter() - t1
        e2e = {"value": ws * E * S * args.steps / e2e_s, "unit": "element-steps/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

    # ---- CPU baseline: the oracle on a bounded sample -------------------------
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(p, args.cpu_steps, 4 * args.cpu_steps, f"block{args.cells} ({E} tets), FP64 oracle")

    # ---- batched and served forms against the plain loop (untimed extras) ----
    extras = None
    if rank == 0 and ws == 1 and not args.no_extras:
        mesh.close()
        torch.cuda.empty_cache()
        extras = {"batch": measure_batch(args, 512, reps=2),
                  "serve": [measure_serve(args, rate, args.extra_queries) for rate in (50.0, 500.0)]}

    if rank == 0:
        line = {
            "metric": "fwd+adjoint element-steps/s", "value": value, "unit": "element-steps/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"block{args.cells}: {args.cells}^3 hex cells x 5 tets = {E} tets, {N} nodes, "
                                   f"{S}-step rollout at dt {p.dt} + adjoint, K={mesh_K(args.K, S)}",
                       "parallelism": f"replicas x{ws}", "l2": "flushed between timed iterations (512 MiB write)",
                       "patch_elems": mesh.info.patch_elems, "block_threads": mesh.info.block_threads,
                       "block_threads_adj": mesh.info.block_threads_adj,
                       "autotune": None if tuned is None else {
                           "K": tuned["K"], "budget": "half the free device memory",
                           "candidates_ms": {_shape_key(t): t["ms"] for t in tuned["timings"]}}},
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                         "alg_bytes_per_launch": abytes, "avg_launch_ms": avg_s * 1e3,
                         "launches_per_step": launches,
                         "timing": "CUDA events around each kernel inside the captured graphs of one extra step",
                         "profiled_kernels_ms_per_step": prof_ms,
                         "in_timed_step": {"avg_launch_ms": avg_s_timed * 1e3, "achieved": achieved_timed,
                                           "frac": achieved_timed / peak,
                                           "how": "the kernel's share of the profiled step x the timed step "
                                                  "/ launches (the per-kernel events remove the overlap of "
                                                  "neighbouring kernels that the timed step has)"},
                         "kernel_share": {k: v[1] / sum(x[1] for x in kt.values()) for k, v in kt.items()},
                         "step": {"alg_bytes": step_bytes, "achieved": step_achieved,
                                  "frac": step_achieved / peak,
                                  "element_steps_per_s_at_peak": E * S / (step_bytes / (peak * 1e9))}},
            "clocks": clk,
            "e2e": e2e,
            "gpu_launches": launches_per_step(S, args.K, mesh.info.n_boundary_nodes > 0) * args.steps,
            "cpu_baseline": cpu,
            "wall_s": t_wall,
        }
        if extras is not None:
            line["batched_vs_plain"] = extras["batch"]
            line["served_vs_plain"] = extras["serve"]
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def mesh_K(K, S):
    import math
    return K if K > 0 else max(1, math.ceil(math.sqrt(max(S, 1))))



# ---------------------------------------------------------------------------
# the other workloads (one JSON line each; the default line is the block)
# ---------------------------------------------------------------------------
def _events_ms(fn, reps=1):
    import torch
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def _grads(problem, dev):
    import torch
    E, N, B = problem.n_elems, problem.n_nodes, problem.n_hinges
    g = {k: torch.zeros(E, dtype=torch.float64, device=dev) for k in ("d_mu", "d_lambda", "d_density")}
    g["d_v0"] = torch.zeros(N, 3, device=dev)
    if B:
        g["d_kb"] = torch.zeros(B, dtype=torch.float64, device=dev)
    return g


def _single_mesh_line(args, name, problem, extra_cfg, cpu_steps=None):
    """Forward rollout + adjoint of one mesh: element-steps/s and steps/s;
    with cpu_steps = (one-thread steps, all-core steps), the oracle's rate on
    that sample of the same mesh beside it."""
    import torch
    from paper_2104_02646_gb300 import gradsim as gs
    gs.load()
    dev = torch.device("cuda", 0)
    ctx = gs.Context(0)
    S = problem.steps
    pe, bt, bta, K = args.patch, args.threads, args.threads_adj, args.K
    tuned = None
    if not args.no_autotune and pe == 0 and bt == 0:
        from paper_2104_02646_gb300 import autotune
        tuned = autotune.tune(ctx, problem, steps=min(S, 20), horizon=S, use_cache=False)
        pe, bt, bta = tuned["patch_elems"], tuned["block_threads"], tuned["block_threads_adj"]
        K = tuned["K"] if K == 0 else K
    mesh = gs.Mesh(ctx, problem, patch_elems=pe, block_threads=bt, block_threads_adj=bta)
    target = torch.tensor(problem.X + 1e-3, dtype=torch.float32, device=dev)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    g = _grads(problem, dev)

    def fwd():
        mesh.reset()
        mesh.rollout(problem.dt, S, K, target, loss)

    def both():
        fwd()
        mesh.adjoint(g)

    for _ in range(args.warmup):
        both()
    t_fwd = min(_events_ms(fwd) for _ in range(args.steps))
    t_all = min(_events_ms(both) for _ in range(args.steps))
    ctx.set_graphs(False)
    t_plain = min(_events_ms(both) for _ in range(max(1, args.steps // 2)))
    ctx.set_graphs(True)
    E = problem.n_elems
    line = {"metric": "fwd+adjoint element-steps/s", "workload": name, "value": E * S / (t_all / 1e3),
            "unit": "element-steps/s", "ms_per_rollout_fwd": t_fwd, "ms_per_rollout_fwd_adj": t_all,
            "fwd_steps_per_s": S / (t_fwd / 1e3), "fwd_adj_steps_per_s": S / (t_all / 1e3),
            "us_per_step_fwd_adj": 1e3 * t_all / S, "plain_loop_value": E * S / (t_plain / 1e3),
            "finite": mesh.check_finite() == 0, "dtype": "f32", "data": "synthetic",
            "config": dict(extra_cfg, elems=E, nodes=problem.n_nodes, hinges=problem.n_hinges, steps=S,
                           dt=problem.dt, patch_elems=mesh.info.patch_elems,
                           block_threads=mesh.info.block_threads, block_threads_adj=mesh.info.block_threads_adj,
                           K=mesh_K(K, S),
                           autotune=None if tuned is None else {_shape_key(t): t["ms"] for t in tuned["timings"]})}
    if cpu_steps is not None and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(problem, cpu_steps[0], cpu_steps[1], f"{name} ({E} elements), FP64 oracle")
    print(json.dumps(line), flush=True)


def workload_bar(args):
    from paper_2104_02646_gb300 import inputs as I
    for v in ("a", "b"):
        _single_mesh_line(args, f"bar1{v}", I.bar(v, steps=1000), {"cells": "4x4x4", "drop": "0.2 m" if v == "a" else "0.02 m"},
                          cpu_steps=(1000, 1000))


def workload_cloth(args):
    from paper_2104_02646_gb300 import inputs as I
    # the stated materials diverge under explicit Euler at dt 1e-4 (reported
    # by `finite`); the stable variant has the same mesh and work
    for v in ("3s", "3"):
        _single_mesh_line(args, f"cloth{v}", I.cloth(v, n=256, steps=500), {"grid": "256x256", "variant": v},
                          cpu_steps=(10, 40) if v == "3s" else None)


def measure_batch(args, n_meshes, reps):
    """Config 4: n heterogeneous meshes, fwd+adj in one launch per kernel per
    step (graphs) against the plain loop (one mesh per launch, one step per
    launch, no graphs) on the same GPU.  Returns a dict."""
    import torch
    from paper_2104_02646_gb300 import gradsim as gs
    from paper_2104_02646_gb300 import inputs as I
    gs.load()
    dev = torch.device("cuda", 0)
    probs = I.batch(n_meshes, steps=300)
    ctx = gs.Context(0)
    t0 = time.perf_counter()
    meshes = [gs.Mesh(ctx, p, patch_elems=args.patch, block_threads=args.threads,
                      block_threads_adj=args.threads_adj) for p in probs]
    t_create = time.perf_counter() - t0
    batch = gs.Batch(ctx, meshes)
    S = 300
    E = sum(p.n_elems for p in probs)
    K = args.K
    if K == 0 and not args.no_autotune:
        from paper_2104_02646_gb300 import autotune
        K = autotune.choose_K(sum(p.n_nodes for p in probs), S, autotune.default_budget())
    targets = [torch.tensor(p.X + 1e-3, dtype=torch.float32, device=dev) for p in probs]
    loss = torch.zeros(len(probs), dtype=torch.float64, device=dev)
    grads = [_grads(p, dev) for p in probs]
    dts = [p.dt for p in probs]

    def batched():
        for m in meshes:
            m.reset()
        batch.rollout(dts, S, K, targets, loss)
        batch.adjoint(grads)

    losses = [torch.zeros(1, dtype=torch.float64, device=dev) for _ in probs]

    def plain():
        for m, p, t, l, g in zip(meshes, probs, targets, losses, grads):
            m.reset()
            m.rollout(p.dt, S, K, t, l)
            m.adjoint(g)

    batched()
    t_b = min(_events_ms(batched) for _ in range(max(1, reps)))
    ctx.set_graphs(False)
    plain()
    t_p = _events_ms(plain)
    ctx.set_graphs(True)
    out = {"metric": "fwd+adjoint element-steps/s", "workload": f"batch{len(probs)}",
           "value": E * S / (t_b / 1e3), "unit": "element-steps/s",
           "plain_loop_value": E * S / (t_p / 1e3), "speedup_vs_plain": t_p / t_b,
           "ms_batched": t_b, "ms_plain": t_p,
           "config": {"meshes": len(probs), "tets": E, "nodes": sum(p.n_nodes for p in probs), "steps": S,
                      "dt": 1e-4, "K": mesh_K(K, S), "mesh_create_s": t_create,
                      "plain_loop": "same kernels, one mesh per launch, one step per launch, no graphs"}}
    batch.close()
    for m in meshes:
        m.close()
    del ctx
    torch.cuda.empty_cache()
    return out


def workload_batch(args):
    """512 heterogeneous meshes: one launch per kernel per step (graphs) vs the
    plain loop (one mesh per launch, one step per launch, no graphs)."""
    line = measure_batch(args, args.meshes, args.steps)
    line.update({"dtype": "f32", "data": "synthetic"})
    print(json.dumps(line), flush=True)


def measure_serve(args, rate, n_queries):
    """Config 5 at one arrival rate: Poisson gradient queries through the
    continuous-batching server vs the plain loop (each query alone, in
    arrival order, one launch per kernel).  Returns a dict."""
    import torch
    from paper_2104_02646_gb300 import gradsim as gs
    from paper_2104_02646_gb300 import inputs as I
    gs.load()
    dev = torch.device("cuda", 0)
    qs = I.query_stream(rate, n_queries, seed=int(rate))
    work = sum(q.problem.n_elems * q.problem.steps for q in qs)
    ctx = gs.Context(0)
    server = gs.Server(ctx, budget=120 << 30)
    t0 = time.perf_counter()
    tickets = []
    for q in qs:
        delay = t0 + q.t_arrival - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        tickets.append(server.submit(q.problem, q.problem.X + q.target_offset))
    res = [server.poll(t, timeout_ms=600000) for t in tickets]
    t_all = time.perf_counter() - t0
    ok = [r for st, r in res if st == gs.GS_OK]
    lat = sorted(r["t_done"] - r["t_submit"] for r in ok)
    stats = server.stats()
    server.close()
    # plain loop: FIFO, one query at a time (no batching, no graphs)
    ctx2 = gs.Context(0)
    ctx2.set_graphs(False)
    clock = 0.0
    plain_lat = []
    busy = 0.0
    for q in qs:
        p = q.problem
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        # service time includes building the mesh, as the server's latency does
        m = gs.Mesh(ctx2, p)
        t = torch.tensor(p.X + q.target_offset, dtype=torch.float32, device=dev)
        l = torch.zeros(1, dtype=torch.float64, device=dev)
        g = _grads(p, dev)
        m.rollout(p.dt, p.steps, 0, t, l)
        m.adjoint(g)
        torch.cuda.synchronize()
        dur = time.perf_counter() - w0
        busy += dur
        clock = max(clock, q.t_arrival) + dur
        plain_lat.append(clock - q.t_arrival)
        m.close()
    plain_lat.sort()
    pct = lambda v, f: v[min(len(v) - 1, int(round(f * (len(v) - 1))))] if v else None
    return {"metric": "p50/p99 query latency and aggregate element-steps/s", "workload": "serve",
            "rate_req_s": rate, "queries": len(qs), "completed": len(ok),
            "p50_s": pct(lat, 0.5), "p99_s": pct(lat, 0.99), "elem_steps_per_s": stats["elem_steps_per_s"],
            "wall_s": t_all, "plain_p50_s": pct(plain_lat, 0.5), "plain_p99_s": pct(plain_lat, 0.99),
            "plain_elem_steps_per_s": work / busy,
            "server_time_s": {k: round(stats[k], 4) for k in
                              ("busy_s", "build_s", "start_s", "rebuild_s", "rt_sync_s", "gpu_wait_s")},
            "server_counts": {k: int(stats[k]) for k in ("ticks", "rebuilds", "rt_syncs")},
            "config": {"budget_GB": 120, "tets": "log-uniform 1e3..2e5", "cloth": "32^2..192^2",
                       "horizon": "100..1000", "dt": 1e-4, "service_time": "mesh build + rollout + adjoint"}}


def workload_serve(args):
    """Poisson gradient queries through the continuous-batching server vs the
    plain loop (each query alone, in arrival order, one launch per kernel)."""
    for rate in [float(r) for r in args.rates.split(",")]:
        line = measure_serve(args, rate, args.queries)
        line["data"] = "synthetic"
        print(json.dumps(line), flush=True)


def workload_recompute(args):
    """The checkpoint / recompute path at size: the 1.3M-tet block over a
    1,000-step rollout + adjoint with every state kept (K = 1) against a
    checkpoint every K = ceil(sqrt(S)) steps, the memory-minimal choice
    (one recomputed forward step per reverse step, less one per segment)."""
    import math as _m
    import torch
    from paper_2104_02646_gb300 import gradsim as gs
    from paper_2104_02646_gb300 import inputs as I
    gs.load()
    dev = torch.device("cuda", 0)
    S = 1000
    p = I.block(n=args.cells, steps=S)
    ctx = gs.Context(0)
    mesh = gs.Mesh(ctx, p, patch_elems=args.patch, block_threads=args.threads, block_threads_adj=args.threads_adj)
    target = torch.tensor(p.X + 1e-3, dtype=torch.float32, device=dev)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    g = _grads(p, dev)
    res = {}
    for K in (1, int(_m.ceil(_m.sqrt(S)))):
        def both():
            mesh.reset()
            mesh.rollout(p.dt, S, K, target, loss)
            mesh.adjoint(g)
        for _ in range(max(1, args.warmup)):
            both()
        res[K] = min(_events_ms(both) for _ in range(max(1, args.steps)))
    K1, Kc = sorted(res)
    state_mb = 48 * p.n_nodes / 1e6
    n_ck = -(-S // Kc)
    line = {"metric": "fwd+adjoint element-steps/s", "workload": f"recompute_block{args.cells}",
            "value": p.n_elems * S / (res[Kc] / 1e3), "unit": "element-steps/s",
            "K1_value": p.n_elems * S / (res[K1] / 1e3), "ms_K1": res[K1], f"ms_K{Kc}": res[Kc],
            "recompute_cost": res[Kc] / res[K1] - 1.0,
            "stored_states_MB": {"K1": (S + 2) * state_mb, f"K{Kc}": (1 + n_ck + Kc + 1) * state_mb},
            "dtype": "f32", "data": "synthetic",
            "config": {"tets": p.n_elems, "nodes": p.n_nodes, "steps": S, "dt": p.dt, "K": [K1, Kc]}}
    print(json.dumps(line), flush=True)
    mesh.close()


def workload_control(args):
    """Time-varying actuation (the visuomotor control input, Sec. 3) driven by
    the App. D controller: (1) a 1,080-tet block, the size of the paper's
    control-fem object, one controller training iteration = controller
    forward, actuated rollout, adjoint with per-step actuation gradients,
    controller backward; (2) the 1.3M-tet block with every element actuated
    every step, against the same rollout + adjoint without actuation."""
    import torch
    from paper_2104_02646_gb300 import autograd as A
    from paper_2104_02646_gb300 import control
    from paper_2104_02646_gb300 import gradsim as gs
    from paper_2104_02646_gb300 import inputs as I
    gs.load()
    dev = torch.device("cuda", 0)
    ctx = gs.Context(0)
    # (1) controller training iteration on a small object
    S1 = 1000
    p = I.block(n=6, steps=S1, seed=3)
    mesh = gs.Mesh(ctx, p)
    x0 = torch.tensor(p.x0, dtype=torch.float32, device=dev)
    v0 = torch.tensor(p.v0, dtype=torch.float32, device=dev)
    t = torch.arange(S1, dtype=torch.float32, device=dev) * p.dt
    ctrl = control.SinusoidController(p.n_elems, omega=2 * 3.14159265 * 20, generator=torch.Generator().manual_seed(0)).to(dev)
    xT = x0 + 0.01
    opt = torch.optim.Adam(ctrl.parameters(), lr=0.05)

    def iteration():
        opt.zero_grad()
        xS, _ = A.actuated_rollout(mesh, p.dt, S1, ctrl(t), x0, v0, K=1)
        loss = ((xS - xT) ** 2).sum()
        loss.backward()
        opt.step()
        return loss

    for _ in range(args.warmup):
        iteration()
    t_it = min(_events_ms(iteration) for _ in range(args.steps))
    line = {"metric": "controller training iterations/s", "workload": "control1080", "value": 1e3 / t_it,
            "unit": "iterations/s", "ms_per_iteration": t_it,
            "fwd_adj_elem_steps_per_s": p.n_elems * S1 / (t_it / 1e3), "dtype": "f32", "data": "synthetic",
            "config": {"tets": p.n_elems, "steps": S1, "dt": p.dt, "controller": "8 sinusoids -> FC (no bias) -> tanh",
                       "actuated": "every element, every step", "K": 1}}
    print(json.dumps(line), flush=True)
    mesh.close()
    # (2) actuation overhead at scale
    S2 = 200
    q = I.block(n=64, steps=S2)
    m2 = gs.Mesh(ctx, q)
    E, N = q.n_elems, q.n_nodes
    seq = (0.05 * torch.sin(torch.arange(S2, device=dev, dtype=torch.float32)[:, None] * 0.1
                            + torch.linspace(0, 6.28, E, device=dev)[None, :])).contiguous()
    tgt = torch.tensor(q.X, dtype=torch.float32, device=dev)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    g = _grads(q, dev)
    g_act = dict(g, d_act_seq=torch.zeros(S2, E, device=dev))

    def run(actuated):
        m2.set_act_seq(seq if actuated else None)
        m2.reset()
        m2.rollout(q.dt, S2, 1, tgt, loss)
        m2.adjoint(g_act if actuated else g)

    res = {}
    for actuated in (False, True):
        for _ in range(args.warmup):
            run(actuated)
        res[actuated] = min(_events_ms(lambda: run(actuated)) for _ in range(args.steps))
    line = {"metric": "fwd+adjoint element-steps/s", "workload": "control_block64", "value": E * S2 / (res[True] / 1e3),
            "unit": "element-steps/s", "unactuated_value": E * S2 / (res[False] / 1e3),
            "ms_actuated": res[True], "ms_unactuated": res[False], "dtype": "f32", "data": "synthetic",
            "config": {"tets": E, "steps": S2, "actuated": "every element, every step; per-step actuation gradients out",
                       "K": 1}}
    print(json.dumps(line), flush=True)


def workload_cloth_air(args):
    """The air model on cloth (App. A.1 lift/drag) and the cloth-control
    workload of Sec. 3: (1) one system-identification iteration on a thrown
    2,048-triangle cloth (the largest of the paper's 64-2048) = rollout of
    1,000 steps with air + adjoint + Adam on the per-node initial velocity;
    (2) the 256^2 cloth ("3s") rollout + adjoint with and without air."""
    import torch
    from paper_2104_02646_gb300 import autograd as A
    from paper_2104_02646_gb300 import gradsim as gs
    from paper_2104_02646_gb300 import inputs as I
    gs.load()
    dev = torch.device("cuda", 0)
    ctx = gs.Context(0)
    S1 = 1000
    p = I.cloth_throw(n=33, steps=S1, seed=0)
    mesh = gs.Mesh(ctx, p)
    f32 = dict(dtype=torch.float32, device=dev)
    mu, lam, rho = (torch.tensor(a, **f32) for a in (p.mu, p.lam, p.rho))
    x0 = torch.tensor(p.x0, **f32)
    v_ref = torch.tensor(p.v0, **f32)
    with torch.no_grad():
        xT, _ = A.rollout(mesh, p.dt, S1, mu, lam, rho, x0, v_ref, K=1)
    v = (v_ref + 0.3).requires_grad_(True)
    opt = torch.optim.Adam([v], lr=0.05)

    def iteration():
        opt.zero_grad()
        xS, _ = A.rollout(mesh, p.dt, S1, mu, lam, rho, x0, v, K=1)
        loss = ((xS - xT) ** 2).sum()
        loss.backward()
        opt.step()

    for _ in range(args.warmup):
        iteration()
    t_it = min(_events_ms(iteration) for _ in range(args.steps))
    line = {"metric": "cloth v0 system-ID iterations/s", "workload": "cloth_throw33", "value": 1e3 / t_it,
            "unit": "iterations/s", "ms_per_iteration": t_it,
            "fwd_adj_tri_steps_per_s": p.n_elems * S1 / (t_it / 1e3), "dtype": "f32", "data": "synthetic",
            "config": {"triangles": p.n_elems, "hinges": p.n_hinges, "steps": S1, "dt": p.dt,
                       "air": dataclasses.asdict(p.air), "optimised": "per-node initial velocity (Adam)", "K": 1}}
    print(json.dumps(line), flush=True)
    mesh.close()
    S2 = 500
    q = I.cloth("3s", n=256, steps=S2)
    m2 = gs.Mesh(ctx, q)
    tgt = torch.tensor(q.X, **f32)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    g = _grads(q, dev)
    res = {}
    for air in (None, I.Air(wind=(0.5, 0.0, 0.2))):
        m2.set_air(air)

        def run():
            m2.reset()
            m2.rollout(q.dt, S2, 1, tgt, loss)
            m2.adjoint(g)

        for _ in range(args.warmup):
            run()
        res[air is not None] = min(_events_ms(run) for _ in range(args.steps))
    line = {"metric": "fwd+adjoint element-steps/s", "workload": "cloth3s_air", "value": q.n_elems * S2 / (res[True] / 1e3),
            "unit": "element-steps/s", "no_air_value": q.n_elems * S2 / (res[False] / 1e3),
            "ms_air": res[True], "ms_no_air": res[False], "dtype": "f32", "data": "synthetic",
            "config": {"grid": "256x256", "triangles": q.n_elems, "hinges": q.n_hinges, "steps": S2, "K": 1,
                       "air": "k_drag 0.6, k_lift 0.4, wind (0.5, 0, 0.2)"}}
    print(json.dumps(line), flush=True)


def workload_render(args):
    """The soft rasteriser (Sec. 2 "Differentiable rendering engine"): (1) one
    frame of the 256^2 cloth (130,050 triangles) at 512^2 and 1024^2, forward
    and backward; (2) the image-loss identification iteration: a thrown
    2,048-triangle cloth, 1,000 steps with air, 4 rendered frames at 128^2
    against target frames, backward through renderer and simulator, Adam on
    the initial velocity."""
    import torch
    from paper_2104_02646_gb300 import autograd as A
    from paper_2104_02646_gb300 import gradsim as gs
    from paper_2104_02646_gb300 import inputs as I
    gs.load()
    dev = torch.device("cuda", 0)
    ctx = gs.Context(0)
    f32 = dict(dtype=torch.float32, device=dev)
    q = I.cloth("3s", n=256, steps=1)
    x = torch.tensor(q.X, **f32)
    col = torch.tensor(I.vertex_colours(q.X, seed=0), **f32)
    spec = I.RenderSpec()
    for res in (512, 1024):
        cam = I.look_at((1.3, 1.2, -0.6), (0.5, 0.3, 0.5), width=res, height=res, fov_deg=50.0)
        r = gs.Raster(ctx, q.n_nodes, q.elems, cam, spec)
        img = torch.empty(res, res, 4, **f32)
        gimg = torch.randn(res, res, 4, generator=torch.Generator().manual_seed(0)).to(dev)
        dx, dc = torch.empty_like(x), torch.empty_like(col)
        for _ in range(args.warmup):
            r.forward(x, col, img)
            r.backward(gimg, dx, dc)
        t_f = min(_events_ms(lambda: r.forward(x, col, img), reps=5) for _ in range(args.steps))
        t_b = min(_events_ms(lambda: r.backward(gimg, dx, dc), reps=5) for _ in range(args.steps))
        # (pixel, triangle) pairs the kernels evaluate: each triangle's clipped box
        u, v, z = _project_np(q.X, cam)
        boxes = _pair_count(u[q.elems], v[q.elems], z[q.elems], cam, spec)
        line = {"metric": "rendered frames/s (forward + backward)", "workload": f"render_cloth256_{res}",
                "value": 1e3 / (t_f + t_b), "unit": "frames/s", "ms_forward": t_f, "ms_backward": t_b,
                "pair_evals_per_frame": boxes, "pair_evals_per_s_forward": boxes / (t_f / 1e3),
                "dtype": "f32", "data": "synthetic",
                "config": {"triangles": q.n_elems, "image": f"{res}x{res}", "sigma_px2": spec.sigma,
                           "gamma": spec.gamma}}
        print(json.dumps(line), flush=True)
        r.close()
    # image-loss identification iteration
    S, n_frames, res = 1000, 4, 128
    p = I.cloth_throw(n=33, steps=S, seed=0)
    mesh = gs.Mesh(ctx, p)
    mu, lam, rho = (torch.tensor(a, **f32) for a in (p.mu, p.lam, p.rho))
    x0 = torch.tensor(p.x0, **f32)
    colp = torch.tensor(I.vertex_colours(p.X, seed=1), **f32)
    cam = I.look_at((1.6, 1.0, -0.8), (0.45, 0.35, 0.45), width=res, height=res, fov_deg=50.0)
    raster = gs.Raster(ctx, p.n_nodes, p.elems, cam, I.RenderSpec(sigma=1.0, gamma=1e-2))

    def frames(v0):
        xx, vv, out = x0, v0, []
        for _ in range(n_frames):
            xx, vv = A.rollout(mesh, p.dt, S // n_frames, mu, lam, rho, xx, vv, K=1)
            out.append(A.render(raster, xx, colp))
        return out

    v_ref = torch.tensor(p.v0, **f32)
    with torch.no_grad():
        target = [f.clone() for f in frames(v_ref)]
    vv0 = (v_ref + 0.3).requires_grad_(True)
    opt = torch.optim.Adam([vv0], lr=0.03)

    def iteration():
        opt.zero_grad()
        loss = sum(((f - t) ** 2).sum() for f, t in zip(frames(vv0), target))
        loss.backward()
        opt.step()

    for _ in range(args.warmup):
        iteration()
    t_it = min(_events_ms(iteration) for _ in range(args.steps))
    line = {"metric": "image-loss v0 identification iterations/s", "workload": "render_cloth_throw33",
            "value": 1e3 / t_it, "unit": "iterations/s", "ms_per_iteration": t_it, "dtype": "f32",
            "data": "synthetic",
            "config": {"triangles": p.n_elems, "steps": S, "frames": n_frames, "image": f"{res}x{res}",
                       "air": "on", "recompute": "each frame's segment is re-run in backward", "K": 1}}
    print(json.dumps(line), flush=True)
    raster.close()
    mesh.close()


def _project_np(X, cam):
    xc = X @ cam.R.T + cam.t
    return cam.fx * xc[:, 0] / xc[:, 2] + cam.cx, cam.fy * xc[:, 1] / xc[:, 2] + cam.cy, xc[:, 2]


def _pair_count(u, v, z, cam, spec):
    """(pixel, triangle) pairs in the triangles' clipped pixel boxes."""
    import math as _m
    r = _m.sqrt(spec.sigma * _m.log((1 - 1e-5) / 1e-5))
    ok = (z > cam.z_near).all(axis=1)
    x0 = np.clip(np.ceil(u.min(axis=1) - r - 0.5), 0, cam.width)
    x1 = np.clip(np.floor(u.max(axis=1) + r - 0.5), -1, cam.width - 1)
    y0 = np.clip(np.ceil(v.min(axis=1) - r - 0.5), 0, cam.height)
    y1 = np.clip(np.floor(v.max(axis=1) + r - 0.5), -1, cam.height - 1)
    n = np.maximum(x1 - x0 + 1, 0) * np.maximum(y1 - y0 + 1, 0)
    return int(n[ok].sum())


def workload_rigid(args):
    """Rigid bodies (App. A.1): 16,384 seeded boxes (98 surface contact
    points each, the ranges of the paper's rigid experiments) dropped on the
    ground, 300 steps, rollout + adjoint in one launch each; and the paper's
    mass loss landscape (a unit-mass cube after a known impulse, 6 rendered
    frames at 96^2, 10 guessed masses)."""
    import torch
    from paper_2104_02646_gb300 import autograd as A
    from paper_2104_02646_gb300 import gradsim as gs
    from paper_2104_02646_gb300 import inputs as I
    gs.load()
    dev = torch.device("cuda", 0)
    ctx = gs.Context(0)
    S, nb = 300, 16384
    bodies = I.rigid_batch(nb, seed=0, n=5, steps=S)
    rig = gs.Rigid(ctx, bodies)
    s0 = torch.tensor(rig.state0(), device=dev)
    sS = torch.empty_like(s0)
    g = {"d_state0": torch.zeros(nb, 13, device=dev), "d_mass": torch.zeros(nb, dtype=torch.float64, device=dev),
         "d_inertia": torch.zeros(nb, 6, dtype=torch.float64, device=dev),
         "d_contact": torch.zeros(nb, 4, dtype=torch.float64, device=dev)}
    seed = torch.ones(nb, 13, device=dev)

    def run():
        rig.rollout(1e-3, S, s0, sS)
        rig.adjoint(g, seed=seed)

    for _ in range(args.warmup):
        run()
    t = min(_events_ms(run) for _ in range(args.steps))
    t_f = min(_events_ms(lambda: rig.rollout(1e-3, S, s0, sS)) for _ in range(args.steps))
    line = {"metric": "rigid fwd+adjoint body-steps/s", "workload": "rigid16384", "value": nb * S / (t / 1e3),
            "unit": "body-steps/s", "ms": t, "ms_forward": t_f,
            "contact_point_steps_per_s": rig.n_points * S / (t / 1e3), "dtype": "f32", "data": "synthetic",
            "finite": rig.check_finite() == gs.GS_OK,
            "config": {"bodies": nb, "points_per_body": rig.n_points // nb, "steps": S, "dt": 1e-3,
                       "launches": "1 rollout + 1 adjoint"}}
    print(json.dumps(line), flush=True)
    rig.close()


WORKLOADS = {"bar": workload_bar, "cloth": workload_cloth, "batch": workload_batch, "serve": workload_serve,
             "control": workload_control, "cloth_air": workload_cloth_air, "render": workload_render,
             "rigid": workload_rigid, "recompute": workload_recompute}

if __name__ == "__main__":
    main()
