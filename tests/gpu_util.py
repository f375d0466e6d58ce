"""Helpers shared by the GPU parity tests: run a Problem through the CUDA
library (via the C-ABI binding) and through the FP64 oracle, and compare."""
import math

import numpy as np

from oracle import oracle as O
from paper_2104_02646_gb300 import inputs as I

# oracle gradient key -> gs_grads field
TET_KEYS = {"tet_mu": "d_mu", "tet_lam": "d_lambda", "tet_rho": "d_density", "x0": "d_x0", "v0": "d_v0"}
CLOTH_KEYS = {"tri_mu": "d_mu", "tri_lam": "d_lambda", "tri_rho": "d_density", "hinge_kb": "d_kb",
              "x0": "d_x0", "v0": "d_v0"}


# FP32 GPU vs FP64 oracle: positions rel-L2 (centroid-removed norm) <= 1e-4
# contact-free, <= 1e-3 with contact; gradients rel-L2 <= 1e-3, cosine >= 0.9999
POS_FREE, POS_CONTACT, GRAD_REL, GRAD_COS = 1e-4, 1e-3, 1e-3, 0.9999


ENTRY_FACTOR = 10.0


def entry_bar(tol, n=None):
    """Per-entry bar that goes with a rel-L2 bar `tol`: ENTRY_FACTOR x tol,
    against |b_i| + rms(b).  A mistake confined to a few entries (a wrong
    index, a dropped term, a flipped sign, two entries swapped) moves them by
    O(1) of their size and fails it; FP32 round-off, including its
    heavier-tailed part near contact, stays inside 1 % per entry."""
    return ENTRY_FACTOR * tol


def check_grads(g_gpu, g_ref, keys, skip=(), entry=True):
    """Per gradient array: rel-L2 <= GRAD_REL, cosine >= GRAD_COS and, entry by
    entry, |a_i - b_i| <= entry_bar(GRAD_REL, n) (|b_i| + rms(b)), so that an
    error confined to a few elements or nodes cannot hide under the norm."""
    for ok, gk in keys.items():
        if ok in skip:
            continue
        a, b = g_gpu[gk], g_ref[ok]
        assert np.all(np.isfinite(a)), gk
        assert rel(a, b) <= GRAD_REL, (gk, rel(a, b))
        assert cosine(a, b) >= GRAD_COS, (gk, cosine(a, b))
        if entry:
            r = entry_ratio(a, b, entry_bar(GRAD_REL))
            assert r <= 1.0, (gk, "entry", r)


def quat_tangent(g_state, q):
    """A rigid body's state gradient [13] with its quaternion part (entries
    3:7) projected on the tangent space of the unit quaternion q: the loss
    depends on r only through the unit sphere, so the component along q is a
    convention of how the step treats off-sphere r, not physics."""
    g = np.array(g_state, dtype=np.float64)
    qn = np.asarray(q, dtype=np.float64) / np.linalg.norm(q)
    g[3:7] -= (g[3:7] @ qn) * qn
    return g


# factor on the problem's own sensitivity for ill-conditioned cases (C20); see
# check_grads_conditioned
COND_FACTOR = 10.0


def fp32_inputs(problem, target):
    """A copy of `problem` (and the target) with every input the GPU receives
    rounded to FP32 (rest and initial positions, velocities, materials)."""
    r32 = lambda z: None if z is None else np.asarray(z, np.float32).astype(np.float64)
    q = I.Problem(**{f: getattr(problem, f) for f in problem.__dataclass_fields__})
    for f in ("X", "x0", "v0", "mu", "lam", "rho", "kb", "act", "hinge_act"):
        setattr(q, f, r32(getattr(problem, f)))
    return q, r32(target)


def check_grads_conditioned(g_gpu, g_ref, g_ref32, keys, skip=()):
    """For rollouts whose gradients are ill-conditioned at FP32 precision (C20:
    contact switching over a long horizon).  kappa = rel-L2 between the
    oracle on the exact inputs and the oracle on the same inputs rounded to
    FP32 is the problem's own sensitivity to one rounding of its inputs; the
    GPU, which rounds at every operation of every step, must stay within
    max(GRAD_REL, COND_FACTOR kappa) of the oracle (measured on such cases:
    1 to 4 kappa).  Returns {key: (rel, kappa)} for reporting."""
    out = {}
    for ok, gk in keys.items():
        if ok in skip:
            continue
        a, b, b32 = g_gpu[gk], g_ref[ok], g_ref32[ok]
        assert np.all(np.isfinite(a)), gk
        kappa = rel(b32, b)
        bar = max(GRAD_REL, COND_FACTOR * kappa)
        r = rel(a, b)
        out[gk] = (r, kappa)
        assert r <= bar, (gk, r, "kappa", kappa)
        assert cosine(a, b) >= min(GRAD_COS, 1.0 - bar * bar), (gk, cosine(a, b), "kappa", kappa)
    print("gradient rel-L2 against the oracle, and the oracle's own FP32-input sensitivity:",
          {k: f"{r:.2e} (kappa {kp:.2e})" for k, (r, kp) in out.items()})
    return out


def entry_ratio(a, b, tol):
    """Largest per-entry error against the bar tol (|b_i| + rms(b)): rows of a
    2-D array (node vectors) are compared by their Euclidean norms.  <= 1 means
    every entry is within the bar."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if a.ndim == 1:
        a, b = a[:, None], b[:, None]
    if a.size == 0:
        return 0.0
    d = np.linalg.norm(a - b, axis=1)
    nb = np.linalg.norm(b, axis=1)
    rms = float(np.sqrt(np.mean(nb * nb)))
    if rms == 0.0:
        return 0.0 if not np.any(d) else float("inf")
    return float(np.max(d / (tol * (nb + rms))))


def state_errors(x, v, ref_x, ref_v, x0):
    """Errors of a final state against the oracle's, measured on what the
    rollout changed: the displacement x - x0 and the velocity.
      disp, vel        rel-L2 of the displacement and of the velocity
      disp_entry,
      vel_entry        entry_ratio numerators at tol = 1 (max over nodes of
                       |err_i| / (|ref_i| + rms(ref)))
      maxabs_bbox      max over nodes |x_i - ref_i| / bbox diagonal (C19)
      pos_centroid     |x - ref| / |ref - centroid(ref)| (C19's position norm)"""
    x, v, ref_x, ref_v, x0 = (np.asarray(t, dtype=np.float64) for t in (x, v, ref_x, ref_v, x0))
    du, dr = x - x0, ref_x - x0
    diag = float(np.linalg.norm(ref_x.max(axis=0) - ref_x.min(axis=0)))
    return {
        "disp": rel(du, dr),
        "vel": rel(v, ref_v),
        "disp_entry": entry_ratio(du, dr, 1.0),
        "vel_entry": entry_ratio(v, ref_v, 1.0),
        "maxabs_bbox": float(np.max(np.linalg.norm(x - ref_x, axis=1)) / diag),
        "pos_centroid": rel_pos(x, ref_x),
    }


def check_state(x, v, ref_x, ref_v, x0, tol, vtol=None, vel_entry=True):
    """Final state against the oracle: rel-L2 of the displacement and of the
    velocity <= tol (vtol), and every node's displacement within
    entry_bar(tol) (|ref_i| + rms(ref)).  The same per-node bar on the
    velocity is asserted when `vel_entry` (runs without contact); with
    contact it is only reported: a node whose contact switches on one step
    earlier or later in FP32 than in FP64 (C20) changes its velocity by a
    whole step's contact impulse while its position barely moves.  Returns
    the errors (state_errors)."""
    vtol = tol if vtol is None else vtol
    e = state_errors(x, v, ref_x, ref_v, x0)
    print("state errors:", {k: f"{val:.3e}" for k, val in e.items()})
    assert e["disp"] <= tol, ("displacement rel-L2", e)
    assert e["vel"] <= vtol, ("velocity rel-L2", e)
    assert e["disp_entry"] <= entry_bar(tol), ("displacement per node", e)
    if vel_entry:
        assert e["vel_entry"] <= entry_bar(vtol), ("velocity per node", e)
    return e


def rel_pos(x, ref):
    """C19 position norm: |x - ref|_2 / |ref - centroid(ref)|_2."""
    return float(np.linalg.norm(x - ref) / np.linalg.norm(ref - ref.mean(axis=0)))


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def cosine(a, b):
    a, b = np.ravel(a), np.ravel(b)
    return float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)))


def make_target(problem, steps, seed=0, scale=1.1):
    """C18: final state of the oracle with reference parameters (mu, lambda
    scaled by `scale`) plus N(0, 1 mm^2) noise."""
    ref = I.Problem(**{f: getattr(problem, f) for f in problem.__dataclass_fields__})
    ref.mu = problem.mu * scale
    ref.lam = problem.lam * scale
    xS, _ = O.Model(ref).rollout(problem.x0, problem.v0, problem.dt, steps)
    return xS + I.position_noise(problem.n_nodes, seed=seed)


def run_gpu(gs, ctx, problem, steps, target=None, K=0, patch_elems=0, block_threads=0, grads=True,
            block_threads_adj=0):
    import torch
    m = gs.Mesh(ctx, problem, patch_elems=patch_elems, block_threads=block_threads,
                block_threads_adj=block_threads_adj)
    N = problem.n_nodes
    dev = "cuda"
    tgt = None if target is None else torch.tensor(target, dtype=torch.float32, device=dev)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    m.rollout(problem.dt, steps, K, tgt, loss if tgt is not None else None)
    x = torch.empty(N, 3, device=dev)
    v = torch.empty(N, 3, device=dev)
    m.get_state(x, v)
    out = {"mesh": m}
    if grads:
        E, B = problem.n_elems, problem.n_hinges
        g = {k: torch.zeros(E, dtype=torch.float64, device=dev) for k in ("d_mu", "d_lambda", "d_density")}
        g["d_x0"] = torch.zeros(N, 3, device=dev)
        g["d_v0"] = torch.zeros(N, 3, device=dev)
        g["d_mass"] = torch.zeros(N, dtype=torch.float64, device=dev)
        if B:
            g["d_kb"] = torch.zeros(B, dtype=torch.float64, device=dev)
        m.adjoint(g)
        torch.cuda.synchronize()
        out.update({k: t.cpu().numpy().astype(np.float64) for k, t in g.items()})
    torch.cuda.synchronize()
    out["x"] = x.cpu().numpy().astype(np.float64)
    out["v"] = v.cpu().numpy().astype(np.float64)
    out["loss"] = float(loss.item())
    return out


def run_oracle(problem, steps, target=None):
    m = O.Model(problem)
    xS, vS = m.rollout(problem.x0, problem.v0, problem.dt, steps)
    out = {"x": xS, "v": vS}
    if target is not None:
        L, g = m.loss_grad(problem.x0, problem.v0, problem.dt, steps, target)
        out["loss"] = L
        out.update(g)
    return out
