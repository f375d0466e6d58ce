"""Helpers shared by the GPU parity tests: run a Problem through the CUDA
library (via the C-ABI binding) and through the FP64 oracle, and compare."""
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


def check_grads(g_gpu, g_ref, keys, skip=()):
    for ok, gk in keys.items():
        if ok in skip:
            continue
        a, b = g_gpu[gk], g_ref[ok]
        assert np.all(np.isfinite(a)), gk
        assert rel(a, b) <= GRAD_REL, (gk, rel(a, b))
        assert cosine(a, b) >= GRAD_COS, (gk, cosine(a, b))


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


def run_gpu(gs, ctx, problem, steps, target=None, K=0, patch_elems=0, block_threads=0, grads=True):
    import torch
    m = gs.Mesh(ctx, problem, patch_elems=patch_elems, block_threads=block_threads)
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
