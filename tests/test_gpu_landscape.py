"""The paper's deformable loss landscape (Sec. 3 "Loss landscapes": a beam
hanging under gravity with mu = lambda = 1000 has a unique, dominant
minimum of the loss there), swept in one batched launch per step on the
CUDA path; the losses agree with the FP64 oracle, and gradient descent on
mu = lambda through the adjoint recovers 1000.  (The rigid-body landscape
over mass is in test_gpu_rigid.py.)
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2104_02646_gb300 import inputs as I

pytestmark = pytest.mark.gpu

GRID = [300.0, 500.0, 700.0, 850.0, 1000.0, 1200.0, 1500.0, 2000.0, 3000.0]


def test_beam_landscape_in_one_batch(gs):
    import torch
    S = 300
    ctx = gs.Context(0)
    probs = [I.hanging_beam(mu, steps=S) for mu in GRID]
    meshes = [gs.Mesh(ctx, p) for p in probs]
    batch = gs.Batch(ctx, meshes)
    batch.rollout([p.dt for p in probs], S, 1)
    xs = []
    for m in meshes:
        x = torch.empty(m.n_nodes, 3, device="cuda")
        m.get_state(x)
        xs.append(x.cpu().numpy().astype(np.float64))
    ref = xs[GRID.index(1000.0)]
    L = [float(((x - ref) ** 2).sum()) for x in xs]
    i1 = GRID.index(1000.0)
    assert L[i1] == 0.0
    assert all(L[i] > L[i + 1] for i in range(i1)), L
    assert all(L[i] < L[i + 1] for i in range(i1, len(L) - 1)), L
    # the same landscape from the oracle
    ref_o, _ = O.Model(probs[i1]).rollout(probs[i1].x0, probs[i1].v0, probs[i1].dt, S)
    for k in (1, 3, 6, 8):
        x_o, _ = O.Model(probs[k]).rollout(probs[k].x0, probs[k].v0, probs[k].dt, S)
        Lo = float(((x_o - ref_o) ** 2).sum())
        assert abs(L[k] - Lo) <= 1e-2 * Lo, (GRID[k], L[k], Lo)
    batch.close()
    for m in meshes:
        m.close()


def test_lame_recovery_through_the_adjoint(gs):
    import torch
    from paper_2104_02646_gb300 import autograd as A
    S = 300
    ctx = gs.Context(0)
    p = I.hanging_beam(1000.0, steps=S)
    mesh = gs.Mesh(ctx, p)
    dev = "cuda"
    f32 = dict(dtype=torch.float32, device=dev)
    x0 = torch.tensor(p.x0, **f32)
    v0 = torch.zeros_like(x0)
    rho = torch.tensor(p.rho, **f32)
    ones = torch.ones(p.n_elems, **f32)
    with torch.no_grad():
        target, _ = A.rollout(mesh, p.dt, S, 1000.0 * ones, 1000.0 * ones, rho, x0, v0, K=1)
    log_mu = torch.tensor(np.log(2500.0), dtype=torch.float64, device=dev, requires_grad=True)
    opt = torch.optim.Adam([log_mu], lr=0.05)
    for _ in range(80):
        opt.zero_grad()
        mu = torch.exp(log_mu).to(torch.float32) * ones
        xS, _ = A.rollout(mesh, p.dt, S, mu, mu, rho, x0, v0, K=1)
        loss = ((xS - target) ** 2).sum()
        loss.backward()
        opt.step()
    assert abs(float(torch.exp(log_mu.detach())) - 1000.0) < 20.0, float(torch.exp(log_mu.detach()))
    mesh.close()
