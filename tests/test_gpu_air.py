"""The lift/drag air model on cloth (App. A.1) on the CUDA path against the
FP64 oracle, and the cloth-control workload of Sec. 3: recovering a thrown
cloth's initial velocity (Table 3, "per-particle velocity") by gradient
descent through the library's adjoint.

Tolerances as for the rest of the path: positions rel-L2 <= 1e-4
contact-free, <= 1e-3 with contact; every gradient rel-L2 <= 1e-3 and
cosine >= 0.9999.
"""
import dataclasses

import numpy as np
import pytest

from paper_2104_02646_gb300 import inputs as I

from gpu_util import CLOTH_KEYS, POS_CONTACT, POS_FREE, check_grads, make_target, rel_pos, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(gs):
    return gs.Context(0)


def _oracle(p, S, tgt):
    from oracle import oracle as O
    m = O.Model(p)
    xS, vS = m.rollout(p.x0, p.v0, p.dt, S)
    L, g = m.loss_grad(p.x0, p.v0, p.dt, S, tgt)
    g["x"], g["v"], g["loss"] = xS, vS, L
    return g


@pytest.mark.parametrize("pe", [0, 64])
def test_thrown_cloth_parity(gs, ctx, pe):
    # 162 triangles in flight (no contact within the horizon), lift and drag
    S = 300
    p = I.cloth_throw(n=10, steps=S, seed=1)
    tgt = make_target(p, S)
    ref = _oracle(p, S, tgt)
    out = run_gpu(gs, ctx, p, S, tgt, patch_elems=pe)
    assert rel_pos(out["x"], ref["x"]) <= POS_FREE
    check_grads(out, ref, CLOTH_KEYS)
    out["mesh"].close()


def test_cloth_with_wind_on_the_sphere_parity(gs, ctx):
    # pressed onto the sphere from step 0 with a cross wind: air + contact
    S = 40
    p = I.cloth("3s", n=12, steps=S, grid_scaled=True, height=0.29)
    p.air = I.Air(k_drag=0.6, k_lift=0.4, wind=(1.5, 0.3, -0.8))
    tgt = make_target(p, S)
    ref = _oracle(p, S, tgt)
    out = run_gpu(gs, ctx, p, S, tgt, patch_elems=64)
    assert rel_pos(out["x"], ref["x"]) <= POS_CONTACT
    check_grads(out, ref, CLOTH_KEYS)
    out["mesh"].close()


def test_air_checkpointing_is_bitwise_invariant(gs, ctx):
    S = 45
    p = I.cloth_throw(n=9, steps=S, seed=2)
    tgt = make_target(p, S)
    a = run_gpu(gs, ctx, p, S, tgt, K=1, patch_elems=64)
    b = run_gpu(gs, ctx, p, S, tgt, K=7, patch_elems=64)
    for k in ("x", "d_v0", "d_x0", "d_mu", "d_lambda", "d_kb", "d_density"):
        np.testing.assert_array_equal(a[k], b[k])
    a["mesh"].close()
    b["mesh"].close()


def test_air_off_is_the_plain_cloth(gs, ctx):
    S = 30
    p = I.cloth_throw(n=8, steps=S, seed=3)
    q = dataclasses.replace(p, air=None)
    tgt = make_target(q, S)
    a = run_gpu(gs, ctx, q, S, tgt)
    m = gs.Mesh(ctx, p)
    m.set_air(None)
    import torch
    t = torch.tensor(tgt, dtype=torch.float32, device="cuda")
    m.rollout(p.dt, S, 0, t)
    x = torch.empty(p.n_nodes, 3, device="cuda")
    m.get_state(x)
    np.testing.assert_array_equal(x.cpu().numpy(), a["x"].astype(np.float32))
    # and with air the state differs
    m.set_air(p.air)
    m.reset()
    m.rollout(p.dt, S, 0)
    m.get_state(x)
    assert np.abs(x.cpu().numpy() - a["x"]).max() > 0
    m.close()
    a["mesh"].close()


def test_air_errors(gs, ctx):
    tet = gs.Mesh(ctx, I.block(n=2, steps=1))
    with pytest.raises(gs.GradsimError) as ei:
        tet.set_air(I.Air())
    assert ei.value.status == gs.GS_EINVAL
    cl = gs.Mesh(ctx, I.cloth("3s", n=6, steps=1))
    for bad in (I.Air(k_drag=-1.0), I.Air(k_lift=float("nan")), I.Air(wind=(0.0, float("inf"), 0.0))):
        with pytest.raises(gs.GradsimError) as ei:
            cl.set_air(bad)
        assert ei.value.status == gs.GS_EINVAL
    srv = gs.Server(ctx, budget=1 << 30)
    with pytest.raises(ValueError):
        srv.submit(I.cloth_throw(n=7, steps=10), np.zeros((49, 3)))
    srv.close()
    tet.close()
    cl.close()


def test_initial_velocity_is_recovered_through_the_adjoint(gs, ctx):
    # control-cloth: the target is where a reference throw lands after
    # 0.05 s; Adam on the per-node initial velocity from a perturbed guess
    import torch
    from paper_2104_02646_gb300 import autograd as A
    S = 500
    p = I.cloth_throw(n=8, steps=S, seed=5)
    mesh = gs.Mesh(ctx, p)
    dev = "cuda"
    mu = torch.tensor(p.mu, dtype=torch.float32, device=dev)
    lam = torch.tensor(p.lam, dtype=torch.float32, device=dev)
    rho = torch.tensor(p.rho, dtype=torch.float32, device=dev)
    x0 = torch.tensor(p.x0, dtype=torch.float32, device=dev)
    v_ref = torch.tensor(p.v0, dtype=torch.float32, device=dev)
    with torch.no_grad():
        xT, _ = A.rollout(mesh, p.dt, S, mu, lam, rho, x0, v_ref)
    v = (v_ref + torch.tensor([0.4, -0.3, 0.25], device=dev)).clone().requires_grad_(True)
    opt = torch.optim.Adam([v], lr=0.05)
    losses = []
    for it in range(30):
        opt.zero_grad()
        xS, _ = A.rollout(mesh, p.dt, S, mu, lam, rho, x0, v)
        loss = ((xS - xT) ** 2).sum()
        loss.backward()
        opt.step()
        losses.append(float(loss.detach()))
    assert losses[-1] < 0.05 * losses[0], losses
    err0 = float(torch.tensor([0.4, -0.3, 0.25]).norm())
    err = float((v.detach() - v_ref).mean(dim=0).norm())
    assert err < 0.25 * err0, (err, err0)
    mesh.close()
