"""Parity at the benchmark sizes of the NEXT workloads, in the launch shapes
the benchmark times: short oracle rollouts of the full meshes with
actuation sequences and air; a window of the 512^2 frame of the 256^2 cloth
(the oracle is exact when given only the triangles whose cutoff box reaches
the window: the others contribute no coverage); sampled bodies of the
16,384-body rigid workload.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from oracle import render_oracle as RO
from paper_2104_02646_gb300 import inputs as I

from gpu_util import (CLOTH_KEYS, GRAD_COS, GRAD_REL, POS_CONTACT, TET_KEYS, check_grads, cosine, make_target,
                      quat_tangent, rel, rel_pos)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(gs):
    return gs.Context(0)


def _adjoint(gs, m, p, S, seq=False, hseq=False):
    import torch
    E, B, N = p.n_elems, p.n_hinges, p.n_nodes
    g = {k: torch.zeros(E, dtype=torch.float64, device="cuda") for k in ("d_mu", "d_lambda", "d_density")}
    g["d_x0"] = torch.zeros(N, 3, device="cuda")
    g["d_v0"] = torch.zeros(N, 3, device="cuda")
    if B:
        g["d_kb"] = torch.zeros(B, dtype=torch.float64, device="cuda")
    if seq:
        g["d_act_seq"] = torch.zeros(S, E, device="cuda")
    if hseq:
        g["d_hinge_act_seq"] = torch.zeros(S, B, device="cuda")
    m.adjoint(g)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy().astype(np.float64) for k, v in g.items()}


def _run(gs, ctx, p, S, tgt, seq=None, hseq=None):
    import torch
    m = gs.Mesh(ctx, p, patch_elems=256, block_threads=128)
    m.set_act_seq(None if seq is None else torch.tensor(seq, dtype=torch.float32, device="cuda"),
                  None if hseq is None else torch.tensor(hseq, dtype=torch.float32, device="cuda"))
    m.rollout(p.dt, S, 1, torch.tensor(tgt, dtype=torch.float32, device="cuda"))
    x = torch.empty(p.n_nodes, 3, device="cuda")
    m.get_state(x)
    out = _adjoint(gs, m, p, S, seq is not None, hseq is not None)
    out["x"] = x.cpu().numpy().astype(np.float64)
    m.close()
    return out


def test_block64_actuated_full_size(gs, ctx):
    S = 2
    p = I.block(n=64, steps=S)
    rng = np.random.default_rng(0)
    seq = 0.1 * rng.uniform(-1, 1, (S, p.n_elems))
    tgt = make_target(p, S)
    om = O.Model(p, act_seq=seq)
    xS, _ = om.rollout(p.x0, p.v0, p.dt, S)
    _, ref = om.loss_grad(p.x0, p.v0, p.dt, S, tgt, act_seq_grad=True)
    out = _run(gs, ctx, p, S, tgt, seq=seq)
    assert rel_pos(out["x"], xS) <= POS_CONTACT
    check_grads(out, ref, TET_KEYS)
    a, b = out["d_act_seq"], ref["tet_act_seq"]
    assert rel(a, b) <= GRAD_REL and cosine(a, b) >= GRAD_COS


def test_cloth256_air_and_hinge_actuation_full_size(gs, ctx):
    S = 8
    p = I.cloth("3s", n=256, steps=S, height=0.29)
    p.air = I.Air(k_drag=0.6, k_lift=0.4, wind=(2.0, 0.5, -1.0))
    rng = np.random.default_rng(1)
    hseq = 0.2 * rng.uniform(-1, 1, (S, p.n_hinges))
    tgt = make_target(p, S)
    om = O.Model(p, hinge_act_seq=hseq)
    xS, _ = om.rollout(p.x0, p.v0, p.dt, S)
    _, ref = om.loss_grad(p.x0, p.v0, p.dt, S, tgt, act_seq_grad=True)
    out = _run(gs, ctx, p, S, tgt, hseq=hseq)
    assert rel_pos(out["x"], xS) <= POS_CONTACT
    check_grads(out, ref, CLOTH_KEYS)
    a, b = out["d_hinge_act_seq"], ref["hinge_act_seq"]
    assert rel(a, b) <= GRAD_REL and cosine(a, b) >= GRAD_COS


def test_render_window_of_the_512_frame(gs, ctx):
    # the benchmark's frame of the 256^2 cloth; a 32 x 32 window of it near the
    # cloth's edge, rendered by the library with every triangle
    import dataclasses
    import torch
    q = I.cloth("3s", n=256, steps=1)
    full = I.look_at((1.3, 1.2, -0.6), (0.5, 0.3, 0.5), width=512, height=512, fov_deg=50.0)
    spec = I.RenderSpec()
    col = I.vertex_colours(q.X, seed=0)
    u, v, z = (t.numpy() for t in RO.project(torch.tensor(q.X), full))
    # a window on the cloth's silhouette: around the projected corner node 0
    x0w, y0w = int(u[0]) - 16, int(v[0]) - 16
    win = dataclasses.replace(full, cx=full.cx - x0w, cy=full.cy - y0w, width=32, height=32)
    r = math.sqrt(RO.cutoff_d2(spec.sigma)) + 1.0
    U, V = u[q.elems], v[q.elems]
    keep = ((U.max(axis=1) + r >= x0w) & (U.min(axis=1) - r <= x0w + 32) &
            (V.max(axis=1) + r >= y0w) & (V.min(axis=1) - r <= y0w + 32))
    F_sub = q.elems[keep]
    assert 0 < len(F_sub) < len(q.elems)
    dimg = np.random.default_rng(2).normal(size=(32, 32, 4))
    img, gx, gc = RO.render_grad(q.X, F_sub, col, win, spec, dimg)
    rast = gs.Raster(ctx, q.n_nodes, q.elems, win, spec)
    x = torch.tensor(q.X, dtype=torch.float32, device="cuda")
    c = torch.tensor(col, dtype=torch.float32, device="cuda")
    out = torch.empty(32, 32, 4, device="cuda")
    rast.forward(x, c, out)
    dx, dc = torch.empty_like(x), torch.empty_like(c)
    rast.backward(torch.tensor(dimg, dtype=torch.float32, device="cuda"), dx, dc)
    o = out.cpu().numpy().astype(np.float64)
    assert 0.05 < o[..., 3].mean() < 0.95  # the window straddles the silhouette
    assert rel(o, img.numpy()) <= 1e-4 and np.abs(o - img.numpy()).max() <= 1e-3
    for a, b in ((dx.cpu().numpy().astype(np.float64), gx.numpy()), (dc.cpu().numpy().astype(np.float64), gc.numpy())):
        assert rel(a, b) <= GRAD_REL and cosine(a, b) >= GRAD_COS
    rast.close()


def test_rigid16384_sampled_bodies(gs, ctx):
    import torch
    S, nb = 300, 16384
    bodies = I.rigid_batch(nb, seed=0, n=5, steps=S)
    rig = gs.Rigid(ctx, bodies)
    s0 = torch.tensor(rig.state0(), device="cuda")
    sS = torch.empty_like(s0)
    rig.rollout(1e-3, S, s0, sS)
    seed = np.random.default_rng(3).normal(size=(nb, 13))
    g = {"d_state0": torch.zeros(nb, 13, device="cuda"), "d_mass": torch.zeros(nb, dtype=torch.float64, device="cuda"),
         "d_inertia": torch.zeros(nb, 6, dtype=torch.float64, device="cuda"),
         "d_contact": torch.zeros(nb, 4, dtype=torch.float64, device="cuda")}
    rig.adjoint(g, seed=torch.tensor(seed, dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    assert rig.check_finite() == gs.GS_OK
    sS = sS.cpu().numpy().astype(np.float64)
    out = {k: v.cpu().numpy().astype(np.float64) for k, v in g.items()}
    for b in (0, 8191, 16383):
        ro = O.Rigid(bodies[b])
        ref_s = ro.rollout(bodies[b].state0, 1e-3, S)
        np.testing.assert_allclose(sS[b, :3], ref_s[:3], atol=1e-3 * (1 + np.abs(ref_s[:3]).max()))
        _, ref = ro.loss_grad(bodies[b].state0, 1e-3, S, None, seed[b])
        q0 = bodies[b].state0[3:7]
        for a, r in ((quat_tangent(out["d_state0"][b], q0), quat_tangent(ref["state0"], q0)),
                     (out["d_contact"][b], ref["contact"]),
                     (out["d_inertia"][b], ref["inertia"])):
            if np.linalg.norm(r) == 0:
                continue
            assert rel(a, r) <= GRAD_REL and cosine(a, r) >= GRAD_COS, (b, rel(a, r))
        assert abs(out["d_mass"][b] - ref["mass"]) <= GRAD_REL * abs(ref["mass"]) + 1e-12
    rig.close()
