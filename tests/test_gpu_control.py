"""Time-varying actuation (the control input of the paper's visuomotor
control experiments, Sec. 3) on the CUDA path against the FP64 oracle, and
the App. D controller (sinusoids -> FC without bias -> tanh) trained through
the library's adjoint.

Tolerances as for the rest of the path: positions rel-L2 <= 1e-3 with
contact; every gradient, including the per-step actuation gradients,
rel-L2 <= 1e-3 and cosine >= 0.9999.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2104_02646_gb300 import inputs as I

from gpu_util import (CLOTH_KEYS, GRAD_COS, GRAD_REL, POS_CONTACT, TET_KEYS, check_grads, cosine, make_target, rel,
                      rel_pos)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(gs):
    return gs.Context(0)


def _seq(S, n, seed, scale=0.2):
    rng = np.random.default_rng(seed)
    t = np.arange(S)[:, None]
    return scale * np.sin(0.05 * t * rng.uniform(0.5, 2.0, n)[None, :] + rng.uniform(0.0, 6.28, n)[None, :])


def _run(gs, ctx, p, S, tgt, seq=None, hseq=None, K=0, pe=0):
    import torch
    dev = "cuda"
    m = gs.Mesh(ctx, p, patch_elems=pe)
    m.set_act_seq(None if seq is None else torch.tensor(seq, dtype=torch.float32, device=dev),
                  None if hseq is None else torch.tensor(hseq, dtype=torch.float32, device=dev))
    t = torch.tensor(tgt, dtype=torch.float32, device=dev)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    m.rollout(p.dt, S, K, t, loss)
    x = torch.empty(p.n_nodes, 3, device=dev)
    v = torch.empty_like(x)
    m.get_state(x, v)
    E, B, N = p.n_elems, p.n_hinges, p.n_nodes
    g = {k: torch.zeros(E, dtype=torch.float64, device=dev) for k in ("d_mu", "d_lambda", "d_density")}
    g["d_x0"] = torch.zeros(N, 3, device=dev)
    g["d_v0"] = torch.zeros(N, 3, device=dev)
    if B:
        g["d_kb"] = torch.zeros(B, dtype=torch.float64, device=dev)
    if seq is not None:
        g["d_act_seq"] = torch.zeros(S, E, device=dev)
    if hseq is not None:
        g["d_hinge_act_seq"] = torch.zeros(S, B, device=dev)
    m.adjoint(g)
    torch.cuda.synchronize()
    out = {k: t_.cpu().numpy().astype(np.float64) for k, t_ in g.items()}
    out["x"] = x.cpu().numpy().astype(np.float64)
    out["loss"] = float(loss.item())
    m.close()
    return out


def _oracle(p, S, tgt, seq=None, hseq=None):
    m = O.Model(p, act_seq=seq, hinge_act_seq=hseq)
    xS, _ = m.rollout(p.x0, p.v0, p.dt, S)
    L, g = m.loss_grad(p.x0, p.v0, p.dt, S, tgt, act_seq_grad=True)
    g["x"] = xS
    g["loss"] = L
    return g


def _check_seq(a, b):
    assert np.all(np.isfinite(a))
    assert rel(a, b) <= GRAD_REL, rel(a, b)
    assert cosine(a, b) >= GRAD_COS, cosine(a, b)


def test_block_actuated_parity(gs, ctx):
    # 135 tets in 3 patches on the ground, random velocities, every element
    # actuated with its own sinusoid
    S = 80
    p = I.block(n=3, steps=S, seed=8)
    seq = _seq(S, p.n_elems, 1)
    tgt = make_target(p, S)
    ref = _oracle(p, S, tgt, seq)
    out = _run(gs, ctx, p, S, tgt, seq, pe=64)
    assert rel_pos(out["x"], ref["x"]) <= POS_CONTACT
    check_grads(out, ref, TET_KEYS)
    _check_seq(out["d_act_seq"], ref["tet_act_seq"])


def test_cloth_actuated_parity(gs, ctx):
    # triangles and hinges actuated, cloth pressed onto the sphere from step 0
    S = 40
    p = I.cloth("3s", n=10, steps=S, grid_scaled=True, height=0.29)
    seq = _seq(S, p.n_elems, 2, 0.1)
    hseq = _seq(S, p.n_hinges, 3, 0.2)
    tgt = make_target(p, S)
    ref = _oracle(p, S, tgt, seq, hseq)
    out = _run(gs, ctx, p, S, tgt, seq, hseq, pe=64)
    assert rel_pos(out["x"], ref["x"]) <= POS_CONTACT
    check_grads(out, ref, CLOTH_KEYS)
    _check_seq(out["d_act_seq"], ref["tri_act_seq"])
    _check_seq(out["d_hinge_act_seq"], ref["hinge_act_seq"])


def test_actuated_checkpointing_is_bitwise_invariant(gs, ctx):
    S = 45
    p = I.block(n=3, steps=S, seed=9)
    seq = _seq(S, p.n_elems, 4)
    tgt = make_target(p, S)
    a = _run(gs, ctx, p, S, tgt, seq, K=1, pe=64)
    b = _run(gs, ctx, p, S, tgt, seq, K=7, pe=64)
    for k in ("x", "d_act_seq", "d_mu", "d_lambda", "d_density", "d_v0", "d_x0"):
        np.testing.assert_array_equal(a[k], b[k])


@pytest.mark.parametrize("S", [30, 100])
def test_step_applies_the_same_rows_as_a_rollout(gs, ctx, S):
    import torch
    p = I.block(n=3, steps=S, seed=10)
    seq = torch.tensor(_seq(S, p.n_elems, 5), dtype=torch.float32, device="cuda")
    xs = []
    for mode in ("step", "rollout"):
        m = gs.Mesh(ctx, p, patch_elems=64)
        m.set_act_seq(seq)
        if mode == "step":
            m.step(p.dt, S)
        else:
            m.rollout(p.dt, S, 1)
        x = torch.empty(p.n_nodes, 3, device="cuda")
        m.get_state(x)
        xs.append(x.cpu().numpy())
        m.close()
    np.testing.assert_array_equal(xs[0], xs[1])


def test_sequence_errors(gs, ctx):
    import ctypes as C
    p = I.block(n=2, steps=1)
    m = gs.Mesh(ctx, p)
    assert gs.load().gs_mesh_set_act_seq(m.h, None, None, -1, gs.GS_MEM_HOST, None) == gs.GS_EINVAL
    bad = np.zeros((3, p.n_elems), dtype=np.float32)
    bad[1, 2] = np.nan
    with pytest.raises(gs.GradsimError) as ei:
        m.set_act_seq(bad, host=True)
    assert ei.value.status == gs.GS_EINVAL
    m.set_act_seq(None)  # clears


def test_controller_trains_through_the_adjoint(gs):
    # App. D controller driving every element of a block; Adam on a final-state
    # loss against the state a reference controller reaches
    import torch
    from paper_2104_02646_gb300 import autograd as A
    from paper_2104_02646_gb300 import control
    ctx = gs.Context(0)
    S = 120
    p = I.block(n=3, steps=S, seed=11)
    mesh = gs.Mesh(ctx, p, patch_elems=64)
    dev = "cuda"
    x0 = torch.tensor(p.x0, dtype=torch.float32, device=dev)
    v0 = torch.tensor(p.v0, dtype=torch.float32, device=dev)
    t = torch.arange(S, dtype=torch.float32, device=dev) * p.dt
    ref = control.SinusoidController(p.n_elems, omega=2 * np.pi * 50, generator=torch.Generator().manual_seed(1)).to(dev)
    with torch.no_grad():
        xT, _ = A.actuated_rollout(mesh, p.dt, S, ref(t), x0, v0)
    ctrl = control.SinusoidController(p.n_elems, omega=2 * np.pi * 50, generator=torch.Generator().manual_seed(2)).to(dev)
    opt = torch.optim.Adam(ctrl.parameters(), lr=0.05)
    losses = []
    for it in range(8):
        opt.zero_grad()
        xS, _ = A.actuated_rollout(mesh, p.dt, S, ctrl(t), x0, v0)
        loss = ((xS - xT) ** 2).sum()
        loss.backward()
        assert torch.isfinite(ctrl.W.grad).all() and ctrl.W.grad.abs().max() > 0
        opt.step()
        losses.append(float(loss.detach()))
    assert losses[-1] < 0.5 * losses[0], losses
