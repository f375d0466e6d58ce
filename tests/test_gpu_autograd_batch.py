"""torch.autograd integration of the checkpointed rollout, and batching:
each mesh gives bitwise the same results alone and inside a batch."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2104_02646_gb300 import inputs as I

from gpu_util import cosine, make_target, rel, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(gs):
    return gs.Context(0)


def test_autograd_rollout_matches_oracle(gs, ctx):
    import torch

    from paper_2104_02646_gb300.autograd import rollout
    p = I.block(n=5, steps=80, seed=31)
    tgt = make_target(p, 80)
    L_ref, g_ref = O.Model(p).loss_grad(p.x0, p.v0, p.dt, 80, tgt)
    dev = "cuda"
    mesh = gs.Mesh(ctx, p, patch_elems=150)
    mu = torch.tensor(p.mu, device=dev, requires_grad=True)
    lam = torch.tensor(p.lam, device=dev, requires_grad=True)
    rho = torch.tensor(p.rho, device=dev, requires_grad=True)
    x0 = torch.tensor(p.x0, device=dev, requires_grad=True)
    v0 = torch.tensor(p.v0, device=dev, requires_grad=True)
    xS, vS = rollout(mesh, p.dt, 80, mu, lam, rho, x0, v0)
    loss = ((xS.double() - torch.tensor(tgt, device=dev)) ** 2).sum()
    loss.backward()
    assert float(loss.detach()) == pytest.approx(L_ref, rel=1e-3)
    for t, k in ((mu, "tet_mu"), (lam, "tet_lam"), (rho, "tet_rho"), (v0, "v0"), (x0, "x0")):
        a = t.grad.detach().cpu().numpy().astype(np.float64)
        assert rel(a, g_ref[k]) <= 1e-3, k
        assert cosine(a, g_ref[k]) >= 0.9999, k


def test_autograd_velocity_seed(gs, ctx):
    # a loss on the final velocity seeds dL/dv(S) only
    import torch

    from paper_2104_02646_gb300.autograd import rollout
    p = I.block(n=4, steps=40, seed=32)
    dev = "cuda"
    mesh = gs.Mesh(ctx, p, patch_elems=100)
    v0 = torch.tensor(p.v0, device=dev, requires_grad=True)
    args = [torch.tensor(a, device=dev) for a in (p.mu, p.lam, p.rho, p.x0)]
    xS, vS = rollout(mesh, p.dt, 40, *args, v0)
    (vS.double() ** 2).sum().backward()
    # the oracle's adjoint seeded with dL/dv(S) = 2 v(S) of its own rollout
    m = O.Model(p)
    _, vS_ref = m.rollout(p.x0, p.v0, p.dt, 40)
    _, g = m.loss_grad(p.x0, p.v0, p.dt, 40, None, vbar=2.0 * vS_ref)
    a = v0.grad.cpu().numpy().astype(np.float64)
    assert rel(a, g["v0"]) <= 1e-3
    assert cosine(a, g["v0"]) >= 0.9999


def test_batch_bitwise_equal_to_alone(gs, ctx):
    import torch
    probs = [I.batch_member(i, steps=60, lo=300, hi=3000, seed=4) for i in range(5)]
    probs.append(I.cloth("3s", n=12, steps=60, grid_scaled=True))
    targets = [make_target(p, 60) for p in probs]
    alone = [run_gpu(gs, ctx, p, 60, t, patch_elems=256) for p, t in zip(probs, targets)]
    meshes = [gs.Mesh(ctx, p, patch_elems=256) for p in probs]
    batch = gs.Batch(ctx, meshes)
    dev = "cuda"
    tg = [torch.tensor(t, dtype=torch.float32, device=dev) for t in targets]
    loss = torch.zeros(len(probs), dtype=torch.float64, device=dev)
    batch.rollout([p.dt for p in probs], 60, 0, tg, loss)
    grads = []
    for p in probs:
        E, N = p.n_elems, p.n_nodes
        g = {k: torch.zeros(E, dtype=torch.float64, device=dev) for k in ("d_mu", "d_lambda", "d_density")}
        g["d_v0"] = torch.zeros(N, 3, device=dev)
        if p.n_hinges:
            g["d_kb"] = torch.zeros(p.n_hinges, dtype=torch.float64, device=dev)
        grads.append(g)
    batch.adjoint(grads)
    torch.cuda.synchronize()
    for i, (m, a) in enumerate(zip(meshes, alone)):
        x = torch.empty(probs[i].n_nodes, 3, device=dev)
        m.get_state(x)
        np.testing.assert_array_equal(x.cpu().numpy(), a["x"].astype(np.float32))
        assert float(loss[i]) == a["loss"]
        for k in grads[i]:
            np.testing.assert_array_equal(grads[i][k].cpu().numpy(), a[k].astype(grads[i][k].cpu().numpy().dtype))


@pytest.mark.gpu
def test_autotune_picks_a_working_shape(gs, ctx, tmp_path):
    from paper_2104_02646_gb300 import autotune as A
    p = I.block(n=8, steps=30, seed=4)
    cache = str(tmp_path / "tune.json")
    r = A.tune(ctx, p, steps=5, cache=cache, candidates=((256, 128), (128, 64), (100000, 128)))
    assert (r["patch_elems"], r["block_threads"]) in ((256, 128), (128, 64))
    assert r["K"] == 1  # a 30-step rollout of 729 nodes fits any budget
    # the too-large patch is skipped, not fatal
    assert any(t["ms"] is None for t in r["timings"])
    again = A.tune(ctx, p, steps=5, cache=cache)
    assert again["cached"] and again["patch_elems"] == r["patch_elems"]
    # the tuned shape gives the same gradients as the default one
    tgt = make_target(p, 30)
    a = run_gpu(gs, ctx, p, 30, tgt, K=r["K"], patch_elems=r["patch_elems"], block_threads=r["block_threads"])
    b = run_gpu(gs, ctx, p, 30, tgt)
    assert rel(a["d_mu"], b["d_mu"]) <= 1e-5
