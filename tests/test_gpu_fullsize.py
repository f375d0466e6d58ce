"""Parity at the full sizes of the benchmark configurations, in the launch
shape the benchmark times (256-element patches, 128 consumer threads).  The
oracle computes whole short rollouts of the full meshes (a few steps of the
1.3M-tet block, ten steps of the 256^2 cloth, sampled members of the
512-mesh batch), and the CUDA path is compared with it element by element.
"""
import numpy as np
import pytest

from paper_2104_02646_gb300 import inputs as I

from gpu_util import (CLOTH_KEYS, POS_CONTACT, TET_KEYS, check_grads, make_target, rel_pos, run_gpu,
                      run_oracle)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(gs):
    return gs.Context(0)


@pytest.mark.parametrize("K", [1, 0])
def test_block64_full_size(gs, ctx, K):
    # 1,310,720 tets on the ground (contact from step 0), heterogeneous
    # materials, random velocities: 2 steps, every state kept (K = 1) and the
    # checkpoint-and-recompute path (library K)
    S = 2
    p = I.block(n=64, steps=S)
    assert p.n_elems == 1310720 and p.n_nodes == 274625
    tgt = make_target(p, S)
    ref = run_oracle(p, S, tgt)
    out = run_gpu(gs, ctx, p, S, tgt, K=K, patch_elems=256, block_threads=128)
    assert rel_pos(out["x"], ref["x"]) <= POS_CONTACT
    assert abs(out["loss"] - ref["loss"]) <= 1e-3 * abs(ref["loss"])
    check_grads(out, ref, TET_KEYS)


def test_cloth_256_full_size(gs, ctx):
    # the stable variant of the 256^2 cloth (130,050 triangles, 194,565 hinges),
    # placed 1 cm below the top of the sphere so that contact, membrane and
    # bending respond from step 0 (a flat cloth in free fall has no material
    # sensitivity): 10 steps
    S = 10
    p = I.cloth("3s", n=256, steps=S, height=0.29)
    assert (p.n_nodes, p.n_elems, p.n_hinges) == (65536, 130050, 194565)
    tgt = make_target(p, S)
    ref = run_oracle(p, S, tgt)
    out = run_gpu(gs, ctx, p, S, tgt, K=1, patch_elems=256, block_threads=128)
    assert rel_pos(out["x"], ref["x"]) <= POS_CONTACT
    check_grads(out, ref, CLOTH_KEYS)


def test_batch_512_sampled_members(gs, ctx):
    # all 512 meshes of the batch workload advance together in one launch per
    # step; sampled members (smallest, median, largest) are compared with the
    # oracle run alone
    import torch
    S = 6
    probs = I.batch(n_meshes=512, steps=S)
    # a seeded N(0, 0.1 m/s) initial velocity field on every member, so that the
    # short rollout strains the solids (6 steps of free fall alone would leave
    # the material gradients at exactly zero)
    rng = np.random.default_rng(11)
    for p in probs:
        p.v0 = rng.normal(0.0, 0.1, p.X.shape)
    sizes = np.array([p.n_elems for p in probs])
    assert 8e6 < sizes.sum() < 14e6
    order = np.argsort(sizes)
    picks = [int(order[0]), int(order[len(order) // 2]), int(order[-1])]
    targets = {i: make_target(probs[i], S) for i in picks}
    dev = "cuda"
    meshes = [gs.Mesh(ctx, p, patch_elems=256, block_threads=128) for p in probs]
    batch = gs.Batch(ctx, meshes)
    tg = [torch.tensor(targets[i] if i in targets else p.X, dtype=torch.float32, device=dev)
          for i, p in enumerate(probs)]
    loss = torch.zeros(len(probs), dtype=torch.float64, device=dev)
    batch.rollout([p.dt for p in probs], S, 1, tg, loss)
    grads = []
    for p in probs:
        E, N = p.n_elems, p.n_nodes
        g = {k: torch.zeros(E, dtype=torch.float64, device=dev) for k in ("d_mu", "d_lambda", "d_density")}
        g["d_v0"] = torch.zeros(N, 3, device=dev)
        g["d_x0"] = torch.zeros(N, 3, device=dev)
        grads.append(g)
    batch.adjoint(grads)
    torch.cuda.synchronize()
    for i in picks:
        ref = run_oracle(probs[i], S, targets[i])
        x = torch.empty(probs[i].n_nodes, 3, device=dev)
        meshes[i].get_state(x)
        assert rel_pos(x.cpu().numpy().astype(np.float64), ref["x"]) <= POS_CONTACT
        out = {k: t.cpu().numpy().astype(np.float64) for k, t in grads[i].items()}
        check_grads(out, ref, TET_KEYS)
    batch.close()
    for m in meshes:
        m.close()
