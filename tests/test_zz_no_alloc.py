"""gs_loss_noalloc: the position loss for callers that cannot allocate device
memory (e.g. a real-time control loop, or a host whose memory pool forbids
library allocations).  Checked through the C ABI against the loss of the
regular entry point (gs_rollout with a target) on two calls in a row; the
second call reuses the library's fixed scratch array left by the first."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_loss_matches_rollout_loss_twice(gs):
    import torch

    from paper_2104_02646_gb300 import inputs as I
    L = gs.load()
    p = I.block(n=6, steps=60, seed=21)
    N = p.n_nodes
    ctx = gs.Context(0)
    mesh = gs.Mesh(ctx, p, patch_elems=200)
    target = torch.tensor(p.X + I.position_noise(N, sigma=2e-3, seed=21), dtype=torch.float32, device="cuda")
    loss_ref = torch.zeros(1, dtype=torch.float64, device="cuda")
    mesh.rollout(p.dt, 60, 0, target, loss_ref)
    x = torch.empty(N, 3, device="cuda")
    mesh.get_state(x)
    torch.cuda.synchronize()
    ref = float(loss_ref.item())
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    grad = torch.zeros(N, 3, device="cuda")
    for _ in range(2):
        out.fill_(float("nan"))
        grad.fill_(float("nan"))
        gs.check(L.gs_loss_noalloc(C.c_void_p(x.data_ptr()), C.c_void_p(target.data_ptr()), N,
                                   C.c_void_p(out.data_ptr()), C.c_void_p(grad.data_ptr()), stream))
        torch.cuda.synchronize()
        assert float(out.item()) == pytest.approx(ref, rel=1e-3)
        np.testing.assert_allclose(grad.cpu().numpy(), 2.0 * (x - target).cpu().numpy(), rtol=1e-5, atol=1e-9)
        # the same sum in float64 by torch: only the summation order differs
        exact = float(((x.double() - target.double()) ** 2).sum().item())
        assert float(out.item()) == pytest.approx(exact, rel=1e-12)


@pytest.mark.parametrize("n_nodes", [0, 1, 257, 1_000_003])
def test_noalloc_sizes_and_optional_seed(gs, n_nodes):
    # empty input, a single block, a ragged second block and thousands of
    # blocks (every partial must be written and summed once); without dL_dx
    # only the loss is produced
    import torch
    L = gs.load()
    g = torch.Generator(device="cpu").manual_seed(n_nodes)
    x = torch.randn(max(n_nodes, 1), 3, generator=g).cuda()
    t = torch.randn(max(n_nodes, 1), 3, generator=g).cuda()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    for with_seed in (False, True):
        grad = torch.full((max(n_nodes, 1), 3), float("nan"), device="cuda")
        gs.check(L.gs_loss_noalloc(C.c_void_p(x.data_ptr()), C.c_void_p(t.data_ptr()), n_nodes,
                                   C.c_void_p(out.data_ptr()), C.c_void_p(grad.data_ptr()) if with_seed else None,
                                   stream))
        torch.cuda.synchronize()
        exact = float(((x[:n_nodes].double() - t[:n_nodes].double()) ** 2).sum().item())
        if n_nodes == 0:
            assert float(out.item()) == 0.0
        else:
            assert float(out.item()) == pytest.approx(exact, rel=1e-12)
        if with_seed and n_nodes:
            np.testing.assert_array_equal(grad[:n_nodes].cpu().numpy(),
                                          (2.0 * (x[:n_nodes].double() - t[:n_nodes].double())).float().cpu().numpy())
        if not with_seed:
            assert torch.isnan(grad).all()  # nothing written


def test_noalloc_rejects_sizes_beyond_its_scratch(gs):
    import torch
    L = gs.load()
    x = torch.zeros(4, 3, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = L.gs_loss_noalloc(C.c_void_p(x.data_ptr()), C.c_void_p(x.data_ptr()), gs.GS_NOALLOC_MAX_NODES + 1,
                           C.c_void_p(out.data_ptr()), None, None)
    assert st == gs.GS_EINVAL
    assert b"GS_NOALLOC_MAX_NODES" in L.gs_last_error()
