"""The soft rasteriser (Sec. 2 "Differentiable rendering engine") on the CUDA
path against its FP64 oracle, and the image-loss loop it closes: a cloth's
initial velocity recovered from rendered frames through the rasteriser's and
the simulator's adjoints.

Tolerances: image rel-L2 <= 1e-4 and max-abs <= 1e-3 (FP32 coverage and
depth-softmax weights against FP64); gradients rel-L2 <= 1e-3, cosine >=
0.9999, as for the rest of the path.
"""
import numpy as np
import pytest

from oracle import render_oracle as RO
from paper_2104_02646_gb300 import inputs as I

from gpu_util import GRAD_COS, GRAD_REL, cosine, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(gs):
    return gs.Context(0)


def _world(cam, u, v, depth):
    xc = np.array([(u - cam.cx) / cam.fx * depth, (v - cam.cy) / cam.fy * depth, depth])
    return cam.R.T @ (xc - cam.t)


def _random_scene(cam, n_tri, seed, spread=1.2):
    rng = np.random.default_rng(seed)
    X, F = [], []
    for k in range(n_tri):
        c = rng.uniform([-0.2 * cam.width, -0.2 * cam.height], [1.2 * cam.width, 1.2 * cam.height])
        d = rng.uniform(1.5, 4.0)
        for _ in range(3):
            X.append(_world(cam, *(c + rng.normal(0, spread * 0.25 * cam.width, 2)), d + rng.normal(0, 0.2)))
        F.append([3 * k, 3 * k + 1, 3 * k + 2])
    X = np.array(X)
    return X, np.array(F), rng.uniform(0.05, 0.95, X.shape)


def _gpu(gs, ctx, X, F, col, cam, spec, dimg=None):
    import torch
    r = gs.Raster(ctx, X.shape[0], F, cam, spec)
    x = torch.tensor(X, dtype=torch.float32, device="cuda")
    c = torch.tensor(col, dtype=torch.float32, device="cuda")
    img = torch.empty(cam.height, cam.width, 4, device="cuda")
    r.forward(x, c, img)
    out = {"img": img.cpu().numpy().astype(np.float64)}
    if dimg is not None:
        dx, dc = torch.empty_like(x), torch.empty_like(c)
        r.backward(torch.tensor(dimg, dtype=torch.float32, device="cuda"), dx, dc)
        out["dx"] = dx.cpu().numpy().astype(np.float64)
        out["dc"] = dc.cpu().numpy().astype(np.float64)
    torch.cuda.synchronize()
    r.close()
    return out


def _check(out, X, F, col, cam, spec, dimg):
    img, gx, gc = RO.render_grad(X, F, col, cam, spec, dimg)
    img = img.numpy()
    assert rel(out["img"], img) <= 1e-4, rel(out["img"], img)
    assert np.abs(out["img"] - img).max() <= 1e-3
    for a, b in ((out["dx"], gx.numpy()), (out["dc"], gc.numpy())):
        assert np.all(np.isfinite(a))
        assert rel(a, b) <= GRAD_REL, rel(a, b)
        assert cosine(a, b) >= GRAD_COS, cosine(a, b)


@pytest.mark.parametrize("w,h,n_tri,seed", [(40, 28, 6, 0), (64, 64, 25, 1), (17, 33, 3, 2)])
def test_random_triangles_parity(gs, ctx, w, h, n_tri, seed):
    # ragged tiles (sizes not multiples of 16), overlaps at several depths,
    # triangles partly off screen
    cam = I.look_at((0.3, 0.4, -2.5), (0.0, 0.0, 0.0), width=w, height=h, fov_deg=50.0)
    X, F, col = _random_scene(cam, n_tri, seed)
    spec = I.RenderSpec(sigma=0.8, gamma=0.02, bg=(0.9, 0.8, 0.7))
    dimg = np.random.default_rng(seed + 10).normal(size=(h, w, 4))
    _check(_gpu(gs, ctx, X, F, col, cam, spec, dimg), X, F, col, cam, spec, dimg)


def test_cloth_surface_parity(gs, ctx):
    # the thrown cloth mid-flight, 162 triangles seen at an angle
    from oracle import oracle as O
    p = I.cloth_throw(n=10, steps=200, seed=1)
    xS, _ = O.Model(p).rollout(p.x0, p.v0, p.dt, 200)
    cam = I.look_at((1.4, 1.1, -0.6), xS.mean(axis=0), width=72, height=56, fov_deg=45.0)
    col = I.vertex_colours(p.X, seed=3)
    spec = I.RenderSpec(sigma=0.6, gamma=5e-3)
    dimg = np.random.default_rng(4).normal(size=(56, 72, 4))
    _check(_gpu(gs, ctx, xS, p.elems, col, cam, spec, dimg), xS, p.elems, col, cam, spec, dimg)


def test_tet_surface_parity(gs, ctx):
    # surface of a 3x3x3-cell block: occlusion between front and back faces
    X, tets = I.hex_block(3, 3, 3, 0.1)
    F = I.surface_faces(tets)
    cam = I.look_at((0.9, 0.8, -0.7), (0.15, 0.15, 0.15), width=48, height=48, fov_deg=45.0)
    col = I.vertex_colours(X, seed=5)
    spec = I.RenderSpec(sigma=0.5, gamma=1e-2)
    dimg = np.random.default_rng(6).normal(size=(48, 48, 4))
    _check(_gpu(gs, ctx, X, F, col, cam, spec, dimg), X, F, col, cam, spec, dimg)


def test_edge_cases(gs, ctx):
    cam = I.look_at((0.0, 0.0, -2.0), (0.0, 0.0, 0.0), width=20, height=20, fov_deg=60.0)
    spec = I.RenderSpec(sigma=0.5, gamma=0.05, bg=(0.2, 0.3, 0.4))
    # no faces: the background, zero gradients
    X = np.zeros((3, 3))
    out = _gpu(gs, ctx, X, np.zeros((0, 3), dtype=np.int32), np.ones((3, 3)) * 0.5, cam, spec, np.ones((20, 20, 4)))
    np.testing.assert_allclose(out["img"][..., :3], np.broadcast_to([0.2, 0.3, 0.4], (20, 20, 3)), atol=1e-7)
    assert np.all(out["img"][..., 3] == 0) and np.all(out["dx"] == 0) and np.all(out["dc"] == 0)
    # one triangle behind the camera (culled) and one covering the whole image
    Xb = np.array([[0.0, 0.0, -3.0], [0.5, 0.0, -3.0], [0.0, 0.5, -3.0]])
    Xw = np.array([_world(cam, -40, -40, 2.0), _world(cam, 80, -30, 2.5), _world(cam, -10, 90, 3.0)])
    X = np.vstack([Xb, Xw])
    F = np.array([[0, 1, 2], [3, 4, 5]])
    col = np.random.default_rng(7).uniform(0.1, 0.9, (6, 3))
    dimg = np.random.default_rng(8).normal(size=(20, 20, 4))
    out = _gpu(gs, ctx, X, F, col, cam, spec, dimg)
    _check(out, X, F, col, cam, spec, dimg)
    assert np.all(out["dx"][:3] == 0)


def test_deterministic(gs, ctx):
    cam = I.look_at((0.3, 0.4, -2.5), (0.0, 0.0, 0.0), width=64, height=48)
    X, F, col = _random_scene(cam, 40, 9)
    spec = I.RenderSpec()
    dimg = np.random.default_rng(9).normal(size=(48, 64, 4))
    a = _gpu(gs, ctx, X, F, col, cam, spec, dimg)
    b = _gpu(gs, ctx, X, F, col, cam, spec, dimg)
    for k in ("img", "dx", "dc"):
        np.testing.assert_array_equal(a[k], b[k])


def test_errors(gs, ctx):
    import torch
    cam = I.look_at((0.0, 0.0, -2.0), (0.0, 0.0, 0.0), width=8, height=8)
    with pytest.raises(gs.GradsimError) as ei:
        gs.Raster(ctx, 3, np.array([[0, 1, 3]]), cam, I.RenderSpec())
    assert ei.value.status == gs.GS_EINVAL
    with pytest.raises(gs.GradsimError) as ei:
        gs.Raster(ctx, 3, np.array([[0, 1, 2]]), cam, I.RenderSpec(sigma=0.0))
    assert ei.value.status == gs.GS_EINVAL
    bad = I.look_at((0.0, 0.0, -2.0), (0.0, 0.0, 0.0), width=8, height=8)
    bad.z_near = -1.0
    with pytest.raises(gs.GradsimError) as ei:
        gs.Raster(ctx, 3, np.array([[0, 1, 2]]), bad, I.RenderSpec())
    assert ei.value.status == gs.GS_EINVAL
    r = gs.Raster(ctx, 3, np.array([[0, 1, 2]]), cam, I.RenderSpec())
    with pytest.raises(gs.GradsimError) as ei:
        r.backward(torch.zeros(8, 8, 4, device="cuda"))
    assert ei.value.status == gs.GS_ESTATE
    r.close()


def test_initial_velocity_from_rendered_frames(gs, ctx):
    # control-cloth from video: three frames of a reference throw are the
    # target; Adam on the initial velocity through render + rollout adjoints
    # (each frame's segment is recomputed in backward: the mesh keeps one
    # stored rollout)
    import torch
    from paper_2104_02646_gb300 import autograd as A
    p = I.cloth_throw(n=8, steps=300, seed=2)
    mesh = gs.Mesh(ctx, p)
    dev = "cuda"
    f32 = dict(dtype=torch.float32, device=dev)
    mu, lam, rho = (torch.tensor(a, **f32) for a in (p.mu, p.lam, p.rho))
    x0 = torch.tensor(p.x0, **f32)
    col = torch.tensor(I.vertex_colours(p.X, seed=1), **f32)
    cam = I.look_at((1.6, 1.0, -0.8), (0.45, 0.35, 0.45), width=64, height=64, fov_deg=50.0)
    raster = gs.Raster(ctx, p.n_nodes, p.elems, cam, I.RenderSpec(sigma=1.0, gamma=1e-2))
    seg = 100

    def frames(v0):
        x, v, out = x0, v0, []
        for _ in range(3):
            x, v = A.rollout(mesh, p.dt, seg, mu, lam, rho, x, v, K=1)
            out.append(A.render(raster, x, col))
        return out

    v_ref = torch.tensor(p.v0, **f32)
    with torch.no_grad():
        target = [f.clone() for f in frames(v_ref)]
    v = (v_ref + torch.tensor([0.3, -0.2, 0.25], device=dev)).requires_grad_(True)
    opt = torch.optim.Adam([v], lr=0.03)
    losses = []
    for it in range(40):
        opt.zero_grad()
        loss = sum(((f - t) ** 2).sum() for f, t in zip(frames(v), target))
        loss.backward()
        assert torch.isfinite(v.grad).all()
        opt.step()
        losses.append(float(loss.detach()))
    assert min(losses[-5:]) < 0.1 * losses[0], losses
    err0 = float(torch.tensor([0.3, -0.2, 0.25]).norm())
    err = float((v.detach() - v_ref).mean(dim=0).norm())
    assert err < 0.3 * err0, (err, err0)
    raster.close()
    mesh.close()
