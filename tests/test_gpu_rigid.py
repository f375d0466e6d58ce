"""Rigid bodies (App. A.1 "Rigid Bodies") on the CUDA path against the FP64
oracle, and the paper's rigid experiment: a body's mass recovered from
rendered frames after a known impulse, with the loss landscape over mass
(Sec. 3 "Loss landscapes": a unit-mass cube, initial guesses 0.1-5 kg).

Tolerances: states rel <= 1e-3 with contact, gradients rel-L2 <= 1e-3 and
cosine >= 0.9999 per body.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2104_02646_gb300 import inputs as I

from gpu_util import GRAD_COS, GRAD_REL, cosine, quat_tangent, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(gs):
    return gs.Context(0)


def _gpu(gs, ctx, bodies, S, dt, seed):
    import torch
    r = gs.Rigid(ctx, bodies)
    s0 = torch.tensor(r.state0(), device="cuda")
    sS = torch.empty_like(s0)
    r.rollout(dt, S, s0, sS)
    B = len(bodies)
    g = {"d_state0": torch.zeros(B, 13, device="cuda"),
         "d_mass": torch.zeros(B, dtype=torch.float64, device="cuda"),
         "d_inertia": torch.zeros(B, 6, dtype=torch.float64, device="cuda"),
         "d_contact": torch.zeros(B, 4, dtype=torch.float64, device="cuda")}
    r.adjoint(g, seed=torch.tensor(seed, dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    out = {k: v.cpu().numpy().astype(np.float64) for k, v in g.items()}
    out["sS"] = sS.cpu().numpy().astype(np.float64)
    out["status"] = r.check_finite()
    r.close()
    return out


def _check_body(out, b, body, S, dt, seed):
    ro = O.Rigid(body)
    sS = ro.rollout(body.state0, dt, S)
    np.testing.assert_allclose(out["sS"][b, :3], sS[:3], atol=1e-3 * (1 + np.abs(sS[:3]).max()))
    np.testing.assert_allclose(out["sS"][b, 3:7], sS[3:7], atol=1e-3)
    _, g = ro.loss_grad(body.state0, dt, S, None, seed[b])
    # dL/dr0 compared on the unit quaternion's tangent space
    q0 = body.state0[3:7]
    pairs = [(quat_tangent(out["d_state0"][b], q0), quat_tangent(g["state0"], q0)), (out["d_inertia"][b], g["inertia"]),
             (out["d_contact"][b], g["contact"])]
    for a, ref in pairs:
        assert np.all(np.isfinite(a))
        if np.linalg.norm(ref) == 0:
            assert np.linalg.norm(a) == 0
            continue
        assert rel(a, ref) <= GRAD_REL, (rel(a, ref), a, ref)
        assert cosine(a, ref) >= GRAD_COS
    assert abs(out["d_mass"][b] - g["mass"]) <= GRAD_REL * abs(g["mass"]) + 1e-12


def _tumbling(n=3):
    return I.box_body(size=(0.25, 0.15, 0.2), density=90.0, contact=(3.0e3, 8.0, 200.0, 0.6), x0=(0.0, 0.16, 0.0),
                      q0=(0.95, 0.2, 0.1, -0.2), v0=(0.8, -0.5, 0.3), w0=(1.0, -2.0, 0.5), n=n)


def test_tumbling_box_parity(gs, ctx):
    S, dt = 250, 1e-3
    body = _tumbling()
    seed = np.random.default_rng(0).normal(size=(1, 13))
    out = _gpu(gs, ctx, [body], S, dt, seed)
    assert out["status"] == gs.GS_OK
    _check_body(out, 0, body, S, dt, seed)


def test_batch_parity_and_batch_invariance(gs, ctx):
    # 64 seeded boxes (98 surface points each): parity on a sample, and each
    # body bitwise the same alone and in the batch
    S, dt = 200, 1e-3
    bodies = I.rigid_batch(64, seed=3, n=5, steps=S)
    for body in bodies:  # lowest point 5 cm above the ground: contact within the horizon
        q = body.state0[3:7]
        w, v = q[0], q[1:]
        low = min((p + 2 * w * np.cross(v, p) + 2 * np.cross(v, np.cross(v, p)))[1] for p in body.points)
        body.state0[1] = 0.05 - low
        body.state0[8] = -abs(body.state0[8])
    seed = np.random.default_rng(1).normal(size=(64, 13))
    out = _gpu(gs, ctx, bodies, S, dt, seed)
    for b in (0, 17, 40, 63):
        _check_body(out, b, bodies[b], S, dt, seed)
    alone = _gpu(gs, ctx, [bodies[17]], S, dt, seed[17:18])
    for k in ("sS", "d_state0", "d_mass", "d_inertia", "d_contact"):
        np.testing.assert_array_equal(alone[k][0], out[k][17])


def test_sphere_contact_parity(gs, ctx):
    S, dt = 300, 1e-3
    body = I.box_body(size=(0.2, 0.2, 0.2), density=60.0, contact=(2.0e3, 5.0, 100.0, 0.4), x0=(0.05, 0.45, 0.02),
                      q0=(0.9, 0.3, 0.0, 0.3), n=3)
    body.scene = I.Contact(plane_on=True, sphere_on=True, sphere_c=(0.0, 0.0, 0.0), sphere_r=0.3)
    seed = np.random.default_rng(2).normal(size=(1, 13))
    out = _gpu(gs, ctx, [body], S, dt, seed)
    _check_body(out, 0, body, S, dt, seed)


def test_points_and_their_adjoint(gs, ctx):
    import torch
    bodies = [_tumbling(), I.box_body(size=(0.3, 0.1, 0.2), q0=(0.7, 0.1, 0.6, 0.3), n=2)]
    r = gs.Rigid(ctx, bodies)
    s = torch.tensor(r.state0(), device="cuda")
    X = torch.empty(r.n_points, 3, device="cuda")
    r.points(s, X)
    ref = []
    for body in bodies:
        q = body.state0[3:7]
        w, v = q[0], q[1:]
        for p in body.points:
            ref.append(body.state0[:3] + p + 2 * w * np.cross(v, p) + 2 * np.cross(v, np.cross(v, p)))
    np.testing.assert_allclose(X.cpu().numpy(), np.array(ref), atol=1e-6)
    # adjoint against the oracle's point loss with zero-step rollouts
    rng = np.random.default_rng(4)
    tgt = np.array(ref) + rng.normal(0, 0.01, (r.n_points, 3))
    gX = 2 * (torch.tensor(np.array(ref), dtype=torch.float32, device="cuda") - torch.tensor(tgt, dtype=torch.float32,
                                                                                            device="cuda"))
    ds = torch.empty_like(s)
    r.points_backward(s, gX.contiguous(), ds)
    off = 0
    for b, body in enumerate(bodies):
        n = len(body.points)
        _, g = O.Rigid(body).loss_grad(body.state0, 1e-3, 0, tgt[off:off + n])
        np.testing.assert_allclose(ds[b].cpu().numpy(), g["state0"], rtol=1e-4, atol=1e-5)
        off += n
    r.close()


def test_errors(gs, ctx):
    import torch
    good = I.box_body()
    for change in ({"mass": -1.0}, {"inertia": (1.0, 1.0, -1.0, 0.0, 0.0, 0.0)},
                   {"contact": (1.0, -2.0, 1.0, 0.5)}):
        import dataclasses
        bad = dataclasses.replace(good, **change)
        with pytest.raises(gs.GradsimError) as ei:
            gs.Rigid(ctx, [bad])
        assert ei.value.status == gs.GS_EINVAL
    r = gs.Rigid(ctx, [good])
    with pytest.raises(gs.GradsimError) as ei:
        r.adjoint({"d_mass": torch.zeros(1, dtype=torch.float64, device="cuda")})
    assert ei.value.status == gs.GS_ESTATE
    r.close()


def _cube_video(gs, ctx, n_frames=6, seg=50):
    """A 1 kg cube given a known impulse, filmed every `seg` steps."""
    import torch
    from paper_2104_02646_gb300 import autograd as A
    body = I.box_body(size=(0.2, 0.2, 0.2), density=125.0, contact=(2.0e4, 40.0, 200.0, 0.5), x0=(0.0, 0.15, 0.0),
                      n=2, steps=n_frames * seg)
    J = torch.tensor([1.2, 2.0, 0.3], device="cuda")  # impulse, N s
    rig = gs.Rigid(ctx, [body])
    cam = I.look_at((0.5, 0.6, -2.2), (0.35, 0.45, 0.0), width=96, height=96, fov_deg=60.0)
    raster = gs.Raster(ctx, 8, body.faces, cam, I.RenderSpec(sigma=1.0, gamma=1e-2))
    col = torch.tensor(I.vertex_colours(body.points, seed=2), dtype=torch.float32, device="cuda")
    s0 = torch.tensor(body.state0, dtype=torch.float32, device="cuda")
    inertia_unit = torch.tensor(body.inertia, dtype=torch.float64, device="cuda") / body.mass
    contact = torch.tensor(body.contact, dtype=torch.float64, device="cuda").reshape(1, 4)

    def frames(mass):
        m = mass.reshape(1)
        I6 = (inertia_unit * m).reshape(1, 6)
        state = torch.cat([s0[:7], J / m.to(torch.float32), s0[10:]]).reshape(1, 13)
        out = []
        for _ in range(n_frames):
            state = A.rigid_rollout(rig, 1e-3, seg, state, m, I6, contact)
            out.append(A.render(raster, A.rigid_points(rig, state), col))
        return out

    return frames


def test_mass_loss_landscape_and_recovery(gs, ctx):
    # Sec. 3 "Loss landscapes": image MSE over frames of a unit-mass cube
    # after a known impulse, as a function of the guessed mass
    import torch
    frames = _cube_video(gs, ctx)
    with torch.no_grad():
        target = [f.clone() for f in frames(torch.tensor(1.0, dtype=torch.float64, device="cuda"))]

    def loss(mass):
        return sum(((f - t) ** 2).mean() for f, t in zip(frames(mass), target))

    grid = [0.5, 0.6, 0.75, 0.9, 1.0, 1.15, 1.4, 2.0, 3.0, 5.0]
    with torch.no_grad():
        L = [float(loss(torch.tensor(m, dtype=torch.float64, device="cuda"))) for m in grid]
    i1 = grid.index(1.0)
    assert L[i1] < 1e-10
    assert all(L[i] > L[i + 1] for i in range(i1)), L       # decreasing towards 1 kg
    assert all(L[i] < L[i + 1] for i in range(i1, len(L) - 1)), L  # increasing past it
    # gradient descent from a 2.5 kg guess
    m = torch.tensor(2.5, dtype=torch.float64, device="cuda", requires_grad=True)
    opt = torch.optim.Adam([m], lr=0.1)
    for _ in range(60):
        opt.zero_grad()
        l = loss(m)
        l.backward()
        opt.step()
        with torch.no_grad():
            m.clamp_(0.3, 10.0)
    assert abs(float(m.detach()) - 1.0) < 0.05, float(m.detach())
