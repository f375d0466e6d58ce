"""Pins of the oracle's air model on cloth (App. A.1 "Deformable Thin-Shells"
adds lift and drag from the air around the cloth; no formula is printed, the
flat-plate reading is stated in the oracle).

Pinned against physics and invariants rather than the formula itself:
terminal velocity of a falling plate (drag balancing gravity, a closed form),
zero force edge-on, independence of the winding, the lift doing no work and
the drag only removing energy, the angle laws of a flat plate (projected-area
drag, sin 2 theta lift), frame covariance and Galilean invariance with the
wind; and the adjoint with air against forward-mode dual numbers and central
finite differences.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2104_02646_gb300 import inputs as I


def _rot(rng):
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    return q * np.sign(np.linalg.det(q))


def _plate(phi, size=0.3):
    """Triangle in the plane through the origin whose normal is
    (sin phi, cos phi, 0): the x-z plane rotated about z by -phi."""
    c, s = math.cos(phi), math.sin(phi)
    t1 = np.array([c, -s, 0.0])   # in-plane, perpendicular to z
    t2 = np.array([0.0, 0.0, 1.0])
    x = np.stack([np.zeros(3), size * t1, size * t2])
    n = np.cross(t1, t2)
    # winding (x1 - x0) x (x2 - x0) is along t1 x t2
    return x, n / np.linalg.norm(n)


def test_falling_plate_reaches_the_drag_terminal_speed():
    # one horizontal triangle (rigid translation: no membrane force) falling
    # from rest: the discrete step's fixed point is where k_D A s^2 = rho_A A g,
    # s* = sqrt(rho_A g / k_D), whatever the area; no lift at normal incidence
    X = np.array([[0.0, 1.0, 0.0], [0.2, 1.0, 0.0], [0.0, 1.0, 0.15]])
    air = I.Air(k_drag=0.6, k_lift=0.4)
    con = I.Contact(plane_on=False)
    m = O.Model(X=X, tris=np.array([[0, 1, 2]]), tri_mu=[10.0], tri_lam=[20.0], tri_rho=[0.2],
                contact=con, air=air)
    _, v = m.rollout(X, np.zeros_like(X), 1e-3, 3000)
    s_star = math.sqrt(0.2 * 9.81 / 0.6)
    np.testing.assert_allclose(v[:, 1], -s_star, rtol=1e-9)
    assert np.abs(v[:, [0, 2]]).max() <= 1e-12  # membrane rounding at rest only
    # without air it would be in free fall at g t
    m0 = O.Model(X=X, tris=np.array([[0, 1, 2]]), tri_mu=[10.0], tri_lam=[20.0], tri_rho=[0.2], contact=con)
    _, v0 = m0.rollout(X, np.zeros_like(X), 1e-3, 3000)
    np.testing.assert_allclose(v0[:, 1], -9.81 * 3.0, rtol=1e-12)


def test_edge_on_motion_and_winding():
    rng = np.random.default_rng(1)
    for _ in range(20):
        x = rng.normal(size=(3, 3))
        t1, t2 = x[1] - x[0], x[2] - x[0]
        v_in_plane = rng.normal() * t1 + rng.normal() * t2
        f = O.air_forces(x, np.tile(v_in_plane, (3, 1)), 0.7, 0.5)
        assert np.abs(f).max() <= 1e-14 * np.abs(v_in_plane).max() ** 2 * np.linalg.norm(np.cross(t1, t2))
        v = rng.normal(size=(3, 3))
        fa = O.air_forces(x, v, 0.7, 0.5, wind=(0.3, -0.1, 0.2))
        fb = O.air_forces(x[[0, 2, 1]], v[[0, 2, 1]], 0.7, 0.5, wind=(0.3, -0.1, 0.2))
        np.testing.assert_allclose(fb[[0, 2, 1]], fa, rtol=1e-13, atol=1e-15)
        # each corner carries a third of the total
        np.testing.assert_allclose(fa[0], fa[1], rtol=1e-15)
        np.testing.assert_allclose(fa[0], fa[2], rtol=1e-15)


def test_lift_does_no_work_and_drag_dissipates():
    rng = np.random.default_rng(2)
    for _ in range(50):
        x = rng.normal(size=(3, 3))
        v = rng.normal(size=(3, 3))
        vbar = v.mean(axis=0)
        lift = O.air_forces(x, v, 0.0, 0.8).sum(axis=0)
        drag = O.air_forces(x, v, 0.8, 0.0).sum(axis=0)
        both = O.air_forces(x, v, 0.8, 0.8).sum(axis=0)
        np.testing.assert_allclose(both, lift + drag, rtol=1e-13, atol=1e-15)
        assert abs(np.dot(lift, vbar)) <= 1e-13 * np.linalg.norm(lift) * np.linalg.norm(vbar)
        # power into the cloth: sum_i f_i . v_i = F . vbar
        P = sum(np.dot(fi, vi) for fi, vi in zip(O.air_forces(x, v, 0.8, 0.8), v))
        assert P <= 1e-15
        assert np.dot(drag, vbar) < 0.0
        # drag is antiparallel to the velocity
        np.testing.assert_allclose(np.cross(drag, vbar), 0.0, atol=1e-13 * np.linalg.norm(drag) * np.linalg.norm(vbar))


def test_flat_plate_angle_laws():
    # a plate moving along +x at speed U with its normal at angle theta to the
    # flow: drag = k_D A U^2 |cos theta| along -x, lift = k_L A U^2 |sin 2 theta| / 2
    # perpendicular to the flow
    U, kD, kL = 2.0, 0.6, 0.4
    for phi in np.linspace(0.05, 1.5, 12):
        x, n = _plate(phi)
        A = 0.5 * np.linalg.norm(np.cross(x[1] - x[0], x[2] - x[0]))
        v = np.tile([U, 0.0, 0.0], (3, 1))
        F = O.air_forces(x, v, kD, kL).sum(axis=0)
        cos_t = n[0]  # n . x_hat
        drag = -F[0]
        lift_vec = F - F[0] * np.array([1.0, 0.0, 0.0])
        np.testing.assert_allclose(drag, kD * A * U * U * abs(cos_t), rtol=1e-12)
        np.testing.assert_allclose(np.linalg.norm(lift_vec), kL * A * U * U * abs(math.sin(2 * math.acos(cos_t))) / 2,
                                   rtol=1e-12)
        # the lift pushes the plate away from the side the flow comes from
        # (towards -n when the plate advances along +n)
        assert np.dot(lift_vec, n) * cos_t <= 0.0


def test_frame_covariance_and_galilean_invariance():
    rng = np.random.default_rng(3)
    for _ in range(20):
        x = rng.normal(size=(3, 3))
        v = rng.normal(size=(3, 3))
        w = rng.normal(size=3)
        f = O.air_forces(x, v, 0.6, 0.4, wind=w)
        R = _rot(rng)
        fr = O.air_forces(x @ R.T + rng.normal(size=3), v @ R.T, 0.6, 0.4, wind=R @ w)
        np.testing.assert_allclose(fr, f @ R.T, rtol=1e-11, atol=1e-13)
        u = rng.normal(size=3)
        fg = O.air_forces(x, v + u, 0.6, 0.4, wind=w + u)
        np.testing.assert_allclose(fg, f, rtol=1e-11, atol=1e-13)


def _throw(n=6, steps=60, seed=4):
    p = I.cloth_throw(n=n, steps=steps, seed=seed)
    m = O.Model(p)
    xS, _ = m.rollout(p.x0, p.v0, p.dt, steps)
    tgt = xS + I.position_noise(p.n_nodes, sigma=1e-3, seed=7)
    return p, m, tgt


def test_air_adjoint_matches_forward_mode():
    S = 60
    p, m, tgt = _throw(steps=S)
    # the reference rollout with slightly different initial velocity
    L, g = m.loss_grad(p.x0, p.v0 * 1.05, p.dt, S, tgt)
    rng = np.random.default_rng(5)
    for key, shape in (("v0", p.v0.shape), ("x0", p.x0.shape), ("tri_mu", (p.n_elems,)), ("hinge_kb", (p.n_hinges,))):
        d = rng.normal(size=shape)
        if key == "x0":
            d *= 1e-3
        L2, dL = m.loss_dir(p.x0, p.v0 * 1.05, p.dt, S, tgt, {key: d})
        assert abs(L2 - L) <= 1e-13 * abs(L)
        ref = float(np.sum(g[key] * d))
        assert abs(dL - ref) <= 1e-9 * max(abs(dL), 1e-30), (key, dL, ref)


def test_air_changes_the_gradient():
    # the air terms reach the adjoint: without them dL/dv0 differs
    S = 60
    p, m, tgt = _throw(steps=S)
    _, g = m.loss_grad(p.x0, p.v0 * 1.05, p.dt, S, tgt)
    q = I.Problem(**{f: getattr(p, f) for f in p.__dataclass_fields__})
    q.air = None
    _, g0 = O.Model(q).loss_grad(p.x0, p.v0 * 1.05, p.dt, S, tgt)
    assert np.linalg.norm(g["v0"] - g0["v0"]) > 1e-3 * np.linalg.norm(g["v0"])


def test_air_adjoint_matches_finite_differences():
    # two triangles with wind, no contact; initial velocities one at a time
    X = np.array([[0.0, 0.5, 0.0], [0.1, 0.5, 0.0], [0.0, 0.52, 0.1], [0.1, 0.55, 0.1]])
    tris = np.array([[0, 1, 2], [1, 3, 2]])
    kw = dict(X=X, tris=tris, tri_mu=[5.0, 5.0], tri_lam=[8.0, 8.0], tri_rho=[0.2, 0.2],
              contact=I.Contact(plane_on=False), air=I.Air(0.6, 0.4, wind=(0.5, 0.0, -0.3)))
    rng = np.random.default_rng(6)
    v0 = rng.normal(0.0, 0.5, X.shape)
    S, dt = 40, 2e-3
    tgt = X + rng.normal(0.0, 1e-2, X.shape)
    m = O.Model(**kw)
    _, g = m.loss_grad(X, v0, dt, S, tgt)
    for (i, k) in [(0, 0), (1, 1), (2, 2), (3, 1)]:
        best = np.inf
        for h in (1e-4, 1e-5, 1e-6):
            vp, vm = v0.copy(), v0.copy()
            vp[i, k] += h
            vm[i, k] -= h
            Lp, _ = m.loss_grad(X, vp, dt, S, tgt)
            Lm, _ = m.loss_grad(X, vm, dt, S, tgt)
            fd = (Lp - Lm) / (2 * h)
            best = min(best, abs(fd - g["v0"][i, k]) / max(abs(fd), 1e-300))
        assert best <= 1e-7, (i, k, best)
    for (i, k) in [(0, 1), (3, 0)]:
        best = np.inf
        for h in (1e-5, 1e-6, 1e-7):
            xp, xm = X.copy(), X.copy()
            xp[i, k] += h
            xm[i, k] -= h
            Lp, _ = m.loss_grad(xp, v0, dt, S, tgt)
            Lm, _ = m.loss_grad(xm, v0, dt, S, tgt)
            fd = (Lp - Lm) / (2 * h)
            best = min(best, abs(fd - g["x0"][i, k]) / max(abs(fd), 1e-300))
        assert best <= 1e-6, (i, k, best)
