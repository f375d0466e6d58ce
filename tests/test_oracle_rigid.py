"""Pins of the rigid-body oracle (App. A.1 "Rigid Bodies": Newton-Euler with
the compliant contact model at the body's points, semi-implicit Euler of
App. B).

Pinned against: the free-flight closed form of the centre of mass; the
exact discrete rotation of a body with isotropic inertia (angle
2 atan(dt |omega| / 2) per step about a fixed axis); the unit quaternion;
conservation of world angular momentum in torque-free flight as dt -> 0
(first-order convergence); the resting box's penetration m g / (4 k_e);
the Coulomb slip deceleration mu g; the box's inertia tensor against a
Monte-Carlo integral; outward surface triangles; and the adjoint against
forward-mode dual numbers and central finite differences.
"""
import math

import numpy as np

from oracle import oracle as O
from paper_2104_02646_gb300 import inputs as I


def _qrot(q, p):
    w, v = q[0], np.asarray(q[1:])
    return p + 2 * w * np.cross(v, p) + 2 * np.cross(v, np.cross(v, p))


def test_box_inertia_and_faces():
    rng = np.random.default_rng(0)
    b = I.box_body(size=(0.3, 0.2, 0.5), density=7.0)
    u = rng.uniform(-0.5, 0.5, (400000, 3)) * np.array([0.3, 0.2, 0.5])
    m = b.mass
    Ixx = m * np.mean(u[:, 1] ** 2 + u[:, 2] ** 2)
    Iyy = m * np.mean(u[:, 0] ** 2 + u[:, 2] ** 2)
    Izz = m * np.mean(u[:, 0] ** 2 + u[:, 1] ** 2)
    np.testing.assert_allclose(b.inertia[:3], [Ixx, Iyy, Izz], rtol=5e-3)
    P = b.points
    for f in b.faces:
        n = np.cross(P[f[1]] - P[f[0]], P[f[2]] - P[f[0]])
        assert np.dot(n, P[f].mean(axis=0)) > 0  # outward
    assert b.faces.shape == (12, 3)


def test_free_flight_closed_forms():
    # no ground: the centre of mass follows the semi-implicit Euler parabola;
    # with isotropic inertia omega stays constant and each step rotates by
    # 2 atan(dt |omega| / 2) about omega (the normalised first-order update)
    b = I.box_body(size=(0.2, 0.2, 0.2), v0=(1.0, 2.0, -0.5), w0=(0.3, -1.2, 2.0))
    b.scene = I.Contact(plane_on=False)
    r = O.Rigid(b)
    dt, S = 1e-3, 700
    sS = r.rollout(b.state0, dt, S)
    n = S
    g = np.array(b.gravity)
    x_ref = b.state0[:3] + n * dt * b.state0[7:10] + g * dt * dt * n * (n + 1) / 2
    np.testing.assert_allclose(sS[:3], x_ref, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(sS[7:10], b.state0[7:10] + n * dt * g, rtol=1e-12)
    w = b.state0[10:13]
    np.testing.assert_allclose(sS[10:13], w, rtol=1e-12, atol=1e-15)
    wl = np.linalg.norm(w)
    ang = n * 2 * math.atan(dt * wl / 2)
    q_ref = np.concatenate([[math.cos(ang / 2)], math.sin(ang / 2) * w / wl])
    np.testing.assert_allclose(sS[3:7], q_ref, atol=1e-12)
    assert abs(np.linalg.norm(sS[3:7]) - 1) < 1e-14


def test_torque_free_angular_momentum_converges():
    # an asymmetric body spinning freely: world angular momentum R I R^T w is
    # conserved by the exact dynamics; the step's drift shrinks with dt
    b = I.box_body(size=(0.1, 0.3, 0.6), w0=(2.0, 0.5, 0.3))
    b.scene = I.Contact(plane_on=False)
    r = O.Rigid(b)

    def Lw(s):
        q = s[3:7]
        Ib = np.diag(b.inertia[:3])
        R = np.stack([_qrot(q, e) for e in np.eye(3)], axis=1)
        return R @ Ib @ R.T @ s[10:13]

    L0 = Lw(b.state0)
    errs = []
    for dt in (2e-3, 1e-3, 5e-4):
        sS = r.rollout(b.state0, dt, int(round(0.5 / dt)))
        errs.append(np.linalg.norm(Lw(sS) - L0) / np.linalg.norm(L0))
    assert errs[0] > errs[1] > errs[2]
    assert 1.7 < errs[0] / errs[1] < 2.3 and 1.7 < errs[1] / errs[2] < 2.3  # first order
    assert errs[2] < 1e-2


def test_resting_box_penetration():
    # a 2.4 kg box settles flat on its 4 bottom corners: each carries m g / 4
    # (a mass other than 1 kg, so that the closed form tells F / m from F m)
    ke = 2.0e4
    b = I.box_body(size=(0.2, 0.2, 0.2), density=300.0, contact=(ke, 30.0, 100.0, 0.5), x0=(0.0, 0.1, 0.0))
    assert abs(b.mass - 2.4) < 1e-12
    r = O.Rigid(b)
    sS = r.rollout(b.state0, 1e-3, 3000)
    C = b.mass * 9.81 / (4 * ke)
    assert abs((0.1 - sS[1]) - C) < 1e-6 * C + 1e-9
    assert np.abs(sS[7:13]).max() < 1e-6


def test_sliding_box_decelerates_at_mu_g():
    # resting box pushed along x: all bottom corners slip, the friction force
    # is mu m g (the normal forces still sum to m g), deceleration mu g
    ke, mu = 1.0e5, 0.4
    b = I.box_body(size=(0.2, 0.2, 0.2), density=125.0, contact=(ke, 60.0, 1.0e5, mu))
    C = b.mass * 9.81 / (4 * ke)
    b.state0[1] = 0.1 - C
    b.state0[7] = 1.0
    r = O.Rigid(b)
    dt, S = 1e-4, 1000
    _, tr = r.rollout(b.state0, dt, S, traj=True)
    vx = tr[:, 7]
    decel = (vx[200] - vx[800]) / (600 * dt)
    assert abs(decel - mu * 9.81) < 0.01 * mu * 9.81, decel


def _tumbling():
    b = I.box_body(size=(0.25, 0.15, 0.2), density=90.0, contact=(3.0e3, 8.0, 200.0, 0.6), x0=(0.0, 0.16, 0.0),
                   q0=(0.95, 0.2, 0.1, -0.2), v0=(0.8, -0.5, 0.3), w0=(1.0, -2.0, 0.5), n=3)
    return b


def test_adjoint_matches_forward_mode():
    b = _tumbling()
    r = O.Rigid(b)
    dt, S = 1e-3, 250
    sS = r.rollout(b.state0, dt, S)
    rng = np.random.default_rng(1)
    target = np.array([sS[:3] + _qrot(sS[3:7], p) for p in b.points]) + rng.normal(0, 1e-2, b.points.shape)
    seed = rng.normal(size=13)
    L, g = r.loss_grad(b.state0, dt, S, target, seed)
    for _ in range(3):
        ds, dm = rng.normal(size=13), rng.normal()
        di, dc = rng.normal(size=6) * 1e-3, rng.normal(size=4) * np.array(b.contact) * 1e-2
        L2, dL = r.loss_dir(b.state0, dt, S, target, seed, ds, dm, di, dc)
        assert abs(L2 - L) <= 1e-13 * abs(L)
        ref = g["state0"] @ ds + g["mass"] * dm + g["inertia"] @ di + g["contact"] @ dc
        assert abs(dL - ref) <= 1e-9 * max(abs(dL), 1e-30), (dL, ref)


def test_adjoint_matches_finite_differences():
    b = _tumbling()
    r = O.Rigid(b)
    dt, S = 1e-3, 120
    rng = np.random.default_rng(2)
    target = b.points + np.array([0.1, 0.12, 0.0]) + rng.normal(0, 1e-2, b.points.shape)
    L, g = r.loss_grad(b.state0, dt, S, target)

    def fd(fn, h):
        return (fn(h) - fn(-h)) / (2 * h)

    for i in (0, 1, 4, 8, 11):
        def f(h, i=i):
            s = b.state0.copy()
            s[i] += h
            return r.loss_grad(s, dt, S, target)[0]
        best = min(abs(fd(f, h) - g["state0"][i]) / max(abs(fd(f, h)), 1e-12) for h in (1e-5, 1e-6, 1e-7))
        assert best <= 1e-6, (i, best)

    def fm(h):
        return O.Rigid(b, mass=b.mass + h).loss_grad(b.state0, dt, S, target)[0]
    best = min(abs(fd(fm, h) - g["mass"]) / abs(fd(fm, h)) for h in (1e-5, 1e-6, 1e-7))
    assert best <= 1e-6, best
    for j in range(4):
        def fc(h, j=j):
            c = list(b.contact)
            c[j] += h * max(abs(c[j]), 1.0)
            return O.Rigid(b, contact=c).loss_grad(b.state0, dt, S, target)[0] / max(abs(b.contact[j]), 1.0)
        best = min(abs(fd(fc, h) - g["contact"][j]) / max(abs(fd(fc, h)), 1e-12) for h in (1e-5, 1e-6, 1e-7))
        assert best <= 1e-5, (j, best)
