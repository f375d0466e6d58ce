"""Pins of the FP64 oracle to the paper and to mathematics (CPU only).

The paper prints no worked numerical example (its only numbers are the
Table 4 timings), so the oracle is pinned by closed forms, invariants,
library routines, central finite differences and forward-mode derivatives,
chosen so that a dropped term, a flipped sign, a wrong index or a transposed
operand anywhere in it breaks at least one test.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2104_02646_gb300 import inputs as I


def rand_rot(rng):
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def rand_tet(rng, h=0.025):
    while True:
        X = rng.normal(size=(4, 3)) * h
        if np.linalg.det((X[1:] - X[0]).T) > 0.3 * h ** 3:
            return X


def rand_tri(rng, h=0.02):
    while True:
        X = rng.normal(size=(3, 3)) * h
        if np.linalg.norm(np.cross(X[1] - X[0], X[2] - X[0])) > 0.3 * h * h:
            return X


MU, LAM = 3.8e4, 5.7e4


# ---------------------------------------------------------------------------
# tetrahedra (App. A.1 / C.1: stable neo-Hookean, U = sum V_e Psi_e, f = -grad U)
# ---------------------------------------------------------------------------

def test_tet_rest_matches_linear_algebra():
    rng = np.random.default_rng(0)
    for _ in range(20):
        X = rand_tet(rng)
        Dminv, V = O.tet_rest(X)
        Dm = (X[1:] - X[0]).T
        np.testing.assert_allclose(Dminv, np.linalg.inv(Dm), rtol=1e-12, atol=1e-9)
        assert V == pytest.approx(np.linalg.det(Dm) / 6.0, rel=1e-12)


def test_tet_zero_force_at_rest_any_rigid_motion():
    rng = np.random.default_rng(1)
    for _ in range(20):
        X = rand_tet(rng)
        Dminv, V = O.tet_rest(X)
        mu, lam = np.exp(rng.uniform(np.log(1e3), np.log(1e6), 2))
        scale = mu * V / 0.025
        f = O.tet_forces(X, Dminv, V, mu, lam)
        assert np.abs(f).max() <= 1e-12 * scale
        R = rand_rot(rng)
        f = O.tet_forces(X @ R.T + rng.normal(size=3), Dminv, V, mu, lam)
        assert np.abs(f).max() <= 1e-11 * scale


@pytest.mark.parametrize("s", [0.7, 0.95, 1.0, 1.1, 1.6])
def test_tet_uniform_stretch_closed_form(s):
    # F = s I  =>  I_C = 3 s^2, J = s^3, cof F = s^2 I,
    # P = [mu s (1 - 1/(3 s^2 + 1)) + lambda (s^3 - alpha) s^2] I, alpha = 1 + 3mu/(4lambda)
    rng = np.random.default_rng(2)
    X = rand_tet(rng)
    Dminv, V = O.tet_rest(X)
    Dm = (X[1:] - X[0]).T
    alpha = 1.0 + 0.75 * MU / LAM
    p = MU * s * (1.0 - 1.0 / (3.0 * s * s + 1.0)) + LAM * (s ** 3 - alpha) * s * s
    H = -V * p * np.linalg.inv(Dm).T
    want = np.vstack([-H.sum(axis=1), H.T])
    got = O.tet_forces(s * X, Dminv, V, MU, LAM)
    np.testing.assert_allclose(got, want, rtol=1e-11, atol=1e-12 * max(np.abs(want).max(), MU * V / 0.025))


def test_tet_actuation_closed_form_at_rest():
    # at F = I with actuation a: P = 3mu/4 I + lambda (1 - alpha) I = -lambda a I
    rng = np.random.default_rng(3)
    X = rand_tet(rng)
    Dminv, V = O.tet_rest(X)
    a = 0.05
    H = -V * (-LAM * a) * np.linalg.inv((X[1:] - X[0]).T).T
    want = np.vstack([-H.sum(axis=1), H.T])
    np.testing.assert_allclose(O.tet_forces(X, Dminv, V, MU, LAM, a), want, rtol=1e-10,
                               atol=1e-12 * np.abs(want).max())


def test_tet_frame_indifference():
    rng = np.random.default_rng(4)
    for _ in range(10):
        X = rand_tet(rng)
        Dminv, V = O.tet_rest(X)
        x = X + rng.normal(size=X.shape) * 0.004
        R = rand_rot(rng)
        e0 = O.tet_energy(x, Dminv, V, MU, LAM)
        e1 = O.tet_energy(x @ R.T + 0.3, Dminv, V, MU, LAM)
        assert e1 == pytest.approx(e0, rel=1e-10)
        f0 = O.tet_forces(x, Dminv, V, MU, LAM)
        f1 = O.tet_forces(x @ R.T + 0.3, Dminv, V, MU, LAM)
        np.testing.assert_allclose(f1, f0 @ R.T, rtol=1e-9, atol=1e-10 * np.abs(f0).max())


def test_tet_momentum_and_torque():
    rng = np.random.default_rng(5)
    for _ in range(10):
        X = rand_tet(rng)
        Dminv, V = O.tet_rest(X)
        x = X + rng.normal(size=X.shape) * 0.005
        f = O.tet_forces(x, Dminv, V, MU, LAM)
        sc = np.abs(f).max()
        assert np.abs(f.sum(axis=0)).max() <= 1e-12 * sc
        assert np.abs(np.cross(x, f).sum(axis=0)).max() <= 1e-12 * sc * 0.1


def test_tet_force_is_minus_energy_gradient():
    rng = np.random.default_rng(6)
    for inverted in (False, True):
        X = rand_tet(rng)
        Dminv, V = O.tet_rest(X)
        x = X + rng.normal(size=X.shape) * 0.005
        if inverted:  # push node 0 through the opposite face: J < 0 stays finite (stable NH)
            c = X[1:].mean(axis=0)
            x[0] = c + 0.5 * (c - X[0])
        f = O.tet_forces(x, Dminv, V, MU, LAM, 0.02)
        assert np.all(np.isfinite(f))
        g = np.zeros(12)
        h = 1e-7 * 0.025
        for k in range(12):
            xp = x.reshape(12).copy(); xp[k] += h
            xm = x.reshape(12).copy(); xm[k] -= h
            g[k] = (O.tet_energy(xp, Dminv, V, MU, LAM, 0.02) - O.tet_energy(xm, Dminv, V, MU, LAM, 0.02)) / (2 * h)
        np.testing.assert_allclose(f.reshape(12), -g, rtol=1e-6, atol=1e-7 * np.abs(g).max())


def test_tet_energy_at_rest_is_the_constant_of_the_formula():
    # Psi(I) = 0 + lambda/2 (1 - alpha)^2 - mu/2 log 4  (App. A.1 energy at F = I)
    rng = np.random.default_rng(7)
    X = rand_tet(rng)
    Dminv, V = O.tet_rest(X)
    alpha = 1.0 + 0.75 * MU / LAM
    want = V * (0.5 * LAM * (1.0 - alpha) ** 2 - 0.5 * MU * math.log(4.0))
    assert O.tet_energy(X, Dminv, V, MU, LAM) == pytest.approx(want, rel=1e-12)


# ---------------------------------------------------------------------------
# membrane triangles
# ---------------------------------------------------------------------------

def test_tri_rest_frame_and_area():
    rng = np.random.default_rng(10)
    for _ in range(10):
        X = rand_tri(rng)
        Dminv, A = O.tri_rest(X)
        assert A == pytest.approx(0.5 * np.linalg.norm(np.cross(X[1] - X[0], X[2] - X[0])), rel=1e-12)
        F = (X[1:] - X[0]).T @ Dminv  # rest F has orthonormal columns
        np.testing.assert_allclose(F.T @ F, np.eye(2), atol=1e-12)


def test_tri_zero_force_at_rest_any_rigid_motion():
    rng = np.random.default_rng(11)
    for _ in range(10):
        X = rand_tri(rng)
        Dminv, A = O.tri_rest(X)
        sc = MU * 0.02
        assert np.abs(O.tri_forces(X, Dminv, A, MU, LAM)).max() <= 1e-12 * sc
        R = rand_rot(rng)
        assert np.abs(O.tri_forces(X @ R.T - 0.2, Dminv, A, MU, LAM)).max() <= 1e-11 * sc


@pytest.mark.parametrize("s", [0.8, 1.0, 1.3])
def test_tri_uniform_stretch_closed_form(s):
    # F = s Q (orthonormal columns): I_C = 2 s^2, J = s^2, dJ/dF = s Q,
    # P = [mu s (1 - 1/(2 s^2 + 1)) + lambda (s^2 - alpha) s] Q, alpha = 1 + 2mu/(3lambda)
    rng = np.random.default_rng(12)
    X = rand_tri(rng)
    Dminv, A = O.tri_rest(X)
    Q = (X[1:] - X[0]).T @ Dminv
    alpha = 1.0 + 2.0 * MU / (3.0 * LAM)
    p = MU * s * (1.0 - 1.0 / (2.0 * s * s + 1.0)) + LAM * (s * s - alpha) * s
    H = -A * p * Q @ Dminv.T
    want = np.vstack([-H.sum(axis=1), H.T])
    got = O.tri_forces(s * X, Dminv, A, MU, LAM)
    np.testing.assert_allclose(got, want, rtol=1e-10, atol=1e-12 * max(np.abs(want).max(), MU * 0.02))


def test_tri_force_is_minus_energy_gradient_and_balanced():
    rng = np.random.default_rng(13)
    for _ in range(5):
        X = rand_tri(rng)
        Dminv, A = O.tri_rest(X)
        x = X + rng.normal(size=X.shape) * 0.003
        f = O.tri_forces(x, Dminv, A, MU, LAM, -0.01)
        g = np.zeros(9)
        h = 1e-7 * 0.02
        for k in range(9):
            xp = x.reshape(9).copy(); xp[k] += h
            xm = x.reshape(9).copy(); xm[k] -= h
            g[k] = (O.tri_energy(xp, Dminv, A, MU, LAM, -0.01) - O.tri_energy(xm, Dminv, A, MU, LAM, -0.01)) / (2 * h)
        np.testing.assert_allclose(f.reshape(9), -g, rtol=1e-6, atol=1e-7 * np.abs(g).max())
        sc = np.abs(f).max()
        assert np.abs(f.sum(axis=0)).max() <= 1e-12 * sc
        assert np.abs(np.cross(x, f).sum(axis=0)).max() <= 1e-12 * sc


# ---------------------------------------------------------------------------
# dihedral bending (App. A.1, Bridson et al. force)
# ---------------------------------------------------------------------------

def make_hinge(theta, rng=None):
    """Edge x3=(0,0,0) -> x4=(0,0,L); wing x1 along +x, wing x2 along -x rotated
    by theta about the edge (flat at theta = 0)."""
    L = 0.02
    x3 = np.array([0.0, 0.0, 0.0])
    x4 = np.array([0.0, 0.0, L])
    x1 = np.array([0.013, 0.0, 0.4 * L])
    w = 0.017
    x2 = np.array([-w * math.cos(theta), w * math.sin(theta), 0.7 * L])
    x = np.array([x1, x2, x3, x4])
    if rng is not None:
        x = x @ rand_rot(rng).T + rng.normal(size=3)
    return x


def test_hinge_angle_matches_construction():
    # atan2 angle of the oracle equals the construction angle (sign by the
    # orientation of the edge): wing x2 turned by theta about the +z edge.
    rng = np.random.default_rng(20)
    for theta in (-1.2, -0.3, 0.0, 0.25, 1.0, 2.5):
        phi = O.hinge_angle(make_hinge(theta, rng))
        assert abs(abs(phi) - abs(theta)) < 1e-12
        if theta != 0.0:
            assert np.sign(phi) == np.sign(O.hinge_angle(make_hinge(abs(theta)))) * np.sign(theta)


def test_hinge_force_zero_when_flat():
    rng = np.random.default_rng(21)
    f = O.hinge_forces(make_hinge(0.0, rng), 1e-2)
    assert np.abs(f).max() < 1e-15


def test_bridson_directions_are_minus_angle_gradient():
    # f_i = s u_i with s = k_b |E|^2/(|N1|+|N2|) sin(phi/2); u_i = -dphi/dx_i,
    # checked against a central finite difference of the atan2 angle and
    # against the oracle's forward-mode derivative of that angle.
    rng = np.random.default_rng(22)
    for theta in (0.3, -0.8, 1.7):
        x = make_hinge(theta, rng)
        x1, x2, x3, x4 = x
        E = x4 - x3
        N1 = np.cross(x1 - x3, x1 - x4)
        N2 = np.cross(x2 - x4, x2 - x3)
        phi = O.hinge_angle(x)
        s = 1.0 * E.dot(E) / (np.linalg.norm(N1) + np.linalg.norm(N2)) * math.sin(phi / 2)
        u = O.hinge_forces(x, 1.0) / s
        g = np.zeros(12)
        h = 1e-8
        for k in range(12):
            xp = x.reshape(12).copy(); xp[k] += h
            xm = x.reshape(12).copy(); xm[k] -= h
            g[k] = (O.hinge_angle(xp) - O.hinge_angle(xm)) / (2 * h)
        np.testing.assert_allclose(u.reshape(12), -g, rtol=1e-6, atol=1e-6 * np.abs(g).max())
        np.testing.assert_allclose(O.hinge_angle_grad(x).reshape(12), g, rtol=1e-6, atol=1e-6 * np.abs(g).max())


def test_hinge_momentum_torque_and_restoring():
    rng = np.random.default_rng(23)
    for theta in (0.4, -0.9):
        x = make_hinge(theta, rng)
        f = O.hinge_forces(x, 3e-3)
        sc = np.abs(f).max()
        assert np.abs(f.sum(axis=0)).max() <= 1e-12 * sc
        assert np.abs(np.cross(x, f).sum(axis=0)).max() <= 1e-12 * sc
        # restoring: the power along the force decreases |phi|
        dphi = (O.hinge_angle_grad(x) * f).sum()
        assert np.sign(dphi) == -np.sign(O.hinge_angle(x))


def test_hinge_actuation_shifts_rest_angle():
    # sin(phi/2 + alpha) = 0 at phi = -2 alpha
    rng = np.random.default_rng(24)
    x = make_hinge(0.5, rng)
    phi = O.hinge_angle(x)
    assert np.abs(O.hinge_forces(x, 1e-2, -phi / 2)).max() < 1e-14
    assert np.abs(O.hinge_forces(x, 1e-2, 0.0)).max() > 1e-6


# ---------------------------------------------------------------------------
# contact and friction (App. A.1 "Contact", App. C.2)
# ---------------------------------------------------------------------------

def contact_model(**kw):
    c = I.Contact(**kw)
    X = np.zeros((1, 3))
    return O.Model(X=X, contact=c)


def test_contact_plane_hand_values():
    m = contact_model(ke=1e4, kd=10.0, kf=1.0, mu_f=0.5, plane_on=True, plane_h=0.0)
    # above the plane: no force
    assert np.all(O.Model.contact_force(m, [0.0, 0.01, 0.0], [0.3, -2.0, 0.0]) == 0.0)
    # penetration C = 0.002, v = (0.1, -0.5, 0): f_n = 1e4*0.002 - 10*(-0.5) = 25
    # sliding |v_s| = 0.1: k_f |v_s| = 0.1 <= mu |f_n| = 12.5 -> stick, f_f = -k_f v_s
    f = m.contact_force([0.0, -0.002, 0.0], [0.1, -0.5, 0.0])
    np.testing.assert_allclose(f, [-0.1, 25.0, 0.0], rtol=1e-14)
    # fast slide |v_s| = 30: k_f |v_s| = 30 > 12.5 -> slip, |f_f| = mu |f_n| along -v_s
    f = m.contact_force([0.0, -0.002, 0.0], [0.0, -0.5, -30.0])
    np.testing.assert_allclose(f, [0.0, 25.0, 12.5], rtol=1e-14)
    # separating fast: the damping term is not clamped (literal reading)
    f = m.contact_force([0.0, -0.001, 0.0], [0.0, 3.0, 0.0])
    np.testing.assert_allclose(f, [0.0, 10.0 - 30.0, 0.0], rtol=1e-14)


def test_contact_sphere_radial_normal():
    m = contact_model(ke=100.0, kd=0.0, kf=0.0, mu_f=0.0, plane_on=False, sphere_on=True,
                      sphere_c=(0.5, 0.0, 0.5), sphere_r=0.3)
    d = np.array([1.0, 2.0, -0.5])
    d /= np.linalg.norm(d)
    x = np.array([0.5, 0.0, 0.5]) + 0.29 * d
    f = m.contact_force(x, [0.0, 0.0, 0.0])
    np.testing.assert_allclose(f, 100.0 * 0.01 * d, rtol=1e-12)


def ground_triangle(rho=0.5, y=0.0, ke=1e3, kd=2.0, kf=50.0, mu_f=0.4):
    X = np.array([[0.0, y, 0.0], [0.1, y, 0.0], [0.0, y, 0.1]])
    c = I.Contact(ke=ke, kd=kd, kf=kf, mu_f=mu_f, plane_on=True, plane_h=0.0)
    return O.Model(X=X, tris=np.array([[0, 2, 1]]), tri_mu=[10.0], tri_lam=[20.0], tri_rho=[rho],
                   contact=c)


def test_resting_contact_equilibrium_depth():
    # a flat triangle settles at the penetration C = m g / k_e of each node
    m = ground_triangle()
    mi = m.masses()
    np.testing.assert_allclose(mi, 0.5 * 0.005 / 3.0, rtol=1e-14)
    X = np.array([[0.0, 0.0, 0.0], [0.1, 0.0, 0.0], [0.0, 0.0, 0.1]])
    xS, vS = m.rollout(X, np.zeros((3, 3)), 1e-4, 20000)
    np.testing.assert_allclose(-xS[:, 1], mi * 9.81 / 1e3, rtol=1e-6)


def test_friction_slip_decelerates_at_mu_g():
    # start in vertical equilibrium (C = m g / k_e, no vertical velocity) and
    # slide along x: in the slip regime |dv/dt| = mu_f g exactly
    m = ground_triangle(kf=1e3)
    mi = m.masses()[0]
    C = mi * 9.81 / 1e3
    X = np.array([[0.0, -C, 0.0], [0.1, -C, 0.0], [0.0, -C, 0.1]])
    v0 = np.tile([1.0, 0.0, 0.0], (3, 1))
    n = 500
    xS, vS = m.rollout(X, v0, 1e-4, n)
    np.testing.assert_allclose(vS[:, 0], 1.0 - 0.4 * 9.81 * n * 1e-4, rtol=1e-12)
    np.testing.assert_allclose(vS[:, 1], 0.0, atol=1e-13)


# ---------------------------------------------------------------------------
# masses and semi-implicit Euler (App. B)
# ---------------------------------------------------------------------------

def test_lumped_mass_totals():
    X, tets = I.hex_block(3, 2, 4, 0.025)
    E = tets.shape[0]
    m = O.Model(X=X, tets=tets, tet_mu=np.full(E, MU), tet_lam=np.full(E, LAM),
                tet_rho=np.full(E, 1000.0))
    assert m.masses().sum() == pytest.approx(1000.0 * 24 * 0.025 ** 3, rel=1e-12)
    # a single tet gives each corner a quarter of its mass
    X1 = rand_tet(np.random.default_rng(30))
    m1 = O.Model(X=X1, tets=np.array([[0, 1, 2, 3]]), tet_mu=[MU], tet_lam=[LAM], tet_rho=[800.0])
    V = np.linalg.det((X1[1:] - X1[0]).T) / 6.0
    np.testing.assert_allclose(m1.masses(), 800.0 * V / 4.0, rtol=1e-12)


def test_free_fall_closed_form():
    # rigid translation under gravity, contact off: elastic forces vanish and
    # v_n = v_0 + n g dt, x_n = x_0 + n dt v_0 + g dt^2 n (n + 1)/2
    p = I.bar("a", steps=300)
    p.contact.plane_on = False
    v0 = np.tile([0.3, 0.5, -0.2], (p.n_nodes, 1))
    m = O.Model(p)
    n, dt = 300, p.dt
    xS, vS = m.rollout(p.X, v0, dt, n)
    g = np.array(p.gravity)
    np.testing.assert_allclose(vS, v0 + n * dt * g, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(xS, p.X + n * dt * v0 + g * dt * dt * n * (n + 1) / 2, rtol=1e-12, atol=1e-13)


def test_pinned_nodes_are_kinematic():
    p = I.bar("a", steps=50)
    pinned = np.zeros(p.n_nodes, dtype=np.uint8)
    pinned[p.X[:, 1] >= p.X[:, 1].max() - 1e-12] = 1  # hang the bar from its top face
    p.pinned = pinned
    m = O.Model(p)
    xS, _ = m.rollout(p.X, np.zeros_like(p.X), p.dt, 200)
    np.testing.assert_array_equal(xS[pinned == 1], p.X[pinned == 1])
    assert xS[pinned == 0][:, 1].min() < p.X[pinned == 0][:, 1].min()


def test_block_inputs_are_conforming_and_positive():
    X, tets = I.hex_block(3, 3, 3, 0.1)
    assert tets.shape == (135, 4) and X.shape == (64, 3)
    Dm = np.transpose(X[tets[:, 1:]] - X[tets[:, :1]], (0, 2, 1))
    vol = np.linalg.det(Dm) / 6.0
    assert np.all(vol > 0)
    assert vol.sum() == pytest.approx(27 * 0.001, rel=1e-12)
    # conforming: every interior triangle face is shared by exactly two tets
    faces = np.sort(np.concatenate([tets[:, [0, 1, 2]], tets[:, [0, 1, 3]], tets[:, [0, 2, 3]],
                                    tets[:, [1, 2, 3]]]), axis=1)
    _, counts = np.unique(faces, axis=0, return_counts=True)
    assert counts.max() == 2
    assert (counts == 1).sum() == 6 * 9 * 2  # boundary faces: 6 sides x 9 squares x 2


def test_workload_counts():
    X, tets = I.hex_block(64, 64, 64, 0.025)
    assert tets.shape[0] == 1_310_720 and X.shape[0] == 274_625
    X, tris, hinges = I.cloth_grid(256)
    assert X.shape[0] == 65_536 and tris.shape[0] == 130_050 and hinges.shape[0] == 194_565
    p = I.bar("a")
    assert p.n_elems == 320 and p.n_nodes == 125


# ---------------------------------------------------------------------------
# the discrete adjoint (App. B) through whole rollouts
# ---------------------------------------------------------------------------

def tiny_cases():
    rng = np.random.default_rng(40)
    cases = []
    # one tet, falling onto the ground with a sliding velocity
    X = rand_tet(rng, 0.05) + np.array([0.0, 0.052, 0.0])
    X[:, 1] -= X[:, 1].min() - 0.0004
    con = I.Contact(ke=1e3, kd=2.0, kf=3.0, mu_f=0.4)
    cases.append(dict(X=X, tets=np.array([[0, 1, 2, 3]]), tet_mu=[2e3], tet_lam=[3e3],
                      tet_rho=[500.0], tet_act=[0.01], contact=con,
                      v0=np.tile([0.2, -0.3, 0.05], (4, 1)), steps=40, dt=2e-4))
    # two tets sharing a face, elastic only
    X2, t2 = I.hex_block(1, 1, 1, 0.05, origin=(0, 0.3, 0))
    cases.append(dict(X=X2, tets=t2[:2], tet_mu=[2e3, 5e3], tet_lam=[3e3, 4e3], tet_rho=[500.0, 900.0],
                      tet_act=None, contact=I.Contact(plane_on=False),
                      v0=rng.normal(0, 0.2, X2.shape), steps=50, dt=2e-4))
    # 4x1x1 bar touching the ground
    X3, t3 = I.hex_block(4, 1, 1, 0.025, origin=(0, 0.0005, 0))
    E3 = t3.shape[0]
    cases.append(dict(X=X3, tets=t3, tet_mu=rng.uniform(1e3, 5e3, E3), tet_lam=rng.uniform(1e3, 5e3, E3),
                      tet_rho=rng.uniform(500, 1500, E3), tet_act=None,
                      contact=I.Contact(ke=2e3, kd=1.0, kf=2.0, mu_f=0.5),
                      v0=np.tile([0.3, -0.1, 0.0], (X3.shape[0], 1)), steps=30, dt=2e-4))
    # one hinge (two triangles) bent, pressed on a sphere
    xh = make_hinge(0.6, None) + np.array([0.5, 0.305, 0.5])
    con = I.Contact(ke=50.0, kd=0.01, kf=0.01, mu_f=0.5, plane_on=False, sphere_on=True,
                    sphere_c=(0.5, 0.0, 0.5), sphere_r=0.31)
    cases.append(dict(X=xh, tris=np.array([[0, 2, 3], [1, 3, 2]]), tri_mu=[10.0, 12.0], tri_lam=[20.0, 25.0],
                      tri_rho=[0.2, 0.3], tri_act=[0.0, 0.01], hinges=np.array([[0, 1, 2, 3]]), kb=[1e-4],
                      hinge_act=[0.05], contact=con, v0=rng.normal(0, 0.05, (4, 3)), steps=40, dt=1e-4))
    return cases


GRAD_KEYS = ["x0", "v0", "tet_mu", "tet_lam", "tet_rho", "tet_act", "tri_mu", "tri_lam", "tri_rho",
             "tri_act", "hinge_kb", "hinge_act", "contact"]


def build_case(c):
    kw = {k: v for k, v in c.items() if k not in ("v0", "steps", "dt")}
    m = O.Model(**kw)
    X = np.asarray(c["X"], dtype=np.float64)
    rng = np.random.default_rng(41)
    xS, _ = m.rollout(X, c["v0"], c["dt"], c["steps"])
    target = xS + rng.normal(0, 1e-3, xS.shape)
    return m, X, target


@pytest.mark.parametrize("case", range(4))
def test_adjoint_matches_central_fd_on_tiny_meshes(case):
    c = tiny_cases()[case]
    m, X, target = build_case(c)
    L, g = m.loss_grad(X, c["v0"], c["dt"], c["steps"], target)
    rng = np.random.default_rng(42)
    for key in GRAD_KEYS:
        if g[key].size == 0:
            continue
        d = rng.normal(size=g[key].shape)
        if key == "contact":
            d *= np.array([1e3, 1.0, 1.0, 0.1])
        dirs = {key: d}
        base = {"x0": X, "v0": np.asarray(c["v0"], float)}
        ad = float((g[key] * d).sum())
        def loss_at(t):
            kw = {k: v for k, v in c.items() if k not in ("v0", "steps", "dt")}
            x0, v0 = base["x0"], base["v0"]
            if key == "x0":
                x0 = x0 + t * d
            elif key == "v0":
                v0 = v0 + t * d
            elif key == "contact":
                con = kw["contact"]
                kw["contact"] = I.Contact(ke=con.ke + t * d[0], kd=con.kd + t * d[1], kf=con.kf + t * d[2],
                                          mu_f=con.mu_f + t * d[3], plane_on=con.plane_on,
                                          plane_h=con.plane_h, sphere_on=con.sphere_on,
                                          sphere_c=con.sphere_c, sphere_r=con.sphere_r)
            else:
                name = {"hinge_kb": "kb"}.get(key, key)
                arr = np.zeros(d.shape) if kw.get(name) is None else np.asarray(kw[name], float)
                kw[name] = arr * (1 + t * d) if name not in ("tet_act", "tri_act", "hinge_act") else arr + t * d
            mm = O.Model(**kw)
            xS, _ = mm.rollout(x0, v0, c["dt"], c["steps"])
            return ((xS - target) ** 2).sum()

        if key in ("tet_mu", "tet_lam", "tet_rho", "tri_mu", "tri_lam", "tri_rho", "hinge_kb"):
            name = {"hinge_kb": "kb"}.get(key, key)
            ad = float((g[key] * d * np.asarray(c[name], float)).sum())  # relative perturbation
        # central differences at several steps: truncation shrinks with the
        # step until FP64 round-off (or a stick/slip kink of the C0 contact
        # law inside the step) takes over; the best one must agree
        errs = []
        for h in (1e-4, 1e-5, 1e-6, 1e-7, 1e-8):
            fd = (loss_at(h) - loss_at(-h)) / (2 * h)
            errs.append(abs(fd - ad) / max(abs(ad), 1e-300))
        assert min(errs) <= 1e-6, (key, errs)


def test_adjoint_matches_forward_mode_with_contact():
    # bar 1b: 1000 steps, the bottom face lands near step 640
    p = I.bar("b", steps=1000)
    m = O.Model(p)
    xS, _ = m.rollout(p.X, p.v0, p.dt, p.steps)
    target = xS + I.position_noise(p.n_nodes, seed=0)
    # reference parameters differ from the simulated ones (system identification)
    p.mu *= 1.1
    m = O.Model(p)
    L, g = m.loss_grad(p.X, p.v0, p.dt, p.steps, target)
    rng = np.random.default_rng(43)
    for key in ("x0", "v0", "tet_mu", "tet_lam", "tet_rho", "contact"):
        d = rng.normal(size=g[key].shape)
        _, dL = m.loss_dir(p.X, p.v0, p.dt, p.steps, target, {key: d})
        assert float((g[key] * d).sum()) == pytest.approx(dL, rel=1e-10), key


def test_uniform_velocity_gradient_closed_form():
    # a uniform change of v0 translates the contact-free mesh rigidly, so
    # <dL/dv0, (d,..,d)> = 2 S dt sum_i (x_i(S) - x*_i) . d
    p = I.bar("a", steps=200)
    m = O.Model(p)
    rng = np.random.default_rng(44)
    xS, _ = m.rollout(p.X, p.v0, p.dt, p.steps)
    target = xS + rng.normal(0, 1e-3, xS.shape)
    L, g = m.loss_grad(p.X, p.v0, p.dt, p.steps, target)
    d = np.array([0.3, -1.0, 0.7])
    want = 2 * p.steps * p.dt * ((xS - target) @ d).sum()
    assert (g["v0"] @ d).sum() == pytest.approx(want, rel=1e-9)


def test_density_gradient_matches_fd_two_tets():
    X, t = I.hex_block(1, 1, 1, 0.05, origin=(0, 0.3, 0))
    kw = dict(X=X, tets=t[:2], tet_mu=[2e3, 4e3], tet_lam=[3e3, 3e3], contact=I.Contact(plane_on=False))
    rho = np.array([700.0, 1300.0])
    m = O.Model(tet_rho=rho, **kw)
    v0 = np.random.default_rng(45).normal(0, 0.1, X.shape)
    xS, _ = m.rollout(X, v0, 2e-4, 60)
    target = xS + 1e-3
    m = O.Model(tet_rho=rho * 1.05, **kw)
    L, g = m.loss_grad(X, v0, 2e-4, 60, target)
    for e in range(2):
        h = 1e-3
        r1, r2 = rho * 1.05, rho * 1.05
        r1 = r1.copy(); r1[e] += h
        r2 = r2.copy(); r2[e] -= h
        l1 = ((O.Model(tet_rho=r1, **kw).rollout(X, v0, 2e-4, 60)[0] - target) ** 2).sum()
        l2 = ((O.Model(tet_rho=r2, **kw).rollout(X, v0, 2e-4, 60)[0] - target) ** 2).sum()
        assert g["tet_rho"][e] == pytest.approx((l1 - l2) / (2 * h), rel=1e-6)
