"""Pins of the oracle's time-varying actuation (the control input of the
paper's visuomotor control experiments, Sec. 3, driving the per-element
actuation of the energy, App. A): row n of the sequence is added to an
element's actuation during step n.

Pinned against: a sequence constant in time (must reproduce static
actuation exactly, and its per-step gradients must sum to the static
gradient); forward-mode dual numbers along random directions; central finite
differences on a tiny mesh; and a zero-padded sequence (steps beyond its end
carry no extra actuation).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2104_02646_gb300 import inputs as I


def _bar(steps, drop=0.02):
    p = I.bar("b", steps=steps)
    p.X = p.X + np.array([0.0, drop - 0.02, 0.0])
    p.x0 = p.X.copy()
    return p


def _target(p, steps):
    m = O.Model(p)
    xS, _ = m.rollout(p.x0, p.v0, p.dt, steps)
    return xS + I.position_noise(p.n_nodes, sigma=1e-3, seed=7)


def test_constant_sequence_equals_static_actuation():
    S = 60
    p = _bar(S)
    c = np.random.default_rng(1).uniform(-0.2, 0.2, p.n_elems)
    tgt = _target(p, S)
    ps = I.Problem(**{f: getattr(p, f) for f in p.__dataclass_fields__})
    ps.act = c
    m_static = O.Model(ps)
    m_seq = O.Model(p, act_seq=np.tile(c, (S, 1)))
    xa, va = m_static.rollout(p.x0, p.v0, p.dt, S)
    xb, vb = m_seq.rollout(p.x0, p.v0, p.dt, S)
    np.testing.assert_array_equal(xa, xb)
    np.testing.assert_array_equal(va, vb)
    La, ga = m_static.loss_grad(p.x0, p.v0, p.dt, S, tgt)
    Lb, gb = m_seq.loss_grad(p.x0, p.v0, p.dt, S, tgt, act_seq_grad=True)
    assert La == Lb
    assert gb["tet_act_seq"].shape == (S, p.n_elems)
    np.testing.assert_allclose(gb["tet_act_seq"].sum(axis=0), ga["tet_act"], rtol=1e-11, atol=1e-18)
    np.testing.assert_allclose(gb["tet_act"], ga["tet_act"], rtol=1e-12, atol=1e-18)
    assert np.abs(gb["tet_act_seq"]).max() > 0


def test_per_step_gradient_matches_forward_mode():
    S = 40
    p = _bar(S)
    rng = np.random.default_rng(2)
    seq = 0.1 * np.sin(np.linspace(0, 3, S))[:, None] * rng.uniform(-1, 1, p.n_elems)[None, :]
    tgt = _target(p, S)
    m = O.Model(p, act_seq=seq)
    L, g = m.loss_grad(p.x0, p.v0, p.dt, S, tgt, act_seq_grad=True)
    for k in range(3):
        d = rng.normal(size=(S, p.n_elems))
        L2, dL = m.loss_dir(p.x0, p.v0, p.dt, S, tgt, {"tet_act_seq": d})
        assert abs(L2 - L) <= 1e-14 * abs(L)
        ref = float(np.sum(g["tet_act_seq"] * d))
        assert abs(dL - ref) <= 1e-10 * max(abs(dL), 1e-30), (dL, ref)


def test_per_step_gradient_matches_finite_differences():
    # 2 tets under gravity on the ground; one sequence entry at a time
    X = np.array([[0, 0.0, 0], [0.1, 0.0, 0], [0, 0.1, 0], [0, 0.0, 0.1], [0.1, 0.1, 0.1]]) + [0, 0.001, 0]
    tets = np.array([[0, 1, 2, 3], [1, 2, 3, 4]])
    con = I.Contact()
    kw = dict(X=X, tets=tets, tet_mu=np.full(2, 2e3), tet_lam=np.full(2, 3e3), tet_rho=np.full(2, 500.0),
              contact=con)
    S, dt = 30, 1e-3
    rng = np.random.default_rng(3)
    seq = rng.uniform(-0.05, 0.05, (S, 2))
    x0, v0 = X.copy(), np.zeros_like(X)
    tgt = X + rng.normal(0, 1e-3, X.shape)
    L, g = O.Model(act_seq=seq, **kw).loss_grad(x0, v0, dt, S, tgt, act_seq_grad=True)
    for (n, e) in [(0, 0), (7, 1), (S - 1, 0), (S // 2, 1)]:
        best = np.inf
        for h in (1e-4, 1e-5, 1e-6, 1e-7):
            sp, sm = seq.copy(), seq.copy()
            sp[n, e] += h
            sm[n, e] -= h
            Lp, _ = O.Model(act_seq=sp, **kw).loss_grad(x0, v0, dt, S, tgt)
            Lm, _ = O.Model(act_seq=sm, **kw).loss_grad(x0, v0, dt, S, tgt)
            fd = (Lp - Lm) / (2 * h)
            best = min(best, abs(fd - g["tet_act_seq"][n, e]) / max(abs(fd), 1e-300))
        assert best <= 1e-6, (n, e, best)


def test_sequence_shorter_than_rollout_is_zero_padded():
    S = 50
    p = _bar(S)
    rng = np.random.default_rng(4)
    short = rng.uniform(-0.1, 0.1, (20, p.n_elems))
    padded = np.vstack([short, np.zeros((S - 20, p.n_elems))])
    xa, _ = O.Model(p, act_seq=short).rollout(p.x0, p.v0, p.dt, S)
    xb, _ = O.Model(p, act_seq=padded).rollout(p.x0, p.v0, p.dt, S)
    np.testing.assert_array_equal(xa, xb)


def test_hinge_sequence_forward_mode():
    S = 25
    p = I.cloth("3s", n=6, steps=S, grid_scaled=True, height=0.29)
    rng = np.random.default_rng(5)
    hseq = rng.uniform(-0.1, 0.1, (S, p.n_hinges))
    tseq = rng.uniform(-0.1, 0.1, (S, p.n_elems))
    tgt = _target(p, S)
    m = O.Model(p, act_seq=tseq, hinge_act_seq=hseq)
    L, g = m.loss_grad(p.x0, p.v0, p.dt, S, tgt, act_seq_grad=True)
    d1, d2 = rng.normal(size=hseq.shape), rng.normal(size=tseq.shape)
    _, dL = m.loss_dir(p.x0, p.v0, p.dt, S, tgt, {"hinge_act_seq": d1, "tri_act_seq": d2})
    ref = float(np.sum(g["hinge_act_seq"] * d1) + np.sum(g["tri_act_seq"] * d2))
    assert abs(dL - ref) <= 1e-9 * max(abs(dL), 1e-30), (dL, ref)
