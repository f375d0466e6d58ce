"""The oracle's threaded loops change nothing: with every core and with one
thread it gives bitwise the same states, loss and gradients (the per-element
work runs in parallel into per-element rows, the node sums stay serial in
element order).  This is what lets the full-horizon parity tests and the
all-cores CPU baseline use the threaded build."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2104_02646_gb300 import inputs as I


def _run(problem, steps, act_seq_grad=False):
    m = O.Model(problem)
    xS, vS = m.rollout(problem.x0, problem.v0, problem.dt, steps)
    target = xS + I.position_noise(problem.n_nodes, seed=3)
    L, g = m.loss_grad(problem.x0, problem.v0, problem.dt, steps, target, act_seq_grad=act_seq_grad)
    return xS, vS, L, g


def _same(a, b):
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert a[2] == b[2]
    for k in a[3]:
        assert np.array_equal(a[3][k], b[3][k]), k


@pytest.fixture()
def all_then_one():
    yield
    O.set_threads(0)


def _cases():
    blk = I.block(n=6, steps=30, seed=2)
    cl = I.cloth("3s", n=12, steps=30, height=0.29)
    thrown = I.cloth_throw(n=8, steps=30)
    act = I.bar("b", steps=30)
    act.act_seq = np.random.default_rng(5).normal(0.0, 0.05, (30, act.n_elems))
    return [("block", blk), ("cloth", cl), ("cloth_air", thrown), ("bar_act_seq", act)]


@pytest.mark.parametrize("name,problem", _cases(), ids=lambda v: v if isinstance(v, str) else "")
def test_threads_bitwise_equal(all_then_one, name, problem):
    steps = 30
    seq = getattr(problem, "act_seq", None) is not None
    O.set_threads(0)
    many = _run(problem, steps, seq)
    assert O.set_threads(1) == 1
    one = _run(problem, steps, seq)
    _same(many, one)
