"""Host logic of the autograd wrappers (CPU, a recording stand-in for the
library's mesh): a mesh stores one rollout, so when two rollout segments
run on it before backward, the earlier segment's backward must first replay
its own forward, and a segment whose stored rollout is still current must
not."""
import torch

from paper_2104_02646_gb300 import autograd as A


class FakeInfo:
    def __init__(self, E, B=0):
        self.n_elems = E
        self.n_hinges = B


class FakeMesh:
    """Records the calls the wrappers make; the 'rollout' adds 1 to x and v."""

    def __init__(self, N=4, E=3):
        self.n_nodes, self.info = N, FakeInfo(E)
        self.calls = []
        self.stored = None
        self.act = None

    def set_act_seq(self, a=None, h=None):
        self.act = None if a is None else a.clone()
        self.calls.append("set_act_seq")

    def set_params(self, mu=None, lam=None, rho=None):
        self.calls.append("set_params")

    def set_state(self, x=None, v=None):
        self.x, self.v = x.clone(), v.clone()
        self.calls.append("set_state")

    def rollout(self, dt, steps, K=0):
        # with an actuation sequence the 'rollout' also adds its sum
        d = 1.0 + (0.0 if self.act is None else float(self.act.sum()))
        self.x, self.v = self.x + d, self.v + d
        self.stored = (self.x.clone(), steps, None if self.act is None else self.act.clone())
        self.calls.append(("rollout", steps))

    def get_state(self, x, v):
        x.copy_(self.x)
        v.copy_(self.v)

    def adjoint(self, g, dLdx=None, dLdv=None):
        # identity Jacobian: dL/dx0 = dL/dx(S), dL/dv0 = dL/dv(S); the stored rollout is consumed
        assert self.stored is not None, "adjoint without a stored rollout"
        # the adjoint must run under the actuation its rollout used
        sa = self.stored[2]
        assert (sa is None and self.act is None) or (sa is not None and self.act is not None
                                                     and torch.equal(sa, self.act)), "stale actuation"
        self.calls.append(("adjoint", self.stored[1]))
        g["d_x0"].copy_(dLdx if dLdx is not None else torch.zeros_like(g["d_x0"]))
        g["d_v0"].copy_(dLdv if dLdv is not None else torch.zeros_like(g["d_v0"]))
        if "d_act_seq" in g:
            # d x(S)/d act[n, e] = 1 for every entry: dL/d act = sum of dL/dx(S) + dL/dv(S)
            s = (0.0 if dLdx is None else float(dLdx.sum())) + (0.0 if dLdv is None else float(dLdv.sum()))
            g["d_act_seq"].fill_(s)
        self.stored = None


def _params(E):
    return torch.ones(E), torch.ones(E), torch.ones(E)


def test_two_segments_on_one_mesh_replay_the_earlier_one():
    m = FakeMesh()
    mu, lam, rho = _params(3)
    x0 = torch.zeros(4, 3, requires_grad=True)
    v0 = torch.zeros(4, 3)
    x1, v1 = A.rollout(m, 1e-3, 10, mu, lam, rho, x0, v0)
    x2, v2 = A.rollout(m, 1e-3, 20, mu, lam, rho, x1, v1)
    (x2.sum() + x1.sum()).backward()
    rollouts = [c for c in m.calls if isinstance(c, tuple)]
    # forward 10, forward 20, backward of the 20-step segment (still stored),
    # then the 10-step segment replays itself before its adjoint
    assert rollouts == [("rollout", 10), ("rollout", 20), ("adjoint", 20), ("rollout", 10), ("adjoint", 10)]
    # identity Jacobians: x0 receives dL/dx1 = 1 (direct) + 1 (through x2)
    assert torch.equal(x0.grad, torch.full((4, 3), 2.0))


def test_a_current_segment_is_not_replayed():
    m = FakeMesh()
    mu, lam, rho = _params(3)
    x0 = torch.zeros(4, 3, requires_grad=True)
    x1, _ = A.rollout(m, 1e-3, 5, mu, lam, rho, x0, torch.zeros(4, 3))
    x1.sum().backward()
    assert [c for c in m.calls if isinstance(c, tuple)] == [("rollout", 5), ("adjoint", 5)]
    # a second, fresh forward + backward after the adjoint consumed the rollout
    m.calls.clear()
    x0b = torch.zeros(4, 3, requires_grad=True)
    y, _ = A.rollout(m, 1e-3, 7, mu, lam, rho, x0b, torch.zeros(4, 3))
    y.sum().backward()
    assert [c for c in m.calls if isinstance(c, tuple)] == [("rollout", 7), ("adjoint", 7)]


def test_interleaved_actuated_rollouts_replay_with_their_own_actuation():
    # two actuated rollouts on one mesh before backward: the first one's
    # backward replays it with its own sequence (not the second's)
    m = FakeMesh()
    a1 = torch.full((10, 3), 0.1, requires_grad=True)
    a2 = torch.full((20, 3), -0.2, requires_grad=True)
    x0 = torch.zeros(4, 3)
    v0 = torch.zeros(4, 3)
    x1, _ = A.actuated_rollout(m, 1e-3, 10, a1, x0, v0)
    x2, _ = A.actuated_rollout(m, 1e-3, 20, a2, x0, v0)
    (x1.sum() + x2.sum()).backward()
    rollouts = [c for c in m.calls if isinstance(c, tuple)]
    assert rollouts == [("rollout", 10), ("rollout", 20), ("adjoint", 20), ("rollout", 10), ("adjoint", 10)]
    assert torch.allclose(a1.grad, torch.full((10, 3), 12.0))
    assert torch.allclose(a2.grad, torch.full((20, 3), 12.0))


def test_plain_rollout_after_an_actuated_one_clears_the_sequence():
    # a plain differentiable rollout after an actuated one runs (and its
    # adjoint re-evaluates forces) without the earlier sequence
    m = FakeMesh()
    mu, lam, rho = _params(3)
    a = torch.full((5, 3), 0.5, requires_grad=True)
    xa, _ = A.actuated_rollout(m, 1e-3, 5, a, torch.zeros(4, 3), torch.zeros(4, 3))
    x0 = torch.zeros(4, 3, requires_grad=True)
    x1, _ = A.rollout(m, 1e-3, 7, mu, lam, rho, x0, torch.zeros(4, 3))
    assert torch.equal(x1, torch.ones(4, 3))  # no actuation added
    (x1.sum() + xa.sum()).backward()
    assert torch.equal(x0.grad, torch.ones(4, 3))
    assert torch.allclose(a.grad, torch.full((5, 3), 12.0))
