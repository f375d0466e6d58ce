"""Failure detection without a GPU fault.

Malformed inputs are refused on the host with GS_EINVAL before any work is
enqueued.  Budgets and a failing allocator give GS_ENOMEM.  Calls out of
order give GS_ESTATE.  A rollout that blows up sets the sticky non-finite
flag, both for a mesh and for a served query.  The kernels' bounded-wait
failure path runs out as designed against a barrier that nothing arrives at.
"""
import ctypes as C
import dataclasses

import numpy as np
import pytest

from paper_2104_02646_gb300 import inputs as I

from gpu_util import make_target

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(gs):
    return gs.Context(0)


def _copy(p, **changes):
    fields = {f: getattr(p, f) for f in p.__dataclass_fields__}
    for k, v in fields.items():
        if isinstance(v, np.ndarray):
            fields[k] = v.copy()
    fields.update(changes)
    return I.Problem(**fields)


def _mutations():
    def out_of_range(p):
        p.elems[3, 2] = p.n_nodes + 5

    def negative_index(p):
        p.elems[1, 0] = -1

    def repeated_node(p):
        p.elems[0, 1] = p.elems[0, 0]

    def inverted(p):
        p.elems[0, [1, 2]] = p.elems[0, [2, 1]]

    def nan_position(p):
        p.X[5, 1] = np.nan

    def zero_mu(p):
        p.mu[7] = 0.0

    def bad_plane(p):
        p.contact = dataclasses.replace(p.contact, plane_n=(0.0, 2.0, 0.0))

    return [out_of_range, negative_index, repeated_node, inverted, nan_position, zero_mu, bad_plane]


@pytest.mark.parametrize("shape", [dict(block_threads=100), dict(block_threads=2048),
                                   dict(block_threads_adj=48), dict(block_threads_adj=1056)])
def test_bad_thread_counts_are_rejected(gs, ctx, shape):
    with pytest.raises(gs.GradsimError) as ei:
        gs.Mesh(ctx, I.block(n=3, steps=1), **shape)
    assert ei.value.status == gs.GS_EINVAL


@pytest.mark.parametrize("mutate", _mutations(), ids=lambda f: f.__name__)
def test_malformed_mesh_is_rejected(gs, ctx, mutate):
    p = _copy(I.block(n=3, steps=1))
    mutate(p)
    with pytest.raises(gs.GradsimError) as ei:
        gs.Mesh(ctx, p)
    assert ei.value.status == gs.GS_EINVAL
    # the context stays usable
    gs.Mesh(ctx, I.block(n=3, steps=1)).close()


def test_budget_gives_enomem(gs):
    small = gs.Context(0, budget=1 << 16)
    with pytest.raises(gs.GradsimError) as ei:
        gs.Mesh(small, I.block(n=6, steps=1))
    assert ei.value.status == gs.GS_ENOMEM
    assert "budget" in str(ei.value)


def test_allocator_returning_null_gives_enomem(gs):
    calls = []

    def alloc(nbytes, stream, user):
        calls.append(nbytes)
        return None

    def free(ptr, nbytes, stream, user):
        pass

    cb = (gs._ALLOC_FN(alloc), gs._FREE_FN(free))
    a = gs.gs_allocator(cb[0], cb[1], None)
    h = gs._vp()
    gs.check(gs.load().gs_create(C.byref(h), 0, 0, C.byref(a)))
    try:
        d, keep = gs.mesh_desc(I.block(n=3, steps=1))
        m = gs._vp()
        st = gs.load().gs_mesh_create(h, C.byref(d), C.byref(m))
        assert st == gs.GS_ENOMEM
        assert b"allocator" in gs.load().gs_last_error()
        assert calls
    finally:
        gs.load().gs_destroy(h)


def test_adjoint_before_rollout_is_estate(gs, ctx):
    import torch
    p = I.block(n=3, steps=1)
    m = gs.Mesh(ctx, p)
    g = {"d_mu": torch.zeros(p.n_elems, dtype=torch.float64, device="cuda")}
    with pytest.raises(gs.GradsimError) as ei:
        m.adjoint(g)
    assert ei.value.status == gs.GS_ESTATE
    # an adjoint consumes its rollout (no keep): a second one is refused too
    m.rollout(p.dt, 3)
    m.adjoint(g)
    with pytest.raises(gs.GradsimError) as ei:
        m.adjoint(g)
    assert ei.value.status == gs.GS_ESTATE


def test_unstable_cloth_sets_the_nonfinite_flag(gs, ctx):
    # the 256^2 cloth with the stated stiffnesses blows up under explicit Euler
    # once it meets the sphere (about step 320; it starts flat and force-free)
    p = I.cloth("3", n=256, steps=500)
    m = gs.Mesh(ctx, p)
    assert m.info.dt_stable < p.dt
    m.rollout(p.dt, 500)
    assert m.status == gs.GS_WUNSTABLE       # the warning at launch
    assert m.check_finite() == gs.GS_ENONFINITE
    assert m.check_finite(reset=True) == gs.GS_ENONFINITE
    m.reset()
    assert m.check_finite() == gs.GS_OK       # cleared; the stable variant runs clean
    q = gs.Mesh(ctx, I.cloth("3s", n=32, steps=50))
    q.rollout(1e-4, 50)
    assert q.check_finite() == gs.GS_OK


def test_server_reports_a_nonfinite_query_and_keeps_serving(gs):
    ctx = gs.Context(0)
    srv = gs.Server(ctx, budget=8 << 30)
    bad = I.cloth("3", n=256, steps=500)
    good = I.block(n=4, steps=50)
    t_bad = srv.submit(bad, bad.X)
    t_good = srv.submit(good, make_target(good, 50))
    st, _ = srv.poll(t_bad, timeout_ms=120000)
    assert st == gs.GS_ENONFINITE
    st, r = srv.poll(t_good, timeout_ms=120000)
    assert st == gs.GS_OK and np.all(np.isfinite(r["d_mu"]))
    srv.close()


def test_bounded_wait_runs_out_and_reports(gs):
    # a barrier that nothing arrives at: the wait gives up after its polls,
    # sets status bit 2 and the kernel returns
    st = C.c_int(-1)
    gs.check(gs.load().gs_selftest_bounded_wait(1000, C.byref(st), None))
    assert st.value == 2
    with pytest.raises(gs.GradsimError) as ei:
        gs.check(gs.load().gs_selftest_bounded_wait(0, C.byref(st), None))
    assert ei.value.status == gs.GS_EINVAL
    # the context is still usable afterwards
    ctx = gs.Context(0)
    p = I.block(n=3, steps=5)
    m = gs.Mesh(ctx, p)
    m.rollout(p.dt, 5)
    assert m.check_finite() == gs.GS_OK
