"""The parity checker itself (CPU): what the GPU tests assert must reject the
mistakes it is there to catch and accept FP32 round-off.  The reference is a
real oracle rollout of a small block."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2104_02646_gb300 import inputs as I

from gpu_util import (GRAD_COS, GRAD_REL, POS_CONTACT, TET_KEYS, check_grads, check_state, cosine, entry_bar,
                      entry_ratio, make_target)


@pytest.fixture(scope="module")
def ref():
    S = 60
    p = I.block(n=4, steps=S, seed=4)
    m = O.Model(p)
    tgt = make_target(p, S)
    xS, vS = m.rollout(p.x0, p.v0, p.dt, S)
    L, g = m.loss_grad(p.x0, p.v0, p.dt, S, tgt)
    return p, xS, vS, L, g


def _fp32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def test_round_off_passes(ref):
    p, xS, vS, L, g = ref
    check_state(_fp32(xS), _fp32(vS), xS, vS, p.x0, POS_CONTACT)
    out = {gk: _fp32(g[ok]) for ok, gk in TET_KEYS.items()}
    check_grads(out, g, TET_KEYS)


def test_mesh_that_never_moved_fails(ref):
    # the failure the old centroid-removed position norm could not see: with
    # x(S) = x(0) its ratio is ~ |displacement| / |spread| << 1e-3 here too
    p, xS, vS, L, g = ref
    from gpu_util import rel_pos
    assert rel_pos(p.x0, xS) < 1e-2
    with pytest.raises(AssertionError):
        check_state(p.x0.copy(), vS, xS, vS, p.x0, POS_CONTACT)
    with pytest.raises(AssertionError):
        check_state(xS, np.zeros_like(vS), xS, vS, p.x0, POS_CONTACT)


def test_one_wrong_node_fails(ref):
    # a velocity sign error on a single node passes neither check
    p, xS, vS, L, g = ref
    k = int(np.argmax(np.linalg.norm(vS, axis=1)))
    v = vS.copy()
    v[k] = -v[k]
    with pytest.raises(AssertionError):
        check_state(xS, v, xS, vS, p.x0, POS_CONTACT)
    # the displacement of one node off by 2 % of the largest displacement
    x = xS.copy()
    d = xS - p.x0
    x[k] += 0.02 * np.max(np.linalg.norm(d, axis=1)) * np.array([1.0, 0.0, 0.0])
    with pytest.raises(AssertionError):
        check_state(x, vS, xS, vS, p.x0, POS_CONTACT)


def test_error_on_one_element_fails_entry_check_not_norm(ref):
    # a sign error on one element of small gradient (a wrong index or a
    # flipped term confined to one element): rel-L2 and cosine stay within
    # the norm bars, the per-entry bar catches it
    p, xS, vS, L, g = ref
    b = g["tet_mu"]
    k = int(np.argmin(np.abs(np.abs(b) - 4e-4 * np.linalg.norm(b))))
    a = b.copy()
    a[k] = -a[k]
    assert np.linalg.norm(a - b) / np.linalg.norm(b) <= GRAD_REL
    assert cosine(a, b) >= GRAD_COS
    assert entry_ratio(a, b, entry_bar(GRAD_REL)) > 1.0
    out = {gk: g[ok].copy() for ok, gk in TET_KEYS.items()}
    out["d_mu"] = a
    with pytest.raises(AssertionError):
        check_grads(out, g, TET_KEYS)


def test_swapped_gradient_entries_fail(ref):
    # a transposed scatter (two elements' results exchanged)
    p, xS, vS, L, g = ref
    out = {gk: g[ok].copy() for ok, gk in TET_KEYS.items()}
    b = out["d_lambda"]
    i, j = int(np.argmax(b)), int(np.argmin(b))
    b[i], b[j] = b[j], b[i]
    with pytest.raises(AssertionError):
        check_grads(out, g, TET_KEYS)


def test_round_off_noise_passes_entry_bar():
    # an error field of FP32-like relative noise at the full norm bar (rel-L2
    # = 1e-3 with Gaussian tails) over a million entries passes the entry bar
    rng = np.random.default_rng(7)
    b = rng.standard_normal(10**6)
    a = b * (1.0 + 1e-3 * rng.standard_normal(10**6))
    assert entry_ratio(a, b, entry_bar(GRAD_REL)) < 1.0


def test_entry_ratio_edge_cases():
    assert entry_ratio(np.zeros(0), np.zeros(0), 1e-3) == 0.0
    assert entry_ratio(np.zeros(5), np.zeros(5), 1e-3) == 0.0
    assert entry_ratio(np.ones(5), np.zeros(5), 1e-3) == float("inf")
    # rows compare by their norms
    b = np.array([[3.0, 4.0, 0.0], [0.0, 0.0, 0.0]])
    a = b + np.array([[0.0, 0.0, 1e-3], [0.0, 0.0, 0.0]])
    rms = np.sqrt((25.0 + 0.0) / 2)
    assert entry_ratio(a, b, 1.0) == pytest.approx(1e-3 / (5.0 + rms))


def test_conditioned_bar_follows_the_oracles_own_sensitivity(ref):
    # an error 5x the norm bar fails while the oracle is well-conditioned and
    # passes once the oracle itself moves by more than a tenth of it under a
    # rounding of its inputs
    from gpu_util import check_grads_conditioned
    p, xS, vS, L, g = ref
    rng = np.random.default_rng(3)
    noisy = lambda b, s: b * (1.0 + s * rng.standard_normal(np.shape(b)))
    gpu = {gk: noisy(g[ok], 5e-3) for ok, gk in TET_KEYS.items()}
    well = {ok: noisy(g[ok], 1e-5) for ok in TET_KEYS}
    with pytest.raises(AssertionError):
        check_grads_conditioned(gpu, g, well, TET_KEYS)
    ill = {ok: noisy(g[ok], 2e-3) for ok in TET_KEYS}
    check_grads_conditioned(gpu, g, ill, TET_KEYS)


def test_fp32_inputs_round_what_the_gpu_receives(ref):
    from gpu_util import fp32_inputs
    p, xS, vS, L, g = ref
    q, t32 = fp32_inputs(p, xS)
    for f in ("X", "x0", "v0", "mu", "lam", "rho"):
        a = getattr(q, f)
        assert np.array_equal(a, a.astype(np.float32).astype(np.float64)), f
        assert np.allclose(a, getattr(p, f), rtol=1e-7, atol=0), f
    assert q.elems is p.elems and np.array_equal(t32, xS.astype(np.float32))
