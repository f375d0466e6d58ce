"""Host logic of the autotuner: state-buffer counts, the choice of the
checkpoint interval under a memory budget, and the cache file."""
import math

import pytest

from paper_2104_02646_gb300 import autotune as A


def test_state_buffers_counts():
    # K = 1 keeps every state: S + 1 states and the current-state buffer
    assert A.state_buffers(200, 1) == 202
    # checkpoints ceil(S/K), K + 1 segment buffers, the current state
    assert A.state_buffers(200, 15) == 1 + 14 + 16
    assert A.state_buffers(57, 8) == 1 + 8 + 9
    assert A.state_buffers(0, 5) == 1 + 1 + 6


def test_choose_K_prefers_least_recompute_that_fits():
    N, S = 274625, 200
    per = N * A.STATE_BYTES
    assert A.choose_K(N, S, 10 ** 12) == 1              # everything fits: no recompute
    assert A.choose_K(N, S, 202 * per) == 1              # exactly fits
    assert A.choose_K(N, S, 201 * per) > 1               # one byte short of K = 1
    K = A.choose_K(N, S, 40 * per)
    assert A.state_buffers(S, K) <= 40
    assert all(A.state_buffers(S, k) > 40 for k in range(1, K))  # the smallest K that fits


def test_choose_K_nothing_fits_gives_fewest_buffers():
    N, S = 1000, 1000
    K = A.choose_K(N, S, 1)
    best = min(A.state_buffers(S, k) for k in range(2, S + 1))
    assert A.state_buffers(S, K) == best
    # among equally small buffer counts (flat near sqrt(S)) the smallest K,
    # which keeps the most checkpoints and recomputes the least
    assert all(A.state_buffers(S, k) > best for k in range(2, K))
    assert abs(K - math.sqrt(S)) <= 0.2 * math.sqrt(S)


@pytest.mark.parametrize("S", [0, 1])
def test_choose_K_trivial_horizons(S):
    assert A.choose_K(10, S, 0) == 1


def test_cache_roundtrip(tmp_path):
    p = str(tmp_path / "tune.json")
    assert A.load_cache(p) == {}
    A.store_cache({"k": {"patch_elems": 256, "block_threads": 128, "ms": 1.5}}, p)
    assert A.load_cache(p)["k"]["patch_elems"] == 256
    with open(p, "w") as f:
        f.write("not json")
    assert A.load_cache(p) == {}


def test_tune_picks_the_fastest_shape_and_reports_adjoint_threads(tmp_path, monkeypatch):
    # the timing of each candidate is faked (no GPU): the tuner must accept
    # candidates with and without an adjoint thread count, skip shapes that
    # could not be built, report the winner's three numbers and cache them
    import torch
    from paper_2104_02646_gb300 import inputs as I
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a: "fake GPU")
    fake_ms = {(256, 128, 0): 2.0, (320, 160, 128): 1.5, (320, 160, 0): 1.7, (100000, 128, 0): None}
    seen = []

    def fake_time(ctx, problem, pe, bt, steps, K, reps, bta=0):
        seen.append((pe, bt, bta))
        return fake_ms[(pe, bt, bta)]

    monkeypatch.setattr(A, "_time_candidate", fake_time)

    class Ctx:
        device = 0

    p = I.block(n=3, steps=20)
    cache = str(tmp_path / "tune.json")
    cands = ((256, 128), (320, 160, 128), (320, 160), (100000, 128))
    r = A.tune(Ctx(), p, steps=5, candidates=cands, budget_bytes=10 ** 12, cache=cache)
    assert seen == [(256, 128, 0), (320, 160, 128), (320, 160, 0), (100000, 128, 0)]
    assert (r["patch_elems"], r["block_threads"], r["block_threads_adj"]) == (320, 160, 128)
    assert r["K"] == 1 and r["ms"] == 1.5
    assert [t["ms"] for t in r["timings"]][-1] is None
    again = A.tune(Ctx(), p, steps=5, candidates=cands, budget_bytes=10 ** 12, cache=cache)
    assert again["cached"] and again["block_threads_adj"] == 128
    # an entry cached before the adjoint count existed reads as "same as the forward"
    entries = A.load_cache(cache)
    key = next(iter(entries))
    del entries[key]["block_threads_adj"]
    A.store_cache(entries, cache)
    old = A.tune(Ctx(), p, steps=5, candidates=cands, budget_bytes=10 ** 12, cache=cache)
    assert old["block_threads_adj"] == 0


def test_default_candidates_are_valid_shapes():
    for c in A.DEFAULT_CANDIDATES:
        assert len(c) in (2, 3)
        assert all(t % 32 == 0 and 0 < t <= 1024 for t in c[1:])
        assert c[0] > 0
