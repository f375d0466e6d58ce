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
