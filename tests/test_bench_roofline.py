"""bench.py's roofline inputs on the benchmark mesh (CPU): the algorithmic
bytes per element-step (the element stream plus the node traffic per tet) and
the count of kernel launches the step claims."""
import bench

E, N, S = 1_310_720, 274_625, 200  # block64


def test_algorithmic_bytes_per_element_step():
    fwd = bench.alg_bytes(True, E, N) / E
    adj = bench.alg_bytes(False, E, N) / E
    # 64 B per tet + 52 (forward) / 88 (adjoint) B per node, N / E = 0.2095 nodes per tet
    assert abs(fwd - (64 + 52 * N / E)) < 1e-12 and round(fwd, 1) == 74.9
    assert abs(adj - (64 + 88 * N / E)) < 1e-12 and round(adj, 1) == 82.4
    assert round(fwd + adj, 1) == 157.3
    assert bench.alg_bytes(False, E, N) == 108_053_080  # bytes per adjoint launch


def test_launch_count_per_benchmark_step():
    # K = 1: reset; checkpoint copy, S (patch + boundary) forward steps, loss
    # and its finalisation; the final state back; seed, two zeroings (w_bar,
    # mu/lambda); S reverse steps; node and element gradients
    k1 = bench.launches_per_step(S, 1, True)
    assert k1 == 1 + (1 + 2 * S + 2) + 1 + (1 + 1 + 2) + 2 * S + 2
    # K > 1 adds, per segment, a checkpoint copy and the segment's recomputed steps
    K = 15
    n_ck = -(-S // K)
    assert bench.launches_per_step(S, K, True) == k1 - 1 + n_ck + 2 * S
    # a mesh without boundary nodes (one patch) has no boundary kernels
    assert bench.launches_per_step(S, 1, False) == k1 - 2 * S
