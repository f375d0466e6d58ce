"""Host-side input generators: counts, structure and ranges of the seeded
workloads (no physics; CPU only)."""
import collections
import math

import numpy as np

from paper_2104_02646_gb300 import inputs as I


def test_surface_faces_form_a_closed_oriented_surface():
    for dims in ((1, 1, 1), (3, 2, 4)):
        X, tets = I.hex_block(*dims, h=0.1)
        F = I.surface_faces(tets)
        a, b, c = dims
        assert len(F) == 4 * (a * b + b * c + c * a)
        # every directed edge appears once and its reverse once: closed and consistently oriented
        directed = collections.Counter()
        for f in F:
            for i in range(3):
                directed[(f[i], f[(i + 1) % 3])] += 1
        assert all(v == 1 for v in directed.values())
        assert all(directed[(q, p)] == 1 for (p, q) in directed)
        # enclosed volume by the divergence theorem equals the block's
        vol = sum(np.dot(X[f[0]], np.cross(X[f[1]], X[f[2]])) for f in F) / 6.0
        assert abs(vol - a * b * c * 1e-3) < 1e-12


def test_box_points_and_inertia():
    pts, faces = I.box_points((0.4, 0.2, 0.6), n=5)
    assert len(pts) == 5 ** 3 - 3 ** 3
    half = np.array([0.2, 0.1, 0.3])
    assert np.allclose(np.abs(pts).max(axis=0), half)
    assert np.all(np.isclose(np.abs(pts) / half, 1.0).any(axis=1))  # on the surface
    assert faces.max() == 7 and len(faces) == 12
    b = I.box_body(size=(0.4, 0.2, 0.6), density=10.0)
    assert abs(b.mass - 10.0 * 0.048) < 1e-12
    assert abs(np.linalg.norm(b.state0[3:7]) - 1.0) < 1e-15


def test_rigid_batch_ranges():
    bodies = I.rigid_batch(64, seed=5, n=3)
    for body in bodies:
        size = 2 * np.abs(body.points).max(axis=0)
        dens = body.mass / np.prod(size)
        assert 2.0 <= dens <= 12.0
        assert 0.2 <= body.contact[3] <= 1.0
        assert abs(np.linalg.norm(body.state0[3:7]) - 1.0) < 1e-12
        assert np.all(np.abs(body.state0[[0, 2]]) <= 6.5)
    assert len({round(b.mass, 9) for b in bodies}) == 64  # seeded, distinct


def test_cloth_throw_and_hanging_beam():
    p = I.cloth_throw(n=9, steps=10, seed=3)
    assert p.n_elems == 2 * 8 * 8 and p.air is not None
    assert p.n_hinges == 3 * 8 * 8 - 2 * 8  # interior edges of an 8 x 8 grid split by one diagonal
    assert np.all(np.isfinite(p.v0)) and p.v0[:, 1].mean() > 0  # thrown upwards
    q = I.cloth_throw(n=9, steps=10, seed=3)
    assert np.array_equal(p.X, q.X) and np.array_equal(p.v0, q.v0)
    beam = I.hanging_beam(1000.0)
    assert beam.pinned.sum() == 3 * 3 and beam.n_elems == 5 * 8 * 2 * 2
    assert np.all(beam.X[beam.pinned.astype(bool), 0] == 0.0)


def test_look_at_camera():
    cam = I.look_at((1.0, 2.0, -3.0), (0.0, 0.5, 0.0), width=80, height=60, fov_deg=45.0)
    assert np.allclose(cam.R @ cam.R.T, np.eye(3), atol=1e-12)
    assert abs(np.linalg.det(cam.R) - 1.0) < 1e-12
    eye = -cam.R.T @ cam.t
    assert np.allclose(eye, (1.0, 2.0, -3.0))
    assert abs(cam.fx - 40.0 / math.tan(math.radians(22.5))) < 1e-9


def _cyclic(t):
    """The three rotations of a triangle (same orientation)."""
    a, b, c = (int(v) for v in t)
    return {(a, b, c), (b, c, a), (c, a, b)}


def test_cloth_hinges_are_the_interior_edges():
    # brute force over the triangles: every edge shared by two triangles is
    # one hinge (x1, x2, x3, x4) whose edge x3-x4 is that edge and whose
    # wing tips x1, x2 are the triangles' third vertices, with (x1, x3, x4)
    # and (x2, x4, x3) oriented as the triangles are; edges on the border
    # carry no hinge (grids of 2, 3 and 7 nodes a side; the 256^2 count is
    # pinned with the workload counts).
    for n in (2, 3, 7):
        X, tris, hinges = I.cloth_grid(n)
        edges = collections.defaultdict(list)
        for t, tri in enumerate(tris):
            for k in range(3):
                edges[frozenset((int(tri[k]), int(tri[(k + 1) % 3])))].append(t)
        interior = {e: ts for e, ts in edges.items() if len(ts) == 2}
        assert all(len(ts) in (1, 2) for ts in edges.values())
        assert len(hinges) == len(interior) == 3 * (n - 1) ** 2 - 2 * (n - 1)
        oriented = set()
        for tri in tris:
            oriented |= _cyclic(tri)
        seen = set()
        for x1, x2, x3, x4 in (tuple(int(v) for v in h) for h in hinges):
            e = frozenset((x3, x4))
            assert e in interior and e not in seen
            seen.add(e)
            assert {frozenset(tris[t]) for t in interior[e]} == {frozenset((x1, x3, x4)), frozenset((x2, x3, x4))}
            assert (x1, x3, x4) in oriented and (x2, x4, x3) in oriented
        # sorted by (min, max) edge node id
        keys = [(min(h[2], h[3]), max(h[2], h[3])) for h in hinges.tolist()]
        assert keys == sorted(keys)


def test_batch_follows_its_recipe():
    # 512 hex blocks: element-count targets log-uniform in [1e3, 1e5], the
    # second and third sides at ratios in [0.5, 2] to the first (before
    # rounding to whole cells), drop heights in
    # [0.05, 0.5] m, E log-uniform in [1e4, 1e6], nu in [0.2, 0.45], dt 1e-4
    ps = I.batch(512)
    assert len(ps) == 512
    E = np.array([p.n_elems for p in ps])
    assert E.sum() == 10_830_100  # the benchmark's batch (about 10.8 M tets)
    assert np.all(E % 5 == 0) and E.min() >= 5
    logE = np.log10(E)
    assert logE.min() > 2.5 and logE.max() < 5.1
    assert 3.7 < np.median(logE) < 4.3  # log-uniform on [3, 5]: median near 4
    for p in ps[:64]:
        ext = p.X.max(axis=0) - p.X.min(axis=0)
        cells = np.rint(ext / 0.025).astype(int)
        assert 5 * np.prod(cells) == p.n_elems
        a = cells[0]
        if a >= 3:  # b / a and c / a were drawn in [0.5, 2]; each side is rounded to whole cells
            for r in cells[1:] / a:
                assert (0.5 * (a - 0.5) - 0.5) / a - 1e-9 <= r <= (2.0 * (a + 0.5) + 0.5) / a + 1e-9, cells
        assert 0.05 <= p.X[:, 1].min() <= 0.5
        mu, lam = p.mu[0], p.lam[0]
        nu = lam / (2.0 * (lam + mu))
        Ey = 2.0 * mu * (1.0 + nu)
        assert 0.2 - 1e-12 <= nu <= 0.45 + 1e-12 and 1e4 * (1 - 1e-9) <= Ey <= 1e6 * (1 + 1e-9)
        assert p.dt == 1e-4 and p.steps == 300
    q = I.batch(4)
    assert all(np.array_equal(a.X, b.X) and np.array_equal(a.mu, b.mu) for a, b in zip(q, ps[:4]))


def test_query_stream_follows_its_recipe():
    # Poisson arrivals at the rate; half tet blocks (targets log-uniform in
    # [1e3, 2e5]), half cloth grids (32^2 .. 192^2); horizons in [100, 1000];
    # dt 1e-4; targets offset by N(0, 1 mm^2)
    rate, n = 200.0, 400
    qs = I.query_stream(rate, n, seed=1)
    t = np.array([q.t_arrival for q in qs])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0) and abs(gaps.mean() * rate - 1.0) < 0.15
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.2  # exponential gaps: coefficient of variation 1
    kinds = np.array([q.problem.kind for q in qs])
    assert 0.4 < (kinds == I.CLOTH).mean() < 0.6
    for q in qs:
        p = q.problem
        assert 100 <= p.steps <= 1000 and p.dt == 1e-4
        if p.kind == I.CLOTH:
            side = int(round(math.sqrt(p.n_nodes)))
            assert side * side == p.n_nodes and 32 <= side <= 192
            assert p.n_elems == 2 * (side - 1) ** 2
        else:
            assert p.n_elems % 5 == 0 and 1e3 / 3 < p.n_elems < 2e5 * 1.5
        assert q.target_offset.shape == (p.n_nodes, 3)
    off = np.concatenate([q.target_offset.ravel() for q in qs])
    assert abs(off.std() - 1e-3) < 2e-5 and abs(off.mean()) < 2e-5


def test_benchmark_workloads_follow_their_recipes():
    # block64: 1.6 m cube of 0.025 m cells on the ground; per-element E
    # log-uniform in [1e4, 1e6] and nu uniform in [0.2, 0.45]; v0 ~ N(0, 0.1^2)
    # per component; density 1000; 200 steps at dt 5e-5
    p = I.block(64)
    assert p.n_elems == 1_310_720 and p.n_nodes == 274_625 and p.steps == 200 and p.dt == 5e-5
    assert p.X[:, 1].min() == 0.0 and np.allclose(p.X.max(axis=0) - p.X.min(axis=0), 1.6)
    nu = p.lam / (2.0 * (p.lam + p.mu))
    Ey = 2.0 * p.mu * (1.0 + nu)
    assert nu.min() >= 0.2 - 1e-12 and nu.max() <= 0.45 + 1e-12 and abs(nu.mean() - 0.325) < 1e-3
    lE = np.log10(Ey)
    assert lE.min() >= 4 - 1e-9 and lE.max() <= 6 + 1e-9 and abs(lE.mean() - 5.0) < 2e-3
    assert abs(p.v0.std() - 0.1) < 1e-3 and abs(p.v0.mean()) < 1e-3
    assert np.all(p.rho == 1000.0) and p.contact.plane_on and not p.contact.sphere_on
    # bars 1a / 1b: 4^3 cells, E 1e5, nu 0.3, bottom face at 0.2 m / 0.02 m
    for v, drop in (("a", 0.2), ("b", 0.02)):
        b = I.bar(v)
        assert b.n_elems == 320 and abs(b.X[:, 1].min() - drop) < 1e-15 and b.dt == 1e-4 and b.steps == 1000
        mu, lam = I.lame(1e5, 0.3)
        assert np.allclose(b.mu, mu) and np.allclose(b.lam, lam) and np.all(b.rho == 1000.0)
        if b.v0 is not None:  # dropped from rest
            assert np.all(b.v0 == 0.0)
    # cloths 3 / 3s: 256^2 nodes over [0, 1]^2 at y = 0.305 above a 0.3 m sphere at (0.5, 0, 0.5)
    for v, mu, lam, kb in (("3", 5e3, 1e4, 1e-2), ("3s", 10.0, 20.0, 1e-6)):
        c = I.cloth(v)
        assert c.n_nodes == 65_536 and c.n_elems == 130_050 and c.n_hinges == 194_565 and c.steps == 500
        assert np.all(c.X[:, 1] == 0.305) and c.X[:, 0].min() == 0.0 and c.X[:, 0].max() == 1.0
        assert np.all(c.mu == mu) and np.all(c.lam == lam) and np.all(c.kb == kb) and np.all(c.rho == 0.2)
        assert c.contact.sphere_on and c.contact.sphere_r == 0.3 and tuple(c.contact.sphere_c) == (0.5, 0.0, 0.5)
