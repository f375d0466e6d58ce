"""Seeded synthetic inputs: meshes, materials and workload configurations.

This module builds the *inputs* of the differentiable explicit step (rest
positions, connectivity, per-element Lame parameters and densities, initial
state, contact and time-step settings).  It holds none of the method's own
arithmetic: no deformation gradients, no forces, no masses, no integration.
Both the CUDA path and the FP64 oracle consume what it produces, so nothing
here may depend on either of them.

Coordinates are y-up; the ground plane is y = h.  All randomness comes from
``numpy.random.default_rng(seed)``.

Workloads (the paper gives only "deformable objects of 100-10000 tets",
Sec. 3 "Timing analysis" / Table 4; these seeded meshes stand in for its
missing mesh datasets):

* ``bar``      4x4x4 hex cells of 0.025 m, 5 tets per cell (320 tets, 125 nodes),
               E = 1e5 Pa, nu = 0.3, density 1000, bottom face at 0.2 m ("1a")
               or 0.02 m ("1b"), dt = 1e-4, 1000 steps.
* ``block``    64^3 cells (1,310,720 tets, 274,625 nodes), E log-uniform in
               [1e4, 1e6] and nu uniform in [0.2, 0.45] per element, initial
               velocity N(0, 0.1^2) per component, bottom face on the ground,
               dt = 5e-5, 200 steps.
* ``cloth``    256^2 node grid over a 1 m square at y = 0.305 draped on a
               sphere of radius 0.3 centred at (0.5, 0, 0.5); "3" keeps the
               stated (explicitly unstable) materials, "3s" the stable variant.
* ``cloth_throw`` a small cloth (64-2048 triangles) thrown through air with
               lift/drag over the ground: the cloth-control episode.
* ``batch``    512 seeded a x b x c hex blocks, 1e3-1e5 tets each.
* ``queries``  a Poisson stream of tet-block / cloth-grid gradient queries.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

# ---------------------------------------------------------------------------
# hex block -> 5 tets per cell
# ---------------------------------------------------------------------------

# local corner c of a unit cell sits at offset (c & 1, (c >> 1) & 1, (c >> 2) & 1)
_CORNER = np.array([[c & 1, (c >> 1) & 1, (c >> 2) & 1] for c in range(8)], dtype=np.int64)

# Two mirror-image 5-tet splits.  Split 0: the central tet uses the corners
# whose offset sum is even and four corner tets cut off the odd corners;
# split 1 is the mirror.  Cells alternate by (ci + cj + ck) parity so that
# every face diagonal joins two nodes of even global parity: the mesh conforms.
_SPLIT = (
    [(0, 3, 5, 6), (1, 0, 3, 5), (2, 0, 3, 6), (4, 0, 5, 6), (7, 3, 5, 6)],
    [(1, 2, 4, 7), (0, 1, 2, 4), (3, 1, 2, 7), (5, 1, 4, 7), (6, 2, 4, 7)],
)


def _orient(template):
    """Order each template tet so its corner offsets have a positive triple product."""
    out = []
    for t in template:
        a, b, c, d = (_CORNER[i] for i in t)
        if int(np.dot(b - a, np.cross(c - a, d - a))) < 0:
            t = (t[0], t[1], t[3], t[2])
        out.append(t)
    return np.array(out, dtype=np.int64)


_SPLIT_ORIENTED = (_orient(_SPLIT[0]), _orient(_SPLIT[1]))


def hex_block(a: int, b: int, c: int, h: float, origin=(0.0, 0.0, 0.0)):
    """Structured block of a x b x c cubes of side ``h`` (a along x, b along y,
    c along z), each split into 5 tets.

    Returns ``(X, tets)``: rest positions float64 [N, 3] with
    N = (a+1)(b+1)(c+1) and tets int32 [5abc, 4], every tet positively
    oriented.  Cells are emitted in x-fastest order, 5 tets per cell.
    """
    i, j, k = np.meshgrid(np.arange(a + 1), np.arange(b + 1), np.arange(c + 1), indexing="ij")
    X = np.stack([i.T.ravel(), j.T.ravel(), k.T.ravel()], axis=1).astype(np.float64) * h
    X += np.asarray(origin, dtype=np.float64)

    ci, cj, ck = np.meshgrid(np.arange(a), np.arange(b), np.arange(c), indexing="ij")
    ci, cj, ck = ci.T.ravel(), cj.T.ravel(), ck.T.ravel()  # x fastest
    parity = (ci + cj + ck) & 1
    # node index of every local corner of every cell: [cells, 8]
    corner_nodes = ((ci[:, None] + _CORNER[None, :, 0])
                    + (a + 1) * ((cj[:, None] + _CORNER[None, :, 1])
                                 + (b + 1) * (ck[:, None] + _CORNER[None, :, 2])))
    tets = np.empty((ci.size, 5, 4), dtype=np.int64)
    for p in (0, 1):
        sel = parity == p
        tets[sel] = corner_nodes[sel][:, _SPLIT_ORIENTED[p]]
    return X, tets.reshape(-1, 4).astype(np.int32)


# ---------------------------------------------------------------------------
# cloth grid
# ---------------------------------------------------------------------------

def cloth_grid(n: int, side: float = 1.0, y0: float = 0.0, origin_xz=(0.0, 0.0)):
    """n x n node grid over a ``side`` square in the x-z plane at height ``y0``.

    Every cell is split by the same diagonal into triangles (a, b, d) and
    (a, d, c), so there are 2 (n-1)^2 triangles.  Returns
    ``(X, tris, hinges)``; each hinge is (x1, x2, x3, x4) with x3-x4 the
    interior edge and x1, x2 the opposite vertices of its two triangles,
    labelled so triangles (x1, x3, x4) and (x2, x4, x3) are consistently
    oriented.  Hinges are sorted by (min, max) edge node id.
    """
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    i, j = i.T.ravel(), j.T.ravel()  # node = i + n*j
    X = np.stack([origin_xz[0] + i * side / (n - 1),
                  np.full(i.shape, float(y0)),
                  origin_xz[1] + j * side / (n - 1)], axis=1).astype(np.float64)
    ci, cj = np.meshgrid(np.arange(n - 1), np.arange(n - 1), indexing="ij")
    ci, cj = ci.T.ravel(), cj.T.ravel()
    a = ci + n * cj
    b = a + 1
    c = a + n
    d = a + n + 1
    tris = np.empty((2 * a.size, 3), dtype=np.int64)
    tris[0::2] = np.stack([a, b, d], axis=1)
    tris[1::2] = np.stack([a, d, c], axis=1)
    hinges = _hinges(tris)
    return X, tris.astype(np.int32), hinges.astype(np.int32)


def _hinges(tris: np.ndarray) -> np.ndarray:
    """Interior edges of a consistently oriented triangle mesh as hinges."""
    # directed half-edges (p -> q) with the opposite vertex o
    p = np.concatenate([tris[:, 0], tris[:, 1], tris[:, 2]])
    q = np.concatenate([tris[:, 1], tris[:, 2], tris[:, 0]])
    o = np.concatenate([tris[:, 2], tris[:, 0], tris[:, 1]])
    lo, hi = np.minimum(p, q), np.maximum(p, q)
    key = lo.astype(np.int64) * (int(tris.max()) + 1) + hi
    order = np.argsort(key, kind="stable")
    key_s = key[order]
    same = np.nonzero(key_s[1:] == key_s[:-1])[0]  # pairs (same, same+1)
    h1, h2 = order[same], order[same + 1]
    # half-edge h1 runs p1 -> q1 inside a triangle (o1, p1, q1) oriented
    # o1 -> p1 -> q1; make x3 = p1, x4 = q1 so triangle (x1, x3, x4) keeps that
    # orientation; the partner half-edge runs q1 -> p1 in (o2, q1, p1) = (x2, x4, x3).
    out = np.stack([o[h1], o[h2], p[h1], q[h1]], axis=1)
    return out


# ---------------------------------------------------------------------------
# materials
# ---------------------------------------------------------------------------

def lame(E, nu):
    """Young's modulus and Poisson ratio -> Lame (mu, lambda), no re-parameterisation."""
    E = np.asarray(E, dtype=np.float64)
    nu = np.asarray(nu, dtype=np.float64)
    return E / (2.0 * (1.0 + nu)), E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))


# ---------------------------------------------------------------------------
# problem description shared by both sides
# ---------------------------------------------------------------------------

TET, CLOTH = 0, 1


@dataclasses.dataclass
class Contact:
    ke: float = 1.0e4
    kd: float = 10.0
    kf: float = 1.0
    mu_f: float = 0.5
    plane_on: bool = True
    plane_n: tuple = (0.0, 1.0, 0.0)
    plane_h: float = 0.0
    sphere_on: bool = False
    sphere_c: tuple = (0.0, 0.0, 0.0)
    sphere_r: float = 0.0


@dataclasses.dataclass
class Air:
    """Air on the cloth surface: drag and lift coefficients (kg/m^3, the
    factor 1/2 rho_air C of a flat plate) against a uniform wind (m/s)."""
    k_drag: float = 0.6
    k_lift: float = 0.4
    wind: tuple = (0.0, 0.0, 0.0)


@dataclasses.dataclass
class Problem:
    """One simulation instance: mesh, parameters, initial state, run length."""
    name: str
    kind: int                       # TET or CLOTH
    X: np.ndarray                   # rest positions [N, 3] float64
    elems: np.ndarray               # [E, 4] (tets) or [T, 3] (triangles) int32
    mu: np.ndarray                  # per element [E] float64
    lam: np.ndarray
    rho: np.ndarray                 # density (tets) or areal density (cloth)
    hinges: Optional[np.ndarray] = None   # [B, 4] int32 (cloth)
    kb: Optional[np.ndarray] = None       # [B] bending stiffness
    act: Optional[np.ndarray] = None      # [E] per-element actuation (default 0)
    hinge_act: Optional[np.ndarray] = None
    pinned: Optional[np.ndarray] = None   # [N] uint8, 1 = kinematic node
    x0: Optional[np.ndarray] = None       # initial positions [N, 3] (default X)
    v0: Optional[np.ndarray] = None       # initial velocities [N, 3] (default 0)
    contact: Contact = dataclasses.field(default_factory=Contact)
    gravity: tuple = (0.0, -9.81, 0.0)
    dt: float = 1.0e-4
    steps: int = 100
    air: Optional[Air] = None             # cloth only: lift/drag air model

    def __post_init__(self):
        if self.x0 is None:
            self.x0 = self.X.copy()
        if self.v0 is None:
            self.v0 = np.zeros_like(self.X)

    @property
    def n_nodes(self):
        return int(self.X.shape[0])

    @property
    def n_elems(self):
        return int(self.elems.shape[0])

    @property
    def n_hinges(self):
        return 0 if self.hinges is None else int(self.hinges.shape[0])


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

def bar(variant: str = "a", steps: int = 1000, cells=(4, 4, 4), h: float = 0.025) -> Problem:
    """Tet bar of 4x4x4 cells (E = 1e5, nu = 0.3, rho = 1000) dropped on the ground.

    variant "a": bottom face at 0.2 m (1000 steps at dt 1e-4 never reach the
    ground); "b": bottom face at 0.02 m (impact near step 640).
    """
    drop = {"a": 0.2, "b": 0.02}[variant]
    X, tets = hex_block(*cells, h=h, origin=(0.0, drop, 0.0))
    mu, lam = lame(1.0e5, 0.3)
    E = tets.shape[0]
    return Problem(name=f"bar1{variant}", kind=TET, X=X, elems=tets,
                   mu=np.full(E, float(mu)), lam=np.full(E, float(lam)),
                   rho=np.full(E, 1000.0), contact=Contact(), dt=1.0e-4, steps=steps)


def block(n: int = 64, steps: int = 200, seed: int = 0, h: float = 0.025) -> Problem:
    """n^3-cell tet block on the ground with heterogeneous materials and a
    random initial velocity field (n = 64 gives 1,310,720 tets)."""
    rng = np.random.default_rng(seed)
    X, tets = hex_block(n, n, n, h=h)
    E = tets.shape[0]
    Ey = np.exp(rng.uniform(math.log(1e4), math.log(1e6), E))
    nu = rng.uniform(0.2, 0.45, E)
    mu, lam = lame(Ey, nu)
    v0 = rng.normal(0.0, 0.1, X.shape)
    return Problem(name=f"block{n}", kind=TET, X=X, elems=tets, mu=mu, lam=lam,
                   rho=np.full(E, 1000.0), v0=v0, contact=Contact(), dt=5.0e-5, steps=steps)


def cloth(variant: str = "3s", n: int = 256, steps: int = 500, grid_scaled: bool = False,
          height: float = 0.305) -> Problem:
    """n x n cloth over [0,1]^2 at y = `height` (0.305: 5 mm above the top of
    the sphere, which it reaches near step 320; below 0.3 the sphere touches
    it from step 0) draped on a sphere (r 0.3 at (0.5, 0, 0.5)).

    "3": mu = 5e3, lambda = 1e4, kb = 1e-2, areal density 0.2, ke = 1e4,
    kd = 10, kf = 1 -- explicitly unstable at dt = 1e-4 (tiny node masses).
    "3s": mu = 10, lambda = 20, kb = 1e-6, ke = 100, kd = 1e-3, kf = 1e-3.
    ``grid_scaled`` multiplies the stiffnesses by ((255/(n-1))^2), the ratio
    of node masses, so a coarser grid keeps the 256^2 grid's time scales.
    """
    X, tris, hinges = cloth_grid(n, 1.0, height)
    T, B = tris.shape[0], hinges.shape[0]
    sc = (255.0 / (n - 1)) ** 2 if grid_scaled else 1.0
    if variant == "3":
        mu, lam, kb = 5.0e3 * sc, 1.0e4 * sc, 1.0e-2 * sc
        con = Contact(ke=1.0e4 * sc, kd=10.0 * sc, kf=1.0 * sc, mu_f=0.5)
    elif variant == "3s":
        mu, lam, kb = 10.0 * sc, 20.0 * sc, 1.0e-6 * sc
        con = Contact(ke=100.0 * sc, kd=1.0e-3 * sc, kf=1.0e-3 * sc, mu_f=0.5)
    else:
        raise ValueError(variant)
    con.plane_on, con.plane_h = True, 0.0
    con.sphere_on, con.sphere_c, con.sphere_r = True, (0.5, 0.0, 0.5), 0.3
    return Problem(name=f"cloth{variant}_{n}", kind=CLOTH, X=X, elems=tris,
                   mu=np.full(T, mu), lam=np.full(T, lam), rho=np.full(T, 0.2),
                   hinges=hinges, kb=np.full(B, kb), contact=con, dt=1.0e-4, steps=steps)


def cloth_throw(n: int = 12, steps: int = 400, seed: int = 0, air: Optional["Air"] = None,
                side: float = 0.5) -> Problem:
    """The cloth-control episode of Sec. 3 (a cloth of 64-2048 triangles sent
    towards a goal by its initial velocity, under lift/drag): an n x n grid
    (2 (n-1)^2 triangles, n in 7..33) of side ``side`` at 0.4 m, tilted by a
    seeded angle, thrown with a seeded common velocity plus a small per-node
    spread, over the ground plane.  Materials of "3s" scaled to the grid.
    """
    rng = np.random.default_rng(seed)
    X, tris, hinges = cloth_grid(n, side, 0.0)
    # tilt about the x axis through the centre, then lift to 0.4 m
    a = rng.uniform(-0.5, 0.5)
    c0 = X.mean(axis=0)
    R = np.array([[1.0, 0.0, 0.0], [0.0, math.cos(a), -math.sin(a)], [0.0, math.sin(a), math.cos(a)]])
    X = (X - c0) @ R.T + np.array([0.5, 0.4, 0.5])
    T, B = tris.shape[0], hinges.shape[0]
    sc = (255.0 / (n - 1)) ** 2 * side ** 2  # node masses relative to the 256^2 unit cloth
    mu, lam, kb = 10.0 * sc, 20.0 * sc, 1.0e-6 * sc
    con = Contact(ke=100.0 * sc, kd=1.0e-3 * sc, kf=1.0e-3 * sc, mu_f=0.5)
    v_common = np.array([rng.uniform(-1.0, 1.0), rng.uniform(0.5, 1.5), rng.uniform(-1.0, 1.0)])
    v0 = v_common + rng.normal(0.0, 0.05, X.shape)
    return Problem(name=f"cloth_throw{n}", kind=CLOTH, X=X, elems=tris,
                   mu=np.full(T, mu), lam=np.full(T, lam), rho=np.full(T, 0.2),
                   hinges=hinges, kb=np.full(B, kb), v0=v0, contact=con, dt=1.0e-4, steps=steps,
                   air=Air() if air is None else air)


# ---------------------------------------------------------------------------
# rendering inputs: cameras, surface triangles, vertex colours
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Camera:
    """Pinhole camera: x_cam = R x + t (camera looks along +z_cam, y_cam down
    the image), pixel (u, v) = (fx x_cam/z_cam + cx, fy y_cam/z_cam + cy);
    pixel (i, j) has its centre at (i + 0.5, j + 0.5).  Depths are normalised
    over [z_near, z_far]."""
    R: np.ndarray          # [3, 3] world -> camera rotation
    t: np.ndarray          # [3]
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    z_near: float = 0.05
    z_far: float = 10.0


def look_at(eye, target, up=(0.0, 1.0, 0.0), width=256, height=256, fov_deg=40.0, z_near=0.05,
            z_far=10.0) -> Camera:
    """Camera at `eye` looking at `target` with `up` towards the image top."""
    eye, target, up = (np.asarray(a, dtype=np.float64) for a in (eye, target, up))
    f = target - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, up)
    r /= np.linalg.norm(r)
    d = np.cross(f, r)  # image down
    R = np.stack([r, d, f])
    t = -R @ eye
    fl = 0.5 * width / math.tan(math.radians(fov_deg) / 2)
    return Camera(R=R, t=t, fx=fl, fy=fl, cx=width / 2, cy=height / 2, width=width, height=height,
                  z_near=z_near, z_far=z_far)


def surface_faces(tets: np.ndarray) -> np.ndarray:
    """Boundary triangles of a tet mesh (faces used by one tet), oriented
    with the outward normal by the right-hand rule, in a fixed order (sorted
    by owning tet, then face)."""
    tets = np.asarray(tets, dtype=np.int64)
    loc = np.array([[1, 2, 3], [0, 3, 2], [0, 1, 3], [0, 2, 1]])  # outward for positively oriented tets
    faces = tets[:, loc].reshape(-1, 3)
    key = np.sort(faces, axis=1)
    _, inv, cnt = np.unique(key, axis=0, return_inverse=True, return_counts=True)
    return faces[cnt[inv.ravel()] == 1].astype(np.int32)


def vertex_colours(X: np.ndarray, seed: int = 0) -> np.ndarray:
    """Seeded smooth per-vertex RGB in [0.1, 0.9] (a colour field over the
    rest shape, so that shading carries positional information)."""
    rng = np.random.default_rng(seed)
    W = rng.normal(size=(3, 3))
    ph = rng.uniform(0.0, 2.0 * math.pi, 3)
    span = np.ptp(X, axis=0).max() or 1.0
    return 0.5 + 0.4 * np.sin(((X - X.min(axis=0)) / span) @ W * 3.0 + ph)


@dataclasses.dataclass
class RenderSpec:
    """Soft rasteriser settings: sigma (pixel^2) sets the width of the soft
    edges, gamma the depth softmax temperature, eps the background's
    normalised depth, bg its colour."""
    sigma: float = 0.5
    gamma: float = 1.0e-3
    eps: float = 1.0e-3
    bg: tuple = (1.0, 1.0, 1.0)


# ---------------------------------------------------------------------------
# rigid bodies
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class RigidBody:
    """A rigid body: contact points and surface triangles in the body frame
    (about the centre of mass), mass, body-frame inertia (Ixx, Iyy, Izz, Ixy,
    Ixz, Iyz), contact parameters (ke, kd, kf, mu), the initial state
    (x, quaternion (w, x, y, z), v, omega) and the scene it moves in."""
    name: str
    points: np.ndarray
    faces: np.ndarray
    mass: float
    inertia: tuple
    contact: tuple
    state0: np.ndarray
    scene: Contact = dataclasses.field(default_factory=lambda: Contact(plane_on=True))
    gravity: tuple = (0.0, -9.81, 0.0)
    dt: float = 1.0e-3
    steps: int = 200


def box_points(size, n: int = 2):
    """Points of an n x n x n lattice on the surface of a box of `size` centred
    at the origin (n = 2: the 8 corners), and the box's 12 surface triangles
    over its corners (indices into the first 8 points, which are the
    corners)."""
    a = np.asarray(size, dtype=np.float64) / 2
    corners = np.array([[sx, sy, sz] for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1)], dtype=np.float64) * a
    pts = [corners]
    if n > 2:
        g = np.linspace(-1.0, 1.0, n)
        lat = np.array([[i, j, k] for i in g for j in g for k in g])
        on_surface = np.isclose(np.abs(lat), 1.0).any(axis=1)
        is_corner = np.isclose(np.abs(lat), 1.0).all(axis=1)
        pts.append(lat[on_surface & ~is_corner] * a)
    # corner index = 4 (x > 0) + 2 (y > 0) + (z > 0); outward-wound faces
    quads = [(0, 1, 3, 2), (4, 6, 7, 5), (0, 4, 5, 1), (2, 3, 7, 6), (0, 2, 6, 4), (1, 5, 7, 3)]
    faces = np.array([t for q in quads for t in ((q[0], q[1], q[2]), (q[0], q[2], q[3]))], dtype=np.int32)
    return np.vstack(pts), faces


def box_body(size=(0.2, 0.2, 0.2), density=125.0, n: int = 2, contact=(1.0e4, 10.0, 100.0, 0.5),
             x0=(0.0, 0.5, 0.0), q0=(1.0, 0.0, 0.0, 0.0), v0=(0.0, 0.0, 0.0), w0=(0.0, 0.0, 0.0),
             dt: float = 1.0e-3, steps: int = 200, name: str = "box") -> RigidBody:
    """A solid box: mass = density x volume, inertia m/12 (b^2 + c^2, ...)
    about its centre."""
    pts, faces = box_points(size, n)
    a, b, c = size
    m = density * a * b * c
    I = (m / 12 * (b * b + c * c), m / 12 * (a * a + c * c), m / 12 * (a * a + b * b), 0.0, 0.0, 0.0)
    q = np.asarray(q0, dtype=np.float64)
    q = q / np.linalg.norm(q)
    state0 = np.concatenate([x0, q, v0, w0]).astype(np.float64)
    return RigidBody(name=name, points=pts, faces=faces, mass=m, inertia=I, contact=tuple(contact), state0=state0,
                     dt=dt, steps=steps)


def rigid_batch(n_bodies: int = 1024, seed: int = 0, n: int = 5, steps: int = 300) -> List[RigidBody]:
    """Seeded boxes in the ranges of the paper's rigid experiments (App. E:
    densities 2-12 kg/m^3 of boxes up to ~2 m, friction coefficient 0.2-1.0,
    random poses and velocities).  The paper's contact stiffnesses (1-500)
    are in unstated units; here k_e makes four corners rest 1 mm deep,
    k_d damps at 0.3 of critical, and k_f is 1-500 x m/100 N s/m so that
    explicit Euler at dt 1e-3 stays stable with a whole face (n^2 points) in
    contact.  n x n x n surface lattice points."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_bodies):
        size = tuple(rng.uniform(0.5, 2.0, 3))
        dens = rng.uniform(2.0, 12.0)
        m = dens * size[0] * size[1] * size[2]
        ke = m * 9.81 / 4 / 1e-3
        kd = 2.0 * math.sqrt(ke * m / 4) * 0.3
        kf = rng.uniform(1.0, 500.0) * m / 100.0
        mu = rng.uniform(0.2, 1.0)
        ax = rng.normal(size=3)
        ang = rng.uniform(0, math.pi)
        q0 = np.concatenate([[math.cos(ang / 2)], math.sin(ang / 2) * ax / np.linalg.norm(ax)])
        x0 = (rng.uniform(-6.5, 6.5), rng.uniform(1.5, 3.0), rng.uniform(-6.5, 6.5))
        v0 = rng.uniform(-2.0, 2.0, 3)
        w0 = rng.uniform(-3.0, 3.0, 3)
        out.append(box_body(size, dens, n=n, contact=(ke, kd, kf, mu), x0=x0, q0=q0, v0=v0, w0=w0, steps=steps,
                            name=f"box{i}"))
    return out


def hanging_beam(mu: float = 1000.0, steps: int = 300, cells=(8, 2, 2), h: float = 0.025,
                 density: float = 100.0, dt: float = 1.0e-3) -> Problem:
    """The beam of the paper's deformable loss landscape (Sec. 3: a beam
    hanging under gravity, Lame parameters mu = lambda = 1000): an 8 x 2 x 2
    cell tet beam of 0.025 m cells, pinned at its x = 0 face, mu = lambda =
    `mu`, density 100 kg/m^3, no ground."""
    X, tets = hex_block(*cells, h=h, origin=(0.0, 0.5, 0.0))
    E = tets.shape[0]
    pin = (X[:, 0] < 1e-9).astype(np.uint8)
    return Problem(name="hanging_beam", kind=TET, X=X, elems=tets, mu=np.full(E, float(mu)),
                   lam=np.full(E, float(mu)), rho=np.full(E, density), pinned=pin,
                   contact=Contact(plane_on=False), dt=dt, steps=steps)


def block_dims(n_tets_target: float, rng) -> tuple:
    """Integer a x b x c (>= 1) with aspect ratios in [0.5, 2] and 5abc ~ target."""
    r1, r2 = np.exp(rng.uniform(math.log(0.5), math.log(2.0), 2))
    s = (n_tets_target / 5.0 / (r1 * r2)) ** (1.0 / 3.0)
    return (max(1, int(round(s))), max(1, int(round(s * r1))), max(1, int(round(s * r2))))


def batch_member(mesh_id: int, steps: int = 300, lo: float = 1e3, hi: float = 1e5,
                 seed: int = 0) -> Problem:
    """One mesh of the heterogeneous batch, seeded by (seed, mesh_id)."""
    rng = np.random.default_rng([seed, mesh_id])
    target = math.exp(rng.uniform(math.log(lo), math.log(hi)))
    a, b, c = block_dims(target, rng)
    drop = rng.uniform(0.05, 0.5)
    Ey = math.exp(rng.uniform(math.log(1e4), math.log(1e6)))
    nu = rng.uniform(0.2, 0.45)
    X, tets = hex_block(a, b, c, h=0.025, origin=(0.0, drop, 0.0))
    mu, lam = lame(Ey, nu)
    E = tets.shape[0]
    return Problem(name=f"batch{mesh_id}", kind=TET, X=X, elems=tets,
                   mu=np.full(E, float(mu)), lam=np.full(E, float(lam)), rho=np.full(E, 1000.0),
                   contact=Contact(), dt=1.0e-4, steps=steps)


def batch(n_meshes: int = 512, steps: int = 300, seed: int = 0, lo: float = 1e3,
          hi: float = 1e5) -> List[Problem]:
    return [batch_member(i, steps=steps, lo=lo, hi=hi, seed=seed) for i in range(n_meshes)]


def position_noise(n_nodes: int, sigma: float = 1.0e-3, seed: int = 0) -> np.ndarray:
    """Seeded N(0, sigma^2) offsets added to a reference final state to form a target."""
    return np.random.default_rng(seed).normal(0.0, sigma, (n_nodes, 3))


@dataclasses.dataclass
class Query:
    """One system-identification gradient query of the serving workload."""
    qid: int
    t_arrival: float
    problem: Problem
    target_offset: np.ndarray


def query_stream(rate: float, n: int, seed: int = 0, tet_range=(1e3, 2e5),
                 cloth_range=(32, 192), horizon=(100, 1000)) -> List[Query]:
    """Poisson arrivals at ``rate`` req/s; half tet blocks, half cloth grids."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for qid in range(n):
        t += rng.exponential(1.0 / rate)
        steps = int(rng.integers(horizon[0], horizon[1] + 1))
        if rng.uniform() < 0.5:
            target = math.exp(rng.uniform(math.log(tet_range[0]), math.log(tet_range[1])))
            a, b, c = block_dims(target, rng)
            drop = rng.uniform(0.05, 0.5)
            Ey = math.exp(rng.uniform(math.log(1e4), math.log(1e6)))
            nu = rng.uniform(0.2, 0.45)
            X, tets = hex_block(a, b, c, h=0.025, origin=(0.0, drop, 0.0))
            mu, lam = lame(Ey, nu)
            E = tets.shape[0]
            p = Problem(name=f"q{qid}", kind=TET, X=X, elems=tets, mu=np.full(E, float(mu)),
                        lam=np.full(E, float(lam)), rho=np.full(E, 1000.0), dt=1.0e-4, steps=steps)
        else:
            m = int(rng.integers(cloth_range[0], cloth_range[1] + 1))
            X, tris, hinges = cloth_grid(m, 1.0, 0.305)
            # the stable "3s" materials scaled with the grid spacing (node mass ~ h^2)
            scale = (255.0 / (m - 1)) ** 2
            T, B = tris.shape[0], hinges.shape[0]
            con = Contact(ke=100.0 * scale, kd=1.0e-3 * scale, kf=1.0e-3 * scale, mu_f=0.5,
                          plane_on=True, plane_h=0.0, sphere_on=True,
                          sphere_c=(0.5, 0.0, 0.5), sphere_r=0.3)
            p = Problem(name=f"q{qid}", kind=CLOTH, X=X, elems=tris,
                        mu=np.full(T, 10.0 * scale), lam=np.full(T, 20.0 * scale),
                        rho=np.full(T, 0.2), hinges=hinges, kb=np.full(B, 1.0e-6 * scale),
                        contact=con, dt=1.0e-4, steps=steps)
        out.append(Query(qid=qid, t_arrival=t, problem=p,
                         target_offset=rng.normal(0.0, 1.0e-3, (p.n_nodes, 3))))
    return out
