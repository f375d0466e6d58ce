"""Pins of the soft-rasteriser oracle (Sec. 2 "Differentiable rendering
engine": SoftRas-style sigmoid edges, DIB-R-style barycentric interpolation;
the reading is stated in oracle/render_oracle.py).

Pinned against geometry and closed forms rather than the oracle's own
formulas: the look-at camera's image of known points and of its field of
view; hard coverage in the sharp limit against exact point-in-triangle tests
on an integer triangle; area preservation of the soft edges; the value on an
edge and at a known distance outside; the probabilistic union of coverages;
the nearest triangle winning the depth softmax; exact reproduction of an
affine colour field; perspective-correct depth against a ray-plane
intersection, both in the interpolated attributes and in the depth softmax's
blend; and the autograd gradients against central differences.
"""
import math

import numpy as np
import torch

from oracle import render_oracle as R
from paper_2104_02646_gb300 import inputs as I


def _cam(w=32, h=24):
    return I.look_at((0.0, 0.0, -2.0), (0.0, 0.0, 0.0), width=w, height=h, fov_deg=60.0)


def _screen_to_world(cam, u, v, depth):
    """World point that projects to (u, v) at camera depth `depth` (inverse of
    the pinhole model, written from the camera axes)."""
    xc = np.array([(u - cam.cx) / cam.fx * depth, (v - cam.cy) / cam.fy * depth, depth])
    return cam.R.T @ (xc - cam.t)


def test_look_at_camera_geometry():
    cam = I.look_at((1.0, 2.0, -3.0), (0.2, 0.1, 0.4), width=64, height=48, fov_deg=50.0)
    u, v, z = R.project(torch.tensor([[0.2, 0.1, 0.4]], dtype=torch.float64), cam)
    assert abs(u.item() - 32.0) < 1e-12 and abs(v.item() - 24.0) < 1e-12
    assert abs(z.item() - math.dist((1.0, 2.0, -3.0), (0.2, 0.1, 0.4))) < 1e-12
    # a point at half the horizontal field of view lands on the image edge
    eye = np.array([1.0, 2.0, -3.0])
    f = np.array([0.2, 0.1, 0.4]) - eye
    f /= np.linalg.norm(f)
    right = np.cross(f, [0.0, 1.0, 0.0])
    right /= np.linalg.norm(right)
    up = np.cross(right, f)
    ang = math.radians(25.0)
    p_right = eye + 2.0 * (math.cos(ang) * f + math.sin(ang) * right)
    p_up = eye + 2.0 * (f + math.tan(ang) * 48 / 64 * up)
    u, v, _ = R.project(torch.tensor(np.stack([p_right, p_up])), cam)
    assert abs(u[0].item() - 64.0) < 1e-9 and abs(v[0].item() - 24.0) < 1e-9
    assert abs(u[1].item() - 32.0) < 1e-9 and abs(v[1].item() - 0.0) < 1e-9  # up is the image top


def _tri_scene(cam, pts2d, depth=2.0, colours=None):
    X = np.stack([_screen_to_world(cam, u, v, depth) for (u, v) in pts2d])
    col = np.tile([0.2, 0.4, 0.6], (len(pts2d), 1)) if colours is None else colours
    return X, np.array([[0, 1, 2]]), col


def test_sharp_limit_is_exact_coverage():
    cam = _cam(32, 32)
    pts = [(3.0, 4.0), (27.0, 9.0), (11.0, 29.0)]
    X, F, col = _tri_scene(cam, pts)
    # every half-integer pixel centre is >= ~0.01 px from these edges, so
    # sigma = 1e-7 px^2 makes each coverage 0 or 1 - Q_MIN
    img = R.render(X, F, col, cam, I.RenderSpec(sigma=1e-7)).numpy()
    (ax, ay), (bx, by), (cx, cy) = pts

    def side(px, py, x0, y0, x1, y1):  # exact for these half-integer centres
        return (x1 - x0) * (py - y0) - (y1 - y0) * (px - x0)

    n = 0
    for j in range(32):
        for i in range(32):
            px, py = i + 0.5, j + 0.5
            s = [side(px, py, ax, ay, bx, by), side(px, py, bx, by, cx, cy), side(px, py, cx, cy, ax, ay)]
            assert all(t != 0 for t in s)
            ins = all(t > 0 for t in s) or all(t < 0 for t in s)
            assert abs(img[j, i, 3] - (1.0 if ins else 0.0)) <= 2 * R.Q_MIN, (i, j)  # 1 - coverage >= Q_MIN
            n += ins
    assert n > 100


def test_soft_edges_preserve_area():
    cam = _cam(64, 64)
    pts = [(10.0, 12.0), (55.0, 20.0), (25.0, 54.0)]
    X, F, col = _tri_scene(cam, pts)
    area = 0.5 * abs((pts[1][0] - pts[0][0]) * (pts[2][1] - pts[0][1]) - (pts[2][0] - pts[0][0]) * (pts[1][1] - pts[0][1]))
    for sigma in (0.3, 1.0):
        A = R.render(X, F, col, cam, I.RenderSpec(sigma=sigma)).numpy()[..., 3]
        assert abs(A.sum() - area) < 0.01 * area, (sigma, A.sum(), area)


def test_edge_value_and_known_distance():
    cam = _cam(16, 16)
    # horizontal edge through pixel centres' row y = 8.5, from x = 1 to 15
    X, F, col = _tri_scene(cam, [(1.0, 8.5), (15.0, 8.5), (8.0, 15.0)])
    sigma = 0.7
    A = R.render(X, F, col, cam, I.RenderSpec(sigma=sigma)).numpy()[..., 3]
    assert abs(A[8, 8] - 0.5) < 1e-9
    for dy in (1, 2):  # rows above the edge, feet of the perpendiculars inside it
        d = float(dy)
        expected = 1.0 / (1.0 + math.exp(d * d / sigma))
        if expected < R.TAU:
            expected = 0.0
        assert abs(A[8 - dy, 8] - expected) < 1e-9, (dy, A[8 - dy, 8], expected)


def test_union_of_coverages():
    cam = _cam(24, 24)
    pa = [(2.0, 3.0), (20.0, 4.0), (6.0, 21.0)]
    pb = [(21.0, 20.0), (4.0, 18.0), (15.0, 2.0)]
    Xa, F, col = _tri_scene(cam, pa, 2.0)
    Xb, _, _ = _tri_scene(cam, pb, 2.5)
    spec = I.RenderSpec(sigma=2.0)
    Aa = R.render(Xa, F, col, cam, spec).numpy()[..., 3]
    Ab = R.render(Xb, F, col, cam, spec).numpy()[..., 3]
    Aab = R.render(np.vstack([Xa, Xb]), np.array([[0, 1, 2], [3, 4, 5]]), np.vstack([col, col]), cam, spec).numpy()[..., 3]
    # away from the clamp (deep overlaps clamp 1 - coverage at Q_MIN)
    ok = (1 - Aa > 1e-5) & (1 - Ab > 1e-5)
    np.testing.assert_allclose(Aab[ok], (1 - (1 - Aa) * (1 - Ab))[ok], rtol=0, atol=1e-12)


def test_nearest_triangle_wins_the_depth_softmax():
    cam = _cam(16, 16)
    pts = [(1.0, 1.0), (15.0, 2.0), (4.0, 15.0)]
    Xn, F, _ = _tri_scene(cam, pts, 1.5)
    Xf, _, _ = _tri_scene(cam, [(15.0, 15.0), (1.0, 14.0), (12.0, 1.0)], 3.0)
    red, green = np.tile([1.0, 0.0, 0.0], (3, 1)), np.tile([0.0, 1.0, 0.0], (3, 1))
    spec = I.RenderSpec(sigma=0.3, gamma=1e-3, bg=(0.0, 0.0, 1.0))
    for near_col, far_col in ((red, green), (green, red)):
        img = R.render(np.vstack([Xn, Xf]), np.array([[0, 1, 2], [3, 4, 5]]), np.vstack([near_col, far_col]), cam,
                       spec).numpy()
        # pixel (7, 7) lies deep inside both triangles
        np.testing.assert_allclose(img[7, 7, :3], near_col[0], atol=1e-6)
        # a pixel far outside both shows the background
        img2 = R.render(Xn, F, near_col, cam, spec).numpy()
        np.testing.assert_allclose(img2[14, 14, :3], spec.bg, atol=1e-9)


def test_affine_colour_field_is_reproduced():
    cam = _cam(32, 32)
    pts = [(2.0, 2.0), (30.0, 5.0), (8.0, 30.0)]
    G = np.array([[0.01, -0.02, 0.015], [0.02, 0.01, -0.01]])
    c0 = np.array([0.3, 0.5, 0.2])
    col = np.array([c0 + np.array(p) @ G for p in pts])
    X, F, _ = _tri_scene(cam, pts, 2.0, col)
    img = R.render(X, F, col, cam, I.RenderSpec(sigma=0.05, gamma=1e-4)).numpy()
    for (i, j) in [(10, 10), (15, 12), (8, 20)]:
        np.testing.assert_allclose(img[j, i, :3], c0 + np.array([i + 0.5, j + 0.5]) @ G, atol=1e-9)


def test_depth_is_perspective_correct():
    # a slanted triangle: the depth interpolated at a pixel (read through the
    # colour channel with colours 1/z_k, interpolated like 1/z) equals the
    # depth where that pixel's ray meets the triangle's plane
    cam = _cam(32, 32)
    X = np.array([[-0.6, -0.5, 0.3], [0.7, -0.4, -0.4], [0.0, 0.6, 0.9]])
    _, _, z = R.project(torch.tensor(X), cam)
    iz = 1.0 / z.numpy()
    spec = I.RenderSpec(sigma=0.05, gamma=1e-4, bg=(0.0, 0.0, 0.0))
    img = R.render(X, np.array([[0, 1, 2]]), np.tile(iz[:, None], (1, 3)), cam, spec).numpy()
    n = np.cross(X[1] - X[0], X[2] - X[0])
    eye = -cam.R.T @ cam.t
    for (i, j) in [(16, 16), (12, 19), (17, 17), (9, 21)]:
        assert img[j, i, 3] > 1 - 2 * R.Q_MIN  # deep inside
        dc = np.array([(i + 0.5 - cam.cx) / cam.fx, (j + 0.5 - cam.cy) / cam.fy, 1.0])
        d = cam.R.T @ dc
        depth = np.dot(n, X[0] - eye) / np.dot(n, d)  # camera depth of eye + s d is s (dc has unit z)
        assert abs(1.0 / img[j, i, 0] - depth) < 1e-6 * depth, (i, j, 1.0 / img[j, i, 0], depth)


def test_depth_softmax_uses_perspective_correct_depth():
    # a slanted triangle (red) over a fronto-parallel one (green) at a depth
    # between its corners' depths; with sharp edges (coverage 1 - Q_MIN deep
    # inside) each pixel's colour is the closed-form softmax over the two
    # triangles' normalised depths, taken where the pixel's ray meets each
    # plane.  Depth interpolated affinely in the screen would give a visibly
    # different blend, which the last check shows.
    cam = _cam(32, 32)
    S = np.stack([_screen_to_world(cam, u, v, d) for (u, v, d) in [(2.0, 2.0, 1.0), (30.0, 3.0, 3.0), (16.0, 30.0, 2.0)]])
    P, _, _ = _tri_scene(cam, [(-20.0, -20.0), (60.0, -20.0), (-20.0, 60.0)], 1.9)
    red, green = np.tile([1.0, 0.0, 0.0], (3, 1)), np.tile([0.0, 1.0, 0.0], (3, 1))
    spec = I.RenderSpec(sigma=1e-4, gamma=0.01, bg=(0.0, 0.0, 0.0))
    img = R.render(np.vstack([S, P]), np.array([[0, 1, 2], [3, 4, 5]]), np.vstack([red, green]), cam, spec).numpy()
    n = np.cross(S[1] - S[0], S[2] - S[0])
    eye = -cam.R.T @ cam.t
    uvS = np.array([(2.0, 2.0), (30.0, 3.0), (16.0, 30.0)])
    zS = np.array([1.0, 3.0, 2.0])
    D = 1.0 - R.Q_MIN
    zh = lambda z: (cam.z_far - z) / (cam.z_far - cam.z_near)

    def red_of(z_s):
        a, b, e = np.exp(zh(z_s) / spec.gamma), np.exp(zh(1.9) / spec.gamma), np.exp(spec.eps / spec.gamma)
        return D * a / (D * a + D * b + e)

    for (i, j) in [(16, 12), (13, 9), (20, 13), (15, 18)]:
        p = np.array([i + 0.5, j + 0.5])
        # screen-space barycentrics of the pixel in the slanted triangle (inside, away from the edges)
        T = np.array([[uvS[0, 0] - uvS[2, 0], uvS[1, 0] - uvS[2, 0]], [uvS[0, 1] - uvS[2, 1], uvS[1, 1] - uvS[2, 1]]])
        l01 = np.linalg.solve(T, p - uvS[2])
        w = np.array([l01[0], l01[1], 1.0 - l01.sum()])
        assert (w > 0.05).all()
        dc = np.array([(p[0] - cam.cx) / cam.fx, (p[1] - cam.cy) / cam.fy, 1.0])
        z_ray = np.dot(n, S[0] - eye) / np.dot(n, cam.R.T @ dc)
        assert abs(1.0 / np.dot(w, 1.0 / zS) - z_ray) < 1e-9 * z_ray  # the same depth, by screen barycentrics
        np.testing.assert_allclose(img[j, i, 0], red_of(z_ray), rtol=0, atol=1e-9)
        np.testing.assert_allclose(img[j, i, 1], 1.0 - red_of(z_ray) - (img[j, i, 2]), rtol=0, atol=1e-9)
        assert abs(red_of(np.dot(w, zS)) - red_of(z_ray)) > 1e-2  # the affine depth's blend is far off


def test_gradients_match_finite_differences():
    cam = _cam(16, 12)
    rng = np.random.default_rng(3)
    X = np.vstack([_screen_to_world(cam, *rng.uniform(0, 16, 2), rng.uniform(1.5, 2.5)) for _ in range(5)])
    F = np.array([[0, 1, 2], [1, 3, 2], [2, 3, 4]])
    col = rng.uniform(0.1, 0.9, (5, 3))
    spec = I.RenderSpec(sigma=1.5, gamma=0.05)
    dimg = rng.normal(size=(12, 16, 4))
    img, gx, gc = R.render_grad(X, F, col, cam, spec, dimg)

    def L(Xp, cp):
        return float((R.render(Xp, F, cp, cam, spec) * torch.tensor(dimg)).sum())

    h = 1e-6
    for (k, c) in [(0, 0), (1, 2), (3, 1), (4, 0), (2, 2)]:
        Xp, Xm = X.copy(), X.copy()
        Xp[k, c] += h
        Xm[k, c] -= h
        fd = (L(Xp, col) - L(Xm, col)) / (2 * h)
        assert abs(fd - gx[k, c].item()) <= 1e-6 * max(1.0, abs(fd)), (k, c, fd, gx[k, c].item())
    for (k, c) in [(0, 1), (3, 2)]:
        cp, cm = col.copy(), col.copy()
        cp[k, c] += h
        cm[k, c] -= h
        fd = (L(X, cp) - L(X, cm)) / (2 * h)
        assert abs(fd - gc[k, c].item()) <= 1e-6 * max(1.0, abs(fd))
