"""FP64 CPU oracle of the differentiable soft rasteriser (test infrastructure
only: the tests, the package smoke check and the benchmark's CPU legs use it;
the library never does).

Sec. 2 "Differentiable rendering engine" of the paper renders the simulated
meshes with SoftRas and DIB-R, which replace the hard edges of rasterised
triangles by sigmoids so that the image is differentiable in the vertex
positions; DIB-R interpolates vertex attributes with differentiable
barycentric weights.  The paper prints no formulas for either, so this module
states one reading and computes it by brute force over every (pixel,
triangle) pair in plain PyTorch CPU float64; gradients are PyTorch autograd
through exactly these operations.

Reading (per pixel p, centre (i + 0.5, j + 0.5); per triangle j with
projected corners a, b, c and camera depths z_a, z_b, z_c):

* projection: x_cam = R x + t; u = fx x/z + cx, v = fy y/z + cy; a triangle
  with a corner at depth <= z_near, or with zero projected area, is skipped;
* barycentric weights w of p; inside when all w >= 0; d^2 = squared distance
  from p to the triangle's boundary (the nearest of its three edges);
* coverage D = sigmoid(+-d^2 / sigma) (+ inside, - outside), with
  q = 1 - D kept >= Q_MIN; a pixel outside with D < TAU is not covered;
* silhouette A = 1 - prod_j q_j (the probabilistic union of the coverages);
* clamped barycentrics wc = max(w, 0) / sum max(w, 0) interpolate the vertex
  colours (C_j) and, perspective-correct, the depth 1/z = sum wc_k / z_k;
  the normalised depth zh = (z_far - z) / (z_far - z_near) (nearer = larger);
* colour I = (sum_j D_j e^{zh_j/gamma} C_j + e^{eps/gamma} bg) /
             (sum_j D_j e^{zh_j/gamma} + e^{eps/gamma})
  (a softmax over depth: with small gamma the nearest covering triangle wins;
  the background sits at normalised depth eps);
* output [H, W, 4] = (I, A).
"""
from __future__ import annotations

import math

import torch

TAU = 1.0e-5   # an outside pixel with coverage below TAU is not covered
Q_MIN = 1.0e-6  # 1 - coverage is kept >= Q_MIN


def cutoff_d2(sigma: float) -> float:
    """Squared distance outside a triangle beyond which its coverage < TAU."""
    return sigma * math.log((1.0 - TAU) / TAU)


def project(x, cam):
    """[N, 3] world positions -> (u, v, z) screen coordinates and camera depth."""
    R = torch.as_tensor(cam.R, dtype=torch.float64)
    t = torch.as_tensor(cam.t, dtype=torch.float64)
    xc = x @ R.T + t
    z = xc[:, 2]
    u = cam.fx * xc[:, 0] / z + cam.cx
    v = cam.fy * xc[:, 1] / z + cam.cy
    return u, v, z


def _cross2(p, q):
    return p[..., 0] * q[..., 1] - p[..., 1] * q[..., 0]


def _seg_d2(p, e0, e1):
    d = e1 - e0
    dd = (d * d).sum(-1).clamp_min(1e-300)  # a zero-length edge: the distance to its point
    t = ((p - e0) * d).sum(-1) / dd
    t = t.clamp(0.0, 1.0)
    c = e0 + t[..., None] * d
    r = p - c
    return (r * r).sum(-1)


def render(x, faces, colours, cam, spec):
    """Image [H, W, 4] (RGB, silhouette) of triangles `faces` [F, 3] over
    vertices `x` [N, 3] with per-vertex `colours` [N, 3] (float64 tensors;
    differentiable in x and colours)."""
    x = torch.as_tensor(x, dtype=torch.float64)
    colours = torch.as_tensor(colours, dtype=torch.float64)
    f = torch.as_tensor(faces, dtype=torch.long)
    H, W = cam.height, cam.width
    u, v, z = project(x, cam)
    scr = torch.stack([u, v], dim=1)
    a, b, c = scr[f[:, 0]], scr[f[:, 1]], scr[f[:, 2]]
    zf = z[f]                                                  # [F, 3]
    A2 = _cross2(b - a, c - a)                                 # twice the signed area
    valid = (zf > cam.z_near).all(dim=1) & (A2.abs() > 1e-12)
    A2s = torch.where(valid, A2, torch.ones_like(A2))
    zs = torch.where(valid[:, None], zf, torch.ones_like(zf))

    jj, ii = torch.meshgrid(torch.arange(H, dtype=torch.float64), torch.arange(W, dtype=torch.float64),
                            indexing="ij")
    p = torch.stack([ii.reshape(-1) + 0.5, jj.reshape(-1) + 0.5], dim=1)[:, None, :]  # [P, 1, 2]
    pa, pb, pc = a[None] - p, b[None] - p, c[None] - p
    w = torch.stack([_cross2(pb, pc), _cross2(pc, pa), _cross2(pa, pb)], dim=-1) / A2s[None, :, None]
    inside = (w >= 0).all(dim=-1)
    d2 = torch.minimum(torch.minimum(_seg_d2(p, a[None], b[None]), _seg_d2(p, b[None], c[None])),
                       _seg_d2(p, c[None], a[None]))
    cover = valid[None] & (inside | (d2 <= cutoff_d2(spec.sigma)))
    tv = torch.where(inside, d2, -d2) / spec.sigma
    q = torch.sigmoid(-tv)
    q = torch.where(q > Q_MIN, q, torch.full_like(q, Q_MIN))
    q = torch.where(cover, q, torch.ones_like(q))
    D = 1.0 - q                                                # 0 where not covered

    wp = torch.where(w > 0, w, torch.zeros_like(w))
    wc = wp / wp.sum(-1, keepdim=True).clamp_min(1e-300)
    iz = (wc / zs[None]).sum(-1)
    zp = 1.0 / torch.where(cover, iz, torch.ones_like(iz))
    zh = (cam.z_far - zp) / (cam.z_far - cam.z_near)
    C = (wc[..., None] * colours[f][None]).sum(-2)             # [P, F, 3]

    A = 1.0 - torch.prod(q, dim=1)
    # softmax over depth; the shift m cancels exactly (detached: no gradient)
    zmax = torch.where(cover, zh, torch.full_like(zh, -1.0)).max(dim=1).values
    m = torch.clamp(zmax, min=spec.eps).detach()
    e = torch.exp((torch.where(cover, zh, m[:, None]) - m[:, None]) / spec.gamma)
    wgt = torch.where(cover, D * e, torch.zeros_like(D))
    wb = torch.exp((spec.eps - m) / spec.gamma)
    bg = torch.as_tensor(spec.bg, dtype=torch.float64)
    num = (wgt[..., None] * C).sum(1) + wb[:, None] * bg
    den = wgt.sum(1) + wb
    I = num / den[:, None]
    return torch.cat([I, A[:, None]], dim=1).reshape(H, W, 4)


def render_grad(x, faces, colours, cam, spec, dimage):
    """(image, dL/dx, dL/dcolours) for the loss L = sum(image * dimage)."""
    xt = torch.as_tensor(x, dtype=torch.float64).clone().requires_grad_(True)
    ct = torch.as_tensor(colours, dtype=torch.float64).clone().requires_grad_(True)
    img = render(xt, faces, ct, cam, spec)
    (img * torch.as_tensor(dimage, dtype=torch.float64)).sum().backward()
    return img.detach(), xt.grad.detach(), ct.grad.detach()
