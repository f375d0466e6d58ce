"""PyTorch autograd integration of the rollout (the paper wraps its kernels as
custom autograd operations, App. A; here the whole checkpointed rollout is one
operation).

``rollout(mesh, dt, steps, mu, lam, rho, x0, v0, K=0)`` returns the final
state (x(S), v(S)) as tensors; calling ``backward`` on any loss of them runs
the library's discrete adjoint (gs_adjoint) with dL/dx(S), dL/dv(S) as seeds
and returns gradients for the per-element Lame parameters, density and the
initial state.  All arithmetic happens in the CUDA library; this module only
marshals tensors.
"""
from __future__ import annotations

import torch

from . import gradsim as gs


def _claim(mesh):
    """A token for the rollout a forward is about to store on `mesh`; a
    later forward on the same mesh replaces the stored rollout."""
    tok = getattr(mesh, "_rollout_seq", 0) + 1
    mesh._rollout_seq = tok
    mesh._rollout_token = tok
    return tok


class Rollout(torch.autograd.Function):
    @staticmethod
    def _run(mesh, dt, steps, K, mu, lam, rho, x0, v0):
        f32 = dict(dtype=torch.float32, device=x0.device)
        # no time-varying actuation: clear one an earlier actuated rollout left
        mesh.set_act_seq(None, None)
        mesh.set_params(mu=mu, lam=lam, rho=rho)
        mesh.set_state(x=x0, v=v0)
        mesh.rollout(dt, steps, K)
        N = mesh.n_nodes
        xS = torch.empty(N, 3, **f32)
        vS = torch.empty(N, 3, **f32)
        mesh.get_state(xS, vS)
        return xS, vS

    @staticmethod
    def forward(ctx, mesh, dt, steps, K, mu, lam, rho, x0, v0):
        dev = x0.device
        f32 = dict(dtype=torch.float32, device=dev)
        args = [t.detach().to(**f32).contiguous() for t in (mu, lam, rho, x0, v0)]
        xS, vS = Rollout._run(mesh, dt, steps, K, *args)
        ctx.mesh = mesh
        ctx.token = _claim(mesh)
        ctx.replay = (dt, steps, K, args)
        ctx.shapes = (mu.dtype, lam.dtype, rho.dtype, x0.dtype, v0.dtype)
        return xS, vS

    @staticmethod
    def backward(ctx, gx, gv):
        mesh = ctx.mesh
        if getattr(mesh, "_rollout_token", None) != ctx.token:
            # a later rollout on this mesh (e.g. the next segment between two
            # rendered frames) replaced the stored states: recompute them
            dt, steps, K, args = ctx.replay
            Rollout._run(mesh, dt, steps, K, *args)
        else:
            # the adjoint re-evaluates the element forces: no actuation sequence
            mesh.set_act_seq(None, None)
        mesh._rollout_token = None  # the adjoint consumes the stored rollout
        dev = gx.device if gx is not None else gv.device
        E, N = mesh.info.n_elems, mesh.n_nodes
        f64 = dict(dtype=torch.float64, device=dev)
        g = {"d_mu": torch.zeros(E, **f64), "d_lambda": torch.zeros(E, **f64), "d_density": torch.zeros(E, **f64),
             "d_x0": torch.zeros(N, 3, dtype=torch.float32, device=dev),
             "d_v0": torch.zeros(N, 3, dtype=torch.float32, device=dev)}
        sx = None if gx is None else gx.detach().to(torch.float32).contiguous()
        sv = None if gv is None else gv.detach().to(torch.float32).contiguous()
        mesh.adjoint(g, dLdx=sx, dLdv=sv)
        tm, tl, tr, tx, tv = ctx.shapes
        return (None, None, None, None, g["d_mu"].to(tm), g["d_lambda"].to(tl), g["d_density"].to(tr),
                g["d_x0"].to(tx), g["d_v0"].to(tv))


def rollout(mesh: "gs.Mesh", dt: float, steps: int, mu, lam, rho, x0, v0, K: int = 0):
    """Differentiable rollout; see the module docstring."""
    return Rollout.apply(mesh, dt, steps, K, mu, lam, rho, x0, v0)


class ActuatedRollout(torch.autograd.Function):
    """Differentiable rollout driven by a time-varying actuation (the control
    input of the paper's visuomotor control experiments, Sec. 3): row n of
    ``act_seq`` [S][n_elems] (and ``hinge_act_seq`` [S][n_hinges]) is added
    to the actuation during step n.  Returns (x(S), v(S)); backward runs the
    library's adjoint and returns the per-step actuation gradients and
    dL/dx0, dL/dv0."""

    @staticmethod
    def _run(mesh, dt, steps, K, a, h, x0, v0):
        f32 = dict(dtype=torch.float32, device=x0.device)
        mesh.set_act_seq(a, h)
        mesh.set_state(x=x0, v=v0)
        mesh.rollout(dt, steps, K)
        N = mesh.n_nodes
        xS = torch.empty(N, 3, **f32)
        vS = torch.empty(N, 3, **f32)
        mesh.get_state(xS, vS)
        return xS, vS

    @staticmethod
    def forward(ctx, mesh, dt, steps, K, act_seq, hinge_act_seq, x0, v0):
        dev = x0.device
        f32 = dict(dtype=torch.float32, device=dev)
        a = None if act_seq is None else act_seq.detach().to(**f32).contiguous()
        h = None if hinge_act_seq is None else hinge_act_seq.detach().to(**f32).contiguous()
        xf = x0.detach().to(**f32).contiguous()
        vf = v0.detach().to(**f32).contiguous()
        xS, vS = ActuatedRollout._run(mesh, dt, steps, K, a, h, xf, vf)
        ctx.mesh = mesh
        ctx.token = _claim(mesh)
        ctx.replay = (dt, steps, K, a, h, xf, vf)
        ctx.steps = steps
        ctx.has = (act_seq is not None, hinge_act_seq is not None)
        ctx.dtypes = (x0.dtype, v0.dtype)
        return xS, vS

    @staticmethod
    def backward(ctx, gx, gv):
        mesh = ctx.mesh
        dt, steps, K, a, h, xf, vf = ctx.replay
        if getattr(mesh, "_rollout_token", None) != ctx.token:
            # a later rollout on this mesh replaced the stored states (and
            # perhaps the actuation): recompute this one's
            ActuatedRollout._run(mesh, dt, steps, K, a, h, xf, vf)
        else:
            # the adjoint re-evaluates the element forces under this rollout's actuation
            mesh.set_act_seq(a, h)
        mesh._rollout_token = None  # the adjoint consumes the stored rollout
        dev = gx.device if gx is not None else gv.device
        S, E, B, N = ctx.steps, mesh.info.n_elems, mesh.info.n_hinges, mesh.n_nodes
        f32 = dict(dtype=torch.float32, device=dev)
        g = {"d_x0": torch.zeros(N, 3, **f32), "d_v0": torch.zeros(N, 3, **f32)}
        if ctx.has[0]:
            g["d_act_seq"] = torch.zeros(S, E, **f32)
        if ctx.has[1]:
            g["d_hinge_act_seq"] = torch.zeros(S, B, **f32)
        sx = None if gx is None else gx.detach().to(torch.float32).contiguous()
        sv = None if gv is None else gv.detach().to(torch.float32).contiguous()
        mesh.adjoint(g, dLdx=sx, dLdv=sv)
        tx, tv = ctx.dtypes
        return (None, None, None, None, g.get("d_act_seq"), g.get("d_hinge_act_seq"), g["d_x0"].to(tx),
                g["d_v0"].to(tv))


def actuated_rollout(mesh: "gs.Mesh", dt: float, steps: int, act_seq, x0, v0, hinge_act_seq=None, K: int = 0):
    """Differentiable rollout under a time-varying actuation; see ActuatedRollout."""
    return ActuatedRollout.apply(mesh, dt, steps, K, act_seq, hinge_act_seq, x0, v0)


class Render(torch.autograd.Function):
    """The soft rasteriser (Sec. 2 "Differentiable rendering engine") as an
    autograd operation: image [H, W, 4] from vertex positions [N, 3] and
    colours [N, 3]; backward runs gs_raster_backward."""

    @staticmethod
    def forward(ctx, raster, x, colours):
        f32 = dict(dtype=torch.float32, device=x.device)
        xs = x.detach().to(**f32).contiguous()
        cs = colours.detach().to(**f32).contiguous()
        img = torch.empty(raster.height, raster.width, 4, **f32)
        raster.forward(xs, cs, img)
        ctx.raster = raster
        ctx.token = _claim(raster)
        ctx.saved = (xs, cs)
        ctx.dtypes = (x.dtype, colours.dtype)
        return img

    @staticmethod
    def backward(ctx, gimg):
        r = ctx.raster
        xs, cs = ctx.saved
        if getattr(r, "_rollout_token", None) != ctx.token:
            # another frame was rendered since: restore this frame's state
            r.forward(xs, cs, torch.empty(r.height, r.width, 4, dtype=torch.float32, device=xs.device))
            r._rollout_token = ctx.token
        dx = torch.empty_like(xs)
        dc = torch.empty_like(cs)
        r.backward(gimg.detach().to(torch.float32).contiguous(), dx, dc)
        return None, dx.to(ctx.dtypes[0]), dc.to(ctx.dtypes[1])


def render(raster, x, colours):
    """Differentiable image [H, W, 4] (RGB, silhouette) of `raster`'s triangles."""
    return Render.apply(raster, x, colours)


class RigidRollout(torch.autograd.Function):
    """Rollout of a set of rigid bodies (App. A.1 "Rigid Bodies") as an
    autograd operation: final states [B, 13] from initial states and the
    per-body mass [B], inertia [B, 6] and contact parameters [B, 4]; backward
    runs gs_rigid_adjoint.  A later rollout on the same body set makes this
    one's backward recompute its states."""

    @staticmethod
    def _run(rigid, dt, steps, state0, mass, inertia, contact):
        rigid.set_params(mass=mass.detach().double().cpu().numpy(), inertia=inertia.detach().double().cpu().numpy(),
                         contact=contact.detach().double().cpu().numpy())
        sS = torch.empty_like(state0)
        rigid.rollout(dt, steps, state0, sS)
        return sS

    @staticmethod
    def forward(ctx, rigid, dt, steps, state0, mass, inertia, contact):
        s0 = state0.detach().to(torch.float32).contiguous()
        sS = RigidRollout._run(rigid, dt, steps, s0, mass, inertia, contact)
        ctx.rigid = rigid
        ctx.token = _claim(rigid)
        ctx.replay = (dt, steps, s0, mass.detach(), inertia.detach(), contact.detach())
        ctx.dtypes = (state0.dtype, mass.dtype, inertia.dtype, contact.dtype)
        return sS

    @staticmethod
    def backward(ctx, gS):
        r = ctx.rigid
        if getattr(r, "_rollout_token", None) != ctx.token:
            dt, steps, s0, m, I, c = ctx.replay
            RigidRollout._run(r, dt, steps, s0, m, I, c)
            r._rollout_token = ctx.token
        dev = gS.device
        B = r.n_bodies
        g = {"d_state0": torch.zeros(B, 13, dtype=torch.float32, device=dev),
             "d_mass": torch.zeros(B, dtype=torch.float64, device=dev),
             "d_inertia": torch.zeros(B, 6, dtype=torch.float64, device=dev),
             "d_contact": torch.zeros(B, 4, dtype=torch.float64, device=dev)}
        r.adjoint(g, seed=gS.detach().to(torch.float32).contiguous())
        ts, tm, ti, tc = ctx.dtypes
        return (None, None, None, g["d_state0"].to(ts), g["d_mass"].to(tm), g["d_inertia"].to(ti),
                g["d_contact"].to(tc))


def rigid_rollout(rigid, dt, steps, state0, mass, inertia, contact):
    """Differentiable rollout of a body set; see RigidRollout."""
    return RigidRollout.apply(rigid, dt, steps, state0, mass, inertia, contact)


class RigidPoints(torch.autograd.Function):
    """World positions [n_points, 3] of the bodies' points at states [B, 13]."""

    @staticmethod
    def forward(ctx, rigid, state):
        s = state.detach().to(torch.float32).contiguous()
        out = torch.empty(rigid.n_points, 3, dtype=torch.float32, device=s.device)
        rigid.points(s, out)
        ctx.rigid = rigid
        ctx.save_for_backward(s)
        return out

    @staticmethod
    def backward(ctx, gX):
        (s,) = ctx.saved_tensors
        ds = torch.empty_like(s)
        ctx.rigid.points_backward(s, gX.detach().to(torch.float32).contiguous(), ds)
        return None, ds


def rigid_points(rigid, state):
    return RigidPoints.apply(rigid, state)

