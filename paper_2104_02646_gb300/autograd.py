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


class Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mesh, dt, steps, K, mu, lam, rho, x0, v0):
        dev = x0.device
        f32 = dict(dtype=torch.float32, device=dev)
        mu_, lam_, rho_ = (t.detach().to(**f32).contiguous() for t in (mu, lam, rho))
        mesh.set_params(mu=mu_, lam=lam_, rho=rho_)
        mesh.set_state(x=x0.detach().to(**f32).contiguous(), v=v0.detach().to(**f32).contiguous())
        mesh.rollout(dt, steps, K)
        N = mesh.n_nodes
        xS = torch.empty(N, 3, **f32)
        vS = torch.empty(N, 3, **f32)
        mesh.get_state(xS, vS)
        ctx.mesh = mesh
        ctx.shapes = (mu.dtype, lam.dtype, rho.dtype, x0.dtype, v0.dtype)
        return xS, vS

    @staticmethod
    def backward(ctx, gx, gv):
        mesh = ctx.mesh
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
    def forward(ctx, mesh, dt, steps, K, act_seq, hinge_act_seq, x0, v0):
        dev = x0.device
        f32 = dict(dtype=torch.float32, device=dev)
        a = None if act_seq is None else act_seq.detach().to(**f32).contiguous()
        h = None if hinge_act_seq is None else hinge_act_seq.detach().to(**f32).contiguous()
        mesh.set_act_seq(a, h)
        mesh.set_state(x=x0.detach().to(**f32).contiguous(), v=v0.detach().to(**f32).contiguous())
        mesh.rollout(dt, steps, K)
        N = mesh.n_nodes
        xS = torch.empty(N, 3, **f32)
        vS = torch.empty(N, 3, **f32)
        mesh.get_state(xS, vS)
        ctx.mesh = mesh
        ctx.steps = steps
        ctx.has = (act_seq is not None, hinge_act_seq is not None)
        ctx.dtypes = (x0.dtype, v0.dtype)
        return xS, vS

    @staticmethod
    def backward(ctx, gx, gv):
        mesh = ctx.mesh
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
