"""ctypes binding of the gradsim C ABI (include/gradsim.h).

Argument marshalling only: every step of the method runs in the CUDA
library.  Function names match the C entry points; the small classes below
(`Context`, `Mesh`, `Batch`, `Server`) only own handles and translate torch
tensors / numpy arrays into pointers.  Loading fails loudly when the library
has not been built: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

GS_OK, GS_EINVAL, GS_ENOMEM, GS_ECUDA, GS_ESTATE, GS_ENONFINITE = 0, -1, -2, -3, -4, -5
GS_ETIMEOUT, GS_ECANCELLED, GS_ENOTFOUND, GS_EUNSUPPORTED = -6, -7, -8, -9
GS_EINDEX, GS_EINTERNAL = -10, -11
GS_BUILD_CHECKED = 1
GS_PENDING, GS_WUNSTABLE = 1, 2
GS_NOALLOC_MAX_NODES = 4194304
GS_TET, GS_CLOTH = 0, 1
GS_MEM_DEVICE, GS_MEM_HOST = 0, 1

_vp = C.c_void_p
_dp = C.POINTER(C.c_double)
_fp = C.POINTER(C.c_float)
_ip = C.POINTER(C.c_int32)


class gs_contact(C.Structure):
    _fields_ = [("ke", C.c_float), ("kd", C.c_float), ("kf", C.c_float), ("mu_f", C.c_float),
                ("plane_on", C.c_int), ("plane_n", C.c_float * 3), ("plane_h", C.c_float),
                ("sphere_on", C.c_int), ("sphere_c", C.c_float * 3), ("sphere_r", C.c_float)]


class gs_mesh_desc(C.Structure):
    _fields_ = [("kind", C.c_int), ("n_nodes", C.c_int), ("n_elems", C.c_int), ("elems", _ip),
                ("n_hinges", C.c_int), ("hinges", _ip), ("X", _dp), ("v0", _dp), ("mu", _dp),
                ("lambda_", _dp), ("density", _dp), ("kb", _dp), ("act", _dp), ("hinge_act", _dp),
                ("pinned", C.POINTER(C.c_uint8)), ("contact", gs_contact), ("gravity", C.c_float * 3),
                ("patch_elems", C.c_int), ("block_threads", C.c_int), ("block_threads_adj", C.c_int)]


class gs_mesh_info(C.Structure):
    _fields_ = [("kind", C.c_int), ("n_nodes", C.c_int), ("n_elems", C.c_int), ("n_hinges", C.c_int),
                ("n_patches", C.c_int), ("n_boundary_nodes", C.c_int), ("patch_elems", C.c_int),
                ("block_threads", C.c_int), ("block_threads_adj", C.c_int), ("dt_stable", C.c_double),
                ("device_bytes", C.c_size_t)]


class gs_camera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int), ("height", C.c_int),
                ("z_near", C.c_float), ("z_far", C.c_float)]


class gs_raster_desc(C.Structure):
    _fields_ = [("n_vertices", C.c_int), ("n_faces", C.c_int), ("faces", C.POINTER(C.c_int)),
                ("camera", gs_camera), ("sigma", C.c_float), ("gamma", C.c_float), ("eps", C.c_float),
                ("bg", C.c_float * 3)]


class gs_rigid_desc(C.Structure):
    _fields_ = [("n_bodies", C.c_int), ("point_begin", C.POINTER(C.c_int)), ("points", _fp), ("mass", _fp),
                ("inertia", _fp), ("contact", _fp), ("scene", gs_contact), ("gravity", C.c_float * 3)]


class gs_rigid_grads(C.Structure):
    _fields_ = [("d_state0", _vp), ("d_mass", _vp), ("d_inertia", _vp), ("d_contact", _vp)]


class gs_air(C.Structure):
    _fields_ = [("k_drag", C.c_float), ("k_lift", C.c_float), ("wind", C.c_float * 3)]


class gs_grads(C.Structure):
    _fields_ = [("d_mu", _vp), ("d_lambda", _vp), ("d_density", _vp), ("d_act", _vp), ("d_kb", _vp),
                ("d_hinge_act", _vp), ("d_mass", _vp), ("d_x0", _vp), ("d_v0", _vp), ("d_act_seq", _vp),
                ("d_hinge_act_seq", _vp)]


_ALLOC_FN = C.CFUNCTYPE(_vp, C.c_size_t, _vp, _vp)
_FREE_FN = C.CFUNCTYPE(None, _vp, C.c_size_t, _vp, _vp)


class gs_allocator(C.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("free", _FREE_FN), ("user", _vp)]


class gs_server_opts(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_size_t), ("max_active", C.c_int), ("K", C.c_int),
                ("use_graphs", C.c_int), ("build_threads", C.c_int)]


class gs_query(C.Structure):
    _fields_ = [("mesh", gs_mesh_desc), ("dt", C.c_float), ("n_steps", C.c_int), ("target", _fp)]


class gs_result(C.Structure):
    _fields_ = [("status", C.c_int), ("loss", C.c_double), ("n_elems", C.c_int), ("n_hinges", C.c_int),
                ("n_nodes", C.c_int), ("d_mu", _dp), ("d_lambda", _dp), ("d_density", _dp), ("d_kb", _dp),
                ("d_x0", _fp), ("d_v0", _fp), ("t_submit", C.c_double), ("t_admit", C.c_double),
                ("t_done", C.c_double)]


class gs_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("rejected", C.c_uint64),
                ("active", C.c_uint64), ("queued", C.c_uint64), ("p50_latency_s", C.c_double),
                ("p99_latency_s", C.c_double), ("elem_steps_per_s", C.c_double), ("admitted_bytes", C.c_size_t),
                ("busy_s", C.c_double), ("build_s", C.c_double), ("start_s", C.c_double), ("rebuild_s", C.c_double),
                ("rt_sync_s", C.c_double), ("gpu_wait_s", C.c_double), ("ticks", C.c_uint64),
                ("rebuilds", C.c_uint64), ("rt_syncs", C.c_uint64)]


class gs_kernel_time(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_uint64), ("total_ms", C.c_double)]


# every entry point of include/gradsim.h with its C signature
_PROTOS = {
    "gs_version": (C.c_int, []),
    "gs_build_flags": (C.c_int, []),
    "gs_last_error": (C.c_char_p, []),
    "gs_create": (C.c_int, [C.POINTER(_vp), C.c_int, C.c_size_t, C.POINTER(gs_allocator)]),
    "gs_destroy": (None, [_vp]),
    "gs_ctx_bytes": (C.c_size_t, [_vp]),
    "gs_set_graphs": (C.c_int, [_vp, C.c_int]),
    "gs_profile": (C.c_int, [_vp, C.c_int]),
    "gs_profile_read": (C.c_int, [_vp, C.POINTER(gs_kernel_time), C.c_int, C.POINTER(C.c_int)]),
    "gs_mesh_create": (C.c_int, [_vp, C.POINTER(gs_mesh_desc), C.POINTER(_vp)]),
    "gs_mesh_destroy": (None, [_vp]),
    "gs_mesh_info_get": (C.c_int, [_vp, C.POINTER(gs_mesh_info)]),
    "gs_mesh_set_params": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, C.c_int, _vp]),
    "gs_mesh_set_state": (C.c_int, [_vp, _vp, _vp, C.c_int, _vp]),
    "gs_mesh_set_act_seq": (C.c_int, [_vp, _vp, _vp, C.c_int, C.c_int, _vp]),
    "gs_mesh_set_air": (C.c_int, [_vp, _vp, _vp]),
    "gs_mesh_get_state": (C.c_int, [_vp, _vp, _vp, C.c_int, _vp]),
    "gs_mesh_reset": (C.c_int, [_vp, _vp]),
    "gs_mesh_check": (C.c_int, [_vp, C.c_int, _vp]),
    "gs_step": (C.c_int, [_vp, C.c_float, C.c_int, _vp]),
    "gs_rollout": (C.c_int, [_vp, C.c_float, C.c_int, C.c_int, _vp, _vp, C.c_int, _vp]),
    "gs_adjoint": (C.c_int, [_vp, _vp, _vp, C.POINTER(gs_grads), C.c_int, C.c_int, _vp]),
    "gs_batch_create": (C.c_int, [_vp, C.POINTER(_vp), C.c_int, C.POINTER(_vp)]),
    "gs_batch_destroy": (None, [_vp]),
    "gs_batch_step": (C.c_int, [_vp, _fp, C.c_int, _vp]),
    "gs_batch_rollout": (C.c_int, [_vp, _fp, C.c_int, C.c_int, C.POINTER(_vp), _vp, _vp]),
    "gs_batch_adjoint": (C.c_int, [_vp, C.POINTER(gs_grads), _vp]),
    "gs_loss_noalloc": (C.c_int, [_vp, _vp, C.c_int, _vp, _vp, _vp]),
    "gs_server_create": (C.c_int, [_vp, C.POINTER(gs_server_opts), C.POINTER(_vp)]),
    "gs_server_destroy": (None, [_vp]),
    "gs_query_submit": (C.c_int, [_vp, C.POINTER(gs_query), C.POINTER(C.c_uint64)]),
    "gs_query_poll": (C.c_int, [_vp, C.c_uint64, C.POINTER(gs_result), C.c_int]),
    "gs_query_cancel": (C.c_int, [_vp, C.c_uint64]),
    "gs_server_stats_get": (C.c_int, [_vp, C.POINTER(gs_server_stats)]),
    "gs_result_free": (None, [C.POINTER(gs_result)]),
    "gs_selftest_bounded_wait": (C.c_int, [C.c_int, C.POINTER(C.c_int), _vp]),
    "gs_raster_create": (C.c_int, [_vp, C.POINTER(gs_raster_desc), C.POINTER(_vp)]),
    "gs_rigid_create": (C.c_int, [_vp, C.POINTER(gs_rigid_desc), C.POINTER(_vp)]),
    "gs_rigid_destroy": (None, [_vp]),
    "gs_rigid_set_params": (C.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "gs_rigid_rollout": (C.c_int, [_vp, C.c_float, C.c_int, _vp, _vp, _vp]),
    "gs_rigid_adjoint": (C.c_int, [_vp, _vp, C.POINTER(gs_rigid_grads), _vp]),
    "gs_rigid_points": (C.c_int, [_vp, _vp, _vp, _vp]),
    "gs_rigid_points_backward": (C.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "gs_rigid_check": (C.c_int, [_vp, C.c_int, _vp]),
    "gs_raster_destroy": (None, [_vp]),
    "gs_raster_set_camera": (C.c_int, [_vp, C.POINTER(gs_camera)]),
    "gs_raster_forward": (C.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "gs_raster_backward": (C.c_int, [_vp, _vp, _vp, _vp, _vp]),
}

_lib = None


def library_path() -> str:
    return _build.LIB_CHECKED if os.environ.get("GRADSIM_CHECKED") == "1" else _build.LIB


def load(build: bool = False):
    """Load libgradsim.so (building it first when ``build`` is set); with the
    environment variable GRADSIM_CHECKED=1, the index-checked build
    libgradsim_check.so instead."""
    global _lib
    if _lib is not None:
        return _lib
    if build:
        _build.build()
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is not built; run __graft_entry__.build() first")
    L = C.CDLL(path)
    for name, (res, args) in _PROTOS.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


class GradsimError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"gradsim status {status}: {msg}")
        self.status = status


def check(status: int) -> int:
    if status < 0:
        raise GradsimError(status, load().gs_last_error().decode())
    return status


# thin wrappers with the C names --------------------------------------------
def _wrap(name):
    def f(*args):
        return getattr(load(), name)(*args)
    f.__name__ = name
    return f


for _n in _PROTOS:
    globals()[_n] = _wrap(_n)


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------
def _stream(stream=None):
    if stream is not None:
        return _vp(stream)
    import torch
    return _vp(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    """Device or host pointer of a torch tensor / numpy array (None -> NULL)."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return _vp(t.ctypes.data)
    return _vp(t.data_ptr())


def _contact(c) -> gs_contact:
    out = gs_contact()
    out.ke, out.kd, out.kf, out.mu_f = c.ke, c.kd, c.kf, c.mu_f
    out.plane_on = int(c.plane_on)
    out.plane_n = (C.c_float * 3)(*c.plane_n)
    out.plane_h = c.plane_h
    out.sphere_on = int(c.sphere_on)
    out.sphere_c = (C.c_float * 3)(*c.sphere_c)
    out.sphere_r = c.sphere_r
    return out


def mesh_desc(problem, patch_elems: int = 0, block_threads: int = 0, block_threads_adj: int = 0):
    """gs_mesh_desc for an ``inputs.Problem``; returns (desc, keep-alive list)."""
    keep = []

    def arr(a, dtype):
        if a is None:
            return None
        a = np.ascontiguousarray(a, dtype=dtype)
        keep.append(a)
        return a

    d = gs_mesh_desc()
    d.kind = int(problem.kind)
    d.n_nodes = problem.n_nodes
    d.n_elems = problem.n_elems
    e = arr(problem.elems, np.int32)
    d.elems = e.ctypes.data_as(_ip)
    if problem.hinges is not None and problem.kind == GS_CLOTH:
        h = arr(problem.hinges, np.int32)
        d.n_hinges = h.shape[0]
        d.hinges = h.ctypes.data_as(_ip)
        d.kb = arr(problem.kb, np.float64).ctypes.data_as(_dp)
        if problem.hinge_act is not None:
            d.hinge_act = arr(problem.hinge_act, np.float64).ctypes.data_as(_dp)
    d.X = arr(problem.X, np.float64).ctypes.data_as(_dp)
    if problem.v0 is not None:
        d.v0 = arr(problem.v0, np.float64).ctypes.data_as(_dp)
    d.mu = arr(problem.mu, np.float64).ctypes.data_as(_dp)
    d.lambda_ = arr(problem.lam, np.float64).ctypes.data_as(_dp)
    d.density = arr(problem.rho, np.float64).ctypes.data_as(_dp)
    if problem.act is not None:
        d.act = arr(problem.act, np.float64).ctypes.data_as(_dp)
    if problem.pinned is not None:
        d.pinned = arr(problem.pinned, np.uint8).ctypes.data_as(C.POINTER(C.c_uint8))
    d.contact = _contact(problem.contact)
    d.gravity = (C.c_float * 3)(*problem.gravity)
    d.patch_elems = int(patch_elems)
    d.block_threads = int(block_threads)
    d.block_threads_adj = int(block_threads_adj)
    return d, keep


class Context:
    """A gs_ctx on one GPU.  ``torch_alloc`` routes device memory through
    PyTorch's caching allocator instead of cudaMallocAsync."""

    def __init__(self, device: int = 0, budget: int = 0, torch_alloc: bool = False):
        self.h = _vp()
        self.device = int(device)
        self._cb = None
        alloc = None
        if torch_alloc:
            import torch

            def _a(nbytes, stream, user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), device, stream or 0)
                except Exception:  # noqa: BLE001 - reported to the library as NULL
                    return None

            def _f(ptr, nbytes, stream, user):
                torch.cuda.caching_allocator_delete(ptr)

            self._cb = (_ALLOC_FN(_a), _FREE_FN(_f))
            alloc = gs_allocator(self._cb[0], self._cb[1], None)
        check(load().gs_create(C.byref(self.h), device, budget, C.byref(alloc) if alloc else None))

    def set_graphs(self, enable: bool):
        check(load().gs_set_graphs(self.h, int(enable)))

    def bytes(self) -> int:
        return load().gs_ctx_bytes(self.h)

    def close(self):
        if self.h:
            load().gs_destroy(self.h)
            self.h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass


class Mesh:
    """A gs_mesh built from an ``inputs.Problem`` (host arrays are copied)."""

    def __init__(self, ctx: Context, problem, patch_elems: int = 0, block_threads: int = 0,
                 block_threads_adj: int = 0):
        self.ctx = ctx
        self.problem = problem
        d, keep = mesh_desc(problem, patch_elems, block_threads, block_threads_adj)
        self.h = _vp()
        check(load().gs_mesh_create(ctx.h, C.byref(d), C.byref(self.h)))
        self.info = gs_mesh_info()
        check(load().gs_mesh_info_get(self.h, C.byref(self.info)))
        self.status = GS_OK
        if getattr(problem, "air", None) is not None:
            self.set_air(problem.air)

    @property
    def n_nodes(self):
        return self.info.n_nodes

    def set_params(self, mu=None, lam=None, rho=None, act=None, kb=None, host=False, stream=None):
        check(load().gs_mesh_set_params(self.h, _ptr(mu), _ptr(lam), _ptr(rho), _ptr(act), _ptr(kb),
                                         GS_MEM_HOST if host else GS_MEM_DEVICE, _stream(stream)))

    def set_state(self, x=None, v=None, host=False, stream=None):
        check(load().gs_mesh_set_state(self.h, _ptr(x), _ptr(v), GS_MEM_HOST if host else GS_MEM_DEVICE,
                                       _stream(stream)))

    def set_air(self, air=None, stream=None):
        """Air on the cloth surface (an object with k_drag, k_lift, wind), or
        None to turn it off."""
        if air is None:
            check(load().gs_mesh_set_air(self.h, None, _stream(stream)))
            return
        a = gs_air(float(air.k_drag), float(air.k_lift), (C.c_float * 3)(*[float(w) for w in air.wind]))
        check(load().gs_mesh_set_air(self.h, C.byref(a), _stream(stream)))

    def set_act_seq(self, act_seq=None, hinge_act_seq=None, host=False, stream=None):
        """Time-varying actuation: row n of act_seq [n_steps][n_elems] (and
        hinge_act_seq [n_steps][n_hinges]) is added during step n; None for
        both clears.  FP32 arrays (device tensors, or host arrays with host=True)."""
        rows = [a.shape[0] for a in (act_seq, hinge_act_seq) if a is not None]
        if len(set(rows)) > 1:
            raise ValueError("actuation sequences need the same number of steps")
        n = rows[0] if rows else 0
        check(load().gs_mesh_set_act_seq(self.h, _ptr(act_seq), _ptr(hinge_act_seq), int(n),
                                         GS_MEM_HOST if host else GS_MEM_DEVICE, _stream(stream)))

    def reset(self, stream=None):
        check(load().gs_mesh_reset(self.h, _stream(stream)))

    def get_state(self, x=None, v=None, host=False, stream=None):
        check(load().gs_mesh_get_state(self.h, _ptr(x), _ptr(v), GS_MEM_HOST if host else GS_MEM_DEVICE,
                                       _stream(stream)))

    def check_finite(self, reset=False, stream=None) -> int:
        return load().gs_mesh_check(self.h, int(reset), _stream(stream))

    def step(self, dt, n, stream=None):
        self.status = check(load().gs_step(self.h, float(dt), int(n), _stream(stream)))

    def rollout(self, dt, n, K=0, target=None, loss_out=None, host=False, stream=None):
        self.status = check(load().gs_rollout(self.h, float(dt), int(n), int(K), _ptr(target), _ptr(loss_out),
                                              GS_MEM_HOST if host else GS_MEM_DEVICE, _stream(stream)))

    def adjoint(self, grads: dict, dLdx=None, dLdv=None, keep=False, host=False, stream=None):
        g = gs_grads(**{k: _ptr(v) for k, v in grads.items()})
        check(load().gs_adjoint(self.h, _ptr(dLdx), _ptr(dLdv), C.byref(g),
                                GS_MEM_HOST if host else GS_MEM_DEVICE, int(keep), _stream(stream)))

    def close(self):
        if self.h:
            load().gs_mesh_destroy(self.h)
            self.h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass


class Batch:
    """Several meshes advanced by one launch per kernel per step."""

    def __init__(self, ctx: Context, meshes):
        self.ctx = ctx
        self.meshes = list(meshes)
        arr = (_vp * len(self.meshes))(*[m.h for m in self.meshes])
        self.h = _vp()
        check(load().gs_batch_create(ctx.h, arr, len(self.meshes), C.byref(self.h)))

    def _dt(self, dt):
        dts = np.ascontiguousarray(np.broadcast_to(np.asarray(dt, np.float32), (len(self.meshes),)))
        return dts, dts.ctypes.data_as(_fp)

    def step(self, dt, n, stream=None):
        keep, p = self._dt(dt)
        return check(load().gs_batch_step(self.h, p, int(n), _stream(stream)))

    def rollout(self, dt, n, K=0, targets=None, loss_out=None, stream=None):
        keep, p = self._dt(dt)
        tg = None
        if targets is not None:
            tg = (_vp * len(self.meshes))(*[(t.data_ptr() if t is not None else None) for t in targets])
        return check(load().gs_batch_rollout(self.h, p, int(n), int(K), tg, _ptr(loss_out), _stream(stream)))

    def adjoint(self, grads, stream=None):
        arr = (gs_grads * len(self.meshes))()
        for i, g in enumerate(grads):
            arr[i] = gs_grads(**{k: _ptr(v) for k, v in g.items()})
        return check(load().gs_batch_adjoint(self.h, arr, _stream(stream)))

    def close(self):
        if self.h:
            load().gs_batch_destroy(self.h)
            self.h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass


def contact_struct(con) -> "gs_contact":
    """gs_contact from an ``inputs.Contact``."""
    c = gs_contact()
    c.ke, c.kd, c.kf, c.mu_f = float(con.ke), float(con.kd), float(con.kf), float(con.mu_f)
    c.plane_on = int(con.plane_on)
    c.plane_n = (C.c_float * 3)(*[float(v) for v in con.plane_n])
    c.plane_h = float(con.plane_h)
    c.sphere_on = int(con.sphere_on)
    c.sphere_c = (C.c_float * 3)(*[float(v) for v in con.sphere_c])
    c.sphere_r = float(con.sphere_r)
    return c


class Rigid:
    """A gs_rigid: a set of independent rigid bodies (``inputs.RigidBody``
    list; they share the scene and gravity of the first)."""

    def __init__(self, ctx: Context, bodies):
        self.ctx = ctx
        self.bodies = list(bodies)
        nb = len(self.bodies)
        pb = np.zeros(nb + 1, dtype=np.int32)
        for b, body in enumerate(self.bodies):
            pb[b + 1] = pb[b] + len(body.points)
        self._pb = pb
        self._pts = np.ascontiguousarray(np.vstack([b.points for b in self.bodies]), dtype=np.float32)
        self._m = np.array([b.mass for b in self.bodies], dtype=np.float32)
        self._I = np.ascontiguousarray([b.inertia for b in self.bodies], dtype=np.float32)
        self._c = np.ascontiguousarray([b.contact for b in self.bodies], dtype=np.float32)
        d = gs_rigid_desc()
        d.n_bodies = nb
        d.point_begin = pb.ctypes.data_as(C.POINTER(C.c_int))
        d.points = self._pts.ctypes.data_as(_fp)
        d.mass = self._m.ctypes.data_as(_fp)
        d.inertia = self._I.ctypes.data_as(_fp)
        d.contact = self._c.ctypes.data_as(_fp)
        d.scene = contact_struct(self.bodies[0].scene)
        d.gravity = (C.c_float * 3)(*[float(g) for g in self.bodies[0].gravity])
        self.h = _vp()
        check(load().gs_rigid_create(ctx.h, C.byref(d), C.byref(self.h)))
        self.n_bodies, self.n_points = nb, int(pb[-1])

    def state0(self):
        return np.ascontiguousarray(np.stack([b.state0 for b in self.bodies]), dtype=np.float32)

    def set_params(self, mass=None, inertia=None, contact=None, stream=None):
        def host(a, shape):
            return None if a is None else np.ascontiguousarray(np.asarray(a, dtype=np.float32).reshape(shape))
        m, I, c = host(mass, (-1,)), host(inertia, (-1, 6)), host(contact, (-1, 4))
        check(load().gs_rigid_set_params(self.h, _ptr(m), _ptr(I), _ptr(c), _stream(stream)))

    def rollout(self, dt, steps, state0, stateS=None, stream=None):
        check(load().gs_rigid_rollout(self.h, float(dt), int(steps), _ptr(state0), _ptr(stateS), _stream(stream)))

    def adjoint(self, grads: dict, seed=None, stream=None):
        g = gs_rigid_grads(**{k: _ptr(v) for k, v in grads.items()})
        check(load().gs_rigid_adjoint(self.h, _ptr(seed), C.byref(g), _stream(stream)))

    def points(self, state, out, stream=None):
        check(load().gs_rigid_points(self.h, _ptr(state), _ptr(out), _stream(stream)))

    def points_backward(self, state, dpoints, dstate, stream=None):
        check(load().gs_rigid_points_backward(self.h, _ptr(state), _ptr(dpoints), _ptr(dstate), _stream(stream)))

    def check_finite(self, reset=False, stream=None) -> int:
        return load().gs_rigid_check(self.h, int(reset), _stream(stream))

    def close(self):
        if self.h:
            load().gs_rigid_destroy(self.h)
            self.h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass


def camera_struct(cam) -> gs_camera:
    """gs_camera from an ``inputs.Camera``."""
    c = gs_camera()
    c.R = (C.c_float * 9)(*[float(v) for v in np.asarray(cam.R, dtype=np.float64).ravel()])
    c.t = (C.c_float * 3)(*[float(v) for v in np.asarray(cam.t, dtype=np.float64).ravel()])
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.width, c.height = int(cam.width), int(cam.height)
    c.z_near, c.z_far = float(cam.z_near), float(cam.z_far)
    return c


class Raster:
    """A gs_raster: the soft rasteriser over a fixed triangle list (faces
    [F, 3] into n_vertices vertices), camera and settings
    (``inputs.RenderSpec``)."""

    def __init__(self, ctx: Context, n_vertices: int, faces, camera, spec):
        self.ctx = ctx
        f = np.ascontiguousarray(faces, dtype=np.int32).reshape(-1, 3)
        self._faces = f
        d = gs_raster_desc()
        d.n_vertices, d.n_faces = int(n_vertices), int(f.shape[0])
        d.faces = f.ctypes.data_as(C.POINTER(C.c_int)) if f.size else None
        d.camera = camera_struct(camera)
        d.sigma, d.gamma, d.eps = float(spec.sigma), float(spec.gamma), float(spec.eps)
        d.bg = (C.c_float * 3)(*[float(b) for b in spec.bg])
        self.h = _vp()
        check(load().gs_raster_create(ctx.h, C.byref(d), C.byref(self.h)))
        self.n_vertices, self.width, self.height = int(n_vertices), int(camera.width), int(camera.height)

    def set_camera(self, camera):
        check(load().gs_raster_set_camera(self.h, C.byref(camera_struct(camera))))

    def forward(self, x, colours, image, stream=None):
        check(load().gs_raster_forward(self.h, _ptr(x), _ptr(colours), _ptr(image), _stream(stream)))

    def backward(self, dimage, dx=None, dcolours=None, stream=None):
        check(load().gs_raster_backward(self.h, _ptr(dimage), _ptr(dx), _ptr(dcolours), _stream(stream)))

    def close(self):
        if self.h:
            load().gs_raster_destroy(self.h)
            self.h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass


class Server:
    """Continuous-batching gradient-query server (gs_server_*)."""

    def __init__(self, ctx: Context, budget: int = 0, max_active: int = 0, K: int = 0, build_threads: int = 0):
        self.ctx = ctx
        o = gs_server_opts(budget, max_active, K, 0, build_threads)
        self.h = _vp()
        check(load().gs_server_create(ctx.h, C.byref(o), C.byref(self.h)))
        self._keep = {}

    def submit(self, problem, target, dt=None, steps=None) -> int:
        if getattr(problem, "air", None) is not None:
            raise ValueError("served queries carry no air model; run a Mesh or Batch instead")
        d, keep = mesh_desc(problem)
        t = np.ascontiguousarray(target, dtype=np.float32)
        q = gs_query(d, float(problem.dt if dt is None else dt), int(problem.steps if steps is None else steps),
                     t.ctypes.data_as(_fp))
        ticket = C.c_uint64(0)
        check(load().gs_query_submit(self.h, C.byref(q), C.byref(ticket)))
        return ticket.value

    def poll(self, ticket: int, timeout_ms: int = 0):
        """(status, result dict or None); result arrays are copied to numpy."""
        r = gs_result()
        st = load().gs_query_poll(self.h, C.c_uint64(ticket), C.byref(r), int(timeout_ms))
        if st in (GS_PENDING, GS_ETIMEOUT) or st == GS_ENOTFOUND:
            return st, None
        out = {"status": st, "loss": r.loss, "t_submit": r.t_submit, "t_admit": r.t_admit, "t_done": r.t_done}
        E, B, N = r.n_elems, r.n_hinges, r.n_nodes
        for name, n, ct in (("d_mu", E, C.c_double), ("d_lambda", E, C.c_double), ("d_density", E, C.c_double),
                            ("d_kb", B, C.c_double), ("d_x0", 3 * N, C.c_float), ("d_v0", 3 * N, C.c_float)):
            ptr = getattr(r, name)
            out[name] = np.ctypeslib.as_array(ptr, shape=(n,)).copy() if (ptr and n) else None
        load().gs_result_free(C.byref(r))
        return st, out

    def cancel(self, ticket: int) -> int:
        return load().gs_query_cancel(self.h, C.c_uint64(ticket))

    def stats(self) -> dict:
        s = gs_server_stats()
        check(load().gs_server_stats_get(self.h, C.byref(s)))
        return {f: getattr(s, f) for f, _ in gs_server_stats._fields_}

    def close(self):
        if self.h:
            load().gs_server_destroy(self.h)
            self.h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass
