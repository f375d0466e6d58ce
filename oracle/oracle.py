"""ctypes front-end of the FP64 CPU oracle (test infrastructure only).

Only the test suite, the package smoke check and the benchmark's CPU-baseline
leg may import this module.  It wraps ``gs_oracle.cpp`` (a plain FP64
restatement of the paper's equations, App. A-C) for numpy inputs built by
``paper_2104_02646_gb300.inputs``.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


class _Model(C.Structure):
    _fields_ = [
        ("n_nodes", C.c_int), ("X", _dp),
        ("n_tets", C.c_int), ("tets", _ip), ("tet_mu", _dp), ("tet_lam", _dp),
        ("tet_rho", _dp), ("tet_act", _dp),
        ("n_tris", C.c_int), ("tris", _ip), ("tri_mu", _dp), ("tri_lam", _dp),
        ("tri_rho", _dp), ("tri_act", _dp),
        ("n_hinges", C.c_int), ("hinges", _ip), ("hinge_kb", _dp), ("hinge_act", _dp),
        ("pinned", C.POINTER(C.c_ubyte)),
        ("gravity", C.c_double * 3),
        ("ke", C.c_double), ("kd", C.c_double), ("kf", C.c_double), ("mu_f", C.c_double),
        ("plane_on", C.c_int), ("plane_n", C.c_double * 3), ("plane_h", C.c_double),
        ("sphere_on", C.c_int), ("sphere_c", C.c_double * 3), ("sphere_r", C.c_double),
        ("n_act_steps", C.c_int), ("tet_act_seq", _dp), ("tri_act_seq", _dp), ("hinge_act_seq", _dp),
        ("air_on", C.c_int), ("k_drag", C.c_double), ("k_lift", C.c_double), ("wind", C.c_double * 3),
    ]


_GRAD_FIELDS = ["x0", "v0", "tet_mu", "tet_lam", "tet_rho", "tet_act", "tri_mu", "tri_lam",
                "tri_rho", "tri_act", "hinge_kb", "hinge_act", "contact", "node_mass",
                "tet_act_seq", "tri_act_seq", "hinge_act_seq"]
_DIR_FIELDS = ["x0", "v0", "tet_mu", "tet_lam", "tet_rho", "tet_act", "tri_mu", "tri_lam",
               "tri_rho", "tri_act", "hinge_kb", "hinge_act", "contact",
               "tet_act_seq", "tri_act_seq", "hinge_act_seq"]
_SEQ = ("tet_act_seq", "tri_act_seq", "hinge_act_seq")


class _Rigid(C.Structure):
    _fields_ = [("n_points", C.c_int), ("points", _dp), ("mass", C.c_double), ("inertia", C.c_double * 6),
                ("contact", C.c_double * 4), ("scene", C.POINTER(_Model))]


class _Grads(C.Structure):
    _fields_ = [(f, _dp) for f in _GRAD_FIELDS]


class _Dirs(C.Structure):
    _fields_ = [(f, _dp) for f in _DIR_FIELDS]


_lib = None


def lib():
    """The compiled oracle.  GS_ORACLE_LIB, if set, names another build of
    the same source to load instead (the tests' copies with a planted
    mistake, which the pins must reject)."""
    global _lib
    if _lib is None:
        L = C.CDLL(os.environ.get("GS_ORACLE_LIB") or _build.build())
        L.orc_tet_rest.argtypes = [_dp, _dp, _dp]
        L.orc_tri_rest.argtypes = [_dp, _dp, _dp]
        L.orc_node_masses.argtypes = [C.POINTER(_Model), _dp]
        L.orc_tet_forces.argtypes = [_dp, _dp, C.c_double, C.c_double, C.c_double, C.c_double, _dp]
        L.orc_tet_energy.argtypes = [_dp, _dp, C.c_double, C.c_double, C.c_double, C.c_double]
        L.orc_tet_energy.restype = C.c_double
        L.orc_tri_forces.argtypes = [_dp, _dp, C.c_double, C.c_double, C.c_double, C.c_double, _dp]
        L.orc_tri_energy.argtypes = [_dp, _dp, C.c_double, C.c_double, C.c_double, C.c_double]
        L.orc_tri_energy.restype = C.c_double
        L.orc_hinge_forces.argtypes = [_dp, C.c_double, C.c_double, _dp]
        L.orc_hinge_angle.argtypes = [_dp]
        L.orc_hinge_angle.restype = C.c_double
        L.orc_hinge_angle_grad.argtypes = [_dp, _dp]
        L.orc_contact_force.argtypes = [C.POINTER(_Model), _dp, _dp, _dp]
        L.orc_air_forces.argtypes = [_dp, _dp, C.c_double, C.c_double, _dp, _dp]
        L.orc_rigid_rollout.argtypes = [C.POINTER(_Rigid), _dp, C.c_double, C.c_int, _dp, _dp]
        L.orc_rigid_loss_grad.argtypes = [C.POINTER(_Rigid), _dp, C.c_double, C.c_int, _dp, _dp, _dp, _dp, _dp,
                                          _dp, _dp]
        L.orc_rigid_loss_dir.argtypes = [C.POINTER(_Rigid), _dp, C.c_double, C.c_int, _dp, _dp, _dp, C.c_double,
                                         _dp, _dp, _dp, _dp]
        L.orc_forces.argtypes = [C.POINTER(_Model), _dp, _dp, _dp]
        L.orc_rollout.argtypes = [C.POINTER(_Model), _dp, _dp, C.c_double, C.c_int, _dp, _dp, _dp]
        L.orc_loss_grad.argtypes = [C.POINTER(_Model), _dp, _dp, C.c_double, C.c_int, _dp, _dp,
                                    _dp, _dp, C.POINTER(_Grads)]
        L.orc_loss_dir.argtypes = [C.POINTER(_Model), _dp, _dp, C.c_double, C.c_int, _dp,
                                   C.POINTER(_Dirs), _dp, _dp]
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_set_threads.restype = C.c_int
        L.orc_max_threads.restype = C.c_int
        _lib = L
    return _lib


def set_threads(n):
    """Threads of the oracle's independent element / node loops (n <= 0: all
    cores); results are bitwise the same for any count.  Returns the count."""
    return int(lib().orc_set_threads(int(n)))


def max_threads():
    return int(lib().orc_max_threads())


def _d(a):
    """float64 C-contiguous view (kept alive by the caller) or None."""
    if a is None:
        return None
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a):
    return None if a is None else a.ctypes.data_as(_dp)


class Model:
    """A problem description in the oracle's C layout.

    Accepts a ``paper_2104_02646_gb300.inputs.Problem`` (tets when
    ``kind == TET``; triangles + hinges when ``kind == CLOTH``) or explicit
    keyword arrays for mixed / tiny test meshes.
    """

    def __init__(self, problem=None, *, X=None, tets=None, tet_mu=None, tet_lam=None,
                 tet_rho=None, tet_act=None, tris=None, tri_mu=None, tri_lam=None,
                 tri_rho=None, tri_act=None, hinges=None, kb=None, hinge_act=None,
                 pinned=None, contact=None, gravity=(0.0, -9.81, 0.0), act_seq=None, hinge_act_seq=None,
                 air=None):
        # act_seq [n_steps][n_elements] (tets or triangles) and hinge_act_seq
        # [n_steps][n_hinges]: actuation added during each step; air: an
        # object with k_drag, k_lift, wind (the triangles' air model)
        if problem is not None:
            air = getattr(problem, "air", None) if air is None else air
            act_seq = getattr(problem, "act_seq", None) if act_seq is None else act_seq
            hinge_act_seq = getattr(problem, "hinge_act_seq", None) if hinge_act_seq is None else hinge_act_seq
            X = problem.X
            contact = problem.contact
            gravity = problem.gravity
            pinned = problem.pinned
            if problem.kind == 0:
                tets, tet_mu, tet_lam, tet_rho, tet_act = (problem.elems, problem.mu, problem.lam,
                                                           problem.rho, problem.act)
            else:
                tris, tri_mu, tri_lam, tri_rho, tri_act = (problem.elems, problem.mu, problem.lam,
                                                           problem.rho, problem.act)
                hinges, kb, hinge_act = problem.hinges, problem.kb, problem.hinge_act
        self._keep = []

        def keep(a, dtype=np.float64):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dtype=dtype)
            self._keep.append(a)
            return a

        m = _Model()
        X = keep(X)
        m.n_nodes = X.shape[0]
        m.X = _p(X)
        self.n_nodes = X.shape[0]
        if tets is not None and len(tets):
            t = keep(tets, np.int32)
            m.n_tets = t.shape[0]
            m.tets = t.ctypes.data_as(_ip)
            m.tet_mu, m.tet_lam, m.tet_rho = _p(keep(tet_mu)), _p(keep(tet_lam)), _p(keep(tet_rho))
            m.tet_act = _p(keep(tet_act))
        self.n_tets = m.n_tets
        if tris is not None and len(tris):
            t = keep(tris, np.int32)
            m.n_tris = t.shape[0]
            m.tris = t.ctypes.data_as(_ip)
            m.tri_mu, m.tri_lam, m.tri_rho = _p(keep(tri_mu)), _p(keep(tri_lam)), _p(keep(tri_rho))
            m.tri_act = _p(keep(tri_act))
        self.n_tris = m.n_tris
        if hinges is not None and len(hinges):
            h = keep(hinges, np.int32)
            m.n_hinges = h.shape[0]
            m.hinges = h.ctypes.data_as(_ip)
            m.hinge_kb = _p(keep(kb))
            m.hinge_act = _p(keep(hinge_act))
        self.n_hinges = m.n_hinges
        if pinned is not None:
            pn = keep(pinned, np.uint8)
            m.pinned = pn.ctypes.data_as(C.POINTER(C.c_ubyte))
        m.gravity = (C.c_double * 3)(*gravity)
        self.n_act_steps = 0
        if act_seq is not None or hinge_act_seq is not None:
            rows = [np.asarray(a).shape[0] for a in (act_seq, hinge_act_seq) if a is not None]
            if len(set(rows)) != 1:
                raise ValueError("actuation sequences need the same number of steps")
            m.n_act_steps = self.n_act_steps = rows[0]
            if act_seq is not None:
                a = keep(act_seq)
                if m.n_tets:
                    m.tet_act_seq = _p(a)
                else:
                    m.tri_act_seq = _p(a)
            if hinge_act_seq is not None:
                m.hinge_act_seq = _p(keep(hinge_act_seq))
        if air is not None:
            m.air_on = 1
            m.k_drag, m.k_lift = float(air.k_drag), float(air.k_lift)
            m.wind = (C.c_double * 3)(*air.wind)
        if contact is not None:
            m.ke, m.kd, m.kf, m.mu_f = contact.ke, contact.kd, contact.kf, contact.mu_f
            m.plane_on = int(contact.plane_on)
            m.plane_n = (C.c_double * 3)(*contact.plane_n)
            m.plane_h = contact.plane_h
            m.sphere_on = int(contact.sphere_on)
            m.sphere_c = (C.c_double * 3)(*contact.sphere_c)
            m.sphere_r = contact.sphere_r
        self.c = m

    # -- whole mesh ---------------------------------------------------------
    def masses(self):
        out = np.zeros(self.n_nodes)
        lib().orc_node_masses(C.byref(self.c), _p(out))
        return out

    def forces(self, x, v):
        x, v = _d(x), _d(v)
        f = np.zeros((self.n_nodes, 3))
        lib().orc_forces(C.byref(self.c), _p(x), _p(v), _p(f))
        return f

    def contact_force(self, x, v):
        x, v = _d(x), _d(v)
        f = np.zeros(3)
        lib().orc_contact_force(C.byref(self.c), _p(x), _p(v), _p(f))
        return f

    def rollout(self, x0, v0, dt, steps, traj=False):
        x0, v0 = _d(x0), _d(v0)
        xS = np.zeros((self.n_nodes, 3))
        vS = np.zeros((self.n_nodes, 3))
        tr = np.zeros((steps + 1, self.n_nodes, 3)) if traj else None
        lib().orc_rollout(C.byref(self.c), _p(x0), _p(v0), dt, steps, _p(xS), _p(vS), _p(tr))
        return (xS, vS, tr) if traj else (xS, vS)

    def loss_grad(self, x0, v0, dt, steps, target=None, xbar=None, vbar=None, act_seq_grad=False):
        """Loss sum |x(S) - target|^2 and every gradient, by the discrete adjoint.
        With ``act_seq_grad`` also the per-step actuation gradients
        (``tet_act_seq`` / ``tri_act_seq`` [S][n], ``hinge_act_seq`` [S][n_hinges])."""
        x0, v0, target, xbar, vbar = _d(x0), _d(v0), _d(target), _d(xbar), _d(vbar)
        N = self.n_nodes
        out = {
            "x0": np.zeros((N, 3)), "v0": np.zeros((N, 3)),
            "tet_mu": np.zeros(self.n_tets), "tet_lam": np.zeros(self.n_tets),
            "tet_rho": np.zeros(self.n_tets), "tet_act": np.zeros(self.n_tets),
            "tri_mu": np.zeros(self.n_tris), "tri_lam": np.zeros(self.n_tris),
            "tri_rho": np.zeros(self.n_tris), "tri_act": np.zeros(self.n_tris),
            "hinge_kb": np.zeros(self.n_hinges), "hinge_act": np.zeros(self.n_hinges),
            "contact": np.zeros(4), "node_mass": np.zeros(N),
        }
        for k, n in zip(_SEQ, (self.n_tets, self.n_tris, self.n_hinges)):
            out[k] = np.zeros((steps, n)) if act_seq_grad else np.zeros(0)
        g = _Grads(**{k: (_p(out[k]) if out[k].size else None) for k in _GRAD_FIELDS})
        L = C.c_double(0.0)
        lib().orc_loss_grad(C.byref(self.c), _p(x0), _p(v0), dt, steps, _p(target), _p(xbar),
                            _p(vbar), C.byref(L), C.byref(g))
        return L.value, out

    def loss_dir(self, x0, v0, dt, steps, target, dirs):
        """Forward-mode (dual number) loss and its derivative along ``dirs``
        (a dict keyed like the gradient outputs, e.g. ``{"tet_mu": d}``)."""
        x0, v0, target = _d(x0), _d(v0), _d(target)
        keep = {k: _d(v) for k, v in dirs.items()}
        for k in keep:
            if k not in _DIR_FIELDS:
                raise KeyError(k)
        d = _Dirs(**{k: _p(v) for k, v in keep.items()})
        L = C.c_double(0.0)
        dL = C.c_double(0.0)
        lib().orc_loss_dir(C.byref(self.c), _p(x0), _p(v0), dt, steps, _p(target), C.byref(d),
                           C.byref(L), C.byref(dL))
        return L.value, dL.value


# -- single elements --------------------------------------------------------

def tet_rest(X):
    X = _d(X).reshape(12)
    Dminv = np.zeros(9)
    V = C.c_double(0.0)
    lib().orc_tet_rest(_p(X), _p(Dminv), C.byref(V))
    return Dminv.reshape(3, 3), V.value


def tri_rest(X):
    X = _d(X).reshape(9)
    Dminv = np.zeros(4)
    A = C.c_double(0.0)
    lib().orc_tri_rest(_p(X), _p(Dminv), C.byref(A))
    return Dminv.reshape(2, 2), A.value


def tet_forces(x, Dminv, V, mu, lam, act=0.0):
    x, Dminv = _d(x).reshape(12), _d(Dminv).reshape(9)
    f = np.zeros(12)
    lib().orc_tet_forces(_p(x), _p(Dminv), V, mu, lam, act, _p(f))
    return f.reshape(4, 3)


def tet_energy(x, Dminv, V, mu, lam, act=0.0):
    x, Dminv = _d(x).reshape(12), _d(Dminv).reshape(9)
    return lib().orc_tet_energy(_p(x), _p(Dminv), V, mu, lam, act)


def tri_forces(x, Dminv, A, mu, lam, act=0.0):
    x, Dminv = _d(x).reshape(9), _d(Dminv).reshape(4)
    f = np.zeros(9)
    lib().orc_tri_forces(_p(x), _p(Dminv), A, mu, lam, act, _p(f))
    return f.reshape(3, 3)


def tri_energy(x, Dminv, A, mu, lam, act=0.0):
    x, Dminv = _d(x).reshape(9), _d(Dminv).reshape(4)
    return lib().orc_tri_energy(_p(x), _p(Dminv), A, mu, lam, act)


def hinge_forces(x, kb, act=0.0):
    x = _d(x).reshape(12)
    f = np.zeros(12)
    lib().orc_hinge_forces(_p(x), kb, act, _p(f))
    return f.reshape(4, 3)


def hinge_angle(x):
    x = _d(x).reshape(12)
    return lib().orc_hinge_angle(_p(x))


def hinge_angle_grad(x):
    x = _d(x).reshape(12)
    g = np.zeros(12)
    lib().orc_hinge_angle_grad(_p(x), _p(g))
    return g.reshape(4, 3)


def air_forces(x, v, k_drag, k_lift, wind=(0.0, 0.0, 0.0)):
    """Air force on the corners of one triangle ([3, 3] positions and
    velocities) under the oracle's flat-plate reading of the air's lift and drag."""
    x = _d(np.asarray(x).reshape(9))
    v = _d(np.asarray(v).reshape(9))
    w = _d(np.asarray(wind).reshape(3))
    f = np.zeros(9)
    lib().orc_air_forces(_p(x), _p(v), float(k_drag), float(k_lift), _p(w), _p(f))
    return f.reshape(3, 3)


class Rigid:
    """One rigid body (an ``inputs.RigidBody``) in the oracle's layout: points,
    mass, inertia, contact parameters and the scene (plane / sphere, gravity)."""

    def __init__(self, body, mass=None, inertia=None, contact=None):
        self._pts = np.ascontiguousarray(body.points, dtype=np.float64)
        self._scene = Model(X=np.zeros((1, 3)), contact=body.scene, gravity=body.gravity)
        r = _Rigid()
        r.n_points = self._pts.shape[0]
        r.points = _p(self._pts)
        r.mass = float(body.mass if mass is None else mass)
        r.inertia = (C.c_double * 6)(*(body.inertia if inertia is None else inertia))
        r.contact = (C.c_double * 4)(*(body.contact if contact is None else contact))
        r.scene = C.pointer(self._scene.c)
        self.c = r

    def rollout(self, state0, dt, steps, traj=False):
        s0 = _d(state0)
        sS = np.zeros(13)
        tr = np.zeros((steps + 1, 13)) if traj else None
        lib().orc_rigid_rollout(C.byref(self.c), _p(s0), dt, steps, _p(sS), _p(tr))
        return (sS, tr) if traj else sS

    def loss_grad(self, state0, dt, steps, target=None, seed=None):
        """(L, {"state0" [13], "mass", "inertia" [6], "contact" [4]}) for
        L = sum_k |X_k(S) - target_k|^2 + seed . state(S)."""
        s0, tg, sd = _d(state0), _d(target), _d(seed)
        L = C.c_double(0.0)
        g = {"state0": np.zeros(13), "mass": np.zeros(1), "inertia": np.zeros(6), "contact": np.zeros(4)}
        lib().orc_rigid_loss_grad(C.byref(self.c), _p(s0), dt, steps, _p(tg), _p(sd), C.byref(L),
                                  _p(g["state0"]), _p(g["mass"]), _p(g["inertia"]), _p(g["contact"]))
        g["mass"] = float(g["mass"][0])
        return L.value, g

    def loss_dir(self, state0, dt, steps, target=None, seed=None, d_state0=None, d_mass=0.0, d_inertia=None,
                 d_contact=None):
        s0, tg, sd = _d(state0), _d(target), _d(seed)
        ds, di, dc = _d(d_state0), _d(d_inertia), _d(d_contact)
        L, dL = C.c_double(0.0), C.c_double(0.0)
        lib().orc_rigid_loss_dir(C.byref(self.c), _p(s0), dt, steps, _p(tg), _p(sd), _p(ds), float(d_mass),
                                 _p(di), _p(dc), C.byref(L), C.byref(dL))
        return L.value, dL.value
