"""FP64 CPU oracle of the differentiable XPBD step (ctypes wrapper of ``xpbd_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py``; the product path never imports it.  It shares no code
with the CUDA library: it takes a ``Scene`` (plain arrays from the seeded generators) and
computes everything else itself.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

from .build import build as _build, LIB_PATH

_lib = None

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)


class _Model(C.Structure):
    _fields_ = [("V", C.c_int32), ("rest_x", _dp), ("inv_mass", _dp),
                ("n_dist", C.c_int32), ("dist_idx", _ip), ("n_bend", C.c_int32), ("bend_idx", _ip),
                ("n_tet", C.c_int32), ("tet_idx", _ip), ("tet_gamma", _dp),
                ("n_colors", C.c_int32), ("color_offsets", _ip), ("color_order", _ip),
                ("tet_coupled", C.c_int32), ("n_memb", C.c_int32), ("memb_idx", _ip), ("memb_uv", _dp)]


class _Params(C.Structure):
    _fields_ = [("dt", C.c_double), ("gravity", C.c_double * 3), ("compliance", _dp),
                ("f_global", _dp), ("f_vertex", _dp), ("collider_flags", C.c_int32),
                ("plane_h", C.c_double), ("sphere", C.c_double * 4),
                ("contact_compliance", C.c_double), ("thickness", C.c_double),
                ("f_vertex_steps", _dp), ("memb_stiffness", _dp)]


class _Direction(C.Structure):
    _fields_ = [("d_compliance", _dp), ("d_x0", _dp), ("d_v0", _dp), ("d_f_global", _dp),
                ("d_f_vertex", _dp), ("d_collider", _dp), ("d_f_vertex_steps", _dp),
                ("d_memb_stiffness", _dp)]


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            _build()
        _lib = C.CDLL(LIB_PATH)
        _lib.oracle_forward.restype = C.c_int
        _lib.oracle_adjoint.restype = C.c_int
        _lib.oracle_tangent.restype = C.c_int
        _lib.oracle_constraint.restype = C.c_int
        _lib.oracle_num_threads.restype = C.c_int
    return _lib


def _d(a):
    if a is None:
        return None, None
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(_ip)


class _Args:
    """Keeps the numpy buffers alive while the C structs point into them."""

    def __init__(self, scene, compliance=None, f_global=None, f_vertex=None, plane_h=None,
                 sphere=None, steps=None, f_vertex_steps=None, memb_stiffness=None):
        keep = []

        def d(a):
            arr, p = _d(a)
            keep.append(arr)
            return p

        def i(a):
            arr, p = _i(a)
            keep.append(arr)
            return p

        s = scene
        self.model = _Model(V=s.V, rest_x=d(s.rest_x), inv_mass=d(s.inv_mass),
                            n_dist=s.n_dist, dist_idx=i(s.dist_idx.reshape(-1)),
                            n_bend=s.n_bend, bend_idx=i(s.bend_idx.reshape(-1)),
                            n_tet=s.n_tet, tet_idx=i(s.tet_idx.reshape(-1)),
                            tet_gamma=d(s.tet_gamma) if s.n_tet else None,
                            n_colors=s.n_colors, color_offsets=i(s.color_offsets),
                            color_order=i(s.color_order),
                            tet_coupled=int(bool(getattr(s, "tet_coupled", False))),
                            n_memb=s.n_memb,
                            memb_idx=i(s.memb_idx.reshape(-1)) if s.n_memb else None,
                            memb_uv=d(s.memb_uv.reshape(-1)) if s.n_memb else None)
        comp = s.compliance if compliance is None else compliance
        fg = s.f_global if f_global is None else f_global
        fv = s.f_vertex if f_vertex is None else f_vertex
        if fg is not None and steps is not None:
            fg = np.asarray(fg, np.float64).reshape(-1, 3)
            if fg.shape[0] < steps:
                raise ValueError("f_global has fewer rows than steps")
        fvs = getattr(s, "f_vertex_steps", None) if f_vertex_steps is None else f_vertex_steps
        if fvs is not None and steps is not None:
            fvs = np.asarray(fvs, np.float64).reshape(-1, s.V, 3)
            if fvs.shape[0] < steps:
                raise ValueError("f_vertex_steps has fewer steps than simulated")
        sph = s.sphere if sphere is None else sphere
        self.params = _Params(dt=s.dt, gravity=(C.c_double * 3)(*s.gravity), compliance=d(comp),
                              f_global=d(fg), f_vertex=d(fv), collider_flags=s.collider_flags,
                              plane_h=s.plane_h if plane_h is None else plane_h,
                              sphere=(C.c_double * 4)(*sph),
                              contact_compliance=s.contact_compliance, thickness=s.thickness,
                              f_vertex_steps=d(fvs),
                              memb_stiffness=(d(s.memb_stiffness if memb_stiffness is None else memb_stiffness)
                                              if s.n_memb else None))
        self.keep = keep


def set_threads(n: int) -> None:
    lib().oracle_set_threads(int(n))


def set_fp32_rounding(on: bool) -> None:
    """Round every state value the forward program produces to float32 (attainable-floor
    measurement); off by default."""
    lib().oracle_set_fp32_rounding(int(bool(on)))


class fp32_rounding:
    """Context manager: run oracle calls with the FP32-rounding emulation on."""

    def __enter__(self):
        set_fp32_rounding(True)
        return self

    def __exit__(self, *exc):
        set_fp32_rounding(False)
        return False


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def forward(scene, steps: Optional[int] = None, iters: Optional[int] = None, *, x0=None, v0=None,
            compliance=None, f_global=None, f_vertex=None, plane_h=None, sphere=None, f_vertex_steps=None,
            memb_stiffness=None):
    """Run the FP64 forward simulation; returns (xs, vs), each [steps+1, V, 3]."""
    steps = scene.steps if steps is None else steps
    iters = scene.iters if iters is None else iters
    a = _Args(scene, compliance, f_global, f_vertex, plane_h, sphere, steps, f_vertex_steps, memb_stiffness)
    x0a, x0p = _d(scene.x0 if x0 is None else x0)
    v0a, v0p = _d(scene.v0 if v0 is None else v0)
    xs = np.zeros((steps + 1, scene.V, 3))
    vs = np.zeros((steps + 1, scene.V, 3))
    lib().oracle_forward(C.byref(a.model), C.byref(a.params), steps, iters, x0p, v0p,
                         xs.ctypes.data_as(_dp), vs.ctypes.data_as(_dp))
    return xs, vs


def forward_multipliers(scene, steps: Optional[int] = None, iters: Optional[int] = None, *, x0=None, v0=None,
                        compliance=None, f_global=None, f_vertex=None, f_vertex_steps=None):
    """Forward simulation returning also what each step ended with: (xs, vs, lam [steps, m]
    by constraint id, lam_c [steps, V, 2] of the plane / sphere contact of each vertex,
    active [steps, V, 2] the contact set)."""
    steps = scene.steps if steps is None else steps
    iters = scene.iters if iters is None else iters
    a = _Args(scene, compliance, f_global, f_vertex, None, None, steps, f_vertex_steps)
    x0a, x0p = _d(scene.x0 if x0 is None else x0)
    v0a, v0p = _d(scene.v0 if v0 is None else v0)
    xs = np.zeros((steps + 1, scene.V, 3))
    vs = np.zeros((steps + 1, scene.V, 3))
    lam = np.zeros((steps, scene.m))
    lamc = np.zeros((steps, scene.V, 2))
    act = np.zeros((steps, scene.V, 2), np.uint8)
    lib().oracle_forward_multipliers(C.byref(a.model), C.byref(a.params), steps, iters, x0p, v0p,
                                     xs.ctypes.data_as(_dp), vs.ctypes.data_as(_dp), lam.ctypes.data_as(_dp),
                                     lamc.ctypes.data_as(_dp), act.ctypes.data_as(C.POINTER(C.c_uint8)))
    return xs, vs, lam, lamc, act.astype(bool)


def forward_memb_multipliers(scene, steps: Optional[int] = None, iters: Optional[int] = None, *, x0=None, v0=None,
                             memb_stiffness=None) -> np.ndarray:
    """The membranes' multipliers (E_uu, E_vv, 2 E_uv rows) each step ended with:
    [steps, n_memb, 3]."""
    steps = scene.steps if steps is None else steps
    iters = scene.iters if iters is None else iters
    a = _Args(scene, None, None, None, None, None, steps, None, memb_stiffness)
    x0a, x0p = _d(scene.x0 if x0 is None else x0)
    v0a, v0p = _d(scene.v0 if v0 is None else v0)
    out = np.zeros((steps, scene.n_memb, 3))
    lib().oracle_forward_memb_multipliers(C.byref(a.model), C.byref(a.params), steps, iters, x0p, v0p,
                                          out.ctypes.data_as(_dp))
    return out


def adjoint(scene, seeds: dict, steps: Optional[int] = None, iters: Optional[int] = None, *,
            seed_dv_T=None, x0=None, v0=None, compliance=None, f_global=None, f_vertex=None,
            plane_h=None, sphere=None, f_vertex_steps=None, memb_stiffness=None) -> dict:
    """Reverse sweep.  ``seeds`` maps step n -> dL/dx_n [V,3].  Returns a dict of FP64
    gradients: compliance [m], x0 [V,3], v0 [V,3], f_global [steps,3], f_vertex [V,3],
    collider [5] (plane h, sphere cx, cy, cz, r), f_vertex_steps [steps,V,3] (the force on
    each vertex at each step), memb_stiffness [n_memb,4] (C00, C11, C01, C22)."""
    steps = scene.steps if steps is None else steps
    iters = scene.iters if iters is None else iters
    a = _Args(scene, compliance, f_global, f_vertex, plane_h, sphere, steps, f_vertex_steps, memb_stiffness)
    x0a, x0p = _d(scene.x0 if x0 is None else x0)
    v0a, v0p = _d(scene.v0 if v0 is None else v0)
    keys = sorted(seeds)
    ss, ssp = _i(np.asarray(keys, np.int32) if keys else np.zeros(1, np.int32))
    sd, sdp = _d(np.stack([np.asarray(seeds[k], np.float64).reshape(-1) for k in keys])
                 if keys else np.zeros(1))
    dv, dvp = _d(None if seed_dv_T is None else np.asarray(seed_dv_T).reshape(-1))
    out = dict(compliance=np.zeros(scene.m), x0=np.zeros((scene.V, 3)), v0=np.zeros((scene.V, 3)),
               f_global=np.zeros((steps, 3)), f_vertex=np.zeros((scene.V, 3)), collider=np.zeros(5),
               f_vertex_steps=np.zeros((steps, scene.V, 3)), memb_stiffness=np.zeros((scene.n_memb, 4)))
    P = lambda k: out[k].ctypes.data_as(_dp)
    lib().oracle_adjoint(C.byref(a.model), C.byref(a.params), steps, iters, x0p, v0p, len(keys),
                         ssp, sdp, dvp, P("compliance"), P("x0"), P("v0"), P("f_global"),
                         P("f_vertex"), P("collider"), P("f_vertex_steps"), P("memb_stiffness"))
    return out


def tangent(scene, direction: dict, steps: Optional[int] = None, iters: Optional[int] = None, *,
            x0=None, v0=None, compliance=None, f_global=None, f_vertex=None, f_vertex_steps=None):
    """Forward-mode derivative along ``direction`` (keys as in ``adjoint``'s output).
    Returns (dxs, dvs), each [steps+1, V, 3]."""
    steps = scene.steps if steps is None else steps
    iters = scene.iters if iters is None else iters
    a = _Args(scene, compliance, f_global, f_vertex, None, None, steps, f_vertex_steps)
    x0a, x0p = _d(scene.x0 if x0 is None else x0)
    v0a, v0p = _d(scene.v0 if v0 is None else v0)
    keep = []

    def dd(k):
        if direction.get(k) is None:
            return None
        arr, p = _d(np.asarray(direction[k]).reshape(-1))
        keep.append(arr)
        return p

    D = _Direction(d_compliance=dd("compliance"), d_x0=dd("x0"), d_v0=dd("v0"),
                   d_f_global=dd("f_global"), d_f_vertex=dd("f_vertex"), d_collider=dd("collider"),
                   d_f_vertex_steps=dd("f_vertex_steps"), d_memb_stiffness=dd("memb_stiffness"))
    dxs = np.zeros((steps + 1, scene.V, 3))
    dvs = np.zeros((steps + 1, scene.V, 3))
    lib().oracle_tangent(C.byref(a.model), C.byref(a.params), steps, iters, x0p, v0p, C.byref(D),
                         dxs.ctypes.data_as(_dp), dvs.ctypes.data_as(_dp))
    return dxs, dvs


def rest_data(scene) -> np.ndarray:
    """Per constraint id: (L, theta0, B[0..8], vol) as derived by the oracle."""
    a = _Args(scene)
    out = np.zeros((scene.m, 12))
    lib().oracle_rest_data(C.byref(a.model), out.ctypes.data_as(_dp))
    return out


KIND = dict(dist=0, bend=1, tet_h=2, tet_d=3, plane=4, sphere=5, memb_uu=6, memb_vv=7, memb_uv=8)
N_INPUTS = {0: 6, 1: 12, 2: 12, 3: 12, 4: 4, 5: 7, 6: 9, 7: 9, 8: 9}


def constraint(kind, q, rest12=None, u=None):
    """One constraint in isolation: (C, grad, H u) by automatic differentiation."""
    k = KIND[kind] if isinstance(kind, str) else int(kind)
    n = N_INPUTS[k]
    q, qp = _d(np.asarray(q, np.float64).reshape(-1))
    r, rp = _d(np.zeros(12) if rest12 is None else np.asarray(rest12, np.float64))
    Cv = C.c_double(0.0)
    g = np.zeros(n)
    hu = np.zeros(n)
    ua, up = _d(None if u is None else np.asarray(u, np.float64).reshape(-1))
    lib().oracle_constraint(k, qp, rp, up, C.byref(Cv), g.ctypes.data_as(_dp),
                            hu.ctypes.data_as(_dp) if u is not None else None)
    return Cv.value, g, (hu if u is not None else None)


def project_one(kind, q, w, rest12, lam, alpha_tilde):
    """One XPBD update of one constraint; returns (q', lambda')."""
    k = KIND[kind] if isinstance(kind, str) else int(kind)
    q = np.array(q, np.float64).reshape(-1)
    wa, wp = _d(np.asarray(w, np.float64))
    ra, rp = _d(np.asarray(rest12, np.float64))
    l = C.c_double(lam)
    lib().oracle_project_one(k, q.ctypes.data_as(_dp), wp, rp, C.byref(l), C.c_double(alpha_tilde))
    return q, l.value


def vjp_one(kind, q, w, rest12, lam, alpha_tilde, qbar, lambar):
    """Reverse of ``project_one``: returns (qbar, lambar, alpha_tilde_bar)."""
    k = KIND[kind] if isinstance(kind, str) else int(kind)
    qa, qp = _d(np.asarray(q, np.float64).reshape(-1))
    wa, wp = _d(np.asarray(w, np.float64))
    ra, rp = _d(np.asarray(rest12, np.float64))
    qb = np.array(qbar, np.float64).reshape(-1)
    lb = C.c_double(lambar)
    ab = C.c_double(0.0)
    lib().oracle_vjp_one(k, qp, wp, rp, C.c_double(lam), C.c_double(alpha_tilde),
                         qb.ctypes.data_as(_dp), C.byref(lb), C.byref(ab))
    return qb, lb.value, ab.value


def project_pair(q, w, rest12, lam, alpha_tilde):
    """One coupled (C_H, C_D) update of one tet; returns (q', lambda'[2])."""
    q = np.array(q, np.float64).reshape(-1)
    wa, wp = _d(np.asarray(w, np.float64))
    ra, rp = _d(np.asarray(rest12, np.float64))
    l = np.array(lam, np.float64)
    aa, ap = _d(np.asarray(alpha_tilde, np.float64))
    lib().oracle_project_pair(q.ctypes.data_as(_dp), wp, rp, l.ctypes.data_as(_dp), ap)
    return q, l


def vjp_pair(q, w, rest12, lam, alpha_tilde, qbar, lambar):
    """Reverse of ``project_pair``: returns (qbar, lambar[2], alpha_tilde_bar[2])."""
    qa, qp = _d(np.asarray(q, np.float64).reshape(-1))
    wa, wp = _d(np.asarray(w, np.float64))
    ra, rp = _d(np.asarray(rest12, np.float64))
    la, lp = _d(np.asarray(lam, np.float64))
    aa, ap = _d(np.asarray(alpha_tilde, np.float64))
    qb = np.array(qbar, np.float64).reshape(-1)
    lb = np.array(lambar, np.float64)
    ab = np.zeros(2)
    lib().oracle_vjp_pair(qp, wp, rp, lp, ap, qb.ctypes.data_as(_dp), lb.ctypes.data_as(_dp),
                          ab.ctypes.data_as(_dp))
    return qb, lb, ab


def project_memb(q, w, B2, lam, alpha_tilde):
    """One membrane update (3x3 multiplier solve); returns (q' [9], lambda' [3])."""
    q = np.array(q, np.float64).reshape(-1)
    wa, wp = _d(np.asarray(w, np.float64))
    ba, bp = _d(np.asarray(B2, np.float64).reshape(-1))
    l = np.array(lam, np.float64)
    aa, ap = _d(np.asarray(alpha_tilde, np.float64).reshape(-1))
    lib().oracle_project_memb(q.ctypes.data_as(_dp), wp, bp, l.ctypes.data_as(_dp), ap)
    return q, l


def vjp_memb(q, w, B2, lam, alpha_tilde, qbar, lambar):
    """Reverse of ``project_memb``: returns (qbar [9], lambar [3], abar4 [4]) with abar4 the
    adjoint of the alpha~ entries (00, 11, 01 = 10, 22)."""
    qa, qp = _d(np.asarray(q, np.float64).reshape(-1))
    wa, wp = _d(np.asarray(w, np.float64))
    ba, bp = _d(np.asarray(B2, np.float64).reshape(-1))
    la, lp = _d(np.asarray(lam, np.float64))
    aa, ap = _d(np.asarray(alpha_tilde, np.float64).reshape(-1))
    qb = np.array(qbar, np.float64).reshape(-1)
    lb = np.array(lambar, np.float64)
    ab = np.zeros(4)
    lib().oracle_vjp_memb(qp, wp, bp, lp, ap, qb.ctypes.data_as(_dp), lb.ctypes.data_as(_dp),
                          ab.ctypes.data_as(_dp))
    return qb, lb, ab
