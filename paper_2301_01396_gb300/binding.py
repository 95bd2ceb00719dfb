"""Python binding of the C ABI in ``include/diffxpbd.h`` (ctypes; argument marshalling only).

Every step of the simulation and of its adjoint runs in the CUDA library
``_lib/libdiffxpbd.so``; this module only passes device pointers, sizes and the current
torch stream.  Importing it does not load the library; the first call does, and raises
``RuntimeError`` if the library is missing (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np
import torch

from .build import LIB_PATH

XPBD_OK = 0
STATUS = {0: "XPBD_OK", 1: "XPBD_ERR_INVALID", 2: "XPBD_ERR_COLORING", 3: "XPBD_ERR_OOM",
          4: "XPBD_ERR_CUDA", 5: "XPBD_ERR_NONFINITE", 6: "XPBD_ERR_TIMEOUT", 7: "XPBD_ERR_BOUNDS"}
COLLIDE_PLANE = 1
COLLIDE_SPHERE = 2
STATIC_MAX_VERTICES = 65536        # limits of xpbd_forward_static (include/diffxpbd.h)
STATIC_MAX_CONSTRAINTS = 393216

_fp = C.POINTER(C.c_float)
_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)


class XpbdModel(C.Structure):
    _fields_ = [("n_vertices", C.c_int32), ("rest_x", _fp), ("inv_mass", _fp),
                ("n_dist", C.c_int32), ("dist_idx", _ip), ("n_bend", C.c_int32), ("bend_idx", _ip),
                ("n_tet", C.c_int32), ("tet_idx", _ip), ("tet_gamma", _fp),
                ("n_colors", C.c_int32), ("color_offsets", _ip), ("color_order", _ip),
                ("exec_mode", C.c_int32), ("tet_coupled", C.c_int32),
                ("n_memb", C.c_int32), ("memb_idx", _ip), ("memb_uv", _fp)]


class XpbdParams(C.Structure):
    _fields_ = [("dt", C.c_float), ("gravity", C.c_float * 3), ("compliance", C.c_void_p),
                ("f_global", C.c_void_p), ("f_vertex", C.c_void_p), ("collider_flags", C.c_int32),
                ("plane_h", C.c_float), ("sphere", C.c_float * 4),
                ("contact_compliance", C.c_float), ("thickness", C.c_float), ("f_vertex_steps", C.c_void_p),
                ("memb_stiffness", C.c_void_p)]


class XpbdGrads(C.Structure):
    _fields_ = [("d_compliance", C.c_void_p), ("d_x0", C.c_void_p), ("d_v0", C.c_void_p),
                ("d_f_global", C.c_void_p), ("d_f_vertex", C.c_void_p), ("d_collider", C.c_void_p),
                ("d_f_vertex_steps", C.c_void_p), ("d_memb_stiffness", C.c_void_p)]


class XpbdImplicitOpts(C.Structure):
    _fields_ = [("cg_tol", C.c_double), ("cg_max_iters", C.c_int32), ("pd_project", C.c_int32),
                ("cg_iters_out", _ip), ("mg_nx", C.c_int32), ("mg_ny", C.c_int32), ("mg_lines", C.c_int32),
                ("mg_sweeps", C.c_int32)]


KERNEL_CLASSES = ("fwd_dist", "fwd_bend", "fwd_tet_h", "fwd_tet_d", "fwd_contact",
                  "replay_dist", "replay_bend", "replay_tet_h", "replay_tet_d", "replay_contact",
                  "vjp_dist", "vjp_bend", "vjp_tet_h", "vjp_tet_d", "vjp_contact",
                  "predict", "velocity", "adjoint_other", "other", "fwd_phase", "replay_phase", "vjp_phase",
                  "fwd_memb", "replay_memb", "vjp_memb")


class XpbdKernelStat(C.Structure):
    _fields_ = [("launches", C.c_int64), ("units", C.c_int64), ("ms", C.c_double),
                ("timed_launches", C.c_int64), ("alg_bytes", C.c_double)]


class XpbdRequest(C.Structure):
    _fields_ = [("handle", C.c_void_p), ("params", XpbdParams), ("steps", C.c_int32), ("iters", C.c_int32),
                ("x0", C.c_void_p), ("v0", C.c_void_p), ("target", C.c_void_p), ("loss_out", C.c_void_p),
                ("grads", XpbdGrads)]


class XpbdServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("admitted", C.c_int64), ("completed", C.c_int64),
                ("pending", C.c_int32), ("active", C.c_int32), ("bytes_in_use", C.c_size_t),
                ("budget", C.c_size_t), ("ticks", C.c_int64), ("items", C.c_int64), ("batches", C.c_int64),
                ("host_wait_s", C.c_double), ("host_build_s", C.c_double)]


class XpbdError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                               "(run __graft_entry__.build()); there is no CPU fallback")
        L = C.CDLL(LIB_PATH)
        for name in ("xpbd_create", "xpbd_destroy", "xpbd_sizes", "xpbd_forward", "xpbd_read_state",
                     "xpbd_loss", "xpbd_adjoint", "xpbd_sync_status", "xpbd_profile", "xpbd_profile_read", "xpbd_forward_static",
                     "xpbd_server_create", "xpbd_server_destroy", "xpbd_server_submit", "xpbd_server_run",
                     "xpbd_server_poll", "xpbd_server_get_stats", "xpbd_exec_info",
                     "xpbd_selftest_wait_timeout", "xpbd_forward_sparse", "xpbd_adjoint_sparse",
                     "xpbd_sparse_slots", "xpbd_sparse_slot", "xpbd_adjoint_implicit",
                     "xpbd_material_compliance", "xpbd_material_gradient", "xpbd_release_workspace"):
            getattr(L, name).restype = C.c_int
        L.xpbd_checkpoint_bytes.restype = C.c_size_t
        L.xpbd_checkpoint_bytes.argtypes = [C.c_void_p, C.c_int32]
        L.xpbd_workspace_bytes.restype = C.c_size_t
        L.xpbd_workspace_bytes.argtypes = [C.c_void_p, C.c_int32]
        L.xpbd_last_error.restype = C.c_char_p
        L.xpbd_request_bytes.restype = C.c_size_t
        L.xpbd_request_bytes.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_int32]
        _lib = L
    return _lib


def _check(st: int):
    if st != XPBD_OK:
        raise XpbdError(st, lib().xpbd_last_error().decode())


def _stream(stream=None) -> C.c_void_p:
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


F32, F64, I32 = torch.float32, torch.float64, torch.int32


def _ptr(t: Optional[torch.Tensor], dtype: Optional[torch.dtype] = None):
    """Device pointer of a contiguous CUDA tensor (of `dtype`, when given: the C ABI reads
    raw memory, so a tensor of another type would be misread, not converted)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected a {dtype} tensor, got {t.dtype}")
    return C.c_void_p(t.data_ptr())


@dataclass
class Params:
    """Per-call parameters (xpbd_params): device tensors plus host scalars."""
    dt: float
    compliance: torch.Tensor                  # [m] float32 cuda
    gravity: Sequence[float] = (0.0, -9.81, 0.0)
    f_global: Optional[torch.Tensor] = None   # [steps,3] float32 cuda
    f_vertex: Optional[torch.Tensor] = None   # [V,3] float32 cuda
    collider_flags: int = 0
    plane_h: float = 0.0
    sphere: Sequence[float] = (0.0, 0.0, 0.0, 0.0)
    contact_compliance: float = 1e-8
    thickness: float = 0.0
    f_vertex_steps: Optional[torch.Tensor] = None   # [steps,V,3] float32 cuda: force per vertex per step
    memb_stiffness: Optional[torch.Tensor] = None   # [n_memb,4] float32 cuda: (C00, C11, C01, C22)

    def c_struct(self) -> XpbdParams:
        for t in (self.compliance, self.f_global, self.f_vertex, self.f_vertex_steps, self.memb_stiffness):
            if t is not None and t.dtype != torch.float32:
                raise ValueError("params tensors must be float32")
        return XpbdParams(dt=self.dt, gravity=(C.c_float * 3)(*self.gravity),
                          compliance=_ptr(self.compliance, F32), f_global=_ptr(self.f_global, F32),
                          f_vertex=_ptr(self.f_vertex, F32), collider_flags=int(self.collider_flags),
                          plane_h=float(self.plane_h), sphere=(C.c_float * 4)(*[float(v) for v in self.sphere]),
                          contact_compliance=float(self.contact_compliance), thickness=float(self.thickness),
                          f_vertex_steps=_ptr(self.f_vertex_steps, F32), memb_stiffness=_ptr(self.memb_stiffness, F32))


def sparse_slots(steps: int, stride: int) -> int:
    """Stored states of a sparse checkpoint buffer (xpbd_sparse_slots); -1 if invalid."""
    return int(lib().xpbd_sparse_slots(int(steps), int(stride)))


def sparse_slot(steps: int, stride: int, step: int) -> int:
    """Slot of `step` in a sparse checkpoint buffer, or -1 if it is not stored."""
    return int(lib().xpbd_sparse_slot(int(steps), int(stride), int(step)))


class Solver:
    """One xpbd_handle: a mesh, its constraints and its coloring, resident on the GPU.

    exec_mode: 0 picks the multi-color phase launches when they cut the launches per
    iteration at least 4-fold, 1 launches one color at a time, 2 uses the phase launches
    whenever the coloring allows any; all three compute the same colored sweep.
    tet_coupled: update each tet's C_H and C_D together by one 2x2 solve; the coloring
    then lists the C_H ids only (``scenes.couple_tets``)."""

    def __init__(self, rest_x, inv_mass, dist_idx=None, bend_idx=None, tet_idx=None, tet_gamma=None,
                 color_offsets=None, color_order=None, exec_mode: int = 0, tet_coupled: bool = False,
                 memb_idx=None, memb_uv=None):
        L = lib()
        keep = []

        def f(a):
            a = np.ascontiguousarray(a, np.float32).reshape(-1)
            keep.append(a)
            return a.ctypes.data_as(_fp)

        def i(a):
            a = np.ascontiguousarray(a, np.int32).reshape(-1)
            keep.append(a)
            return a.ctypes.data_as(_ip)

        z2 = np.zeros((0, 2), np.int32)
        z4 = np.zeros((0, 4), np.int32)
        dist_idx = z2 if dist_idx is None else np.asarray(dist_idx)
        bend_idx = z4 if bend_idx is None else np.asarray(bend_idx)
        tet_idx = z4 if tet_idx is None else np.asarray(tet_idx)
        md = XpbdModel(n_vertices=int(np.asarray(rest_x).shape[0]), rest_x=f(rest_x), inv_mass=f(inv_mass),
                       n_dist=int(dist_idx.shape[0]), dist_idx=i(dist_idx),
                       n_bend=int(bend_idx.shape[0]), bend_idx=i(bend_idx),
                       n_tet=int(tet_idx.shape[0]), tet_idx=i(tet_idx),
                       tet_gamma=f(tet_gamma) if (tet_gamma is not None and len(tet_gamma)) else None,
                       n_colors=int(len(color_offsets) - 1), color_offsets=i(color_offsets),
                       color_order=i(color_order), exec_mode=int(exec_mode),
                       tet_coupled=int(bool(tet_coupled)),
                       n_memb=int(0 if memb_idx is None else np.asarray(memb_idx).shape[0]),
                       memb_idx=i(memb_idx) if memb_idx is not None and len(memb_idx) else None,
                       memb_uv=f(memb_uv) if memb_uv is not None and len(memb_uv) else None)
        h = C.c_void_p()
        _check(L.xpbd_create(C.byref(md), C.byref(h)))
        self._h = h
        nv, nc, ncol = C.c_int32(), C.c_int32(), C.c_int32()
        _check(L.xpbd_sizes(h, C.byref(nv), C.byref(nc), C.byref(ncol)))
        self.V, self.m, self.n_colors = nv.value, nc.value, ncol.value
        self.n_memb = int(md.n_memb)

    @classmethod
    def from_scene(cls, sc, exec_mode: int = 0) -> "Solver":
        return cls(sc.rest_x, sc.inv_mass, sc.dist_idx, sc.bend_idx, sc.tet_idx, sc.tet_gamma,
                   sc.color_offsets, sc.color_order, exec_mode, getattr(sc, "tet_coupled", False),
                   getattr(sc, "memb_idx", None), getattr(sc, "memb_uv", None))

    def exec_info(self) -> dict:
        """{"phases": bool, "launches_per_iteration": int} of the handle's execution plan."""
        u, n = C.c_int32(), C.c_int32()
        _check(lib().xpbd_exec_info(self._h, C.byref(u), C.byref(n)))
        return {"phases": bool(u.value), "launches_per_iteration": n.value}

    def close(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.xpbd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    # -- sizes
    def checkpoint_bytes(self, steps: int) -> int:
        return int(lib().xpbd_checkpoint_bytes(self._h, steps))

    def workspace_bytes(self, iters: int) -> int:
        return int(lib().xpbd_workspace_bytes(self._h, iters))

    def release_workspace(self):
        """xpbd_release_workspace: free the handle's working buffers until its next call."""
        _check(lib().xpbd_release_workspace(self._h))

    def new_checkpoints(self, steps: int, device="cuda") -> torch.Tensor:
        """[(steps+1), 2, V, 4] float32: per step (x,y,z,w) positions then velocities."""
        return torch.empty((steps + 1, 2, self.V, 4), dtype=torch.float32, device=device)

    # -- calls
    def forward(self, params: Params, steps: int, iters: int, x0: torch.Tensor, v0: torch.Tensor,
                checkpoints: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        ck = self.new_checkpoints(steps, x0.device) if checkpoints is None else checkpoints
        p = params.c_struct()
        _check(lib().xpbd_forward(self._h, C.byref(p), int(steps), int(iters), _ptr(x0, F32), _ptr(v0, F32),
                                  _ptr(ck, F32), _stream(stream)))
        return ck

    def forward_sparse(self, params: Params, steps: int, iters: int, x0: torch.Tensor, v0: torch.Tensor,
                       stride: int, checkpoints: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        """xpbd_forward_sparse: stores the state only at every `stride`-th step and the last
        step.  Returns [sparse_slots(steps, stride), 2, V, 4]; slot of step n: sparse_slot()."""
        n = sparse_slots(steps, stride)
        if n < 0:
            raise XpbdError(1, f"bad steps/stride: {steps}/{stride}")
        ck = (torch.empty((n, 2, self.V, 4), dtype=torch.float32, device=x0.device)
              if checkpoints is None else checkpoints)
        p = params.c_struct()
        _check(lib().xpbd_forward_sparse(self._h, C.byref(p), int(steps), int(iters), _ptr(x0, F32), _ptr(v0, F32),
                                         int(stride), _ptr(ck, F32), _stream(stream)))
        return ck

    def forward_static(self, params: Params, steps: int, iters: int, x0: torch.Tensor, v0: torch.Tensor,
                       checkpoints: torch.Tensor, stream=None) -> torch.Tensor:
        """xpbd_forward_static: the forward simulation without any device allocation by the
        library, for callers that cannot allocate while they simulate (the checkpoint buffer
        is the caller's).  Limited to STATIC_MAX_VERTICES vertices and STATIC_MAX_CONSTRAINTS
        multiplier slots (one per constraint, four per membrane); calls
        whose GPU work overlaps on one device race on the library's shared working array."""
        p = params.c_struct()
        _check(lib().xpbd_forward_static(self._h, C.byref(p), int(steps), int(iters), _ptr(x0, F32), _ptr(v0, F32),
                                         _ptr(checkpoints, F32), _stream(stream)))
        return checkpoints

    def read_state(self, checkpoints: torch.Tensor, step: int, stream=None):
        x = torch.empty((self.V, 3), dtype=torch.float32, device=checkpoints.device)
        v = torch.empty_like(x)
        _check(lib().xpbd_read_state(self._h, _ptr(checkpoints, F32), int(step), _ptr(x, F32), _ptr(v, F32), _stream(stream)))
        return x, v

    def loss(self, checkpoints: torch.Tensor, targets: dict, stream=None):
        """targets: {step: [V,3] float32 cuda}.  Returns (loss [1] float64, seeds [k,V,3])."""
        keys = sorted(targets)
        tg = torch.stack([targets[k] for k in keys]).contiguous()
        seeds = torch.empty_like(tg)
        out = torch.empty(1, dtype=torch.float64, device=checkpoints.device)
        ks = (C.c_int32 * len(keys))(*keys)
        _check(lib().xpbd_loss(self._h, _ptr(checkpoints, F32), len(keys), ks, _ptr(tg, F32), _ptr(out, F64),
                               _ptr(seeds, F32), _stream(stream)))
        return out, seeds

    def adjoint(self, params: Params, steps: int, iters: int, checkpoints: torch.Tensor, seeds: dict,
                seed_dv_T: Optional[torch.Tensor] = None, want=("compliance", "x0", "v0", "f_global",
                                                                 "f_vertex", "collider"),
                out: Optional[dict] = None, stream=None, stride: Optional[int] = None) -> dict:
        """seeds: {step: dL/dx_step [V,3] float32 cuda}.  Returns float64 gradients.  With
        `stride`, `checkpoints` is a sparse buffer from forward_sparse with that stride."""
        dev = checkpoints.device
        keys = sorted(seeds)
        sd = torch.stack([seeds[k] for k in keys]).contiguous() if keys else None
        shapes = dict(compliance=(self.m,), x0=(self.V, 3), v0=(self.V, 3), f_global=(max(steps, 1), 3),
                      f_vertex=(self.V, 3), collider=(5,), f_vertex_steps=(max(steps, 1), self.V, 3),
                      memb_stiffness=(self.n_memb, 4))
        if out is None:
            out = {k: torch.empty(shapes[k], dtype=torch.float64, device=dev) for k in want}
        g = XpbdGrads(d_compliance=_ptr(out.get("compliance"), F64), d_x0=_ptr(out.get("x0"), F64),
                      d_v0=_ptr(out.get("v0"), F64), d_f_global=_ptr(out.get("f_global"), F64),
                      d_f_vertex=_ptr(out.get("f_vertex"), F64), d_collider=_ptr(out.get("collider"), F64),
                      d_f_vertex_steps=_ptr(out.get("f_vertex_steps"), F64),
                      d_memb_stiffness=_ptr(out.get("memb_stiffness"), F64))
        p = params.c_struct()
        ks = (C.c_int32 * max(len(keys), 1))(*keys)
        if stride is None:
            _check(lib().xpbd_adjoint(self._h, C.byref(p), int(steps), int(iters), _ptr(checkpoints, F32),
                                      len(keys), ks, _ptr(sd, F32), _ptr(seed_dv_T, F32), C.byref(g), _stream(stream)))
        else:
            _check(lib().xpbd_adjoint_sparse(self._h, C.byref(p), int(steps), int(iters), _ptr(checkpoints, F32),
                                             int(stride), len(keys), ks, _ptr(sd, F32), _ptr(seed_dv_T, F32), C.byref(g),
                                             _stream(stream)))
        return out

    def adjoint_implicit(self, params: Params, steps: int, iters: int, checkpoints: torch.Tensor, seeds: dict,
                         seed_dv_T: Optional[torch.Tensor] = None,
                         want=("compliance", "x0", "v0", "f_global", "f_vertex"), cg_tol: float = 1e-10,
                         cg_max_iters: int = 5000, pd_project: bool = True, multigrid=None, stream=None):
        """The paper's implicit adjoint (xpbd_adjoint_implicit).  Returns (float64 gradients,
        conjugate-gradient iterations per step).  `multigrid` = (nx, ny[, lines[, sweeps]])
        preconditions the solve with the grid multigrid V-cycle (block Jacobi when None)."""
        dev = checkpoints.device
        keys = sorted(seeds)
        sd = torch.stack([seeds[k] for k in keys]).contiguous() if keys else None
        shapes = dict(compliance=(self.m,), x0=(self.V, 3), v0=(self.V, 3), f_global=(max(steps, 1), 3),
                      f_vertex=(self.V, 3), f_vertex_steps=(max(steps, 1), self.V, 3), memb_stiffness=(self.n_memb, 4))
        out = {k: torch.empty(shapes[k], dtype=torch.float64, device=dev) for k in want}
        g = XpbdGrads(d_compliance=_ptr(out.get("compliance"), F64), d_x0=_ptr(out.get("x0"), F64),
                      d_v0=_ptr(out.get("v0"), F64), d_f_global=_ptr(out.get("f_global"), F64),
                      d_f_vertex=_ptr(out.get("f_vertex"), F64), d_collider=None,
                      d_f_vertex_steps=_ptr(out.get("f_vertex_steps"), F64),
                      d_memb_stiffness=_ptr(out.get("memb_stiffness"), F64))
        its = (C.c_int32 * max(steps, 1))()
        mg = tuple(multigrid) + (0, 0) if multigrid else (0, 0, 0, 0)
        o = XpbdImplicitOpts(cg_tol=float(cg_tol), cg_max_iters=int(cg_max_iters), pd_project=int(bool(pd_project)),
                             cg_iters_out=C.cast(its, _ip), mg_nx=int(mg[0]), mg_ny=int(mg[1]), mg_lines=int(mg[2]),
                             mg_sweeps=int(mg[3]))
        p = params.c_struct()
        ks = (C.c_int32 * max(len(keys), 1))(*keys)
        _check(lib().xpbd_adjoint_implicit(self._h, C.byref(p), int(steps), int(iters), _ptr(checkpoints, F32),
                                           len(keys), ks, _ptr(sd, F32), _ptr(seed_dv_T, F32), C.byref(g), C.byref(o),
                                           _stream(stream)))
        return out, list(its)[:steps]

    def material_compliance(self, tet_material: torch.Tensor, a: torch.Tensor, b: torch.Tensor,
                            compliance: torch.Tensor, stream=None) -> torch.Tensor:
        """Writes the tet entries of `compliance` from materials mu = a^2, lambda = b^2
        (xpbd_material_compliance); returns `compliance`."""
        _check(lib().xpbd_material_compliance(self._h, int(a.numel()), _ptr(tet_material, I32), _ptr(a, F32), _ptr(b, F32),
                                              _ptr(compliance, F32), _stream(stream)))
        return compliance

    def material_gradient(self, tet_material: torch.Tensor, a: torch.Tensor, b: torch.Tensor,
                          d_compliance: torch.Tensor, stream=None):
        """(dL/da, dL/db) float64 from a compliance gradient (xpbd_material_gradient)."""
        da = torch.empty(a.numel(), dtype=torch.float64, device=a.device)
        db = torch.empty_like(da)
        _check(lib().xpbd_material_gradient(self._h, int(a.numel()), _ptr(tet_material, I32), _ptr(a, F32), _ptr(b, F32),
                                            _ptr(d_compliance, F64), _ptr(da, F64), _ptr(db, F64), _stream(stream)))
        return da, db

    def sync_status(self, stream=None):
        _check(lib().xpbd_sync_status(self._h, _stream(stream)))

    def selftest_wait_timeout(self, stream=None):
        """Queue one phase-kernel CTA whose bounded waits all run out (its producer issues
        no copies); the next sync_status() raises XPBD_ERR_TIMEOUT."""
        _check(lib().xpbd_selftest_wait_timeout(self._h, _stream(stream)))

    def profile(self, enable: bool = True):
        """Reset the launch counters; time every launch with CUDA events while enabled."""
        _check(lib().xpbd_profile(self._h, int(bool(enable))))

    def profile_read(self) -> dict:
        """{class: {launches, units, ms, timed_launches}} since the last profile() call."""
        arr = (XpbdKernelStat * len(KERNEL_CLASSES))()
        _check(lib().xpbd_profile_read(self._h, arr))
        return {n: dict(launches=a.launches, units=a.units, ms=a.ms, timed_launches=a.timed_launches,
                        alg_bytes=a.alg_bytes) for n, a in zip(KERNEL_CLASSES, arr)}


def params_from_scene(sc, device="cuda", compliance=None) -> Params:
    """Device params of a scenes.Scene (uploads compliance and forces as float32)."""
    t = lambda a: None if a is None else torch.as_tensor(np.asarray(a, np.float32), device=device).contiguous()
    return Params(dt=float(sc.dt), compliance=t(sc.compliance if compliance is None else compliance),
                  gravity=tuple(float(g) for g in sc.gravity), f_global=t(sc.f_global), f_vertex=t(sc.f_vertex),
                  collider_flags=int(sc.collider_flags), plane_h=float(sc.plane_h),
                  sphere=tuple(float(v) for v in sc.sphere), contact_compliance=float(sc.contact_compliance),
                  thickness=float(sc.thickness), f_vertex_steps=t(getattr(sc, "f_vertex_steps", None)),
                  memb_stiffness=t(sc.memb_stiffness) if getattr(sc, "n_memb", 0) else None)


class XPBDSolve(torch.autograd.Function):
    """Differentiable XPBD rollout: positions at the key steps as a function of
    (compliance, x0, v0, f_global, f_vertex, collider = [plane_h, cx, cy, cz, r]).
    backward runs the library's reverse sweep; float64 gradients are cast to each input's
    dtype."""

    @staticmethod
    def forward(ctx, solver: Solver, cfg: dict, key_steps: tuple, compliance, x0, v0, f_global,
                f_vertex, collider):
        steps, iters = cfg["steps"], cfg["iters"]
        col = [float(v) for v in collider.detach().cpu().tolist()] if collider is not None else [0.0] * 5
        p = Params(dt=cfg["dt"], compliance=compliance.detach().contiguous(), gravity=cfg.get("gravity", (0, -9.81, 0)),
                   f_global=None if f_global is None else f_global.detach().contiguous(),
                   f_vertex=None if f_vertex is None else f_vertex.detach().contiguous(),
                   collider_flags=cfg.get("collider_flags", 0), plane_h=col[0], sphere=col[1:5],
                   contact_compliance=cfg.get("contact_compliance", 1e-8), thickness=cfg.get("thickness", 0.0))
        ck = solver.forward(p, steps, iters, x0.detach().contiguous(), v0.detach().contiguous())
        outs = [solver.read_state(ck, k)[0] for k in key_steps]
        ctx.save_for_backward(ck)
        ctx.solver, ctx.params, ctx.cfg, ctx.key_steps = solver, p, cfg, key_steps
        ctx.dtypes = [None if t is None else t.dtype for t in (compliance, x0, v0, f_global, f_vertex, collider)]
        ctx.devices = [None if t is None else t.device for t in (compliance, x0, v0, f_global, f_vertex, collider)]
        return tuple(outs)

    @staticmethod
    def backward(ctx, *grads):
        (ck,) = ctx.saved_tensors
        seeds = {}
        for k, g in zip(ctx.key_steps, grads):
            if g is None:
                continue
            g = g.to(torch.float32).contiguous()
            seeds[k] = seeds[k] + g if k in seeds else g
        want = [n for n, t in zip(("compliance", "x0", "v0", "f_global", "f_vertex", "collider"), ctx.dtypes)
                if t is not None]
        gr = ctx.solver.adjoint(ctx.params, ctx.cfg["steps"], ctx.cfg["iters"], ck, seeds, want=tuple(want))
        res = []
        for name, dt, dev in zip(("compliance", "x0", "v0", "f_global", "f_vertex", "collider"), ctx.dtypes,
                                 ctx.devices):
            res.append(None if dt is None else gr[name].to(device=dev, dtype=dt))
        return (None, None, None, *res)


def simulate(solver: Solver, cfg: dict, compliance, x0, v0, f_global=None, f_vertex=None, collider=None,
             key_steps=None):
    """Autograd entry point: returns the positions [V,3] at each key step (default: the last)."""
    ks = (cfg["steps"],) if key_steps is None else tuple(key_steps)
    return XPBDSolve.apply(solver, cfg, ks, compliance, x0, v0, f_global, f_vertex, collider)


class Server:
    """Continuous-batching server (xpbd_server_*): forward + loss + full reverse sweep per
    request, with every resident request advanced by each launch of the dispatch kernel.

    submit() keeps references to the request's tensors (and allocates its float64 outputs)
    until poll() reports it done; result() then returns {"loss": [1], <gradient groups>}."""

    def __init__(self, budget: int = 0, max_slots: int = 64, stream=None):
        self._stream = torch.cuda.current_stream() if stream is None else stream
        s = C.c_void_p()
        _check(lib().xpbd_server_create(C.c_size_t(int(budget)), int(max_slots), C.c_void_p(self._stream.cuda_stream),
                                        C.byref(s)))
        self._s = s
        self._live = {}
        self._done = {}

    def close(self):
        if getattr(self, "_s", None) is not None and _lib is not None:
            _lib.xpbd_server_destroy(self._s)
            self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def request_bytes(solver: "Solver", steps: int, iters: int, collider_flags: int = 0) -> int:
        return int(lib().xpbd_request_bytes(solver.handle, int(steps), int(iters), int(collider_flags)))

    def submit(self, solver: "Solver", params: Params, steps: int, iters: int, x0: torch.Tensor, v0: torch.Tensor,
               target: torch.Tensor, want=("compliance", "x0", "v0")) -> int:
        dev = x0.device
        shapes = dict(compliance=(solver.m,), x0=(solver.V, 3), v0=(solver.V, 3), f_global=(max(steps, 1), 3),
                      f_vertex=(solver.V, 3), collider=(5,))
        out = {k: torch.empty(shapes[k], dtype=torch.float64, device=dev) for k in want}
        out["loss"] = torch.empty(1, dtype=torch.float64, device=dev)
        g = XpbdGrads(d_compliance=_ptr(out.get("compliance"), F64), d_x0=_ptr(out.get("x0"), F64), d_v0=_ptr(out.get("v0"), F64),
                      d_f_global=_ptr(out.get("f_global"), F64), d_f_vertex=_ptr(out.get("f_vertex"), F64),
                      d_collider=_ptr(out.get("collider"), F64))
        req = XpbdRequest(handle=solver.handle, params=params.c_struct(), steps=int(steps), iters=int(iters),
                          x0=_ptr(x0, F32), v0=_ptr(v0, F32), target=_ptr(target, F32), loss_out=_ptr(out["loss"], F64), grads=g)
        t = C.c_uint64()
        _check(lib().xpbd_server_submit(self._s, C.byref(req), C.byref(t)))
        self._live[t.value] = (solver, params, x0, v0, target, out)
        return t.value

    def run(self, max_ticks: int = 64) -> int:
        active = C.c_int32()
        _check(lib().xpbd_server_run(self._s, int(max_ticks), C.byref(active)))
        return active.value

    def poll(self, ticket: int) -> bool:
        if ticket in self._done:
            return True
        d = C.c_int32()
        _check(lib().xpbd_server_poll(self._s, C.c_uint64(ticket), C.byref(d)))
        if d.value:
            self._done[ticket] = self._live.pop(ticket)[-1]
        return bool(d.value)

    def result(self, ticket: int) -> dict:
        return self._done[ticket]

    def drain(self, tickets, max_ticks: int = 64):
        """Run until every ticket in `tickets` is done."""
        pending = [t for t in tickets if t not in self._done]
        while pending:
            self.run(max_ticks)
            pending = [t for t in pending if not self.poll(t)]

    def stats(self) -> dict:
        st = XpbdServerStats()
        _check(lib().xpbd_server_get_stats(self._s, C.byref(st)))
        return {f: getattr(st, f) for f, _ in XpbdServerStats._fields_}
