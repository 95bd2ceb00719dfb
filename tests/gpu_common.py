"""Shared helpers of the GPU parity tests: run a scene through the C ABI and the oracle on
identical (FP32-representable) inputs."""
import numpy as np
import torch

import oracle

from paper_2301_01396_gb300 import binding, scenes

GRAD_KEYS = ("compliance", "x0", "v0", "f_global", "f_vertex", "collider")


def to_dev(a):
    return torch.as_tensor(np.asarray(a, np.float32), device="cuda").contiguous()


def gpu_forward(sc, steps=None, iters=None, solver=None):
    steps = sc.steps if steps is None else steps
    iters = sc.iters if iters is None else iters
    solver = solver or binding.Solver.from_scene(sc)
    p = binding.params_from_scene(sc)
    ck = solver.forward(p, steps, iters, to_dev(sc.x0), to_dev(sc.v0))
    torch.cuda.synchronize()
    solver.sync_status()
    ckn = ck.cpu().numpy().astype(np.float64)
    return solver, p, ck, ckn[:, 0, :, :3], ckn[:, 1, :, :3]


def gpu_adjoint(sc, seeds, steps=None, iters=None):
    steps = sc.steps if steps is None else steps
    iters = sc.iters if iters is None else iters
    solver, p, ck, xs, vs = gpu_forward(sc, steps, iters)
    gr = solver.adjoint(p, steps, iters, ck, {k: to_dev(v) for k, v in seeds.items()})
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in gr.items()}, xs


def rel_err(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


# Element-wise gradient bound.  Every entry j of a gradient group must satisfy
#   |g_j - r_j| <= ELEM_TOL * (|r_j| + ELEM_FLOOR * max_i |r_i|),
# i.e. 2 % relative error for entries within three decades of the group's largest, and an
# absolute 2e-5 * max|r| below that.  The group-norm bound (1e-3) can hide a wrong
# gradient on a few boundary hinges, pinned-vertex springs or contact vertices under large
# entries; a wrong update there is O(1) relative, 50x this bound.  Entries far below the
# group's scale carry float32 cancellation of large terms (their absolute error is set by
# the group's scale, not their own), hence the floor.
ELEM_TOL = 2e-2
ELEM_FLOOR = 1e-3


def elem_err(a, b, floor=ELEM_FLOOR):
    """max_j |a_j - b_j| / (|b_j| + floor * max|b|): the worst entry's error relative to its
    own size, floored at `floor` times the group's largest entry."""
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    if a.size == 0:
        return 0.0
    s = np.abs(b).max()
    if s == 0:
        return float(np.abs(a).max())
    return float(np.max(np.abs(a - b) / (np.abs(b) + floor * s)))


# Where float32 rounding moves a gradient past the bounds above (stiff constraints,
# strains near float32 resolution, compliance gradients of nearly slack constraints), the
# bounds become these multiples of the "floor": the same errors of the oracle's own
# float32-rounding emulation (oracle.fp32_rounding).  The emulation rounds the state
# (positions, multipliers) after every projection; the GPU also rounds every intermediate
# and runs the reverse sweep in float32, so its errors exceed the floor somewhat (measured:
# 1.0-1.65x in L2, up to 2.3x per entry, on the stiff membranes); a wrong update is orders
# of magnitude beyond.
FLOOR_FACTOR = 2.0
ELEM_FLOOR_FACTOR = 3.0


def oracle_adjoint_floor(sc, seeds, *args, **kw):
    """The oracle's gradients, and the same from its float32-rounding emulation."""
    ref = oracle.adjoint(sc, seeds, *args, **kw)
    with oracle.fp32_rounding():
        ref32 = oracle.adjoint(sc, seeds, *args, **kw)
    return ref, ref32


def check_grad(tag, got, ref, tol=1e-3, elem_tol=ELEM_TOL, ref32=None):
    """Assert a gradient group against the oracle's: relative L2 error below `tol` and every
    entry within the element-wise bound (with `ref32`, the oracle's float32-rounding run,
    both bounds are at least FLOOR_FACTOR / ELEM_FLOOR_FACTOR times its errors).  Prints
    the errors (one PARITY line per group)."""
    got = np.asarray(got, np.float64).reshape(np.shape(ref))
    e, ee = rel_err(got, ref), elem_err(got, ref)
    msg = f"PARITY {tag}: rel {e:.3e} elem {ee:.3e}"
    if ref32 is not None:
        ref32 = np.asarray(ref32, np.float64).reshape(np.shape(ref))
        f, fe = rel_err(ref32, ref), elem_err(ref32, ref)
        tol, elem_tol = max(tol, FLOOR_FACTOR * f), max(elem_tol, ELEM_FLOOR_FACTOR * fe)
        msg += f" (float32 floor: rel {f:.3e} elem {fe:.3e})"
    print(msg)
    assert e < tol, f"{tag}: relative error {e:.3e} (bound {tol:.3e})"
    assert ee < elem_tol, f"{tag}: element-wise error {ee:.3e} (bound {elem_tol:.3e})"
    return e, ee


def _contact_values(sc, xs, vs):
    out = []
    g = np.asarray(sc.gravity)
    for n in range(xs.shape[0] - 1):
        f = np.zeros_like(xs[n])
        if sc.f_global is not None:
            f += sc.f_global[n]
        if sc.f_vertex is not None:
            f += sc.f_vertex
        w = sc.inv_mass[:, None]
        p = xs[n] + sc.dt * vs[n] + sc.dt ** 2 * (w * f + (w > 0) * g)
        if sc.collider_flags & scenes.COLLIDE_PLANE:
            out.append(p[:, 1] - sc.plane_h - sc.thickness)
        if sc.collider_flags & scenes.COLLIDE_SPHERE:
            c = np.asarray(sc.sphere[:3])
            out.append(np.linalg.norm(p - c, axis=1) - sc.sphere[3] - sc.thickness)
    return np.concatenate(out) if out else np.zeros(0)


def contact_signs_agree(sc, xs, vs, xs_ref, vs_ref):
    """The contact tests C(p) < 0 evaluated on the GPU trajectory and on the oracle's give
    the same activity for every vertex and step."""
    a, b = _contact_values(sc, xs, vs), _contact_values(sc, xs_ref, vs_ref)
    return bool(np.all((a < 0) == (b < 0)))


def contact_margin(sc, xs, vs):
    """Smallest |C(p)| of the contact tests over all steps (FP64 oracle trajectory): the
    activity decisions of FP32 and FP64 agree when this is well above rounding level."""
    if not sc.collider_flags:
        return np.inf
    m = np.inf
    g = np.asarray(sc.gravity)
    for n in range(xs.shape[0] - 1):
        f = np.zeros_like(xs[n])
        if sc.f_global is not None:
            f += sc.f_global[n]
        if sc.f_vertex is not None:
            f += sc.f_vertex
        w = sc.inv_mass[:, None]
        p = xs[n] + sc.dt * vs[n] + sc.dt ** 2 * (w * f + (w > 0) * g)
        if sc.collider_flags & scenes.COLLIDE_PLANE:
            m = min(m, np.abs(p[:, 1] - sc.plane_h - sc.thickness).min())
        if sc.collider_flags & scenes.COLLIDE_SPHERE:
            c = np.asarray(sc.sphere[:3])
            m = min(m, np.abs(np.linalg.norm(p - c, axis=1) - sc.sphere[3] - sc.thickness).min())
    return m
