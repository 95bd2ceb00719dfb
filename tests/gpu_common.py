"""Shared helpers of the GPU parity tests: run a scene through the C ABI and the oracle on
identical (FP32-representable) inputs."""
import numpy as np
import torch

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
