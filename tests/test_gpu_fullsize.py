"""Parity at the full sizes of the cloth, ground-cloth, tet-block and 2950^2 sphere-cloth
workloads, in the launch configuration bench.py times (per-color kernels, 256-thread
blocks over whole colors).

The 256^2 cloth (325,125 constraints) and the 32^3 tet block (327,680 constraints) run in
the oracle at full size.  The 2950^2 cloth (52,179,606 constraints) is compared on a
window: every color pass moves information at most two vertices (a bending hinge spans
rows j-1..j+1), so after I iterations of K color passes the vertices farther than
R = 2 K I from a window's edge do not see that edge, and the oracle run on the window
reproduces the full run there.  Gradients are compared where seeds and their reverse
propagation stay R away from the edge."""
import numpy as np
import pytest
import torch

import oracle
from paper_2301_01396_gb300 import binding, scenes
from tests.gpu_common import contact_margin, contact_signs_agree, gpu_forward, rel_err, to_dev

pytestmark = pytest.mark.gpu

POS_TOL = 1e-5
GRAD_TOL = 1e-3


def _at_state(sc, xs, vs, n, steps, iters=None):
    """The scene restarted from the (FP32-rounded) oracle state of step n."""
    fg = None if sc.f_global is None else sc.f_global[n:n + steps]
    return sc.with_(x0=scenes.f32(xs[n]), v0=scenes.f32(vs[n]), steps=steps,
                    iters=sc.iters if iters is None else iters, f_global=fg)


def _grad_parity(sc, seeds, keys=("compliance", "x0", "v0")):
    ref = oracle.adjoint(sc, seeds)
    solver, p, ck, xs, _ = gpu_forward(sc)
    got = solver.adjoint(p, sc.steps, sc.iters, ck, {k: to_dev(v) for k, v in seeds.items()})
    torch.cuda.synchronize()
    for k in keys:
        e = rel_err(got[k].cpu().numpy().reshape(ref[k].shape), ref[k])
        assert e < GRAD_TOL, f"{k}: relative error {e:.3e}"


def test_ground_cloth_256_forward_first_steps():
    sc = scenes.ground_cloth(256, steps=8)
    xs_ref, _ = oracle.forward(sc)
    _, _, _, xs, _ = gpu_forward(sc)
    assert np.abs(xs - xs_ref).max() < POS_TOL


def test_ground_cloth_256_contact_regime():
    """From the oracle state of step 15, when the tilted cloth's low edge reaches the
    ground: forward over steps 15-18 and the reverse sweep over steps 16-18.  Over this
    window every contact test is at least 1e-5 away from its decision boundary."""
    sc = scenes.ground_cloth(256, steps=18)
    xs, vs = oracle.forward(sc)
    start = 15
    sub = _at_state(sc, xs, vs, start, 3)
    xs_ref, vs_ref = oracle.forward(sub)
    assert (xs_ref[-1, :, 1] <= sc.plane_h + 1e-6).sum() > 100        # contacts are active
    assert contact_margin(sub, xs_ref, vs_ref) > 1e-5
    _, _, _, xg, vg = gpu_forward(sub)
    assert contact_signs_agree(sub, xg, vg, xs_ref, vs_ref)
    assert np.abs(xg - xs_ref).max() < POS_TOL
    sub2 = _at_state(sc, xs, vs, start + 1, 2)
    rng = np.random.default_rng(2)
    _grad_parity(sub2, {2: scenes.f32(rng.standard_normal((sc.V, 3)))})


def test_tet_block_32_forward_to_contact():
    sc = scenes.tet_block(32, steps=16)
    xs_ref, vs_ref = oracle.forward(sc)
    assert (xs_ref[-1, :, 1] <= sc.plane_h + 1e-6).sum() > 100
    assert contact_margin(sc, xs_ref, vs_ref) > 1e-6
    _, _, _, xs, vs = gpu_forward(sc)
    assert contact_signs_agree(sc, xs, vs, xs_ref, vs_ref)
    assert np.abs(xs - xs_ref).max() < POS_TOL


def test_tet_block_32_adjoint_in_contact():
    sc = scenes.tet_block(32, steps=15)
    xs, vs = oracle.forward(sc)
    sub = _at_state(sc, xs, vs, 13, 2)
    rng = np.random.default_rng(3)
    _grad_parity(sub, {2: scenes.f32(rng.standard_normal((sc.V, 3)))})


# --------------------------------------------------------------------------- 2950^2 cloth

def _window(full, n, i0, j0, w):
    """The sub-scene of an n x n grid scene on vertices i0 <= i < i0+w, j0 <= j < j0+w,
    keeping every constraint whose vertices all lie inside, in the same color order."""
    ii = np.arange(full.V) % n
    jj = np.arange(full.V) // n
    inside = (ii >= i0) & (ii < i0 + w) & (jj >= j0) & (jj < j0 + w)
    local = np.full(full.V, -1, np.int64)
    local[inside] = (jj[inside] - j0) * w + (ii[inside] - i0)
    keep_d = inside[full.dist_idx].all(1)
    keep_b = inside[full.bend_idx].all(1)
    nd, nb = int(keep_d.sum()), int(keep_b.sum())
    new_id = np.full(full.m, -1, np.int64)
    new_id[:full.n_dist][keep_d] = np.arange(nd)
    new_id[full.n_dist:][keep_b] = nd + np.arange(nb)
    offs = [0]
    order = []
    for c in range(full.n_colors):
        ids = full.color_order[full.color_offsets[c]:full.color_offsets[c + 1]]
        ids = new_id[ids]
        ids = ids[ids >= 0]
        order.append(ids)
        offs.append(offs[-1] + ids.shape[0])
    sel = np.nonzero(inside)[0][np.argsort(local[inside])]
    comp = np.concatenate([full.compliance[:full.n_dist][keep_d], full.compliance[full.n_dist:][keep_b]])
    sub = full.with_(rest_x=full.rest_x[sel], inv_mass=full.inv_mass[sel],
                     dist_idx=local[full.dist_idx[keep_d]].astype(np.int32),
                     bend_idx=local[full.bend_idx[keep_b]].astype(np.int32),
                     color_offsets=np.asarray(offs, np.int32),
                     color_order=np.concatenate(order).astype(np.int32),
                     x0=full.x0[sel], v0=full.v0[sel], compliance=comp,
                     f_vertex=None if full.f_vertex is None else full.f_vertex[sel])
    return sub, sel, np.nonzero(keep_d)[0], full.n_dist + np.nonzero(keep_b)[0]


@pytest.fixture(scope="module")
def big_cloth():
    return scenes.sphere_cloth(2950, steps=1, iters=15)


def test_sphere_cloth_2950_forward_window(big_cloth):
    full = big_cloth
    n, I = 2950, 15
    R = 2 * 16 * I + 4
    w = 2 * R + 64
    i0 = j0 = (n - w) // 2
    sub, sel, _, _ = _window(full, n, i0, j0, w)
    xs_ref, _ = oracle.forward(sub, 1, I)
    _, _, _, xs, _ = gpu_forward(full, 1, I)
    core = np.zeros((w, w), bool)
    core[R:w - R, R:w - R] = True
    core = core.reshape(-1)
    err = np.abs(xs[1][sel][core] - xs_ref[1][core]).max()
    assert err < POS_TOL, err
    assert core.sum() >= 64 * 64


def test_sphere_cloth_2950_adjoint_window(big_cloth):
    """Reverse sweep over one step of 3 iterations; the seed lives on a core 3R from the
    window edge, gradients are compared on the band within R of that core.

    At this resolution (3.4e-4 m edges, coordinates near 0.5 m) float32 state rounding
    alone moves the compliance gradient by a few percent: the strains it depends on are
    near float32 resolution.  The compliance tolerance is therefore max(1e-3, 4 x floor),
    where the floor is the oracle's own change when its state is rounded to float32
    (oracle.fp32_rounding)."""
    full = big_cloth
    n, I = 2950, 3
    R = 2 * 16 * I + 4
    w = 6 * R + 48
    i0, j0 = 1200, 1400
    sub, sel, kd, kb = _window(full, n, i0, j0, w)
    rng = np.random.default_rng(5)
    li, lj = np.meshgrid(np.arange(w), np.arange(w), indexing="xy")
    dist_edge = np.minimum(np.minimum(li, w - 1 - li), np.minimum(lj, w - 1 - lj)).reshape(-1)
    seed_local = scenes.f32(rng.standard_normal((sub.V, 3)) * (dist_edge >= 3 * R)[:, None])
    ref = oracle.adjoint(sub, {1: seed_local}, 1, I)
    seed_full = np.zeros((full.V, 3), np.float32)
    seed_full[sel] = seed_local
    solver, p, ck, _, _ = gpu_forward(full, 1, I)
    got = solver.adjoint(p, 1, I, ck, {1: to_dev(seed_full)})
    torch.cuda.synchronize()
    band = dist_edge >= 2 * R
    for k in ("x0", "v0", "f_vertex"):
        g = got[k].cpu().numpy()[sel][band]
        assert rel_err(g, ref[k][band]) < GRAD_TOL, k
    # everything outside the window is untouched by the seed
    outside = np.ones(full.V, bool)
    outside[sel] = False
    assert np.abs(got["x0"].cpu().numpy()[outside]).max() == 0.0
    gc = got["compliance"].cpu().numpy()
    ids = np.concatenate([kd, kb])
    with oracle.fp32_rounding():
        ref32 = oracle.adjoint(sub, {1: seed_local}, 1, I)
    floor = rel_err(ref32["compliance"], ref["compliance"])
    err = rel_err(gc[ids], ref["compliance"])
    print(f"2950^2 window: compliance-gradient error {err:.3e}, float32 rounding floor {floor:.3e}")
    assert err < max(GRAD_TOL, 4.0 * floor), (err, floor)
    assert rel_err(got["f_global"].cpu().numpy()[:1], ref["f_global"]) < GRAD_TOL


def test_membrane_cloth_256_full_size():
    """The material-estimation membrane workload at its full size (65,536 vertices, 130,050
    StVK triangles + 129,540 hinges, 8x8-tile coloring, 30 iterations) in the phase
    kernels bench.py times, over one step, with a smooth start velocity field (0.3 m/s, one
    wavelength across the sheet) so that the sheet strains and every gradient group is
    nonzero (the bench's flat fall keeps it strain-free for 20 steps).  The stiff
    membranes (K ~ 1e3 N/m on 4 mm triangles) amplify float32 rounding in the reverse
    sweep to ~9e-4, so the gradient bound is max(1e-3, 4 x floor) with the floor measured
    by the oracle's float32 emulation."""
    sc = scenes.membrane_cloth(256, pins=(), steps=1, iters=30, seed=9, coloring="tiled", tile=8)
    sc.collider_flags = scenes.COLLIDE_PLANE
    sc.plane_h = -0.6
    x, z = sc.x0[:, 0], sc.x0[:, 2]
    sc.v0 = scenes.f32(0.3 * np.stack([np.sin(2 * np.pi * z + 0.3), np.sin(2 * np.pi * (x + z)),
                                        np.cos(2 * np.pi * x - 0.7)], axis=1))
    solver = binding.Solver.from_scene(sc)
    assert solver.exec_info()["phases"]
    rng = np.random.default_rng(42)
    seeds = {sc.steps: scenes.f32(rng.standard_normal((sc.V, 3)))}
    keys = ("compliance", "x0", "v0", "f_vertex", "memb_stiffness")
    xs_ref, _ = oracle.forward(sc)
    ref = oracle.adjoint(sc, seeds)
    with oracle.fp32_rounding():
        ref32 = oracle.adjoint(sc, seeds)
    _, p, ck, xs, _ = gpu_forward(sc, solver=solver)
    assert np.abs(xs - xs_ref).max() < POS_TOL
    got = solver.adjoint(p, sc.steps, sc.iters, ck, {k: to_dev(v) for k, v in seeds.items()}, want=keys)
    torch.cuda.synchronize()
    for k in keys:
        assert np.abs(ref[k]).max() > 0, k
        floor = rel_err(ref32[k], ref[k])
        e = rel_err(got[k].cpu().numpy().reshape(ref[k].shape), ref[k])
        print(f"membrane 256^2 {k}: error {e:.3e}, float32 floor {floor:.3e}")
        assert e < max(GRAD_TOL, 4.0 * floor), (k, e, floor)
