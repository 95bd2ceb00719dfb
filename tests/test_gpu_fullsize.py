"""Parity at the full sizes of the cloth, ground-cloth, tet-block and 2950^2 sphere-cloth
workloads.  The 2950^2 cloth runs twice: with the 16-color pattern coloring (one launch
per color), and in the configuration bench.py times (the 64-color tiled coloring with
32 x 32 tiles, executed by the multi-color phase kernels: 1536-vertex groups, full
256-constraint stages and the reverse stage ring).

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
from tests import helpers
from tests.gpu_common import (check_grad, contact_margin, contact_signs_agree, gpu_forward, oracle_adjoint_floor,
                              rel_err, to_dev)

pytestmark = pytest.mark.gpu

POS_TOL = 1e-5
GRAD_TOL = 1e-3


def _at_state(sc, xs, vs, n, steps, iters=None):
    """The scene restarted from the (FP32-rounded) oracle state of step n."""
    fg = None if sc.f_global is None else sc.f_global[n:n + steps]
    return sc.with_(x0=scenes.f32(xs[n]), v0=scenes.f32(vs[n]), steps=steps,
                    iters=sc.iters if iters is None else iters, f_global=fg)


def _grad_parity(tag, sc, seeds, keys=("compliance", "x0", "v0")):
    ref, ref32 = oracle_adjoint_floor(sc, seeds)
    solver, p, ck, xs, _ = gpu_forward(sc)
    got = solver.adjoint(p, sc.steps, sc.iters, ck, {k: to_dev(v) for k, v in seeds.items()})
    torch.cuda.synchronize()
    for k in keys:
        check_grad(f"{tag} {k}", got[k].cpu().numpy(), ref[k], GRAD_TOL, ref32=ref32[k])


def test_ground_cloth_256_forward_first_steps():
    sc = scenes.ground_cloth(256, steps=8)
    xs_ref, _ = oracle.forward(sc)
    _, _, _, xs, _ = gpu_forward(sc)
    assert np.abs(xs - xs_ref).max() < POS_TOL


def test_ground_cloth_256_error_vs_step_full_horizon():
    """Config 2 over its full horizon (100 steps of 30 iterations): the largest position
    error against the oracle at every step (printed every 10 steps).  The oracle's own
    float32-rounding emulation stays within 1.1e-6 m of it over the 100 steps, so a float32
    implementation can stay within the 1e-5 m position tolerance; the bound asserted over
    the whole horizon is that tolerance.  (Over 100 steps the cloth lies on the ground, and
    a contact whose predicted position is within float32 rounding of the plane could be
    decided differently by float32 and float64; none is on this trajectory.)"""
    sc = scenes.ground_cloth(256)
    xs_ref, _ = oracle.forward(sc)
    _, _, _, xs, _ = gpu_forward(sc)
    err = np.abs(xs - xs_ref).max(axis=(1, 2))
    print("PARITY config2 error vs step: " + " ".join(f"{n}:{err[n]:.1e}" for n in range(0, sc.steps + 1, 10)))
    assert err.max() < POS_TOL, err.max()


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
    _grad_parity("ground_cloth_256", sub2, {2: scenes.f32(rng.standard_normal((sc.V, 3)))})


def test_tet_block_32_forward_to_contact():
    sc = scenes.tet_block(32, steps=16)
    xs_ref, vs_ref = oracle.forward(sc)
    assert (xs_ref[-1, :, 1] <= sc.plane_h + 1e-6).sum() > 100
    assert contact_margin(sc, xs_ref, vs_ref) > 1e-6
    _, _, _, xs, vs = gpu_forward(sc)
    assert contact_signs_agree(sc, xs, vs, xs_ref, vs_ref)
    err = np.abs(xs - xs_ref).max(axis=(1, 2))
    print("PARITY config3 error vs step: " + " ".join(f"{n}:{err[n]:.1e}" for n in range(sc.steps + 1)))
    assert err.max() < POS_TOL


def test_tet_block_32_adjoint_in_contact():
    sc = scenes.tet_block(32, steps=15)
    xs, vs = oracle.forward(sc)
    sub = _at_state(sc, xs, vs, 13, 2)
    rng = np.random.default_rng(3)
    _grad_parity("tet_block_32", sub, {2: scenes.f32(rng.standard_normal((sc.V, 3)))})


# --------------------------------------------------------------------------- 2950^2 cloth

@pytest.fixture(scope="module")
def big_cloth():
    return scenes.sphere_cloth(2950, steps=1, iters=15)


def test_sphere_cloth_2950_forward_window(big_cloth):
    full = big_cloth
    n, I = 2950, 15
    R = 2 * 16 * I + 4
    w = 2 * R + 64
    i0 = j0 = (n - w) // 2
    sub, sel, _, _ = helpers.grid_window(full, n, i0, j0, w)
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
    near float32 resolution.  Every group's bounds are therefore max(1e-3, 2 x floor)
    (L2) and max(2e-2, 3 x floor) (per entry), where the floor is the oracle's own change
    when its state is rounded to float32 (oracle.fp32_rounding)."""
    full = big_cloth
    n, I = 2950, 3
    R = 2 * 16 * I + 4
    w = 6 * R + 48
    i0, j0 = 1200, 1400
    sub, sel, kd, kb = helpers.grid_window(full, n, i0, j0, w)
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
    with oracle.fp32_rounding():
        ref32 = oracle.adjoint(sub, {1: seed_local}, 1, I)
    for k in ("x0", "v0", "f_vertex"):
        g = got[k].cpu().numpy()[sel][band]
        check_grad(f"pattern_2950 {k}", g, ref[k][band], GRAD_TOL, ref32=ref32[k][band])
    # everything outside the window is untouched by the seed
    outside = np.ones(full.V, bool)
    outside[sel] = False
    assert np.abs(got["x0"].cpu().numpy()[outside]).max() == 0.0
    gc = got["compliance"].cpu().numpy()
    ids = np.concatenate([kd, kb])
    check_grad("pattern_2950 compliance", gc[ids], ref["compliance"], GRAD_TOL, ref32=ref32["compliance"])
    check_grad("pattern_2950 f_global", got["f_global"].cpu().numpy()[:1], ref["f_global"], GRAD_TOL)


def test_membrane_cloth_256_full_size():
    """The material-estimation membrane workload at its full size (65,536 vertices, 130,050
    StVK triangles + 129,540 hinges, 8x8-tile coloring, 30 iterations) in the phase
    kernels bench.py times, over one step, with a smooth start velocity field (0.3 m/s, one
    wavelength across the sheet) so that the sheet strains and every gradient group is
    nonzero (the bench's flat fall keeps it strain-free for 20 steps).  The stiff
    membranes (K ~ 1e3 N/m on 4 mm triangles) amplify float32 rounding in the reverse
    sweep to ~9e-4, so the gradient bounds are max(1e-3, 2 x floor) (L2) and
    max(2e-2, 3 x floor) (per entry), with the floors measured by the oracle's float32
    emulation."""
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
        check_grad(f"membrane_256 {k}", got[k].cpu().numpy(), ref[k], GRAD_TOL, ref32=ref32[k])


# ------------------------------------------------------------ the benched configuration

BENCH_TILE = 32


@pytest.fixture(scope="module")
def bench_cloth():
    """The benched 2950^2 cloth: tiled coloring with 32 x 32 tiles (64 colors, 4 phases of
    16), one step, started with a smooth velocity field (0.3 m/s, one wavelength across the
    sheet) so that every constraint is strained.  For this step the sphere stays below the
    sheet: the phase kernels are what is under test (contacts run in their own kernel,
    compared with the oracle by the smaller contact scenes)."""
    sc = scenes.sphere_cloth(2950, steps=1, iters=2, coloring="tiled", tile=BENCH_TILE)
    x, z = sc.x0[:, 0], sc.x0[:, 2]
    sc.v0 = scenes.f32(0.3 * np.stack([np.sin(2 * np.pi * z + 0.3), np.sin(2 * np.pi * (x + z)),
                                        np.cos(2 * np.pi * x - 0.7)], axis=1))
    return sc


def _bench_solver(sc):
    solver = binding.Solver.from_scene(sc)      # the default execution mode, as bench.py creates it
    info = solver.exec_info()
    assert info["phases"] and info["launches_per_iteration"] == 4, info
    return solver


def test_bench_configuration_forward_window(bench_cloth):
    """Forward over one step of 2 iterations.  With K = 64 colors a vertex farther than
    R = 2 K I + 4 = 260 from the window's edge does not see that edge; the window (608^2,
    aligned to the tile grid) keeps the full run's color order, so the oracle reproduces the
    full run on its 88 x 88 core."""
    full = bench_cloth
    n, I = 2950, 2
    R = 2 * full.n_colors * I + 4
    w = (2 * R + 64 + BENCH_TILE - 1) // BENCH_TILE * BENCH_TILE
    i0, j0 = BENCH_TILE * 40, BENCH_TILE * 44
    sub, sel, _, _ = helpers.grid_window(full, n, i0, j0, w)
    xs_ref, _ = oracle.forward(sub, 1, I)
    _, _, _, xs, _ = gpu_forward(full, 1, I, solver=_bench_solver(full))
    core = np.zeros((w, w), bool)
    core[R:w - R, R:w - R] = True
    core = core.reshape(-1)
    assert core.sum() >= 64 * 64
    moved = np.abs(xs_ref[1][core] - full.x0[sel][core]).max()
    err = np.abs(xs[1][sel][core] - xs_ref[1][core]).max()
    print(f"PARITY bench_2950 positions: max error {err:.3e} m (motion {moved:.3e} m)")
    assert moved > 1e-3
    assert err < POS_TOL, err


def test_bench_configuration_adjoint_window(bench_cloth):
    """Reverse sweep over the same step (2 iterations, the reverse stage ring of the phase
    kernels): the seed lives on a core 3R from the window's edge, every per-vertex gradient
    group is compared on the band within R of that core (and is zero beyond it on both
    sides), and the compliance gradient on every constraint of the window."""
    full = bench_cloth
    n, I = 2950, 2
    R = 2 * full.n_colors * I + 4
    w = (6 * R + 48 + BENCH_TILE - 1) // BENCH_TILE * BENCH_TILE
    i0, j0 = BENCH_TILE * 20, BENCH_TILE * 30
    sub, sel, kd, kb = helpers.grid_window(full, n, i0, j0, w)
    rng = np.random.default_rng(15)
    li, lj = np.meshgrid(np.arange(w), np.arange(w), indexing="xy")
    dist_edge = np.minimum(np.minimum(li, w - 1 - li), np.minimum(lj, w - 1 - lj)).reshape(-1)
    seed_local = scenes.f32(rng.standard_normal((sub.V, 3)) * (dist_edge >= 3 * R)[:, None])
    ref = oracle.adjoint(sub, {1: seed_local}, 1, I)
    with oracle.fp32_rounding():
        ref32 = oracle.adjoint(sub, {1: seed_local}, 1, I)
    seed_full = np.zeros((full.V, 3), np.float32)
    seed_full[sel] = seed_local
    solver = _bench_solver(full)
    _, p, ck, _, _ = gpu_forward(full, 1, I, solver=solver)
    got = solver.adjoint(p, 1, I, ck, {1: to_dev(seed_full)})
    torch.cuda.synchronize()
    solver.sync_status()
    band = dist_edge >= 2 * R
    for k in ("x0", "v0", "f_vertex"):
        g = got[k].cpu().numpy()
        check_grad(f"bench_2950 {k}", g[sel][band], ref[k][band], GRAD_TOL, ref32=ref32[k][band])
        assert np.abs(ref[k][~band]).max() == 0.0, k
        assert np.abs(g[sel][~band]).max() == 0.0, k
        outside = np.ones(full.V, bool)
        outside[sel] = False
        assert np.abs(g[outside]).max() == 0.0, k
    ids = np.concatenate([kd, kb])
    gc = got["compliance"].cpu().numpy()
    check_grad("bench_2950 compliance", gc[ids], ref["compliance"], GRAD_TOL, ref32=ref32["compliance"])
    rest = np.ones(full.m, bool)
    rest[ids] = False
    assert np.abs(gc[rest]).max() == 0.0
    check_grad("bench_2950 f_global", got["f_global"].cpu().numpy()[:1], ref["f_global"], GRAD_TOL)
    assert np.all(got["collider"].cpu().numpy() == 0)
