"""GPU (sm_103a, through the C ABI) versus the FP64 oracle, element by element.

Tolerances: positions within 1e-5 m (relative to the 1 m scenes) over the horizon; each
gradient group within 1e-3 relative L2 error and each of its entries within 2 % of its own
size (floored at 1e-3 of the group's largest entry), with the same FP32-rounded seed dL/dx
fed to both sides; where the oracle's own float32-rounding emulation already moves a group
further, the bounds are twice that floor (tests/gpu_common.py)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2301_01396_gb300 import binding, scenes
from tests import helpers
from tests.gpu_common import (GRAD_KEYS, check_grad, contact_margin, contact_signs_agree, gpu_adjoint,
                              gpu_forward, oracle_adjoint_floor, rel_err, to_dev)

pytestmark = pytest.mark.gpu

POS_TOL = 1e-5
GRAD_TOL = 1e-3


def _cases():
    both = helpers.small_sphere_cloth(24, steps=6, iters=8)
    both.collider_flags = scenes.COLLIDE_PLANE | scenes.COLLIDE_SPHERE
    both.plane_h = float(np.float32(both.sphere[1] + both.sphere[3] + 0.003))
    both.v0 = scenes.f32(both.v0 + np.array([0.0, -1.4, 0.0]))
    return {
        # the 16x16 stiff cloth over its first 10 steps (20 iterations each); its 50-step
        # horizon is ill-conditioned (tests/test_conditioning.py)
        "plain_cloth_16": scenes.plain_cloth(16, steps=10),
        "ground_cloth_32": helpers.small_cloth(32, bending=True, diagonals="one", steps=8, iters=10,
                                               plane_h=-0.03, v_scale=0.3, seed=33),
        "tets_4": helpers.small_tets(4, steps=8, iters=6, y0=0.004, v_scale=0.05),
        # each tet's C_H and C_D by one 2x2 solve (per-color launches in every mode), on
        # softer tets: with inverse moduli down to 1e-5 the coupled sweep amplifies float32
        # rounding past these bounds within 3 steps (tests/test_oracle_coupled.py)
        "tets_4_coupled": scenes.couple_tets(helpers.small_tets(4, steps=8, iters=6, y0=0.004, v_scale=0.05,
                                                                alpha=(1e-4, 1e-2))),
        "sphere_cloth_24": helpers.small_sphere_cloth(24, steps=6, iters=8),
        "both_colliders_24": both,
        # 16,384 vertices: more than one shared-memory group, so the phase plan has many
        # CTAs per phase (tiled coloring: 4 phases of 16 colors) or a mix of multi- and
        # single-color runs (pattern coloring)
        "tiled_cloth_128": helpers.small_cloth(128, bending=True, diagonals="both", pins=(), steps=3, iters=4,
                                               v_scale=0.3, seed=60, coloring="tiled", tile=16),
        "pattern_cloth_128": helpers.small_cloth(128, bending=True, diagonals="both", pins=((0, 0),), steps=3,
                                                 iters=4, v_scale=0.3, seed=61),
    }


CASES = list(_cases().keys())


@pytest.fixture(scope="module")
def cases():
    return _cases()


@pytest.mark.parametrize("name", CASES)
def test_forward_matches_oracle(name, cases):
    sc = cases[name]
    xs_ref, vs_ref = oracle.forward(sc)
    assert contact_margin(sc, xs_ref, vs_ref) > 1e-5
    _, _, _, xs, vs = gpu_forward(sc)
    assert contact_signs_agree(sc, xs, vs, xs_ref, vs_ref)
    err = np.abs(xs - xs_ref).max()
    assert err < POS_TOL, f"max position error {err:.3e}"
    pinned = sc.inv_mass == 0
    assert np.all(xs[:, pinned] == np.float32(sc.x0[pinned]))


@pytest.mark.parametrize("name", CASES)
def test_adjoint_matches_oracle(name, cases):
    sc = cases[name]
    rng = np.random.default_rng(7)
    N = sc.steps
    seeds = {N: scenes.f32(rng.standard_normal((sc.V, 3))), N // 2: scenes.f32(rng.standard_normal((sc.V, 3)))}
    ref, ref32 = oracle_adjoint_floor(sc, seeds)
    got, _ = gpu_adjoint(sc, seeds)
    for k in GRAD_KEYS:
        if k == "f_global" and sc.f_global is None and np.abs(ref[k]).max() == 0:
            continue
        if k == "collider" and not sc.collider_flags:
            assert np.all(got[k] == 0)
            continue
        r, r32 = ref[k], ref32[k]
        g = got[k].reshape(r.shape) if k != "f_global" else got[k][:N]
        if k == "collider":
            sel = [0] if sc.collider_flags == scenes.COLLIDE_PLANE else \
                  [1, 2, 3, 4] if sc.collider_flags == scenes.COLLIDE_SPHERE else [0, 1, 2, 3, 4]
            r, g, r32 = r[sel], g[sel], r32[sel]
        check_grad(f"{name} {k}", g, r, GRAD_TOL, ref32=r32)


def _keyframe_force_scene():
    """A cloth on the sphere driven by a force per vertex per step (the keyframe example's
    control variables) on top of the global and wind forces."""
    sc = helpers.small_sphere_cloth(10, steps=5, iters=3, seed=4)
    rng = np.random.default_rng(31)
    m_i = 2.56 / sc.V
    sc.f_vertex_steps = scenes.f32(0.3 * m_i * 9.81 * rng.standard_normal((sc.steps, sc.V, 3)))
    return sc


def test_per_step_vertex_forces_match_oracle():
    sc = _keyframe_force_scene()
    xs_ref, vs_ref = oracle.forward(sc)
    assert contact_margin(sc, xs_ref, vs_ref) > 1e-5
    solver, p, ck, xs, vs = gpu_forward(sc)
    assert contact_signs_agree(sc, xs, vs, xs_ref, vs_ref)
    assert np.abs(xs - xs_ref).max() < POS_TOL
    rng = np.random.default_rng(32)
    seeds = {sc.steps: scenes.f32(rng.standard_normal((sc.V, 3))), 2: scenes.f32(rng.standard_normal((sc.V, 3)))}
    ref, ref32 = oracle_adjoint_floor(sc, seeds)
    got = solver.adjoint(p, sc.steps, sc.iters, ck, {k: to_dev(v) for k, v in seeds.items()},
                         want=GRAD_KEYS + ("f_vertex_steps",))
    torch.cuda.synchronize()
    for k in ("compliance", "x0", "v0", "f_global", "f_vertex", "f_vertex_steps"):
        check_grad(f"keyframe_forces {k}", got[k].cpu().numpy(), ref[k], GRAD_TOL, ref32=ref32[k])
    fvs = got["f_vertex_steps"].cpu().numpy()
    assert np.allclose(fvs.sum(0), got["f_vertex"].cpu().numpy(), rtol=1e-12, atol=0)


def test_loss_and_seed_match_definition():
    sc = helpers.small_cloth(9, steps=5, iters=4)
    solver, p, ck, xs, _ = gpu_forward(sc)
    rng = np.random.default_rng(3)
    targets = {5: scenes.f32(xs[5] + 0.01 * rng.standard_normal(xs[5].shape)),
               2: scenes.f32(xs[2] + 0.01 * rng.standard_normal(xs[2].shape))}
    loss, seeds = solver.loss(ck, {k: to_dev(v) for k, v in targets.items()})
    torch.cuda.synchronize()
    ref = sum(0.5 * np.sum((xs[k] - targets[k]) ** 2) for k in targets)
    assert abs(loss.item() - ref) <= 1e-6 * ref
    s = seeds.cpu().numpy()
    assert np.allclose(s[0], xs[2] - targets[2], atol=1e-7)
    assert np.allclose(s[1], xs[5] - targets[5], atol=1e-7)


def test_deterministic_bitwise():
    sc = helpers.small_sphere_cloth(16, steps=4, iters=5)
    rng = np.random.default_rng(1)
    seeds = {4: scenes.f32(rng.standard_normal((sc.V, 3)))}
    a, xa = gpu_adjoint(sc, seeds)
    b, xb = gpu_adjoint(sc, seeds)
    assert np.array_equal(xa, xb)
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def test_mixed_type_colors_and_greedy_order():
    """A coloring whose colors mix distance and bending constraints (greedy over all
    constraints): the library splits each color by type; results follow the oracle."""
    sc = helpers.small_cloth(12, bending=True, steps=4, iters=5, plane_h=-0.02, v_scale=0.3, seed=5)
    offs, order = scenes.greedy_coloring(sc)
    sc = sc.with_(color_offsets=offs, color_order=order)
    xs_ref, vs_ref = oracle.forward(sc)
    assert contact_margin(sc, xs_ref, vs_ref) > 1e-5
    _, _, _, xs, _ = gpu_forward(sc)
    assert np.abs(xs - xs_ref).max() < POS_TOL
    rng = np.random.default_rng(2)
    seeds = {sc.steps: scenes.f32(rng.standard_normal((sc.V, 3)))}
    ref, ref32 = oracle_adjoint_floor(sc, seeds)
    got, _ = gpu_adjoint(sc, seeds)
    for k in ("compliance", "x0", "v0"):
        check_grad(f"greedy_order {k}", got[k], ref[k], GRAD_TOL, ref32=ref32[k])


def test_zero_steps_and_single_iteration():
    sc = helpers.small_cloth(7, steps=3, iters=1, v_scale=0.2)
    rng = np.random.default_rng(4)
    seed = scenes.f32(rng.standard_normal((sc.V, 3)))
    got, xs = gpu_adjoint(sc, {0: seed}, steps=0, iters=1)
    assert np.array_equal(xs[0], np.float32(sc.x0))
    assert np.allclose(got["x0"], seed) and np.all(got["v0"] == 0) and np.all(got["compliance"] == 0)
    xs_ref, _ = oracle.forward(sc, 3, 1)
    _, _, _, xs, _ = gpu_forward(sc, 3, 1)
    assert np.abs(xs - xs_ref).max() < POS_TOL
    seeds = {3: seed}
    ref, ref32 = oracle_adjoint_floor(sc, seeds, 3, 1)
    got, _ = gpu_adjoint(sc, seeds, 3, 1)
    for k in ("compliance", "x0", "v0"):
        check_grad(f"single_iteration {k}", got[k], ref[k], GRAD_TOL, ref32=ref32[k])


def test_no_constraints_is_ballistic():
    V = 300
    rng = np.random.default_rng(8)
    x0 = scenes.f32(rng.standard_normal((V, 3)))
    sc = scenes.Scene(rest_x=x0, inv_mass=scenes.f32(np.full(V, 2.0)), dist_idx=np.zeros((0, 2), np.int32),
                      bend_idx=np.zeros((0, 4), np.int32), tet_idx=np.zeros((0, 4), np.int32),
                      tet_gamma=np.zeros(0), color_offsets=np.zeros(1, np.int32),
                      color_order=np.zeros(0, np.int32), x0=x0, v0=scenes.f32(rng.standard_normal((V, 3))),
                      compliance=np.zeros(0), steps=5, iters=2)
    xs_ref, _ = oracle.forward(sc)
    _, _, _, xs, _ = gpu_forward(sc)
    assert np.abs(xs - xs_ref).max() < POS_TOL


def test_autograd_function_matches_adjoint():
    sc = helpers.small_sphere_cloth(10, steps=4, iters=4)
    solver = binding.Solver.from_scene(sc)
    cfg = dict(steps=sc.steps, iters=sc.iters, dt=sc.dt, gravity=sc.gravity, collider_flags=sc.collider_flags,
               contact_compliance=sc.contact_compliance, thickness=sc.thickness)
    comp = to_dev(sc.compliance).requires_grad_()
    x0 = to_dev(sc.x0).requires_grad_()
    v0 = to_dev(sc.v0).requires_grad_()
    fg = to_dev(sc.f_global).requires_grad_()
    fv = to_dev(sc.f_vertex).requires_grad_()
    col = torch.tensor([sc.plane_h, *sc.sphere], dtype=torch.float64, requires_grad=True)
    (xT,) = binding.simulate(solver, cfg, comp, x0, v0, fg, fv, col)
    rng = np.random.default_rng(6)
    target = to_dev(xT.detach().cpu().numpy() + 0.01 * rng.standard_normal((sc.V, 3)))
    loss = 0.5 * ((xT - target) ** 2).sum()
    loss.backward()
    seeds = {sc.steps: scenes.f32((xT - target).detach().cpu().numpy())}
    ref, ref32 = oracle_adjoint_floor(sc, seeds)
    grads = {"compliance": comp.grad, "x0": x0.grad, "v0": v0.grad, "f_global": fg.grad, "f_vertex": fv.grad}
    for k, g in grads.items():
        check_grad(f"autograd {k}", g.cpu().numpy(), ref[k], GRAD_TOL, ref32=ref32[k])
    check_grad("autograd sphere", col.grad.numpy()[1:], ref["collider"][1:], GRAD_TOL, ref32=ref32["collider"][1:])


def test_nonfinite_state_is_reported():
    """A NaN compliance makes the step non-finite; the library reports it as a status
    (the kernels never trap)."""
    sc = helpers.small_cloth(6, steps=2, iters=2)
    comp = sc.compliance.copy()
    comp[0] = np.nan
    solver = binding.Solver.from_scene(sc)
    p = binding.params_from_scene(sc, compliance=comp)
    solver.forward(p, 2, 2, to_dev(sc.x0), to_dev(sc.v0))
    with pytest.raises(binding.XpbdError, match="NONFINITE"):
        solver.sync_status()
    solver.sync_status()   # cleared after being reported


@pytest.mark.parametrize("name", CASES)
def test_phase_plan_matches_per_color_launches(name, cases):
    """The multi-color phase launches (exec_mode 2) and one launch per color (exec_mode 1)
    run the same constraint updates in the same order, and the phase plan is used for these
    colorings.  Built with FMA contraction off (nvcc -fmad=false) the two modes agree bit
    for bit on every case here; with contraction on, the compiler fuses a few multiply-adds
    differently in the two kernels, so positions first differ by one float32 ulp and the
    contact-sensitive scenes carry that to ~4e-5 in the compliance gradient: the bounds are
    those of rounding, far below what one skipped or reordered update would give."""
    sc = cases[name]
    rng = np.random.default_rng(9)
    seeds = {sc.steps: scenes.f32(rng.standard_normal((sc.V, 3)))}
    out = []
    for mode in (2, 1):   # 2: the phase plan whenever the coloring allows one
        solver = binding.Solver.from_scene(sc, exec_mode=mode)
        info = solver.exec_info()
        assert info["phases"] == (mode == 2), info
        if mode == 2:
            assert info["launches_per_iteration"] < sc.n_colors
        p = binding.params_from_scene(sc)
        ck = solver.forward(p, sc.steps, sc.iters, to_dev(sc.x0), to_dev(sc.v0))
        gr = solver.adjoint(p, sc.steps, sc.iters, ck, {k: to_dev(v) for k, v in seeds.items()})
        torch.cuda.synchronize()
        out.append((ck[:, 0, :, :3].cpu().numpy(), {k: v.cpu().numpy() for k, v in gr.items()}))
    (x0, g0), (x1, g1) = out
    assert np.abs(x0 - x1).max() <= 1e-6
    for k in g0:
        assert rel_err(g0[k], g1[k]) <= 2e-4, k


def test_config1_workload_loss_and_gradients():
    """Config 1 on its own workload over the well-conditioned 10-step horizon: the 16 x 16
    stiff cloth (930 springs, compliance 1e-7, 20 iterations), the loss 1/2 |x_T - x*|^2
    against a target made (by the oracle) with seeded lognormal(0, 0.5) compliances, and
    its gradient with respect to all 930 compliances and v0.

    The target differs from the simulated cloth by at most ~4e-7 m (stiff springs stretch by
    m g alpha ~ 1e-8 m), the size of float32 position rounding: the loss and the end-to-end
    gradient are not resolvable in float32 (the oracle's own float32-rounding emulation
    moves the seed by ~66 % and the gradients by 20-50 %).  So the gradient is compared
    element by element with the same float32-rounded seed fed to both sides, and the GPU's
    own loss and seed are checked against twice that float32 floor."""
    sc = scenes.plain_cloth(16, steps=10)
    T = sc.steps
    xt, _ = oracle.forward(scenes.plain_cloth(16, steps=10, target=True))
    target = scenes.f32(xt[T])
    xs_ref, _ = oracle.forward(sc)
    with oracle.fp32_rounding():
        xs32, _ = oracle.forward(sc)
    solver, p, ck, xs, _ = gpu_forward(sc)
    assert np.abs(xs - xs_ref).max() < POS_TOL
    loss, seeds = solver.loss(ck, {T: to_dev(target)})
    torch.cuda.synchronize()
    seed_ref = xs_ref[T] - target
    loss_ref = 0.5 * float(np.sum(seed_ref ** 2))
    loss32 = 0.5 * float(np.sum((xs32[T] - target) ** 2))
    floor = abs(loss32 - loss_ref) / loss_ref
    err = abs(loss.item() - loss_ref) / loss_ref
    print(f"PARITY config1 loss: rel {err:.3e} (float32 floor {floor:.3e})")
    assert err < max(1e-3, 2.0 * floor)
    assert rel_err(seeds[0].cpu().numpy(), seed_ref) < max(1e-3, 2.0 * rel_err(xs32[T] - target, seed_ref))
    # the gradient of the workload's loss, same seed on both sides
    seed = scenes.f32(seed_ref)
    ref, ref32 = oracle_adjoint_floor(sc, {T: seed})
    got = solver.adjoint(p, T, sc.iters, ck, {T: to_dev(seed)}, want=("compliance", "v0"))
    torch.cuda.synchronize()
    assert got["compliance"].shape == (930,)
    for k in ("compliance", "v0"):
        check_grad(f"config1 {k}", got[k].cpu().numpy(), ref[k], GRAD_TOL, ref32=ref32[k])
