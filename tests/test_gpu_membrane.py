"""Orthotropic StVK membranes on the GPU (per-color kernels k_proj_memb / k_vjp_memb and
the stiffness chain rule) against the FP64 oracle, and the entry points that run or
refuse them."""
import numpy as np
import pytest
import torch

import oracle
from paper_2301_01396_gb300 import binding, scenes
from tests.gpu_common import (check_grad, contact_margin, contact_signs_agree, gpu_adjoint, gpu_forward,
                              oracle_adjoint_floor, rel_err, to_dev)

pytestmark = pytest.mark.gpu

POS_TOL = 1e-5
GRAD_TOL = 1e-3
KEYS = ("compliance", "x0", "v0", "f_vertex", "memb_stiffness")


def _hanging():
    # 16x16 sheet, two corners pinned, per-triangle stiffness spread 0.3, random start
    # velocities; float32-rounding floors (oracle emulation): positions 3.7e-7 m,
    # gradients <= 1.8e-5
    sc = scenes.membrane_cloth(16, steps=6, iters=8, seed=5)
    rng = np.random.default_rng(51)
    v = 0.3 * rng.standard_normal(sc.x0.shape)
    v[sc.inv_mass == 0] = 0.0
    sc.v0 = scenes.f32(v)
    return sc


def _on_sphere():
    # free sheet falling onto a sphere (contacts from step 1); floors <= 1.2e-5
    sc = scenes.membrane_cloth(16, steps=6, iters=8, seed=6, pins=())
    sc.x0 = scenes.f32(sc.x0 + np.array([-0.5, 0.0, -0.5]))
    sc.collider_flags = scenes.COLLIDE_SPHERE
    sc.sphere = (0.0, -0.3, 0.0, 0.29)
    sc.v0 = scenes.f32(np.tile([0.0, -0.5, 0.0], (sc.V, 1)))
    return sc


CASES = {"hanging": _hanging, "on_sphere": _on_sphere}


@pytest.mark.parametrize("name", list(CASES))
def test_membrane_forward_and_adjoint_match_oracle(name):
    sc = CASES[name]()
    xs_ref, vs_ref, _, _, act = oracle.forward_multipliers(sc)
    if sc.collider_flags:
        assert act.any() and contact_margin(sc, xs_ref, vs_ref) > 1e-5
    solver, p, ck, xs, vs = gpu_forward(sc)
    assert solver.n_memb == sc.n_memb
    if sc.collider_flags:
        assert contact_signs_agree(sc, xs, vs, xs_ref, vs_ref)
    err = np.abs(xs - xs_ref).max()
    assert err < POS_TOL, f"max position error {err:.3e}"
    rng = np.random.default_rng(7)
    N = sc.steps
    seeds = {N: scenes.f32(rng.standard_normal((sc.V, 3))), N // 2: scenes.f32(rng.standard_normal((sc.V, 3)))}
    ref, ref32 = oracle_adjoint_floor(sc, seeds)
    gr = solver.adjoint(p, N, sc.iters, ck, {k: to_dev(v) for k, v in seeds.items()},
                        want=KEYS + (("collider",) if sc.collider_flags else ()))
    torch.cuda.synchronize()
    solver.sync_status()
    for k in KEYS + (("collider",) if sc.collider_flags else ()):
        g, r, r32 = gr[k].cpu().numpy(), ref[k], ref32[k]
        if k == "collider":
            sel = [0] if sc.collider_flags == scenes.COLLIDE_PLANE else [1, 2, 3, 4]
            g, r, r32 = g[sel], r[sel], r32[sel]
        check_grad(f"membrane {sc.name} {k}", g, r, GRAD_TOL, ref32=r32)


def test_membrane_deterministic_static_and_sparse():
    """Two runs agree bit for bit; the allocation-free forward and the sparse-checkpoint
    reverse sweep give the same bits as the allocating forward and the dense sweep."""
    sc = _hanging()
    solver = binding.Solver.from_scene(sc, exec_mode=1)
    p = binding.params_from_scene(sc)
    x0, v0 = to_dev(sc.x0), to_dev(sc.v0)
    ck = solver.forward(p, sc.steps, sc.iters, x0, v0)
    ck2 = solver.forward(p, sc.steps, sc.iters, x0, v0)
    cks = solver.forward_static(p, sc.steps, sc.iters, x0, v0, solver.new_checkpoints(sc.steps))
    torch.cuda.synchronize()
    assert torch.equal(ck, ck2) and torch.equal(ck, cks)
    seeds = {sc.steps: to_dev(np.random.default_rng(3).standard_normal((sc.V, 3)))}
    g1 = solver.adjoint(p, sc.steps, sc.iters, ck, seeds, want=KEYS)
    g2 = solver.adjoint(p, sc.steps, sc.iters, ck, seeds, want=KEYS)
    ckp = solver.forward_sparse(p, sc.steps, sc.iters, x0, v0, 4)
    g3 = solver.adjoint(p, sc.steps, sc.iters, ckp, seeds, want=KEYS, stride=4)
    torch.cuda.synchronize()
    solver.sync_status()
    for k in KEYS:
        assert torch.equal(g1[k], g2[k]) and torch.equal(g1[k], g3[k]), k


def test_membrane_invalid_stiffness_is_reported():
    sc = scenes.membrane_cloth(4, steps=1, iters=1)
    K = sc.memb_stiffness.copy()
    K[2, 2] = 2.0 * np.sqrt(K[2, 0] * K[2, 1])        # C01^2 > C00 C11: not positive definite
    solver = binding.Solver.from_scene(sc)
    p = binding.params_from_scene(sc.with_(memb_stiffness=K))
    solver.forward(p, 1, 1, to_dev(sc.x0), to_dev(sc.v0))
    with pytest.raises(binding.XpbdError) as e:
        solver.sync_status()
    assert e.value.status == 5 and "membrane stiffness" in str(e.value)


def test_membrane_models_are_refused_by_serving():
    sc = scenes.membrane_cloth(4, steps=2, iters=2)
    solver = binding.Solver.from_scene(sc)
    p = binding.params_from_scene(sc)
    x0, v0 = to_dev(sc.x0), to_dev(sc.v0)
    srv = binding.Server(max_slots=2)
    with pytest.raises(binding.XpbdError) as e:
        srv.submit(solver, p, sc.steps, sc.iters, x0, v0, x0)
    assert "membranes" in str(e.value)
    srv.close()


def _tiled():
    # 64x64 sheet with the tiled coloring (16x16 blocks): the phase plan runs its colors in
    # multi-color launches; pinned corners, random start velocities
    sc = scenes.membrane_cloth(64, steps=5, iters=6, seed=8, coloring="tiled", tile=16)
    rng = np.random.default_rng(52)
    v = 0.3 * rng.standard_normal(sc.x0.shape)
    v[sc.inv_mass == 0] = 0.0
    sc.v0 = scenes.f32(v)
    return sc


def test_membrane_phase_plan_matches_oracle_and_per_color():
    """Membranes in the multi-color phase kernels (exec_mode 2) against the oracle, and
    against one launch per color (exec_mode 1) within rounding (FMA contraction differs
    between the two kernels, as for the other constraint types)."""
    sc = _tiled()
    xs_ref, _ = oracle.forward(sc)
    rng = np.random.default_rng(9)
    N = sc.steps
    seeds = {N: scenes.f32(rng.standard_normal((sc.V, 3))), 2: scenes.f32(rng.standard_normal((sc.V, 3)))}
    ref, ref32 = oracle_adjoint_floor(sc, seeds)
    out = {}
    for mode in (2, 1):
        solver = binding.Solver.from_scene(sc, exec_mode=mode)
        info = solver.exec_info()
        assert info["phases"] == (mode == 2), info
        if mode == 2:
            assert info["launches_per_iteration"] < sc.n_colors
        _, p, ck, xs, _ = gpu_forward(sc, solver=solver)
        gr = solver.adjoint(p, N, sc.iters, ck, {k: to_dev(v) for k, v in seeds.items()}, want=KEYS)
        torch.cuda.synchronize()
        solver.sync_status()
        err = np.abs(xs - xs_ref).max()
        assert err < POS_TOL, (mode, err)
        for k in KEYS:
            check_grad(f"membrane_mode{mode} {k}", gr[k].cpu().numpy(), ref[k], GRAD_TOL, ref32=ref32[k])
        out[mode] = (xs, {k: gr[k].cpu().numpy() for k in KEYS})
    assert np.abs(out[2][0] - out[1][0]).max() <= 1e-6
    for k in KEYS:
        assert rel_err(out[2][1][k], out[1][1][k]) <= 2e-4, k
