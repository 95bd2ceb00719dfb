"""Coupled tet updates on the GPU (each tet's C_H and C_D from one 2x2 solve) against the
FP64 oracle, and the entry points that run or refuse them."""
import numpy as np
import pytest
import torch

import oracle
from paper_2301_01396_gb300 import binding, scenes
from tests import helpers
from tests.gpu_common import check_grad, gpu_adjoint, gpu_forward, oracle_adjoint_floor, rel_err, to_dev

pytestmark = pytest.mark.gpu

POS_TOL = 1e-5
GRAD_TOL = 1e-3


def _uncoupled_block():
    # 6^3 cells x 5 = 1080 tets with per-tet inverse moduli log-uniform in [1e-4, 1e-2],
    # tumbling freely (no contacts: the comparison covers the pair update alone).  Stiffer
    # tets (down to 1e-5) make the coupled sweep amplify float32 rounding beyond these
    # bounds within a few steps (tests/test_oracle_coupled.py).
    return helpers.small_tets(6, steps=4, iters=8, y0=0.05, plane=False, v_scale=0.05, alpha=(1e-4, 1e-2))


def _block():
    return scenes.couple_tets(_uncoupled_block())


def test_coupled_block_matches_oracle():
    sc = _block()
    xs_ref, _ = oracle.forward(sc)
    _, _, _, xs, _ = gpu_forward(sc)
    err = np.abs(xs - xs_ref).max()
    assert err < POS_TOL, f"max position error {err:.3e}"
    rng = np.random.default_rng(17)
    seeds = {sc.steps: scenes.f32(rng.standard_normal((sc.V, 3))), 2: scenes.f32(rng.standard_normal((sc.V, 3)))}
    ref, ref32 = oracle_adjoint_floor(sc, seeds)
    got, _ = gpu_adjoint(sc, seeds)
    for k in ("compliance", "x0", "v0", "f_vertex"):
        check_grad(f"coupled_block {k}", got[k], ref[k], GRAD_TOL, ref32=ref32[k])


def test_coupled_differs_from_one_at_a_time():
    """The flag changes the update: the same block with C_H and C_D updated one after the
    other ends elsewhere (the oracle agrees on both)."""
    sc = _block()
    un = _uncoupled_block()
    _, _, _, xc, _ = gpu_forward(sc)
    _, _, _, xu, _ = gpu_forward(un)
    assert np.abs(xc - xu).max() > 1e-4
    assert np.abs(xu - oracle.forward(un)[0]).max() < POS_TOL


def test_coupled_phase_plan_matches_per_color_and_oracle():
    """Pairs in the multi-color phase kernels (exec_mode 2; each chunk stages the C_H records
    with their C_D shadows) against one launch per color (within rounding: FMA contraction
    differs between the kernels) and against the oracle."""
    sc = _block()
    rng = np.random.default_rng(19)
    seeds = {sc.steps: scenes.f32(rng.standard_normal((sc.V, 3)))}
    ref, ref32 = oracle_adjoint_floor(sc, seeds)
    xs_ref, _ = oracle.forward(sc)
    out = {}
    for mode in (2, 1):
        solver = binding.Solver.from_scene(sc, exec_mode=mode)
        info = solver.exec_info()
        assert info["phases"] == (mode == 2), info
        _, p, ck, xs, _ = gpu_forward(sc, solver=solver)
        gr = solver.adjoint(p, sc.steps, sc.iters, ck, {k: to_dev(v) for k, v in seeds.items()},
                            want=("compliance", "x0", "v0", "f_vertex"))
        torch.cuda.synchronize()
        solver.sync_status()
        assert np.abs(xs - xs_ref).max() < POS_TOL, mode
        out[mode] = (xs, {k: v.cpu().numpy() for k, v in gr.items()})
        for k, v in out[mode][1].items():
            check_grad(f"coupled_mode{mode} {k}", v, ref[k], GRAD_TOL, ref32=ref32[k])
    assert np.abs(out[2][0] - out[1][0]).max() <= 1e-6
    for k in out[2][1]:
        assert rel_err(out[2][1][k], out[1][1][k]) <= 2e-4, k


def test_serving_refuses_coupled_models():
    sc = scenes.couple_tets(helpers.small_tets(2, steps=2, iters=2))
    solver = binding.Solver.from_scene(sc)
    p = binding.params_from_scene(sc)
    srv = binding.Server(max_slots=2)
    x0, v0 = to_dev(sc.x0), to_dev(sc.v0)
    with pytest.raises(binding.XpbdError) as e:
        srv.submit(solver, p, sc.steps, sc.iters, x0, v0, x0)
    assert "coupled" in str(e.value)
    srv.close()
