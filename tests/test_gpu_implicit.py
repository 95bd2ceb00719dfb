"""The paper's implicit adjoint on the GPU (xpbd_adjoint_implicit) against the dense
implicit-adjoint oracle: same linearisation states (the XPBD forward), block projection,
pinned-vertex filtering and contact blocks; the GPU solves by preconditioned CG."""
import numpy as np
import pytest
import torch

import oracle
from oracle import implicit
from paper_2301_01396_gb300 import binding, scenes
from tests import helpers
from tests.gpu_common import check_grad, contact_margin, gpu_forward, rel_err, to_dev

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-3
KEYS = ("compliance", "x0", "v0", "f_global", "f_vertex")


def _cases():
    ground = helpers.small_cloth(8, bending=True, diagonals="one", pins=(), steps=4, iters=6, v_scale=0.3,
                                 plane_h=-0.02, seed=33)
    ground.v0 = scenes.f32(ground.v0 + np.array([0.0, -0.6, 0.0]))
    return {
        "pinned_cloth": helpers.small_cloth(8, bending=True, diagonals="both", pins=((0, 0), (-1, 0)), steps=4,
                                            iters=6, v_scale=0.3, seed=12),
        "ground_cloth": ground,
        "tets": helpers.small_tets(2, steps=3, iters=6, y0=0.05, plane=False, v_scale=0.05),
        "tets_coupled": scenes.couple_tets(helpers.small_tets(2, steps=3, iters=6, y0=0.05, plane=False,
                                                              v_scale=0.05)),
        "membrane": _membrane(),
    }


def _membrane():
    # a pinned 8x8 orthotropic StVK sheet with bending, random start velocities
    sc = scenes.membrane_cloth(8, steps=3, iters=6, seed=8, pins=((0, 0),), stiffness=(60.0, 30.0, 10.0, 20.0))
    rng = np.random.default_rng(9)
    v = 0.3 * rng.standard_normal(sc.x0.shape)
    v[sc.inv_mass == 0] = 0.0
    sc.v0 = scenes.f32(v)
    return sc


@pytest.mark.parametrize("name", ["pinned_cloth", "ground_cloth", "tets", "tets_coupled", "membrane"])
@pytest.mark.parametrize("pd", [True, False])
def test_implicit_adjoint_matches_oracle(name, pd):
    sc = _cases()[name]
    xs_ref, vs_ref, lam, lamc, act = oracle.forward_multipliers(sc)
    if sc.collider_flags:
        assert contact_margin(sc, xs_ref, vs_ref) > 1e-5
        assert act.any()
    rng = np.random.default_rng(8)
    seeds = {sc.steps: scenes.f32(rng.standard_normal((sc.V, 3))), 1: scenes.f32(rng.standard_normal((sc.V, 3)))}
    ref = implicit.adjoint(sc, seeds, pd=pd)
    with oracle.fp32_rounding():
        ref32 = implicit.adjoint(sc, seeds, pd=pd)
    solver, p, ck, xs, _ = gpu_forward(sc)
    keys = KEYS + ("f_vertex_steps",) + (("memb_stiffness",) if sc.n_memb else ())
    got, its = solver.adjoint_implicit(p, sc.steps, sc.iters, ck, {k: to_dev(v) for k, v in seeds.items()},
                                       want=keys, pd_project=pd)
    torch.cuda.synchronize()
    solver.sync_status()
    assert all(0 < n < 5000 for n in its), its
    for k in keys:
        check_grad(f"implicit {name} pd{int(pd)} {k}", got[k].cpu().numpy(), ref[k], GRAD_TOL, ref32=ref32[k])


def test_phase_plan_handle_gives_the_same_gradient():
    """The solve runs on the per-color records whatever execution mode the handle has."""
    sc = helpers.small_cloth(64, bending=True, diagonals="both", pins=(), steps=2, iters=4, v_scale=0.3, seed=70,
                             coloring="tiled", tile=16)
    rng = np.random.default_rng(9)
    seeds = {sc.steps: to_dev(rng.standard_normal((sc.V, 3)))}
    out = []
    for mode in (2, 1):
        solver = binding.Solver.from_scene(sc, exec_mode=mode)
        p = binding.params_from_scene(sc)
        ck = solver.forward(p, sc.steps, sc.iters, to_dev(sc.x0), to_dev(sc.v0))
        g, _ = solver.adjoint_implicit(p, sc.steps, sc.iters, ck, seeds)
        torch.cuda.synchronize()
        out.append({k: v.cpu().numpy() for k, v in g.items()})
    for k in KEYS:
        assert rel_err(out[0][k], out[1][k]) < 1e-4, k


def test_collider_gradient_is_refused():
    sc = _cases()["ground_cloth"]
    solver, p, ck, _, _ = gpu_forward(sc)
    g = binding.XpbdGrads(d_compliance=None, d_x0=None, d_v0=None, d_f_global=None, d_f_vertex=None,
                          d_collider=ck.data_ptr(), d_f_vertex_steps=None)
    import ctypes as C
    o = binding.XpbdImplicitOpts(cg_tol=1e-8, cg_max_iters=10, pd_project=1, cg_iters_out=None)
    pc = p.c_struct()
    st = binding.lib().xpbd_adjoint_implicit(solver._h, C.byref(pc), sc.steps, sc.iters, C.c_void_p(ck.data_ptr()),
                                             0, None, None, None, C.byref(g), C.byref(o), None)
    assert st == 1


# ---- grid multigrid preconditioner (xpbd_implicit_opts.mg_*): the same solve, fewer iterations

def _ground_grid(n, steps=4, seed=41):
    """A cloth falling onto the ground (one diagonal, hinges on the axis-aligned edges), two
    corner pins: slack early steps (fold mechanisms along the diagonal), contacts later."""
    sc = helpers.small_cloth(n, bending=True, diagonals="one", pins=((0, 0), (-1, 0)), steps=steps, iters=8,
                             v_scale=0.2, plane_h=-0.03, seed=seed)
    sc.v0 = scenes.f32(sc.v0 + np.where(sc.inv_mass[:, None] > 0, np.array([0.0, -0.8, 0.0]), 0.0))
    return sc


@pytest.mark.parametrize("name,n,lines", [("pinned_cloth", 8, 0), ("ground_cloth", 8, 1), ("membrane", 8, 0),
                                          ("ground21_lines", 21, 1), ("ground21_points", 21, 0),
                                          ("ground24_lines", 24, 1)])
def test_multigrid_preconditioner_matches_oracle(name, n, lines):
    """Multigrid-preconditioned CG reaches the oracle's gradients (dense direct solves) on
    grids of 1 to 4 levels (21: odd sides 21 -> 11 -> 6 -> 3; 24: 24 -> 12 -> 6 -> 3), with
    point and diagonal-line smoothing, and needs no more iterations than block Jacobi."""
    sc = _cases()[name] if n == 8 else _ground_grid(n, seed=43 if n == 24 else 41)
    if n != 8:   # the GPU's float32 forward meets the same contact set as the oracle's
        xs_ref, vs_ref, _, _, act = oracle.forward_multipliers(sc)
        assert contact_margin(sc, xs_ref, vs_ref) > 1e-5 and act.any()
    rng = np.random.default_rng(18)
    seeds = {sc.steps: scenes.f32(rng.standard_normal((sc.V, 3))), 1: scenes.f32(rng.standard_normal((sc.V, 3)))}
    ref = implicit.adjoint(sc, seeds, pd=True)
    with oracle.fp32_rounding():
        ref32 = implicit.adjoint(sc, seeds, pd=True)
    solver, p, ck, xs, _ = gpu_forward(sc)
    keys = KEYS + (("memb_stiffness",) if sc.n_memb else ())
    dseeds = {k: to_dev(v) for k, v in seeds.items()}
    got, its = solver.adjoint_implicit(p, sc.steps, sc.iters, ck, dseeds, want=keys, multigrid=(n, n, lines))
    jac, its_j = solver.adjoint_implicit(p, sc.steps, sc.iters, ck, dseeds, want=keys)
    torch.cuda.synchronize()
    solver.sync_status()
    print(f"{name}: CG iterations per step, multigrid {its}, block Jacobi {its_j}")
    assert all(0 < k < 5000 for k in its), its
    assert max(its) <= max(its_j), (its, its_j)
    for k in keys:
        check_grad(f"implicit multigrid {name} {k}", got[k].cpu().numpy(), ref[k], GRAD_TOL, ref32=ref32[k])
        assert rel_err(got[k].cpu().numpy(), jac[k].cpu().numpy()) < 1e-6, k


def test_multigrid_is_deterministic_and_sweeps_cut_iterations():
    sc = _ground_grid(32, steps=3)
    solver, p, ck, _, _ = gpu_forward(sc)
    rng = np.random.default_rng(3)
    seeds = {sc.steps: to_dev(rng.standard_normal((sc.V, 3)))}
    a, its1 = solver.adjoint_implicit(p, sc.steps, sc.iters, ck, seeds, multigrid=(32, 32, 1, 1))
    b, its1b = solver.adjoint_implicit(p, sc.steps, sc.iters, ck, seeds, multigrid=(32, 32, 1, 1))
    _, its2 = solver.adjoint_implicit(p, sc.steps, sc.iters, ck, seeds, multigrid=(32, 32, 1, 2))
    _, its_j = solver.adjoint_implicit(p, sc.steps, sc.iters, ck, seeds)
    torch.cuda.synchronize()
    print(f"32^2 ground cloth: multigrid 1 sweep {its1}, 2 sweeps {its2}, block Jacobi {its_j}")
    assert its1 == its1b
    for k in a:
        assert torch.equal(a[k], b[k]), k
    assert max(its2) <= max(its1) and 4 * max(its1) < max(its_j), (its1, its2, its_j)


def test_multigrid_rejects_a_non_grid_model():
    sc = _cases()["pinned_cloth"]
    solver, p, ck, _, _ = gpu_forward(sc)
    seeds = {sc.steps: to_dev(np.ones((sc.V, 3)))}
    with pytest.raises(binding.XpbdError, match="vertex count"):
        solver.adjoint_implicit(p, sc.steps, sc.iters, ck, seeds, multigrid=(8, 9, 0))
    with pytest.raises(binding.XpbdError, match="mg_lines"):
        solver.adjoint_implicit(p, sc.steps, sc.iters, ck, seeds, multigrid=(8, 8, 2))
    # the right vertex count read as a 4 x 16 grid: constraints then couple vertices
    # more than two cells apart
    with pytest.raises(binding.XpbdError, match="two grid cells"):
        solver.adjoint_implicit(p, sc.steps, sc.iters, ck, seeds, multigrid=(4, 16, 0))
    tets = _cases()["tets"]
    solver, p, ck, _, _ = gpu_forward(tets)
    with pytest.raises(binding.XpbdError, match="two grid cells"):
        solver.adjoint_implicit(p, tets.steps, tets.iters, ck, {tets.steps: to_dev(np.ones((tets.V, 3)))},
                                multigrid=(tets.V, 1, 0))
