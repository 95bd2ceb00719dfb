"""Tet materials on the GPU (mu = a^2, lambda = b^2 per material): the compliance expansion
and the chain rule to (a, b) against the oracle's."""
import numpy as np
import pytest
import torch

import oracle
from oracle import materials
from paper_2301_01396_gb300 import binding, scenes
from tests import helpers
from tests.gpu_common import check_grad, oracle_adjoint_floor, rel_err, to_dev

pytestmark = pytest.mark.gpu


def test_material_compliance_and_gradient_match_oracle():
    sc = helpers.small_tets(3, steps=4, iters=4, y0=0.05, plane=False, v_scale=0.05)
    mat, a, b = scenes.tet_materials(sc.n_tet, 5, seed=6)
    solver = binding.Solver.from_scene(sc)
    d_mat = torch.as_tensor(mat, device="cuda")
    d_a, d_b = to_dev(a), to_dev(b)
    comp = solver.material_compliance(d_mat, d_a, d_b, to_dev(sc.compliance))
    torch.cuda.synchronize()
    solver.sync_status()
    ref_c = materials.compliance(sc, mat, a.astype(np.float64), b.astype(np.float64))
    assert rel_err(comp.cpu().numpy(), ref_c) < 1e-6
    sc.compliance = scenes.f32(comp.cpu().numpy())
    p = binding.params_from_scene(sc)
    ck = solver.forward(p, sc.steps, sc.iters, to_dev(sc.x0), to_dev(sc.v0))
    rng = np.random.default_rng(3)
    seed = scenes.f32(rng.standard_normal((sc.V, 3)))
    gr = solver.adjoint(p, sc.steps, sc.iters, ck, {sc.steps: to_dev(seed)}, want=("compliance",))
    da, db = solver.material_gradient(d_mat, d_a, d_b, gr["compliance"])
    torch.cuda.synchronize()
    ref, ref32 = oracle_adjoint_floor(sc, {sc.steps: seed})
    rda, rdb = materials.gradient(sc, ref["compliance"], mat, a.astype(np.float64), b.astype(np.float64))
    fda, fdb = materials.gradient(sc, ref32["compliance"], mat, a.astype(np.float64), b.astype(np.float64))
    check_grad("materials a", da.cpu().numpy(), rda, 1e-3, ref32=fda)
    check_grad("materials b", db.cpu().numpy(), rdb, 1e-3, ref32=fdb)
    da2, db2 = solver.material_gradient(d_mat, d_a, d_b, gr["compliance"])
    assert torch.equal(da, da2) and torch.equal(db, db2)        # fixed-order sums


def test_material_id_out_of_range_is_reported():
    sc = helpers.small_tets(2, steps=1, iters=1)
    solver = binding.Solver.from_scene(sc)
    mat = torch.zeros(sc.n_tet, dtype=torch.int32, device="cuda")
    mat[3] = 7
    solver.material_compliance(mat, to_dev(np.ones(2)), to_dev(np.ones(2)), to_dev(sc.compliance))
    with pytest.raises(binding.XpbdError) as e:
        solver.sync_status()
    assert e.value.status == 1
