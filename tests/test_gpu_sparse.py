"""Sparse checkpoints: the stored states equal the dense forward's, and the reverse sweep
that recomputes the states between them gives gradients bit-identical to the dense one."""
import numpy as np
import pytest
import torch

from paper_2301_01396_gb300 import binding, scenes
from tests import helpers
from tests.gpu_common import to_dev

pytestmark = pytest.mark.gpu

KEYS = ("compliance", "x0", "v0", "f_global", "f_vertex", "collider", "f_vertex_steps")


def _sphere_cloth():
    sc = helpers.small_sphere_cloth(12, steps=7, iters=3, seed=4)
    rng = np.random.default_rng(8)
    sc.f_vertex_steps = scenes.f32(0.3 * 2.56 / sc.V * 9.81 * rng.standard_normal((sc.steps, sc.V, 3)))
    return sc


def _scenes():
    return {
        "sphere_cloth": _sphere_cloth(),
        "ground_cloth_tiled": helpers.small_cloth(64, bending=True, diagonals="both", pins=(), steps=7, iters=3,
                                                  v_scale=0.3, plane_h=-0.02, seed=33, coloring="tiled", tile=16),
        "tets": helpers.small_tets(3, steps=7, iters=3, y0=0.004, v_scale=0.05),
        "tets_coupled": scenes.couple_tets(helpers.small_tets(3, steps=7, iters=3, y0=0.004, v_scale=0.05)),
    }


@pytest.mark.parametrize("name", ["sphere_cloth", "ground_cloth_tiled", "tets", "tets_coupled"])
@pytest.mark.parametrize("stride", [1, 2, 3, 7, 10])
def test_sparse_equals_dense(name, stride):
    sc = _scenes()[name]
    solver = binding.Solver.from_scene(sc)
    p = binding.params_from_scene(sc)
    x0, v0 = to_dev(sc.x0), to_dev(sc.v0)
    rng = np.random.default_rng(5)
    seeds = {k: to_dev(rng.standard_normal((sc.V, 3))) for k in (2, 5, sc.steps)}   # 2 and 5 are not stored
    ck = solver.forward(p, sc.steps, sc.iters, x0, v0)
    cks = solver.forward_sparse(p, sc.steps, sc.iters, x0, v0, stride)
    torch.cuda.synchronize()
    solver.sync_status()
    assert cks.shape[0] == binding.sparse_slots(sc.steps, stride)
    for n in range(sc.steps + 1):
        s = binding.sparse_slot(sc.steps, stride, n)
        if s >= 0:
            assert torch.equal(cks[s], ck[n]), n
    ref = solver.adjoint(p, sc.steps, sc.iters, ck, seeds, want=KEYS)
    got = solver.adjoint(p, sc.steps, sc.iters, cks, seeds, want=KEYS, stride=stride)
    torch.cuda.synchronize()
    solver.sync_status()
    for k in KEYS:
        assert torch.equal(got[k], ref[k]), k


def test_loss_reads_a_sparse_buffer_by_slot():
    sc = _scenes()["sphere_cloth"]
    solver = binding.Solver.from_scene(sc)
    p = binding.params_from_scene(sc)
    ck = solver.forward(p, sc.steps, sc.iters, to_dev(sc.x0), to_dev(sc.v0))
    cks = solver.forward_sparse(p, sc.steps, sc.iters, to_dev(sc.x0), to_dev(sc.v0), 3)
    target = to_dev(scenes.f32(sc.x0 + 0.01))
    l_dense, s_dense = solver.loss(ck, {6: target})
    l_sparse, s_sparse = solver.loss(cks, {binding.sparse_slot(sc.steps, 3, 6): target})
    assert torch.equal(l_dense, l_sparse) and torch.equal(s_dense, s_sparse)


def test_bad_stride_is_rejected():
    sc = _scenes()["sphere_cloth"]
    solver = binding.Solver.from_scene(sc)
    p = binding.params_from_scene(sc)
    with pytest.raises(binding.XpbdError) as e:
        solver.forward_sparse(p, sc.steps, sc.iters, to_dev(sc.x0), to_dev(sc.v0), 0)
    assert e.value.status == 1
