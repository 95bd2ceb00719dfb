"""The allocation-free forward entry point (xpbd_forward_static) against xpbd_forward.

xpbd_forward_static serves callers that cannot allocate device memory while they simulate
(another allocator owns the memory under a fixed budget, or cudaMalloc's implicit device
synchronisation is not acceptable in their loop); it keeps its working state in one fixed
array inside the library, whose device address xpbd_create looks up.  This file is
collected last on purpose, and each test also passes when run alone in a fresh process."""
import numpy as np
import pytest
import torch

from paper_2301_01396_gb300 import binding, scenes
from tests import helpers
from tests.gpu_common import to_dev

pytestmark = pytest.mark.gpu

POS_TOL = 1e-5   # the position tolerance of the parity tests


def _device_memory():
    """(free device bytes, bytes the caching allocator holds, its allocation count)."""
    torch.cuda.synchronize()
    st = torch.cuda.memory_stats()
    return (torch.cuda.mem_get_info()[0], st.get("reserved_bytes.all.current", 0),
            st.get("allocation.all.allocated", 0))


def test_static_forward_allocates_nothing_on_a_fresh_handle():
    """A fresh handle calls the static entry point before anything else (so nothing of the
    allocating path's workspace exists), then once more with every buffer in place: across
    that warm call the device's free memory and the caching allocator are unchanged.  Only
    then is the allocating entry point run, and the results compared."""
    sc = helpers.small_cloth(32, bending=True, diagonals="one", steps=5, iters=6, plane_h=-0.03,
                             v_scale=0.3, seed=31)
    solver = binding.Solver.from_scene(sc, exec_mode=1)
    p = binding.params_from_scene(sc)
    x0, v0 = to_dev(sc.x0), to_dev(sc.v0)
    ck1, ck2 = solver.new_checkpoints(sc.steps), solver.new_checkpoints(sc.steps)
    solver.forward_static(p, sc.steps, sc.iters, x0, v0, ck1)     # first call: kernels load
    before = _device_memory()
    solver.forward_static(p, sc.steps, sc.iters, x0, v0, ck2)
    after = _device_memory()
    solver.sync_status()
    assert after == before, (before, after)
    assert torch.equal(ck1, ck2)
    ref = solver.forward(p, sc.steps, sc.iters, x0, v0)
    torch.cuda.synchronize()
    assert (ck2 - ref)[:, :, :, :3].abs().max().item() <= POS_TOL


def test_static_forward_matches_allocating_forward_on_two_calls():
    """Two calls in a row with different inputs (the second sees what the first left in the
    shared array), each compared with the allocating entry point on the same inputs."""
    sc = helpers.small_cloth(48, bending=True, diagonals="one", steps=6, iters=8, plane_h=-0.03,
                             v_scale=0.3, seed=33)
    # the allocating entry point in its color-by-color mode, the launch structure the static
    # entry point uses (the multi-color phase mode is compared with it in the parity tests)
    solver = binding.Solver.from_scene(sc, exec_mode=1)
    p = binding.params_from_scene(sc)
    x0 = to_dev(sc.x0)
    inputs = [to_dev(sc.v0), to_dev(0.5 * sc.v0 + np.array([0.0, -0.4, 0.0]) * (sc.inv_mass[:, None] > 0))]
    for v0 in inputs:
        ref = solver.forward(p, sc.steps, sc.iters, x0, v0)
        got = solver.forward_static(p, sc.steps, sc.iters, x0, v0, solver.new_checkpoints(sc.steps))
        torch.cuda.synchronize()
        solver.sync_status()
        d = (got - ref)[:, :, :, :3].abs().max().item()
        assert d <= POS_TOL, d


def test_static_forward_on_a_phase_plan_handle():
    """A handle in the multi-color phase mode (a tiled coloring): the static entry point
    still runs one launch per color, which agrees with the phase kernels to float32
    rounding."""
    sc = helpers.small_cloth(64, bending=True, diagonals="both", steps=4, iters=6, plane_h=-0.03,
                             v_scale=0.3, seed=35, coloring="tiled", tile=16)
    solver = binding.Solver.from_scene(sc)
    assert solver.exec_info()["phases"]
    p = binding.params_from_scene(sc)
    x0, v0 = to_dev(sc.x0), to_dev(sc.v0)
    ref = solver.forward(p, sc.steps, sc.iters, x0, v0)
    for _ in range(2):
        got = solver.forward_static(p, sc.steps, sc.iters, x0, v0, solver.new_checkpoints(sc.steps))
        torch.cuda.synchronize()
        solver.sync_status()
        assert (got - ref)[:, :, :, :3].abs().max().item() <= POS_TOL


def test_static_forward_at_its_vertex_limit():
    """The 256 x 256 ground cloth (65,536 vertices, exactly the limit; 325,125 constraints)
    is accepted and matches the allocating entry point."""
    sc = scenes.ground_cloth(256, steps=2)
    assert sc.V == binding.STATIC_MAX_VERTICES and sc.m <= binding.STATIC_MAX_CONSTRAINTS
    solver = binding.Solver.from_scene(sc)
    p = binding.params_from_scene(sc)
    x0, v0 = to_dev(sc.x0), to_dev(sc.v0)
    got = solver.forward_static(p, sc.steps, sc.iters, x0, v0, solver.new_checkpoints(sc.steps))
    ref = solver.forward(p, sc.steps, sc.iters, x0, v0)
    torch.cuda.synchronize()
    solver.sync_status()
    assert (got - ref)[:, :, :, :3].abs().max().item() <= POS_TOL


def test_static_forward_tet_block_with_contacts():
    sc = helpers.small_tets(4, steps=5, iters=6, y0=0.004, v_scale=0.05)
    solver = binding.Solver.from_scene(sc, exec_mode=1)
    p = binding.params_from_scene(sc)
    x0, v0 = to_dev(sc.x0), to_dev(sc.v0)
    ref = solver.forward(p, sc.steps, sc.iters, x0, v0)
    for _ in range(2):
        got = solver.forward_static(p, sc.steps, sc.iters, x0, v0, solver.new_checkpoints(sc.steps))
        torch.cuda.synchronize()
        assert (got - ref)[:, :, :, :3].abs().max().item() <= POS_TOL


def test_static_forward_coupled_tets():
    sc = scenes.couple_tets(helpers.small_tets(4, steps=5, iters=6, y0=0.004, v_scale=0.05))
    solver = binding.Solver.from_scene(sc, exec_mode=1)
    p = binding.params_from_scene(sc)
    x0, v0 = to_dev(sc.x0), to_dev(sc.v0)
    ref = solver.forward(p, sc.steps, sc.iters, x0, v0)
    got = solver.forward_static(p, sc.steps, sc.iters, x0, v0, solver.new_checkpoints(sc.steps))
    torch.cuda.synchronize()
    solver.sync_status()
    assert torch.equal(got, ref)


def test_static_forward_rejects_models_beyond_its_limit():
    sc = scenes.plain_cloth(257, steps=1, iters=1)          # 66,049 vertices > 65,536
    assert sc.V > binding.STATIC_MAX_VERTICES
    solver = binding.Solver.from_scene(sc)
    p = binding.params_from_scene(sc)
    with pytest.raises(binding.XpbdError) as e:
        solver.forward_static(p, 1, 1, to_dev(sc.x0), to_dev(sc.v0), solver.new_checkpoints(1))
    assert e.value.status == 7 and "at most 65536 vertices" in str(e.value)
    assert f"this model has {sc.V} vertices" in str(e.value)
