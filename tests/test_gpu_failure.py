"""Failure detection in the phase kernels without a GPU fault: a launch whose staged copies
are never issued makes every bounded wait run out; the kernel latches the timeout bit and
returns, the host reads XPBD_ERR_TIMEOUT, and the same context then simulates correctly."""
import numpy as np
import pytest
import torch

from paper_2301_01396_gb300 import binding
from tests import helpers
from tests.gpu_common import to_dev

pytestmark = pytest.mark.gpu


def _scene():
    return helpers.small_cloth(64, bending=True, diagonals="both", pins=(), steps=2, iters=3, v_scale=0.3,
                               seed=70, coloring="tiled", tile=16)


def test_bounded_wait_reports_timeout_and_context_stays_usable():
    sc = _scene()
    solver = binding.Solver.from_scene(sc, exec_mode=2)
    assert solver.exec_info()["phases"]
    p = binding.params_from_scene(sc)
    ref = solver.forward(p, sc.steps, sc.iters, to_dev(sc.x0), to_dev(sc.v0))
    torch.cuda.synchronize()
    solver.sync_status()
    solver.selftest_wait_timeout()
    with pytest.raises(binding.XpbdError) as e:
        solver.sync_status()
    assert e.value.status == 6 and "gave up waiting" in str(e.value)
    solver.sync_status()   # reported once, then cleared
    got = solver.forward(p, sc.steps, sc.iters, to_dev(sc.x0), to_dev(sc.v0))
    torch.cuda.synchronize()
    solver.sync_status()
    assert torch.equal(got, ref)


def test_selftest_needs_phase_kernels():
    sc = _scene()
    solver = binding.Solver.from_scene(sc, exec_mode=1)
    with pytest.raises(binding.XpbdError) as e:
        solver.selftest_wait_timeout()
    assert e.value.status == 1
