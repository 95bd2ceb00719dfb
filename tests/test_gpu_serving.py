"""Continuous-batching server: each request's result is the same alone and in a mix of
requests of different sizes, horizons and iteration counts admitted while others run; it
matches the one-request C-ABI path and the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2301_01396_gb300 import binding, scenes
from tests import helpers
from tests.gpu_common import check_grad, oracle_adjoint_floor, rel_err, to_dev

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-3
KEYS = ("compliance", "x0", "v0", "f_vertex", "collider")


def _requests():
    """Cloth requests of several sizes and horizons, some on a ground plane, some pinned."""
    out = []
    for k, (n, steps, iters, ground, pins) in enumerate([(12, 5, 4, True, ((0, 0),)), (24, 3, 6, False, ()),
                                                         (40, 4, 3, True, ((0, 0), (-1, 0))), (17, 6, 5, True, ()),
                                                         (33, 2, 7, False, ((5, 0),))]):
        sc = helpers.small_cloth(n, bending=True, diagonals="one", steps=steps, iters=iters, pins=pins,
                                 plane_h=-0.02 if ground else None, v_scale=0.3, seed=40 + k)
        rng = np.random.default_rng(100 + k)
        target = scenes.f32(sc.x0 + 0.05 * rng.standard_normal(sc.x0.shape))
        out.append((sc, target))
    return out


def _submit(server, sc, target, keep):
    solver = binding.Solver.from_scene(sc)
    p = binding.params_from_scene(sc)
    x0, v0, tg = to_dev(sc.x0), to_dev(sc.v0), to_dev(target)
    keep.append((solver, p, x0, v0, tg))
    return server.submit(solver, p, sc.steps, sc.iters, x0, v0, tg, want=KEYS)


def _host(res):
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in res.items()}


def test_alone_equals_mix_and_single_request_api():
    reqs = _requests()
    # alone: one server per request
    alone = []
    for sc, target in reqs:
        srv = binding.Server(max_slots=4)
        keep = []
        t = _submit(srv, sc, target, keep)
        srv.drain([t], max_ticks=16)
        alone.append(_host(srv.result(t)))
        srv.close()
    # mix: continuous admission, new requests arrive while earlier ones run
    srv = binding.Server(max_slots=8)
    keep = []
    tickets = []
    for j, (sc, target) in enumerate(reqs):
        tickets.append(_submit(srv, sc, target, keep))
        srv.run(max_ticks=7 + 3 * j)            # advance the resident ones before the next arrives
    srv.drain(tickets, max_ticks=16)
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["active"] == 0 and st["bytes_in_use"] == 0
    assert st["items"] > st["ticks"]              # passes of several requests shared launches
    for j, t in enumerate(tickets):
        mixed = _host(srv.result(t))
        for k in alone[j]:
            assert np.array_equal(mixed[k], alone[j][k]), (j, k)
    # the one-request API on the same inputs, launched color by color like the server (its
    # multi-color phase launches are compared with this mode in the parity tests): the same
    # element code compiled into other kernels, so the two agree to float32 rounding
    for j, (sc, target) in enumerate(reqs):
        solver = binding.Solver.from_scene(sc, exec_mode=1)
        p = binding.params_from_scene(sc)
        ck = solver.forward(p, sc.steps, sc.iters, to_dev(sc.x0), to_dev(sc.v0))
        loss, seeds = solver.loss(ck, {sc.steps: to_dev(target)})
        gr = solver.adjoint(p, sc.steps, sc.iters, ck, {sc.steps: seeds[0]}, want=KEYS)
        ref = _host(gr)
        assert abs(loss.item() - alone[j]["loss"][0]) <= 1e-9 * abs(loss.item())
        for k in KEYS:
            assert rel_err(alone[j][k], ref[k]) <= 1e-5, (j, k)


def test_matches_oracle():
    sc, target = _requests()[3]
    srv = binding.Server(max_slots=2)
    keep = []
    t = _submit(srv, sc, target, keep)
    srv.drain([t])
    got = _host(srv.result(t))
    xs, _ = oracle.forward(sc)
    seed = xs[-1] - target
    assert abs(got["loss"][0] - 0.5 * np.sum(seed ** 2)) <= 1e-4 * got["loss"][0]
    ref, ref32 = oracle_adjoint_floor(sc, {sc.steps: scenes.f32(seed)})
    for k in ("compliance", "x0", "v0", "f_vertex"):
        check_grad(f"serving {k}", got[k], ref[k], GRAD_TOL, ref32=ref32[k])


def test_admission_waits_for_memory():
    """Three equal requests and a budget for 1.5 of them: they run one after another."""
    sc, target = _requests()[2]
    reqs = [(sc, target), (sc, scenes.f32(target + 0.01)), (sc, scenes.f32(target - 0.01))]
    need = binding.Server.request_bytes(binding.Solver.from_scene(sc), sc.steps, sc.iters, sc.collider_flags)
    budget = int(need * 1.5)
    srv = binding.Server(budget=budget, max_slots=8)
    keep = []
    tickets = [_submit(srv, sc, target, keep) for sc, target in reqs]
    max_active = 0
    pending = list(tickets)
    while pending:
        max_active = max(max_active, srv.run(8))
        pending = [t for t in pending if not srv.poll(t)]
    assert max_active == 1
    assert srv.stats()["completed"] == 3


def test_oversized_request_is_rejected():
    sc, target = _requests()[2]
    srv = binding.Server(budget=1 << 20, max_slots=2)
    with pytest.raises(binding.XpbdError) as e:
        _submit(srv, sc, target, [])
    assert e.value.status == 3
