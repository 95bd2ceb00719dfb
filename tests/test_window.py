"""The window argument the full-size GPU parity tests rest on, checked on the oracle alone.

A color pass moves information at most two grid vertices (a bending hinge spans rows
j-1..j+1), so after I iterations of K colors a vertex farther than R = 2 K I + 4 from a
window's edge does not see that edge: the oracle run on the window reproduces the full run
there, bit for bit, when the window keeps the full run's color order.  Here both runs are
the oracle's, on the benched cloth's tiled coloring (64 colors, 32 x 32 tiles) at a size
the oracle runs in seconds."""
import numpy as np

import oracle
from paper_2301_01396_gb300 import scenes
from tests import helpers


def _cloth(n, iters):
    sc = scenes.sphere_cloth(n, steps=1, iters=iters, coloring="tiled", tile=32)
    x, z = sc.x0[:, 0], sc.x0[:, 2]
    sc.v0 = scenes.f32(0.3 * np.stack([np.sin(2 * np.pi * z + 0.3), np.sin(2 * np.pi * (x + z)),
                                        np.cos(2 * np.pi * x - 0.7)], axis=1))
    return sc


def test_forward_window_core_is_the_full_run():
    n, I = 700, 2
    full = _cloth(n, I)
    R = 2 * full.n_colors * I + 4
    w = 608
    xs, _ = oracle.forward(full, 1, I)
    sub, sel, _, _ = helpers.grid_window(full, n, 32, 64, w)
    xw, _ = oracle.forward(sub, 1, I)
    core = np.zeros((w, w), bool)
    core[R:w - R, R:w - R] = True
    core = core.reshape(-1)
    assert np.array_equal(xs[1][sel][core], xw[1][core])
    assert np.abs(xs[1][sel][~core] - xw[1][~core]).max() > 1e-6      # the edge does differ


def test_adjoint_window_band_is_the_full_run():
    n, I = 900, 1
    full = _cloth(n, I)
    R = 2 * full.n_colors * I + 4
    w = 6 * R + 48
    sub, sel, kd, kb = helpers.grid_window(full, n, 20, 30, w)
    li, lj = np.meshgrid(np.arange(w), np.arange(w), indexing="xy")
    dist_edge = np.minimum(np.minimum(li, w - 1 - li), np.minimum(lj, w - 1 - lj)).reshape(-1)
    rng = np.random.default_rng(15)
    seed_local = scenes.f32(rng.standard_normal((sub.V, 3)) * (dist_edge >= 3 * R)[:, None])
    seed_full = np.zeros((full.V, 3), np.float32)
    seed_full[sel] = seed_local
    gw = oracle.adjoint(sub, {1: seed_local}, 1, I)
    gf = oracle.adjoint(full, {1: seed_full}, 1, I)
    band = dist_edge >= 2 * R
    for k in ("x0", "v0", "f_vertex"):
        assert np.array_equal(gf[k][sel][band], gw[k][band]), k
        assert np.abs(gw[k][~band]).max() == 0.0 and np.abs(gf[k][sel][~band]).max() == 0.0, k
    ids = np.concatenate([kd, kb])
    assert np.array_equal(gf["compliance"][ids], gw["compliance"])
    assert np.abs(gw["compliance"]).max() > 0
    rest = np.ones(full.m, bool)
    rest[ids] = False
    assert np.abs(gf["compliance"][rest]).max() == 0.0
    assert np.allclose(gf["f_global"], gw["f_global"], rtol=1e-12, atol=0)
