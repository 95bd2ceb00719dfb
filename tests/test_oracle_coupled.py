"""Pins of the oracle's coupled tet update: a tet's hydrostatic and deviatoric constraints
projected together by one 2x2 solve (the volumetric model of Sec. 3.2 follows Macklin and
Mueller 2021, whose update is this coupled one), and its reverse."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2301_01396_gb300 import scenes
from tests.helpers import rel, small_tets


def _tet(rng, gamma=1.2):
    r = np.zeros(12)
    r[2:11] = np.linalg.inv(rng.standard_normal((3, 3)) + 2 * np.eye(3)).reshape(-1)
    r[11] = gamma
    return r


def _fd_grad(oracle_mod, kind, q, r, h=1e-6):
    return np.array([(oracle_mod.constraint(kind, q + h * e, r)[0] - oracle_mod.constraint(kind, q - h * e, r)[0])
                     / (2 * h) for e in np.eye(12)])


def test_coupled_update_solves_the_linearised_pair(oracle_mod):
    """After one coupled update both linearised conditions hold at once,
    C_k(q) + grad C_k . (q' - q) + alpha~_k lambda'_k = 0 for k = H, D, and the position
    change is W (grad C_H dlambda_H + grad C_D dlambda_D).  Gradients by central
    differences of C."""
    rng = np.random.default_rng(21)
    for trial in range(4):
        r = _tet(rng)
        q = rng.standard_normal(12)
        w = rng.uniform(0.5, 2.0, 4)
        if trial == 1:
            w[2] = 0.0                                     # one pinned vertex
        lam = rng.standard_normal(2) * 0.1
        at = rng.uniform(0.05, 0.5, 2)
        q2, lam2 = oracle_mod.project_pair(q, w, r, lam, at)
        gH, gD = _fd_grad(oracle_mod, "tet_h", q, r), _fd_grad(oracle_mod, "tet_d", q, r)
        CH, CD = oracle_mod.constraint("tet_h", q, r)[0], oracle_mod.constraint("tet_d", q, r)[0]
        dq = q2 - q
        assert abs(CH + gH @ dq + at[0] * lam2[0]) < 1e-8 * max(1.0, abs(CH))
        assert abs(CD + gD @ dq + at[1] * lam2[1]) < 1e-8 * max(1.0, abs(CD))
        dl = lam2 - lam
        W = np.repeat(w, 3)
        assert rel(dq, W * (gH * dl[0] + gD * dl[1])) < 1e-8


def test_coupled_update_differs_from_sequential_pair(oracle_mod):
    """The coupled update is not two single updates in a row: the sequential pair leaves
    the first constraint's linearised condition violated where the gradients overlap."""
    rng = np.random.default_rng(22)
    r = _tet(rng)
    q = rng.standard_normal(12)
    w = np.ones(4)
    at = np.array([0.1, 0.2])
    qc, _ = oracle_mod.project_pair(q, w, r, np.zeros(2), at)
    q1, lh = oracle_mod.project_one("tet_h", q, w, r, 0.0, at[0])
    q1, ld = oracle_mod.project_one("tet_d", q1, w, r, 0.0, at[1])
    gH = _fd_grad(oracle_mod, "tet_h", q, r)
    CH = oracle_mod.constraint("tet_h", q, r)[0]
    assert abs(gH @ (q1 - q) + CH + at[0] * lh) > 1e-3
    assert rel(qc, q1) > 1e-3


def test_coupled_vjp_matches_fd_jacobian(oracle_mod):
    """The reverse of the coupled update equals the transpose of its finite-difference
    Jacobian with respect to (q, lambda_H, lambda_D, alpha~_H, alpha~_D)."""
    rng = np.random.default_rng(23)
    for trial in range(3):
        r = _tet(rng)
        q = rng.standard_normal(12)
        w = rng.uniform(0.5, 2.0, 4)
        if trial == 2:
            w[0] = 0.0
        lam = rng.standard_normal(2) * 0.2
        at = rng.uniform(0.05, 0.5, 2)

        def F(z):
            q2, l2 = oracle_mod.project_pair(z[:12], w, r, z[12:14], z[14:16])
            return np.r_[q2, l2]

        z0 = np.r_[q, lam, at]
        h = 1e-6
        J = np.stack([(F(z0 + h * e) - F(z0 - h * e)) / (2 * h) for e in np.eye(16)], axis=1)
        qbar = rng.standard_normal(12)
        lbar = rng.standard_normal(2)
        qb, lb, ab = oracle_mod.vjp_pair(q, w, r, lam, at, qbar, lbar)
        assert rel(np.r_[qb, lb, ab], J.T @ np.r_[qbar, lbar]) < 1e-7


def _residuals(oracle_mod, sc, iters):
    xs, _, lam, _, _ = oracle_mod.forward_multipliers(sc, iters=iters)
    rd = oracle_mod.rest_data(sc)
    nt, x = sc.n_tet, xs[-1]
    out = np.zeros(sc.m)
    for j in range(sc.m):
        t = j % nt
        r = rd[j].copy()
        vol, r[11] = r[11], sc.tet_gamma[t]
        Cj = oracle_mod.constraint("tet_h" if j < nt else "tet_d", x[sc.tet_idx[t]], r)[0]
        out[j] = Cj + sc.compliance[j] / vol / sc.dt ** 2 * lam[-1, j]
    return out


def test_coupled_iteration_reaches_both_conditions(oracle_mod):
    """Gauss-Seidel over coupled tets drives C_k + alpha~_k lambda_k to zero for both
    constraints of every tet (the fixed point of the XPBD iteration), and after a few
    iterations leaves a smaller residual than the one-constraint-at-a-time sweep."""
    sc = small_tets(2, steps=6, iters=3, y0=0.004, v_scale=0.05)
    cs = scenes.couple_tets(sc)
    assert np.abs(_residuals(oracle_mod, cs, 60)).max() < 1e-10
    assert np.abs(_residuals(oracle_mod, cs, 3)).max() < 0.2 * np.abs(_residuals(oracle_mod, sc, 3)).max()


def test_couple_tets_coloring(oracle_mod):
    """The coupled coloring lists every C_H id once and no C_D id; a scene whose tet
    block has no C_D in any color keeps its vertex-disjointness."""
    sc = small_tets(2)
    cs = scenes.couple_tets(sc)
    scenes.validate_coloring(cs)
    assert cs.n_colored == sc.m - sc.n_tet
    assert np.all(np.sort(cs.color_order) == np.arange(sc.n_tet))
    with pytest.raises(ValueError):
        scenes.validate_coloring(cs.with_(tet_coupled=False))


def test_coupled_sweep_sensitivity_on_stiff_tets(oracle_mod):
    """Finding: on stiff tets (inverse moduli down to 1e-5) the coupled sweep is far more
    sensitive to its start state than the one-constraint sweep.  The rest state carries a
    pre-stress (gamma = 1 + alpha_H / alpha_D), so every step rebuilds two large multipliers
    of opposite pull along nearly parallel gradients (parallel at F = I) from lambda = 0,
    and the positions are a small difference of large terms.  In exact arithmetic a 1e-8
    perturbation of x0 grows about 67-fold within 6 steps coupled and shrinks (0.22x)
    uncoupled; with inverse moduli in [1e-4, 1e-2] both sweeps shrink it (0.5x).  (The GPU
    parity cases of the coupled path therefore use the softer range.)"""
    def growth(alpha, coupled):
        sc = small_tets(4, steps=6, iters=10, y0=0.05, plane=False, v_scale=0.05, alpha=alpha)
        if coupled:
            sc = scenes.couple_tets(sc)
        d = np.random.default_rng(0).standard_normal(sc.x0.shape) * 1e-8
        xa, _ = oracle_mod.forward(sc)
        xb, _ = oracle_mod.forward(sc, x0=sc.x0 + d)
        return np.abs(xa[-1] - xb[-1]).max() / np.abs(d).max()
    assert growth((1e-5, 1e-3), True) > 30.0
    assert growth((1e-5, 1e-3), False) < 1.0
    assert growth((1e-4, 1e-2), True) < 1.0


def test_coupled_update_falls_back_to_c_h_when_c_d_is_degenerate(oracle_mod):
    """A tet collapsed to a point has F = 0, so C_D = |F| has no gradient: the pair update
    is then the single C_H update (which moves nothing either, cof F = 0, but builds
    lambda_H against alpha~_H), and lambda_D is left alone."""
    rng = np.random.default_rng(24)
    r = _tet(rng)
    q = np.tile(rng.standard_normal(3), 4)
    w = np.ones(4)
    at = np.array([0.2, 0.3])
    lam = np.array([0.1, -0.4])
    q2, lam2 = oracle_mod.project_pair(q, w, r, lam, at)
    q1, lh = oracle_mod.project_one("tet_h", q, w, r, lam[0], at[0])
    assert np.array_equal(q2, q1) and lam2[0] == lh and lam2[1] == lam[1]
    CH = oracle_mod.constraint("tet_h", q, r)[0]
    assert abs(lh - (lam[0] + (-CH - at[0] * lam[0]) / at[0])) < 1e-12
