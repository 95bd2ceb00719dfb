"""Pins of the oracle's orthotropic StVK membrane (Sec. "Cloth Material Parameter
Estimation"): C = (E_uu, E_vv, 2 E_uv) of the Green strain E = (F^T F - I)/2 per triangle,
compliance block (A K)^-1 with K = [C00 C01 .; C01 C11 .; . . C22], the three multipliers
solved together, and its reverse."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2301_01396_gb300 import scenes
from tests.helpers import rel

KINDS = ("memb_uu", "memb_vv", "memb_uv")


def _rest12(B2):
    r = np.zeros(12)
    r[2:6] = np.asarray(B2, np.float64).reshape(-1)
    return r


def _tri(rng):
    uv = rng.standard_normal((3, 2))
    Dm = np.stack([uv[1] - uv[0], uv[2] - uv[0]], axis=1)
    if np.linalg.det(Dm) < 0:
        uv[[1, 2]] = uv[[2, 1]]
        Dm = np.stack([uv[1] - uv[0], uv[2] - uv[0]], axis=1)
    return uv, np.linalg.inv(Dm)


def _C(oracle_mod, q, B2):
    return np.array([oracle_mod.constraint(k, q, _rest12(B2))[0] for k in KINDS])


def _grads(oracle_mod, q, B2):
    return np.stack([oracle_mod.constraint(k, q, _rest12(B2))[1] for k in KINDS])


def test_green_strain_of_an_affine_map(oracle_mod):
    """Vertices x_i = R F uv_i + t (any rotation R, translation t, 3x2 map F): the constraint
    is (E_uu, E_vv, 2 E_uv) of E = (F^T F - I)/2 computed from F directly."""
    rng = np.random.default_rng(31)
    for _ in range(5):
        uv, B2 = _tri(rng)
        F = rng.standard_normal((3, 2))
        Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
        x = uv @ F.T @ Q.T + rng.standard_normal(3)
        E = 0.5 * ((Q @ F).T @ (Q @ F) - np.eye(2))
        got = _C(oracle_mod, x.reshape(-1), B2)
        assert np.allclose(got, [E[0, 0], E[1, 1], 2 * E[0, 1]], atol=1e-12)
    # the rest shape (F = the embedding of the identity) is strain free
    uv, B2 = _tri(rng)
    x = np.stack([uv[:, 0], np.zeros(3), uv[:, 1]], axis=1)
    assert np.abs(_C(oracle_mod, x.reshape(-1), B2)).max() < 1e-14


def test_membrane_derivatives(oracle_mod):
    """AD gradient vs central differences; the Hessian is constant (E is quadratic in x)
    and symmetric; forces sum to zero (translation invariance)."""
    rng = np.random.default_rng(32)
    uv, B2 = _tri(rng)
    q = rng.standard_normal(9)
    q2 = rng.standard_normal(9)
    h = 1e-6
    for k in KINDS:
        r = _rest12(B2)
        _, g, _ = oracle_mod.constraint(k, q, r)
        g_fd = np.array([(oracle_mod.constraint(k, q + h * e, r)[0] - oracle_mod.constraint(k, q - h * e, r)[0]) / (2 * h)
                         for e in np.eye(9)])
        assert rel(g, g_fd) < 1e-8
        H = np.stack([oracle_mod.constraint(k, q, r, u=e)[2] for e in np.eye(9)], axis=1)
        H2 = np.stack([oracle_mod.constraint(k, q2, r, u=e)[2] for e in np.eye(9)], axis=1)
        assert np.abs(H - H.T).max() < 1e-12 * max(1.0, np.abs(H).max())
        assert np.abs(H - H2).max() < 1e-12 * max(1.0, np.abs(H).max())
        assert np.abs(g.reshape(3, 3).sum(0)).max() < 1e-12 * max(1.0, np.abs(g).max())


def _alpha_tilde(K, area, dt):
    c00, c11, c01, c22 = K
    A = np.zeros((3, 3))
    A[:2, :2] = np.linalg.inv(np.array([[c00, c01], [c01, c11]]))
    A[2, 2] = 1.0 / c22
    return A / (area * dt * dt)


def test_membrane_update_solves_the_linearised_system(oracle_mod):
    """After one update all three linearised conditions hold at once,
    C_k + grad C_k . dx + (A~ lambda')_k = 0, with dx = W G^T dlambda (gradients by central
    differences)."""
    rng = np.random.default_rng(33)
    for trial in range(4):
        uv, B2 = _tri(rng)
        q = (np.stack([uv[:, 0], np.zeros(3), uv[:, 1]], axis=1) + 0.2 * rng.standard_normal((3, 3))).reshape(-1)
        w = rng.uniform(0.5, 2.0, 3)
        if trial == 1:
            w[0] = 0.0
        at = _alpha_tilde(rng.uniform(0.5, 2.0, 4) * np.array([1.0, 1.0, 0.2, 1.0]), 0.7, 0.9)
        lam = 0.1 * rng.standard_normal(3)
        q2, lam2 = oracle_mod.project_memb(q, w, B2, lam, at)
        h = 1e-6
        G = np.stack([[(_C(oracle_mod, q + h * e, B2)[k] - _C(oracle_mod, q - h * e, B2)[k]) / (2 * h)
                       for e in np.eye(9)] for k in range(3)])
        C0 = _C(oracle_mod, q, B2)
        dq = q2 - q
        assert np.abs(C0 + G @ dq + at @ lam2).max() < 1e-8 * max(1.0, np.abs(C0).max())
        assert rel(dq, np.repeat(w, 3) * (G.T @ (lam2 - lam))) < 1e-7


@pytest.mark.parametrize("axis", ["warp", "weft"])
def test_uniaxial_stretch_reduces_to_the_scalar_update(oracle_mod, axis):
    """Unit right triangle (u, v) = (0,0), (1,0), (0,1) with C01 = 0 and only the vertex on
    the stretched axis free, stretched by e along it: the shear and the other normal strain
    stay zero, so the update is the scalar XPBD update of E along that axis with
    compliance 1/(A C dt^2), C = C00 for the warp and C11 for the weft (A = 1/2)."""
    e, dt, w = 0.1, 0.05, 3.0
    K = (800.0, 300.0, 0.0, 200.0)
    x = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    free = 1 if axis == "warp" else 2
    comp = 0 if axis == "warp" else 2
    x[free, comp] += e
    wv = np.zeros(3)
    wv[free] = w
    at = _alpha_tilde(K, 0.5, dt)
    q2, lam2 = oracle_mod.project_memb(x.reshape(-1), wv, np.eye(2), np.zeros(3), at)
    s = 1.0 + e
    C = 0.5 * (s * s - 1.0)
    a = 1.0 / (0.5 * (K[0] if axis == "warp" else K[1]) * dt * dt)
    dl = -C / (w * s * s + a)
    expect = x.copy()
    expect[free, comp] = s + w * s * dl
    assert np.allclose(q2.reshape(3, 3), expect, atol=1e-13)
    assert abs(lam2[0 if axis == "warp" else 1] - dl) < 1e-13
    assert abs(lam2[1 if axis == "warp" else 0]) < 1e-13 and abs(lam2[2]) < 1e-13


def test_membrane_vjp_matches_fd_jacobian(oracle_mod):
    """The reverse of one update equals the transposed finite-difference Jacobian in
    (q, lambda, alpha~ entries 00, 11, 01 = 10, 22)."""
    rng = np.random.default_rng(34)
    for trial in range(3):
        uv, B2 = _tri(rng)
        q = (np.stack([uv[:, 0], np.zeros(3), uv[:, 1]], axis=1) + 0.2 * rng.standard_normal((3, 3))).reshape(-1)
        w = rng.uniform(0.5, 2.0, 3)
        if trial == 2:
            w[1] = 0.0
        lam = 0.1 * rng.standard_normal(3)
        a4 = np.array([0.8, 0.6, 0.1, 0.5])

        def A(a):
            return np.array([[a[0], a[2], 0.0], [a[2], a[1], 0.0], [0.0, 0.0, a[3]]])

        def F(z):
            q2, l2 = oracle_mod.project_memb(z[:9], w, B2, z[9:12], A(z[12:16]))
            return np.r_[q2, l2]

        z0 = np.r_[q, lam, a4]
        h = 1e-6
        J = np.stack([(F(z0 + h * e) - F(z0 - h * e)) / (2 * h) for e in np.eye(16)], axis=1)
        qbar, lbar = rng.standard_normal(9), rng.standard_normal(3)
        qb, lb, ab = oracle_mod.vjp_memb(q, w, B2, lam, A(a4), qbar, lbar)
        assert rel(np.r_[qb, lb, ab], J.T @ np.r_[qbar, lbar]) < 1e-7


def _membrane_scene():
    sc = scenes.membrane_cloth(6, steps=5, iters=4, seed=4)
    rng = np.random.default_rng(35)
    v = 0.3 * rng.standard_normal(sc.x0.shape)
    v[sc.inv_mass == 0] = 0.0
    sc.v0 = scenes.f32(v)
    return sc


def test_membrane_rest_state_is_fixed_without_gravity(oracle_mod):
    sc = scenes.membrane_cloth(6, steps=4, iters=5).with_(gravity=(0.0, 0.0, 0.0))
    xs, _ = oracle_mod.forward(sc)
    assert np.abs(xs - xs[0]).max() < 1e-12


def test_membrane_adjoint_equals_tangent(oracle_mod):
    sc = _membrane_scene()
    rng = np.random.default_rng(36)
    N = sc.steps
    seed_T = rng.standard_normal((sc.V, 3))
    gr = oracle_mod.adjoint(sc, {N: seed_T})
    dirs = {"memb_stiffness": sc.memb_stiffness * rng.standard_normal(sc.memb_stiffness.shape),
            "compliance": sc.compliance * rng.standard_normal(sc.m),
            "x0": 1e-3 * rng.standard_normal((sc.V, 3)), "v0": rng.standard_normal((sc.V, 3))}
    for key, d in dirs.items():
        dxs, _ = oracle_mod.tangent(sc, {key: d})
        lhs = float(np.sum(gr[key] * d))
        rhs = float(np.sum(dxs[N] * seed_T))
        assert abs(lhs - rhs) <= 1e-9 * max(abs(rhs), 1e-12) + 1e-14, (key, lhs, rhs)


def test_membrane_stiffness_gradient_matches_central_fd(oracle_mod):
    sc = _membrane_scene()
    rng = np.random.default_rng(37)
    N = sc.steps
    xs, _ = oracle_mod.forward(sc)
    target = xs[N] + 0.01 * rng.standard_normal((sc.V, 3))
    gr = oracle_mod.adjoint(sc, {N: xs[N] - target})

    def loss(K):
        x, _ = oracle_mod.forward(sc, memb_stiffness=K)
        d = x[N] - target
        return 0.5 * float(np.sum(d * d))

    g = gr["memb_stiffness"]
    for _ in range(8):
        t, c = rng.integers(sc.n_memb), rng.integers(4)
        h = 1e-5 * sc.memb_stiffness[t, c]
        Kp, Km = sc.memb_stiffness.astype(np.float64), sc.memb_stiffness.astype(np.float64)
        Kp[t, c] += h
        Km[t, c] -= h
        fd = (loss(Kp) - loss(Km)) / (2 * h)
        assert abs(fd - g[t, c]) <= 1e-5 * abs(g[t, c]) + 1e-6 * np.abs(g).max(), (t, c, fd, g[t, c])


def test_membrane_coloring(oracle_mod):
    sc = scenes.membrane_cloth(7)
    scenes.validate_coloring(sc)
    assert sc.n_memb == 2 * 6 * 6 and sc.n_colored == sc.m + sc.n_memb
    tiled = scenes.membrane_cloth(40, coloring="tiled", tile=8)
    scenes.validate_coloring(tiled)                      # vertex-disjoint colors, every id once
    assert tiled.n_colors == 4 * 16
    assert np.array_equal(np.sort(tiled.color_order), np.sort(scenes.membrane_cloth(40).color_order))
    K = sc.memb_stiffness.astype(np.float64)
    assert np.all(K[:, 0] * K[:, 1] - K[:, 2] ** 2 > 0) and np.all(K[:, 3] > 0)


def _one_triangle(K, w, vx, dt):
    """Unit right triangle in the x-z plane, (u, v) = (x, z), vertices 0 and 2 pinned,
    vertex 1 moving along the warp."""
    x = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    return scenes.Scene(rest_x=x, inv_mass=np.array([0.0, w, 0.0]), dist_idx=np.zeros((0, 2), np.int32),
                        bend_idx=np.zeros((0, 4), np.int32), tet_idx=np.zeros((0, 4), np.int32), tet_gamma=np.zeros(0),
                        color_offsets=np.array([0, 1], np.int32), color_order=np.array([0], np.int32), x0=x.copy(),
                        v0=np.array([[0.0, 0.0, 0.0], [vx, 0.0, 0.0], [0.0, 0.0, 0.0]]), compliance=np.zeros(0),
                        dt=dt, gravity=(0.0, 0.0, 0.0), steps=1, iters=1,
                        memb_idx=np.array([[0, 1, 2]], np.int32), memb_uv=x[:, [0, 2]][None],
                        memb_stiffness=np.array([K], np.float64))


def test_scene_level_membrane_update_closed_form(oracle_mod):
    """One step, one iteration of a scene with one triangle: the rest area (1/2), the
    map K -> alpha~ = (A K)^-1 / dt^2 with C01 != 0 and the warp/weft assignment all enter
    the closed form.  At the free vertex only E_uu and the shear row have gradients
    (s e_x and e_z); the shear row has no residual, so S reduces to the 2x2 of (E_uu, E_vv)
    rows [[w s^2 + a00, a01], [a01, a11]] against (-C_uu, 0): the E_vv multiplier is
    -a01 dlambda_uu / a11 (its sign follows alpha~'s off-diagonal)."""
    K = (800.0, 300.0, 200.0, 150.0)
    w, vx, dt = 2.0, 3.0, 0.05
    sc = _one_triangle(K, w, vx, dt)
    xs, _ = oracle_mod.forward(sc)
    lam = oracle_mod.forward_memb_multipliers(sc)[0, 0]
    Km = np.array([[K[0], K[2], 0.0], [K[2], K[1], 0.0], [0.0, 0.0, K[3]]])
    at = np.linalg.inv(0.5 * Km) / dt ** 2
    s = 1.0 + vx * dt
    C = 0.5 * (s * s - 1.0)
    S2 = np.array([[w * s * s + at[0, 0], at[0, 1]], [at[0, 1], at[1, 1]]])
    dl = np.linalg.solve(S2, [-C, 0.0])
    assert abs(xs[1, 1, 0] - (s + w * s * dl[0])) < 1e-13
    assert np.abs(xs[1, 1, 1:]).max() < 1e-15 and np.allclose(xs[1, [0, 2]], sc.x0[[0, 2]])
    assert np.allclose(lam, [dl[0], dl[1], 0.0], rtol=1e-12, atol=1e-15)
    assert abs(dl[1]) > 1e-6 * abs(dl[0])                 # the off-diagonal is exercised
