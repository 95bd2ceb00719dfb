"""Pins of the implicit-adjoint oracle (the paper's Eq. adjointXPBD with PD-projected
blocks): an independent augmented-system solve, the converged limit of the discrete
adjoint, and the properties of the projection."""
import numpy as np
import pytest

import oracle
from oracle import implicit
from paper_2301_01396_gb300 import scenes
from tests.helpers import rel, small_cloth, small_tets

KEYS = ("compliance", "x0", "v0", "f_global", "f_vertex", "f_vertex_steps")


def _seeds(sc, seed):
    rng = np.random.default_rng(seed)
    return {sc.steps: rng.standard_normal((sc.V, 3)), 1: rng.standard_normal((sc.V, 3))}


def test_schur_form_equals_augmented_system():
    """Eliminating the multipliers (Schur form) and solving the transposed augmented system
    [[M - sum lambda hess C, grad C^T], [-grad C, alpha~]] give the same gradients."""
    sc = small_cloth(4, bending=True, diagonals="both", pins=((0, 0),), steps=3, iters=4, v_scale=0.3, seed=3)
    seeds = _seeds(sc, 1)
    a = implicit.adjoint(sc, seeds, pd=False)
    b = implicit.adjoint(sc, seeds, pd=False, kkt=True)
    for k in KEYS:
        assert rel(a[k], b[k]) < 1e-10, k


@pytest.mark.parametrize("name", ["cloth", "tets"])
def test_exact_derivative_of_the_exactly_solved_step(name):
    """With every step solved exactly (Newton on the step's KKT system) and no projection,
    the implicit adjoint is the exact derivative of the trajectory: central finite
    differences of the loss agree."""
    if name == "cloth":
        sc = small_cloth(4, bending=True, diagonals="both", pins=((0, 0),), steps=3, iters=4, v_scale=0.3, seed=5)
    else:
        sc = small_tets(1, steps=3, iters=4, y0=0.05, plane=False, v_scale=0.05)
    traj = implicit.kkt_forward(sc)
    rng = np.random.default_rng(2)
    target = traj[0][-1] + 0.01 * rng.standard_normal((sc.V, 3))
    g = implicit.adjoint(sc, {sc.steps: traj[0][-1] - target}, pd=False, trajectory=traj)

    def loss(**kw):
        return 0.5 * np.sum((implicit.kkt_forward(sc, **kw)[0][-1] - target) ** 2)

    for j in rng.choice(sc.m, 4, replace=False):
        h = 1e-5 * sc.compliance[j]
        cp, cm = sc.compliance.copy(), sc.compliance.copy()
        cp[j] += h
        cm[j] -= h
        fd = (loss(compliance=cp) - loss(compliance=cm)) / (2 * h)
        assert abs(fd - g["compliance"][j]) <= 1e-5 * abs(g["compliance"][j]) + 1e-8 * np.abs(g["compliance"]).max()
    free = np.flatnonzero(sc.inv_mass > 0)
    for key, base in (("x0", sc.x0), ("v0", sc.v0)):
        for i in rng.choice(free, 2, replace=False):
            c = int(rng.integers(3))
            h = 1e-6
            bp, bm = np.array(base, np.float64), np.array(base, np.float64)
            bp[i, c] += h
            bm[i, c] -= h
            fd = (loss(**{key: bp}) - loss(**{key: bm})) / (2 * h)
            assert abs(fd - g[key][i, c]) <= 1e-5 * abs(g[key][i, c]) + 1e-8 * np.abs(g[key]).max(), (key, i, c)


def test_xpbd_fixed_point_is_not_the_exact_step():
    """XPBD iterated to convergence satisfies C + alpha~ lambda = 0 but not the primal
    equation M (x - p) = grad C^T lambda, so its end state differs from the exactly solved
    step (the implicit adjoint linearises there; its gradient is not the limit of the
    discrete adjoint)."""
    sc = small_cloth(4, bending=True, diagonals="both", pins=((0, 0),), steps=1, iters=2000, v_scale=0.3, seed=5)
    xs_x, _, _, _, _ = oracle.forward_multipliers(sc)
    xs_k = implicit.kkt_forward(sc)[0]
    d = np.abs(xs_x[1] - xs_k[1]).max()
    assert 1e-9 < d < 1e-2


def test_projection_gives_psd_blocks_and_keeps_psd_ones():
    rng = np.random.default_rng(4)
    for kind, q, r in [(0, rng.standard_normal(6), np.r_[1.5, np.zeros(11)]),
                       (1, rng.standard_normal(12), np.zeros(12)),
                       (3, rng.standard_normal(12), np.r_[0, 0, np.eye(3).reshape(-1), 1.0]),
                       (5, np.r_[rng.standard_normal(3), 0.1, 0.2, 0.3, 0.5], np.zeros(12))]:
        for lam in (-0.7, 0.9):
            g, B = implicit._block(kind, q, r, lam, 0.3, pd=True)
            assert np.allclose(B, B.T)
            assert np.linalg.eigvalsh(B).min() > -1e-10 * max(1.0, np.abs(B).max())
            nv = B.shape[0] // 3
            if nv > 1:   # translations stay in the null space
                t = np.tile(rng.standard_normal(3), nv)
                assert np.abs(B @ t).max() < 1e-9 * max(1.0, np.abs(B).max())
            _, B0 = implicit._block(kind, q, r, lam, 0.3, pd=False)
            if np.linalg.eigvalsh(B0).min() > 1e-12:
                assert np.allclose(B, B0, rtol=1e-9, atol=1e-12)


def test_force_gradients_follow_pbar():
    """f_global and f_vertex are the sums of the per-step per-vertex force gradient."""
    sc = small_cloth(4, bending=True, pins=((0, 0),), steps=3, iters=5, v_scale=0.3, seed=6)
    a = implicit.adjoint(sc, _seeds(sc, 3))
    assert rel(a["f_vertex_steps"].sum(0), a["f_vertex"]) < 1e-12
    assert rel(a["f_vertex_steps"].sum(1), a["f_global"]) < 1e-12
    assert np.all(a["f_vertex_steps"][:, 0] == 0.0)      # the pinned vertex


def _membrane_sheet(steps=3, iters=4):
    sc = scenes.membrane_cloth(4, steps=steps, iters=iters, seed=8, pins=((0, 0),), stiffness=(60.0, 30.0, 10.0, 20.0))
    rng = np.random.default_rng(9)
    v = 0.3 * rng.standard_normal(sc.x0.shape)
    v[sc.inv_mass == 0] = 0.0
    sc.v0 = scenes.f32(v)
    return sc


def test_membrane_schur_form_equals_augmented_system():
    """Membranes as 3-row blocks: the Schur form (B_t = G^T alpha~^-1 G - sum lambda_k
    hess C_k) and the augmented system with the 3x3 compliance blocks give the same
    gradients, the stiffness gradient included."""
    sc = _membrane_sheet()
    seeds = _seeds(sc, 5)
    a = implicit.adjoint(sc, seeds, pd=False)
    b = implicit.adjoint(sc, seeds, pd=False, kkt=True)
    for k in KEYS + ("memb_stiffness",):
        assert rel(a[k], b[k]) < 1e-10, k
    assert np.abs(a["memb_stiffness"]).max() > 0


def test_membrane_exact_derivative_of_the_exactly_solved_step():
    """The implicit adjoint with membranes is the exact derivative of the exactly solved
    trajectory: central differences in the stiffness, x0 and v0 agree."""
    sc = _membrane_sheet()
    traj = implicit.kkt_forward(sc)
    rng = np.random.default_rng(6)
    target = traj[0][-1] + 0.01 * rng.standard_normal((sc.V, 3))
    g = implicit.adjoint(sc, {sc.steps: traj[0][-1] - target}, pd=False, trajectory=traj)

    def loss(**kw):
        return 0.5 * np.sum((implicit.kkt_forward(sc, **kw)[0][-1] - target) ** 2)

    K = sc.memb_stiffness.astype(np.float64)
    gm = g["memb_stiffness"]
    for _ in range(6):
        t, c = int(rng.integers(sc.n_memb)), int(rng.integers(4))
        h = 1e-5 * K[t, c]
        kp, km = K.copy(), K.copy()
        kp[t, c] += h
        km[t, c] -= h
        fd = (loss(memb_stiffness=kp) - loss(memb_stiffness=km)) / (2 * h)
        assert abs(fd - gm[t, c]) <= 1e-5 * abs(gm[t, c]) + 1e-6 * np.abs(gm).max(), (t, c, fd, gm[t, c])
    free = np.flatnonzero(sc.inv_mass > 0)
    for key, base in (("x0", sc.x0), ("v0", sc.v0)):
        for i in rng.choice(free, 2, replace=False):
            c = int(rng.integers(3))
            h = 1e-6
            bp, bm = np.array(base, np.float64), np.array(base, np.float64)
            bp[i, c] += h
            bm[i, c] -= h
            fd = (loss(**{key: bp}) - loss(**{key: bm})) / (2 * h)
            assert abs(fd - g[key][i, c]) <= 1e-5 * abs(g[key][i, c]) + 1e-8 * np.abs(g[key]).max(), (key, i, c)


def test_membrane_projected_block_is_psd_with_translations_in_its_null_space():
    rng = np.random.default_rng(7)
    uv = rng.standard_normal((3, 2))
    B2 = np.linalg.inv(np.stack([uv[1] - uv[0], uv[2] - uv[0]], axis=1))
    at3 = implicit._memb_alpha((50.0, 20.0, 5.0, 10.0), 0.4, 0.05)
    for lam3 in (np.array([0.4, -0.3, 0.2]), np.array([-2.0, -1.0, 0.5])):
        q = rng.standard_normal(9)
        G, B = implicit._memb_block(q, B2, lam3, at3, pd=True)
        assert np.allclose(B, B.T)
        assert np.linalg.eigvalsh(B).min() > -1e-10 * max(1.0, np.abs(B).max())
        t = np.tile(rng.standard_normal(3), 3)
        assert np.abs(B @ t).max() < 1e-9 * max(1.0, np.abs(B).max())


def test_membrane_alpha_is_the_inverse_scaled_stiffness():
    """The implicit oracle's membrane compliance: alpha~ (A K dt^2) = I for the printed
    inverse-compliance matrix A [C00 C01; C01 C11; C22], and its stiffness gradient is the
    chain rule through it (central differences of <G, alpha~(K)>)."""
    K, A, dt = np.array([50.0, 20.0, 5.0, 10.0]), 0.4, 0.05
    Km = np.array([[K[0], K[2], 0.0], [K[2], K[1], 0.0], [0.0, 0.0, K[3]]])
    at = implicit._memb_alpha(K, A, dt)
    assert np.allclose(at @ (A * Km * dt * dt), np.eye(3), atol=1e-12)
    sc = scenes.membrane_cloth(2)
    sc.memb_stiffness = np.array([K, K * 1.5])
    Gbar = np.random.default_rng(3).standard_normal((2, 3, 3))
    g = implicit._memb_alpha_grad(sc, Gbar, None, dt)
    areas = [a for _, a in implicit._memb_rest(sc)]
    for t in range(2):
        for p in range(4):
            h = 1e-6 * sc.memb_stiffness[t, p]
            kp, km = sc.memb_stiffness[t].copy(), sc.memb_stiffness[t].copy()
            kp[p] += h
            km[p] -= h
            fd = (np.sum(Gbar[t] * implicit._memb_alpha(kp, areas[t], dt))
                  - np.sum(Gbar[t] * implicit._memb_alpha(km, areas[t], dt))) / (2 * h)
            assert abs(fd - g[t, p]) <= 1e-6 * abs(g[t, p]) + 1e-12
