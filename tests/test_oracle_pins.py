"""Pins of the FP64 oracle to facts fixed by the paper and by mathematics (no GPU).

Each test checks the oracle against something other than itself: a closed form, an
invariant the paper states, brute-force finite differences, or the forward-mode tangent
(dual numbers through the forward program, which shares no derivative code with the
hand-derived reverse sweep)."""
import numpy as np
import pytest

from paper_2301_01396_gb300 import scenes
from tests.helpers import rel, single_spring, small_cloth, small_sphere_cloth, small_tets


# --------------------------------------------------------------------------- closed forms

def _spring_recurrence(L, e0, w, alpha, dt, steps, g=9.81):
    """Closed-form single-spring recurrence (Sec. 3.1, Eq. xpbd with one constraint): one
    pinned end, one free mass below it, stretch e = l - L and rate u = dl/dt.  The first
    iteration gives dlambda = -C/(w + alpha~) so C' = C alpha~/(w + alpha~); every later
    iteration gives dlambda = 0.  Returns e_n and de_n/dalpha."""
    at = alpha / dt ** 2
    r = at / (w + at)
    dr = (1.0 / dt ** 2) * w / (w + at) ** 2
    e, u, de, du = e0, 0.0, 0.0, 0.0
    es, des = [e], [de]
    for _ in range(steps):
        ep = e + dt * u + dt * dt * g
        dep = de + dt * du
        e1 = r * ep
        de1 = dr * ep + r * dep
        u, du = (e1 - e) / dt, (de1 - de) / dt
        e, de = e1, de1
        es.append(e)
        des.append(de)
    return np.array(es), np.array(des)


@pytest.mark.parametrize("iters", [1, 4])
def test_single_spring_closed_form(oracle_mod, iters):
    sc = single_spring(L=0.5, stretch0=0.01, mass=0.01, alpha=1e-3)
    steps = 40
    xs, vs = oracle_mod.forward(sc, steps, iters)
    L = 0.5
    e0 = -sc.x0[1, 1] - L                                  # inputs are FP32-rounded
    e_ref, de_ref = _spring_recurrence(L, e0, sc.inv_mass[1], float(sc.compliance[0]), sc.dt, steps)
    e = -xs[:, 1, 1] - L
    assert np.max(np.abs(e - e_ref)) < 1e-12
    assert np.all(xs[:, 0, :] == 0.0)                    # pinned vertex never moves
    assert np.max(np.abs(xs[:, 1, [0, 2]])) == 0.0       # motion stays on the axis
    # d e_N / d alpha: reverse sweep and tangent against the differentiated recurrence
    seed = np.zeros((2, 3))
    seed[1, 1] = -1.0                                      # L = l_N = -y_N  ->  dL/dy_N = -1
    gr = oracle_mod.adjoint(sc, {steps: seed}, steps, iters)
    assert abs(gr["compliance"][0] - de_ref[-1]) < 1e-9 * max(1.0, abs(de_ref[-1]))
    dxs, _ = oracle_mod.tangent(sc, {"compliance": np.ones(1)}, steps, iters)
    assert np.max(np.abs(-dxs[:, 1, 1] - de_ref)) < 1e-9 * max(1.0, np.abs(de_ref).max())


def test_single_spring_hooke_equilibrium(oracle_mod):
    """Static equilibrium l - L = m g alpha (Hooke's law with stiffness 1/alpha)."""
    m, alpha = 0.01, 0.05
    sc = single_spring(L=0.5, mass=m, alpha=alpha)
    xs, _ = oracle_mod.forward(sc, 3000, 1)
    e = -xs[-1, 1, 1] - 0.5
    assert abs(e - 9.81 * float(sc.compliance[0]) / sc.inv_mass[1]) < 1e-10


# --------------------------------------------------------------------------- constraints

def _rot(rng):
    q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1
    return q


def test_dihedral_angle_closed_form(oracle_mod):
    """theta for a hinge whose two wings are each lifted by beta out of the flat
    configuration is -2 beta (sign convention of the signed atan2 angle), invariant under
    rigid motions, and C = theta - theta0 wraps into (-pi, pi]."""
    rng = np.random.default_rng(0)
    for beta in np.linspace(-1.4, 1.4, 15):
        x0, x1 = np.zeros(3), np.array([1.0, 0, 0])
        x2 = np.array([0.3, np.cos(beta), np.sin(beta)])
        x3 = np.array([0.6, -np.cos(beta), np.sin(beta)])
        q = np.stack([x0, x1, x2, x3])
        R, t = _rot(rng), rng.standard_normal(3)
        for qq in (q, q @ R.T + t):
            C, g, _ = oracle_mod.constraint("bend", qq)
            assert abs(C - (-2 * beta)) < 1e-12
    # wrap: theta0 close to +pi, theta close to -pi -> C small
    q = np.stack([np.zeros(3), [1.0, 0, 0], [0.3, np.cos(1.5), np.sin(1.5)], [0.6, -np.cos(1.5), np.sin(1.5)]])
    r = np.zeros(12)
    r[1] = 3.0
    C, _, _ = oracle_mod.constraint("bend", q, r)
    assert abs(C - (-3.0 - 3.0 + 2 * np.pi)) < 1e-12


def test_tet_constraints_closed_form(oracle_mod):
    rng = np.random.default_rng(1)
    Xr = rng.standard_normal((4, 3))
    Dm = (Xr[1:] - Xr[0]).T
    B = np.linalg.inv(Dm)
    for s in (0.7, 1.0, 1.3):
        R, t = _rot(rng), rng.standard_normal(3)
        X = (s * Xr) @ R.T + t                # F = s R
        r = np.zeros(12)
        r[2:11] = B.reshape(-1)
        r[11] = 1.0
        CH, _, _ = oracle_mod.constraint("tet_h", X, r)
        CD, _, _ = oracle_mod.constraint("tet_d", X, r)
        assert abs(CH - (s ** 3 - 1.0)) < 1e-11
        assert abs(CD - np.sqrt(3.0) * s) < 1e-11


def test_rest_data_and_tet_volumes(oracle_mod):
    """Rest lengths equal the grid spacing (or its diagonal), flat hinges have theta0 = 0,
    and the 5-tet split tiles each cube: corner tets h^3/6, central tet h^3/3."""
    sc = small_cloth(5)
    rd = oracle_mod.rest_data(sc)
    h = 1.0 / 4
    L = rd[:sc.n_dist, 0]
    assert np.all((np.abs(L - h) < 1e-7) | (np.abs(L - h * np.sqrt(2)) < 1e-7))
    assert np.max(np.abs(rd[sc.n_dist:sc.n_dist + sc.n_bend, 1])) < 1e-12
    tb = scenes.tet_block(3, size=0.3, steps=1)
    rd = oracle_mod.rest_data(tb)
    vol = rd[:tb.n_tet, 11].reshape(-1, 5)
    hh = 0.1
    assert np.allclose(np.sort(vol, axis=1), np.array([1, 1, 1, 1, 2]) * hh ** 3 / 6, rtol=1e-6)
    assert abs(vol.sum() - 0.3 ** 3) < 1e-6 * 0.3 ** 3


@pytest.mark.parametrize("kind", ["dist", "bend", "tet_h", "tet_d", "plane", "sphere"])
def test_constraint_derivatives_fd(oracle_mod, kind):
    """AD gradient vs central differences of C; AD Hessian-vector product vs central
    differences of the gradient; Hessian symmetry; translation invariance (element
    forces sum to zero, Sec. 4.4.1)."""
    rng = np.random.default_rng(2)
    n = oracle_mod.N_INPUTS[oracle_mod.KIND[kind]]
    nv = {"dist": 2, "bend": 4, "tet_h": 4, "tet_d": 4, "plane": 1, "sphere": 1}[kind]
    r = np.zeros(12)
    if kind == "dist":
        r[0] = 0.3
    if kind.startswith("tet"):
        r[2:11] = np.linalg.inv(rng.standard_normal((3, 3)) + 2 * np.eye(3)).reshape(-1)
        r[11] = 1.1
    if kind in ("plane", "sphere"):
        r[11] = 0.01
    q = rng.standard_normal(n)
    if kind == "sphere":
        q[6] = 0.4
    h = 1e-6
    C0, g, _ = oracle_mod.constraint(kind, q, r)
    g_fd = np.array([(oracle_mod.constraint(kind, q + h * e, r)[0] - oracle_mod.constraint(kind, q - h * e, r)[0]) / (2 * h)
                     for e in np.eye(n)])
    assert rel(g, g_fd) < 1e-8
    H = np.stack([oracle_mod.constraint(kind, q, r, u=e)[2] for e in np.eye(n)], axis=1)
    assert np.max(np.abs(H - H.T)) < 1e-9 * max(1.0, np.abs(H).max())
    H_fd = np.stack([(oracle_mod.constraint(kind, q + h * e, r)[1] - oracle_mod.constraint(kind, q - h * e, r)[1]) / (2 * h)
                     for e in np.eye(n)], axis=1)
    assert np.max(np.abs(H - H_fd)) < 1e-6 * max(1.0, np.abs(H).max())
    if kind in ("dist", "bend", "tet_h", "tet_d"):
        gv = g[:3 * nv].reshape(nv, 3)
        assert np.max(np.abs(gv.sum(0))) < 1e-12 * max(1.0, np.abs(gv).max())
        Hv = H[:3 * nv, :3 * nv].reshape(nv, 3, nv, 3)
        assert np.max(np.abs(Hv.sum(0))) < 1e-9 * max(1.0, np.abs(H).max())


@pytest.mark.parametrize("kind", ["dist", "bend", "tet_h", "tet_d", "plane", "sphere"])
def test_projection_vjp_matches_fd_jacobian(oracle_mod, kind):
    """The reverse of one XPBD update equals the transpose of the finite-difference
    Jacobian of that update with respect to (inputs, lambda, alpha~)."""
    rng = np.random.default_rng(3)
    n = oracle_mod.N_INPUTS[oracle_mod.KIND[kind]]
    nv = {"dist": 2, "bend": 4, "tet_h": 4, "tet_d": 4, "plane": 1, "sphere": 1}[kind]
    r = np.zeros(12)
    if kind == "dist":
        r[0] = 0.8
    if kind.startswith("tet"):
        r[2:11] = np.linalg.inv(rng.standard_normal((3, 3)) + 2 * np.eye(3)).reshape(-1)
        r[11] = 1.05
    if kind == "bend":
        r[1] = 0.2
    q = rng.standard_normal(n)
    if kind == "sphere":
        q[6] = 2.5
    if kind == "plane":
        q[3] = q[1] + 0.3
    w = rng.uniform(0.5, 2.0, nv)
    w[0] = 0.0 if kind in ("dist", "bend") else w[0]       # one pinned vertex
    lam, at = 0.37, 0.21

    def F(z):
        qq, ll, aa = z[:n], z[n], z[n + 1]
        q2, l2 = oracle_mod.project_one(kind, qq, w, r, ll, aa)
        return np.r_[q2, l2]

    z0 = np.r_[q, lam, at]
    h = 1e-6
    J = np.stack([(F(z0 + h * e) - F(z0 - h * e)) / (2 * h) for e in np.eye(n + 2)], axis=1)
    qbar = rng.standard_normal(n)
    lbar = rng.standard_normal()
    qb, lb, ab = oracle_mod.vjp_one(kind, q, w, r, lam, at, qbar, lbar)
    ref = J.T @ np.r_[qbar, lbar]
    got = np.r_[qb, lb, ab]
    assert rel(got, ref) < 1e-7


def test_distance_update_jacobian_symmetry(oracle_mod):
    """Sec. 4.4.1: M d(dx)/dx is symmetric and its rows and columns sum to zero (checked
    for a distance constraint between two free vertices)."""
    rng = np.random.default_rng(4)
    q = rng.standard_normal(6)
    w = np.array([2.0, 0.5])
    r = np.zeros(12)
    r[0] = 0.6

    def F(qq):
        return oracle_mod.project_one("dist", qq, w, r, 0.1, 0.3)[0]

    h = 1e-6
    J = np.stack([(F(q + h * e) - F(q - h * e)) / (2 * h) for e in np.eye(6)], axis=1)
    Mm = np.diag(np.repeat(1.0 / w, 3))
    A = Mm @ (J - np.eye(6))
    assert np.max(np.abs(A - A.T)) < 1e-7
    Ab = A.reshape(2, 3, 2, 3)
    assert np.max(np.abs(Ab.sum(0))) < 1e-7 and np.max(np.abs(Ab.sum(2))) < 1e-7


# --------------------------------------------------------------------------- invariants

def test_rest_state_is_fixed_without_gravity(oracle_mod):
    sc = small_cloth(6, bending=True, gravity=(0.0, 0.0, 0.0), steps=10, iters=5)
    xs, vs = oracle_mod.forward(sc)
    assert np.max(np.abs(xs - sc.rest_x[None])) < 1e-15
    assert np.max(np.abs(vs)) < 1e-13


def test_pinned_vertices_never_move(oracle_mod):
    sc = small_cloth(6, bending=True, steps=15, iters=4, jitter=0.01, plane_h=-0.05)
    xs, _ = oracle_mod.forward(sc)
    pinned = sc.inv_mass == 0
    assert np.all(xs[:, pinned, :] == sc.x0[None, pinned, :])
    assert np.max(np.abs(xs[-1, ~pinned] - sc.x0[~pinned])) > 1e-3   # the rest did move


@pytest.mark.parametrize("which", ["cloth", "tets"])
def test_linear_momentum_conserved(oracle_mod, which):
    """No pins, gravity or collisions: every projection moves mass-weighted positions by
    sum_i grad_i C dlambda = 0 (translation invariance), so sum m v is constant."""
    if which == "cloth":
        sc = small_cloth(5, bending=True, pins=(), gravity=(0.0, 0.0, 0.0), jitter=0.02,
                         v_scale=0.5, steps=8, iters=3)
    else:
        sc = small_tets(2, plane=False, gravity=(0.0, 0.0, 0.0), jitter=0.005, v_scale=0.3,
                        steps=6, iters=3)
    xs, vs = oracle_mod.forward(sc)
    m = 1.0 / sc.inv_mass
    P = np.einsum("i,nij->nj", m, vs)
    assert np.max(np.abs(P - P[0])) < 1e-12 * max(1.0, np.abs(P[0]).max() + np.abs(m[:, None] * vs[0]).sum())


# --------------------------------------------------------------------------- full adjoint

def _loss_and_seed(xs, target, step):
    d = xs[step] - target
    return 0.5 * float(np.sum(d * d)), d


def _scenes_for_adjoint():
    return {
        "cloth_plane": small_cloth(5, bending=True, steps=6, iters=3, plane_h=-0.02, jitter=0.002,
                                   v_scale=0.2, seed=7),
        "tets_plane": small_tets(2, steps=6, iters=3, y0=0.004, v_scale=0.05),
        "tets_coupled": scenes.couple_tets(small_tets(2, steps=6, iters=3, y0=0.004, v_scale=0.05)),
        "cloth_sphere": small_sphere_cloth(6, steps=5, iters=3),
        "cloth_both": _both_colliders(),
    }


def _both_colliders():
    """Plane just above the sphere's top: vertices falling onto the top penetrate both
    colliders in the same step (plane first, then sphere, within the collision pass)."""
    sc = small_sphere_cloth(6, steps=5, iters=3)
    sc.collider_flags = scenes.COLLIDE_PLANE | scenes.COLLIDE_SPHERE
    sc.plane_h = float(np.float32(sc.sphere[1] + sc.sphere[3] + 0.003))
    sc.v0 = scenes.f32(sc.v0 + np.array([0.0, -1.4, 0.0]))     # reach inside the sphere in one step
    return sc


@pytest.mark.parametrize("name", ["cloth_plane", "tets_plane", "tets_coupled", "cloth_sphere", "cloth_both"])
def test_adjoint_equals_tangent(oracle_mod, name):
    """<dL/du, du> from the reverse sweep equals <dL/dx_N, dx_N/du du> from the
    forward-mode tangent, for every parameter group."""
    sc = _scenes_for_adjoint()[name]
    rng = np.random.default_rng(11)
    xs, _ = oracle_mod.forward(sc)
    N = sc.steps
    seed_T = rng.standard_normal((sc.V, 3))
    seed_mid = rng.standard_normal((sc.V, 3))
    mid = N // 2
    gr = oracle_mod.adjoint(sc, {N: seed_T, mid: seed_mid})
    dirs = {
        "compliance": sc.compliance * rng.standard_normal(sc.m),
        "x0": rng.standard_normal((sc.V, 3)) * 1e-3,
        "v0": rng.standard_normal((sc.V, 3)),
        "f_global": rng.standard_normal((N, 3)),
        "f_vertex": rng.standard_normal((sc.V, 3)),
        "collider": rng.standard_normal(5),
        "f_vertex_steps": rng.standard_normal((N, sc.V, 3)),
    }
    for key, d in dirs.items():
        dxs, _ = oracle_mod.tangent(sc, {key: d})
        lhs = float(np.sum(gr[key] * d))
        rhs = float(np.sum(dxs[N] * seed_T) + np.sum(dxs[mid] * seed_mid))
        assert abs(lhs - rhs) <= 1e-9 * max(abs(rhs), 1e-12) + 1e-14, (key, lhs, rhs)


@pytest.mark.parametrize("name", ["cloth_plane", "tets_plane", "tets_coupled", "cloth_sphere", "cloth_both"])
def test_adjoint_matches_central_fd(oracle_mod, name):
    """Central finite differences of the FP64 forward simulation, on seeded parameter
    subsets; parameters whose perturbation changes the contact set are skipped."""
    sc = _scenes_for_adjoint()[name]
    rng = np.random.default_rng(12)
    N = sc.steps
    xs, _ = oracle_mod.forward(sc)
    target = xs[N] + 0.01 * rng.standard_normal((sc.V, 3))
    _, seed = _loss_and_seed(xs, target, N)
    gr = oracle_mod.adjoint(sc, {N: seed})

    def loss(**kw):
        x, _ = oracle_mod.forward(sc, **kw)
        return _loss_and_seed(x, target, N)[0]

    checks = 0
    for j in rng.choice(sc.m, 6, replace=False):
        h = 1e-4 * sc.compliance[j]
        cp, cm = sc.compliance.copy(), sc.compliance.copy()
        cp[j] += h
        cm[j] -= h
        fd = (loss(compliance=cp) - loss(compliance=cm)) / (2 * h)
        assert abs(fd - gr["compliance"][j]) <= 1e-5 * abs(gr["compliance"][j]) + 1e-9 * np.abs(gr["compliance"]).max()
        checks += 1
    for key, base in (("x0", sc.x0), ("v0", sc.v0)):
        for _ in range(4):
            i, c = rng.integers(sc.V), rng.integers(3)
            h = 1e-6
            bp, bm = base.copy(), base.copy()
            bp[i, c] += h
            bm[i, c] -= h
            fd = (loss(**{key: bp}) - loss(**{key: bm})) / (2 * h)
            assert abs(fd - gr[key][i, c]) <= 1e-5 * abs(gr[key][i, c]) + 1e-7 * np.abs(gr[key]).max()
            checks += 1
    if sc.collider_flags & scenes.COLLIDE_PLANE:
        h = 1e-7
        fd = (loss(plane_h=sc.plane_h + h) - loss(plane_h=sc.plane_h - h)) / (2 * h)
        assert abs(fd - gr["collider"][0]) <= 1e-5 * abs(gr["collider"][0]) + 1e-10
    if sc.collider_flags & scenes.COLLIDE_SPHERE:
        for c in range(4):
            h = 1e-7
            sp, sm = list(sc.sphere), list(sc.sphere)
            sp[c] += h
            sm[c] -= h
            fd = (loss(sphere=sp) - loss(sphere=sm)) / (2 * h)
            assert abs(fd - gr["collider"][1 + c]) <= 1e-5 * abs(gr["collider"][1 + c]) + 1e-10
        fg = sc.f_global
        for _ in range(3):
            n, c = rng.integers(N), rng.integers(3)
            h = 1e-3 * np.abs(fg).max()
            fp, fm = fg.copy(), fg.copy()
            fp[n, c] += h
            fm[n, c] -= h
            fd = (loss(f_global=fp) - loss(f_global=fm)) / (2 * h)
            assert abs(fd - gr["f_global"][n, c]) <= 1e-5 * abs(gr["f_global"][n, c]) + 1e-9 * np.abs(gr["f_global"]).max()
    assert checks > 0


def test_force_gradient_identity(oracle_mod):
    """Sec. 5.6: force gradients come straight from the adjoint: the per-vertex force
    gradient summed over vertices equals the per-step global force gradient summed over
    steps (both are dt^2 w pbar accumulated)."""
    sc = small_sphere_cloth(6, steps=4, iters=2)
    rng = np.random.default_rng(5)
    gr = oracle_mod.adjoint(sc, {sc.steps: rng.standard_normal((sc.V, 3))})
    assert rel(gr["f_vertex"].sum(0), gr["f_global"].sum(0)) < 1e-12


def test_per_step_vertex_force_gradient_identities(oracle_mod):
    """The keyframe example's control variables, one force per vertex per step (Sec.
    "Keyframe Simulation"): their gradient dt^2 w pbar_n, summed over steps, is the
    time-constant per-vertex force gradient, and summed over vertices, each step's global
    force gradient; pinned vertices (w = 0) get none."""
    sc = small_sphere_cloth(6, steps=4, iters=2)
    sc.inv_mass = sc.inv_mass.copy()
    sc.inv_mass[0] = 0.0
    sc.v0 = sc.v0.copy()
    sc.v0[0] = 0.0
    rng = np.random.default_rng(6)
    gr = oracle_mod.adjoint(sc, {sc.steps: rng.standard_normal((sc.V, 3)), 2: rng.standard_normal((sc.V, 3))})
    fvs = gr["f_vertex_steps"]
    assert fvs.shape == (sc.steps, sc.V, 3)
    assert rel(fvs.sum(0), gr["f_vertex"]) < 1e-12
    assert rel(fvs.sum(1), gr["f_global"]) < 1e-12
    assert np.all(fvs[:, 0] == 0.0)


def test_per_step_vertex_force_matches_central_fd(oracle_mod):
    """The forward applies F_{n,i} at step n and the reverse sweep's gradient for it agrees
    with central finite differences of the loss."""
    sc = small_cloth(5, bending=True, steps=5, iters=3, plane_h=-0.02, v_scale=0.2, seed=21)
    rng = np.random.default_rng(22)
    sc.f_vertex_steps = 0.05 * rng.standard_normal((sc.steps, sc.V, 3))
    xs, _ = oracle_mod.forward(sc)
    x_free, _ = oracle_mod.forward(sc, f_vertex_steps=np.zeros_like(sc.f_vertex_steps))
    assert np.abs(xs[-1] - x_free[-1]).max() > 1e-6          # the forces move the cloth
    target = xs[-1] + 0.01 * rng.standard_normal((sc.V, 3))
    gr = oracle_mod.adjoint(sc, {sc.steps: xs[-1] - target})
    for n, i, c in [(0, 7, 1), (2, 12, 0), (4, 18, 2)]:
        h = 1e-4
        fp, fm = sc.f_vertex_steps.copy(), sc.f_vertex_steps.copy()
        fp[n, i, c] += h
        fm[n, i, c] -= h
        lp = 0.5 * np.sum((oracle_mod.forward(sc, f_vertex_steps=fp)[0][-1] - target) ** 2)
        lm = 0.5 * np.sum((oracle_mod.forward(sc, f_vertex_steps=fm)[0][-1] - target) ** 2)
        fd = (lp - lm) / (2 * h)
        g = gr["f_vertex_steps"][n, i, c]
        assert abs(fd - g) <= 1e-6 * abs(g) + 1e-10, (n, i, c, fd, g)


def test_total_gradient_is_sum_of_constraint_contributions(oracle_mod):
    """With alpha_j = s alpha_j0, dL/ds at s = 1 equals sum_j alpha_j0 dL/dalpha_j."""
    sc = small_cloth(5, bending=True, steps=5, iters=3, plane_h=-0.02, v_scale=0.2, seed=9)
    rng = np.random.default_rng(13)
    xs, _ = oracle_mod.forward(sc)
    target = xs[-1] + 0.01 * rng.standard_normal((sc.V, 3))
    gr = oracle_mod.adjoint(sc, {sc.steps: xs[-1] - target})

    def loss(s):
        x, _ = oracle_mod.forward(sc, compliance=sc.compliance * s)
        return 0.5 * np.sum((x[-1] - target) ** 2)

    h = 1e-5
    fd = (loss(1 + h) - loss(1 - h)) / (2 * h)
    assert abs(fd - np.sum(sc.compliance * gr["compliance"])) < 1e-6 * abs(fd)


def test_initial_velocity_gradient_is_adjoint_state(oracle_mod):
    """Sec. 5.5: dL/dv0 is read from the adjoint state: for a single spring with the loss
    on x_1, dL/dv0 = dt * pbar and dL/dx0 = pbar + dL/dx_1 (d v_1 / d x_0 path vanishes
    with no velocity seed)."""
    sc = single_spring(alpha=1e-3)
    seed = np.zeros((2, 3))
    seed[1] = [0.3, -0.7, 0.2]
    gr = oracle_mod.adjoint(sc, {1: seed}, 1, 1)
    assert rel(gr["v0"], sc.dt * gr["x0"]) < 1e-13


def test_fp32_rounding_emulation_is_off_by_default(oracle_mod):
    """The FP32-rounding emulation (used to measure attainable float32 agreement) changes
    nothing unless switched on, and when on every state value is float-representable."""
    sc = small_cloth(6, steps=3, iters=2, plane_h=-0.02, v_scale=0.2)
    a, _ = oracle_mod.forward(sc)
    with oracle_mod.fp32_rounding():
        b, vb = oracle_mod.forward(sc)
    c, _ = oracle_mod.forward(sc)
    assert np.array_equal(a, c)
    assert np.array_equal(b, b.astype(np.float32).astype(np.float64))
    assert np.array_equal(vb, vb.astype(np.float32).astype(np.float64))
    assert 0 < np.abs(a - b).max() < 1e-5


def test_material_gradient_matches_central_fd(oracle_mod):
    """Tet materials (mu = a^2, lambda = b^2): the chain rule from the compliance gradient to
    (a, b) agrees with central finite differences of the loss over the material parameters."""
    from oracle import materials
    sc = small_tets(2, steps=4, iters=4, y0=0.004, v_scale=0.05, plane=False)   # smooth: no contact set
    mat, a, b = scenes.tet_materials(sc.n_tet, 3, seed=4)
    a, b = a.astype(np.float64), b.astype(np.float64)
    rng = np.random.default_rng(14)
    comp = materials.compliance(sc, mat, a, b)
    xs, _ = oracle_mod.forward(sc, compliance=comp)
    target = xs[-1] + 0.005 * rng.standard_normal((sc.V, 3))
    gr = oracle_mod.adjoint(sc, {sc.steps: xs[-1] - target}, compliance=comp)
    da, db = materials.gradient(sc, gr["compliance"], mat, a, b)

    def loss(a_, b_):
        x, _ = oracle_mod.forward(sc, compliance=materials.compliance(sc, mat, a_, b_))
        return 0.5 * np.sum((x[-1] - target) ** 2)

    for k in range(3):
        for arr, g in ((a, da), (b, db)):
            h = 1e-7 * arr[k]   # the loss is strongly curved in a, b (compliance ~ 1/a^2)
            ap, am = arr.copy(), arr.copy()
            ap[k] += h
            am[k] -= h
            fd = (loss(ap, b) - loss(am, b)) / (2 * h) if arr is a else (loss(a, ap) - loss(a, am)) / (2 * h)
            assert abs(fd - g[k]) <= 1e-5 * abs(g[k]) + 1e-9 * np.abs(g).max(), (k, fd, g[k])
