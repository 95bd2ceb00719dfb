"""Pins of the oracle's contact projection to closed forms (Sec. 4.6: collisions as stiff
compliant springs with a user-set thickness; reading R12: contacts detected once per step
at the predicted positions, an active contact is an equality spring for all iterations of
that step).

Each contact is a one-vertex constraint with C = y - h - t (plane) or C = |x - c| - r - t
(sphere), gradient the surface normal, so one XPBD update from lambda = 0 moves the vertex
along the normal by w C / (w + alpha~) and leaves C' = C alpha~ / (w + alpha~); every later
iteration gives dlambda = 0 because C' + alpha~ lambda' = 0.  A vertex resting on a collider
settles where that spring balances gravity: a depth m g alpha below the surface (Hooke's
law with stiffness 1/alpha).  These values, their derivatives in the collider parameters,
and the detect-once rule are checked here against the oracle's forward, reverse sweep and
tangent."""
import numpy as np
import pytest

from paper_2301_01396_gb300 import scenes
from paper_2301_01396_gb300.scenes import Scene, f32

DT = 1.0 / 60.0
G = 9.81


def _points(x0, v0, mass, *, flags, alpha_c, thickness, plane_h=0.0, sphere=(0.0, 0.0, 0.0, 0.0),
            gravity=(0.0, -G, 0.0), dist=None, dist_alpha=0.0, rest=None):
    """Free vertices (optionally one spring between vertices 0 and 1) and colliders."""
    x0 = f32(x0)
    V = x0.shape[0]
    inv = np.where(np.asarray(mass, np.float64) > 0, 1.0 / np.maximum(np.asarray(mass, np.float64), 1e-300), 0.0)
    nd = 0 if dist is None else 1
    return Scene(rest_x=f32(x0 if rest is None else rest), inv_mass=f32(np.broadcast_to(inv, (V,))),
                 dist_idx=np.array([dist] if nd else [], np.int32).reshape(nd, 2), bend_idx=np.zeros((0, 4), np.int32),
                 tet_idx=np.zeros((0, 4), np.int32), tet_gamma=np.zeros(0),
                 color_offsets=np.array([0, nd], np.int32) if nd else np.zeros(1, np.int32),
                 color_order=np.arange(nd, dtype=np.int32), x0=x0, v0=f32(v0),
                 compliance=f32([dist_alpha] * nd), dt=DT, gravity=gravity, collider_flags=flags,
                 plane_h=plane_h, sphere=tuple(float(v) for v in f32(sphere)), contact_compliance=alpha_c,
                 thickness=thickness, name="points")


def _predicted(sc):
    x0 = sc.x0.astype(np.float64)
    v0 = sc.v0.astype(np.float64)
    w = sc.inv_mass.astype(np.float64)[:, None]
    return x0 + sc.dt * v0 + sc.dt ** 2 * (w > 0) * np.asarray(sc.gravity)


# ------------------------------------------------------------------------- plane

@pytest.mark.parametrize("iters", [1, 3])
def test_plane_one_update_closed_form(oracle_mod, iters):
    """Vertices predicted below y = h + t move up along the normal to
    y' - h - t = (y_p - h - t) alpha~/(w + alpha~); x and z are untouched; vertices
    predicted above are untouched.  Later iterations change nothing.  The derivatives
    dy'/dh = 1 - r, dy'/dy_p = r (r = alpha~/(w + alpha~)) are those of the reverse sweep."""
    m, h, t = 0.01, -0.02, 0.003
    w = float(f32(1.0 / m))
    alpha = w / 3.0 * DT ** 2                        # r = 1/4
    y0 = np.array([-0.01, -0.015, -0.016, -0.02, -0.03, 0.01])
    rng = np.random.default_rng(1)
    x0 = np.stack([rng.uniform(0, 1, 6), y0, rng.uniform(0, 1, 6)], 1)
    v0 = np.stack([rng.normal(0, 0.2, 6), np.full(6, -0.3), rng.normal(0, 0.2, 6)], 1)
    sc = _points(x0, v0, m, flags=scenes.COLLIDE_PLANE, alpha_c=alpha, thickness=t, plane_h=h)
    p = _predicted(sc)
    C = p[:, 1] - h - t
    active = C < 0
    assert active.sum() == 5 and np.abs(C).min() > 5e-4
    at = alpha / DT ** 2
    r = at / (w + at)
    expect = p.copy()
    expect[active, 1] = h + t + C[active] * r
    xs, vs = oracle_mod.forward(sc, 1, iters)
    assert np.abs(xs[1] - expect).max() < 1e-14
    assert np.abs(vs[1] - (expect - sc.x0) / DT).max() < 1e-11
    assert np.all(xs[1][active, 1] > p[active, 1])                  # pushed out, not in
    # reverse sweep: L = sum of all final coordinates
    gr = oracle_mod.adjoint(sc, {1: np.ones((6, 3))}, 1, iters)
    assert abs(gr["collider"][0] - active.sum() * (1.0 - r)) < 1e-12
    assert np.all(gr["collider"][1:] == 0.0)
    dy = np.where(active, r, 1.0)
    assert np.abs(gr["x0"][:, 1] - dy).max() < 1e-12 and np.abs(gr["x0"][:, [0, 2]] - 1.0).max() < 1e-12
    assert np.abs(gr["v0"][:, 1] - DT * dy).max() < 1e-14
    # tangent in h agrees
    dxs, _ = oracle_mod.tangent(sc, {"collider": np.array([1.0, 0, 0, 0, 0])}, 1, iters)
    assert np.abs(dxs[1][:, 1] - np.where(active, 1.0 - r, 0.0)).max() < 1e-12


@pytest.mark.parametrize("iters", [1, 4])
def test_plane_resting_depth_is_hooke(oracle_mod, iters):
    """A vertex released on the plane settles m g alpha below h + t, and the settled height
    follows h one to one (dy/dh = 1) and forgets its start (dy/dy0 = 0)."""
    m, h, t = 0.01, 0.1, 0.002
    w = float(f32(1.0 / m))
    alpha = w * DT ** 2                              # r = 1/2: converges as 0.71^n
    sc = _points([[0.3, h + t, 0.4]], [[0.0, 0.0, 0.0]], m, flags=scenes.COLLIDE_PLANE, alpha_c=alpha,
                 thickness=t, plane_h=h)
    N = 300
    xs, vs = oracle_mod.forward(sc, N, iters)
    mass = 1.0 / float(sc.inv_mass[0])
    depth = mass * G * alpha
    assert abs(xs[N, 0, 1] - (sc.x0[0, 1] * 0 + h + t - depth)) < 1e-12
    assert abs(vs[N, 0, 1]) < 1e-10 and xs[N, 0, 0] == np.float32(0.3)
    seed = np.zeros((1, 3))
    seed[0, 1] = 1.0
    gr = oracle_mod.adjoint(sc, {N: seed}, N, iters)
    assert abs(gr["collider"][0] - 1.0) < 1e-9
    assert abs(gr["x0"][0, 1]) < 1e-9


# ------------------------------------------------------------------------- sphere

@pytest.mark.parametrize("iters", [1, 3])
def test_sphere_one_update_closed_form(oracle_mod, iters):
    """Vertices predicted inside |x - c| = r + t move out radially to
    |x' - c| - r - t = (|p - c| - r - t) alpha~/(w + alpha~) with their direction from c
    unchanged; vertices outside are untouched.  Derivatives in (c, r) and x0 follow from
    x' = c + (p - c) rr + (r + t)(1 - rr) n, n = (p - c)/|p - c|."""
    m, t = 0.02, 0.004
    c = np.array([0.1, -0.2, 0.3])
    R = 0.25
    sc0 = _points(np.zeros((1, 3)), np.zeros((1, 3)), m, flags=scenes.COLLIDE_SPHERE, alpha_c=0.0,
                  thickness=t, sphere=(*c, R))
    c = np.asarray(sc0.sphere[:3], np.float64)
    R = float(sc0.sphere[3])
    rng = np.random.default_rng(2)
    dirs = rng.normal(size=(8, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    radii = np.array([0.20, 0.24, 0.25, 0.251, 0.30, 0.22, 0.35, 0.10])
    x0 = c + dirs * radii[:, None]
    w = float(f32(1.0 / m))
    alpha = 0.4 * w * DT ** 2                        # rr = 0.4/1.4
    sc = _points(x0, np.zeros((8, 3)), m, flags=scenes.COLLIDE_SPHERE, alpha_c=alpha, thickness=t,
                 sphere=(*c, R), gravity=(0.0, 0.0, 0.0))
    p = _predicted(sc)
    d = np.linalg.norm(p - c, axis=1)
    n = (p - c) / d[:, None]
    Cp = d - R - t
    active = Cp < 0
    assert active.sum() == 6 and np.abs(Cp).min() > 5e-4
    at = alpha / DT ** 2
    rr = at / (w + at)
    expect = p.copy()
    expect[active] = c + n[active] * (R + t + Cp[active] * rr)[:, None]
    xs, _ = oracle_mod.forward(sc, 1, iters)
    assert np.abs(xs[1] - expect).max() < 1e-14
    assert np.all(np.linalg.norm(xs[1][active] - c, axis=1) > d[active])
    # reverse sweep for L = sum_i u_i . x'_i
    u = rng.normal(size=(8, 3))
    gr = oracle_mod.adjoint(sc, {1: u}, 1, iters)
    dr = sum((1 - rr) * u[i] @ n[i] for i in np.nonzero(active)[0])
    dc = np.zeros(3)
    dx0 = u.copy()
    I3 = np.eye(3)
    for i in np.nonzero(active)[0]:
        P = I3 - np.outer(n[i], n[i])
        dc += ((1 - rr) * I3 - (R + t) * (1 - rr) * P / d[i]) @ u[i]
        dx0[i] = (rr * I3 + (R + t) * (1 - rr) * P / d[i]) @ u[i]
    assert abs(gr["collider"][4] - dr) < 1e-12
    assert np.abs(gr["collider"][1:4] - dc).max() < 1e-12
    assert gr["collider"][0] == 0.0
    assert np.abs(gr["x0"] - dx0).max() < 1e-12


def test_sphere_resting_depth_at_the_top_is_hooke(oracle_mod):
    """A vertex released on top of the sphere settles m g alpha below the surface, radially
    (gravity is along the normal there); the settled height follows r and c_y one to one."""
    m, t = 0.01, 0.001
    sc0 = _points(np.zeros((1, 3)), np.zeros((1, 3)), m, flags=scenes.COLLIDE_SPHERE, alpha_c=0.0,
                  thickness=t, sphere=(0.5, -0.35, 0.5, 0.3))
    cx, cy, cz, R = (float(v) for v in sc0.sphere)
    w = float(f32(1.0 / m))
    alpha = w * DT ** 2
    top = [[cx, cy + R + t, cz]]
    sc = _points(top, np.zeros((1, 3)), m, flags=scenes.COLLIDE_SPHERE, alpha_c=alpha, thickness=t,
                 sphere=(cx, cy, cz, R))
    N = 250
    xs, _ = oracle_mod.forward(sc, N, 2)
    depth = (1.0 / float(sc.inv_mass[0])) * G * alpha
    assert abs(xs[N, 0, 1] - (cy + R + t - depth)) < 1e-10
    assert xs[N, 0, 0] == np.float32(cx) and xs[N, 0, 2] == np.float32(cz)
    seed = np.zeros((1, 3))
    seed[0, 1] = 1.0
    gr = oracle_mod.adjoint(sc, {N: seed}, N, 2)
    assert abs(gr["collider"][4] - 1.0) < 1e-8 and abs(gr["collider"][2] - 1.0) < 1e-8
    assert abs(gr["collider"][1]) < 1e-8 and abs(gr["collider"][3]) < 1e-8


# ------------------------------------------------------------------ detect once (R12)

def _spring_pair(yA, yB, L, *, at_s, at_c, t, h=0.0):
    """Vertex 0 pinned at (0, yA, 0), vertex 1 free at (0, yB, 0), one spring of rest length
    L between them (from the rest positions), no gravity, a plane at h."""
    m = 0.01
    w = float(np.float32(1.0 / m))
    return _points([[0.0, yA, 0.0], [0.0, yB, 0.0]], np.zeros((2, 3)), [0.0, m], flags=scenes.COLLIDE_PLANE,
                   alpha_c=at_c * w * DT ** 2, thickness=t, plane_h=h, gravity=(0.0, 0.0, 0.0), dist=(0, 1),
                   dist_alpha=at_s * w * DT ** 2, rest=[[0.0, yA, 0.0], [0.0, yA + (L if yB > yA else -L), 0.0]])


@pytest.mark.parametrize("iters", [1, 3])
def test_vertex_not_in_contact_at_prediction_is_never_projected(oracle_mod, iters):
    """Predicted 2 cm above the plane, the vertex is pulled 5.6 cm down (to 3.6 cm below
    the plane) by a spring in the first iteration.  Its contact was inactive at the
    predicted position, so no iteration of this step touches it: it ends where the spring
    alone puts it, C' = C alpha~_s/(w + alpha~_s) from the spring's closed form."""
    t = 0.001
    sc = _spring_pair(-0.1, 0.02, 0.05, at_s=0.25, at_c=0.01, t=t)
    w, at_s = float(sc.inv_mass[1]), float(sc.compliance[0]) / DT ** 2
    L = float(sc.rest_x[1, 1]) - float(sc.rest_x[0, 1])
    C = (float(sc.x0[1, 1]) - float(sc.x0[0, 1])) - L
    yB = float(sc.x0[0, 1]) + L + C * at_s / (w + at_s)
    xs, _ = oracle_mod.forward(sc, 1, iters)
    assert abs(xs[1, 1, 1] - yB) < 1e-14
    assert xs[1, 1, 1] < -0.03                     # left below the plane for this step


def test_contact_active_at_prediction_stays_an_equality(oracle_mod):
    """Predicted 1 cm below the plane, the vertex is pulled 4.8 cm up (above the plane) by a
    spring, then the contact pass runs on it all the same (it was detected at the
    prediction) and, with no clamp on lambda, pulls it back toward the plane:
    y'' = y' - (y' - h - t) w/(w + alpha~_c)."""
    t = 0.001
    sc = _spring_pair(0.1, -0.01, 0.05, at_s=0.25, at_c=0.01, t=t)
    w, at_s, at_c = float(sc.inv_mass[1]), float(sc.compliance[0]) / DT ** 2, sc.contact_compliance / DT ** 2
    L = float(sc.rest_x[0, 1]) - float(sc.rest_x[1, 1])
    C = (float(sc.x0[0, 1]) - float(sc.x0[1, 1])) - L
    y1 = float(sc.x0[1, 1]) + w * C / (w + at_s)     # the spring update, lambda = 0
    assert y1 > t
    y2 = y1 - w * (y1 - t) / (w + at_c)              # the contact update, lambda_c = 0
    xs, _ = oracle_mod.forward(sc, 1, 1)
    assert abs(xs[1, 1, 1] - y2) < 1e-14
