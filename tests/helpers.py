"""Small hand-built scenes for the oracle pins and the GPU parity tests."""
import numpy as np

from paper_2301_01396_gb300 import scenes
from paper_2301_01396_gb300.scenes import Scene, f32


def single_spring(L=0.5, stretch0=0.0, mass=0.01, alpha=1e-3, dt=1.0 / 60.0):
    """Vertex 0 pinned at the origin, vertex 1 hanging below it on one spring of rest
    length L (the rest positions define L), both on the y axis."""
    rest = np.array([[0.0, 0.0, 0.0], [0.0, -L, 0.0]])
    x0 = np.array([[0.0, 0.0, 0.0], [0.0, -(L + stretch0), 0.0]])
    return Scene(rest_x=f32(rest), inv_mass=f32([0.0, 1.0 / mass]),
                 dist_idx=np.array([[0, 1]], np.int32), bend_idx=np.zeros((0, 4), np.int32),
                 tet_idx=np.zeros((0, 4), np.int32), tet_gamma=np.zeros(0),
                 color_offsets=np.array([0, 1], np.int32), color_order=np.array([0], np.int32),
                 x0=f32(x0), v0=np.zeros((2, 3)), compliance=f32([alpha]), dt=dt,
                 gravity=(0.0, -9.81, 0.0), steps=10, iters=1, name="single_spring")


def small_cloth(n=5, *, bending=True, diagonals="both", pins=((0, 0), (-1, 0)), seed=0,
                plane_h=None, steps=4, iters=3, gravity=(0.0, -9.81, 0.0), jitter=0.0,
                v_scale=0.0, stretch=1e-3, bend=1e-2, coloring="pattern", tile=48):
    g = scenes.cloth_grid(n, 1.0, areal_density=2.56, diagonals=diagonals, bending=bending, pins=pins,
                          coloring=coloring, tile=tile)
    rng = np.random.default_rng(seed)
    alpha = scenes.lognormal_cloth_compliance(rng, g["dist_idx"].shape[0], g["bend_idx"].shape[0],
                                              stretch=stretch, bend=bend)
    sc = scenes._cloth_scene(g, alpha, dt=1.0 / 60.0, steps=steps, iters=iters, gravity=gravity,
                             name=f"small_cloth_{n}")
    if jitter:
        sc.x0 = f32(sc.x0 + jitter * rng.standard_normal(sc.x0.shape))
    if v_scale:
        v = v_scale * rng.standard_normal(sc.x0.shape)
        v[sc.inv_mass == 0] = 0.0
        sc.v0 = f32(v)
    if plane_h is not None:
        sc.collider_flags = scenes.COLLIDE_PLANE
        sc.plane_h = plane_h
    return sc


def small_tets(n=2, *, steps=3, iters=3, seed=3, y0=0.02, plane=True, gravity=(0.0, -9.81, 0.0),
               jitter=0.0, v_scale=0.0, alpha=(1e-5, 1e-3)):
    sc = scenes.tet_block(n, size=0.2, y0=y0, steps=steps, iters=iters, seed=seed, alpha_lo=alpha[0],
                          alpha_hi=alpha[1])
    sc.gravity = gravity
    rng = np.random.default_rng(seed + 100)
    if jitter:
        sc.x0 = f32(sc.x0 + jitter * rng.standard_normal(sc.x0.shape))
    if v_scale:
        sc.v0 = f32(v_scale * rng.standard_normal(sc.x0.shape))
    if not plane:
        sc.collider_flags = 0
    return sc


def small_sphere_cloth(n=6, *, steps=4, iters=3, seed=4):
    """A small unpinned cloth dropped on a sphere whose top sits just below it, with
    per-step global forces and a per-vertex force field."""
    g = scenes.cloth_grid(n, 1.0, areal_density=2.56, diagonals="both", bending=True, pins=())
    rng = np.random.default_rng(seed)
    alpha = scenes.lognormal_cloth_compliance(rng, g["dist_idx"].shape[0], g["bend_idx"].shape[0],
                                              stretch=1e-3, bend=1e-2)
    V = n * n
    m_i = 2.56 / V
    sc = scenes._cloth_scene(g, alpha, dt=1.0 / 60.0, steps=steps, iters=iters,
                             collider_flags=scenes.COLLIDE_SPHERE,
                             sphere=tuple(float(v) for v in f32([0.47, -0.31, 0.52, 0.3])),
                             contact_compliance=1e-6, name=f"small_sphere_{n}")
    sc.v0 = f32(np.tile([0.0, -0.6, 0.0], (V, 1)) + 0.05 * rng.standard_normal((V, 3)))
    sc.f_global = f32(0.3 * m_i * 9.81 * rng.standard_normal((steps, 3)))
    sc.f_vertex = f32(0.3 * m_i * 9.81 * rng.standard_normal((V, 3)))
    return sc


def grid_window(full, n, i0, j0, w):
    """The sub-scene of an n x n grid scene on vertices i0 <= i < i0+w, j0 <= j < j0+w,
    keeping every constraint whose vertices all lie inside, in the same color order."""
    ii = np.arange(full.V) % n
    jj = np.arange(full.V) // n
    inside = (ii >= i0) & (ii < i0 + w) & (jj >= j0) & (jj < j0 + w)
    local = np.full(full.V, -1, np.int64)
    local[inside] = (jj[inside] - j0) * w + (ii[inside] - i0)
    keep_d = inside[full.dist_idx].all(1)
    keep_b = inside[full.bend_idx].all(1)
    nd, nb = int(keep_d.sum()), int(keep_b.sum())
    new_id = np.full(full.m, -1, np.int64)
    new_id[:full.n_dist][keep_d] = np.arange(nd)
    new_id[full.n_dist:][keep_b] = nd + np.arange(nb)
    offs = [0]
    order = []
    for c in range(full.n_colors):
        ids = full.color_order[full.color_offsets[c]:full.color_offsets[c + 1]]
        ids = new_id[ids]
        ids = ids[ids >= 0]
        order.append(ids)
        offs.append(offs[-1] + ids.shape[0])
    sel = np.nonzero(inside)[0][np.argsort(local[inside])]
    comp = np.concatenate([full.compliance[:full.n_dist][keep_d], full.compliance[full.n_dist:][keep_b]])
    sub = full.with_(rest_x=full.rest_x[sel], inv_mass=full.inv_mass[sel],
                     dist_idx=local[full.dist_idx[keep_d]].astype(np.int32),
                     bend_idx=local[full.bend_idx[keep_b]].astype(np.int32),
                     color_offsets=np.asarray(offs, np.int32),
                     color_order=np.concatenate(order).astype(np.int32),
                     x0=full.x0[sel], v0=full.v0[sel], compliance=comp,
                     f_vertex=None if full.f_vertex is None else full.f_vertex[sel])
    return sub, sel, np.nonzero(keep_d)[0], full.n_dist + np.nonzero(keep_b)[0]


def rel(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
