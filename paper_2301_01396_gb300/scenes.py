"""Seeded synthetic scene generators.

This module is the one piece of code shared by the CUDA path (its tests, ``bench.py``)
and the FP64 oracle's tests.  It builds meshes, constraint topology, graph colorings,
masses, start states and seeded parameter draws, and nothing else: it evaluates no
constraint, projects nothing and differentiates nothing.  Rest lengths, rest angles,
reference shape matrices and rest volumes are computed independently by each side from
``rest_x``.

Every float this module emits is rounded to a value FP32 represents exactly, so the FP32
GPU path and the FP64 oracle start from identical inputs.

Constraint id space (used by ``compliance`` and the coloring):
    [0, nd)                 distance constraints        (``dist_idx`` rows)
    [nd, nd+nb)             dihedral bending hinges     (``bend_idx`` rows: edge v0-v1, wings v2, v3)
    [nd+nb, nd+nb+nt)       tet hydrostatic  C_H = det F - gamma
    [nd+nb+nt, nd+nb+2nt)   tet deviatoric   C_D = ||F||_F
Compliance units: distance and bending constraints take the constraint compliance alpha
directly (Sec. 3.1, Eq. xpbdUenergy); tet constraints take the inverse Lame modulus
alpha_hat, and the constraint compliance is alpha_hat / V_e (V_e the rest volume).

Workload recipes follow the five synthetic configurations: plain pinned cloth (16x16),
cloth with bending on a ground plane (256x256), a 5-tet-per-cube block falling on a ground
plane (32^3 cells), a 2950x2950 cloth draped on a sphere with per-frame and per-vertex
forces, and a mixed serving stream.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import Optional

import numpy as np

COLLIDE_PLANE = 1
COLLIDE_SPHERE = 2


def f32(a) -> np.ndarray:
    """Round to FP32-representable values, returned as float64."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


@dataclass
class Scene:
    """A complete simulation input: topology, coloring, start state and parameters."""

    rest_x: np.ndarray                  # [V,3] rest positions (define L, theta0, Dm^-1, V_e)
    inv_mass: np.ndarray                # [V] w = 1/m, 0 = pinned
    dist_idx: np.ndarray                # [nd,2] int32
    bend_idx: np.ndarray                # [nb,4] int32  (edge v0,v1; wing v2 side A, wing v3 side B)
    tet_idx: np.ndarray                 # [nt,4] int32  (positively oriented)
    tet_gamma: np.ndarray               # [nt] hydrostatic rest offset gamma
    color_offsets: np.ndarray           # [K+1] int32
    color_order: np.ndarray             # [m] int32 global constraint ids, color by color
    x0: np.ndarray                      # [V,3]
    v0: np.ndarray                      # [V,3]
    compliance: np.ndarray              # [m]
    dt: float = 1.0 / 60.0
    gravity: tuple = (0.0, -9.81, 0.0)
    steps: int = 1
    iters: int = 1
    collider_flags: int = 0
    plane_h: float = 0.0
    sphere: tuple = (0.0, 0.0, 0.0, 0.0)   # cx, cy, cz, r
    contact_compliance: float = 1e-8
    thickness: float = 0.0
    f_global: Optional[np.ndarray] = None  # [steps,3] force added to every vertex at step n
    f_vertex: Optional[np.ndarray] = None  # [V,3] time-constant per-vertex force
    f_vertex_steps: Optional[np.ndarray] = None  # [steps,V,3] force on each vertex at each step
    tet_coupled: bool = False           # project each tet's C_H and C_D together (2x2 solve);
                                        # the coloring then lists C_H ids only
    # orthotropic StVK membrane triangles (coloring ids m + t): vertices, the warp/weft (u, v)
    # rest coordinates of each triangle's vertices, and (C00, C11, C01, C22) per triangle
    memb_idx: np.ndarray = field(default_factory=lambda: np.zeros((0, 3), np.int32))
    memb_uv: np.ndarray = field(default_factory=lambda: np.zeros((0, 3, 2)))
    memb_stiffness: np.ndarray = field(default_factory=lambda: np.zeros((0, 4)))
    name: str = "scene"
    meta: dict = field(default_factory=dict)

    @property
    def V(self) -> int:
        return int(self.rest_x.shape[0])

    @property
    def n_dist(self) -> int:
        return int(self.dist_idx.shape[0])

    @property
    def n_bend(self) -> int:
        return int(self.bend_idx.shape[0])

    @property
    def n_tet(self) -> int:
        return int(self.tet_idx.shape[0])

    @property
    def m(self) -> int:
        return self.n_dist + self.n_bend + 2 * self.n_tet

    @property
    def n_memb(self) -> int:
        return int(self.memb_idx.shape[0])

    @property
    def n_colored(self) -> int:
        """Constraint ids the coloring lists: the scalar ones (all but the C_D ids when each
        tet's two constraints are projected together), then one id m + t per membrane."""
        return self.m - (self.n_tet if self.tet_coupled else 0) + self.n_memb

    @property
    def n_colors(self) -> int:
        return int(self.color_offsets.shape[0] - 1)

    def with_(self, **kw) -> "Scene":
        return replace(self, **kw)


# ----------------------------------------------------------------------------------------
# coloring helpers (host logic: graph coloring is an input of the solver, Sec. 3.1)
# ----------------------------------------------------------------------------------------

def constraint_vertices(scene: Scene, cid: int) -> tuple:
    nd, nb, nt = scene.n_dist, scene.n_bend, scene.n_tet
    if cid < nd:
        return tuple(int(v) for v in scene.dist_idx[cid])
    cid -= nd
    if cid < nb:
        return tuple(int(v) for v in scene.bend_idx[cid])
    cid -= nb
    if cid < 2 * nt:
        return tuple(int(v) for v in scene.tet_idx[cid % nt])
    cid -= 2 * nt
    if cid < scene.n_memb:
        return tuple(int(v) for v in scene.memb_idx[cid])
    raise IndexError("constraint id out of range")


def _vertex_table(scene: Scene) -> np.ndarray:
    """[m, 4] vertex ids of every constraint, -1 padded."""
    rows = [np.pad(scene.dist_idx, ((0, 0), (0, 2)), constant_values=-1) if scene.n_dist else
            np.zeros((0, 4), np.int64)]
    rows.append(scene.bend_idx.astype(np.int64) if scene.n_bend else np.zeros((0, 4), np.int64))
    rows.append(scene.tet_idx.astype(np.int64) if scene.n_tet else np.zeros((0, 4), np.int64))
    rows.append(scene.tet_idx.astype(np.int64) if scene.n_tet else np.zeros((0, 4), np.int64))
    rows.append(np.pad(scene.memb_idx.astype(np.int64), ((0, 0), (0, 1)), constant_values=-1) if scene.n_memb
                else np.zeros((0, 4), np.int64))
    return np.concatenate(rows, axis=0)


def validate_coloring(scene: Scene) -> None:
    """Raise ValueError unless every constraint appears exactly once and no two
    constraints of one color share a vertex."""
    order = np.asarray(scene.color_order, np.int64)
    offs = np.asarray(scene.color_offsets, np.int64)
    n = scene.n_colored
    if offs[0] != 0 or offs[-1] != n or np.any(np.diff(offs) < 0):
        raise ValueError("bad color offsets")
    ids = np.concatenate([np.arange(scene.m - (scene.n_tet if scene.tet_coupled else 0)),
                          scene.m + np.arange(scene.n_memb)])
    if order.shape[0] != n or np.any(np.sort(order) != ids):
        raise ValueError("coloring is not a permutation of the constraints")
    table = _vertex_table(scene)
    for c in range(scene.n_colors):
        ids = order[offs[c]:offs[c + 1]]
        verts = table[ids].reshape(-1)
        verts = verts[verts >= 0]
        if np.unique(verts).shape[0] != verts.shape[0]:
            raise ValueError(f"color {c} has a vertex shared by two constraints")


def greedy_coloring(scene: Scene, groups=None):
    """First-fit greedy coloring of the constraint graph (constraints adjacent when they
    share a vertex).  ``groups`` is an optional list of constraint-id arrays colored
    separately (so every color holds one constraint type).  Returns (offsets, order)."""
    table = _vertex_table(scene)
    if groups is None:
        groups = [np.arange(scene.m)]
    offsets = [0]
    order = []
    for ids in groups:
        vert_colors = {}
        buckets: list = []
        for cid in ids:
            vs = [int(v) for v in table[cid] if v >= 0]
            used = set()
            for v in vs:
                used |= vert_colors.get(v, set())
            c = 0
            while c in used:
                c += 1
            if c == len(buckets):
                buckets.append([])
            buckets[c].append(int(cid))
            for v in vs:
                vert_colors.setdefault(v, set()).add(c)
        for b in buckets:
            order.extend(sorted(b, key=lambda j: table[j][0]))
            offsets.append(len(order))
    return np.asarray(offsets, np.int32), np.asarray(order, np.int32)


# ----------------------------------------------------------------------------------------
# cloth grid
# ----------------------------------------------------------------------------------------

def _grid_topology(n: int, diagonals: str, bending: bool):
    """Edges and hinges of an n x n vertex grid, vertex (i, j) -> j*n + i, grouped into
    vertex-disjoint color classes (pattern coloring of the regular grid)."""
    I, J = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")  # I[j, i] = i
    vid = lambda i, j: (j * n + i)
    classes = []   # list of (kind, idx array [k, 2|4])

    def add_edges(a, b, key):
        for par in (0, 1):
            sel = (key % 2) == par
            if np.any(sel):
                classes.append(("dist", np.stack([a[sel], b[sel]], axis=1)))

    # structural: horizontal (i,j)-(i+1,j), colored by i parity
    i, j = I[:, :-1].ravel(), J[:, :-1].ravel()
    add_edges(vid(i, j), vid(i + 1, j), i)
    # structural: vertical (i,j)-(i,j+1), colored by j parity
    i, j = I[:-1, :].ravel(), J[:-1, :].ravel()
    add_edges(vid(i, j), vid(i, j + 1), j)
    if diagonals in ("one", "both"):
        i, j = I[:-1, :-1].ravel(), J[:-1, :-1].ravel()
        add_edges(vid(i, j), vid(i + 1, j + 1), i)
    if diagonals == "both":
        i, j = I[:-1, :-1].ravel(), J[:-1, :-1].ravel()
        add_edges(vid(i + 1, j), vid(i, j + 1), i)
    if bending:
        # triangulation with diagonal (i,j)-(i+1,j+1): quad (i,j) -> T1=(i,j),(i+1,j),(i+1,j+1)
        # and T2=(i,j),(i+1,j+1),(i,j+1).  Hinges on interior axis-aligned edges only.
        # horizontal hinge edge (i,j)-(i+1,j), 1<=j<=n-2: wings (i+1,j+1) [T1 of quad (i,j)]
        # and (i,j-1) [T2 of quad (i,j-1)]
        i, j = I[1:-1, :-1].ravel(), J[1:-1, :-1].ravel()
        h = np.stack([vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j - 1)], axis=1)
        for pi in (0, 1):
            for pj in (0, 1):
                sel = ((i % 2) == pi) & ((j % 2) == pj)
                if np.any(sel):
                    classes.append(("bend", h[sel]))
        # vertical hinge edge (i,j)-(i,j+1), 1<=i<=n-2: wings (i-1,j) [T1 of quad (i-1,j)]
        # and (i+1,j+1) [T2 of quad (i,j)], ordered so side A/B match the horizontal case
        i, j = I[:-1, 1:-1].ravel(), J[:-1, 1:-1].ravel()
        h = np.stack([vid(i, j), vid(i, j + 1), vid(i - 1, j), vid(i + 1, j + 1)], axis=1)
        for pi in (0, 1):
            for pj in (0, 1):
                sel = ((i % 2) == pi) & ((j % 2) == pj)
                if np.any(sel):
                    classes.append(("bend", h[sel]))
    return classes


def cloth_grid(n: int, size: float = 1.0, *, vertex_mass: Optional[float] = None,
               areal_density: float = 2.56, diagonals: str = "both", bending: bool = False,
               pins=((0, 0), (-1, 0)), y0: float = 0.0, origin=(0.0, 0.0), coloring: str = "pattern",
               tile: int = 32) -> dict:
    """An n x n vertex cloth square in the x-z plane at height y0.

    coloring="pattern": one color per constraint family and parity (2 per edge family, 4
    per hinge family).  coloring="tiled": the grid is cut into tile x tile blocks of
    vertices, each constraint belongs to the block of its first vertex, and blocks are
    classed by the parities of their block coordinates (4 classes); the colors are the
    pattern colors restricted to one class, ordered class by class.  Blocks of one class
    are a block apart, so within a class every block's constraints only touch that block
    and its one-vertex border: a class's 16 colors run block by block.

    Returns the raw arrays (positions, masses, topology, coloring) of a cloth grid; the
    ``cloth_*`` config builders below turn them into a Scene."""
    if n < 2:
        raise ValueError("grid needs n >= 2")
    h = size / (n - 1)
    I, J = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    x = np.stack([origin[0] + I.ravel() * h, np.full(n * n, y0), origin[1] + J.ravel() * h], axis=1)
    if vertex_mass is None:
        vertex_mass = areal_density * size * size / (n * n)
    w = np.full(n * n, 1.0 / vertex_mass)
    for (pi, pj) in pins:
        pi = pi % n
        pj = pj % n
        w[pj * n + pi] = 0.0
    classes = _grid_topology(n, diagonals, bending)
    if coloring == "tiled":
        if tile < 4:
            raise ValueError("tile must be >= 4 (a hinge spans three rows)")
        tiled = []
        for cls in range(4):
            for kind, idx in classes:
                first = idx[:, 0]
                ti, tj = (first % n) // tile, (first // n) // tile
                sel = ((ti % 2) + 2 * (tj % 2)) == cls
                if np.any(sel):
                    tiled.append((kind, idx[sel]))
        classes = tiled
    elif coloring != "pattern":
        raise ValueError("coloring must be 'pattern' or 'tiled'")
    dist = [c[1] for c in classes if c[0] == "dist"]
    bend = [c[1] for c in classes if c[0] == "bend"]
    dist_idx = np.concatenate(dist).astype(np.int32) if dist else np.zeros((0, 2), np.int32)
    bend_idx = np.concatenate(bend).astype(np.int32) if bend else np.zeros((0, 4), np.int32)
    nd = dist_idx.shape[0]
    offsets = [0]
    order = []
    d0 = 0
    b0 = nd
    for kind, idx in classes:
        k = idx.shape[0]
        if kind == "dist":
            order.append(np.arange(d0, d0 + k))
            d0 += k
        else:
            order.append(np.arange(b0, b0 + k))
            b0 += k
        offsets.append(offsets[-1] + k)
    return dict(rest_x=f32(x), inv_mass=f32(w), dist_idx=dist_idx, bend_idx=bend_idx,
                color_offsets=np.asarray(offsets, np.int32),
                color_order=(np.concatenate(order).astype(np.int32) if order else np.zeros(0, np.int32)))


def _cloth_scene(g: dict, compliance: np.ndarray, **kw) -> Scene:
    V = g["rest_x"].shape[0]
    return Scene(rest_x=g["rest_x"], inv_mass=g["inv_mass"], dist_idx=g["dist_idx"],
                 bend_idx=g["bend_idx"], tet_idx=np.zeros((0, 4), np.int32),
                 tet_gamma=np.zeros(0), color_offsets=g["color_offsets"],
                 color_order=g["color_order"], x0=g["rest_x"].copy(), v0=np.zeros((V, 3)),
                 compliance=f32(compliance), **kw)


def plain_cloth(n: int = 16, *, compliance: float = 1e-7, steps: int = 50, iters: int = 20,
                seed: int = 1, target: bool = False) -> Scene:
    """Plain XPBD cloth: 1 m square, 0.01 kg per vertex, two top corners pinned,
    structural + both shear diagonals, uniform compliance, gravity, dt = 1/60.
    With ``target``: the per-constraint compliance is multiplied by exp(0.5 z),
    z ~ N(0, 1) (seeded), as used to produce the target trajectory."""
    g = cloth_grid(n, 1.0, vertex_mass=0.01, diagonals="both", bending=False)
    nd = g["dist_idx"].shape[0]
    alpha = np.full(nd, compliance)
    if target:
        rng = np.random.default_rng(seed)
        alpha = alpha * np.exp(0.5 * rng.standard_normal(nd))
    return _cloth_scene(g, alpha, dt=1.0 / 60.0, steps=steps, iters=iters,
                        name=f"plain_cloth_{n}")


def membrane_cloth(n: int = 32, size: float = 1.0, *, areal_density: float = 0.2, pins=((0, 0), (-1, 0)),
                   stiffness=(2000.0, 800.0, 300.0, 400.0), spread: float = 0.3, bend: float = 1e-2,
                   bending: bool = True, seed: int = 9, steps: int = 30, iters: int = 10,
                   dt: float = 1.0 / 60.0, coloring: str = "pattern", tile: int = 32) -> Scene:
    """Orthotropic StVK membrane cloth (Sec. "Cloth Material Parameter Estimation"): an
    n x n vertex sheet in the x-z plane, warp u along x and weft v along z (the rest
    positions are the pattern coordinates), two triangles per grid cell, each carrying the
    Green-strain membrane constraint with its own stiffness (C00, C11, C01, C22): the
    base ``stiffness`` with C00, C11, C22 scaled by exp(spread z) (seeded normal z) and
    C01 = nu sqrt(C00 C11) with the base's nu, so every K stays positive definite; plus
    dihedral bending with lognormal compliance around ``bend`` on interior edges.
    coloring="pattern": 8 membrane colors (cell parities x triangle), then the bending
    colors.  coloring="tiled": as cloth_grid's, the pattern colors restricted to 4 classes
    of tile x tile vertex blocks (by the block of each element's first vertex), class by
    class, so that a class's colors run block by block (the phase plan)."""
    if n < 2:
        raise ValueError("grid needs n >= 2")
    h = size / (n - 1)
    I, J = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    x = np.stack([I.ravel() * h, np.zeros(n * n), J.ravel() * h], axis=1)
    w = np.full(n * n, n * n / (areal_density * size * size))
    for (pi, pj) in pins:
        w[(pj % n) * n + (pi % n)] = 0.0
    vid = lambda i, j: j * n + i
    ci, cj = np.meshgrid(np.arange(n - 1), np.arange(n - 1), indexing="xy")
    ci, cj = ci.ravel(), cj.ravel()
    tris, order_m, offsets = [], [], [0]
    t0 = 0
    for tri in (0, 1):
        for pi in (0, 1):
            for pj in (0, 1):
                sel = ((ci % 2) == pi) & ((cj % 2) == pj)
                i, j = ci[sel], cj[sel]
                if tri == 0:
                    t = np.stack([vid(i, j), vid(i + 1, j), vid(i + 1, j + 1)], axis=1)
                else:
                    t = np.stack([vid(i, j), vid(i + 1, j + 1), vid(i, j + 1)], axis=1)
                tris.append(t)
                order_m.append(np.arange(t0, t0 + t.shape[0]))
                t0 += t.shape[0]
                offsets.append(offsets[-1] + t.shape[0])
    memb_idx = np.concatenate(tris).astype(np.int32)
    nm = memb_idx.shape[0]
    uv = x[:, [0, 2]][memb_idx]                                  # [nm, 3, 2]
    bend_cls = [c[1] for c in _grid_topology(n, "none", bending) if c[0] == "bend"] if bending else []
    bend_idx = np.concatenate(bend_cls).astype(np.int32) if bend_cls else np.zeros((0, 4), np.int32)
    nb = bend_idx.shape[0]
    order = [o + nb for o in order_m]                            # membrane ids m + t (m = nb)
    b0 = 0
    for c in bend_cls:
        order.append(np.arange(b0, b0 + c.shape[0]))
        b0 += c.shape[0]
        offsets.append(offsets[-1] + c.shape[0])
    if coloring == "tiled":
        if tile < 4:
            raise ValueError("tile must be >= 4")
        # first vertex of each colored id: membranes (ids nb + t) then bending (ids 0..nb-1)
        fv = np.empty(nb + nm, np.int64)
        fv[nb:] = memb_idx[:, 0]
        if nb:
            fv[:nb] = bend_idx[:, 0]
        cls_of = lambda ids: ((fv[ids] % n) // tile % 2) + 2 * ((fv[ids] // n) // tile % 2)
        t_order, t_offs = [], [0]
        for cls in range(4):
            for ids in order:
                sel = ids[cls_of(ids) == cls]
                if sel.shape[0]:
                    t_order.append(sel)
                    t_offs.append(t_offs[-1] + sel.shape[0])
        order, offsets = t_order, t_offs
    elif coloring != "pattern":
        raise ValueError("coloring must be 'pattern' or 'tiled'")
    rng = np.random.default_rng(seed)
    c00, c11, c01, c22 = stiffness
    nu = c01 / np.sqrt(c00 * c11)
    z = rng.standard_normal((nm, 3))
    k00 = c00 * np.exp(spread * z[:, 0])
    k11 = c11 * np.exp(spread * z[:, 1])
    k22 = c22 * np.exp(spread * z[:, 2])
    K = np.stack([k00, k11, nu * np.sqrt(k00 * k11), k22], axis=1)
    alpha_b = bend * np.exp(0.5 * rng.standard_normal(nb))
    xr = f32(x)
    return Scene(rest_x=xr, inv_mass=f32(w), dist_idx=np.zeros((0, 2), np.int32), bend_idx=bend_idx,
                 tet_idx=np.zeros((0, 4), np.int32), tet_gamma=np.zeros(0),
                 color_offsets=np.asarray(offsets, np.int32),
                 color_order=np.concatenate(order).astype(np.int32), x0=xr.copy(), v0=np.zeros((n * n, 3)),
                 compliance=f32(alpha_b), dt=dt, steps=steps, iters=iters,
                 memb_idx=memb_idx, memb_uv=f32(uv), memb_stiffness=f32(K), name=f"membrane_cloth_{n}")


def lognormal_cloth_compliance(rng, nd: int, nb: int, stretch: float = 1e-4,
                               bend: float = 1e-2) -> np.ndarray:
    return np.concatenate([stretch * np.exp(0.5 * rng.standard_normal(nd)),
                           bend * np.exp(0.5 * rng.standard_normal(nb))])


def ground_cloth(n: int = 256, *, steps: int = 100, iters: int = 30, seed: int = 2,
                 plane_h: float = -0.6, pins=(), tilt: float = 0.3) -> Scene:
    """Cloth with stretch/shear springs (one diagonal) and dihedral bending, per-constraint
    lognormal compliance, falling onto a ground plane.  No vertex is pinned; the sheet
    starts flat and at rest, tilted by `tilt` radians about the x axis (through its centre
    line z = 0.5), so it reaches the ground progressively."""
    g = cloth_grid(n, 1.0, areal_density=2.56, diagonals="one", bending=True, pins=pins)
    if tilt:
        x = g["rest_x"].copy()
        z = x[:, 2] - 0.5
        x[:, 1] = x[:, 1] + np.sin(tilt) * z
        x[:, 2] = 0.5 + np.cos(tilt) * z
        g["rest_x"] = f32(x)
    rng = np.random.default_rng(seed)
    alpha = lognormal_cloth_compliance(rng, g["dist_idx"].shape[0], g["bend_idx"].shape[0])
    return _cloth_scene(g, alpha, dt=1.0 / 60.0, steps=steps, iters=iters,
                        collider_flags=COLLIDE_PLANE, plane_h=plane_h, contact_compliance=1e-8,
                        name=f"ground_cloth_{n}")


def sphere_cloth(n: int = 2950, *, steps: int = 60, iters: int = 15, seed: int = 4,
                 radius: float = 0.3, force_scale: float = 0.2, coloring: str = "pattern",
                 tile: int = 32) -> Scene:
    """High-resolution cloth (structural + both diagonals + bending) with no pins, falling
    on an analytic sphere, driven by a per-frame global force G_n (3 per step) and a
    time-constant smooth per-vertex wind field W."""
    g = cloth_grid(n, 1.0, areal_density=2.56, diagonals="both", bending=True, pins=(),
                   coloring=coloring, tile=tile)
    rng = np.random.default_rng(seed)
    centre = np.array([0.5, -0.35, 0.5]) + rng.uniform(-0.05, 0.05, 3)
    alpha = lognormal_cloth_compliance(rng, g["dist_idx"].shape[0], g["bend_idx"].shape[0])
    V = n * n
    m_i = 2.56 / V
    amp = force_scale * m_i * 9.81
    phase = rng.uniform(0, 2 * np.pi, 3)
    t = np.arange(steps)[:, None]
    f_global = amp * np.sin(2 * np.pi * t / 60.0 + phase[None, :])
    # smooth wind: a few low-order Fourier modes over the rest (x, z) coordinates
    x = g["rest_x"]
    W = np.zeros((V, 3))
    for _ in range(3):
        kx, kz = rng.integers(1, 4, 2)
        ph = rng.uniform(0, 2 * np.pi)
        a = rng.normal(0, 0.3, 3)
        W += amp * a[None, :] * np.sin(2 * np.pi * (kx * x[:, 0:1] + kz * x[:, 2:3]) + ph)
    return _cloth_scene(g, alpha, dt=1.0 / 60.0, steps=steps, iters=iters,
                        collider_flags=COLLIDE_SPHERE, sphere=tuple(float(v) for v in f32(np.r_[centre, radius])),
                        contact_compliance=1e-8, f_global=f32(f_global), f_vertex=f32(W),
                        name=f"sphere_cloth_{n}")


# ----------------------------------------------------------------------------------------
# tetrahedral block
# ----------------------------------------------------------------------------------------

# 5-tet corner-cut split of a unit cube; corners numbered by bits (x=1, y=2, z=4).
_EVEN_TETS = ((0, 1, 2, 4), (3, 1, 2, 7), (5, 1, 4, 7), (6, 2, 4, 7), (1, 2, 4, 7))
_ODD_TETS = ((1, 0, 3, 5), (2, 0, 3, 6), (4, 0, 5, 6), (7, 3, 5, 6), (0, 3, 5, 6))


def tet_block(n: int = 32, *, size: float = 1.0, density: float = 1000.0, y0: float = 0.05,
              steps: int = 120, iters: int = 20, seed: int = 3, plane_h: float = 0.0,
              alpha_lo: float = 1e-6, alpha_hi: float = 1e-3) -> Scene:
    """n^3 cube cells split into 5 tets each (mirrored parity so faces conform), falling on
    a ground plane.  Per tet, two inverse moduli are drawn log-uniform in [alpha_lo,
    alpha_hi]; the smaller is the hydrostatic one (1/lambda) and the larger the deviatoric
    one (1/mu), so lambda >= mu (Poisson ratio >= 1/4), and gamma = 1 + alpha_H / alpha_D
    in (1, 2] makes the rest state an equilibrium."""
    h = size / n
    N1 = n + 1
    I, J, K = np.meshgrid(np.arange(N1), np.arange(N1), np.arange(N1), indexing="ij")
    vid = lambda i, j, k: i + N1 * (j + N1 * k)
    x = np.zeros((N1 ** 3, 3))
    x[vid(I, J, K).ravel()] = np.stack([I.ravel() * h, y0 + J.ravel() * h, K.ravel() * h], 1)
    ci, cj, ck = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    ci, cj, ck = ci.ravel(), cj.ravel(), ck.ravel()
    corner = np.stack([vid(ci + (b & 1), cj + ((b >> 1) & 1), ck + ((b >> 2) & 1)) for b in range(8)], 1)
    odd = ((ci + cj + ck) % 2) == 1
    tets_by_slot = []
    for s in range(5):
        t = np.where(odd[:, None], corner[:, list(_ODD_TETS[s])], corner[:, list(_EVEN_TETS[s])])
        tets_by_slot.append(t)
    tets = np.stack(tets_by_slot, axis=1)          # [cells, 5, 4]
    # orient positively (mesh construction: swap two vertices where the signed volume < 0)
    P = x[tets]
    vol6 = np.einsum("...i,...i->...", np.cross(P[..., 1, :] - P[..., 0, :], P[..., 2, :] - P[..., 0, :]),
                     P[..., 3, :] - P[..., 0, :])
    neg = vol6 < 0
    tets[neg, 1], tets[neg, 2] = tets[neg, 2].copy(), tets[neg, 1].copy()
    vol = np.abs(vol6) / 6.0
    # lumped mass
    mass = np.zeros(N1 ** 3)
    np.add.at(mass, tets.reshape(-1, 4), np.repeat((density * vol.reshape(-1) / 4.0)[:, None], 4, 1))
    # coloring: cell parity class (8) x tet slot (5); hydrostatic then deviatoric per class
    cls = (ci % 2) + 2 * (cj % 2) + 4 * (ck % 2)
    tet_idx = tets.reshape(-1, 4).astype(np.int32)
    nt = tet_idx.shape[0]
    tet_id = np.arange(nt).reshape(-1, 5)
    offsets = [0]
    order = []
    for c in range(8):
        cells = np.nonzero(cls == c)[0]
        for s in range(5):
            ids = tet_id[cells, s]
            order.append(ids)            # hydrostatic constraint ids = tet id
            offsets.append(offsets[-1] + ids.shape[0])
            order.append(ids + nt)       # deviatoric constraint ids = nt + tet id
            offsets.append(offsets[-1] + ids.shape[0])
    rng = np.random.default_rng(seed)
    la, lb = np.log(alpha_lo), np.log(alpha_hi)
    a1 = np.exp(rng.uniform(la, lb, nt))
    a2 = np.exp(rng.uniform(la, lb, nt))
    aH, aD = np.minimum(a1, a2), np.maximum(a1, a2)
    gamma = 1.0 + aH / aD
    V = N1 ** 3
    xr = f32(x)
    return Scene(rest_x=xr, inv_mass=f32(1.0 / mass), dist_idx=np.zeros((0, 2), np.int32),
                 bend_idx=np.zeros((0, 4), np.int32), tet_idx=tet_idx, tet_gamma=f32(gamma),
                 color_offsets=np.asarray(offsets, np.int32),
                 color_order=np.concatenate(order).astype(np.int32), x0=xr.copy(),
                 v0=np.zeros((V, 3)), compliance=f32(np.concatenate([aH, aD])),
                 dt=1.0 / 120.0, steps=steps, iters=iters, collider_flags=COLLIDE_PLANE,
                 plane_h=plane_h, contact_compliance=1e-8, name=f"tet_block_{n}")


def couple_tets(scene: Scene) -> Scene:
    """The same scene with each tet's C_H and C_D projected together: the C_D ids
    (n_dist + n_bend + n_tet ...) leave the coloring, colors left empty are dropped, and
    every C_H id stands for its tet's pair."""
    first_d = scene.n_dist + scene.n_bend + scene.n_tet
    order = np.asarray(scene.color_order, np.int64)
    offs = np.asarray(scene.color_offsets, np.int64)
    new_order, new_offs = [], [0]
    for c in range(scene.n_colors):
        ids = order[offs[c]:offs[c + 1]]
        ids = ids[ids < first_d]
        if ids.shape[0]:
            new_order.append(ids)
            new_offs.append(new_offs[-1] + ids.shape[0])
    return scene.with_(tet_coupled=True, color_offsets=np.asarray(new_offs, np.int32),
                       color_order=(np.concatenate(new_order).astype(np.int32) if new_order
                                    else np.zeros(0, np.int32)))


# ----------------------------------------------------------------------------------------
# serving stream
# ----------------------------------------------------------------------------------------

def serving_requests(n_requests: int = 2000, *, seed: int = 5, side_lo: int = 32,
                     side_hi: int = 512, steps_lo: int = 20, steps_hi: int = 200,
                     iters_lo: int = 10, iters_hi: int = 40) -> list:
    """Parameters of a seeded request trace: per request the cloth side, horizon,
    iteration count, pins, ground plane and the seed of its compliance draw."""
    rng = np.random.default_rng(seed)
    out = []
    for r in range(n_requests):
        side = int(rng.integers(side_lo, side_hi + 1))
        npins = int(rng.integers(0, 5))
        pins = tuple((int(p), 0) for p in rng.choice(side, size=npins, replace=False))
        out.append(dict(side=side, steps=int(rng.integers(steps_lo, steps_hi + 1)),
                        iters=int(rng.integers(iters_lo, iters_hi + 1)), pins=pins,
                        ground=bool(rng.integers(0, 2)), seed=int(rng.integers(0, 2 ** 31))))
    return out


def request_scene(req: dict) -> Scene:
    """The cloth scene of one serving request (ground-plane cloth law with its own pins)."""
    n = req["side"]
    g = cloth_grid(n, 1.0, areal_density=2.56, diagonals="one", bending=True, pins=req["pins"])
    rng = np.random.default_rng(req["seed"])
    alpha = lognormal_cloth_compliance(rng, g["dist_idx"].shape[0], g["bend_idx"].shape[0])
    return _cloth_scene(g, alpha, dt=1.0 / 60.0, steps=req["steps"], iters=req["iters"],
                        collider_flags=COLLIDE_PLANE if req["ground"] else 0, plane_h=-0.6,
                        contact_compliance=1e-8, name=f"request_{n}")


def perturbed_target_compliance(scene: Scene, seed: int, sigma: float = 0.5) -> np.ndarray:
    """Per-constraint compliance multiplied by exp(sigma z), z ~ N(0,1): the seeded
    'ground truth' material used to make target trajectories."""
    rng = np.random.default_rng(seed)
    return f32(scene.compliance * np.exp(sigma * rng.standard_normal(scene.m)))


def tet_materials(n_tet: int, n_materials: int, *, seed: int = 7, mu=(1e3, 1e6), lam_over_mu=(1.0, 4.0)):
    """Materials randomly distributed over the tets (the paper's volumetric example uses 100
    over all tets): returns (tet_material [n_tet] int32, a [n_materials], b [n_materials])
    with mu = a^2 log-uniform in `mu` and lambda = b^2 = mu * U(lam_over_mu) (lambda >= mu, the
    same ordering as tet_block's moduli)."""
    rng = np.random.default_rng(seed)
    mat = rng.integers(0, n_materials, n_tet).astype(np.int32)
    mu_k = np.exp(rng.uniform(np.log(mu[0]), np.log(mu[1]), n_materials))
    lam_k = mu_k * rng.uniform(lam_over_mu[0], lam_over_mu[1], n_materials)
    return mat, f32(np.sqrt(mu_k)), f32(np.sqrt(lam_k))
