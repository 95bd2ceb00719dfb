"""The paper's implicit adjoint (Sec. "Adjoint State Computation", Eq. adjointXPBD;
Sec. "Positive Definite Projection"), written plainly for small meshes.  Test
infrastructure: only the tests, the smoke check and the bench's CPU leg use it.

Reading (derived here in reverse mode; the paper's index form is not transcribed).  Step n
ends at x_{n+1} with multipliers lambda; at convergence x_{n+1} = p_n + M^-1 grad C^T lambda
and C + alpha~ lambda = 0.  Linearising both and eliminating d lambda:

    A dx_{n+1} = M dp_n - sum_j grad C_j^T (lambda_j / alpha~_j) d alpha~_j,
    A = M + sum_j B_j,   B_j = grad C_j^T grad C_j / alpha~_j - lambda_j hess C_j,

(active contacts are constraints with the contact compliance).  With `pd`, every block
B_j is replaced by its positive semi-definite projection, taken in the constraint's
relative coordinates (the positions of its vertices relative to one of them: every
constraint is translation invariant, so B_j = T^T B_rel T) by clamping negative
eigenvalues to 0.  The reverse step, given the adjoint xbar of x_{n+1} (with the
velocity adjoint folded in as vbar/dt), solves A y = xbar on the free vertices (pinned
vertices are filtered out of the system, Sec. "Linear System Filtering"), then
pbar = M y on free vertices, pbar = xbar - (A y) on pinned ones, and
alphabar~_j += -(lambda_j / alpha~_j) grad C_j . y.  The rest of the sweep (prediction,
velocity, forces, seeds) is the discrete adjoint's.

Dense 3V x 3V matrices and a direct solve: a few hundred vertices at most.
Collider-parameter gradients are not formed."""
from typing import Optional

import numpy as np

import oracle


def _constraint_table(scene):
    """(kind, vertex ids, rest12) for every constraint id, in the oracle's order."""
    rest = oracle.rest_data(scene)
    nd, nb, nt = scene.n_dist, scene.n_bend, scene.n_tet
    out = []
    for j in range(scene.m):
        r = np.zeros(12)
        if j < nd:
            out.append((0, scene.dist_idx[j], np.r_[rest[j, 0], np.zeros(11)]))
        elif j < nd + nb:
            r[1] = rest[j, 1]
            out.append((1, scene.bend_idx[j - nd], r))
        else:
            t = (j - nd - nb) % nt
            r[2:11] = rest[j, 2:11]
            r[11] = scene.tet_gamma[t]
            out.append((2 if j < nd + nb + nt else 3, scene.tet_idx[t], r))
    return out


def _alpha_tilde(scene, compliance, dt):
    at = np.asarray(compliance, np.float64) / (dt * dt)
    if scene.n_tet:
        rest = oracle.rest_data(scene)
        k = scene.n_dist + scene.n_bend
        at[k:] = at[k:] / rest[k:, 11]
    return at


def _block(kind, q, rest12, lam, at, pd):
    """Value-free block data of one constraint at q: (grad [n], B [n x n]) over its vertex
    coordinates (collider parameters dropped), B projected when `pd`."""
    n = oracle.N_INPUTS[kind]
    nv = 3 * (2 if kind == 0 else 4 if kind in (1, 2, 3) else 1)
    C, g, _ = oracle.constraint(kind, q, rest12)
    H = np.zeros((nv, nv))
    for c in range(nv):
        u = np.zeros(n)
        u[c] = 1.0
        H[:, c] = oracle.constraint(kind, q, rest12, u)[2][:nv]
    g = g[:nv]
    H = 0.5 * (H + H.T)
    B = np.outer(g, g) / at - lam * H
    if pd:
        if kind in (4, 5):                      # one vertex: no translation null space
            w, U = np.linalg.eigh(B)
            B = (U * np.maximum(w, 0.0)) @ U.T
        else:                                   # relative coordinates: drop the first vertex
            Br = B[3:, 3:]
            w, U = np.linalg.eigh(Br)
            Br = (U * np.maximum(w, 0.0)) @ U.T
            k = nv // 3
            T = np.zeros((nv - 3, nv))
            for a in range(1, k):
                T[3 * (a - 1):3 * a, 3 * a:3 * a + 3] = np.eye(3)
                T[3 * (a - 1):3 * a, 0:3] = -np.eye(3)
            B = T.T @ Br @ T
    return g, B


def _degenerate(kind, q):
    if kind in (0, 5):
        return np.linalg.norm(q[0:3] - q[3:6]) < 1e-12
    if kind == 1:
        x = q.reshape(4, 3)
        e = x[1] - x[0]
        return (np.linalg.norm(e) < 1e-12 or np.linalg.norm(np.cross(e, x[2] - x[0])) < 1e-12
                or np.linalg.norm(np.cross(x[3] - x[0], e)) < 1e-12)
    return False


def assemble(scene, x, lam, lamc, active, at, pd: bool):
    """A = M + sum_j B_j over the constraints and active contacts at positions x [V,3];
    returns (A [3V,3V], list of (vertex ids, grad) per constraint id or None)."""
    V = scene.V
    m = np.where(scene.inv_mass > 0, 1.0 / np.where(scene.inv_mass > 0, scene.inv_mass, 1.0), 0.0)
    A = np.diag(np.repeat(m, 3))
    grads = []
    for j, (kind, vs, r) in enumerate(_constraint_table(scene)):
        q = x[vs].reshape(-1)
        if _degenerate(kind, q) or at[j] <= 0:
            grads.append(None)
            continue
        g, B = _block(kind, q, r, lam[j], at[j], pd)
        idx = np.concatenate([np.arange(3 * v, 3 * v + 3) for v in vs])
        A[np.ix_(idx, idx)] += B
        grads.append((vs, g))
    atc = scene.contact_compliance / scene.dt ** 2
    for i in range(V):
        for which in (0, 1):
            if not active[i, which]:
                continue
            kind = 4 if which == 0 else 5
            r = np.zeros(12)
            r[11] = scene.thickness
            q = np.r_[x[i], [scene.plane_h]] if which == 0 else np.r_[x[i], scene.sphere]
            if kind == 5 and _degenerate(5, q):
                continue
            g, B = _block(kind, q, r, lamc[i, which], atc, pd)
            A[3 * i:3 * i + 3, 3 * i:3 * i + 3] += B
    return A, grads


def kkt_forward(scene, steps: Optional[int] = None, *, compliance=None, x0=None, v0=None, newton: int = 30):
    """Each step solved exactly instead of by XPBD iterations: Newton's method on
    M (x - p) - grad C^T lambda = 0, C + alpha~ lambda = 0 (no colliders; constraints as
    given).  XPBD drives only the second equation to zero; this forward is the step map
    whose exact derivative the implicit adjoint computes.  Returns (xs, vs, lam, lam_c,
    active) like oracle.forward_multipliers."""
    if scene.collider_flags:
        raise ValueError("the exact forward takes no colliders")
    steps = scene.steps if steps is None else steps
    dt = scene.dt
    V, m = scene.V, scene.m
    w = np.asarray(scene.inv_mass, np.float64)
    free = np.repeat(w > 0, 3)
    mass = np.repeat(np.where(w > 0, 1.0 / np.where(w > 0, w, 1.0), 0.0), 3)
    comp = scene.compliance if compliance is None else compliance
    at = _alpha_tilde(scene, comp, dt)
    table = _constraint_table(scene)
    g_acc = np.asarray(scene.gravity, np.float64)
    x = np.asarray(scene.x0 if x0 is None else x0, np.float64).reshape(-1).copy()
    v = np.asarray(scene.v0 if v0 is None else v0, np.float64).reshape(-1).copy()
    xs, vs, lams = [x.reshape(V, 3).copy()], [v.reshape(V, 3).copy()], []
    for n in range(steps):
        f = np.zeros((V, 3))
        if scene.f_global is not None:
            f += np.asarray(scene.f_global, np.float64)[n]
        if scene.f_vertex is not None:
            f += np.asarray(scene.f_vertex, np.float64)
        if getattr(scene, "f_vertex_steps", None) is not None:
            f += np.asarray(scene.f_vertex_steps, np.float64)[n]
        acc = w[:, None] * f + (w[:, None] > 0) * g_acc
        p = x + dt * v + dt * dt * acc.reshape(-1)
        xn, lam = p.copy(), np.zeros(m)
        for _ in range(newton):
            H = np.diag(mass)
            G = np.zeros((m, 3 * V))
            Cv = np.zeros(m)
            for j, (kind, vs_j, r) in enumerate(table):
                q = xn.reshape(V, 3)[vs_j].reshape(-1)
                n_in = oracle.N_INPUTS[kind]
                nv = 3 * len(vs_j)
                Cv[j], g, _ = oracle.constraint(kind, q, r)
                idx = np.concatenate([np.arange(3 * u, 3 * u + 3) for u in vs_j])
                G[j, idx] = g[:nv]
                for c in range(nv):
                    e = np.zeros(n_in)
                    e[c] = 1.0
                    H[idx, idx[c]] -= lam[j] * oracle.constraint(kind, q, r, e)[2][:nv]
            r1 = mass * (xn - p) - G.T @ lam
            r2 = Cv + at * lam
            nf = int(free.sum())
            K = np.zeros((nf + m, nf + m))
            K[:nf, :nf] = H[np.ix_(free, free)]
            K[:nf, nf:] = -G[:, free].T
            K[nf:, :nf] = G[:, free]
            K[nf:, nf:] = np.diag(at)
            d = np.linalg.solve(K, -np.r_[r1[free], r2])
            xn[free] += d[:nf]
            lam += d[nf:]
            if np.abs(d).max() < 1e-14:
                break
        v = (xn - x) / dt
        x = xn
        xs.append(x.reshape(V, 3).copy())
        vs.append(v.reshape(V, 3).copy())
        lams.append(lam.copy())
    return (np.array(xs), np.array(vs), np.array(lams), np.zeros((steps, V, 2)),
            np.zeros((steps, V, 2), bool))


def adjoint(scene, seeds: dict, steps: Optional[int] = None, iters: Optional[int] = None, *, pd: bool = True,
            seed_dv_T=None, kkt: bool = False, trajectory=None) -> dict:
    """Implicit-adjoint gradients: compliance [m], x0, v0 [V,3], f_global [steps,3],
    f_vertex [V,3], f_vertex_steps [steps,V,3].  The linearisation points are the XPBD
    forward's end-of-step states and multipliers, or `trajectory` (as returned by
    kkt_forward).  `kkt` solves each step's augmented system
    [[M - sum lambda hess C, grad C^T], [-grad C, alpha~]] instead of the Schur form (a
    cross-check; contacts and PD projection are then not allowed)."""
    steps = scene.steps if steps is None else steps
    iters = scene.iters if iters is None else iters
    dt = scene.dt
    xs, vs, lam, lamc, act = trajectory if trajectory is not None else oracle.forward_multipliers(scene, steps, iters)
    at = _alpha_tilde(scene, scene.compliance, dt)
    V, m = scene.V, scene.m
    w = np.asarray(scene.inv_mass, np.float64)
    free = np.repeat(w > 0, 3)
    xbar = np.zeros(3 * V)
    vbar = np.zeros(3 * V) if seed_dv_T is None else np.asarray(seed_dv_T, np.float64).reshape(-1).copy()
    if steps in seeds:
        xbar += np.asarray(seeds[steps], np.float64).reshape(-1)
    abar = np.zeros(m)
    fvs = np.zeros((steps, V, 3))
    for n in range(steps - 1, -1, -1):
        tot = xbar + vbar / dt
        if kkt:
            if act[n].any() or pd:
                raise ValueError("the KKT cross-check takes no contacts and no projection")
            y, abar_n = _kkt_step(scene, xs[n + 1], lam[n], at, tot, free)
        else:
            A, grads = assemble(scene, xs[n + 1], lam[n], lamc[n], act[n], at, pd)
            y = np.zeros(3 * V)
            y[free] = np.linalg.solve(A[np.ix_(free, free)], tot[free])
            abar_n = np.zeros(m)
            for j, gv in enumerate(grads):
                if gv is None:
                    continue
                vs_j, g = gv
                abar_n[j] = -(lam[n][j] / at[j]) * float(g @ y.reshape(V, 3)[vs_j].reshape(-1))
        if kkt:
            A, _ = assemble(scene, xs[n + 1], lam[n], lamc[n], act[n], at, False)
        mass = np.repeat(np.where(w > 0, 1.0 / np.where(w > 0, w, 1.0), 0.0), 3)
        pbar = np.where(free, mass * y, tot - A @ y)
        abar += abar_n
        fb = (dt * dt) * np.repeat(w, 3) * pbar
        fvs[n] = fb.reshape(V, 3)
        xbar = pbar - vbar / dt
        vbar = dt * pbar
        if n in seeds:
            xbar = xbar + np.asarray(seeds[n], np.float64).reshape(-1)
    scale = np.full(m, 1.0 / (dt * dt))
    if scene.n_tet:
        k = scene.n_dist + scene.n_bend
        scale[k:] /= oracle.rest_data(scene)[k:, 11]
    return dict(compliance=abar * scale, x0=xbar.reshape(V, 3), v0=vbar.reshape(V, 3),
                f_global=fvs.sum(1), f_vertex=fvs.sum(0), f_vertex_steps=fvs)


def _kkt_step(scene, x, lam, at, tot, free):
    """Transposed augmented system of one step, solved densely: returns (y, alphabar~)."""
    V, m = scene.V, scene.m
    w = np.asarray(scene.inv_mass, np.float64)
    Hm = np.diag(np.repeat(np.where(w > 0, 1.0 / np.where(w > 0, w, 1.0), 0.0), 3))
    G = np.zeros((m, 3 * V))
    keep = np.zeros(m, bool)
    for j, (kind, vs, r) in enumerate(_constraint_table(scene)):
        q = x[vs].reshape(-1)
        if _degenerate(kind, q) or at[j] <= 0:
            continue
        keep[j] = True
        n = oracle.N_INPUTS[kind]
        nv = 3 * len(vs)
        _, g, _ = oracle.constraint(kind, q, r)
        idx = np.concatenate([np.arange(3 * v, 3 * v + 3) for v in vs])
        G[j, idx] = g[:nv]
        for c in range(nv):
            u = np.zeros(n)
            u[c] = 1.0
            Hm[idx, idx[c]] -= lam[j] * oracle.constraint(kind, q, r, u)[2][:nv]
    Gf = G[keep][:, free]
    nf, mk = Gf.shape[1], Gf.shape[0]
    K = np.zeros((nf + mk, nf + mk))
    K[:nf, :nf] = 0.5 * (Hm[np.ix_(free, free)] + Hm[np.ix_(free, free)].T)
    K[:nf, nf:] = Gf.T
    K[nf:, :nf] = -Gf
    K[nf:, nf:] = np.diag(at[keep])
    rhs = np.zeros(nf + mk)
    rhs[:nf] = tot[free]
    sol = np.linalg.solve(K, rhs)
    y = np.zeros(3 * V)
    y[free] = sol[:nf]
    abar = np.zeros(m)
    abar[keep] = -lam[keep] * sol[nf:]
    return y, abar
