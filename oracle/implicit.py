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

A membrane (three rows E_uu, E_vv, 2 E_uv with a 3x3 compliance block alpha~_t) enters
as one block: B_t = G_t^T alpha~_t^-1 G_t - sum_k lambda_k hess C_k, and its reverse
step gives the matrix alphabar~_t += -(alpha~_t^-1 G_t y) lambda_t^T, then dL/dK through
alpha~_t = (A K)^-1 / dt^2.

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


def _memb_rest(scene):
    """Per membrane: Dm^-1 (2x2) of its (u, v) rest coordinates and its rest area."""
    out = []
    for t in range(scene.n_memb):
        uv = np.asarray(scene.memb_uv[t], np.float64)
        Dm = np.stack([uv[1] - uv[0], uv[2] - uv[0]], axis=1)
        out.append((np.linalg.inv(Dm), abs(np.linalg.det(Dm)) / 2.0))
    return out


def _memb_alpha(K, area, dt):
    """alpha~ = (A K)^-1 / dt^2, K = [C00 C01 0; C01 C11 0; 0 0 C22]."""
    c00, c11, c01, c22 = (float(v) for v in K)
    Km = np.array([[c00, c01, 0.0], [c01, c11, 0.0], [0.0, 0.0, c22]])
    return np.linalg.inv(area * Km) / (dt * dt)


def _memb_alphas(scene, stiffness, dt):
    K = np.asarray(scene.memb_stiffness if stiffness is None else stiffness, np.float64).reshape(-1, 4)
    return [_memb_alpha(K[t], area, dt) for t, (_, area) in enumerate(_memb_rest(scene))]


def _memb_alpha_grad(scene, abar_m, stiffness, dt):
    """dL/d(C00, C11, C01, C22) per membrane from the matrices alphabar~_t: with
    M = A K, d alpha~ = -M^-1 (A dK) M^-1 / dt^2 for each parameter's dK."""
    K = np.asarray(scene.memb_stiffness if stiffness is None else stiffness, np.float64).reshape(-1, 4)
    out = np.zeros((scene.n_memb, 4))
    units = [np.diag([1.0, 0.0, 0.0]), np.diag([0.0, 1.0, 0.0]),
             np.array([[0.0, 1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 0.0]]), np.diag([0.0, 0.0, 1.0])]
    for t, (_, area) in enumerate(_memb_rest(scene)):
        c00, c11, c01, c22 = K[t]
        Mi = np.linalg.inv(area * np.array([[c00, c01, 0.0], [c01, c11, 0.0], [0.0, 0.0, c22]]))
        for k, dK in enumerate(units):
            da = -Mi @ (area * dK) @ Mi / (dt * dt)
            out[t, k] = float(np.sum(abar_m[t] * da))
    return out


def _memb_rows(q, B2):
    """The three rows' gradients G [3, 9] and Hessians [3, 9, 9] at q (by the oracle's AD)."""
    r = np.zeros(12)
    r[2:6] = np.asarray(B2, np.float64).reshape(-1)
    G = np.zeros((3, 9))
    H = np.zeros((3, 9, 9))
    for k in range(3):
        G[k] = oracle.constraint(6 + k, q, r)[1]
        for c in range(9):
            u = np.zeros(9)
            u[c] = 1.0
            H[k][:, c] = oracle.constraint(6 + k, q, r, u)[2]
        H[k] = 0.5 * (H[k] + H[k].T)
    return G, H


def _psd_rel(B, nv):
    """Positive semi-definite part of B taken in relative coordinates (drop the first
    vertex: B = T^T B_rel T), negative eigenvalues of B_rel clamped to 0."""
    Br = B[3:, 3:]
    w, U = np.linalg.eigh(Br)
    Br = (U * np.maximum(w, 0.0)) @ U.T
    k = nv // 3
    T = np.zeros((nv - 3, nv))
    for a in range(1, k):
        T[3 * (a - 1):3 * a, 3 * a:3 * a + 3] = np.eye(3)
        T[3 * (a - 1):3 * a, 0:3] = -np.eye(3)
    return T.T @ Br @ T


def _memb_block(q, B2, lam3, at3, pd):
    """A membrane's block: (G [3, 9], B = G^T alpha~^-1 G - sum_k lambda_k hess C_k)."""
    G, H = _memb_rows(q, B2)
    B = G.T @ np.linalg.inv(at3) @ G - np.einsum("k,kij->ij", np.asarray(lam3, np.float64), H)
    B = 0.5 * (B + B.T)
    if pd:
        B = _psd_rel(B, 9)
    return G, B


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
            B = _psd_rel(B, nv)
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


def assemble(scene, x, lam, lamc, active, at, pd: bool, lam_m=None, at_m=None):
    """A = M + sum_j B_j over the constraints, membranes and active contacts at positions
    x [V,3]; returns (A [3V,3V], list of (vertex ids, grad) per constraint id or None,
    list of (vertex ids, G [3, 9]) per membrane)."""
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
    mgrads = []
    for t, (B2, _) in enumerate(_memb_rest(scene)):
        vs = scene.memb_idx[t]
        G, B = _memb_block(x[vs].reshape(-1), B2, lam_m[t], at_m[t], pd)
        idx = np.concatenate([np.arange(3 * v, 3 * v + 3) for v in vs])
        A[np.ix_(idx, idx)] += B
        mgrads.append((vs, G))
    return A, grads, mgrads


def _rows(scene, x, lam, lam_m, at, at_m):
    """Every constraint row at positions x [3V]: the scalar constraints, then each
    membrane's three rows.  Returns (C [R], G [R, 3V], sum of lambda-weighted Hessians
    [3V, 3V], block-diagonal alpha~ [R, R], kept rows [R] bool)."""
    V, m, nm = scene.V, scene.m, scene.n_memb
    R = m + 3 * nm
    Cv, G, Hs = np.zeros(R), np.zeros((R, 3 * V)), np.zeros((3 * V, 3 * V))
    Ab, keep = np.zeros((R, R)), np.zeros(R, bool)
    X = x.reshape(V, 3)
    for j, (kind, vs, r) in enumerate(_constraint_table(scene)):
        q = X[vs].reshape(-1)
        if _degenerate(kind, q) or at[j] <= 0:
            continue
        keep[j] = True
        n_in = oracle.N_INPUTS[kind]
        nv = 3 * len(vs)
        Cv[j], g, _ = oracle.constraint(kind, q, r)
        idx = np.concatenate([np.arange(3 * u, 3 * u + 3) for u in vs])
        G[j, idx] = g[:nv]
        for c in range(nv):
            e = np.zeros(n_in)
            e[c] = 1.0
            Hs[idx, idx[c]] += lam[j] * oracle.constraint(kind, q, r, e)[2][:nv]
        Ab[j, j] = at[j]
    for t, (B2, _) in enumerate(_memb_rest(scene)):
        vs = scene.memb_idx[t]
        q = X[vs].reshape(-1)
        rr = np.zeros(12)
        rr[2:6] = B2.reshape(-1)
        Gm, Hm = _memb_rows(q, B2)
        idx = np.concatenate([np.arange(3 * u, 3 * u + 3) for u in vs])
        rows = m + 3 * t + np.arange(3)
        for k in range(3):
            Cv[rows[k]] = oracle.constraint(6 + k, q, rr)[0]
            G[rows[k], idx] = Gm[k]
            Hs[np.ix_(idx, idx)] += lam_m[t][k] * Hm[k]
        Ab[np.ix_(rows, rows)] = at_m[t]
        keep[rows] = True
    return Cv, G, Hs, Ab, keep


def kkt_forward(scene, steps: Optional[int] = None, *, compliance=None, x0=None, v0=None, newton: int = 30,
                memb_stiffness=None):
    """Each step solved exactly instead of by XPBD iterations: Newton's method on
    M (x - p) - grad C^T lambda = 0, C + alpha~ lambda = 0 (no colliders; constraints and
    membrane rows as given).  XPBD drives only the second equation to zero; this forward is
    the step map whose exact derivative the implicit adjoint computes.  Returns (xs, vs,
    lam, lam_c, active, lam_m) like oracle.forward_multipliers plus the membranes'
    multipliers [steps, n_memb, 3]."""
    if scene.collider_flags:
        raise ValueError("the exact forward takes no colliders")
    steps = scene.steps if steps is None else steps
    dt = scene.dt
    V, m, nm = scene.V, scene.m, scene.n_memb
    w = np.asarray(scene.inv_mass, np.float64)
    free = np.repeat(w > 0, 3)
    mass = np.repeat(np.where(w > 0, 1.0 / np.where(w > 0, w, 1.0), 0.0), 3)
    comp = scene.compliance if compliance is None else compliance
    at = _alpha_tilde(scene, comp, dt)
    at_m = _memb_alphas(scene, memb_stiffness, dt)
    g_acc = np.asarray(scene.gravity, np.float64)
    x = np.asarray(scene.x0 if x0 is None else x0, np.float64).reshape(-1).copy()
    v = np.asarray(scene.v0 if v0 is None else v0, np.float64).reshape(-1).copy()
    xs, vs, lams, lams_m = [x.reshape(V, 3).copy()], [v.reshape(V, 3).copy()], [], []
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
        xn, lam = p.copy(), np.zeros(m + 3 * nm)
        for _ in range(newton):
            Cv, G, Hs, Ab, _ = _rows(scene, xn, lam[:m], lam[m:].reshape(nm, 3), at, at_m)
            H = np.diag(mass) - Hs
            r1 = mass * (xn - p) - G.T @ lam
            r2 = Cv + Ab @ lam
            nf = int(free.sum())
            R = m + 3 * nm
            K = np.zeros((nf + R, nf + R))
            K[:nf, :nf] = H[np.ix_(free, free)]
            K[:nf, nf:] = -G[:, free].T
            K[nf:, :nf] = G[:, free]
            K[nf:, nf:] = Ab
            d = np.linalg.solve(K, -np.r_[r1[free], r2])
            xn[free] += d[:nf]
            lam += d[nf:]
            if np.abs(d).max() < 1e-14:
                break
        v = (xn - x) / dt
        x = xn
        xs.append(x.reshape(V, 3).copy())
        vs.append(v.reshape(V, 3).copy())
        lams.append(lam[:m].copy())
        lams_m.append(lam[m:].reshape(nm, 3).copy())
    return (np.array(xs), np.array(vs), np.array(lams), np.zeros((steps, V, 2)),
            np.zeros((steps, V, 2), bool), np.array(lams_m).reshape(steps, nm, 3))


def adjoint(scene, seeds: dict, steps: Optional[int] = None, iters: Optional[int] = None, *, pd: bool = True,
            seed_dv_T=None, kkt: bool = False, trajectory=None) -> dict:
    """Implicit-adjoint gradients: compliance [m], x0, v0 [V,3], f_global [steps,3],
    f_vertex [V,3], f_vertex_steps [steps,V,3], memb_stiffness [n_memb,4].  The
    linearisation points are the XPBD forward's end-of-step states and multipliers, or
    `trajectory` (as returned by kkt_forward).  `kkt` solves each step's augmented system
    [[M - sum lambda hess C, grad C^T], [-grad C, alpha~]] instead of the Schur form (a
    cross-check; contacts and PD projection are then not allowed)."""
    steps = scene.steps if steps is None else steps
    iters = scene.iters if iters is None else iters
    dt = scene.dt
    if trajectory is None:
        xs, vs, lam, lamc, act = oracle.forward_multipliers(scene, steps, iters)
        lam_m = (oracle.forward_memb_multipliers(scene, steps, iters) if scene.n_memb
                 else np.zeros((steps, 0, 3)))
    else:
        xs, vs, lam, lamc, act = trajectory[:5]
        lam_m = trajectory[5] if len(trajectory) > 5 else np.zeros((steps, 0, 3))
    at = _alpha_tilde(scene, scene.compliance, dt)
    at_m = _memb_alphas(scene, None, dt)
    V, m, nm = scene.V, scene.m, scene.n_memb
    w = np.asarray(scene.inv_mass, np.float64)
    free = np.repeat(w > 0, 3)
    xbar = np.zeros(3 * V)
    vbar = np.zeros(3 * V) if seed_dv_T is None else np.asarray(seed_dv_T, np.float64).reshape(-1).copy()
    if steps in seeds:
        xbar += np.asarray(seeds[steps], np.float64).reshape(-1)
    abar = np.zeros(m)
    abar_m = np.zeros((nm, 3, 3))
    fvs = np.zeros((steps, V, 3))
    for n in range(steps - 1, -1, -1):
        tot = xbar + vbar / dt
        if kkt:
            if act[n].any() or pd:
                raise ValueError("the KKT cross-check takes no contacts and no projection")
            y, abar_n, abar_mn = _kkt_step(scene, xs[n + 1], lam[n], lam_m[n], at, at_m, tot, free)
        else:
            A, grads, mgrads = assemble(scene, xs[n + 1], lam[n], lamc[n], act[n], at, pd, lam_m[n], at_m)
            y = np.zeros(3 * V)
            y[free] = np.linalg.solve(A[np.ix_(free, free)], tot[free])
            abar_n = np.zeros(m)
            for j, gv in enumerate(grads):
                if gv is None:
                    continue
                vs_j, g = gv
                abar_n[j] = -(lam[n][j] / at[j]) * float(g @ y.reshape(V, 3)[vs_j].reshape(-1))
            abar_mn = np.zeros((nm, 3, 3))
            for t, (vs_t, G) in enumerate(mgrads):
                z = np.linalg.solve(at_m[t], G @ y.reshape(V, 3)[vs_t].reshape(-1))
                abar_mn[t] = -np.outer(z, lam_m[n][t])
        if kkt:
            A, _, _ = assemble(scene, xs[n + 1], lam[n], lamc[n], act[n], at, False, lam_m[n], at_m)
        mass = np.repeat(np.where(w > 0, 1.0 / np.where(w > 0, w, 1.0), 0.0), 3)
        pbar = np.where(free, mass * y, tot - A @ y)
        abar += abar_n
        abar_m += abar_mn
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
                f_global=fvs.sum(1), f_vertex=fvs.sum(0), f_vertex_steps=fvs,
                memb_stiffness=_memb_alpha_grad(scene, abar_m, None, dt))


def _kkt_step(scene, x, lam, lam_m, at, at_m, tot, free):
    """Transposed augmented system of one step, solved densely: returns (y, alphabar~ of
    the scalar constraints, alphabar~ matrices of the membranes)."""
    V, m, nm = scene.V, scene.m, scene.n_memb
    w = np.asarray(scene.inv_mass, np.float64)
    Cv, G, Hs, Ab, keep = _rows(scene, np.asarray(x, np.float64).reshape(-1), lam, lam_m, at, at_m)
    Hm = np.diag(np.repeat(np.where(w > 0, 1.0 / np.where(w > 0, w, 1.0), 0.0), 3)) - Hs
    Gf = G[keep][:, free]
    nf, mk = Gf.shape[1], Gf.shape[0]
    K = np.zeros((nf + mk, nf + mk))
    K[:nf, :nf] = 0.5 * (Hm[np.ix_(free, free)] + Hm[np.ix_(free, free)].T)
    K[:nf, nf:] = Gf.T
    K[nf:, :nf] = -Gf
    K[nf:, nf:] = Ab[np.ix_(keep, keep)]
    rhs = np.zeros(nf + mk)
    rhs[:nf] = tot[free]
    sol = np.linalg.solve(K, rhs)
    y = np.zeros(3 * V)
    y[free] = sol[:nf]
    mu = np.zeros(m + 3 * nm)
    mu[keep] = sol[nf:]
    abar = np.zeros(m)
    sk = keep[:m]
    abar[sk] = -lam[sk] * mu[:m][sk]
    abar_m = np.zeros((nm, 3, 3))
    for t in range(nm):
        abar_m[t] = -np.outer(mu[m + 3 * t:m + 3 * t + 3], lam_m[t])
    return y, abar, abar_m
