"""Tet materials (Sec. "Volumetric Material Parameter Estimation"): mu_k = a_k^2,
lambda_k = b_k^2; a tet of material k has alpha_hat_D = 1/a_k^2 and alpha_hat_H = 1/b_k^2.
Test infrastructure: only the tests, the smoke check and the bench's CPU leg use it."""
import numpy as np


def compliance(scene, tet_material, a, b, base=None):
    """Per-constraint compliance (caller order) with the tet entries from the materials."""
    c = np.array(scene.compliance if base is None else base, np.float64)
    k = scene.n_dist + scene.n_bend
    nt = scene.n_tet
    mat = np.asarray(tet_material)
    c[k:k + nt] = 1.0 / np.asarray(b, np.float64)[mat] ** 2
    c[k + nt:k + 2 * nt] = 1.0 / np.asarray(a, np.float64)[mat] ** 2
    return c


def gradient(scene, d_compliance, tet_material, a, b):
    """dL/da, dL/db from dL/dcompliance: d(1/a^2)/da = -2/a^3, summed over each material."""
    k = scene.n_dist + scene.n_bend
    nt = scene.n_tet
    mat = np.asarray(tet_material)
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    gh = np.asarray(d_compliance, np.float64)[k:k + nt]
    gd = np.asarray(d_compliance, np.float64)[k + nt:k + 2 * nt]
    da = np.bincount(mat, weights=gd, minlength=len(a)) * (-2.0 / a ** 3)
    db = np.bincount(mat, weights=gh, minlength=len(b)) * (-2.0 / b ** 3)
    return da, db
