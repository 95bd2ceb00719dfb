"""Conditioning of the parity workloads, measured on the FP64 oracle alone.

The stiff 16x16 cloth (compliance 1e-7, two pinned corners, 20 iterations) falling from a
flat start buckles: perturbations of the start state at FP32 rounding level (1e-7 m) grow
by more than 1e3 within 50 steps, so no FP32 computation can agree with FP64 to 1e-5 m over
that horizon.  Over its first 10 steps the growth stays below 10x, which is the horizon on
which positions and gradients are compared element by element."""
import numpy as np

import oracle
from paper_2301_01396_gb300 import scenes


def _amplification(sc, steps, eps=1e-7, seed=0):
    rng = np.random.default_rng(seed)
    xs, _ = oracle.forward(sc, steps)
    x0 = sc.x0 + eps * rng.standard_normal(sc.x0.shape) * (sc.inv_mass[:, None] > 0)
    xp, _ = oracle.forward(sc, steps, x0=x0)
    return float(np.abs(xp - xs).max() / eps)


def test_plain_cloth_long_horizon_is_ill_conditioned():
    sc = scenes.plain_cloth(16)
    assert _amplification(sc, 50) > 1e3


def test_plain_cloth_short_horizon_is_well_conditioned():
    sc = scenes.plain_cloth(16)
    assert _amplification(sc, 10) < 10.0
