"""Host-side rules of the binding (no GPU): the integrator step count is the
smallest k with gamma/(1 + alpha^2) B dt / k <= 1/2 (the explicit-step bound
Heun's method needs on the precession frequency)."""
import math

import numpy as np

from paper_1603_09493_gb300 import api


def test_stable_substeps_is_the_smallest_admissible_count():
    gamma = 1.76085963023e-1                                 # rad / (ps T)
    rng = np.random.default_rng(0)
    for B, dt, alpha in zip(rng.uniform(0.01, 500.0, 200), rng.uniform(0.01, 1.0, 200), rng.uniform(0.0, 1.0, 200)):
        k = api.stable_substeps(B, dt, alpha)
        rate = gamma / (1.0 + alpha * alpha) * B * dt
        assert k >= 1 and rate / k <= 0.5 * (1 + 1e-12)
        assert k == 1 or rate / (k - 1) > 0.5
    # the census numbers: 28 steps per 0.1 ps at alpha 0.1 for a bound near 800 T (the exchange spectrum)
    assert api.stable_substeps(800.0, 0.1, 0.1) == 28
    assert api.stable_substeps(0.0, 0.1, 0.1) == 1
    assert api.stable_substeps(1.0, 0.1, 0.0, courant=0.25) == math.ceil(gamma * 0.1 / 0.25)
