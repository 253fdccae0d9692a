"""Critical-field search of Sec. II.C with the FP64 oracle LLG (oracle; test
infrastructure).

Grid {0, sigma/2, ..., 4 sigma} of constant fields antiparallel (target bit)
or parallel (previous bit) to the head-field direction, then two refinements
that each evaluate the midpoint of the bracket between the last field with
the good outcome and the first with the bad one; H_crit is the last good field
(4 sigma if no bad outcome occurs; a bad outcome at zero field aborts with
BER = 1).  Each field value of each design is one oracle LLG run; the runs of
one level are integrated together as one oracle batch only because the
islands are independent.
"""
from __future__ import annotations

import numpy as np

from . import ber as oracle_ber
from .llg import Batch


def search(ops, islands, params, direction, sigma_T, role, head_map=None, levels=3):
    """Returns (h_crit_T [D], ber [D], aborted [D])."""
    sign = -1.0 if role == "targ" else 1.0
    D = len(islands)
    sigma_T = np.asarray(sigma_T, np.float64)
    direction = np.asarray(direction, np.float64)

    def good_outcomes(designs, mults):
        sub = islands.subset(np.asarray(designs))
        sub.Hext_T = np.array([sign * m * sigma_T[d] * direction[d] for d, m in zip(designs, mults)], np.float32)
        switched = Batch(ops, sub, params, head_map=head_map).run()["switched"]
        return switched if role == "targ" else ~switched

    grid = [0.5 * k for k in range(9)]
    g0 = good_outcomes([d for d in range(D) for _ in grid], grid * D).reshape(D, len(grid))
    lo = np.zeros(D)
    hi = np.full(D, np.inf)
    aborted = ~g0[:, 0]
    for d in range(D):
        if aborted[d]:
            continue
        bad = [k for k in range(len(grid)) if not g0[d, k]]
        if bad:
            lo[d], hi[d] = grid[bad[0] - 1], grid[bad[0]]
        else:
            lo[d] = 4.0
    for _ in range(levels - 1):
        act = [d for d in range(D) if not aborted[d] and np.isfinite(hi[d])]
        if not act:
            break
        mids = [0.5 * (lo[d] + hi[d]) for d in act]
        g = good_outcomes(act, mids)
        for d, mid, ok in zip(act, mids, g):
            if ok:
                lo[d] = mid
            else:
                hi[d] = mid
    h_crit = lo * sigma_T
    ber = np.array([1.0 if aborted[d] else oracle_ber.ber_from_hcrit(h_crit[d], sigma_T[d]) for d in range(D)])
    return h_crit, ber, aborted
