"""Critical-field search and write bit-error rates (Sec. II.C, Eqs. 1-2), batched
over designs on the GPU path.

For every design the paper applies, besides the moving head field, a constant
field H_ext antiparallel (target bit) or parallel (previous bit) to the head
field, and searches the critical H_ext at which writing the target fails (or the
previous bit gets overwritten) on the grid {0, ..., 4 sigma} with an initial
step of sigma/2, refined twice; sigma = 0.015 H_A, H_A = 2 K1,hard / Js.  The
error rate is the Gaussian tail BER = 1/2 [1 - erf(H_crit / sqrt(2 sigma^2))].

Readings (the paper gives the grid and the number of refinements only):
* a refinement halves the step and evaluates the midpoint of the bracket
  [last field with the good outcome, first field with the bad one];
* H_crit is the last field with the good outcome after the refinements;
* no bad outcome up to 4 sigma: H_crit = 4 sigma (the paper always found the
  critical field inside the grid);
* a bad outcome already at H_ext = 0 aborts the design: BER = 1 (the early
  abort of Fig. 1);
* the H_ext direction is the unit head-field direction at the island centre
  under the pole (sign - for the target, + for the previous bit).

Every level of the search is one batch of islands (designs x grid points)
through the library; this module only builds the batches and reads flags.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import _lib as L
from .synth import Islands

MU0 = 4e-7 * math.pi


def sfd_sigma_T(K1_hard_J_m3: float, Js_T: float, frac: float = 0.015) -> float:
    """sigma = 0.015 mu0 H_A in tesla, mu0 H_A = 2 K1 mu0 / Js."""
    return frac * 2.0 * K1_hard_J_m3 * MU0 / Js_T


def ber_from_hcrit(h_crit_T: float, sigma_T: float) -> float:
    return 0.5 * math.erfc(h_crit_T / (math.sqrt(2.0) * sigma_T))


@dataclass
class SearchResult:
    h_crit_T: np.ndarray        # [D]
    ber: np.ndarray             # [D]
    aborted: np.ndarray         # [D] bad outcome at H_ext = 0
    n_runs: int                 # LLG island-runs spent


def _with_field(isl: Islands, idx, H: np.ndarray) -> Islands:
    sub = isl.subset(idx)
    sub.Hext_T = H.astype(np.float32)
    return sub


def critical_field_search(run_flags, islands: Islands, direction: np.ndarray, sigma_T: np.ndarray,
                          role: str, levels: int = 3, step: float = 0.5, top: float = 4.0) -> SearchResult:
    """run_flags(Islands, designs) -> switched flags [B] (one batch of LLG runs);
    designs [B] holds the design index of every island of the batch.

    islands: one island per design (its position is the bit's position);
    direction: [D][3] unit head-field direction; sigma_T: [D]; role 'targ'
    (H_ext antiparallel, good outcome = switched) or 'prev' (parallel, good
    outcome = not switched)."""
    D = len(islands)
    sign = -1.0 if role == "targ" else 1.0
    sigma_T = np.asarray(sigma_T, np.float64)
    direction = np.asarray(direction, np.float64)
    grid = np.arange(0.0, top + 1e-9, step)                 # multiples of sigma
    G = grid.size
    idx = np.repeat(np.arange(D), G)
    mult = np.tile(grid, D)
    H = sign * (mult * sigma_T[idx])[:, None] * direction[idx]
    sw = np.asarray(run_flags(_with_field(islands, idx, H), idx), bool).reshape(D, G)
    good = sw if role == "targ" else ~sw
    runs = D * G
    aborted = ~good[:, 0]
    lo = np.zeros(D)                                        # last good multiple
    hi = np.full(D, np.inf)                                 # first bad multiple
    for d in range(D):
        bad = np.where(~good[d])[0]
        if aborted[d]:
            continue
        if bad.size == 0:
            lo[d] = top
        else:
            first = bad[0]
            lo[d], hi[d] = grid[first - 1], grid[first]
    active = np.where(~aborted & np.isfinite(hi))[0]
    for _ in range(levels - 1):
        if active.size == 0:
            break
        mid = 0.5 * (lo[active] + hi[active])
        Hm = sign * (mid * sigma_T[active])[:, None] * direction[active]
        swm = np.asarray(run_flags(_with_field(islands, active, Hm), active), bool)
        gm = swm if role == "targ" else ~swm
        runs += active.size
        lo[active] = np.where(gm, mid, lo[active])
        hi[active] = np.where(gm, hi[active], mid)
    h = lo * sigma_T
    ber = np.array([1.0 if aborted[d] else ber_from_hcrit(h[d], sigma_T[d]) for d in range(D)])
    return SearchResult(h_crit_T=h, ber=ber, aborted=aborted, n_runs=runs)


def gpu_flag_runner(ctx, params, n_intervals: int, map_id: int = -1, precision: int = L.PREC_BF16X3):
    """run_flags for critical_field_search on the batched GPU path."""
    def run(isl: Islands, designs=None):
        return ctx.run_batch(isl, params, n_intervals, precision=precision, map_id=map_id)["switched"]
    return run
