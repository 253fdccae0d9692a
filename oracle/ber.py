"""Bit-error-rate formulas of Sec. II.C, plain FP64 (oracle; test infrastructure).

* switching-field distribution: sigma = 0.015 H_A with H_A = 2 K1,hard / Js
  (in tesla: mu0 H_A = 2 K1 mu0 / Js);
* Eqs. (1)-(2): BER = 1/2 [1 - erf(H_crit / sqrt(2 sigma^2))];
* Eq. (3) with tau = exp(E_B / kT) / f0: BER_adj = t_write / tau;
* BER_tot = BER_targ + BER_prev + BER_adj.
"""
from __future__ import annotations

import math

MU0 = 4e-7 * math.pi


def sfd_sigma_T(K1_hard_J_m3: float, Js_T: float, frac: float = 0.015) -> float:
    return frac * 2.0 * K1_hard_J_m3 * MU0 / Js_T


def ber_from_hcrit(H_crit: float, sigma: float) -> float:
    return 0.5 * (1.0 - math.erf(H_crit / math.sqrt(2.0 * sigma * sigma)))


def ber_adj(E_B_kT: float, f0_Hz: float = 130e9, t_write_s: float = 1e-9) -> float:
    tau = math.exp(E_B_kT) / f0_Hz
    return t_write_s / tau


def ber_tot(targ: float, prev: float, adj: float) -> float:
    return targ + prev + adj
