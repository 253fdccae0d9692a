"""Adjacent-track erasure rate (Sec. II.C, Eq. 3) from energy barriers computed
by the nudged elastic band on the GPU (bpm_neb_run).

The adjacent bit sits in the head's fringing field with the head frozen at the
down-track position of the lowest barrier (2 nm behind the trailing edge in
the paper); its switching barrier E_B gives the lifetime
tau = exp(E_B / kT) / f0 (f0 = 130 GHz, T = 300 K) and, for a field exposure
t_write = 1 ns per pass,

    BER_adj = t_write / tau = t_write f0 exp(-E_B / kT).

BER_tot = BER_targ + BER_prev + BER_adj.  This module builds the band runs and
evaluates Eq. (3); every band iteration runs in the library.
"""
from __future__ import annotations

import math

import numpy as np

from . import _lib as L
from . import api

KB = 1.380649e-23          # J/K


def ber_adj(E_B_J, T_K: float = 300.0, f0_Hz: float = 130e9, t_write_s: float = 1e-9):
    """Eq. (3): t_write f0 exp(-E_B / kT), elementwise."""
    E = np.asarray(E_B_J, np.float64)
    return t_write_s * f0_Hz * np.exp(-E / (KB * T_K))


def ber_tot(targ, prev, adj):
    return np.asarray(targ) + np.asarray(prev) + np.asarray(adj)


def stable_step(ctx, mesh_id: int, islands, params, map_id: int = -1, courant: float = 0.4) -> float:
    """Band step (m^3/MJ) with step * max(Ms_i) * |B|_max <= courant, the bound of the
    explicit update on the stiffest (exchange) mode; |B|_max is the library's field
    bound of the islands (bpm_stable_substeps)."""
    bound = ctx.stable_substeps(islands, params, map_id)[1]
    Ms = ctx.get_operator(mesh_id, L.OP_NODAL_MS_F64)
    ms_max = float(np.max(Ms)) * 1e-6 * float(np.max(np.asarray(islands.Ms_scale, np.float64)))
    return courant / (ms_max * bound)


def barriers(ctx, islands, params, n_images: int = 12, max_iters: int = 2000, climb_after: int = 400,
             spring: float = 1.0, step=None, precision: int = L.PREC_BF16X3, map_id: int = -1,
             force_tol: float = 0.0, T_K: float = 300.0) -> dict:
    """Energy barriers (J and kT) and BER_adj of every island in the fringing field
    of the head frozen at params.x0_nm (params.uniform_T and each island's
    Hext_T add a uniform field; params.term_mask selects the terms)."""
    mid = int(np.asarray(islands.mesh_id)[0])
    if step is None:
        step = stable_step(ctx, mid, islands, params, map_id)
    out = ctx.neb(islands, n_images, max_iters, step, spring, climb_after, precision=precision, map_id=map_id,
                  head_x_nm=params.x0_nm, uniform_T=params.uniform_T, term_mask=params.term_mask,
                  force_tol=force_tol)
    out["E_B_kT"] = out["E_B"] / (KB * T_K)
    out["ber_adj"] = ber_adj(out["E_B"], T_K)
    out["step"] = step
    return out


def barrier_kT_from_ber(ber: float, f0_Hz: float = 130e9, t_write_s: float = 1e-9) -> float:
    """Eq. (3) inverted: E_B / kT = ln(t_write f0 / BER_adj)."""
    return math.log(t_write_s * f0_Hz / ber)
