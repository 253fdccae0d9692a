"""Model evaluation of one write-head / media design (Sec. II.A, the flow chart of
Fig. 4): the design's Table I parameters build the main pole and its trailing
shield, whose field is solved on the GPU (bpm_head_field_solve); the
critical-field searches of the target and the previous bit (Sec. II.C, Eqs.
1-2) run as batched LLG recording simulations under that field; a target that
cannot be written at H_ext = 0 aborts the evaluation with BER_tot = 1;
otherwise the adjacent-track bit's energy barrier in the fringing field (NEB)
gives BER_adj (Eq. 3), and BER_tot = BER_targ + BER_prev + BER_adj.

Readings (where the paper gives no number):
* media (Sec. II.B): 12 nm dots, 12 nm bit height, down-track pitch 13.5 nm,
  cross-track pitch 11.7 nm, Js = 0.7 T in both phases, K1_soft = 0.2
  K1_hard, as printed; the soft phase on top, 6 nm thick (the paper puts the
  middle of the soft phase 9 nm below the ABS, 6 nm above the islands), then
  the 1 nm interlayer carrying A_ex,int (the hard phase's top slab) and 5 nm
  of hard phase; A = 10 pJ/m elsewhere; a 481-node mesh (37-node planes, 13
  planes);
* frame: island bottoms at z = 0, tops at 12 nm, the ABS 6 nm above them (the
  paper's head-media spacing), the soft under-layer 2 nm below the islands;
* the head moves along -x at 13.5 m/s (the pole's trailing edge is its +x
  side), and a write window lasts one bit period, 13.5 nm / 13.5 m/s = 1 ns
  (the paper's t_write), with the 0.1 ns field rise at its start; a bit is
  written as it crosses the trailing edge, and the down-track offset is the
  target's distance past the trailing edge (into the trailing gap) when the
  window ends and the current reverses; the previous bit lies one pitch
  further along and spends the window in the gap and under the shield; the
  cross-track offset shifts the head across the track;
* the adjacent-track bit sits one cross-track pitch away (at half a
  down-track pitch in the staggered layout; on the previously written side in
  the shingled one), with the head frozen where the bit is 2 nm past the
  trailing edge (the paper's position of the lowest barrier);
* the H_ext direction of the critical-field searches is the head field's at
  the trailing edge, under the track's centre, at the islands' mid-height;
* a rate above 1 (an Arrhenius rate with a vanishing barrier, or the sum of
  the three) is taken as 1, a probability;
* the shield is the wrap-around body of bpm_head_field_solve: trailing and side
  blocks at Table I's gaps, Table I's thickness as their height.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import _lib as L
from . import adjacent, hcrit, synth

MU0 = 4e-7 * math.pi

# Table I: free parameters, (lower bound, initial value, upper bound)
TABLE1 = {
    "trailing_shield_gap_nm": (5.0, 9.0, 20.0),
    "trailing_edge_angle_deg": (5.0, 20.0, 45.0),
    "side_shield_gap_nm": (5.0, 16.0, 20.0),
    "side_edge_angle_deg": (5.0, 15.0, 45.0),
    "pole_tip_width_nm": (5.0, 14.0, 20.0),
    "pole_tip_taper_angle_deg": (75.0, 75.0, 75.0),
    "shield_thickness_nm": (3.0, 10.0, 20.0),
    "K1_hard_MJ_m3": (0.5, 0.8, 1.2),
    "A_ex_int_pJ_m": (1.0, 2.0, 10.0),
    "down_track_offset_nm": (0.0, 6.8, 8.0),
    "cross_track_offset_nm": (-8.0, 0.0, 8.0),
}

# Sec. II.B media
DOWN_PITCH_NM, CROSS_PITCH_NM = 13.5, 11.7
DOT_NM, HEIGHT_NM, JS_MEDIA_T = 12.0, 12.0, 0.7
HEAD_SPACING_NM = 6.0
VELOCITY_M_S = 13.5
A_BULK = 10e-12
Z_ABS_NM = HEIGHT_NM + HEAD_SPACING_NM
Z_SUL_NM = -2.0
WINDOW_PS = DOWN_PITCH_NM / (VELOCITY_M_S * 1e-3)      # one bit period
ADJ_BEHIND_TRAILING_NM = 2.0


def initial_design() -> dict:
    """Table I's initial design."""
    return {k: v[1] for k, v in TABLE1.items()}


def pole_geometry(p: dict, panel_nm: float = 3.0) -> dict:
    """bpm_pole_geometry fields of a design (in the media frame above)."""
    return synth.pole_geometry(pole_tip_width_nm=p["pole_tip_width_nm"],
                               trailing_edge_angle_deg=p["trailing_edge_angle_deg"],
                               side_edge_angle_deg=p["side_edge_angle_deg"],
                               taper_angle_deg=p["pole_tip_taper_angle_deg"],
                               z_abs_nm=Z_ABS_NM, z_sul_nm=Z_SUL_NM, sul_image=1,
                               trailing_shield_gap_nm=p["trailing_shield_gap_nm"],
                               shield_thickness_nm=p["shield_thickness_nm"], shield_panel_nm=panel_nm,
                               side_shield_gap_nm=p["side_shield_gap_nm"])


def media(p: dict):
    """Island mesh and region table (hard, hard interface, soft) of a design."""
    mesh = synth.layered_island_mesh(DOT_NM, HEIGHT_NM / 2, HEIGHT_NM / 2, rings=3, hard_slabs=6, soft_slabs=6,
                                     seed=7)
    ms = JS_MEDIA_T / MU0
    k1 = p["K1_hard_MJ_m3"] * 1e6
    mats = synth.ecc_materials(Ms_hard=ms, Ku_hard=k1, A_hard=A_BULK, Ms_soft=ms, Ku_soft=0.2 * k1,
                               A_soft=A_BULK, interlayer_scale=p["A_ex_int_pJ_m"] * 1e-12 / A_BULK)
    return mesh, mats


def head_grid():
    """The head map's grid: (nx, ny, nz, h, origin) covering every position the bits take."""
    return 64, 64, 18, 1.0, (-30.0, -28.0, 0.0)


def bit_positions(p: dict, layout: str = "staggered") -> dict:
    """Media-frame positions (x, y) of the target, previous and adjacent bits; the cross-track
    offset moves the head, i.e. every bit by -offset in the head's frame."""
    dy = -p["cross_track_offset_nm"]
    adj = {"centered": (0.0, CROSS_PITCH_NM), "staggered": (DOWN_PITCH_NM / 2, CROSS_PITCH_NM),
           "shingled": (0.0, -CROSS_PITCH_NM)}[layout]
    return {"targ": (0.0, dy), "prev": (DOWN_PITCH_NM, dy), "adj": (adj[0], adj[1] + dy)}


def run_params(p: dict) -> synth.RunParams:
    """The write window: the head moves along -x for one bit period and leaves the target
    down_track_offset past its trailing edge (map x = +offset) when the window ends."""
    v = -VELOCITY_M_S
    x_end = -p["down_track_offset_nm"]                 # head position at the end: target at +offset
    x0 = x_end - v * 1e-3 * WINDOW_PS
    return synth.RunParams(dt_ps=0.1, t_end_ps=WINDOW_PS, alpha=0.1, rise_ps=100.0, v_m_per_s=v, x0_nm=x0,
                           use_map=True, substeps=0)


def field_direction(hm: synth.HeadMap, map_xyz) -> np.ndarray:
    """Unit head-field direction at the voxel nearest a map point (the H_ext direction of the
    critical-field search)."""
    nz, ny, nx = hm.B_T.shape[:3]
    i = np.rint((np.asarray(map_xyz, np.float64) - hm.origin_nm) / hm.h_nm).astype(int)
    i = np.clip(i, 0, [nx - 1, ny - 1, nz - 1])
    b = hm.B_T[i[2], i[1], i[0]].astype(np.float64)
    return b / np.linalg.norm(b)


def evaluate(ctx, p: dict, layout: str = "staggered", precision: int = L.PREC_BF16X3, panel_nm: float = 3.0,
             neb_images: int = 9, neb_iters: int = 1500) -> dict:
    """BER_targ, BER_prev, BER_adj and BER_tot of one design (Fig. 4), with what they came from."""
    t = {"start": time.perf_counter()}
    nx, ny, nz, h, org = head_grid()
    hm = ctx.head_field(pole_geometry(p, panel_nm), nx, ny, nz, h, org)
    hid = ctx.headmap_upload(hm)
    t["head"] = time.perf_counter()
    mesh, mats = media(p)
    mid = ctx.mesh_upload(mesh, mats)
    t["media"] = time.perf_counter()
    pos = bit_positions(p, layout)
    q = run_params(p)
    sigma = hcrit.sfd_sigma_T(p["K1_hard_MJ_m3"] * 1e6, JS_MEDIA_T)
    direction = field_direction(hm, (0.0, pos["targ"][1], HEIGHT_NM / 2))
    run = hcrit.gpu_flag_runner(ctx, q, q.n_intervals, map_id=hid, precision=precision)
    targ = hcrit.critical_field_search(run, synth.nominal_islands(1, mid, pos["targ"]), direction[None], [sigma],
                                       "targ")
    t["targ"] = time.perf_counter()
    out = {"layout": layout, "sigma_T": sigma, "direction": direction.tolist(),
           "h_crit_targ_sigma": float(targ.h_crit_T[0] / sigma), "ber_targ": float(targ.ber[0]),
           "aborted": bool(targ.aborted[0]), "llg_island_runs": int(targ.n_runs)}
    if targ.aborted[0]:
        out.update(ber_prev=None, ber_adj=None, ber_tot=1.0)
    else:
        prev = hcrit.critical_field_search(run, synth.nominal_islands(1, mid, pos["prev"]), direction[None],
                                           [sigma], "prev")
        t["prev"] = time.perf_counter()
        qa = synth.RunParams(dt_ps=0.1, rise_ps=0.0, use_map=True, v_m_per_s=0.0,
                             x0_nm=pos["adj"][0] - ADJ_BEHIND_TRAILING_NM)
        bar = adjacent.barriers(ctx, synth.nominal_islands(1, mid, pos["adj"]), qa, n_images=neb_images,
                                max_iters=neb_iters, climb_after=neb_iters // 5, precision=precision, map_id=hid)
        t["adj"] = time.perf_counter()
        out.update(h_crit_prev_sigma=float(prev.h_crit_T[0] / sigma), ber_prev=float(prev.ber[0]),
                   E_B_kT=float(bar["E_B_kT"][0]), ber_adj=min(1.0, float(bar["ber_adj"][0])),
                   llg_island_runs=int(targ.n_runs + prev.n_runs))
        out["ber_tot"] = min(1.0, float(adjacent.ber_tot(out["ber_targ"], out["ber_prev"], out["ber_adj"])))
    ctx.mesh_release(mid)              # a loop uploads one mesh and one map per design
    ctx.headmap_release(hid)
    stamps = list(t.items())
    out["seconds"] = {k: stamps[i][1] - stamps[i - 1][1] for i, (k, _) in enumerate(stamps) if i > 0}
    return out


def design_from_unit(u, keys, base=None) -> dict:
    """A design whose parameters `keys` take the unit-cube coordinates u within their Table I
    bounds, the rest their initial values (or base's)."""
    p = dict(base or initial_design())
    for k, x in zip(keys, np.asarray(u, np.float64)):
        lo, _, hi = TABLE1[k]
        p[k] = lo + (hi - lo) * float(x)
    return p


def optimise(ctx, keys, n_init: int, iters: int, seed: int = 0, layout: str = "staggered", log=None, **kw):
    """The optimisation loop of Sec. II.A on log10(BER_tot): a maximin Latin hypercube of n_init
    designs over the parameters `keys` (the rest at Table I's initial values), then `iters` EGO
    iterations (kriging, expected improvement), every design evaluated by `evaluate`; steps
    taken while all scores are equal are space-filling instead (see below)."""
    from . import ego
    d = len(keys)
    C = synth.lhs_candidates(64, n_init, d, seed=seed)
    j, _ = ego.lhs_maximin(ctx, C)
    X0 = C[j]
    evals = []

    def f(U):
        ys = []
        for u in np.atleast_2d(U):
            r = evaluate(ctx, design_from_unit(u, keys), layout=layout, **kw)
            r["unit"] = [float(x) for x in u]
            evals.append(r)
            if log:
                log(r)
            ys.append(math.log10(max(r["ber_tot"], 1e-300)))
        return np.array(ys)

    X, y = X0, f(X0)
    # while every design evaluated so far scores the same (typically BER_tot = 1: none writes its
    # target), a kriging model has nothing to fit; take the candidate farthest from the designs
    # evaluated (a space-filling step) until the scores differ, then hand over to EGO
    explore = 0
    while np.ptp(y) == 0 and explore < iters:
        C = synth.unit_points(2000, d, seed * 1000 + 7, explore)
        gap = np.min(np.linalg.norm(C[:, None] - X[None], axis=2), axis=1)
        u = C[int(np.argmax(gap))][None]
        X, y = np.concatenate([X, u]), np.concatenate([y, f(u)])
        explore += 1
    hist = []
    if np.ptp(y) > 0 and iters > explore:
        draws = lambda it: [synth.theta_unit_draws(32, d, seed * 1000 + 5 + it, r) for r in range(4)]
        cands = lambda it: (synth.unit_points(2000, d, seed * 1000 + 6, 2 * it),
                            synth.unit_points(2000, d, seed * 1000 + 6, 2 * it + 1))
        X, y, hist = ego.ego(ctx, f, X, y, iters - explore, draws, cands)
    best = int(np.argmin(y))
    return {"keys": list(keys), "X": X, "log10_ber_tot": y, "best": design_from_unit(X[best], keys),
            "best_log10_ber_tot": float(y[best]), "evaluations": evals, "space_filling_steps": explore,
            "max_ei": [float(e) for _, e in hist]}
