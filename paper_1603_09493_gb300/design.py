"""The write-head and media design problem that the surrogate screens (Sec. II.A
optimisation loop; Sec. II.B and Table I free parameters; Fig. 3 track layouts).

A design is 12 parameters of island and head together:

  diameter, soft-layer thickness, hard-layer thickness, Ms scale, Ku scale,
  interlayer exchange scale (Table I row A_ex,int), bit pitch, track layout
  (centered, staggered, shingled), head peak field, head field tilt, head
  field width (the down-track gradient, peak / (width sqrt e)), head velocity.

Each realisation of a design carries 4 jitter values: the Ms and Ku factors, an
easy-axis tilt in the down-track plane and a down-track position offset.  The
surrogate sees the 16 numbers.  Its two labels are the error events of
Sec. II.C: the target island switches (it is written), and the adjacent-track
island of the layout flips in the head's fringing field.

Readings (the paper gives its own head and media parameters, not these ranges):
* geometry and exchange scale take the levels of a 3 x 3 x 3 x 3 grid (81
  meshes, coarse: two node rings per plane, 1 nm slabs), the velocity one of 4
  levels, the layout one of 3; the other parameters are continuous;
* every island's top sits at z = 16 nm of the head map, 5 nm below the
  air-bearing surface, whatever its thickness;
* a design's head field is the synthetic pole-tip field with its peak, tilt and
  width; up to 256 heads share one map, as a 16 x 16 array of 64 nm blocks
  along its down-track (x, head frame) and cross-track (y) axes, and an island
  samples its design's head through an offset of 64 nm times the head's block
  coordinates (islands and the moving head stay within 20 nm of their block's
  centre, so no lookup reaches a neighbouring block; with offsets below 1 um
  the FP32 lookup coordinate keeps a resolution of 6e-5 nm, a head-field error
  of about 1e-5 T);
* the pitch (9-14 nm) and field width (6-12 nm) ranges are wide enough that
  both error events occur among random designs;
* the head centre reaches the target at 100 ps (x0 = -v * 100 ps), the fields
  rise over 100 ps, the run lasts 250 ps;
* the adjacent island carries the realisation's Ms and Ku factors and tilt, at
  its layout's offset from the target: (0, +p) centered, (+p/2, +p) staggered,
  (0, -p) shingled (the previously written side).
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass

import numpy as np

from . import _lib as L
from . import evolve, synth

KEYS = ("diameter_nm", "t_soft_nm", "t_hard_nm", "Ms_scale", "Ku_scale", "A_int_scale", "pitch_nm", "layout",
        "B_peak_T", "tilt_deg", "width_nm", "v_m_per_s")
RANGES = dict(diameter_nm=(6.0, 10.0), t_soft_nm=(2.0, 4.0), t_hard_nm=(5.0, 9.0), Ms_scale=(0.85, 1.15),
              Ku_scale=(0.8, 1.2), A_int_scale=(0.1, 0.6), pitch_nm=(9.0, 14.0), layout=(0.0, 2.0),
              B_peak_T=(1.0, 1.6), tilt_deg=(10.0, 40.0), width_nm=(6.0, 12.0), v_m_per_s=(10.0, 30.0))
LEVELS = dict(diameter_nm=(6.0, 8.0, 10.0), t_soft_nm=(2.0, 3.0, 4.0), t_hard_nm=(5.0, 7.0, 9.0),
              A_int_scale=(0.1, 0.3, 0.6), layout=(0.0, 1.0, 2.0), v_m_per_s=(10.0, 50.0 / 3.0, 70.0 / 3.0, 30.0))
LAYOUTS = ("centered", "staggered", "shingled")
GEOMETRY_KEYS = ("diameter_nm", "t_soft_nm", "t_hard_nm", "A_int_scale")
HEAD_KEYS = ("B_peak_T", "tilt_deg", "width_nm")
JITTER = dict(Ms=0.05, Ku=0.05, tilt_deg=2.0, pos_nm=1.0)
T_END_PS = 250.0
Z_TOP_NM = 16.0
BLOCK_NM = 64
BLOCKS = 16                      # blocks per map axis
HEADS_PER_MAP = BLOCKS * BLOCKS


def values(Z) -> dict:
    """Unit-cube designs Z [N][12] -> parameter values [N] per key; the gridded
    parameters take the level of their equal-width cell."""
    Z = np.asarray(Z, np.float64)
    out = {}
    for k, key in enumerate(KEYS):
        if key in LEVELS:
            lev = np.asarray(LEVELS[key])
            out[key] = lev[np.minimum((Z[:, k] * len(lev)).astype(np.int64), len(lev) - 1)]
        else:
            lo, hi = RANGES[key]
            out[key] = lo + (hi - lo) * Z[:, k]
    return out


def geometry_index(v: dict) -> np.ndarray:
    """Index into the 81-mesh grid of each design's (diameter, t_soft, t_hard, A_int)."""
    idx = np.zeros(len(v["diameter_nm"]), np.int64)
    for key in GEOMETRY_KEYS:
        lev = np.asarray(LEVELS[key])
        idx = idx * len(lev) + np.argmin(np.abs(v[key][:, None] - lev[None, :]), axis=1)
    return idx


def grid_meshes():
    """The 81 (mesh, materials) pairs of the geometry grid, in geometry_index order."""
    out = []
    k = 0
    for d in LEVELS["diameter_nm"]:
        for ts in LEVELS["t_soft_nm"]:
            for th in LEVELS["t_hard_nm"]:
                for a in LEVELS["A_int_scale"]:
                    m = synth.layered_island_mesh(d, th, ts, rings=2, hard_slabs=int(th), soft_slabs=int(ts),
                                                  seed=700 + k)
                    m.xyz_nm = m.xyz_nm.copy()
                    m.xyz_nm[:, 2] += Z_TOP_NM - m.height_nm        # top 5 nm below the air-bearing surface
                    out.append((m, synth.ecc_materials(interlayer_scale=a)))
                    k += 1
    return out


def upload_grid(ctx) -> list:
    return [ctx.mesh_upload(m, mats) for m, mats in grid_meshes()]


def head_block(h) -> tuple:
    """Block coordinates (down-track, cross-track) of head h within its map."""
    h = np.asarray(h) % HEADS_PER_MAP
    return h // BLOCKS, h % BLOCKS


def head_stack(heads) -> synth.HeadMap:
    """One map holding the heads [H][3] (peak T, tilt deg, width nm): head h is
    the synthetic pole-tip map of that head (18 planes, island top at z = 16 nm)
    in the block spanning x in [64 bx - 32, 64 bx + 32), y in [64 by - 32,
    64 by + 32) nm, (bx, by) = head_block(h)."""
    heads = np.asarray(heads, np.float64)
    H = len(heads)
    if not 1 <= H <= HEADS_PER_MAP:
        raise ValueError(f"1..{HEADS_PER_MAP} heads per map")
    nby, nbx = min(H, BLOCKS), (H + BLOCKS - 1) // BLOCKS
    blocks = [synth.synthetic_head_map(nx=BLOCK_NM, ny=BLOCK_NM, nz=18, B_peak_T=float(b), tilt_deg=float(t),
                                       sx_nm=float(w), sy_nm=float(w), z_top_nm=Z_TOP_NM) for b, t, w in heads]
    nz = blocks[0].B_T.shape[0]
    B = np.zeros((nz, nby * BLOCK_NM, nbx * BLOCK_NM, 3), np.float32)
    for h, blk in enumerate(blocks):
        bx, by = head_block(h)
        B[:, by * BLOCK_NM:(by + 1) * BLOCK_NM, bx * BLOCK_NM:(bx + 1) * BLOCK_NM] = blk.B_T
    return synth.HeadMap(B_T=B, origin_nm=blocks[0].origin_nm.copy(), h_nm=blocks[0].h_nm,
                         info=dict(heads=heads.tolist(), block_nm=BLOCK_NM))


@dataclass
class Realisations:
    """Design-major realisations of designs: rows d * J .. d * J + J - 1 belong to design d."""
    v: dict                 # parameter values per row
    head: np.ndarray        # [N] index into the heads of the row's batch
    heads: np.ndarray       # [H][3] peak, tilt, width
    ms: np.ndarray          # [N] Ms factor
    ku: np.ndarray          # [N] Ku factor
    tilt: np.ndarray        # [N] easy-axis tilt (rad) towards +x
    dx: np.ndarray          # [N] down-track offset (nm)
    X: np.ndarray           # [N][16] surrogate features

    def __len__(self):
        return len(self.ms)


def features(v: dict, ms, ku, tilt, dx) -> np.ndarray:
    """[N][16]: the 12 design values scaled to [-1, 1] by RANGES, then the 4 jitter
    values in units of three standard deviations."""
    N = len(ms)
    X = np.zeros((N, 16), np.float32)
    for k, key in enumerate(KEYS):
        lo, hi = RANGES[key]
        X[:, k] = 2.0 * (np.asarray(v[key], np.float64) - lo) / (hi - lo) - 1.0
    X[:, 12] = (np.asarray(ms) - 1.0) / (3 * JITTER["Ms"])
    X[:, 13] = (np.asarray(ku) - 1.0) / (3 * JITTER["Ku"])
    X[:, 14] = np.asarray(tilt) / (3 * math.radians(JITTER["tilt_deg"]))
    X[:, 15] = np.asarray(dx) / (3 * JITTER["pos_nm"])
    return X


def realisations(Z, n_jitter: int, seed: int, first_index: int, heads=None, head_of_design=None) -> Realisations:
    """n_jitter jittered realisations of each design Z [D][12].  The heads are the
    designs' own (one per design) unless heads [H][3] and head_of_design [D] are
    given, in which case design d's head parameters are replaced by heads[head_of_design[d]]."""
    Z = np.asarray(Z, np.float64)
    D, J = len(Z), int(n_jitter)
    v = values(Z)
    if heads is None:
        heads = np.stack([v[k] for k in HEAD_KEYS], 1)
        head_of_design = np.arange(D)
    heads = np.asarray(heads, np.float64)
    head_of_design = np.asarray(head_of_design, np.int64)
    for k, key in enumerate(HEAD_KEYS):
        v[key] = heads[head_of_design, k]
    v = {key: np.repeat(val, J) for key, val in v.items()}
    idx = np.arange(first_index, first_index + D * J, dtype=np.uint64)
    ms = 1.0 + JITTER["Ms"] * synth.counter_normal(seed, 700, idx)
    ku = 1.0 + JITTER["Ku"] * synth.counter_normal(seed, 701, idx)
    tilt = math.radians(JITTER["tilt_deg"]) * synth.counter_normal(seed, 702, idx)
    dx = JITTER["pos_nm"] * synth.counter_normal(seed, 703, idx)
    return Realisations(v=v, head=np.repeat(head_of_design, J), heads=heads, ms=ms, ku=ku, tilt=tilt, dx=dx,
                        X=features(v, ms, ku, tilt, dx))


def adjacent_offset(layout, pitch):
    """Offset (down-track, cross-track) of the adjacent-track island from the target."""
    layout = np.asarray(layout).astype(np.int64)
    p = np.asarray(pitch, np.float64)
    ox = np.where(layout == 1, 0.5 * p, 0.0)
    oy = np.where(layout == 2, -p, p)
    return ox, oy


def islands(R: Realisations, grid_ids, rows):
    """Target and adjacent islands (synth.Islands) of the realisation rows."""
    rows = np.asarray(rows, np.int64)
    geo = geometry_index({k: R.v[k][rows] for k in GEOMETRY_KEYS})
    mid = np.asarray(grid_ids, np.int32)[geo]
    Ms = (R.v["Ms_scale"][rows] * R.ms[rows]).astype(np.float32)
    Ku = (R.v["Ku_scale"][rows] * R.ku[rows]).astype(np.float32)
    u = np.stack([np.sin(R.tilt[rows]), np.zeros(len(rows)), np.cos(R.tilt[rows])], 1).astype(np.float32)
    bx, by = head_block(R.head[rows])
    x0, y0 = BLOCK_NM * bx.astype(np.float64), BLOCK_NM * by.astype(np.float64)
    ox, oy = adjacent_offset(R.v["layout"][rows], R.v["pitch_nm"][rows])
    mk = lambda px, py: synth.Islands(mesh_id=mid.copy(), Ms_scale=Ms.copy(), Ku_scale=Ku.copy(), u=u.copy(),
                                      pos_nm=np.stack([px, py], 1).astype(np.float32),
                                      Hext_T=np.zeros((len(rows), 3), np.float32))
    return mk(x0 + R.dx[rows], y0), mk(x0 + R.dx[rows] + ox, y0 + oy)


def run_params(v_m_per_s: float) -> synth.RunParams:
    return synth.RunParams(dt_ps=0.1, alpha=0.1, rise_ps=100.0, v_m_per_s=float(v_m_per_s),
                           x0_nm=-0.1 * float(v_m_per_s), use_map=True, t_end_ps=T_END_PS, substeps=0)


def llg_labels(ctx, grid_ids, R: Realisations, precision: int = L.PREC_BF16X3) -> np.ndarray:
    """LLG labels [N][2] (target switched, adjacent island flipped) of every
    realisation: one batch per (group of 256 heads, velocity level), the group's
    heads in one stacked map."""
    Y = np.zeros((len(R), 2), np.float32)
    group = R.head // HEADS_PER_MAP
    for g in np.unique(group):
        hid = ctx.headmap_upload(head_stack(R.heads[g * HEADS_PER_MAP:(g + 1) * HEADS_PER_MAP]))
        for v in LEVELS["v_m_per_s"]:
            rows = np.where((group == g) & np.isclose(R.v["v_m_per_s"], v))[0]
            if rows.size == 0:
                continue
            tgt, adj = islands(R, grid_ids, rows)
            out = ctx.run_batch(synth.Islands.concat([tgt, adj]), run_params(v), int(round(T_END_PS / 0.1)),
                                precision=precision, map_id=hid)
            if np.any(out["status"] != 0):
                raise RuntimeError("an island of a label batch reported a failure")
            n = rows.size
            Y[rows, 0] = out["switched"][:n]
            Y[rows, 1] = out["switched"][n:]
    return Y


def training_set(ctx, grid_ids, N: int, n_heads: int, seed: int, first_index: int = 0):
    """N uniform designs, one realisation each, whose heads are drawn from a pool of
    n_heads uniform head designs; returns (X, Y, R)."""
    Z = synth.counter_uniform(seed, 710, np.arange(first_index * 12, (first_index + N) * 12)).reshape(N, 12)
    Zh = synth.counter_uniform(seed, 711, np.arange(first_index * 3, (first_index + n_heads) * 3)).reshape(n_heads, 3)
    heads = np.stack([RANGES[k][0] + (RANGES[k][1] - RANGES[k][0]) * Zh[:, j] for j, k in enumerate(HEAD_KEYS)], 1)
    R = realisations(Z, 1, seed, first_index, heads=heads, head_of_design=np.arange(N) % n_heads)
    return R.X, llg_labels(ctx, grid_ids, R), R


def metrics(P, Y) -> dict:
    """Accuracy at 1/2, Brier score and ROC AUC of probabilities P [N] against labels Y [N]."""
    P = np.asarray(P, np.float64)
    Y = np.asarray(Y, np.float64) > 0.5
    pos, neg = P[Y], P[~Y]
    if pos.size and neg.size:
        allv = np.concatenate([pos, neg])
        ranks = np.empty(allv.size)
        order = np.argsort(allv, kind="stable")
        ranks[order] = np.arange(1, allv.size + 1)
        for val in np.unique(allv):                    # average ranks of ties
            tie = allv == val
            ranks[tie] = ranks[tie].mean()
        auc = (ranks[:pos.size].sum() - pos.size * (pos.size + 1) / 2) / (pos.size * neg.size)
    else:
        auc = float("nan")
    return dict(accuracy=float(np.mean((P > 0.5) == Y)), brier=float(np.mean((P - Y) ** 2)), auc=float(auc),
                positive_fraction=float(Y.mean()))


def search(ctx, sur, grid_ids, cfg: evolve.SearchConfig):
    """The generational design loop of evolve.search on this problem: each
    generation the surrogate screens the population on fresh jitter samples, the
    best-screened designs that are not elites yet are solved with LLG (each with
    its own head), and the elites are mutated into the next population."""
    P, K, Js, Jv = cfg.population, cfg.top_k, cfg.n_jitter_screen, cfg.n_jitter_verify
    d = len(KEYS)
    Z = synth.counter_uniform(cfg.seed, 720, np.arange(P * d, dtype=np.uint64)).reshape(P, d)
    elite_Z, elite_obj, elite_rates = np.zeros((0, d)), np.zeros(0), np.zeros((0, 2))
    res = evolve.SearchResult(best_Z=None, best_rates=None)
    for g in range(cfg.generations):
        n_el = len(elite_Z)
        t0 = time.perf_counter()
        Rs = realisations(Z, Js, cfg.seed + 1, first_index=g * P * Js)
        s_obj = sur.screen(Rs.X, P, Js).sum(1)
        res.screen_s += time.perf_counter() - t0
        cand = n_el + np.argsort(s_obj[n_el:], kind="stable")[:K]
        t0 = time.perf_counter()
        Rv = realisations(Z[cand], Jv, cfg.seed + 2, first_index=g * P * Jv)
        rates = evolve.error_rates(llg_labels(ctx, grid_ids, Rv), len(cand), Jv)
        res.verify_s += time.perf_counter() - t0
        res.verified_islands += 2 * len(cand) * Jv
        res.llg_only_islands += 2 * (P - n_el) * Jv
        pool_Z = np.concatenate([elite_Z, Z[cand]])
        pool_obj = np.concatenate([elite_obj, rates.sum(1)])
        pool_rates = np.concatenate([elite_rates, rates])
        keep = np.argsort(pool_obj, kind="stable")[:K]
        elite_Z, elite_obj, elite_rates = pool_Z[keep], pool_obj[keep], pool_rates[keep]
        res.history.append(dict(generation=g, best_verified=float(elite_obj[0]),
                                screened_of_verified=s_obj[cand].tolist(), verified=rates.sum(1).tolist()))
        if g + 1 < cfg.generations:
            Z = evolve.next_population(elite_Z, P, g + 1, cfg)
    res.best_Z, res.best_rates = elite_Z[0], elite_rates[0]
    return res
