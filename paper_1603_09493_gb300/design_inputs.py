"""Seeded inputs of the write-head and media design problem (Sec. II.A
optimisation loop; Sec. II.B and Table I free parameters; Fig. 3 track
layouts): the design parameters and their grid, the island meshes of the
geometry grid, the stacked head maps, jittered realisations of designs, their
surrogate features and their islands.  Input generators only, like synth: no
field, no time stepping, no library call.

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
from dataclasses import dataclass

import numpy as np

from . import synth

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


def nominal(Z) -> Realisations:
    """One realisation of each design without jitter (Ms and Ku factors 1, no tilt, no offset)."""
    R = realisations(Z, 1, seed=0, first_index=0)
    R.ms[:] = 1.0
    R.ku[:] = 1.0
    R.tilt[:] = 0.0
    R.dx[:] = 0.0
    R.X = features(R.v, R.ms, R.ku, R.tilt, R.dx)
    return R




def parity_designs() -> np.ndarray:
    """Three designs that share the grid's middle geometry (d 8 nm, soft 3 nm, hard 7 nm,
    exchange scale 0.3), one velocity level, a 12 nm head field width and a 9 nm pitch, with
    their own Ms, Ku, layout, tilt and head peaks of 1.05, 1.14 and 1.19 T: their critical
    fields lie inside the search grid (the write margin of the first, the previous-bit margins
    of the other two), the cases whose critical-field bit-error rates are compared with the
    oracle's."""
    Z = synth.counter_uniform(61, 0, np.arange(6 * 12)).reshape(6, 12)[[1, 3, 4]]
    for key in GEOMETRY_KEYS + ("v_m_per_s",):
        Z[:, KEYS.index(key)] = 0.5
    Z[:, KEYS.index("B_peak_T")] = [0.08, 0.24, 0.32]
    Z[:, KEYS.index("width_nm")] = 1.0
    Z[:, KEYS.index("pitch_nm")] = 0.0
    return Z


def critical_field_inputs(Z, role: str, K1_hard: float = 0.9e6, Ms_hard: float = 0.8e6):
    """The critical-field search's inputs for designs Z (Sec. II.C): the nominal islands
    (the previous bit one pitch behind the target, down-track), the unit head-field
    directions (0, sin tilt, -cos tilt), sigma = 0.015 mu0 H_A of each design's hard layer
    (T), and the realisations.  mesh_id holds the geometry-grid index."""
    R = nominal(Z)
    D = len(R)
    tgt, _ = islands(R, np.arange(81), np.arange(D))
    if role == "prev":
        tgt.pos_nm[:, 0] -= R.v["pitch_nm"].astype(np.float32)
    th = np.radians(R.v["tilt_deg"])
    direction = np.stack([np.zeros(D), np.sin(th), -np.cos(th)], 1)
    mu0 = 4e-7 * math.pi
    sigma = 0.015 * 2.0 * K1_hard * R.v["Ku_scale"] * mu0 / (mu0 * Ms_hard * R.v["Ms_scale"])
    return tgt, direction, sigma, R
