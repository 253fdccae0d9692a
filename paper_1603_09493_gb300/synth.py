"""Seeded synthetic inputs for the batched ECC-island LLG path.

This module holds input generators only -- island meshes, per-island jitter
tables, the write-head field map and workload presets -- and none of the
method's arithmetic (no FEM assembly, no fields, no time stepping).  Both the
CUDA path and the FP64 oracle read the arrays it returns.

Geometry follows the exchange-coupled-composite island of Sec. II.B / Fig. 3
(a soft nucleation layer on top of a hard storage layer, coupled through an
interlayer exchange constant, Table I row A_ex,int); the sizes are the
workload's (8 nm cylinder, soft 3 nm on hard 7 nm, 12.7 nm square lattice).
The paper's own head fields came from a FEM/BEM head solve (Sec. II.A); the
synthetic map here is a Gaussian pole-tip field with a cross-track tilt that
stands in for it.

Random draws use a counter-based generator (SplitMix64 finaliser applied to
seed/stream/index counters, Box-Muller for normals) so that any island's draw
is reproducible on its own.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MU0 = 4e-7 * math.pi

# region ids of the layered island mesh
REGION_HARD = 0
REGION_HARD_INTERFACE = 1   # slab of hard tets directly below the soft/hard interface
REGION_SOFT = 2

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def _splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (Steele, Lea, Flood 2014) on uint64 arrays."""
    with np.errstate(over="ignore"):
        z = (x + np.uint64(0x9E3779B97F4A7C15)) & _M64
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _M64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _M64
        return z ^ (z >> np.uint64(31))


def counter_uniform(seed: int, stream: int, index) -> np.ndarray:
    """Uniform doubles in (0, 1) keyed by (seed, stream, index)."""
    idx = np.asarray(index, dtype=np.uint64)
    with np.errstate(over="ignore"):
        key = _splitmix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) ^
                          (np.uint64(stream) * np.uint64(0xD1B54A32D192ED03)))
        z = _splitmix64(key ^ (idx * np.uint64(0x9E3779B97F4A7C15)))
    # 53 random bits -> (0,1), never exactly 0
    return ((z >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def counter_normal(seed: int, stream: int, index) -> np.ndarray:
    """Standard normals keyed by (seed, stream, index) via Box-Muller."""
    idx = np.asarray(index, dtype=np.uint64)
    u1 = counter_uniform(seed, stream, idx * np.uint64(2))
    u2 = counter_uniform(seed, stream, idx * np.uint64(2) + np.uint64(1))
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


# --------------------------------------------------------------------------
# island mesh
# --------------------------------------------------------------------------

@dataclass
class IslandMesh:
    xyz_nm: np.ndarray        # [n][3] float64, z up, island bottom at z = 0
    tets: np.ndarray          # [nt][4] int32, positively oriented
    tet_region: np.ndarray    # [nt] int32
    z_interface_nm: float
    height_nm: float
    info: dict = field(default_factory=dict)

    @property
    def n_nodes(self) -> int:
        return int(self.xyz_nm.shape[0])

    @property
    def n_tets(self) -> int:
        return int(self.tets.shape[0])


def _disk_nodes_and_triangles(rings: int):
    """Concentric hexagonal rings: ring k holds 6k nodes; zipper triangulation."""
    pts = [(0.0, 0.0)]
    ring_start = [0]
    for k in range(1, rings + 1):
        ring_start.append(len(pts))
        for j in range(6 * k):
            th = 2.0 * math.pi * j / (6 * k)
            pts.append((k / rings * math.cos(th), k / rings * math.sin(th)))
    tris = []
    for j in range(6):
        tris.append((0, 1 + j, 1 + (j + 1) % 6))
    for k in range(2, rings + 1):
        p, q = 6 * (k - 1), 6 * k
        a0, b0 = ring_start[k - 1], ring_start[k]
        i = j = 0
        while i < p or j < q:
            next_a = (i + 1) / p
            next_b = (j + 1) / q
            if j < q and (i == p or next_b <= next_a):
                tris.append((a0 + i % p, b0 + j, b0 + (j + 1) % q))
                j += 1
            else:
                tris.append((a0 + i, b0 + j % q, a0 + (i + 1) % p))
                i += 1
    return np.array(pts, dtype=np.float64), np.array(tris, dtype=np.int64), rings


def layered_island_mesh(diameter_nm: float = 8.0, t_hard_nm: float = 7.0,
                        t_soft_nm: float = 3.0, rings: int = 2,
                        hard_slabs: int = 7, soft_slabs: int = 3,
                        aspect: float = 1.0, seed: int = 0,
                        perturb: float = 0.12) -> IslandMesh:
    """Seeded layered P1-tetrahedral mesh of an ECC island.

    The cross-section is a disk (or an equal-area ellipse of axis ratio
    `aspect`) of concentric hexagonal node rings; it is extruded through
    `hard_slabs` + `soft_slabs` node planes, the soft/hard interface being a
    node plane, and every prism is cut into three tetrahedra by the
    sorted-global-index rule (conforming across neighbouring prisms).  Interior
    nodes of each plane are moved in-plane by a seeded uniform displacement of
    up to `perturb` ring spacings; the outer ring stays on the polygon.
    """
    uv, tris, K = _disk_nodes_and_triangles(rings)
    n2 = uv.shape[0]
    R = 0.5 * diameter_nm
    ax, ay = math.sqrt(aspect), 1.0 / math.sqrt(aspect)
    interior = np.zeros(n2, dtype=bool)
    interior[: 1 + 3 * (K - 1) * K] = True          # rings 0..K-1
    zs = list(np.linspace(0.0, t_hard_nm, hard_slabs + 1))
    zs += list(np.linspace(t_hard_nm, t_hard_nm + t_soft_nm, soft_slabs + 1)[1:])
    n_planes = len(zs)
    xyz = np.zeros((n_planes * n2, 3))
    for p, z in enumerate(zs):
        idx = np.arange(n2, dtype=np.uint64) + np.uint64(p * n2)
        d = np.stack([counter_uniform(seed, 101, idx), counter_uniform(seed, 102, idx)], 1)
        d = (2.0 * d - 1.0) * perturb / K
        d[~interior] = 0.0
        xy = uv + d
        xyz[p * n2:(p + 1) * n2, 0] = R * ax * xy[:, 0]
        xyz[p * n2:(p + 1) * n2, 1] = R * ay * xy[:, 1]
        xyz[p * n2:(p + 1) * n2, 2] = z
    tets, regs = [], []
    for p in range(n_planes - 1):
        if p < hard_slabs - 1:
            reg = REGION_HARD
        elif p == hard_slabs - 1:
            reg = REGION_HARD_INTERFACE
        else:
            reg = REGION_SOFT
        for tri in tris:
            v0, v1, v2 = sorted(int(t) for t in tri)
            b0, b1, b2 = p * n2 + v0, p * n2 + v1, p * n2 + v2
            t0, t1, t2 = b0 + n2, b1 + n2, b2 + n2
            for tet in ((b0, b1, b2, t2), (b0, b1, t1, t2), (b0, t0, t1, t2)):
                tets.append(list(tet))
                regs.append(reg)
    tets = np.array(tets, dtype=np.int64)
    # orient positively
    x = xyz[tets]
    vol6 = np.einsum("ij,ij->i", x[:, 1] - x[:, 0], np.cross(x[:, 2] - x[:, 0], x[:, 3] - x[:, 0]))
    neg = vol6 < 0
    tets[neg, 2], tets[neg, 3] = tets[neg, 3].copy(), tets[neg, 2].copy()
    x = xyz[tets]
    vol6 = np.einsum("ij,ij->i", x[:, 1] - x[:, 0], np.cross(x[:, 2] - x[:, 0], x[:, 3] - x[:, 0]))
    if np.any(vol6 <= 1e-12):
        raise ValueError("degenerate tetrahedron in generated mesh; reduce perturb")
    return IslandMesh(xyz_nm=xyz, tets=tets.astype(np.int32),
                      tet_region=np.array(regs, dtype=np.int32),
                      z_interface_nm=float(t_hard_nm),
                      height_nm=float(t_hard_nm + t_soft_nm),
                      info=dict(diameter_nm=diameter_nm, t_hard_nm=t_hard_nm,
                                t_soft_nm=t_soft_nm, rings=rings, hard_slabs=hard_slabs,
                                soft_slabs=soft_slabs, aspect=aspect, seed=seed,
                                perturb=perturb, nodes_per_plane=n2, planes=n_planes))


def polygon_area_nm2(mesh: IslandMesh) -> float:
    """Area of the outer node ring polygon (the exact cross-section of the mesh)."""
    info = mesh.info
    K, n2 = info["rings"], info["nodes_per_plane"]
    ring = mesh.xyz_nm[1 + 3 * (K - 1) * K:n2, :2]
    x, y = ring[:, 0], ring[:, 1]
    return 0.5 * float(np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y))


def ecc_materials(Ms_hard=0.8e6, Ku_hard=0.9e6, A_hard=10e-12,
                  Ms_soft=1.0e6, Ku_soft=0.0, A_soft=10e-12,
                  interlayer_scale=0.3) -> np.ndarray:
    """Region table [3][3] = (Ms A/m, Ku J/m^3, A J/m) for hard, hard-interface, soft."""
    return np.array([[Ms_hard, Ku_hard, A_hard],
                     [Ms_hard, Ku_hard, A_hard * interlayer_scale],
                     [Ms_soft, Ku_soft, A_soft]], dtype=np.float64)


# --------------------------------------------------------------------------
# per-island jitter
# --------------------------------------------------------------------------

@dataclass
class Islands:
    mesh_id: np.ndarray     # [B] int32
    Ms_scale: np.ndarray    # [B] float32
    Ku_scale: np.ndarray    # [B] float32
    u: np.ndarray           # [B][3] float32 easy axis (unit)
    pos_nm: np.ndarray      # [B][2] float32 island centre in the media frame
    Hext_T: np.ndarray      # [B][3] float32 constant per-island field

    def __len__(self):
        return int(self.mesh_id.shape[0])

    def subset(self, idx) -> "Islands":
        return Islands(self.mesh_id[idx], self.Ms_scale[idx], self.Ku_scale[idx],
                       self.u[idx], self.pos_nm[idx], self.Hext_T[idx])

    @staticmethod
    def concat(parts) -> "Islands":
        return Islands(*[np.concatenate([getattr(p, f) for p in parts])
                         for f in ("mesh_id", "Ms_scale", "Ku_scale", "u", "pos_nm", "Hext_T")])


def nominal_islands(B: int, mesh_id: int = 0, pos_nm=(0.0, 0.0), Hext_T=(0.0, 0.0, 0.0)) -> Islands:
    return Islands(mesh_id=np.full(B, mesh_id, np.int32),
                   Ms_scale=np.ones(B, np.float32), Ku_scale=np.ones(B, np.float32),
                   u=np.tile(np.array([0, 0, 1], np.float32), (B, 1)),
                   pos_nm=np.tile(np.asarray(pos_nm, np.float32), (B, 1)),
                   Hext_T=np.tile(np.asarray(Hext_T, np.float32), (B, 1)))


def jittered_islands(B: int, seed: int, mesh_id: int = 0, sigma_ms: float = 0.05,
                     sigma_ku: float = 0.05, sigma_tilt_deg: float = 2.0,
                     sigma_pos_nm: float = 1.0, lattice_pos_nm=(0.0, 0.0),
                     first_index: int = 0) -> Islands:
    """Per-island Gaussian jitter of Ms, Ku, easy-axis tilt and position.

    Stream ids: 1 Ms, 2 Ku, 3/4 tilt x/y, 5/6 position x/y; index = island.
    """
    idx = np.arange(first_index, first_index + B, dtype=np.uint64)
    ms = 1.0 + sigma_ms * counter_normal(seed, 1, idx)
    ku = 1.0 + sigma_ku * counter_normal(seed, 2, idx)
    tx = np.deg2rad(sigma_tilt_deg) * counter_normal(seed, 3, idx)
    ty = np.deg2rad(sigma_tilt_deg) * counter_normal(seed, 4, idx)
    u = np.stack([np.tan(tx), np.tan(ty), np.ones(B)], 1)
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    px = lattice_pos_nm[0] + sigma_pos_nm * counter_normal(seed, 5, idx)
    py = lattice_pos_nm[1] + sigma_pos_nm * counter_normal(seed, 6, idx)
    return Islands(mesh_id=np.full(B, mesh_id, np.int32),
                   Ms_scale=ms.astype(np.float32), Ku_scale=ku.astype(np.float32),
                   u=u.astype(np.float32), pos_nm=np.stack([px, py], 1).astype(np.float32),
                   Hext_T=np.zeros((B, 3), np.float32))


# --------------------------------------------------------------------------
# synthetic write-head field map
# --------------------------------------------------------------------------

@dataclass
class HeadMap:
    B_T: np.ndarray            # [nz][ny][nx][3] float32 (mu0*H in tesla)
    origin_nm: np.ndarray      # [3] float32: (x, y, z) of voxel (0,0,0)
    h_nm: float
    info: dict = field(default_factory=dict)


def synthetic_head_map(nx=64, ny=64, nz=16, h_nm=1.0, B_peak_T=1.3, tilt_deg=25.0,
                       sx_nm=8.0, sy_nm=8.0, decay_nm=12.0, d_top_nm=5.0,
                       z_top_nm=10.0, d_ref_nm=6.5) -> HeadMap:
    """Gaussian pole-tip field with a cross-track tilt, stands in for a head solve.

    Axes: x down-track in the head frame (x = 0 under the pole centre), y
    cross-track, z height in the media frame (island top at z_top_nm, which
    sits d_top_nm below the air-bearing surface).  The field points along
    (0, sin tilt, -cos tilt), peaks at B_peak_T at depth d_ref_nm (the middle
    of the soft layer) and decays exponentially with depth.
    """
    xs = (np.arange(nx) - nx // 2) * h_nm
    ys = (np.arange(ny) - ny // 2) * h_nm
    zs = np.arange(nz) * h_nm
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    depth = d_top_nm + (z_top_nm - Z)
    amp = B_peak_T * np.exp(-X ** 2 / (2 * sx_nm ** 2) - Y ** 2 / (2 * sy_nm ** 2)) \
        * np.exp(-(depth - d_ref_nm) / decay_nm)
    th = math.radians(tilt_deg)
    B = np.stack([np.zeros_like(amp), amp * math.sin(th), -amp * math.cos(th)], -1)
    return HeadMap(B_T=B.astype(np.float32),
                   origin_nm=np.array([xs[0], ys[0], zs[0]], np.float32), h_nm=float(h_nm),
                   info=dict(B_peak_T=B_peak_T, tilt_deg=tilt_deg, sx_nm=sx_nm, sy_nm=sy_nm,
                             decay_nm=decay_nm, d_ref_nm=d_ref_nm))


def pole_geometry(**overrides) -> dict:
    """Main-pole geometry for the head-field solve (field names of bpm_pole_geometry): Table I's
    initial design (pole tip width 14 nm, trailing edge angle 20 deg, side edge angle 15 deg,
    taper 75 deg), the yoke edge 153 nm above the ABS, CoFe at 2.4 T (Table II), a 20 nm deep
    ABS footprint, and the frame of synthetic_head_map: island tops at z = 10 nm, the ABS 6 nm
    above them (the paper's head-media spacing), the soft under-layer 20 nm below the ABS.  No
    shields unless their gaps are given (Table I's initial design: trailing gap 9 nm, side gap
    16 nm, thickness 10 nm)."""
    g = dict(pole_tip_width_nm=14.0, trailing_edge_angle_deg=20.0, side_edge_angle_deg=15.0,
             taper_angle_deg=75.0, abs_thickness_nm=20.0, yoke_edge_nm=153.0, Js_T=2.4,
             z_abs_nm=16.0, z_sul_nm=-4.0, sul_image=1, trailing_shield_gap_nm=0.0, shield_thickness_nm=0.0,
             shield_panel_nm=2.0, side_shield_gap_nm=0.0)
    g.update(overrides)
    return g


# --------------------------------------------------------------------------
# run parameters and workload presets
# --------------------------------------------------------------------------

# term mask bits (same meaning on both sides of the boundary)
TERM_EXCHANGE = 1
TERM_ANISOTROPY = 2
TERM_DEMAG = 4
TERM_HEAD = 8
TERM_UNIFORM = 16
TERM_ALL = 31


@dataclass
class RunParams:
    dt_ps: float = 0.1          # output / sampling interval
    substeps: int = 1           # integrator steps per output interval
    t0_ps: float = 0.0
    t_end_ps: float = 100.0
    alpha: float = 0.1
    rise_ps: float = 100.0      # linear field ramp time
    v_m_per_s: float = 20.0     # head velocity (down-track, +x)
    x0_nm: float = -10.0        # head-centre x at t = 0
    use_map: bool = False
    uniform_T: tuple = (0.0, 0.0, 0.0)
    term_mask: int = TERM_ALL

    @property
    def n_intervals(self) -> int:
        return int(round((self.t_end_ps - self.t0_ps) / self.dt_ps))


def uniform_field(B_T: float, angle_deg: float) -> tuple:
    """Field of magnitude B_T in the xz-plane at angle_deg from +z."""
    a = math.radians(angle_deg)
    return (B_T * math.sin(a), 0.0, B_T * math.cos(a))


def census_run_params(t_end_ps: float = 0.1) -> RunParams:
    """The census workload's run: head map moving at 20 m/s from 10 nm before the
    island, 100 ps field rise, damping 0.1, 0.1 ps output intervals."""
    return RunParams(dt_ps=0.1, alpha=0.1, rise_ps=100.0, v_m_per_s=20.0, x0_nm=-10.0, use_map=True,
                     t_end_ps=t_end_ps)


def head_field_direction(tilt_deg: float = 25.0) -> np.ndarray:
    """Unit direction of the synthetic head field, (0, sin tilt, -cos tilt)."""
    th = math.radians(tilt_deg)
    return np.array([0.0, math.sin(th), -math.cos(th)])


def outcome_census(B: int = 1024, seed: int = 5, mesh_id: int = 0, H_max_T: float = 0.3):
    """A recording census of Sec. II.C shape: B jittered islands written by the head
    moving at 20 m/s from 2 nm before them (100 ps rise, damping 0.1, 300 ps),
    island b under a constant field of (b / B) H_max_T opposing the head field, so
    that the outcomes range from nearly all switched to nearly none.  Returns
    (Islands, RunParams)."""
    isl = jittered_islands(B, seed=seed, mesh_id=mesh_id)
    mag = H_max_T * np.arange(B) / B
    isl.Hext_T[:] = (-mag[:, None] * head_field_direction()[None, :]).astype(np.float32)
    p = RunParams(dt_ps=0.1, alpha=0.1, rise_ps=100.0, v_m_per_s=20.0, x0_nm=-2.0, use_map=True, t_end_ps=300.0)
    return isl, p


def small_island_mesh(seed: int = 0) -> IslandMesh:
    """~200-node island: 19-node disk x 11 planes (hard 7 x 1 nm, soft 3 x 1 nm)."""
    return layered_island_mesh(8.0, 7.0, 3.0, rings=2, hard_slabs=7, soft_slabs=3, seed=seed)


def census_island_mesh(seed: int = 1) -> IslandMesh:
    """~1500-node island: 91-node disk x 17 planes (hard 11, soft 5 slabs)."""
    return layered_island_mesh(8.0, 7.0, 3.0, rings=5, hard_slabs=11, soft_slabs=5, seed=seed)


def variant_island_mesh(diameter_nm: float, soft_ratio: float, elliptical: bool,
                        target_nodes: int, seed: int) -> IslandMesh:
    """Island of a design variant: total height 10 nm, t_soft/t_hard = soft_ratio,
    circle or 1.5:1 equal-area ellipse, ring/plane counts chosen to approach
    target_nodes with a node spacing near isotropic."""
    t_hard = 10.0 / (1.0 + soft_ratio)
    t_soft = 10.0 - t_hard
    best = None
    for K in range(2, 14):
        n2 = 1 + 3 * K * (K + 1)
        planes = max(4, int(round(target_nodes / n2)))
        slabs = planes - 1
        soft = max(1, int(round(slabs * t_soft / 10.0)))
        hard = max(2, slabs - soft)
        n = n2 * (hard + soft + 1)
        score = abs(n - target_nodes) / target_nodes + 0.15 * abs(
            math.log((diameter_nm / 2 / K) / (10.0 / slabs)))
        if best is None or score < best[0]:
            best = (score, K, hard, soft)
    _, K, hard, soft = best
    return layered_island_mesh(diameter_nm, t_hard, t_soft, rings=K, hard_slabs=hard,
                               soft_slabs=soft, aspect=1.5 if elliptical else 1.0, seed=seed)


# --------------------------------------------------------------------------
# surrogate inputs
# --------------------------------------------------------------------------

def mlp_init_params(sizes, seed: int) -> np.ndarray:
    """Flat initial parameters of an MLP with layer widths `sizes` (input first):
    per layer W [out][in] ~ N(0, 1/in) from the counter generator, then b = 0."""
    out, k = [], 0
    for i, (fan_in, fan_out) in enumerate(zip(sizes[:-1], sizes[1:])):
        idx = np.arange(fan_in * fan_out, dtype=np.uint64)
        W = counter_normal(seed, 1000 + i, idx) / math.sqrt(fan_in)
        out.append(W.astype(np.float32))
        out.append(np.zeros(fan_out, np.float32))
    return np.concatenate(out)


def unflatten_params(flat, sizes):
    """Flat vector -> [(W [out][in], b [out]), ...] (float64), the oracle's layout."""
    res, off = [], 0
    for fan_in, fan_out in zip(sizes[:-1], sizes[1:]):
        W = np.asarray(flat[off:off + fan_in * fan_out], np.float64).reshape(fan_out, fan_in)
        off += fan_in * fan_out
        b = np.asarray(flat[off:off + fan_out], np.float64)
        off += fan_out
        res.append((W, b))
    return res


def flatten_params(params) -> np.ndarray:
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in params]).astype(np.float64)


# --------------------------------------------------------------------------
# uneven batches: design variants and track layouts
# --------------------------------------------------------------------------

def design_variants(n_min: int = 500, n_max: int = 4000, seed: int = 2):
    """The 16 design variants of the uneven workload: diameter 6-10 nm (4
    values) x soft/hard thickness ratio 0.2 or 0.5 x circular or 1.5:1
    elliptical cross-section, with target node counts spread over
    [n_min, n_max] in variant order."""
    out = []
    k = 0
    for d in (6.0, 22.0 / 3.0, 26.0 / 3.0, 10.0):
        for ratio in (0.2, 0.5):
            for ell in (False, True):
                target = int(round(n_min + (n_max - n_min) * k / 15.0))
                mesh = variant_island_mesh(d, ratio, ell, target, seed=seed * 100 + k)
                out.append(dict(mesh=mesh, diameter_nm=d, soft_ratio=ratio, elliptical=ell, target_nodes=target))
                k += 1
    return out


def layout_offsets(layout: str, pitch_nm: float = 12.7):
    """Positions (down-track x, cross-track y) of the target island and of the
    adjacent-track islands under the fringing field: centered and shingled
    writing have neighbours at (0, +-p); in staggered writing the adjacent
    rows are shifted by half a pitch down-track, (+-p/2, +-p) (the effective
    down-track separation is halved, Sec. IV).  Shingled writing keeps only
    the previously written side.  Returns (target, [adjacent...])."""
    p = float(pitch_nm)
    if layout == "centered":
        return (0.0, 0.0), [(0.0, p), (0.0, -p)]
    if layout == "staggered":
        return (0.0, 0.0), [(0.5 * p, p), (-0.5 * p, -p)]
    if layout == "shingled":
        return (0.0, 0.0), [(0.0, -p)]
    raise ValueError(layout)


def uneven_batch(variants, mesh_ids, realisations: int, seed: int, layout: str = "centered",
                 pitch_nm: float = 12.7):
    """Jittered targets plus adjacent-track islands for every variant; returns
    (Islands, role) with role 0 = target, 1 = adjacent."""
    parts, roles = [], []
    (tx, ty), adj = layout_offsets(layout, pitch_nm)
    for v, (var, mid) in enumerate(zip(variants, mesh_ids)):
        for r, (px, py) in enumerate([(tx, ty)] + adj):
            isl = jittered_islands(realisations, seed=seed, mesh_id=mid, lattice_pos_nm=(px, py),
                                   first_index=(v * 8 + r) * realisations)
            parts.append(isl)
            roles.append(np.full(realisations, 0 if r == 0 else 1, np.int32))
    return Islands.concat(parts), np.concatenate(roles)


# --------------------------------------------------------------------------
# surrogate screening designs
# --------------------------------------------------------------------------

SCREEN_RANGES = dict(Ms_scale=(0.85, 1.15), Ku_scale=(0.75, 1.25), tilt_x_deg=(-4.0, 4.0),
                     tilt_y_deg=(-4.0, 4.0), pos_x_nm=(-1.5, 1.5), pos_y_nm=(-1.5, 1.5),
                     B_ext_T=(0.55, 1.05), angle_deg=(160.0, 180.0))


def screening_designs(N: int, seed: int, mesh_id: int = 0, first_index: int = 0):
    """Random candidate designs for the surrogate: per island uniform draws of
    the parameters in SCREEN_RANGES (Ms and Ku scale, easy-axis tilt, position,
    magnitude and angle from +z of a constant field in the xz-plane).  Returns
    (Islands, X) with X [N][16] the features scaled to [-1, 1] (unused features
    zero)."""
    idx = np.arange(first_index, first_index + N, dtype=np.uint64)
    keys = list(SCREEN_RANGES)
    U = np.stack([counter_uniform(seed, 200 + k, idx) for k in range(len(keys))], 1)
    val = {k: lo + (hi - lo) * U[:, j] for j, (k, (lo, hi)) in enumerate(SCREEN_RANGES.items())}
    tx, ty = np.deg2rad(val["tilt_x_deg"]), np.deg2rad(val["tilt_y_deg"])
    u = np.stack([np.tan(tx), np.tan(ty), np.ones(N)], 1)
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    a = np.deg2rad(val["angle_deg"])
    H = np.stack([val["B_ext_T"] * np.sin(a), np.zeros(N), val["B_ext_T"] * np.cos(a)], 1)
    isl = Islands(mesh_id=np.full(N, mesh_id, np.int32), Ms_scale=val["Ms_scale"].astype(np.float32),
                  Ku_scale=val["Ku_scale"].astype(np.float32), u=u.astype(np.float32),
                  pos_nm=np.stack([val["pos_x_nm"], val["pos_y_nm"]], 1).astype(np.float32),
                  Hext_T=H.astype(np.float32))
    X = np.zeros((N, 16), np.float32)
    X[:, :len(keys)] = 2.0 * U - 1.0
    return isl, X


# --------------------------------------------------------------------------
# random inputs of the global optimiser (Latin hypercubes, candidate points)
# --------------------------------------------------------------------------
def lhs_candidates(T: int, n: int, d: int, seed: int) -> np.ndarray:
    """T random Latin hypercubes of n points in [0, 1)^d, [T][n][d]: in every
    column the points fall one per stratum [j/n, (j+1)/n), each at a uniform
    offset inside its stratum."""
    out = np.empty((T, n, d))
    for t in range(T):
        for k in range(d):
            base = (t * d + k) * n
            perm = np.argsort(counter_uniform(seed, 300, np.arange(base, base + n)), kind="stable")
            off = counter_uniform(seed, 301, np.arange(base, base + n))
            out[t, :, k] = (perm + off) / n
    return out


def unit_points(N: int, d: int, seed: int, stream: int) -> np.ndarray:
    """N uniform points in (0, 1)^d, [N][d]."""
    return counter_uniform(seed, 400 + stream, np.arange(N * d)).reshape(N, d)


def theta_unit_draws(T: int, d: int, seed: int, round_: int) -> np.ndarray:
    """Unit uniforms [T][d] for round `round_` of the correlation-length search."""
    return counter_uniform(seed, 500 + round_, np.arange(T * d)).reshape(T, d)


def branin01(X: np.ndarray) -> np.ndarray:
    """Branin's test function on [0,1]^2 (x1 in [-5, 10], x2 in [0, 15]); global
    minimum 0.397887 at three points."""
    x1 = -5.0 + 15.0 * X[:, 0]
    x2 = 15.0 * X[:, 1]
    a, b, c, r, s, t = 1.0, 5.1 / (4 * math.pi ** 2), 5.0 / math.pi, 6.0, 10.0, 1.0 / (8 * math.pi)
    return a * (x2 - b * x1 ** 2 + c * x1 - r) ** 2 + s * (1 - t) * np.cos(x1) + s
