"""Trilinear lookup of the write-head field map, FP64 (oracle; test infrastructure).

Sec. II.A / II.C: the precomputed head field is moved over the island at the
head velocity and scaled by the current rise; the field between grid points is
interpolated.  Reading: trilinear interpolation of the map values, positions
outside the grid clamped to the grid box (edge voxel value).
"""
from __future__ import annotations

import numpy as np


def trilinear(B_map: np.ndarray, origin_nm, h_nm: float, p_nm: np.ndarray) -> np.ndarray:
    """B_map [nz][ny][nx][3], p_nm [..., 3] (x, y, z) -> field [..., 3] (float64)."""
    Bm = np.asarray(B_map, dtype=np.float64)
    nz, ny, nx = Bm.shape[:3]
    dims = np.array([nx, ny, nz], dtype=np.float64)
    if np.any(dims < 2):
        raise ValueError("head map needs at least two points along every axis")
    f = (np.asarray(p_nm, np.float64) - np.asarray(origin_nm, np.float64)) / float(h_nm)
    f = np.clip(f, 0.0, dims - 1.0)
    i0 = np.minimum(np.floor(f), dims - 2.0)
    w = f - i0
    i0 = i0.astype(np.int64)
    out = np.zeros(f.shape[:-1] + (3,))
    for dz in (0, 1):
        wz = w[..., 2] if dz else 1.0 - w[..., 2]
        for dy in (0, 1):
            wy = w[..., 1] if dy else 1.0 - w[..., 1]
            for dx in (0, 1):
                wx = w[..., 0] if dx else 1.0 - w[..., 0]
                v = Bm[i0[..., 2] + dz, i0[..., 1] + dy, i0[..., 0] + dx]
                out += (wx * wy * wz)[..., None] * v
    return out
