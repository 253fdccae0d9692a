"""P1 finite elements on tetrahedra, plain FP64 (oracle; test infrastructure).

The paper treats the island with finite-element micromagnetics (abstract;
Sec. II.A "hybrid finite element/boundary element method") but does not write
the discretisation down.  Reading used here (textbook P1 FEM):

* nodal magnetisation, linear shape functions phi_i on each tetrahedron;
* lumped nodal volume V_i = sum over tets t containing i of vol_t / 4;
* nodal material values are lumped volume averages of the region values;
* exchange stiffness K_ij = sum_t A_t vol_t grad(phi_i).grad(phi_j), so that
  the exchange field at node i is B_i = -(2 / (Ms_i V_i)) sum_j K_ij m_j;
* the interlayer exchange A_ex,int of Fig. 3 / Table I enters as the A of the
  slab of hard tets directly below the soft/hard interface.

Lengths are in nm, so K carries a factor 1e-9 and V a factor 1e-27 when
converted to SI; `exchange_matrix_T` returns the operator in tesla.
"""
from __future__ import annotations

import numpy as np


def tet_geometry(xyz_nm: np.ndarray, tets: np.ndarray):
    """Volumes [nt] (nm^3) and shape-function gradients [nt][4][3] (1/nm).

    phi = barycentric coordinates: for J = [x1-x0, x2-x0, x3-x0] (columns),
    (phi_1, phi_2, phi_3) = J^{-1} (x - x0) and phi_0 = 1 - phi_1 - phi_2 - phi_3.
    """
    x = xyz_nm[tets]                                   # [nt][4][3]
    J = np.stack([x[:, 1] - x[:, 0], x[:, 2] - x[:, 0], x[:, 3] - x[:, 0]], axis=2)
    vol = np.linalg.det(J) / 6.0
    Jinv = np.linalg.inv(J)                            # rows = grad phi_1..3
    grads = np.empty((tets.shape[0], 4, 3))
    grads[:, 1:, :] = Jinv
    grads[:, 0, :] = -Jinv.sum(axis=1)
    return vol, grads


def lumped_volumes(n: int, tets: np.ndarray, vol: np.ndarray) -> np.ndarray:
    V = np.zeros(n)
    for k in range(4):
        np.add.at(V, tets[:, k], vol / 4.0)
    return V


def laplacian(n: int, tets: np.ndarray, vol: np.ndarray, grads: np.ndarray,
              coeff: np.ndarray | None = None) -> np.ndarray:
    """Dense K_ij = sum_t c_t vol_t grad(phi_i).grad(phi_j) (units nm * c)."""
    c = np.ones(tets.shape[0]) if coeff is None else coeff
    K = np.zeros((n, n))
    local = np.einsum("tid,tjd->tij", grads, grads) * (c * vol)[:, None, None]
    for a in range(4):
        for b in range(4):
            np.add.at(K, (tets[:, a], tets[:, b]), local[:, a, b])
    return K


def nodal_average(n: int, tets: np.ndarray, vol: np.ndarray, V: np.ndarray,
                  tet_values: np.ndarray) -> np.ndarray:
    out = np.zeros(n)
    for k in range(4):
        np.add.at(out, tets[:, k], tet_values * vol / 4.0)
    return out / V


class MeshOperators:
    """Everything the oracle needs about one island mesh, in FP64."""

    def __init__(self, xyz_nm, tets, tet_region, region_mats, with_demag=True):
        self.xyz = np.asarray(xyz_nm, dtype=np.float64)
        self.tets = np.asarray(tets, dtype=np.int64)
        self.region = np.asarray(tet_region, dtype=np.int64)
        mats = np.asarray(region_mats, dtype=np.float64)
        self.n = self.xyz.shape[0]
        self.vol, self.grads = tet_geometry(self.xyz, self.tets)
        self.V = lumped_volumes(self.n, self.tets, self.vol)
        Ms_t, Ku_t, A_t = mats[self.region, 0], mats[self.region, 1], mats[self.region, 2]
        self.Ms = nodal_average(self.n, self.tets, self.vol, self.V, Ms_t)      # A/m
        self.Ku = nodal_average(self.n, self.tets, self.vol, self.V, Ku_t)      # J/m^3
        self.K_A = laplacian(self.n, self.tets, self.vol, self.grads, A_t)      # J/m * nm
        # exchange operator in tesla: B_ex = -S m, S = 2 K / (Ms V) (nm -> m: 1e-9 / 1e-27)
        self.S = (2.0 * 1e18) * self.K_A / (self.Ms * self.V)[:, None]
        self.demag = None
        if with_demag:
            from . import demag
            self.demag = demag.fredkin_koehler_matrix(self.xyz, self.tets, self.vol, self.grads, self.V)

    def exchange_field(self, m: np.ndarray, Ms_scale: np.ndarray) -> np.ndarray:
        """m [B][n][3] -> B_ex [B][n][3] in tesla for islands with Ms scaled by Ms_scale."""
        return -np.einsum("ij,bjc->bic", self.S, m) / Ms_scale[:, None, None]

    def exchange_lambda_max(self) -> float:
        """Largest eigenvalue of S (tesla per unit m); S = D K with D > 0 diagonal."""
        d = np.sqrt((2.0 * 1e18) / (self.Ms * self.V))
        sym = d[:, None] * self.K_A * d[None, :]
        return float(np.linalg.eigvalsh(sym)[-1])
