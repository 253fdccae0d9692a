"""Demagnetising operator by the Fredkin-Koehler FEM/BEM split, plain FP64
(oracle; test infrastructure).

The paper's solver is a hybrid finite-element/boundary-element method
(Sec. II.A, citing Schrefl et al. 2005) but the paper does not write it out.
Reading used (Fredkin & Koehler, IEEE Trans. Magn. 26, 415 (1990); double-layer
weights of Lindholm, IEEE Trans. Magn. 20, 2025 (1984)), with H = -grad(u):

1. u1 solves the Neumann problem  int grad(u1).grad(v) = int M.grad(v)  for all
   P1 test functions v, with zero mean (u1 = 0 outside the island);
2. on the boundary, u2 = B u1 with B = D + diag(Omega_i / 4pi - 1), where
   D_ij = (1/4pi) int phi_j(y) n_y.(x_i - y) / |x_i - y|^3 dS_y (double layer)
   and Omega_i is the interior solid angle at boundary node i;
3. u2 is harmonic inside the island (P1 Dirichlet problem);
4. H_t = -grad(u1 + u2) per tetrahedron, projected to the nodes by the lumped
   (volume-weighted) average.

M -> H is linear, so the operator is materialised as the dense matrix N of
H = -N M with row/column index c * n + i (component-planar).  Dense LU solves
(numpy.linalg.solve) stand for the two Poisson problems.
"""
from __future__ import annotations

import math

import numpy as np


def boundary_faces(xyz: np.ndarray, tets: np.ndarray) -> np.ndarray:
    """Faces [nf][3] that belong to exactly one tet, ordered so that
    (y2 - y1) x (y3 - y1) points out of the island."""
    faces, opp = [], []
    for k in range(4):
        idx = [a for a in range(4) if a != k]
        faces.append(tets[:, idx])
        opp.append(tets[:, k])
    faces = np.concatenate(faces)
    opp = np.concatenate(opp)
    key = np.sort(faces, axis=1)
    _, inv, counts = np.unique(key, axis=0, return_inverse=True, return_counts=True)
    once = counts[inv.ravel()] == 1
    f, o = faces[once].copy(), opp[once]
    y = xyz[f]
    nrm = np.cross(y[:, 1] - y[:, 0], y[:, 2] - y[:, 0])
    flip = np.einsum("ij,ij->i", nrm, xyz[o] - y[:, 0]) > 0
    f[flip, 1], f[flip, 2] = f[flip, 2].copy(), f[flip, 1].copy()
    return f


def solid_angle(r1: np.ndarray, r2: np.ndarray, r3: np.ndarray) -> np.ndarray:
    """Signed solid angle of triangle (r1, r2, r3) (vectors from the observer),
    positive when the triangle's normal (r2-r1)x(r3-r1) points away from the
    observer -- van Oosterom & Strackee, IEEE Trans. Biomed. Eng. 30, 125 (1983)."""
    l1, l2, l3 = (np.linalg.norm(r, axis=-1) for r in (r1, r2, r3))
    num = np.einsum("...i,...i->...", r1, np.cross(r2, r3))
    den = (l1 * l2 * l3 + np.einsum("...i,...i->...", r1, r2) * l3
           + np.einsum("...i,...i->...", r1, r3) * l2 + np.einsum("...i,...i->...", r2, r3) * l1)
    return 2.0 * np.arctan2(num, den)


def interior_solid_angles(xyz: np.ndarray, tets: np.ndarray, nodes: np.ndarray) -> np.ndarray:
    """Interior solid angle at each node: sum over the tets around it of the
    solid angle that the opposite face subtends at the node."""
    omega = np.zeros(xyz.shape[0])
    for a in range(4):
        others = [b for b in range(4) if b != a]
        x = xyz[tets[:, a]]
        w = np.abs(solid_angle(*(xyz[tets[:, b]] - x for b in others)))
        np.add.at(omega, tets[:, a], w)
    return omega[nodes]


def lindholm_weights(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """w_k = int_T phi_k(s) n.(s - x) / |s - x|^3 dS for a flat triangle T with
    vertices y[..., k, :] (counter-clockwise about n) and observers x[..., :].

    Closed form (Lindholm 1984, restated): with rho_k = y_k - x, side k from
    vertex k to k+1 of length s_k and unit vector xi_k, zeta = n.rho_1,
    eta_k = (n x xi_k).rho_k, gamma_kj = xi_k.xi_j,
    P_k = ln((|rho_k| + |rho_k+1| + s_k) / (|rho_k| + |rho_k+1| - s_k)) and the
    signed solid angle Omega:
        w_k = s_{k+1} / (2A) * (-eta_{k+1} Omega + zeta sum_j gamma_{k+1,j} P_j).
    The weights sum to Omega.  Observers must not be vertices of T.
    """
    rho = y - x[..., None, :]                           # [..., 3, 3]
    e = np.roll(y, -1, axis=-2) - y                     # side k: y_{k+1} - y_k
    s = np.linalg.norm(e, axis=-1)
    xi = e / s[..., None]
    cr = np.cross(y[..., 1, :] - y[..., 0, :], y[..., 2, :] - y[..., 0, :])
    two_area = np.linalg.norm(cr, axis=-1)
    n = cr / two_area[..., None]
    zeta = np.einsum("...i,...i->...", n, rho[..., 0, :])
    eta = np.einsum("...ki,...ki->...k", np.cross(n[..., None, :], xi), rho)
    gamma = np.einsum("...ki,...ji->...kj", xi, xi)
    lr = np.linalg.norm(rho, axis=-1)
    lsum = lr + np.roll(lr, -1, axis=-1)
    P = np.log((lsum + s) / (lsum - s))
    omega = solid_angle(rho[..., 0, :], rho[..., 1, :], rho[..., 2, :])
    w = np.empty_like(s)
    for k in range(3):
        k1 = (k + 1) % 3
        w[..., k] = s[..., k1] / two_area * (-eta[..., k1] * omega
                                             + zeta * np.einsum("...j,...j->...", gamma[..., k1, :], P))
    return w


def double_layer_matrix(xyz: np.ndarray, faces: np.ndarray, bnodes: np.ndarray) -> np.ndarray:
    """D [nb][nb], D_ij = (1/4pi) int phi_j n.(x_i - y)/|x_i - y|^3 dS = -(1/4pi) sum_T w_j."""
    nb = bnodes.shape[0]
    pos = -np.ones(xyz.shape[0], dtype=np.int64)
    pos[bnodes] = np.arange(nb)
    fl = pos[faces]                                     # local boundary indices
    D = np.zeros((nb, nb))
    yT = xyz[faces]                                     # [nf][3][3]
    chunk = max(1, 400000 // max(1, faces.shape[0]))
    for i0 in range(0, nb, chunk):
        rows = np.arange(i0, min(nb, i0 + chunk))
        x = xyz[bnodes[rows]]                           # [r][3]
        touching = np.any(fl[None, :, :] == rows[:, None, None], axis=2)   # [r][nf]
        X = np.broadcast_to(x[:, None, :], (rows.size, faces.shape[0], 3)).copy()
        Y = np.broadcast_to(yT[None], (rows.size,) + yT.shape).copy()
        # keep the formula away from the singular vertex case; those weights are zero
        X[touching] = 0.0
        Y[touching] = np.array([[1.0, 0, 0], [0, 1.0, 0], [0, 0, 1.0]]) + 10.0
        w = lindholm_weights(X, Y)                      # [r][nf][3]
        w[touching] = 0.0
        for k in range(3):
            np.add.at(D, (np.repeat(rows, faces.shape[0]), np.tile(fl[:, k], rows.size)),
                      (-w[:, :, k] / (4.0 * math.pi)).ravel())
    return D


def rhs_matrix(n: int, tets: np.ndarray, vol: np.ndarray, grads: np.ndarray) -> np.ndarray:
    """R [n][3n]: (R M)_i = int M.grad(phi_i) for nodal P1 M (column c*n + k)."""
    R = np.zeros((n, 3 * n))
    for a in range(4):
        for b in range(4):
            for c in range(3):
                np.add.at(R, (tets[:, a], c * n + tets[:, b]), vol * grads[:, a, c] / 4.0)
    return R


def fredkin_koehler_matrix(xyz, tets, vol, grads, V, return_parts=False):
    """Dense N [3n][3n] with H = -N M (index c*n + i)."""
    from .fem import laplacian
    n = xyz.shape[0]
    K = laplacian(n, tets, vol, grads)
    R = rhs_matrix(n, tets, vol, grads)
    # 1. Neumann problem with zero-mean gauge (Lagrange multiplier)
    aug = np.zeros((n + 1, n + 1))
    aug[:n, :n] = K
    aug[:n, n] = 1.0
    aug[n, :n] = 1.0
    rhs = np.zeros((n + 1, 3 * n))
    rhs[:n] = R
    u1 = np.linalg.solve(aug, rhs)[:n]
    # 2. boundary values of u2
    faces = boundary_faces(xyz, tets)
    bnodes = np.unique(faces)
    D = double_layer_matrix(xyz, faces, bnodes)
    omega = interior_solid_angles(xyz, tets, bnodes)
    Bmat = D + np.diag(omega / (4.0 * math.pi) - 1.0)
    u2 = np.zeros_like(u1)
    u2[bnodes] = Bmat @ u1[bnodes]
    # 3. harmonic extension into the interior
    interior = np.setdiff1d(np.arange(n), bnodes)
    if interior.size:
        u2[interior] = np.linalg.solve(K[np.ix_(interior, interior)],
                                       -K[np.ix_(interior, bnodes)] @ u2[bnodes])
    u = u1 + u2
    # 4. N_{c i, :} = (1/V_i) sum_{t ni i} (vol_t/4) sum_{k in t} grad(phi_k)[c] u_k
    P = np.zeros((3 * n, n))
    for a in range(4):
        for b in range(4):
            for c in range(3):
                np.add.at(P, (c * n + tets[:, a], tets[:, b]), vol * grads[:, b, c] / 4.0)
    N = (P @ u) / np.tile(V, 3)[:, None]
    if return_parts:
        return N, dict(K=K, R=R, u1=u1, u2=u2, faces=faces, bnodes=bnodes, D=D, omega=omega)
    return N
