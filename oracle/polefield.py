"""Field of a saturated write-head main pole, FP64 (oracle; test infrastructure).

Sec. II.A computes the write field below the saturated head, with the yoke,
return pole and coil replaced by a charge sheet of density Js at the yoke edge
153 nm above the ABS, and the soft under-layer (SUL) taken into account by
mirroring the pole at its upper surface.  Table I gives the pole's free
parameters (pole tip width, trailing edge angle, side edge angle, taper angle
of the ABS footprint, 75 deg); Table II its saturation polarisation (CoFe,
2.4 T).

Readings (where the paper gives no number or formula):
* the pole is uniformly magnetised at Js along -z (saturated, towards the
  media), so its field is that of the surface charges sigma = M . n on its
  faces; the face at the yoke edge carries -Js/mu0, which is the charge sheet;
* ABS footprint: trailing edge of width w at x = 0, narrowing towards the
  leading edge at the taper angle from the trailing edge, `abs_thickness_nm`
  deep down-track (leading width at least w/10); the trailing face leans
  down-track by the trailing edge angle, the side faces flare cross-track by
  the side edge angle (both from the vertical); the leading face is vertical;
  every face is split into two triangles along the diagonal from its first
  corner below; the non-planar side faces from their trailing corner at the
  ABS, so that the two sides mirror each other;
* the SUL has unbounded permeability: the magnetic potential is constant on
  its surface, which the mirror image of the pole with charges of the
  opposite sign gives;
* shields are not modelled.

The field is evaluated by numerical quadrature of the Coulomb integral
    mu0 H(P) = (Js (m . n) / 4 pi) int (P - Q) / |P - Q|^3 dA_Q
over every triangle: 8 x 8 Gauss-Legendre points on the triangle mapped from
the unit square, on sub-triangles split four ways until each is smaller than a
quarter of its distance to P.
"""
from __future__ import annotations

import math

import numpy as np

JS_COFE_T = 2.4


def pole_vertices(g: dict) -> dict:
    """The eight corners of the pole (nm): ABS footprint (z = z_abs) and yoke edge."""
    w, D, H = float(g["pole_tip_width_nm"]), float(g["abs_thickness_nm"]), float(g["yoke_edge_nm"])
    tt = math.tan(math.radians(g["trailing_edge_angle_deg"]))
    ts = math.tan(math.radians(g["side_edge_angle_deg"]))
    wl = max(w - 2.0 * D / math.tan(math.radians(g["taper_angle_deg"])), 0.1 * w)
    z0 = float(g["z_abs_nm"])
    z1 = z0 + H
    return {
        "trail_l": (0.0, -w / 2, z0), "trail_r": (0.0, w / 2, z0),
        "lead_r": (-D, wl / 2, z0), "lead_l": (-D, -wl / 2, z0),
        "trail_l_top": (H * tt, -(w / 2 + H * ts), z1), "trail_r_top": (H * tt, w / 2 + H * ts, z1),
        "lead_r_top": (-D, wl / 2 + H * ts, z1), "lead_l_top": (-D, -(wl / 2 + H * ts), z1),
    }


def pole_triangles(g: dict) -> tuple[np.ndarray, np.ndarray]:
    """Triangles [T][3][3] (nm) with outward normals, and the charge of each as Js (m . n),
    tesla (m = -z); with g["sul_image"] the mirrored triangles and opposite charges follow."""
    v = pole_vertices(g)
    faces = [  # each face as a loop of corners
        ("trail_l", "trail_r", "lead_r", "lead_l"),                  # ABS
        ("trail_l_top", "trail_r_top", "lead_r_top", "lead_l_top"),  # yoke edge (charge sheet)
        ("trail_l", "trail_r", "trail_r_top", "trail_l_top"),        # trailing face
        ("lead_l", "lead_r", "lead_r_top", "lead_l_top"),            # leading face
        ("trail_r", "lead_r", "lead_r_top", "trail_r_top"),          # side +y
        ("trail_l", "lead_l", "lead_l_top", "trail_l_top"),          # side -y
    ]
    centre = np.mean(np.array(list(v.values())), axis=0)
    tris, charge = [], []
    for f in faces:
        p = [np.array(v[k]) for k in f]
        for a, b, c in ((p[0], p[1], p[2]), (p[0], p[2], p[3])):
            n = np.cross(b - a, c - a)
            if np.linalg.norm(n) < 1e-9:
                continue
            if np.dot(n, (a + b + c) / 3 - centre) < 0:
                b, c = c, b
                n = -n
            tris.append(np.array([a, b, c]))
            charge.append(-float(g["Js_T"]) * n[2] / np.linalg.norm(n))
    tris = np.array(tris)
    charge = np.array(charge)
    if g.get("sul_image", 0):
        img = tris.copy()
        img[..., 2] = 2.0 * float(g["z_sul_nm"]) - img[..., 2]
        img = img[:, [0, 2, 1]]          # keep the winding outward after the mirror
        tris = np.concatenate([tris, img])
        charge = np.concatenate([charge, -charge])
    return tris, charge


_GL_X, _GL_W = np.polynomial.legendre.leggauss(8)


def _triangle_rule(tri: np.ndarray):
    """Quadrature points [N][3] and weights [N] (area included) on one triangle: the unit square
    (s, t) mapped by Q = a + s (b - a) + s t (c - b), Jacobian s |(b - a) x (c - b)|."""
    a, b, c = tri
    s = 0.5 * (_GL_X + 1.0)
    ws = 0.5 * _GL_W
    S, T = np.meshgrid(s, s, indexing="ij")
    W = np.outer(ws, ws) * S
    Q = a + S[..., None] * (b - a) + (S * T)[..., None] * (c - b)
    jac = np.linalg.norm(np.cross(b - a, c - b))
    return Q.reshape(-1, 3), (W * jac).reshape(-1)


def _coulomb(tri: np.ndarray, P: np.ndarray, ratio: float = 0.25, depth: int = 0) -> np.ndarray:
    """int over the triangle of (P - Q) / |P - Q|^3 dA, adaptively."""
    centroid = tri.mean(axis=0)
    diam = max(np.linalg.norm(tri[i] - tri[j]) for i, j in ((0, 1), (1, 2), (2, 0)))
    if diam > ratio * np.linalg.norm(P - centroid) and depth < 40:
        a, b, c = tri
        ab, bc, ca = (a + b) / 2, (b + c) / 2, (c + a) / 2
        return sum(_coulomb(np.array(t), P, ratio, depth + 1) for t in
                   ((a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca)))
    Q, W = _triangle_rule(tri)
    d = P - Q
    r3 = np.linalg.norm(d, axis=1) ** 3
    return (W[:, None] * d / r3[:, None]).sum(axis=0)


def field(g: dict, points_nm: np.ndarray) -> np.ndarray:
    """mu0 H (tesla) of the saturated pole at points [..., 3] (nm), outside the pole."""
    tris, charge = pole_triangles(g)
    P = np.asarray(points_nm, np.float64).reshape(-1, 3)
    out = np.zeros_like(P)
    for k, p in enumerate(P):
        for tri, q in zip(tris, charge):
            out[k] += q / (4.0 * math.pi) * _coulomb(tri, p)
    return out.reshape(np.shape(points_nm))


def field_map(g: dict, nx: int, ny: int, nz: int, h_nm: float, origin_nm) -> np.ndarray:
    """The field on the voxel grid [nz][ny][nx][3] (voxel (ix, iy, iz) at origin + h (ix, iy, iz))."""
    o = np.asarray(origin_nm, np.float64)
    zs, ys, xs = (o[2] + h_nm * np.arange(nz), o[1] + h_nm * np.arange(ny), o[0] + h_nm * np.arange(nx))
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    return field(g, np.stack([X, Y, Z], -1))
