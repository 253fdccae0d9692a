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
* the shield (trailing and side blocks, when their gaps are given) is solved
  as described below.

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


# --------------------------------------------------------------------------------------------
# Wrap-around shield (Sec. II.A, Table I gaps and thickness).  Readings: the shield has unbounded
# permeability, so its surface is an equipotential of the magnetic potential and it carries no
# net magnetic charge.  Its trailing block stands on the ABS with its leading face parallel to
# the pole's trailing face at the trailing shield gap (down-track, at the ABS),
# shield_thickness_nm high (Table I's shield thickness read as the height above the ABS), 30 nm
# deep down-track and 40 nm wider than the pole tip on each side; each side block has its inner
# face parallel to the pole's flared side at the side shield gap, as high, from 10 nm behind the
# leading edge to 0.5 nm short of the trailing block, out to the trailing block's extent.  The
# surface is cut into flat triangles carrying uniform charge (collocation at the triangle
# centroids), and the under-layer image applies to them too.
# --------------------------------------------------------------------------------------------

SHIELD_DEPTH_NM = 30.0
SHIELD_MARGIN_NM = 40.0
SIDE_LEAD_NM = 10.0        # side shields start this far behind the leading edge
SIDE_CLEAR_NM = 0.5        # and stop this far short of the trailing shield


def shield_blocks(g: dict):
    """The shield's blocks as (corner, three edge vectors): the trailing block, and with a side
    shield gap the two side blocks, whose inner faces lean out with the pole's flared sides (the
    paper builds every shield face parallel to the opposite pole face); one body."""
    tt = math.tan(math.radians(g["trailing_edge_angle_deg"]))
    ts = math.tan(math.radians(g["side_edge_angle_deg"]))
    w = float(g["pole_tip_width_nm"])
    W = w + 2 * SHIELD_MARGIN_NM
    T = float(g["shield_thickness_nm"])
    z0 = float(g["z_abs_nm"])
    gap_t = float(g.get("trailing_shield_gap_nm", 0.0))
    gap_s = float(g.get("side_shield_gap_nm", 0.0))
    blocks = []
    if gap_t > 0:
        blocks.append((np.array([gap_t, -W / 2, z0]), np.array([SHIELD_DEPTH_NM, 0, 0]), np.array([0, W, 0]),
                       np.array([T * tt, 0, T])))
    if gap_s > 0:
        x0 = -float(g["abs_thickness_nm"]) - SIDE_LEAD_NM
        x1 = max(gap_t, 0.0) - SIDE_CLEAR_NM
        inner = w / 2 + gap_s
        reach = W / 2 - inner
        blocks.append((np.array([x0, inner, z0]), np.array([x1 - x0, 0, 0]), np.array([0, reach, 0]),
                       np.array([0, T * ts, T])))
        blocks.append((np.array([x0, -W / 2, z0]), np.array([x1 - x0, 0, 0]), np.array([0, reach, 0]),
                       np.array([0, -T * ts, T])))
    return blocks


def has_shield(g: dict) -> bool:
    return float(g.get("trailing_shield_gap_nm", 0.0)) > 0 or float(g.get("side_shield_gap_nm", 0.0)) > 0


def shield_panels(g: dict):
    """Triangles [N][3][3] of the shield's blocks (outward winding) and their areas [N]: each face
    a grid of about shield_panel_nm squares (parallelograms), each cell split along the diagonal
    from its first corner."""
    panel = float(g.get("shield_panel_nm") or 2.0)
    tris, areas = [], []
    for corner, dx, dy, dz in shield_blocks(g):
        centre = corner + (dx + dy + dz) / 2
        faces = [(corner, dx, dy), (corner + dz, dx, dy), (corner, dy, dz), (corner + dx, dy, dz),
                 (corner, dx, dz), (corner + dy, dx, dz)]
        for origin, u, v in faces:
            nu = max(1, math.ceil(np.linalg.norm(u) / panel - 1e-9))
            nv = max(1, math.ceil(np.linalg.norm(v) / panel - 1e-9))
            for i in range(nu):
                for j in range(nv):
                    p = lambda a, b: origin + (a / nu) * u + (b / nv) * v
                    for a, b, c in ((p(i, j), p(i + 1, j), p(i + 1, j + 1)),
                                    (p(i, j), p(i + 1, j + 1), p(i, j + 1))):
                        n = np.cross(b - a, c - a)
                        if np.dot(n, (a + b + c) / 3 - centre) < 0:
                            b, c = c, b
                        tris.append(np.array([a, b, c]))
                        areas.append(0.5 * np.linalg.norm(n))
    return np.array(tris), np.array(areas)


def _potential(tri: np.ndarray, P: np.ndarray, ratio: float = 0.25, depth: int = 0) -> float:
    """int over the triangle of 1 / |P - Q| dA by quadrature: a point on the triangle becomes the
    first corner of three sub-triangles (the map from the unit square then cancels the 1/R
    singularity); elsewhere sub-triangles are split four ways until small against their
    distance to P."""
    a, b, c = tri
    n = np.cross(b - a, c - a)
    area2 = np.linalg.norm(n)
    n = n / area2
    h = np.dot(P - a, n)
    if abs(h) < 1e-12 * math.sqrt(area2):
        # barycentric coordinates of P in the triangle's plane
        w1 = np.dot(np.cross(c - b, P - b), n) / area2
        w2 = np.dot(np.cross(a - c, P - c), n) / area2
        w3 = 1 - w1 - w2
        if min(w1, w2, w3) > -1e-12:
            return sum(_potential_from_corner(np.array([P, u, v])) for u, v in ((a, b), (b, c), (c, a)))
    centroid = tri.mean(axis=0)
    diam = max(np.linalg.norm(tri[i] - tri[j]) for i, j in ((0, 1), (1, 2), (2, 0)))
    if diam > ratio * np.linalg.norm(P - centroid) and depth < 40:
        ab, bc, ca = (a + b) / 2, (b + c) / 2, (c + a) / 2
        return sum(_potential(np.array(t), P, ratio, depth + 1) for t in
                   ((a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca)))
    Q, W = _triangle_rule(tri)
    return float((W / np.linalg.norm(P - Q, axis=1)).sum())


def _potential_from_corner(tri: np.ndarray, depth: int = 0) -> float:
    # the triangle's first corner is the evaluation point; wedges wider than half their shorter
    # side are halved at the far edge, so that the rule sees a smooth integrand along it
    P, b, c = tri
    if np.linalg.norm(np.cross(b - P, c - P)) < 1e-14:
        return 0.0
    if np.linalg.norm(c - b) > 0.5 * min(np.linalg.norm(b - P), np.linalg.norm(c - P)) and depth < 30:
        m = (b + c) / 2
        return (_potential_from_corner(np.array([P, b, m]), depth + 1) +
                _potential_from_corner(np.array([P, m, c]), depth + 1))
    Q, W = _triangle_rule(tri)
    return float((W / np.linalg.norm(P - Q, axis=1)).sum())


def potential_closed(tris: np.ndarray, P: np.ndarray) -> np.ndarray:
    """int 1/|P - Q| dA over every triangle [T][3][3] (winding gives the normal n), in closed form:
    with P0 the foot of P on a triangle's plane at signed height h, each edge (ends at s- < s+
    along its unit direction from P0's projection, outward in-plane normal m, distance d of the
    edge line from P0, distances R-, R+ of its ends from P) contributes
        d ln((R+ + s+)/(R- + s-)) - |h| [atan(d s+/(R0^2 + |h| R+)) - atan(d s-/(R0^2 + |h| R-))],
    R0^2 = d^2 + h^2: the integral of 1/R over the plane in polar coordinates about P0, taken
    edge by edge (pinned against quadrature in the tests)."""
    tris = np.asarray(tris, np.float64)
    P = np.asarray(P, np.float64)
    n = np.cross(tris[:, 1] - tris[:, 0], tris[:, 2] - tris[:, 0])
    n /= np.linalg.norm(n, axis=1)[:, None]
    h = np.einsum("ij,ij->i", P - tris[:, 0], n)
    ah = np.abs(h)
    P0 = P - h[:, None] * n
    tot = np.zeros(len(tris))
    for i in range(3):
        p, q = tris[:, i], tris[:, (i + 1) % 3]
        e = q - p
        L = np.linalg.norm(e, axis=1)
        t = e / L[:, None]
        m = np.cross(t, n)
        sm = np.einsum("ij,ij->i", p - P0, t)
        sp = np.einsum("ij,ij->i", q - P0, t)
        d = np.einsum("ij,ij->i", p - P0, m)
        Rm = np.linalg.norm(p - P, axis=1)
        Rp = np.linalg.norm(q - P, axis=1)
        R02 = d * d + h * h
        with np.errstate(divide="ignore", invalid="ignore"):
            fwd = np.log((Rp + sp) / (Rm + sm))
            bwd = np.log((Rm - sm) / (Rp - sp))
        lg = np.where(sp + sm >= 0, np.where(Rm + sm > 0, fwd, 0.0), bwd)
        lg = np.where(np.isfinite(lg), lg, 0.0)      # P on the edge line: d = 0, no contribution
        tot += d * lg - ah * (np.arctan2(d * sp, R02 + ah * Rp) - np.arctan2(d * sm, R02 + ah * Rm))
    return tot


def _potential_rows(tris: np.ndarray, P: np.ndarray) -> np.ndarray:
    return potential_closed(tris, P)


def _coulomb_rows(tris: np.ndarray, P: np.ndarray, ratio: float = 0.25) -> np.ndarray:
    """int (P - Q)/|P - Q|^3 dA over every triangle [T] -> [T][3]: one 8 x 8 rule for the
    triangles far from P (all at once), the adaptive rule for the others."""
    out = np.empty((len(tris), 3))
    centroid = tris.mean(axis=1)
    diam = np.max(np.linalg.norm(tris[:, [0, 1, 2]] - tris[:, [1, 2, 0]], axis=2), axis=1)
    far = diam <= ratio * np.linalg.norm(P - centroid, axis=1)
    s = 0.5 * (_GL_X + 1.0)
    ws = 0.5 * _GL_W
    S, T = np.meshgrid(s, s, indexing="ij")
    Wg = (np.outer(ws, ws) * S).reshape(-1)
    S, T = S.reshape(-1), T.reshape(-1)
    f = tris[far]
    a, b, c = f[:, 0], f[:, 1], f[:, 2]
    Q = a[:, None] + S[None, :, None] * (b - a)[:, None] + (S * T)[None, :, None] * (c - b)[:, None]
    jac = np.linalg.norm(np.cross(b - a, c - b), axis=1)
    d = P - Q
    r3 = np.linalg.norm(d, axis=2) ** 3
    out[far] = jac[:, None] * (Wg[None, :, None] * d / r3[..., None]).sum(axis=1)
    for k in np.where(~far)[0]:
        out[k] = _coulomb(tris[k], P, ratio)
    return out


def bem_equipotential(tris: np.ndarray, areas: np.ndarray, phi_ext: np.ndarray, image_z=None):
    """Charges q [N] (as mu0 sigma, tesla) on the triangles of a body of unbounded permeability
    that make the total potential mu0 phi_ext + mu0 phi_q the same constant Phi at every triangle
    centroid, with sum q A = 0 (no net charge); with image_z, the body's mirror image in
    z = image_z carries -q.  phi_ext [N]: the applied mu0 phi at the centroids (tesla nm).
    Returns (q, Phi)."""
    N = len(tris)
    cent = tris.mean(axis=1)
    img = None
    if image_z is not None:
        img = tris.copy()
        img[..., 2] = 2.0 * image_z - img[..., 2]
        img = img[:, [0, 2, 1]]
    A = np.zeros((N + 1, N + 1))
    for i in range(N):
        row = _potential_rows(tris, cent[i])
        if img is not None:
            row = row - _potential_rows(img, cent[i])
        A[i, :N] = row / (4 * math.pi)
        A[i, N] = -1.0
    A[N, :N] = areas
    rhs = np.concatenate([-np.asarray(phi_ext, np.float64), [0.0]])
    x = np.linalg.solve(A, rhs)
    return x[:N], x[N]


def pole_potential(g: dict, points: np.ndarray) -> np.ndarray:
    """mu0 phi (tesla nm) of the pole's charges (and their images) at points [M][3]."""
    tris, charge = pole_triangles(g)
    return np.array([sum(q / (4 * math.pi) * v for q, v in zip(charge, _potential_rows(tris, p)))
                     for p in np.asarray(points, np.float64)])


def shield_charges(g: dict):
    """The shield's triangles, their charges q (tesla) and the shield's potential Phi."""
    tris, areas = shield_panels(g)
    phi = pole_potential(g, tris.mean(axis=1))
    q, Phi = bem_equipotential(tris, areas, phi, float(g["z_sul_nm"]) if g.get("sul_image", 0) else None)
    return tris, q, Phi


def field_with_shield(g: dict, points_nm: np.ndarray) -> np.ndarray:
    """mu0 H (tesla) of the pole and, when g has a trailing shield gap, the shield's induced
    charges (and their images), at points [..., 3] (nm)."""
    B = field(g, points_nm)
    if not has_shield(g):
        return B
    tris, q, _ = shield_charges(g)
    if g.get("sul_image", 0):
        img = tris.copy()
        img[..., 2] = 2.0 * float(g["z_sul_nm"]) - img[..., 2]
        tris = np.concatenate([tris, img[:, [0, 2, 1]]])
        q = np.concatenate([q, -q])
    P = np.asarray(points_nm, np.float64).reshape(-1, 3)
    out = B.reshape(-1, 3).copy()
    for k, p in enumerate(P):
        out[k] += (q[:, None] / (4.0 * math.pi) * _coulomb_rows(tris, p)).sum(axis=0)
    return out.reshape(np.shape(points_nm))
