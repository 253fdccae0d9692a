"""Pins of the oracle's Fredkin-Koehler demag operator.

Independent checks: brute-force quadrature of the double-layer integral,
solid angles of known configurations, the constant-potential identity of the
boundary operator (two independent solid-angle computations must agree), the
trace of the volume-averaged demag tensor, and the magnetometric factor of the
same polygonal prism from a surface-charge double integral."""
import math

import numpy as np
import pytest

from oracle import demag, fem
from paper_1603_09493_gb300 import synth


def _tri_rule(a, b, c, order):
    """Collapsed Gauss-Legendre rule on triangle (a, b, c): points, weights."""
    g, w = np.polynomial.legendre.leggauss(order)
    g, w = 0.5 * (g + 1), 0.5 * w
    S, T = np.meshgrid(g, g, indexing="ij")
    WS, WT = np.meshgrid(w, w, indexing="ij")
    s, t = S.ravel(), T.ravel()
    pts = a + s[:, None] * ((b - a) + t[:, None] * (c - b))
    area2 = np.linalg.norm(np.cross(b - a, c - a))
    return pts, (WS * WT).ravel() * s * area2


def _subdivide(a, b, c, levels):
    tris = [(a, b, c)]
    for _ in range(levels):
        nxt = []
        for p, q, r in tris:
            pq, qr, rp = (p + q) / 2, (q + r) / 2, (r + p) / 2
            nxt += [(p, pq, rp), (pq, q, qr), (rp, qr, r), (pq, qr, rp)]
        tris = nxt
    return tris


def test_lindholm_weights_match_quadrature():
    y = np.array([[0.0, 0.0, 0.0], [2.0, 0.3, 0.1], [0.4, 1.7, -0.2]])
    n = np.cross(y[1] - y[0], y[2] - y[0])
    n /= np.linalg.norm(n)
    # barycentric coordinates for the shape functions
    Tm = np.stack([y[1] - y[0], y[2] - y[0], n], 1)
    observers = [np.array([0.7, 0.6, 1.0]), np.array([0.7, 0.6, -0.4]),
                 np.array([3.0, -1.0, 0.5]), np.array([0.8, 0.5, 0.15]),
                 np.array([-1.0, 2.0, -2.0])]
    for x in observers:
        acc = np.zeros(3)
        for tri in _subdivide(y[0], y[1], y[2], 4):
            p, w = _tri_rule(*tri, 12)
            lam = np.linalg.solve(Tm, (p - y[0]).T).T
            phi = np.stack([1 - lam[:, 0] - lam[:, 1], lam[:, 0], lam[:, 1]], 1)
            r = p - x
            ker = (r @ n) / np.linalg.norm(r, axis=1) ** 3
            acc += (w * ker) @ phi
        wl = demag.lindholm_weights(x[None], y[None])[0]
        assert np.allclose(wl, acc, rtol=1e-7, atol=1e-9), (x, wl, acc)
        om = demag.solid_angle(*(y[k] - x for k in range(3)))
        assert abs(wl.sum() - om) < 1e-12


def test_solid_angle_of_cube_face_from_centre():
    c = np.array([0.5, 0.5, 0.5])
    # top face z = 1 split into two triangles, normal +z (away from the centre)
    f1 = [np.array(v, float) - c for v in ([0, 0, 1], [1, 0, 1], [1, 1, 1])]
    f2 = [np.array(v, float) - c for v in ([0, 0, 1], [1, 1, 1], [0, 1, 1])]
    om = demag.solid_angle(*f1) + demag.solid_angle(*f2)
    assert abs(om - 4 * math.pi / 6) < 1e-14
    # reversed orientation flips the sign
    assert abs(demag.solid_angle(f1[0], f1[2], f1[1]) + demag.solid_angle(*f1)) < 1e-15


@pytest.fixture(scope="module")
def small_parts():
    m = synth.small_island_mesh()
    ops = fem.MeshOperators(m.xyz_nm, m.tets, m.tet_region, synth.ecc_materials(), with_demag=False)
    N, parts = demag.fredkin_koehler_matrix(ops.xyz, ops.tets, ops.vol, ops.grads, ops.V,
                                            return_parts=True)
    return m, ops, N, parts


def test_interior_solid_angles(small_parts):
    m, ops, _, parts = small_parts
    allnodes = np.arange(ops.n)
    om_all = demag.interior_solid_angles(ops.xyz, ops.tets, allnodes)
    interior = np.setdiff1d(allnodes, parts["bnodes"])
    assert np.abs(om_all[interior] - 4 * math.pi).max() < 1e-12
    # nodes inside the flat top and bottom faces see half space
    z = ops.xyz[:, 2]
    n2 = m.info["nodes_per_plane"]
    K = m.info["rings"]
    face_inner = [i for i in allnodes if (i % n2) < 1 + 3 * (K - 1) * K and
                  (abs(z[i]) < 1e-12 or abs(z[i] - m.height_nm) < 1e-12)]
    assert np.abs(om_all[face_inner] - 2 * math.pi).max() < 1e-12


def test_boundary_operator_maps_constant_to_minus_constant(small_parts):
    _, ops, _, parts = small_parts
    # (D + diag(Omega/4pi - 1)) 1 = -1 : Lindholm weights (triangles) against
    # the interior solid angles (tetrahedra), two independent computations
    D, om = parts["D"], parts["omega"]
    Bmat = D + np.diag(om / (4 * math.pi) - 1.0)
    assert np.abs(Bmat.sum(axis=1) + 1.0).max() < 1e-12


def _avg_tensor(N, V):
    n = V.shape[0]
    T = np.zeros((3, 3))
    for c in range(3):
        M = np.zeros(3 * n)
        M[c * n:(c + 1) * n] = 1.0
        NM = N @ M
        for r in range(3):
            T[r, c] = float(NM[r * n:(r + 1) * n] @ V) / V.sum()
    return T


def test_demag_trace_converges_to_one():
    errs = []
    for K, hs, ss in [(2, 7, 3), (3, 10, 5)]:
        m = synth.layered_island_mesh(8, 7, 3, rings=K, hard_slabs=hs, soft_slabs=ss, seed=1)
        ops = fem.MeshOperators(m.xyz_nm, m.tets, m.tet_region, synth.ecc_materials())
        T = _avg_tensor(ops.demag, ops.V)
        errs.append(abs(np.trace(T) - 1.0))
        assert abs(T[0, 0] - T[1, 1]) < 1e-3            # hexagonal symmetry
        assert np.abs(T - np.diag(np.diag(T))).max() < 2e-3
    assert errs[0] < 0.06 and errs[1] < errs[0] * 0.6, errs


def _polygon_self_potential_integral(poly):
    """int_P int_P dS dS' / |r - r'| for a convex polygon (CCW vertices):
    inner integral in closed form (edge sum of distance * log factor),
    outer by quadrature on a fan subdivision."""
    c = poly.mean(axis=0)
    tot = 0.0
    nv = poly.shape[0]
    for k in range(nv):
        a, b = poly[k], poly[(k + 1) % nv]
        for tri in _subdivide(np.append(c, 0.0), np.append(a, 0.0), np.append(b, 0.0), 2):
            p, w = _tri_rule(*tri, 10)
            p = p[:, :2]
            val = np.zeros(p.shape[0])
            for e in range(nv):
                ya, yb = poly[e], poly[(e + 1) % nv]
                s = np.linalg.norm(yb - ya)
                t = (yb - ya) / s
                nout = np.array([t[1], -t[0]])
                d = (ya - p) @ nout
                ra = np.linalg.norm(ya - p, axis=1)
                rb = np.linalg.norm(yb - p, axis=1)
                val += d * np.log((ra + rb + s) / (ra + rb - s))
            tot += float(w @ val)
    return tot


def _polygon_pair_integral(poly, L):
    c = poly.mean(axis=0)
    pts, wts = [], []
    nv = poly.shape[0]
    for k in range(nv):
        a, b = poly[k], poly[(k + 1) % nv]
        for tri in _subdivide(np.append(c, 0.0), np.append(a, 0.0), np.append(b, 0.0), 1):
            p, w = _tri_rule(*tri, 8)
            pts.append(p[:, :2])
            wts.append(w)
    p = np.concatenate(pts)
    w = np.concatenate(wts)
    d2 = ((p[:, None, :] - p[None, :, :]) ** 2).sum(-1)
    return float(w @ (1.0 / np.sqrt(d2 + L * L)) @ w)


def test_prism_magnetometric_factor_against_surface_charge_integral():
    m = synth.census_island_mesh()
    ops = fem.MeshOperators(m.xyz_nm, m.tets, m.tet_region, synth.ecc_materials())
    T = _avg_tensor(ops.demag, ops.V)
    K, n2 = m.info["rings"], m.info["nodes_per_plane"]
    poly = m.xyz_nm[1 + 3 * (K - 1) * K:n2, :2]
    L = m.height_nm
    V = synth.polygon_area_nm2(m) * L
    Nzz = (2 * _polygon_self_potential_integral(poly) - 2 * _polygon_pair_integral(poly, L)) / (4 * math.pi * V)
    assert 0.2 < Nzz < 0.35
    assert abs(T[2, 2] - Nzz) < 0.03 * Nzz, (T[2, 2], Nzz)
    assert abs(T[0, 0] - (1 - Nzz) / 2) < 0.03 * (1 - Nzz) / 2


def test_thin_film_limit():
    m = synth.layered_island_mesh(40.0, 0.5, 0.5, rings=6, hard_slabs=1, soft_slabs=1,
                                  seed=2, perturb=0.0)
    ops = fem.MeshOperators(m.xyz_nm, m.tets, m.tet_region, synth.ecc_materials())
    T = _avg_tensor(ops.demag, ops.V)
    K, n2 = m.info["rings"], m.info["nodes_per_plane"]
    poly = m.xyz_nm[1 + 3 * (K - 1) * K:n2, :2]
    L = m.height_nm
    V = synth.polygon_area_nm2(m) * L
    Nzz = (2 * _polygon_self_potential_integral(poly) - 2 * _polygon_pair_integral(poly, L)) / (4 * math.pi * V)
    assert Nzz > 0.9
    # one slab per layer of 3.3 nm x 0.5 nm elements: coarse, 7 % allowed
    assert abs(T[2, 2] - Nzz) < 0.07 * Nzz and T[0, 0] < 0.06, (T[2, 2], Nzz)


def test_demag_energy_positive(small_parts):
    _, ops, N, _ = small_parts
    rng = np.random.default_rng(1)
    W = np.tile(ops.V, 3)
    for _ in range(20):
        M = rng.standard_normal(3 * ops.n)
        assert M @ (W * (N @ M)) > 0
