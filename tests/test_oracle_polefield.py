"""The oracle's field of a saturated main pole (oracle/polefield.py) against
what the mathematics fixes: a uniformly magnetised rectangular prism has a
closed-form field (its two charged faces, each a sum of arctangents and
logarithms over the corners, written out here from the integral); far from
the pole the field is that of a point dipole of moment Js V; the under-layer
image makes the field normal to the under-layer surface; the pole is
mirror-symmetric across y = 0; and the quadrature has converged."""
import math

import numpy as np
import pytest

from oracle import polefield
from paper_1603_09493_gb300 import synth


def _rect(x1, x2, y1, y2, zf, P):
    # int over the rectangle [x1, x2] x [y1, y2] at height zf of (P - Q) / |P - Q|^3 dA
    out = np.zeros(3)
    z = P[2] - zf
    for i, u in enumerate((P[0] - x1, P[0] - x2)):
        for j, v in enumerate((P[1] - y1, P[1] - y2)):
            R = math.sqrt(u * u + v * v + z * z)
            lv = math.log(v + R) if v >= 0 else math.log((u * u + z * z) / (R - v))
            lu = math.log(u + R) if u >= 0 else math.log((v * v + z * z) / (R - u))
            out += (-1) ** (i + j) * np.array([-lv, -lu, math.atan(u * v / (z * R))])
    return out


def _prism_field(w, D, H, z0, Js, P):
    # m = -z: the bottom face carries +Js, the top face -Js (as mu0 sigma)
    c = Js / (4 * math.pi)
    return c * (_rect(-D, 0.0, -w / 2, w / 2, z0, P) - _rect(-D, 0.0, -w / 2, w / 2, z0 + H, P))


def _box_geometry(**kw):
    return synth.pole_geometry(trailing_edge_angle_deg=0.0, side_edge_angle_deg=0.0, taper_angle_deg=90.0,
                               sul_image=0, **kw)


def test_rectangular_prism_matches_closed_form():
    g = _box_geometry(pole_tip_width_nm=12.0, abs_thickness_nm=20.0, yoke_edge_nm=60.0)
    rng = np.random.default_rng(0)
    pts = np.stack([rng.uniform(-40, 25, 24), rng.uniform(-25, 25, 24), rng.uniform(-10, 15, 24)], 1)
    pts = np.concatenate([pts, [[-10.0, 0.0, 15.0], [0.0, 6.0, 14.0], [-25.0, 10.0, 90.0]]])  # near edges, beside
    got = polefield.field(g, pts)
    want = np.array([_prism_field(12.0, 20.0, 60.0, g["z_abs_nm"], 2.4, p) for p in pts])
    scale = np.abs(want).max()
    assert scale > 0.5                                      # near the ABS the field is of order Js/2
    assert np.abs(got - want).max() <= 1e-9 * scale


def _signed_volume(tris):
    return sum(np.dot(a, np.cross(b, c)) for a, b, c in tris) / 6.0


def test_far_field_is_the_dipole_of_moment_Js_V():
    g = synth.pole_geometry(sul_image=0)
    tris, _ = polefield.pole_triangles(g)
    V = _signed_volume(tris)
    assert V > 0                                            # outward winding
    # volume of the prism-like pole against the box bound: positive and below the bounding box
    assert V < 200 * 120 * 153
    centre = np.mean(tris.reshape(-1, 3), axis=0)
    m = np.array([0.0, 0.0, -2.4 * V])                      # mu0 m, T nm^3
    for d in ([1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, -1], [-2, 1, 3]):
        rhat = np.array(d, float) / np.linalg.norm(d)
        r = 1.0e6                                           # the next multipole is ~ size / r = 1e-4
        P = centre + r * rhat
        want = (3 * np.dot(m, rhat) * rhat - m) / (4 * math.pi * r ** 3)
        got = polefield.field(g, P[None])[0]
        assert np.linalg.norm(got - want) <= 1e-3 * np.linalg.norm(want)


def test_under_layer_image_makes_the_field_normal_to_it():
    g = synth.pole_geometry()
    xs = np.linspace(-30, 20, 5)
    pts = np.array([[x, y, g["z_sul_nm"]] for x in xs for y in (-12.0, 0.0, 7.0)])
    B = polefield.field(g, pts)
    assert np.abs(B[:, 2]).max() > 0.05
    assert np.abs(B[:, :2]).max() <= 1e-9 * np.abs(B[:, 2]).max()
    # without the image the same points see a tangential field
    B0 = polefield.field({**g, "sul_image": 0}, pts)
    assert np.abs(B0[:, :2]).max() > 1e-2


def test_mirror_symmetry_and_convergence():
    g = synth.pole_geometry()
    rng = np.random.default_rng(1)
    pts = np.stack([rng.uniform(-30, 20, 8), rng.uniform(1, 20, 8), rng.uniform(0, 15, 8)], 1)
    B = polefield.field(g, pts)
    Bm = polefield.field(g, pts * np.array([1, -1, 1]))
    assert np.allclose(Bm, B * np.array([1, -1, 1]), rtol=0, atol=1e-10)
    # under the pole the field points into the media and the under-layer doubles it roughly
    under = polefield.field(g, np.array([[-5.0, 0.0, 10.0]]))[0]
    alone = polefield.field({**g, "sul_image": 0}, np.array([[-5.0, 0.0, 10.0]]))[0]
    assert under[2] < alone[2] < 0
    # a finer subdivision changes nothing
    tris, q = polefield.pole_triangles(g)
    P = np.array([-3.0, 2.0, 14.5])
    fine = sum(c / (4 * math.pi) * polefield._coulomb(t, P, ratio=0.1) for t, c in zip(tris, q))
    assert np.abs(fine - polefield.field(g, P[None])[0]).max() <= 1e-10


def test_geometry_readings():
    g = synth.pole_geometry()
    v = polefield.pole_vertices(g)
    w = g["pole_tip_width_nm"]
    # trailing edge w wide at x = 0 on the ABS, footprint narrowing at the taper angle
    assert v["trail_r"][1] - v["trail_l"][1] == pytest.approx(w)
    wl = v["lead_r"][1] - v["lead_l"][1]
    assert (w - wl) / 2 == pytest.approx(g["abs_thickness_nm"] / math.tan(math.radians(75.0)))
    # trailing face leans down-track, sides flare, by their angles over the yoke height
    H = g["yoke_edge_nm"]
    assert v["trail_r_top"][0] == pytest.approx(H * math.tan(math.radians(20.0)))
    assert v["trail_r_top"][1] - v["trail_r"][1] == pytest.approx(H * math.tan(math.radians(15.0)))
    tris, q = polefield.pole_triangles(g)
    assert tris.shape == (24, 3, 3) and np.allclose(q[12:], -q[:12])
    # the ABS triangles carry +Js, the yoke-edge ones -Js (the charge sheet)
    abs_tris = np.all(np.isclose(tris[:12, :, 2], g["z_abs_nm"]), axis=1)
    top_tris = np.all(np.isclose(tris[:12, :, 2], g["z_abs_nm"] + H), axis=1)
    assert np.allclose(q[:12][abs_tris], 2.4) and np.allclose(q[:12][top_tris], -2.4)


def test_closed_form_panel_potential_against_quadrature():
    # the oracle's closed-form panel potential (the shield solve's matrix entries) against the
    # quadrature of the same integral: on the triangle, beside it, above and below, far away
    rng = np.random.default_rng(3)
    for _ in range(4):
        tri = rng.uniform(-3, 3, (3, 3))
        cent = tri.mean(axis=0)
        n = np.cross(tri[1] - tri[0], tri[2] - tri[0])
        n /= np.linalg.norm(n)
        for P in (cent, cent + 0.3 * n, cent - 2.0 * n, tri[0] + 0.5 * (tri[1] - tri[0]) + 1e-3 * n,
                  tri[1] + 2.0 * (tri[1] - tri[2]), cent + 20.0 * rng.normal(size=3)):
            want = polefield._potential(tri, P, ratio=0.1)
            got = polefield.potential_closed(tri[None], P)[0]
            assert abs(got - want) <= 1e-9 * abs(want), (P, got, want)


def _icosphere(level, radius):
    t = (1 + math.sqrt(5)) / 2
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
         (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    v = [np.array(p, float) / np.linalg.norm(p) for p in v]
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4), (11, 10, 2),
         (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9), (4, 9, 5), (2, 4, 11),
         (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(level):
        cache, nf = {}, []

        def mid(i, j):
            key = (min(i, j), max(i, j))
            if key not in cache:
                m = v[i] + v[j]
                v.append(m / np.linalg.norm(m))
                cache[key] = len(v) - 1
            return cache[key]
        for a, b, c in f:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        f = nf
    tris = np.array([[radius * v[i] for i in tri] for tri in f])
    for k, tr in enumerate(tris):                      # outward winding
        if np.dot(np.cross(tr[1] - tr[0], tr[2] - tr[0]), tr.mean(axis=0)) < 0:
            tris[k] = tr[[0, 2, 1]]
    areas = 0.5 * np.linalg.norm(np.cross(tris[:, 1] - tris[:, 0], tris[:, 2] - tris[:, 0]), axis=1)
    return tris, areas


def test_soft_sphere_in_a_uniform_field():
    # a sphere of unbounded permeability in a uniform field B0 z: the surface is an equipotential
    # with no net charge, and the induced charge (3 B0 cos theta) has the dipole moment
    # 4 pi a^3 B0 (the field outside is B0 plus that dipole's); the error of the flat panels falls
    # with refinement
    a, B0 = 10.0, 0.5
    errs = []
    for level in (2, 3):
        tris, areas = _icosphere(level, a)
        cent = tris.mean(axis=1)
        q, Phi = polefield.bem_equipotential(tris, areas, -B0 * cent[:, 2])
        moment = (q[:, None] * areas[:, None] * cent).sum(axis=0)
        want = 4 * math.pi * a ** 3 * B0
        errs.append(abs(moment[2] - want) / want)
        assert abs(Phi) <= 1e-9 and np.abs(moment[:2]).max() <= 1e-6 * want
        assert abs((q * areas).sum()) <= 1e-9 * want / a
    print("sphere moment errors", errs)
    assert errs[0] / errs[1] > 3.0 and errs[1] <= 0.011    # second order in the panel size


def test_shield_interior_is_at_the_shield_potential():
    # the solved shield: inside a closed equipotential surface the potential is that constant;
    # the pole's potential plus the shield's (and the images') at interior points of the block
    g = synth.pole_geometry(trailing_shield_gap_nm=9.0, shield_thickness_nm=10.0, shield_panel_nm=3.0)
    tris, q, Phi = polefield.shield_charges(g)
    areas = polefield.shield_panels(g)[1]
    assert abs((q * areas).sum()) <= 1e-9 * np.abs(q * areas).sum()
    img = tris.copy()
    img[..., 2] = 2 * g["z_sul_nm"] - img[..., 2]
    img = img[:, [0, 2, 1]]
    tt = math.tan(math.radians(g["trailing_edge_angle_deg"]))
    inner = [np.array([9.0 + 15.0 + 5.0 * tt, y, g["z_abs_nm"] + 5.0]) for y in (-30.0, 0.0, 20.0)]
    pole_phi = polefield.pole_potential(g, np.array(inner))
    for P, pp in zip(inner, pole_phi):
        shield_phi = ((polefield.potential_closed(tris, P) - polefield.potential_closed(img, P)) * q).sum() / (4 * math.pi)
        assert abs(pp + shield_phi - Phi) <= 2e-3 * abs(Phi), (pp + shield_phi, Phi)
    # the pole drives the shield: its potential is not the under-layer's (zero)
    assert abs(Phi) > 0.1


def test_side_shields_join_the_equipotential_body():
    # trailing and side blocks form one body: the potential is the same constant inside each
    # block; its charges sum to zero; the side shields pull the fringing field at the adjacent
    # track (one cross-track pitch from the pole's centre, past the trailing edge)
    g = synth.pole_geometry(trailing_shield_gap_nm=9.0, side_shield_gap_nm=16.0, shield_thickness_nm=10.0,
                            shield_panel_nm=4.0)
    blocks = polefield.shield_blocks(g)
    assert len(blocks) == 3
    tris, q, Phi = polefield.shield_charges(g)
    areas = polefield.shield_panels(g)[1]
    assert abs((q * areas).sum()) <= 1e-9 * np.abs(q * areas).sum()
    img = tris.copy()
    img[..., 2] = 2 * g["z_sul_nm"] - img[..., 2]
    img = img[:, [0, 2, 1]]
    inner = [corner + 0.5 * (dx + dy + dz) for corner, dx, dy, dz in blocks]
    pole_phi = polefield.pole_potential(g, np.array(inner))
    for P, pp in zip(inner, pole_phi):
        v = pp + ((polefield.potential_closed(tris, P) - polefield.potential_closed(img, P)) * q).sum() / (4 * math.pi)
        assert abs(v - Phi) <= 3e-3 * abs(Phi), (P, v, Phi)
    # the side blocks clear the pole: inner faces the side gap outside the pole's flared sides
    corner, dx, dy, dz = blocks[1]
    assert corner[1] == pytest.approx(g["pole_tip_width_nm"] / 2 + 16.0)
    assert dz[1] / dz[2] == pytest.approx(math.tan(math.radians(g["side_edge_angle_deg"])))
    adj = np.array([[2.0, 11.7, 9.0]])
    with_sides = polefield.field_with_shield(g, adj)[0]
    trailing_only = polefield.field_with_shield(dict(g, side_shield_gap_nm=0.0), adj)[0]
    assert abs(with_sides[2]) < abs(trailing_only[2])
