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
