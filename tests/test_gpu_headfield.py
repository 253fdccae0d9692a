"""The head-field solve of a saturated main pole (bpm_head_field_solve) against
the oracle's quadrature of the same charges (oracle/polefield.py), its device
output, its argument checks, and a recording run under the solved field."""
import os

import numpy as np
import pytest

from oracle import polefield
from paper_1603_09493_gb300 import _lib as L
from paper_1603_09493_gb300 import api, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not os.path.exists(L.LIB_PATH):
        from paper_1603_09493_gb300 import build
        build.build()
    c = api.Context(0)
    yield c
    c.close()


GEOMETRIES = [
    synth.pole_geometry(),
    synth.pole_geometry(pole_tip_width_nm=5.0, trailing_edge_angle_deg=45.0, side_edge_angle_deg=5.0, sul_image=0),
    synth.pole_geometry(pole_tip_width_nm=20.0, trailing_edge_angle_deg=5.0, side_edge_angle_deg=40.0,
                        abs_thickness_nm=35.0),
]


@pytest.mark.parametrize("k", range(len(GEOMETRIES)))
def test_pole_field_matches_oracle(ctx, k):
    g = GEOMETRIES[k]
    nx, ny, nz, h, org = 48, 40, 16, 1.0, (-36.0, -20.0, 0.0)
    hm = ctx.head_field(g, nx, ny, nz, h, org)
    assert hm.B_T.shape == (nz, ny, nx, 3)
    rng = np.random.default_rng(k)
    idx = np.stack([rng.integers(0, nx, 48), rng.integers(0, ny, 48), rng.integers(0, nz, 48)], 1)
    idx = np.concatenate([idx, [[36, 20, 15], [26, 20, 15], [36, 27, 15], [0, 0, 0]]])   # under the pole
    pts = np.asarray(org) + h * idx
    want = polefield.field(g, pts)
    got = hm.B_T[idx[:, 2], idx[:, 1], idx[:, 0]].astype(np.float64)
    err = float(np.abs(got - want).max())
    print(f"geometry {k}: max |B| {np.abs(want).max():.3f} T, max |dB| {err:.2e} T")
    assert err <= 1e-6
    assert want[-4:-2, 2].max() < -0.5                       # into the media under the pole


def test_device_output_equals_host(ctx):
    import torch
    g = GEOMETRIES[0]
    host = ctx.head_field(g, 64, 64, 16, 1.0, (-48.0, -32.0, 0.0))
    dev = torch.empty((16, 64, 64, 3), dtype=torch.float32, device="cuda")
    ctx.head_field(g, 64, 64, 16, 1.0, (-48.0, -32.0, 0.0), out=dev)
    assert np.array_equal(dev.cpu().numpy(), host.B_T)


def test_bad_geometry_and_grids_are_refused(ctx):
    g = GEOMETRIES[0]
    for bad in (dict(pole_tip_width_nm=0.0), dict(Js_T=-1.0), dict(trailing_edge_angle_deg=85.0),
                dict(taper_angle_deg=0.0), dict(z_sul_nm=20.0)):
        with pytest.raises(L.BpmError) as ei:
            ctx.head_field({**g, **bad}, 8, 8, 4, 1.0, (-4.0, -4.0, 0.0))
        assert ei.value.code == L.BPM_ERR_ARG
    for org, nz in (((-4.0, -4.0, 0.0), 17), ((-4.0, -4.0, -5.0), 4)):   # reaches the ABS; the under-layer
        with pytest.raises(L.BpmError):
            ctx.head_field(g, 8, 8, nz, 1.0, org)


def test_recording_under_the_solved_field(ctx):
    # the solved map drives a batch like any head map: islands that start under the pole tilt
    # towards -z, and stay finite and unit-length
    hm = ctx.head_field(synth.pole_geometry(), 64, 48, 16, 1.0, (-48.0, -24.0, 0.0))
    hid = ctx.headmap_upload(hm)
    mesh, mats = synth.small_island_mesh(), synth.ecc_materials()
    mid = ctx.mesh_upload(mesh, mats)
    isl = synth.jittered_islands(32, seed=9, mesh_id=mid)
    p = synth.RunParams(dt_ps=0.1, t_end_ps=50.0, alpha=0.1, rise_ps=20.0, use_map=True, x0_nm=10.0,
                        v_m_per_s=20.0, substeps=0)
    out = ctx.run_batch(isl, p, p.n_intervals, map_id=hid)
    assert np.all(out["status"] == 0)
    m = out["m"][:, :, :mesh.xyz_nm.shape[0]]
    assert np.allclose(np.linalg.norm(m, axis=1), 1.0, atol=1e-5)
    assert m[:, 2].mean() < 0.95


SHIELDED = synth.pole_geometry(trailing_shield_gap_nm=9.0, shield_thickness_nm=10.0, shield_panel_nm=6.0)


def test_trailing_shield_field_matches_oracle(ctx):
    # the trailing shield's boundary-element solve (same panels on both sides: the library's LU
    # in FP64 on the GPU against the oracle's dense solve) and the field of pole, shield and
    # their images against the oracle's quadrature
    nx, ny, nz, h, org = 48, 40, 16, 1.0, (-36.0, -20.0, 0.0)
    hm = ctx.head_field(SHIELDED, nx, ny, nz, h, org)
    rng = np.random.default_rng(5)
    idx = np.stack([rng.integers(0, nx, 24), rng.integers(0, ny, 24), rng.integers(0, nz, 24)], 1)
    idx = np.concatenate([idx, [[26, 20, 15], [38, 20, 15], [41, 20, 12], [45, 20, 15]]])
    pts = np.asarray(org) + h * idx
    want = polefield.field_with_shield(SHIELDED, pts)
    got = hm.B_T[idx[:, 2], idx[:, 1], idx[:, 0]].astype(np.float64)
    err = float(np.abs(got - want).max())
    print(f"with shield: max |B| {np.abs(want).max():.3f} T, max |dB| {err:.2e} T")
    assert err <= 1e-6
    # the shield turns the field at the trailing edge towards itself and weakens its
    # perpendicular part there; under the pole centre it changes little
    bare = polefield.field(SHIELDED, pts[-4:])
    assert want[-3, 0] > bare[-3, 0] + 0.05 and want[-3, 2] > bare[-3, 2] + 0.05
    assert abs(want[-4, 2] - bare[-4, 2]) < 0.1 * abs(bare[-4, 2])


def test_wrap_around_shield_matches_oracle(ctx):
    # trailing and side shields as one equipotential body, against the oracle's solve
    g = dict(SHIELDED, side_shield_gap_nm=16.0)
    nx, ny, nz, h, org = 48, 40, 16, 1.0, (-36.0, -20.0, 0.0)
    hm = ctx.head_field(g, nx, ny, nz, h, org)
    rng = np.random.default_rng(6)
    idx = np.stack([rng.integers(0, nx, 16), rng.integers(0, ny, 16), rng.integers(0, nz, 16)], 1)
    idx = np.concatenate([idx, [[38, 32, 15], [30, 38, 12]]])
    pts = np.asarray(org) + h * idx
    want = polefield.field_with_shield(g, pts)
    got = hm.B_T[idx[:, 2], idx[:, 1], idx[:, 0]].astype(np.float64)
    err = float(np.abs(got - want).max())
    print(f"wrap-around shield: max |B| {np.abs(want).max():.3f} T, max |dB| {err:.2e} T")
    assert err <= 1e-6


def test_trailing_shield_at_default_panels(ctx):
    # the default 2 nm panels (over four thousand unknowns): the solve passes its residual check
    # and converges to the 6 nm panels' field within the discretisation error
    fine = synth.pole_geometry(trailing_shield_gap_nm=9.0, shield_thickness_nm=10.0)
    a = ctx.head_field(fine, 48, 40, 16, 1.0, (-36.0, -20.0, 0.0)).B_T
    b = ctx.head_field(SHIELDED, 48, 40, 16, 1.0, (-36.0, -20.0, 0.0)).B_T
    assert np.all(np.isfinite(a))
    assert np.abs(a - b).max() <= 0.05 * np.abs(a).max()
    assert not np.array_equal(a, ctx.head_field(synth.pole_geometry(), 48, 40, 16, 1.0, (-36.0, -20.0, 0.0)).B_T)
