"""Host logic of the model evaluation (Fig. 4) and its optimisation loop, without
a GPU: Table I's values, the readings of the media and the write window, and the
flow of one evaluation (abort when the target cannot be written, BER_tot as the
sum of the three rates) with closed-form stand-ins for the LLG outcomes and the
energy barrier."""
import math

import numpy as np
import pytest

from paper_1603_09493_gb300 import adjacent, model, synth


def test_table1_and_media_readings():
    p = model.initial_design()
    # Table I's initial design
    assert p["trailing_shield_gap_nm"] == 9.0 and p["trailing_edge_angle_deg"] == 20.0
    assert p["pole_tip_width_nm"] == 14.0 and p["pole_tip_taper_angle_deg"] == 75.0
    assert p["K1_hard_MJ_m3"] == 0.8 and p["A_ex_int_pJ_m"] == 2.0 and p["down_track_offset_nm"] == 6.8
    mesh, mats = model.media(p)
    z = mesh.xyz_nm[:, 2]
    assert z.min() == 0.0 and z.max() == 12.0
    assert np.isclose(np.ptp(mesh.xyz_nm[:, 0]), 12.0)
    ms = 0.7 / (4e-7 * math.pi)
    assert np.allclose(mats[:, 0], ms)
    assert mats[0, 1] == 0.8e6 and mats[2, 1] == pytest.approx(0.16e6)        # K1_soft = 0.2 K1_hard
    assert mats[1, 2] == pytest.approx(2e-12) and mats[0, 2] == 10e-12       # A_ex,int at the interface
    g = model.pole_geometry(p)
    assert g["z_abs_nm"] == 18.0 and g["z_sul_nm"] < 0.0                     # 6 nm above the island tops
    assert g["trailing_shield_gap_nm"] == 9.0 and g["shield_thickness_nm"] == 10.0
    assert g["side_shield_gap_nm"] == 16.0


def test_write_window_and_bit_positions():
    for off in (0.0, 4.0, 8.0):
        for layout in ("centered", "staggered", "shingled"):
            p = dict(model.initial_design(), down_track_offset_nm=off, cross_track_offset_nm=3.0)
            q = model.run_params(p)
            pos = model.bit_positions(p, layout)
            assert q.v_m_per_s < 0 and q.t_end_ps == pytest.approx(1000.0)    # 13.5 nm at 13.5 m/s
            x_end = q.x0_nm + q.v_m_per_s * 1e-3 * q.t_end_ps
            assert pos["targ"][0] - x_end == pytest.approx(off)              # past the trailing edge
            assert pos["prev"][0] - pos["targ"][0] == pytest.approx(model.DOWN_PITCH_NM)
            assert pos["targ"][1] == -3.0                                    # the head moved across
            assert abs(pos["adj"][1] - pos["targ"][1]) == pytest.approx(model.CROSS_PITCH_NM)
            nx, ny, nz, h, org = model.head_grid()
            for x, y in pos.values():       # every bit stays inside the head map during the window
                for xm in (x - q.x0_nm, x - x_end):
                    assert org[0] + 6 <= xm <= org[0] + h * (nx - 1) - 6
                assert org[1] + 6 <= y <= org[1] + h * (ny - 1) - 6
    u = np.array([0.0, 1.0, 0.5])
    keys = ["trailing_shield_gap_nm", "pole_tip_width_nm", "K1_hard_MJ_m3"]
    d = model.design_from_unit(u, keys)
    assert d["trailing_shield_gap_nm"] == 5.0 and d["pole_tip_width_nm"] == 20.0
    assert d["K1_hard_MJ_m3"] == pytest.approx(0.85) and d["A_ex_int_pJ_m"] == 2.0


class _FakeCtx:
    def head_field(self, g, nx, ny, nz, h, origin):
        B = np.zeros((nz, ny, nx, 3), np.float32)
        B[..., 2] = -1.0
        return synth.HeadMap(B_T=B, origin_nm=np.asarray(origin, np.float32), h_nm=h)

    def headmap_upload(self, hm):
        return 0

    def mesh_upload(self, mesh, mats):
        return 0

    def mesh_release(self, mid):
        pass

    def headmap_release(self, hid):
        pass


def test_evaluation_flow(monkeypatch):
    # stand-ins: the target switches unless H_ext opposes the head by more than 2.3 sigma, the
    # previous bit flips once H_ext along the head exceeds 1.1 sigma; the barrier is 55 kT
    p = model.initial_design()
    sigma = model.hcrit.sfd_sigma_T(p["K1_hard_MJ_m3"] * 1e6, model.JS_MEDIA_T)
    calls = []

    def runner(ctx, q, n, map_id=-1, precision=0):
        def run(isl, designs=None):
            h = isl.Hext_T @ np.array([0.0, 0.0, -1.0]) / sigma          # along the head field, in sigma
            calls.append(len(isl))
            target = isl.pos_nm[:, 0] < model.DOWN_PITCH_NM / 2          # the previous bit is a pitch on
            return np.where(target, h > -thr["targ"], h > thr["prev"])
        return run

    thr = {"targ": 2.3, "prev": 1.1}
    monkeypatch.setattr(model.hcrit, "gpu_flag_runner", runner)
    monkeypatch.setattr(model.adjacent, "barriers",
                        lambda ctx, isl, q, **kw: {"E_B_kT": np.array([55.0]),
                                                   "ber_adj": adjacent.ber_adj([55.0 * adjacent.KB * 300.0])})
    r = model.evaluate(_FakeCtx(), p)
    # the searches bracket the thresholds at sigma / 8 (grid sigma / 2, two refinements)
    assert r["h_crit_targ_sigma"] == pytest.approx(2.25) and r["h_crit_prev_sigma"] == pytest.approx(1.0)
    assert r["ber_targ"] == pytest.approx(0.5 * math.erfc(2.25 / math.sqrt(2)))
    assert r["ber_tot"] == pytest.approx(r["ber_targ"] + r["ber_prev"] + r["ber_adj"])
    assert r["ber_adj"] == pytest.approx(130e9 * 1e-9 * math.exp(-55.0))
    # a vanishing barrier: the Arrhenius rate exceeds 1 and is taken as 1
    monkeypatch.setattr(model.adjacent, "barriers",
                        lambda ctx, isl, q, **kw: {"E_B_kT": np.array([0.5]),
                                                   "ber_adj": adjacent.ber_adj([0.5 * adjacent.KB * 300.0])})
    r = model.evaluate(_FakeCtx(), p)
    assert r["ber_adj"] == 1.0 and r["ber_tot"] == 1.0
    assert np.allclose(r["direction"], [0, 0, -1]) and not r["aborted"]
    # a head that cannot write the target even without H_ext: BER_tot = 1, no further runs
    thr["targ"] = -1.0
    calls.clear()
    r = model.evaluate(_FakeCtx(), p)
    assert r["aborted"] and r["ber_tot"] == 1.0 and r["ber_prev"] is None and len(calls) == 1


def test_optimisation_loop_without_spread_explores(monkeypatch):
    # every design scoring BER_tot = 1 leaves nothing to fit: the loop takes space-filling steps
    # (each the candidate farthest from the designs so far) and never calls the kriging code
    keys = ["pole_tip_width_nm", "K1_hard_MJ_m3"]
    seen = []
    monkeypatch.setattr(model, "evaluate", lambda ctx, p, **kw: seen.append(p) or {"ber_tot": 1.0, "aborted": True})
    from paper_1603_09493_gb300 import ego
    monkeypatch.setattr(ego, "lhs_maximin", lambda ctx, C: (0, None))
    monkeypatch.setattr(ego, "ego", lambda *a, **k: (_ for _ in ()).throw(AssertionError("kriging on flat data")))
    res = model.optimise(None, keys, n_init=5, iters=3, seed=2)
    assert res["space_filling_steps"] == 3 and len(seen) == 8 and len(res["log10_ber_tot"]) == 8
    U = res["X"]
    for k in range(5, 8):       # each new point is the farthest candidate from the ones before it
        assert np.min(np.linalg.norm(U[:k] - U[k], axis=1)) > 0.05
