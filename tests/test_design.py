"""Host logic of the surrogate's design problem (no GPU): the parameter grid and
its meshes, the stacked head map, the realisations' layout and features, the
island positions of each track layout, and the screening metrics."""
import math

import numpy as np
import pytest

from paper_1603_09493_gb300 import design, synth


def test_values_snap_the_gridded_parameters_and_scale_the_rest():
    Z = synth.counter_uniform(3, 0, np.arange(500 * 12)).reshape(500, 12)
    v = design.values(Z)
    for k, key in enumerate(design.KEYS):
        lo, hi = design.RANGES[key]
        assert np.all(v[key] >= lo - 1e-12) and np.all(v[key] <= hi + 1e-12), key
        if key in design.LEVELS:
            lev = np.asarray(design.LEVELS[key])
            assert np.all(np.isin(v[key], lev)), key
            cell = np.minimum((Z[:, k] * len(lev)).astype(int), len(lev) - 1)
            assert np.array_equal(v[key], lev[cell])
        else:
            assert np.allclose(v[key], lo + (hi - lo) * Z[:, k])
    # the cell edges: 0 -> first level, 1 -> last level
    edge = design.values(np.vstack([np.zeros(12), np.ones(12)]))
    assert edge["v_m_per_s"][0] == 10.0 and edge["v_m_per_s"][1] == 30.0 and edge["layout"][1] == 2.0


def test_geometry_grid_order_thickness_and_top_height():
    meshes = design.grid_meshes()
    assert len(meshes) == 81
    v = {k: [] for k in design.GEOMETRY_KEYS}
    for d in design.LEVELS["diameter_nm"]:
        for ts in design.LEVELS["t_soft_nm"]:
            for th in design.LEVELS["t_hard_nm"]:
                for a in design.LEVELS["A_int_scale"]:
                    for key, val in zip(design.GEOMETRY_KEYS, (d, ts, th, a)):
                        v[key].append(val)
    idx = design.geometry_index({k: np.asarray(val) for k, val in v.items()})
    assert np.array_equal(idx, np.arange(81))
    for i, (m, mats) in enumerate(meshes):
        z = m.xyz_nm[:, 2]
        assert abs(z.max() - design.Z_TOP_NM) < 1e-12                       # top 5 nm below the ABS
        assert abs((z.max() - z.min()) - (v["t_soft_nm"][i] + v["t_hard_nm"][i])) < 1e-12
        assert abs(m.info["diameter_nm"] - v["diameter_nm"][i]) < 1e-12
        assert abs(mats[1, 2] - mats[0, 2] * v["A_int_scale"][i]) < 1e-24  # interlayer exchange scale


def test_head_stack_holds_each_head_in_its_own_block():
    rng = np.random.default_rng(2)
    heads = np.stack([rng.uniform(1.0, 1.6, 19), rng.uniform(10, 40, 19), rng.uniform(6, 12, 19)], 1)
    hm = design.head_stack(heads)
    assert hm.B_T.shape == (18, 16 * design.BLOCK_NM, 2 * design.BLOCK_NM, 3)   # 16 x 2 blocks
    assert np.allclose(hm.origin_nm, [-32.0, -32.0, 0.0])
    for h, (b, t, w) in enumerate(heads):
        bx, by = design.head_block(h)
        assert (bx, by) == (h // 16, h % 16)
        one = synth.synthetic_head_map(nx=64, ny=64, nz=18, B_peak_T=b, tilt_deg=t, sx_nm=w, sy_nm=w,
                                       z_top_nm=design.Z_TOP_NM)
        blk = hm.B_T[:, 64 * by:64 * (by + 1), 64 * bx:64 * (bx + 1)]
        assert np.array_equal(blk, one.B_T)
        # the peak of block h sits at its centre (index 32, 32), the field direction is the head's tilt
        iz, iy, ix = np.unravel_index(np.argmax(np.linalg.norm(blk, axis=-1)), blk.shape[:3])
        assert iy == 32 and ix == 32
        f = blk[iz, iy, ix]
        assert math.isclose(math.degrees(math.atan2(f[1], -f[2])), t, abs_tol=1e-4)
    with pytest.raises(ValueError):
        design.head_stack(np.ones((design.HEADS_PER_MAP + 1, 3)))


def test_realisations_are_design_major_with_bounded_features():
    D, J = 7, 5
    Z = synth.counter_uniform(4, 0, np.arange(D * 12)).reshape(D, 12)
    R = design.realisations(Z, J, seed=9, first_index=100)
    assert len(R) == D * J and R.X.shape == (D * J, 16)
    v = design.values(Z)
    for key in design.KEYS:
        assert np.allclose(R.v[key], np.repeat(v[key], J)), key
    assert np.array_equal(R.head, np.repeat(np.arange(D), J))
    assert np.all(np.abs(R.X[:, :12]) <= 1.0 + 1e-6)
    # jitter draws are keyed by (seed, index): the same rows give the same draws
    R2 = design.realisations(Z[2:3], J, seed=9, first_index=100 + 2 * J)
    assert np.array_equal(R2.ms, R.ms[2 * J:3 * J]) and np.array_equal(R2.dx, R.dx[2 * J:3 * J])
    # a pool of heads replaces the designs' own head parameters
    heads = np.array([[1.1, 12.0, 7.0], [1.5, 33.0, 9.0]])
    R3 = design.realisations(Z, 1, seed=9, first_index=0, heads=heads, head_of_design=np.arange(D) % 2)
    for k, key in enumerate(design.HEAD_KEYS):
        assert np.allclose(R3.v[key], heads[np.arange(D) % 2, k])
    lo, hi = design.RANGES["B_peak_T"]
    assert np.allclose(R3.X[:, design.KEYS.index("B_peak_T")], 2 * (R3.v["B_peak_T"] - lo) / (hi - lo) - 1)


def test_islands_sit_at_their_layout_offsets_in_their_head_block():
    D = 40                              # 40 heads: blocks in two down-track columns and a third
    Z = synth.counter_uniform(5, 0, np.arange(D * 12)).reshape(D, 12)
    R = design.realisations(Z, 2, seed=3, first_index=0)
    grid = list(range(1000, 1081))
    tgt, adj = design.islands(R, grid, np.arange(len(R)))
    v = R.v
    y0 = 64.0 * (R.head % 16)
    x0 = 64.0 * (R.head // 16)
    assert np.allclose(tgt.pos_nm[:, 0], x0 + R.dx, atol=1e-4) and np.allclose(tgt.pos_nm[:, 1], y0)
    p = v["pitch_nm"]
    lay = v["layout"].astype(int)
    want_x = x0 + R.dx + np.where(lay == 1, 0.5 * p, 0.0)
    want_y = y0 + np.where(lay == 2, -p, p)
    assert np.allclose(adj.pos_nm[:, 0], want_x, atol=1e-5) and np.allclose(adj.pos_nm[:, 1], want_y, atol=1e-4)
    assert np.array_equal(tgt.mesh_id, adj.mesh_id)
    assert np.array_equal(tgt.mesh_id, np.asarray(grid)[design.geometry_index(v)])
    assert np.allclose(tgt.Ms_scale, v["Ms_scale"] * R.ms, rtol=1e-6)
    assert np.allclose(np.linalg.norm(tgt.u, axis=1), 1.0, atol=1e-6)
    # every island stays within 21 nm of its block's centre (cross-track), inside the 64 nm block
    assert np.all(np.abs(adj.pos_nm[:, 1] - y0) <= 14.0 + 1e-6)


def test_metrics_against_brute_force():
    rng = np.random.default_rng(0)
    P = rng.uniform(size=300).round(2)                 # ties on purpose
    Y = (rng.uniform(size=300) < P).astype(float)
    m = design.metrics(P, Y)
    pos, neg = P[Y > 0.5], P[Y < 0.5]
    pairs = (pos[:, None] > neg[None, :]).sum() + 0.5 * (pos[:, None] == neg[None, :]).sum()
    assert math.isclose(m["auc"], pairs / (pos.size * neg.size), rel_tol=1e-12)
    assert math.isclose(m["accuracy"], np.mean((P > 0.5) == (Y > 0.5)))
    assert math.isclose(m["brier"], np.mean((P - Y) ** 2))


def _rule_labels(R):
    # closed-form stand-in for the LLG labels: the target is written when the head's peak field
    # beats the realisation's Ku factor times the design's Ku scale; the adjacent island flips when
    # the pitch is below 11 nm
    tgt = R.v["B_peak_T"] > 1.3 * R.v["Ku_scale"] * R.ku
    adj = R.v["pitch_nm"] < 11.0
    return np.stack([tgt, adj], 1).astype(np.float32)


class _RuleSurrogate:
    # screens with the same rule, read back from the features
    def screen(self, X, D, J):
        def val(key, col):
            lo, hi = design.RANGES[key]
            return lo + (hi - lo) * (X[:, col] + 1.0) / 2.0
        ku = 1.0 + 3 * design.JITTER["Ku"] * X[:, 13]
        tgt = val("B_peak_T", design.KEYS.index("B_peak_T")) > 1.3 * val("Ku_scale", 4) * ku
        adj = val("pitch_nm", 6) < 11.0
        from paper_1603_09493_gb300 import evolve
        return evolve.error_rates(np.stack([tgt, adj], 1).astype(np.float32), D, J)


def test_design_search_loop_against_a_closed_form_rule(monkeypatch):
    from paper_1603_09493_gb300 import evolve
    calls = []

    def fake_labels(ctx, grid, R, precision=None):
        calls.append(len(R))
        return _rule_labels(R)

    monkeypatch.setattr(design, "llg_labels", fake_labels)
    cfg = evolve.SearchConfig(generations=5, population=64, top_k=8, n_jitter_screen=16, n_jitter_verify=16, seed=7)
    res = design.search(None, _RuleSurrogate(), list(range(81)), cfg)
    best = [h["best_verified"] for h in res.history]
    assert all(b1 <= b0 for b0, b1 in zip(best, best[1:]))                  # elitism
    assert best[-1] <= 1.0 / 16 and res.best_rates.sum() == best[-1]
    v = design.values(res.best_Z[None])
    assert v["pitch_nm"][0] >= 11.0 and v["B_peak_T"][0] > 1.3 * v["Ku_scale"][0]
    assert calls == [8 * 16] * 5 and res.verified_islands == 5 * 2 * 8 * 16
    assert res.llg_only_islands == 2 * 16 * (64 + 4 * 56)
