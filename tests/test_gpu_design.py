"""The surrogate on the write-head and media design problem (12 design and 4
jitter inputs; labels from LLG batches of the 81-mesh geometry grid with the
moving head map and the layout's adjacent-track island).

* heads stacked side by side in one map give the islands the fields of their
  own heads: the state after 20 ps matches one map per head to 1e-4, and the
  switch outcomes after the full run agree;
* the network trained on LLG labels of random designs predicts fresh LLG
  solves of unseen designs and heads (accuracy, AUC, Brier score, and the
  per-design screened error rates against the LLG-counted rates);
* screening with it picks designs whose LLG-verified error rates are lower
  than those of random designs of the same population."""
import os

import numpy as np
import pytest

from paper_1603_09493_gb300 import _lib as L
from paper_1603_09493_gb300 import api, design, evolve, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not os.path.exists(L.LIB_PATH):
        from paper_1603_09493_gb300 import build
        build.build()
    c = api.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def grid(ctx):
    return design.upload_grid(ctx)


def test_stacked_heads_give_each_island_its_own_head(ctx, grid):
    Z = synth.counter_uniform(11, 0, np.arange(20 * 12)).reshape(20, 12)
    Z[:, design.KEYS.index("v_m_per_s")] = 0.6                       # one velocity level
    R = design.realisations(Z, 3, seed=12, first_index=0)             # 20 heads: 16 x 2 blocks
    p = design.run_params(float(R.v["v_m_per_s"][0]))
    hid = ctx.headmap_upload(design.head_stack(R.heads))
    tgt, adj = design.islands(R, grid, np.arange(len(R)))
    isl = synth.Islands.concat([tgt, adj])
    short = ctx.run_batch(isl, p, 200, map_id=hid)
    full = ctx.run_batch(isl, p, int(round(design.T_END_PS / 0.1)), map_id=hid)
    agree, worst = [], 0.0
    for h in range(len(R.heads)):
        rows = np.where(R.head == h)[0]
        one = design.Realisations(v={k: val[rows] for k, val in R.v.items()}, head=np.zeros(rows.size, np.int64),
                                  heads=R.heads[h:h + 1], ms=R.ms[rows], ku=R.ku[rows], tilt=R.tilt[rows],
                                  dx=R.dx[rows], X=R.X[rows])
        hid1 = ctx.headmap_upload(design.head_stack(one.heads))
        t1, a1 = design.islands(one, grid, np.arange(rows.size))
        isl1 = synth.Islands.concat([t1, a1])
        both = np.concatenate([rows, rows + len(R)])
        s1 = ctx.run_batch(isl1, p, 200, map_id=hid1)
        f1 = ctx.run_batch(isl1, p, int(round(design.T_END_PS / 0.1)), map_id=hid1)
        n1 = s1["m"].shape[-1]                  # the largest mesh of this head's islands
        assert not np.any(short["m"][both][:, :, n1:])
        worst = max(worst, float(np.abs(short["m"][both][:, :, :n1] - s1["m"]).max()))
        agree.append(np.mean(full["switched"][both] == f1["switched"]))
    print(f"stacked vs one map per head: max |dm| after 20 ps {worst:.2e}, outcome agreement {np.mean(agree):.4f}")
    assert worst <= 1e-4
    assert np.mean(agree) >= 0.98


def test_surrogate_on_the_design_problem(ctx, grid):
    X, Y, _ = design.training_set(ctx, grid, N=8192, n_heads=64, seed=31)
    Xh, Yh, Rh = design.training_set(ctx, grid, N=2048, n_heads=16, seed=32, first_index=10 ** 6)
    print(f"labels: target switched {Y[:, 0].mean():.3f}, adjacent flipped {Y[:, 1].mean():.3f}")
    assert 0.1 < Y[:, 0].mean() < 0.95 and Y[:, 1].mean() > 0.01   # both events occur
    sizes = [16, 256, 256, 256, 256, 2]
    sur = ctx.surrogate((16, 256, 4, 2), synth.mlp_init_params(sizes, seed=6))
    try:
        curve = sur.train(X, Y, epochs=60, batch=512, lr=2e-3, weight_decay=1e-4)
        assert curve[-16:].mean() < 0.6 * curve[:16].mean()
        P = sur.infer(Xh)
        mt = design.metrics(P[:, 0], Yh[:, 0])
        ma = design.metrics(P[:, 1], Yh[:, 1])
        print("held-out target:", mt)
        print("held-out adjacent:", ma)
        base = max(Yh[:, 0].mean(), 1 - Yh[:, 0].mean())
        assert mt["accuracy"] >= base + 0.1 and mt["auc"] >= 0.85
        assert ma["auc"] >= 0.8
        # per-design screened rates against LLG-counted rates over the same 32 realisations
        D, J = 48, 32
        Zd = synth.counter_uniform(33, 0, np.arange(D * 12)).reshape(D, 12)
        Rd = design.realisations(Zd, J, seed=34, first_index=0)
        screened = sur.screen(Rd.X, D, J)
        counted = evolve.error_rates(design.llg_labels(ctx, grid, Rd), D, J)
        err = np.abs(screened - counted)
        print(f"screened vs LLG-counted rates over {D} designs x {J}: mean |d| {err.mean(0)}, max {err.max(0)}")
        assert err[:, 0].mean() <= 0.1 and err[:, 1].mean() <= 0.1
        # screening gain: the 8 best-screened of the 48 designs against 8 of them taken at random
        obj = screened.sum(1)
        pick = np.argsort(obj, kind="stable")[:8]
        rnd = np.arange(D)[::6][:8]
        print(f"LLG objective of the screened picks {counted[pick].sum(1).mean():.3f}, "
              f"of random designs {counted[rnd].sum(1).mean():.3f}")
        assert counted[pick].sum(1).mean() < counted[rnd].sum(1).mean()
    finally:
        sur.destroy()


def test_critical_field_ber_of_designs_matches_oracle(ctx, grid):
    # the write and previous-bit BERs (Sec. II.C, Eqs. 1-2) of three designs that share a mesh
    # and a velocity level, each under its own head in one stacked map: the library's
    # critical-field search against the oracle's (stored by tests/golden/make_headline_golden.py
    # design-ber) on the same islands, map and step count; both take every decision from switch
    # outcomes, so the critical fields agree to one finest-grid step sigma/8
    import sys
    sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
    ref = np.load(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "design_ber.npz"))
    Z = design.parity_designs()
    assert np.allclose(Z, ref["Z"])
    k = int(ref["k"])
    for r, role in enumerate(("targ", "prev")):
        tgt, direction, sigma, R = design.critical_field_inputs(Z, role)
        assert np.allclose(sigma, ref["sigma_T"], rtol=1e-12)
        if role == "targ":      # the library's count for the strongest field of the grid is the oracle's
            probe = tgt.subset(np.arange(3))
            probe.mesh_id = np.asarray(grid, np.int32)[probe.mesh_id]
            probe.Hext_T = (4.0 * sigma[:, None] * direction).astype(np.float32)
            hid = ctx.headmap_upload(design.head_stack(R.heads))
            assert ctx.stable_substeps(probe, design.run_params(float(R.v["v_m_per_s"][0])), hid)[0] == k
        got = design.critical_field_ber(ctx, grid, Z, role, precision=L.PREC_BF16X3, substeps=k)
        print(role, "gpu H_crit/sigma", got.h_crit_T / sigma, "BER", got.ber,
              "oracle", ref["h_crit_T"][r] / sigma, ref["ber"][r])
        assert np.array_equal(got.aborted, ref["aborted"][r])
        assert np.all(np.abs(got.h_crit_T - ref["h_crit_T"][r]) <= sigma / 8 + 1e-12)
