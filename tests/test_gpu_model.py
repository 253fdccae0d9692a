"""The model evaluation of Fig. 4 on the GPU: a design's head field solved from its
Table I geometry, the critical-field searches of its target and previous bits,
the adjacent bit's barrier, and BER_tot; each part is tested against the oracle
in its own file, this one checks that they compose."""
import os

import numpy as np
import pytest

from paper_1603_09493_gb300 import _lib as L
from paper_1603_09493_gb300 import api, model

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not os.path.exists(L.LIB_PATH):
        from paper_1603_09493_gb300 import build
        build.build()
    c = api.Context(0)
    yield c
    c.close()


def _check(r):
    assert 0.0 < r["ber_tot"] <= 1.0 and 0.0 < r["ber_targ"] <= 1.0
    assert np.isclose(np.linalg.norm(r["direction"]), 1.0) and r["direction"][2] < 0      # into the media
    assert r["sigma_T"] == pytest.approx(0.015 * 2 * r["K1"] * 1e6 * 4e-7 * np.pi / 0.7)   # 0.015 H_A
    if r["aborted"]:
        assert r["ber_tot"] == 1.0 and r["ber_prev"] is None
    else:
        assert 0.0 <= r["ber_prev"] <= 1.0 and 0.0 <= r["ber_adj"] <= 1.0
        assert r["ber_tot"] == pytest.approx(min(1.0, r["ber_targ"] + r["ber_prev"] + r["ber_adj"]))
        assert np.isfinite(r["E_B_kT"])


def test_model_evaluation_composes(ctx):
    init = model.initial_design()
    soft = dict(init, K1_hard_MJ_m3=0.5, pole_tip_width_nm=20.0, A_ex_int_pJ_m=10.0)
    out = []
    for p in (init, soft):
        r = model.evaluate(ctx, p)
        r["K1"] = p["K1_hard_MJ_m3"]
        print({k: r[k] for k in ("ber_targ", "ber_prev", "ber_adj", "ber_tot", "h_crit_targ_sigma", "aborted")},
              r["seconds"])
        _check(r)
        out.append(r)
    # softer media under a wider pole cannot be harder to write
    assert out[1]["h_crit_targ_sigma"] * out[1]["sigma_T"] >= out[0]["h_crit_targ_sigma"] * out[0]["sigma_T"] - 1e-12
