"""Host-side rules of the library and the binding (no GPU): the integrator step
count is the smallest k with gamma/(1 + alpha^2) B dt / k <= 1/2 (the
explicit-step bound Heun's method needs on the precession frequency), computed
by the library itself (bpm_substeps_for_bound, host arithmetic); the
critical-field search of Sec. II.C makes the oracle search's decisions when
both see the same outcomes."""
import math
import os

import numpy as np
import pytest

from paper_1603_09493_gb300 import _lib as L
from paper_1603_09493_gb300 import api


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(L.LIB_PATH):
        from paper_1603_09493_gb300 import build
        build.build()
    return L.load()


def test_library_step_count_is_the_smallest_admissible_count(lib):
    gamma = 1.76085963023e-1                                 # rad / (ps T)
    rng = np.random.default_rng(0)
    for B, dt, alpha in zip(rng.uniform(0.01, 500.0, 200), rng.uniform(0.01, 1.0, 200), rng.uniform(0.0, 1.0, 200)):
        k = api.substeps_for_bound(B, dt, alpha)
        rate = gamma / (1.0 + alpha * alpha) * B * dt
        assert k >= 1 and rate / k <= 0.5 * (1 + 1e-12)
        assert k == 1 or rate / (k - 1) > 0.5
    # the census numbers: 28 steps per 0.1 ps at alpha 0.1 for a bound near 800 T (the exchange spectrum)
    assert api.substeps_for_bound(800.0, 0.1, 0.1) == 28
    assert api.substeps_for_bound(0.0, 0.1, 0.1) == 1
    assert api.substeps_for_bound(1.0, 0.1, 0.0) == math.ceil(gamma * 0.1 / 0.5)
    # the same rule as the oracle's, on the oracle's own bound of a batch
    from oracle import fem, llg
    from paper_1603_09493_gb300 import synth
    mesh = synth.small_island_mesh()
    ops = fem.MeshOperators(mesh.xyz_nm, mesh.tets, mesh.tet_region, synth.ecc_materials(), with_demag=False)
    for seed, alpha in ((1, 0.1), (2, 0.02), (3, 1.0)):
        isl = synth.jittered_islands(64, seed=seed)
        p = synth.RunParams(dt_ps=0.1, alpha=alpha, use_map=False, uniform_T=synth.uniform_field(0.5, 170.0))
        b = llg.Batch(ops, isl, p, demag=np.zeros((1, 1)))
        assert api.substeps_for_bound(llg.field_bound(b), p.dt_ps, alpha) == llg.stable_substeps(b)
    # arguments outside the rule's domain are refused
    k = ctypes_int()
    for args in ((-1.0, 0.1, 0.1), (1.0, 0.0, 0.1), (1.0, 0.1, -0.5)):
        assert lib.bpm_substeps_for_bound(*args, k) == L.BPM_ERR_ARG


def ctypes_int():
    import ctypes
    return ctypes.byref(ctypes.c_int32())


def _threshold_rule(isl, role):
    # closed-form stand-in for the LLG switched flags: the bad outcome starts once |H_ext| reaches
    # the island's threshold (carried in Ku_scale, in tesla); bad is "not switched" for the target
    # bit and "switched" for the previous bit
    h = np.linalg.norm(isl.Hext_T.astype(np.float64), axis=1)
    bad = h >= isl.Ku_scale.astype(np.float64)
    return ~bad if role == "targ" else bad                  # targ: good = switched; prev: good = not


def test_critical_field_search_matches_the_oracle_search(monkeypatch):
    from oracle import hcrit as ohcrit
    from paper_1603_09493_gb300 import hcrit, synth

    sigma = np.array([0.04] * 10)
    # thresholds in units of sigma: inside the grid, on grid points, at 0 (abort), beyond 4 sigma
    tau = sigma * np.array([0.0, 0.3, 0.5, 1.0, 1.37, 2.25, 3.9, 4.0, 4.2, 7.0])
    rng = np.random.default_rng(1)
    direction = rng.standard_normal((10, 3))
    direction /= np.linalg.norm(direction, axis=1, keepdims=True)
    isl = synth.nominal_islands(10)
    isl.Ku_scale = tau.astype(np.float32)
    for role in ("targ", "prev"):
        class FakeBatch:
            def __init__(self, ops, sub, params, head_map=None):
                self.sub = sub

            def run(self):
                return {"switched": _threshold_rule(self.sub, role)}

        monkeypatch.setattr(ohcrit, "Batch", FakeBatch)
        h_o, ber_o, ab_o = ohcrit.search(None, isl, None, direction, sigma, role)
        res = hcrit.critical_field_search(lambda sub, designs: _threshold_rule(sub, role), isl, direction, sigma,
                                          role)
        assert np.array_equal(res.aborted, ab_o) and np.array_equal(res.h_crit_T, h_o)
        # the same Gaussian tail, erfc on one side and 1 - erf on the other: equal up to the
        # cancellation of 1 - erf at 4 sigma (~3e-12 relative)
        assert np.allclose(res.ber, ber_o, rtol=1e-9, atol=0)
        assert res.aborted.tolist() == [True] + [False] * 9 and np.all(res.ber[0] == 1.0)
        # the last good field brackets the threshold to sigma/8 (two halvings of sigma/2); none past 4 sigma
        inside = (tau > 0) & (tau <= 4.0 * sigma)
        assert np.all(res.h_crit_T[inside] < tau[inside] + 1e-12)
        assert np.all(res.h_crit_T[inside] >= tau[inside] - sigma[inside] / 8 - 1e-12)
        assert np.all(res.h_crit_T[tau > 4.0 * sigma] == 4.0 * sigma[tau > 4.0 * sigma])


def test_error_rate_formulas_match_the_oracle():
    # Eqs. 1-3 as the product computes them against the oracle's own statements of them
    import math

    from oracle import ber as ober
    from oracle import neb as oneb
    from paper_1603_09493_gb300 import adjacent, hcrit

    for K1, Js in ((0.9e6, 1.0), (1.5e6, 0.8), (3.0e5, 1.2)):
        assert math.isclose(hcrit.sfd_sigma_T(K1, Js), ober.sfd_sigma_T(K1, Js), rel_tol=1e-15)
    for mult in np.linspace(0.0, 6.0, 25):
        s = 0.035
        # the oracle states Eq. 1 as 1 - erf, exact to ~1e-16 absolute; the product uses erfc
        assert math.isclose(hcrit.ber_from_hcrit(mult * s, s), ober.ber_from_hcrit(mult * s, s), rel_tol=1e-9,
                            abs_tol=1e-15)
    E_J = np.linspace(10.0, 80.0, 15) * 1.380649e-23 * 300.0      # 10 .. 80 kT at 300 K
    got = adjacent.ber_adj(E_J)
    ref = np.array([ober.ber_adj(float(x)) for x in oneb.barrier_kT(E_J)])
    assert np.allclose(got, ref, rtol=1e-12, atol=0)
    for b, e in zip(got, oneb.barrier_kT(E_J)):
        assert math.isclose(adjacent.barrier_kT_from_ber(float(b)), float(e), rel_tol=1e-12)
    assert adjacent.ber_tot(1e-4, 2e-5, 3e-6) == ober.ber_tot(1e-4, 2e-5, 3e-6)


def test_ego_loop_makes_the_oracle_loops_choices(monkeypatch):
    # the product's EGO loop (theta search, search set, EI argmax, bookkeeping) with its likelihood
    # and kriging calls answered by the oracle: it must propose exactly the oracle loop's designs
    from oracle import ego as oego
    from paper_1603_09493_gb300 import ego, synth

    class OracleKriging:
        def __init__(self, ctx, X, y, theta, nugget=1e-10):
            self.gp = oego.fit(np.asarray(X, float), np.asarray(y, float), np.asarray(theta, float), nugget)

        def predict(self, C, f_min):
            return oego.predict(self.gp, np.asarray(C, float), f_min)

        def __enter__(self):
            return self

        def __exit__(self, *exc):
            pass

    monkeypatch.setattr(ego, "nll", lambda ctx, X, y, th, nugget=1e-10:
                        np.array([oego.nll(np.asarray(X, float), np.asarray(y, float), t, nugget)
                                  for t in np.asarray(th, float)]))
    monkeypatch.setattr(ego, "Kriging", OracleKriging)
    C = synth.lhs_candidates(20, 12, 2, seed=3)
    X0 = C[oego.maximin_select(C)[0]]
    draws = lambda it: [synth.theta_unit_draws(16, 2, 5 + it, r) for r in range(3)]
    cands = lambda it: (synth.unit_points(300, 2, 6, 2 * it), synth.unit_points(300, 2, 6, 2 * it + 1))
    X, y, hist = ego.ego(None, synth.branin01, X0, synth.branin01(X0), 5, draws, cands)
    Xo, yo, histo = oego.ego(synth.branin01, X0, synth.branin01(X0), 5, draws, cands)
    assert np.array_equal(X, Xo) and np.array_equal(y, yo)
    for (t, e), (to, eo) in zip(hist, histo):
        assert np.array_equal(t, to) and e == eo


def test_a_missing_library_fails_loudly(monkeypatch, tmp_path):
    # no CPU fallback: without the built library the binding raises before any work
    import pytest

    from paper_1603_09493_gb300 import _lib as L
    monkeypatch.setattr(L, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        L.load(str(tmp_path / "libbpmllg.so"))
