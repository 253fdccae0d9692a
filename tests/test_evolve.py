"""Host logic of the surrogate-assisted design search (no GPU): the mutation and
selection operator, the jitter samples, the error rates, and the generational
loop run against a closed-form switching rule in place of the LLG solver and
the surrogate."""
import numpy as np
import pytest

from paper_1603_09493_gb300 import evolve, synth


def test_next_population_layout_and_bounds():
    cfg = evolve.SearchConfig(population=64, top_k=8, seed=4)
    elite = synth.counter_uniform(9, 0, np.arange(8 * 4)).reshape(8, 4)
    Z = evolve.next_population(elite, 64, 3, cfg)
    assert Z.shape == (64, 4) and np.all((Z >= 0.0) & (Z <= 1.0))
    assert np.array_equal(Z[:8], elite)                                     # elites first
    n_fresh = int(round(cfg.fresh * 64))
    mut = Z[8:64 - n_fresh]
    step = cfg.sigma_mut * cfg.decay ** 3
    parents = elite[np.arange(len(mut)) % 8]
    assert np.abs(mut - parents).max() <= 6.0 * step                        # reflection keeps steps short
    assert np.array_equal(evolve.next_population(elite, 64, 3, cfg), Z)     # keyed by (seed, generation)
    assert not np.array_equal(evolve.next_population(elite, 64, 4, cfg)[8:], Z[8:])
    with pytest.raises(ValueError):
        evolve.next_population(elite, 9, 1, cfg)             # 8 elites + 2 fresh > 9


def test_samples_are_design_major_with_the_fringe_field():
    Z = np.array([[0.5, 0.5, 1.0, 1.0], [0.0, 1.0, 0.0, 0.0]])
    J = 4000
    tgt, adj, X = evolve.samples(Z, J, seed=1, first_index=0)
    assert X.shape == (2 * J, 16) and len(tgt.Ms_scale) == 2 * J
    assert np.allclose(adj.Hext_T, evolve.FRINGE * tgt.Hext_T, rtol=1e-6, atol=0)
    for f in ("Ms_scale", "Ku_scale", "u", "pos_nm"):
        assert np.array_equal(getattr(adj, f), getattr(tgt, f))
    # design 0: field 1.05 T along 180 degrees; design 1: 0.55 T along 160 degrees
    assert np.allclose(np.linalg.norm(tgt.Hext_T[:J], axis=1), 1.05, rtol=1e-6)
    assert np.allclose(tgt.Hext_T[J:, 0] / 0.55, np.sin(np.deg2rad(160.0)), rtol=1e-5)
    assert np.all(X[:J, 6] == 1.0) and np.all(X[J:, 6] == -1.0) and np.all(X[:, 8:] == 0.0)
    # jitter about the design values: Ms 3 %, Ku 7 %
    ms, ku = tgt.Ms_scale.reshape(2, J), tgt.Ku_scale.reshape(2, J)
    assert abs(ms[0].mean() - 1.0) < 0.003 and abs(ms[0].std() / 1.0 - evolve.JITTER["Ms"]) < 0.003
    assert abs(ku[1].mean() - 1.25) < 0.005 and abs(ku[1].std() / 1.25 - evolve.JITTER["Ku"]) < 0.004


def test_error_rates():
    Y = np.array([[1, 0], [0, 0], [1, 1], [1, 0], [1, 1], [1, 1]], np.float32)   # 2 designs x 3 samples
    r = evolve.error_rates(Y, 2, 3)
    assert np.allclose(r, [[1 / 3, 1 / 3], [0.0, 2 / 3]])


def _rule(tgt):
    # closed-form stand-in: an island switches when its field exceeds 0.8 T x Ku scale
    return np.linalg.norm(tgt.Hext_T, axis=1) > 0.8 * tgt.Ku_scale


class _FakeSurrogate:
    def screen(self, X, D, J):
        lo, hi = synth.SCREEN_RANGES["Ku_scale"]
        ku = lo + (hi - lo) * (X[:, 1] + 1.0) / 2.0
        lo, hi = synth.SCREEN_RANGES["B_ext_T"]
        b = lo + (hi - lo) * (X[:, 6] + 1.0) / 2.0
        Y = np.stack([b > 0.8 * ku, evolve.FRINGE * b > 0.8 * ku], 1).astype(np.float32)
        return evolve.error_rates(Y, D, J)


def test_search_loop_against_a_closed_form_rule(monkeypatch):
    monkeypatch.setattr(evolve, "llg_outcomes",
                        lambda ctx, mid, p, tgt, adj: np.stack([_rule(tgt), _rule(adj)], 1).astype(np.float32))
    cfg = evolve.SearchConfig(generations=4, population=64, top_k=8, n_jitter_screen=16, n_jitter_verify=16, seed=7)
    res = evolve.search(None, _FakeSurrogate(), 0, cfg)
    best = [h["best_verified"] for h in res.history]
    assert all(b1 <= b0 for b0, b1 in zip(best, best[1:]))                  # elitism
    assert best[-1] <= 1.0 / 16                                             # a design inside the window
    assert res.best_rates.sum() == best[-1]
    # the first generation verifies 8 of 64; later ones 8 of the 56 that are not elites
    assert res.verified_islands == 4 * 2 * 8 * 16
    assert res.llg_only_islands == 2 * 16 * (64 + 3 * 56)
