"""Surrogate-assisted design search over media and write-field parameters.

The paper optimises its write head and media with efficient global
optimisation (Sec. II.A), whose screening model is a Gaussian process.  This
loop puts the MLP surrogate in that place:

* a design is (Ms scale, Ku scale, write-field magnitude, write-field angle),
  drawn in the unit cube over `synth.SCREEN_RANGES`;
* every island of a design carries its own jitter of Ms, Ku, easy axis and
  position (Sec. II.C's switching-field distribution comes from such jitter);
* the two error events are those of Sec. II.C: the target island fails to
  switch (a write error), and an island of the adjacent track, which sees
  `FRINGE` times the write field, flips (an adjacent-track error);
* the objective of a design is the sum of the two error rates over its jitter.

Each generation the surrogate screens the whole population on fresh jitter
samples (`bpm_surrogate_screen`); only the `top_k` best-screened designs are
solved with the batched LLG path.  The best verified designs are kept (elitist
(mu + lambda) selection) and mutated into the next population, with a fraction
of fresh uniform draws; the mutation and selection operator is this module's,
not the paper's.  The LLG cost of solving every design of every generation is
reported beside the loop's, at the loop's own measured LLG rate."""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import _lib as L
from . import api, synth

DESIGN_KEYS = ("Ms_scale", "Ku_scale", "B_ext_T", "angle_deg")
JITTER = dict(Ms=0.03, Ku=0.07, tilt_deg=2.0, pos_nm=1.0)
FRINGE = 0.75          # the adjacent-track island sees this fraction of the write field


@dataclass
class SearchConfig:
    generations: int = 20
    population: int = 256
    top_k: int = 32
    n_jitter_screen: int = 64
    n_jitter_verify: int = 4096
    sigma_mut: float = 0.15      # mutation step in unit-cube coordinates, generation 0
    decay: float = 0.8           # per-generation factor of the mutation step
    fresh: float = 0.25          # fraction of every later population drawn afresh
    seed: int = 4


def design_values(Z) -> dict:
    """Unit-cube designs [D][4] -> physical values per key."""
    Z = np.asarray(Z, np.float64)
    out = {}
    for k, key in enumerate(DESIGN_KEYS):
        lo, hi = synth.SCREEN_RANGES[key]
        out[key] = lo + (hi - lo) * Z[:, k]
    return out


def samples(Z, n_jitter: int, seed: int, first_index: int, mesh_id: int = 0):
    """The jitter samples of designs Z [D][4], design-major ([D * n_jitter]):
    target islands, adjacent-track islands (the same island parameters under
    FRINGE times the field) and surrogate features X [D * n_jitter][16] (the
    realised parameters scaled by SCREEN_RANGES to [-1, 1], as in
    `synth.screening_designs`)."""
    v = design_values(Z)
    D, J = len(Z), int(n_jitter)
    idx = np.arange(first_index, first_index + D * J, dtype=np.uint64)
    rep = lambda a: np.repeat(np.asarray(a, np.float64), J)
    real = dict(Ms_scale=rep(v["Ms_scale"]) * (1.0 + JITTER["Ms"] * synth.counter_normal(seed, 500, idx)),
                Ku_scale=rep(v["Ku_scale"]) * (1.0 + JITTER["Ku"] * synth.counter_normal(seed, 501, idx)),
                tilt_x_deg=JITTER["tilt_deg"] * synth.counter_normal(seed, 502, idx),
                tilt_y_deg=JITTER["tilt_deg"] * synth.counter_normal(seed, 503, idx),
                pos_x_nm=JITTER["pos_nm"] * synth.counter_normal(seed, 504, idx),
                pos_y_nm=JITTER["pos_nm"] * synth.counter_normal(seed, 505, idx),
                B_ext_T=rep(v["B_ext_T"]), angle_deg=rep(v["angle_deg"]))
    tx, ty = np.deg2rad(real["tilt_x_deg"]), np.deg2rad(real["tilt_y_deg"])
    u = np.stack([np.tan(tx), np.tan(ty), np.ones(D * J)], 1)
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    a = np.deg2rad(real["angle_deg"])
    H = np.stack([real["B_ext_T"] * np.sin(a), np.zeros(D * J), real["B_ext_T"] * np.cos(a)], 1)
    mk = lambda field: synth.Islands(mesh_id=np.full(D * J, mesh_id, np.int32),
                                     Ms_scale=real["Ms_scale"].astype(np.float32),
                                     Ku_scale=real["Ku_scale"].astype(np.float32), u=u.astype(np.float32),
                                     pos_nm=np.stack([real["pos_x_nm"], real["pos_y_nm"]], 1).astype(np.float32),
                                     Hext_T=field.astype(np.float32))
    X = np.zeros((D * J, 16), np.float32)
    for k, (key, (lo, hi)) in enumerate(synth.SCREEN_RANGES.items()):
        X[:, k] = 2.0 * (real[key] - lo) / (hi - lo) - 1.0
    return mk(H), mk(FRINGE * H), X


def run_params(t_end_ps: float = 100.0) -> synth.RunParams:
    """Constant per-island field from t = 0, damping 0.1, no head map."""
    return synth.RunParams(dt_ps=0.1, t_end_ps=t_end_ps, alpha=0.1, rise_ps=0.0, use_map=False)


def llg_outcomes(ctx: api.Context, mesh_id: int, p: synth.RunParams, target, adjacent) -> np.ndarray:
    """LLG labels [N][2]: (target switched, adjacent island flipped), one batch."""
    isl = synth.Islands.concat([target, adjacent])
    p.substeps = ctx.stable_substeps(isl, p)[0]
    out = ctx.run_batch(isl, p, p.n_intervals, precision=L.PREC_BF16X3)
    if np.any(out["status"] != 0):
        raise RuntimeError("an island of the verification batch reported a failure")
    n = len(target.Ms_scale)
    return np.stack([out["switched"][:n], out["switched"][n:]], 1).astype(np.float32)


def error_rates(Y, n_designs: int, n_jitter: int) -> np.ndarray:
    """[D][2]: fraction of write errors (target not switched) and of adjacent flips."""
    Y = np.asarray(Y, np.float64).reshape(n_designs, n_jitter, 2)
    return np.stack([1.0 - Y[:, :, 0].mean(1), Y[:, :, 1].mean(1)], 1)


def next_population(elite_Z, P: int, gen: int, cfg: SearchConfig) -> np.ndarray:
    """Elites first, then Gaussian mutants of the elites in turn (step
    sigma_mut * decay^gen, reflected into the unit cube), then fresh uniform
    draws; keyed by (seed, generation) only."""
    elite_Z = np.asarray(elite_Z, np.float64)
    K, d = elite_Z.shape
    n_fresh = int(round(cfg.fresh * P))
    n_mut = P - K - n_fresh
    if n_mut < 0:
        raise ValueError("population too small for the elites and the fresh draws")
    base = np.uint64(gen) * np.uint64(P * d)
    step = cfg.sigma_mut * cfg.decay ** gen
    noise = synth.counter_normal(cfg.seed, 600, base + np.arange(n_mut * d, dtype=np.uint64)).reshape(n_mut, d)
    mut = elite_Z[np.arange(n_mut) % K] + step * noise
    mut = np.abs(mut)                                  # reflect at 0 and at 1
    mut = np.where(mut > 1.0, 2.0 - mut, mut)
    mut = np.clip(mut, 0.0, 1.0)
    fresh = synth.counter_uniform(cfg.seed, 601, base + np.arange(n_fresh * d, dtype=np.uint64)).reshape(n_fresh, d)
    return np.concatenate([elite_Z, mut, fresh])


@dataclass
class SearchResult:
    best_Z: np.ndarray
    best_rates: np.ndarray           # verified (write error rate, adjacent flip rate) of the best design
    history: list = field(default_factory=list)
    screen_s: float = 0.0
    verify_s: float = 0.0
    verified_islands: int = 0
    llg_only_islands: int = 0

    @property
    def llg_only_s(self) -> float:
        """Time to solve every design of every generation with LLG, at the measured LLG rate."""
        return self.verify_s * self.llg_only_islands / max(self.verified_islands, 1)


def search(ctx: api.Context, sur: api.Surrogate, mesh_id: int, cfg: SearchConfig, t_end_ps: float = 100.0):
    """The generational loop; see the module docstring."""
    P, K, Js, Jv = cfg.population, cfg.top_k, cfg.n_jitter_screen, cfg.n_jitter_verify
    p = run_params(t_end_ps)
    Z = synth.counter_uniform(cfg.seed, 602, np.arange(P * 4, dtype=np.uint64)).reshape(P, 4)
    elite_Z = np.zeros((0, 4))
    elite_obj = np.zeros(0)
    elite_rates = np.zeros((0, 2))
    res = SearchResult(best_Z=None, best_rates=None)
    for g in range(cfg.generations):
        n_el = len(elite_Z)
        t0 = time.perf_counter()
        _, _, X = samples(Z, Js, cfg.seed + 1, first_index=g * P * Js, mesh_id=mesh_id)
        screened = sur.screen(X, P, Js)
        s_obj = screened.sum(1)
        res.screen_s += time.perf_counter() - t0
        # the elites are already verified: verify the best-screened of the rest
        cand = n_el + np.argsort(s_obj[n_el:], kind="stable")[:K]
        t0 = time.perf_counter()
        tgt, adj, _ = samples(Z[cand], Jv, cfg.seed + 2, first_index=g * P * Jv, mesh_id=mesh_id)
        rates = error_rates(llg_outcomes(ctx, mesh_id, p, tgt, adj), len(cand), Jv)
        res.verify_s += time.perf_counter() - t0
        res.verified_islands += 2 * len(cand) * Jv
        res.llg_only_islands += 2 * (P - n_el) * Jv
        pool_Z = np.concatenate([elite_Z, Z[cand]])
        pool_obj = np.concatenate([elite_obj, rates.sum(1)])
        pool_rates = np.concatenate([elite_rates, rates])
        keep = np.argsort(pool_obj, kind="stable")[:K]
        elite_Z, elite_obj, elite_rates = pool_Z[keep], pool_obj[keep], pool_rates[keep]
        res.history.append(dict(generation=g, best_verified=float(elite_obj[0]),
                                screened_of_verified=s_obj[cand].tolist(), verified=rates.sum(1).tolist()))
        if g + 1 < cfg.generations:
            Z = next_population(elite_Z, P, g + 1, cfg)
    res.best_Z, res.best_rates = elite_Z[0], elite_rates[0]
    return res
