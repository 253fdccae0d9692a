"""The write-head and media design problem that the surrogate screens (Sec. II.A
optimisation loop; Sec. II.B and Table I free parameters; Fig. 3 track
layouts), on the library: LLG labels of realisations of designs, the held-out
metrics of the surrogate, the paper's critical-field bit-error rates of designs
(Sec. II.C, Eqs. 1-2), and the surrogate-assisted design search.  The designs,
their grid, head maps, jitter and islands come from design_inputs, which also
states the readings of the problem."""
from __future__ import annotations

import time

import numpy as np

from . import _lib as L
from . import evolve, hcrit, synth
from .design_inputs import (BLOCK_NM, BLOCKS, GEOMETRY_KEYS, HEAD_KEYS, HEADS_PER_MAP, JITTER, KEYS, LAYOUTS,  # noqa: F401
                            LEVELS, RANGES, T_END_PS, Z_TOP_NM, Realisations, adjacent_offset,
                            critical_field_inputs, features, parity_designs,
                            geometry_index, grid_meshes, head_block, head_stack, islands, nominal, realisations,
                            run_params, values)

def upload_grid(ctx) -> list:
    """Upload the 81 meshes of the geometry grid; their mesh ids in geometry_index order."""
    return [ctx.mesh_upload(m, mats) for m, mats in grid_meshes()]


def llg_labels(ctx, grid_ids, R: Realisations, precision: int = L.PREC_BF16X3) -> np.ndarray:
    """LLG labels [N][2] (target switched, adjacent island flipped) of every
    realisation: one batch per (group of 256 heads, velocity level), the group's
    heads in one stacked map."""
    Y = np.zeros((len(R), 2), np.float32)
    group = R.head // HEADS_PER_MAP
    for g in np.unique(group):
        hid = ctx.headmap_upload(head_stack(R.heads[g * HEADS_PER_MAP:(g + 1) * HEADS_PER_MAP]))
        for v in LEVELS["v_m_per_s"]:
            rows = np.where((group == g) & np.isclose(R.v["v_m_per_s"], v))[0]
            if rows.size == 0:
                continue
            tgt, adj = islands(R, grid_ids, rows)
            out = ctx.run_batch(synth.Islands.concat([tgt, adj]), run_params(v), int(round(T_END_PS / 0.1)),
                                precision=precision, map_id=hid)
            if np.any(out["status"] != 0):
                raise RuntimeError("an island of a label batch reported a failure")
            n = rows.size
            Y[rows, 0] = out["switched"][:n]
            Y[rows, 1] = out["switched"][n:]
    return Y


def training_set(ctx, grid_ids, N: int, n_heads: int, seed: int, first_index: int = 0):
    """N uniform designs, one realisation each, whose heads are drawn from a pool of
    n_heads uniform head designs; returns (X, Y, R)."""
    Z = synth.counter_uniform(seed, 710, np.arange(first_index * 12, (first_index + N) * 12)).reshape(N, 12)
    Zh = synth.counter_uniform(seed, 711, np.arange(first_index * 3, (first_index + n_heads) * 3)).reshape(n_heads, 3)
    heads = np.stack([RANGES[k][0] + (RANGES[k][1] - RANGES[k][0]) * Zh[:, j] for j, k in enumerate(HEAD_KEYS)], 1)
    R = realisations(Z, 1, seed, first_index, heads=heads, head_of_design=np.arange(N) % n_heads)
    return R.X, llg_labels(ctx, grid_ids, R), R


def critical_field_ber(ctx, grid_ids, Z, role: str = "targ", K1_hard: float = 0.9e6, Ms_hard: float = 0.8e6,
                       precision: int = L.PREC_BF16X3, substeps: int = 0) -> hcrit.SearchResult:
    """Bit-error rate of each design by the critical-field search of Sec. II.C (Eqs. 1-2)
    on its nominal island under its own head: role 'targ' writes the target against a
    constant field antiparallel to the head field, role 'prev' holds the previously
    written bit (one pitch behind the target, down-track) against a parallel one;
    sigma = 0.015 H_A of the design's hard layer.  Each level of the search is one batch
    per velocity level, the designs' heads stacked in maps of 256; substeps 0 takes the
    library's stable step count of each batch."""
    tgt, direction, sigma, R = critical_field_inputs(Z, role, K1_hard, Ms_hard)
    D = len(R)
    tgt.mesh_id = np.asarray(grid_ids, np.int32)[tgt.mesh_id]
    maps = [ctx.headmap_upload(head_stack(R.heads[g * HEADS_PER_MAP:(g + 1) * HEADS_PER_MAP]))
            for g in range((D + HEADS_PER_MAP - 1) // HEADS_PER_MAP)]
    n_int = int(round(T_END_PS / 0.1))

    def run_flags(isl, designs):
        designs = np.asarray(designs)
        out = np.zeros(len(isl), bool)
        group = designs // HEADS_PER_MAP
        for g in np.unique(group):
            for v in LEVELS["v_m_per_s"]:
                rows = np.where((group == g) & np.isclose(R.v["v_m_per_s"][designs], v))[0]
                if rows.size:
                    q = run_params(v)
                    q.substeps = int(substeps)
                    res = ctx.run_batch(isl.subset(rows), q, n_int, precision=precision, map_id=maps[g])
                    if np.any(res["status"] != 0):
                        raise RuntimeError("an island of a critical-field batch reported a failure")
                    out[rows] = res["switched"]
        return out

    return hcrit.critical_field_search(run_flags, tgt, direction, sigma, role)


def metrics(P, Y) -> dict:
    """Accuracy at 1/2, Brier score and ROC AUC of probabilities P [N] against labels Y [N]."""
    P = np.asarray(P, np.float64)
    Y = np.asarray(Y, np.float64) > 0.5
    pos, neg = P[Y], P[~Y]
    if pos.size and neg.size:
        allv = np.concatenate([pos, neg])
        ranks = np.empty(allv.size)
        order = np.argsort(allv, kind="stable")
        ranks[order] = np.arange(1, allv.size + 1)
        for val in np.unique(allv):                    # average ranks of ties
            tie = allv == val
            ranks[tie] = ranks[tie].mean()
        auc = (ranks[:pos.size].sum() - pos.size * (pos.size + 1) / 2) / (pos.size * neg.size)
    else:
        auc = float("nan")
    return dict(accuracy=float(np.mean((P > 0.5) == Y)), brier=float(np.mean((P - Y) ** 2)), auc=float(auc),
                positive_fraction=float(Y.mean()))


def search(ctx, sur, grid_ids, cfg: evolve.SearchConfig):
    """The generational design loop of evolve.search on this problem: each
    generation the surrogate screens the population on fresh jitter samples, the
    best-screened designs that are not elites yet are solved with LLG (each with
    its own head), and the elites are mutated into the next population."""
    P, K, Js, Jv = cfg.population, cfg.top_k, cfg.n_jitter_screen, cfg.n_jitter_verify
    d = len(KEYS)
    Z = synth.counter_uniform(cfg.seed, 720, np.arange(P * d, dtype=np.uint64)).reshape(P, d)
    elite_Z, elite_obj, elite_rates = np.zeros((0, d)), np.zeros(0), np.zeros((0, 2))
    res = evolve.SearchResult(best_Z=None, best_rates=None)
    for g in range(cfg.generations):
        n_el = len(elite_Z)
        t0 = time.perf_counter()
        Rs = realisations(Z, Js, cfg.seed + 1, first_index=g * P * Js)
        s_obj = sur.screen(Rs.X, P, Js).sum(1)
        res.screen_s += time.perf_counter() - t0
        cand = n_el + np.argsort(s_obj[n_el:], kind="stable")[:K]
        t0 = time.perf_counter()
        Rv = realisations(Z[cand], Jv, cfg.seed + 2, first_index=g * P * Jv)
        rates = evolve.error_rates(llg_labels(ctx, grid_ids, Rv), len(cand), Jv)
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
            Z = evolve.next_population(elite_Z, P, g + 1, cfg)
    res.best_Z, res.best_rates = elite_Z[0], elite_rates[0]
    res.elite_Z, res.elite_rates = elite_Z, elite_rates
    return res


def rank_by_ber(ctx, grid_ids, Z) -> dict:
    """BER_targ + BER_prev (Eqs. 1-2, critical-field search) of the designs Z and the
    best of them: the paper's error rates of the write, where counted jitter samples
    no longer resolve the differences between designs."""
    t0 = time.perf_counter()
    rt = critical_field_ber(ctx, grid_ids, Z, "targ")
    rp = critical_field_ber(ctx, grid_ids, Z, "prev")
    tot = rt.ber + rp.ber
    b = int(np.argmin(tot))
    return dict(ber_targ=rt.ber, ber_prev=rp.ber, ber_sum=tot, best=b, best_Z=np.asarray(Z)[b],
                runs=rt.n_runs + rp.n_runs, seconds=time.perf_counter() - t0)
