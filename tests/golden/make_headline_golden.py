"""Write the FP64 oracle's results for the headline parity tests (test infrastructure).

Only the oracle (oracle/) and the seeded input generators (synth) run here; no
value comes from the CUDA path.  The oracle needs about an hour of host time
for these runs, more than a test may take, so its results are stored:

  census      tests/golden/census_first_100ps.npz
              64 islands sampled from the 4096-island census workload (the
              bench's: 1547-node mesh, jitter seed 1, 64x64x16 head map moving
              at 20 m/s from x0 = -10 nm, 100 ps rise, alpha 0.1), integrated
              over the first 100 ps with the workload's step count k; the
              volume-averaged m_z after every 0.1 ps interval, and every
              node's m every 10 ps (stored as int16, m = q / 32767, a rounding
              of at most 1.6e-5).
  outcomes    tests/golden/outcome_census_209.npz
              1024 jittered islands of the 209-node mesh written by the moving
              head (synth.outcome_census, a Sec. II.C recording simulation: the
              head field plus a constant field H_ext opposing it, spread over
              the islands so that a real fraction of them switches), 300 ps;
              the switch flag, first crossing time and final volume-averaged
              m_z of every island.

  design-ber  tests/golden/design_ber.npz
              the critical-field search of Sec. II.C (Eqs. 1-2) for the three
              designs of design_inputs.parity_designs, both roles (target and
              previous bit), each design under its own head in one stacked
              map, with the step count of the strongest constant field of the
              grid: the critical fields, error rates and aborts.

  python tests/golden/make_headline_golden.py census|outcomes|design-ber [--workers N]
"""
from __future__ import annotations

import argparse
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
GOLDEN = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# census workload
CENSUS_B = 4096
CENSUS_SAMPLES = 64
CENSUS_INTERVALS = 1000          # 100 ps at 0.1 ps
CENSUS_SNAPSHOT_EVERY = 100      # full state every 10 ps


def census_params():
    from paper_1603_09493_gb300 import synth
    return synth.census_run_params(t_end_ps=CENSUS_INTERVALS * 0.1)


def census_sample_index() -> np.ndarray:
    return np.round(np.linspace(0, CENSUS_B - 1, CENSUS_SAMPLES)).astype(np.int64)


def outcome_islands(mesh_id: int = 0):
    from paper_1603_09493_gb300 import synth
    return synth.outcome_census(mesh_id=mesh_id)[0]


def outcome_params():
    from paper_1603_09493_gb300 import synth
    return synth.outcome_census()[1]


def _census_chunk(args):
    idx, k = args
    from oracle import fem, llg
    from paper_1603_09493_gb300 import synth
    mesh = synth.census_island_mesh()
    mats = synth.ecc_materials()
    hm = synth.synthetic_head_map()
    ops = fem.MeshOperators(mesh.xyz_nm, mesh.tets, mesh.tet_region, mats)
    p = census_params()
    p.substeps = k
    b = llg.Batch(ops, synth.jittered_islands(CENSUS_B, seed=1).subset(idx), p, head_map=hm)
    mz, steps = [], [0]

    def on_step(m, t):
        steps[0] += 1
        if steps[0] % k == 0:
            mz.append(b.mz_avg(m))

    r = b.run(sample_every=CENSUS_SNAPSHOT_EVERY, on_step=on_step)
    return np.array(mz), np.array(r["samples"])


def _outcome_chunk(args):
    lo, hi, k = args
    from oracle import fem, llg
    from paper_1603_09493_gb300 import synth
    mesh = synth.small_island_mesh()
    ops = fem.MeshOperators(mesh.xyz_nm, mesh.tets, mesh.tet_region, synth.ecc_materials())
    p = outcome_params()
    p.substeps = k
    b = llg.Batch(ops, outcome_islands().subset(np.arange(lo, hi)), p, head_map=synth.synthetic_head_map())
    r = b.run()
    return r["switched"], r["t_sw"], r["mz"], r["status"]


def _design_ber_one(args):
    d, role, k = args
    from oracle import fem
    from oracle import hcrit as ohcrit
    from paper_1603_09493_gb300 import design_inputs as DI
    Z = DI.parity_designs()
    tgt, direction, sigma, R = DI.critical_field_inputs(Z, role)
    mesh, mats = DI.grid_meshes()[int(tgt.mesh_id[0])]
    ops = fem.MeshOperators(mesh.xyz_nm, mesh.tets, mesh.tet_region, mats)
    p = DI.run_params(float(R.v["v_m_per_s"][0]))
    p.substeps = k
    hm = DI.head_stack(R.heads)
    h, ber, ab = ohcrit.search(ops, tgt.subset([d]), p, direction[d:d + 1], sigma[d:d + 1], role, head_map=hm)
    return float(h[0]), float(ber[0]), bool(ab[0])


def _pool(workers):
    # one BLAS thread per worker process; spawned, so that no parent state is forked
    os.environ["OMP_NUM_THREADS"] = "1"
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    os.environ["MKL_NUM_THREADS"] = "1"
    return mp.get_context("spawn").Pool(workers)


def make_census(workers: int):
    from oracle import fem, llg
    from paper_1603_09493_gb300 import synth
    mesh = synth.census_island_mesh()
    ops = fem.MeshOperators(mesh.xyz_nm, mesh.tets, mesh.tet_region, synth.ecc_materials(), with_demag=False)
    p = census_params()
    k = llg.stable_substeps(llg.Batch(ops, synth.jittered_islands(CENSUS_B, seed=1), p,
                                      head_map=synth.synthetic_head_map(), demag=np.zeros((1, 1))))
    idx = census_sample_index()
    chunks = np.array_split(idx, workers)
    t = time.time()
    with _pool(workers) as pool:
        res = pool.map(_census_chunk, [(c, k) for c in chunks])
    mz = np.concatenate([r[0] for r in res], axis=1)                  # [intervals][samples]
    snaps = np.concatenate([r[1] for r in res], axis=1)               # [snapshots][samples][n][3]
    q = np.round(snaps * 32767.0).astype(np.int16)
    isl = synth.jittered_islands(CENSUS_B, seed=1).subset(idx)
    out = os.path.join(GOLDEN, "census_first_100ps.npz")
    np.savez_compressed(out, k=k, index=idx, mz=mz, m_q=q, snapshot_every=CENSUS_SNAPSHOT_EVERY,
                        Ms_scale=isl.Ms_scale, Ku_scale=isl.Ku_scale, u=isl.u, pos_nm=isl.pos_nm,
                        n_nodes=mesh.n_nodes, xyz_sum=float(mesh.xyz_nm.sum()))
    print(f"census: k={k}, {len(idx)} islands, {mz.shape[0]} intervals, {time.time() - t:.0f} s -> {out}")


def make_outcomes(workers: int):
    from oracle import fem, llg
    from paper_1603_09493_gb300 import synth
    mesh = synth.small_island_mesh()
    ops = fem.MeshOperators(mesh.xyz_nm, mesh.tets, mesh.tet_region, synth.ecc_materials(), with_demag=False)
    p = outcome_params()
    isl = outcome_islands()
    k = llg.stable_substeps(llg.Batch(ops, isl, p, head_map=synth.synthetic_head_map(), demag=np.zeros((1, 1))))
    bounds = np.linspace(0, len(isl), 4 * workers + 1).astype(int)
    t = time.time()
    with _pool(workers) as pool:
        res = pool.map(_outcome_chunk, [(bounds[i], bounds[i + 1], k) for i in range(len(bounds) - 1)])
    sw = np.concatenate([r[0] for r in res])
    tsw = np.concatenate([r[1] for r in res])
    mz = np.concatenate([r[2] for r in res])
    st = np.concatenate([r[3] for r in res])
    out = os.path.join(GOLDEN, "outcome_census_209.npz")
    np.savez_compressed(out, k=k, switched=sw, t_sw=tsw, mz=mz, status=st, Ms_scale=isl.Ms_scale,
                        Ku_scale=isl.Ku_scale, u=isl.u, pos_nm=isl.pos_nm, Hext_T=isl.Hext_T,
                        t_end_ps=outcome_params().t_end_ps)
    print(f"outcomes: k={k}, {sw.sum()} of {sw.size} switched, {time.time() - t:.0f} s -> {out}")


def make_design_ber(workers: int):
    from oracle import fem, llg
    from paper_1603_09493_gb300 import design_inputs as DI
    Z = DI.parity_designs()
    tgt, direction, sigma, R = DI.critical_field_inputs(Z, "targ")
    assert len(set(tgt.mesh_id.tolist())) == 1 and len(set(R.v["v_m_per_s"].tolist())) == 1
    mesh, mats = DI.grid_meshes()[int(tgt.mesh_id[0])]
    ops = fem.MeshOperators(mesh.xyz_nm, mesh.tets, mesh.tet_region, mats, with_demag=False)
    probe = tgt.subset(np.arange(len(tgt)))
    probe.Hext_T = (4.0 * sigma[:, None] * direction).astype(np.float32)
    p = DI.run_params(float(R.v["v_m_per_s"][0]))
    k = llg.stable_substeps(llg.Batch(ops, probe, p, head_map=DI.head_stack(R.heads), demag=np.zeros((1, 1))))
    tasks = [(d, role, k) for role in ("targ", "prev") for d in range(len(Z))]
    t = time.time()
    with _pool(min(workers, len(tasks))) as pool:
        res = pool.map(_design_ber_one, tasks)
    h = np.array([r[0] for r in res]).reshape(2, len(Z))
    ber = np.array([r[1] for r in res]).reshape(2, len(Z))
    ab = np.array([r[2] for r in res]).reshape(2, len(Z))
    out = os.path.join(GOLDEN, "design_ber.npz")
    np.savez_compressed(out, k=k, roles=np.array(["targ", "prev"]), h_crit_T=h, ber=ber, aborted=ab, sigma_T=sigma,
                        Z=Z)
    print(f"design-ber: k={k}, H_crit/sigma {h / sigma[None, :]}, {time.time() - t:.0f} s -> {out}")


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["census", "outcomes", "design-ber"])
    ap.add_argument("--workers", type=int, default=os.cpu_count() or 1)
    a = ap.parse_args()
    {"census": make_census, "outcomes": make_outcomes, "design-ber": make_design_ber}[a.what](a.workers)
