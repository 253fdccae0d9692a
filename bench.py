#!/usr/bin/env python
"""Throughput of the batched ECC-island LLG path (island-ns/s).

Workload: 4096 jittered ECC islands sharing one ~1500-node P1 cylinder mesh
(8 nm, soft 3 nm on hard 7 nm), synthetic 64x64x16 head-field map at 1 nm,
head moving at 20 m/s, alpha 0.1, output interval 0.1 ps split into the
stable number of Heun steps.  One bench step = one output interval for every
island (one CUDA-graph replay: per Heun step two demag GEMMs and the two Heun
stage kernels).  value = islands * simulated ns / device seconds, all ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision bf16x3|fp32|bf16]
  python bench.py --impl reference     # the FP64 CPU oracle on the host cores
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "island-ns/s batched LLG (mixed vs plain, same outcomes); surrogate evals/s"
UNIT = "island-ns/s"
DT_PS = 0.1
B_ISLANDS = 4096
SM_FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # 152 SMs x 128 FP32 lanes x FMA x 2.07 GHz


def workload(seed: int = 1):
    from paper_1603_09493_gb300 import synth
    mesh = synth.census_island_mesh(seed=seed)
    mats = synth.ecc_materials()
    hm = synth.synthetic_head_map()
    return mesh, mats, hm, synth.census_run_params(t_end_ps=DT_PS)


def config_dict(mesh, k, precision, B, n_gpus):
    return {"workload": f"census batch: {B} jittered ECC islands per GPU on one {mesh.n_nodes}-node P1 cylinder "
                        "mesh (8 nm, soft 3 nm / hard 7 nm), 64x64x16 head map at 1 nm, 20 m/s, 0.1 ps intervals",
            "islands_per_gpu": B, "nodes": mesh.n_nodes, "heun_steps_per_interval": k, "dt_ps": DT_PS,
            "demag_precision": precision, "parallelism": f"islands sharded over {n_gpus} GPU(s), no collective",
            "l2": "per-step working set (state, stages, demag operand and field, BF16/FP32 operator) > 129 MB L2"}


def sample_clocks_start(log_path: str = ""):
    """nvidia-smi clock samples every 100 ms until sample_clocks_stop; the raw
    samples also go to log_path when one is given."""
    try:
        f = open(log_path or os.devnull, "w")
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "100"],
                                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        return proc, f
    except Exception:
        return None, None


def sample_clocks_stop(proc, f, gpu_index):
    if proc is None:
        return None
    proc.terminate()
    try:
        out, _ = proc.communicate(timeout=5)
    except Exception:
        proc.kill()
        return None
    sm, mx, reasons = [], 0.0, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in out.strip().splitlines():
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 9 or parts[0] != str(gpu_index):
            continue
        try:
            sm.append(float(parts[1]))
            mx = max(mx, float(parts[2]))
        except ValueError:
            continue
        for nm, v in zip(names, parts[5:9]):
            if v.lower() == "active":
                reasons.add(nm)
    if f is not None:
        f.write(out)
        f.close()
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def gemm_peak(pk):
    """Denominator of the GEMM roofline.  The GEMM duration is taken launch by
    launch with CUDA events (bpm_batch_kernel_times, right after the timed
    region, same stream and launch configuration), a kernel timed alone at the
    clocks of the run (2.0-2.07 GHz), so the burst cuBLAS figure applies; the
    sustained one was taken over seconds of back-to-back GEMMs at a median SM
    clock of about 1.5 GHz."""
    if pk:
        return pk["bf16_tflops"], "MEASURED_PEAKS bf16_tflops (burst; kernel timed launch by launch)"
    return 1900.0, "fallback (1.9 PFLOP/s bf16 burst)"


# DRAM bytes (read + write) of one demag-GEMM launch from ncu
# (dram__bytes_read.sum + dram__bytes_write.sum, mean of two launches), keyed by
# (precision, islands, nodes) of the captured workload:
#   ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum \
#       --clock-control none -k regex:k_gemm_grouped -s 10 -c 2 --csv \
#       python bench.py --steps 2 --warmup 1 --no-cpu --no-e2e --no-extras --no-autotune
# (k_gemm_grouped<3,256,32>, N-major tile order).  Remove an entry when the kernel changes.
NCU_GEMM_TRAFFIC = {(1, 4096, 1547): 412.97e6 + 60.92e6}


def gemm_traffic(prec, B, n):
    return NCU_GEMM_TRAFFIC.get((int(prec), int(B), int(n)))


# Warp instructions per island-node of the Heun stage kernels (two islands per CTA, BF16x3
# operand) from ncu's smsp__inst_executed.sum of one launch over the 1024 islands of one chain
# (2048 islands, two chains) of the 1547-node mesh (profiles/heun_stages_census_2048.md: 24.30 M
# and 26.87 M).  Remove when the kernels change.
NCU_STAGE_WARP_INSTR = {1547: (24.30e6 / (1024 * 1547), 26.87e6 / (1024 * 1547))}
SM_COUNT = 152
ISSUE_PER_SM_CLK = 4           # one warp instruction per scheduler per cycle, four schedulers per SM


# ---------------------------------------------------------------------------
# The FP64 oracle on the host cores: spawned worker processes, each with its
# own copy of the census mesh operators and a pinned number of BLAS threads.

_WORKER = {}


def _oracle_worker_init(barrier):
    from oracle import fem
    mesh, mats, hm, _ = workload()
    _WORKER["ops"] = fem.MeshOperators(mesh.xyz_nm, mesh.tets, mesh.tet_region, mats)
    _WORKER["hm"] = hm
    barrier.wait()


def _oracle_worker_run(task):
    """task = (islands, params, m0 or None) -> final m of the islands."""
    from oracle import llg
    isl, p, m0 = task
    return llg.Batch(_WORKER["ops"], isl, p, head_map=_WORKER["hm"]).run(m0)["m"]


class OraclePool:
    """Worker processes with the census workload's oracle operators built, each
    with `threads` BLAS threads (pinned through the environment before numpy
    loads); the constructor returns once every worker holds them, so that
    timing starts after the set-up."""

    def __init__(self, workers: int, threads: int = 1):
        import multiprocessing as mp
        for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[v] = str(int(threads))
        ctx = mp.get_context("spawn")
        barrier = ctx.Barrier(workers + 1)
        self.workers = workers
        self.pool = ctx.Pool(workers, initializer=_oracle_worker_init, initargs=(barrier,))
        barrier.wait()

    def run(self, tasks):
        return self.pool.map(_oracle_worker_run, tasks, chunksize=1)

    def close(self):
        self.pool.close()
        self.pool.join()


def host_cores() -> int:
    return len(os.sched_getaffinity(0))


def oracle_step_count(p):
    """The workload's integrator step count by the oracle's own rule (over all its islands)."""
    from oracle import fem, llg
    from paper_1603_09493_gb300 import synth
    mesh, mats, hm, _ = workload()
    ops = fem.MeshOperators(mesh.xyz_nm, mesh.tets, mesh.tet_region, mats, with_demag=False)
    return llg.stable_substeps(llg.Batch(ops, synth.jittered_islands(B_ISLANDS, seed=1), p, head_map=hm,
                                         demag=np.zeros((1, 1))))


def cpu_baseline(p, k, target_s=15.0):
    """The oracle on all host cores: one process integrating one island per core
    as one batch, its BLAS pinned to as many threads as the host has cores, for
    a bounded number of 0.1 ps intervals sized to about target_s seconds."""
    from paper_1603_09493_gb300 import synth
    W = host_cores()
    isl = synth.jittered_islands(W, seed=1)
    pool = OraclePool(1, threads=W)
    try:
        def run(nint):
            q = type(p)(**{**p.__dict__})
            q.substeps, q.t0_ps, q.t_end_ps = k, 0.0, nint * DT_PS
            t = time.perf_counter()
            pool.run([(isl, q, None)])
            return time.perf_counter() - t
        t1 = run(1)
        nint = int(max(1, min(40, round(target_s / max(t1, 1e-3)))))
        t = run(nint)
    finally:
        pool.close()
    return {"value": W * nint * DT_PS * 1e-3 / t, "unit": UNIT, "cores": W, "kind": "oracle",
            "workers": f"one process, its BLAS pinned to {W} threads (one per host core)",
            "sample": f"{W} islands in one oracle batch x {nint} intervals ({nint * k} Heun steps) of the census "
                      f"workload, numpy FP64, {t:.1f} s"}


def stable_k(ctx, hid, isl, p):
    """The library's integrator step count for this workload (bpm_stable_substeps)."""
    return ctx.stable_substeps(isl, p, hid)[0]


def measure_plain(ctx, isl, p, hid, prec, n, islands=8, intervals=2):
    """The one-island-per-launch FP32 GEMV form on a few islands of the same
    workload, and the batched path on the same islands for the same-outcome check."""
    sub = isl.subset(np.arange(islands))
    plain = ctx.run_plain(sub, p, intervals, map_id=hid)
    mixed = ctx.run_batch(sub, p, intervals, precision=prec, map_id=hid)
    value = islands * intervals * DT_PS * 1e-3 / (plain["device_ms"] * 1e-3)
    return {"value": value, "unit": UNIT, "islands": islands, "intervals": intervals,
            "form": "one island per launch, FP32 GEMV demag streamed from HBM, single-island stage kernels",
            "vs_mixed_max_abs_dm": float(np.abs(plain["m"] - mixed["m"]).max()),
            "same_switch_flags": bool(np.array_equal(plain["switched"], mixed["switched"]))}


def measure_plain_f64(ctx, isl, p, hid, mesh, mats, islands=2, intervals=1):
    """The one-island-per-launch FP64 form (every step in FP64, the FP64 demag
    matrix streamed per Heun stage) on a few islands of the same workload."""
    mid = ctx.mesh_upload(mesh, mats, keep_f64=True)
    sub = isl.subset(np.arange(islands))
    sub.mesh_id[:] = mid
    out = ctx.run_plain_f64(sub, p, intervals, map_id=hid)
    return {"value": islands * intervals * DT_PS * 1e-3 / (out["device_ms"] * 1e-3), "unit": UNIT,
            "islands": islands, "intervals": intervals,
            "form": "one island per launch, FP64 GEMV demag with the FP64 operator, FP64 field and Heun kernels"}


def measure_parity(ctx, hid):
    """Switch outcomes of the BF16x3 batch against the FP64 oracle's, stored by
    tests/golden/make_headline_golden.py: 1024 jittered islands of the 209-node
    mesh written by the moving head against an opposing field spread over the
    islands (synth.outcome_census, 300 ps)."""
    from paper_1603_09493_gb300 import _lib as L
    from paper_1603_09493_gb300 import synth
    path = os.path.join(ROOT, "tests", "golden", "outcome_census_209.npz")
    if not os.path.exists(path):
        return None
    ref = np.load(path)
    mid = ctx.mesh_upload(synth.small_island_mesh(), synth.ecc_materials())
    isl, p = synth.outcome_census(mesh_id=mid)
    p.substeps = int(ref["k"])
    out = ctx.run_batch(isl, p, p.n_intervals, precision=L.PREC_BF16X3, map_id=hid)
    both = (out["t_sw"] > 0) & (ref["t_sw"] > 0)
    return {"outcome_agreement": float(np.mean(out["switched"] == ref["switched"])), "islands": len(isl),
            "switched_fraction": float(np.mean(ref["switched"])),
            "max_abs_dt_sw_ps": float(np.abs(out["t_sw"][both] - ref["t_sw"][both]).max()) if both.any() else None,
            "against": "FP64 oracle outcomes (tests/golden/outcome_census_209.npz)",
            "workload": "1024 jittered islands, 209-node mesh, head map from x0 = -2 nm at 20 m/s, opposing "
                        "field 0-0.3 T spread over the islands, 300 ps, BF16x3 demag"}


def measure_uneven(ctx, hm, hid, realisations=512, steps=3):
    """Config 2: 16 design variants (518-3906 nodes), `realisations` jittered
    targets each plus their adjacent-track islands, in one batch (grouped demag
    GEMM over all mesh groups, one stage launch per occupancy class), for the
    centered, staggered and shingled layouts; device time of `steps` intervals
    per layout, and the grouped GEMM's roofline."""
    from paper_1603_09493_gb300 import _lib as L
    from paper_1603_09493_gb300 import synth
    variants = synth.design_variants()
    mats = synth.ecc_materials()
    mids = [ctx.mesh_upload(v["mesh"], mats) for v in variants]
    import torch
    stream = torch.cuda.ExternalStream(ctx.stream_ptr)
    pk = peaks()
    peak, peak_source = gemm_peak(pk)
    out = {"variants": len(variants), "nodes": [min(v["mesh"].n_nodes for v in variants),
                                                 max(v["mesh"].n_nodes for v in variants)],
           "realisations": realisations, "layouts": {}}
    for layout in ("staggered", "centered", "shingled"):
        isl, role = synth.uneven_batch(variants, mids, realisations=realisations, seed=2, layout=layout)
        p = synth.census_run_params()
        p.substeps = 0
        k = ctx.stable_substeps(isl, p, hid)[0]
        with ctx.batch(isl, p, precision=L.PREC_BF16X3, map_id=hid) as bt:
            bt.advance(1)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            bt.advance(steps)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1) / steps
            ok = bool(np.all(bt.read()["status"] == 0))
            entry = {"islands": len(isl), "adjacent_islands": int(np.sum(role == 1)), "heun_steps_per_interval": k,
                     "value": len(isl) * DT_PS * 1e-3 / (ms * 1e-3), "unit": UNIT, "ms_per_interval": ms,
                     "launches_per_interval": bt.graph_kernels(), "status_ok": ok}
            if layout == "staggered":
                kt = bt.kernel_times(reps=4)
                flops = sum(6.0 * int(np.sum(isl.mesh_id == mid)) * (3 * v["mesh"].n_nodes) ** 2
                            for mid, v in zip(mids, variants))
                entry["roofline"] = {"bound": "tensor", "achieved": flops / (kt["gemm_ms"] * 1e-3) / 1e12,
                                     "peak": peak, "unit": "TFLOP/s", "peak_source": peak_source,
                                     "frac": flops / (kt["gemm_ms"] * 1e-3) / 1e12 / peak, "traffic": None,
                                     "kernel": "grouped demag GEMM over the 16 mesh groups (one launch)"}
                entry["kernel_ms"] = kt
        out["layouts"][layout] = entry
    return out


def measure_neb(ctx, mid, hm, hid, D=64, P=16, iters=400, mesh=None, mats=None):
    """Adjacent-track barriers (Sec. II.C, Eq. 3): D islands of the census mesh on
    the adjacent track (12.7 nm cross-track), head frozen 2 nm into the map, one
    band of P images each, BF16x3 demag; wall-clock of the bpm_neb_run call."""
    from paper_1603_09493_gb300 import adjacent, synth
    isl = synth.jittered_islands(D, seed=4, mesh_id=mid)
    isl.pos_nm[:, 1] += 12.7
    p = synth.RunParams(dt_ps=0.1, rise_ps=0.0, v_m_per_s=0.0, x0_nm=2.0, use_map=True)
    step = adjacent.stable_step(ctx, mid, isl, p, hid)
    ctx.neb(isl, P, 2, step, 1.0, -1, map_id=hid, head_x_nm=p.x0_nm)           # warm-up
    t = time.perf_counter()
    out = adjacent.barriers(ctx, isl, p, n_images=P, max_iters=iters, climb_after=iters // 2, step=step,
                            map_id=hid)
    wall = time.perf_counter() - t
    kt = out["E_B_kT"]
    oracle = None
    if mesh is not None:
        # the FP64 oracle band on one band of the same workload, two updates
        from oracle import fem
        from oracle import neb as oneb
        ops = fem.MeshOperators(mesh.xyz_nm, mesh.tets, mesh.tet_region, mats)
        t = time.perf_counter()
        oneb.island_band(ops, isl.subset(np.arange(1)), p, hm, oneb.great_circle_path(ops.n, P)[None], 2, step, 1.0)
        to = time.perf_counter() - t
        oracle = {"value": P * 2 / to, "unit": "band-image updates/s", "kind": "oracle", "cores": 1,
                  "workers": "one process (numpy FP64; its BLAS may thread the matrix products)",
                  "sample": f"1 band x {P} images x 2 updates, {to:.1f} s"}
    return {"image_updates_per_s": D * P * out["iters"] / wall, "unit": "band-image updates/s", "bands": D,
            "cpu_baseline": oracle,
            "images": P, "iters": out["iters"], "wall_s": wall, "max_force": out["max_force"],
            "E_B_kT_median": float(np.median(kt)), "E_B_kT_min": float(np.min(kt)),
            "ber_adj_median": float(np.median(out["ber_adj"])),
            "note": "each update: one BF16x3 demag GEMM over all images, energy/field and band kernels; "
                    "wall-clock incl. buffer setup and convergence checks every 50 updates"}


def measure_head_field(ctx, nx=64, ny=64, nz=18, reps=20):
    """The head-field solve of the saturated main pole (Table I's initial design) on a head map
    of the census frame, written to device memory; CUDA events on the context stream."""
    import torch
    from paper_1603_09493_gb300 import synth
    g = synth.pole_geometry(z_abs_nm=18.0, z_sul_nm=-2.0)
    out = torch.empty((nz, ny, nx, 3), dtype=torch.float32, device="cuda")
    org = (-48.0, -32.0, 0.0)
    ctx.head_field(g, nx, ny, nz, 1.0, org, out=out)
    stream = torch.cuda.ExternalStream(ctx.stream_ptr)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        ctx.head_field(g, nx, ny, nz, 1.0, org, out=out)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    B = out.cpu().numpy()
    # with Table I's initial trailing shield (9 nm gap, 10 nm thick, 2 nm panels): the boundary-
    # element solve (matrix, LU, triangular solves, residual check) and the field, one call
    gs = dict(g, trailing_shield_gap_nm=9.0, shield_thickness_nm=10.0, shield_panel_nm=2.0)
    torch.cuda.synchronize()
    t = time.perf_counter()
    ctx.head_field(gs, nx, ny, nz, 1.0, org, out=out)
    torch.cuda.synchronize()
    ms_shield = (time.perf_counter() - t) * 1e3
    Bs = out.cpu().numpy()
    # the oracle's quadrature on a bounded sample of voxels
    from oracle import polefield
    pts = np.array([[-10.0, 0.0, 17.0], [0.0, 7.0, 17.0], [-30.0, 20.0, 5.0], [5.0, -10.0, 12.0]])
    t = time.perf_counter()
    polefield.field(g, pts)
    o_vox = len(pts) / (time.perf_counter() - t)
    return {"voxels": nx * ny * nz, "ms_per_map": ms, "voxels_per_s": nx * ny * nz / (ms * 1e-3),
            "triangles": 24, "peak_under_pole_T": float(B[17, 32, 38, 2]),
            "with_trailing_shield": {"ms_per_map": ms_shield, "gap_nm": 9.0, "thickness_nm": 10.0, "panel_nm": 2.0,
                                     "under_pole_T": float(Bs[17, 32, 38, 2]),
                                     "trailing_edge_T": [float(v) for v in Bs[17, 32, 48]],
                                     "trailing_edge_without_T": [float(v) for v in B[17, 32, 48]],
                                     "note": "wall-clock of one call: panel matrix, LU and solves on the GPU, "
                                             "residual check, field of pole, shield and images"},
            "form": "saturated CoFe main pole (Table I initial design) as surface charges, charge sheet at the "
                    "yoke edge, under-layer image; closed form per triangle, FP64, one thread per voxel",
            "cpu_baseline": {"voxels_per_s": o_vox, "kind": "oracle", "cores": 1,
                             "sample": f"{len(pts)} voxels, adaptive Gauss-Legendre quadrature of the same charges"}}


def measure_model_evaluation(ctx):
    """One model evaluation of Fig. 4 for Table I's initial design (staggered layout): head field
    solved with its wrap-around shield, critical-field searches, NEB, BER_tot; wall-clock."""
    from paper_1603_09493_gb300 import model
    t = time.perf_counter()
    r = model.evaluate(ctx, model.initial_design())
    r["wall_s"] = time.perf_counter() - t
    r["design"] = "Table I initial design"
    return r


def measure_ego(ctx, n=240, d=12, T=256, N=1 << 20):
    """EGO steps on the GPU (Sec. II.A) at the paper's scale of ten or more training
    designs per parameter: a batch of T likelihood evaluations (one Cholesky each)
    and the expected improvement at N candidates; wall-clock of each call."""
    from paper_1603_09493_gb300 import ego, synth
    X = synth.unit_points(n, d, 12, 0)
    y = np.sin(3.0 * X).sum(1)
    th = 10.0 ** (0.5 + synth.theta_unit_draws(T, d, 12, 0))
    ego.nll(ctx, X, y, th[:8])                                                 # warm-up
    t = time.perf_counter()
    v = ego.nll(ctx, X, y, th)
    t_nll = time.perf_counter() - t
    C = synth.unit_points(N, d, 12, 1)
    with ego.Kriging(ctx, X, y, th[int(np.argmin(v))]) as gp:
        gp.predict(C[:4096], float(y.min()))
        t = time.perf_counter()
        gp.predict(C, float(y.min()))
        t_ei = time.perf_counter() - t
    # the FP64 oracle on bounded samples of the same calls
    from oracle import ego as oego
    t = time.perf_counter()
    for q in range(16):
        oego.nll(X, y, th[q])
    o_nll = 16 / (time.perf_counter() - t)
    gpo = oego.fit(X, y, th[int(np.argmin(v))])
    t = time.perf_counter()
    oego.predict(gpo, C[:16384], float(y.min()))
    o_ei = 16384 / (time.perf_counter() - t)
    return {"nll_evals_per_s": T / t_nll, "ei_candidates_per_s": N / t_ei, "train_designs": n, "params": d,
            "theta_batch": T, "candidates": N, "note": "FP64; wall-clock per library call incl. host<->device copies",
            "cpu_baseline": {"nll_evals_per_s": o_nll, "ei_candidates_per_s": o_ei, "kind": "oracle",
                             "cores": 1, "workers": "one process (numpy FP64; its BLAS may thread the products)",
                             "sample": "16 likelihood evaluations; EI at 16384 candidates (numpy FP64)"}}


def measure_surrogate(ctx, torch, stream, n_infer=262144, n_train=65536, batch=4096, reps=20):
    """Surrogate MLP 16-256x4-2 (BF16 tensor-core GEMMs): inference evals/s on a
    device-resident screening batch, training samples/s (AdamW steps)."""
    from paper_1603_09493_gb300 import synth
    sizes = [16, 256, 256, 256, 256, 2]
    sur = ctx.surrogate((16, 256, 4, 2), synth.mlp_init_params(sizes, seed=3))
    g = torch.Generator(device="cpu").manual_seed(0)
    X = (torch.rand((n_infer, 16), generator=g) * 2 - 1).to("cuda")
    Xt = (torch.rand((n_train, 16), generator=g) * 2 - 1).numpy()
    Yt = (torch.rand((n_train, 2), generator=g) < 0.3).float().numpy()
    for _ in range(3):
        sur.infer(X)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        sur.infer(X)
    e1.record(stream)
    e1.synchronize()
    infer_s = e0.elapsed_time(e1) * 1e-3 / reps
    # screening: per-design error rates over 64 jitter samples each (inference + FP64 per-design means)
    n_jit = 64
    n_des = n_infer // n_jit
    for _ in range(3):
        sur.screen(X, n_des, n_jit)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        sur.screen(X, n_des, n_jit)
    e1.record(stream)
    e1.synchronize()
    screen_s = e0.elapsed_time(e1) * 1e-3 / reps
    sur.train(Xt[:batch], Yt[:batch], epochs=1, batch=batch, lr=1e-3, weight_decay=1e-4)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sur.train(Xt, Yt, epochs=1, batch=batch, lr=1e-3, weight_decay=1e-4)
    train_s = time.perf_counter() - t0
    flops_fwd = 2.0 * sum(a * b for a, b in zip(sizes[:-1], sizes[1:]))
    sur.destroy()
    return {"infer_evals_per_s": n_infer / infer_s, "infer_batch": n_infer,
            "infer_tflops": flops_fwd * n_infer / infer_s / 1e12,
            "screen_samples_per_s": n_infer / screen_s, "screen_designs": n_des, "screen_jitter": n_jit,
            "train_samples_per_s": n_train / train_s, "train_batch": batch,
            "note": "inference and screening timed with CUDA events on device-resident inputs; training "
                    "wall-clock per call including the host->device copy of the data"}


def measure_search(ctx, generations=8, population=256, top_k=16, n_jit_screen=64, n_jit_verify=64,
                   n_train=32768, n_heads=128, n_heldout=4096):
    """The surrogate on the write-head and media design problem (design.py: 12
    design and 4 jitter inputs, labels from LLG batches over the 81-mesh
    geometry grid with the moving head map and the layout's adjacent-track
    island): LLG labels of random designs, training, held-out error against
    fresh LLG solves of unseen designs and heads, then the surrogate-assisted
    design search.  Wall-clock of each part; the LLG-only time is every design
    of every generation solved at the loop's own LLG rate."""
    from paper_1603_09493_gb300 import design, evolve, synth
    grid = design.upload_grid(ctx)
    t0 = time.perf_counter()
    X, Y, _ = design.training_set(ctx, grid, n_train, n_heads, seed=41)
    label_s = time.perf_counter() - t0
    Xh, Yh, _ = design.training_set(ctx, grid, n_heldout, 16, seed=42, first_index=10 ** 6)
    sur = ctx.surrogate((16, 256, 4, 2), synth.mlp_init_params([16, 256, 256, 256, 256, 2], seed=4))
    t0 = time.perf_counter()
    sur.train(X, Y, epochs=40, batch=512, lr=2e-3, weight_decay=1e-4)
    train_s = time.perf_counter() - t0
    P = sur.infer(Xh)
    held = {"target": design.metrics(P[:, 0], Yh[:, 0]), "adjacent": design.metrics(P[:, 1], Yh[:, 1])}
    cfg = evolve.SearchConfig(generations=generations, population=population, top_k=top_k,
                              n_jitter_screen=n_jit_screen, n_jitter_verify=n_jit_verify, seed=43)
    res = design.search(ctx, sur, grid, cfg)
    sur.destroy()
    # the paper's write error rates (Eqs. 1-2, critical-field search) of the final elites
    ranked = design.rank_by_ber(ctx, grid, res.elite_Z)
    best = design.values(res.best_Z[None])
    best_ber = design.values(ranked["best_Z"][None])
    loop_s = res.screen_s + res.verify_s
    return {"problem": "12 design parameters (diameter, t_soft, t_hard, Ms, Ku, interlayer exchange, pitch, "
                       "layout, head peak, tilt, width, velocity) + 4 jitter values; labels: target switched, "
                       "adjacent-track island flipped; 81-mesh geometry grid, moving head map, 250 ps",
            "train_labels": n_train, "label_islands": 2 * n_train, "heads": n_heads, "heldout_labels": n_heldout,
            "heldout": held, "generations": generations, "population": population, "top_k": top_k,
            "n_jitter_screen": n_jit_screen, "n_jitter_verify": n_jit_verify,
            "best_design": {k: float(v[0]) for k, v in best.items()},
            "best_write_error_rate": float(res.best_rates[0]), "best_adjacent_flip_rate": float(res.best_rates[1]),
            "elites_by_ber": {"ber_targ": ranked["ber_targ"].tolist(), "ber_prev": ranked["ber_prev"].tolist(),
                              "best_ber_targ_plus_prev": float(ranked["ber_sum"][ranked["best"]]),
                              "best_design": {k: float(v[0]) for k, v in best_ber.items()},
                              "llg_runs": int(ranked["runs"]), "seconds": ranked["seconds"],
                              "method": "critical-field search of Sec. II.C on each elite's nominal island under "
                                        "its head, sigma = 0.015 H_A, BER = erfc(H_crit / (sqrt 2 sigma)) / 2"},
            "best_per_generation": [h["best_verified"] for h in res.history],
            "train_labels_s": label_s, "train_s": train_s, "screen_s": res.screen_s, "verify_s": res.verify_s,
            "llg_only_s": res.llg_only_s, "loop_vs_llg_only": res.llg_only_s / loop_s,
            "note": f"{n_jit_verify} LLG jitter samples per verified design (not 4096); an error rate of 0 means "
                    "none of the verified samples failed; wall-clock incl. host copies and head-map uploads"}


def main_surrogate_study(args):
    """The surrogate's label-count study on the design problem: LLG labels of
    random designs in rounds, training on the growing set, held-out error
    against fresh LLG solves after each round; one JSON line."""
    import torch
    from paper_1603_09493_gb300 import api, design, synth
    torch.cuda.set_device(0)
    ctx = api.Context(0, stream=torch.cuda.Stream())
    grid = design.upload_grid(ctx)
    Xh, Yh, _ = design.training_set(ctx, grid, 8192, 16, seed=52, first_index=10 ** 7)
    Xs, Ys, rows = [], [], []
    t_label = 0.0
    per_round = args.study_round
    for r in range(args.study_rounds):
        t0 = time.perf_counter()
        X, Y, _ = design.training_set(ctx, grid, per_round, 128, seed=51, first_index=r * per_round)
        t_label += time.perf_counter() - t0
        Xs.append(X)
        Ys.append(Y)
        Xa, Ya = np.concatenate(Xs), np.concatenate(Ys)
        sur = ctx.surrogate((16, 256, 4, 2), synth.mlp_init_params([16, 256, 256, 256, 256, 2], seed=4))
        t0 = time.perf_counter()
        sur.train(Xa, Ya, epochs=max(10, int(40 * 32768 / len(Xa))), batch=1024, lr=2e-3, weight_decay=1e-4)
        t_train = time.perf_counter() - t0
        P = sur.infer(Xh)
        sur.destroy()
        rows.append({"labels": len(Xa), "target": design.metrics(P[:, 0], Yh[:, 0]),
                     "adjacent": design.metrics(P[:, 1], Yh[:, 1]), "label_s_total": t_label, "train_s": t_train})
        print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    ctx.close()
    print(json.dumps({"workload": "surrogate label-count study on the design problem", "heldout_labels": 8192,
                      "rounds": rows}))
    return 0


def main_paper_loop(args):
    """The paper's optimisation loop (Sec. II.A, Fig. 4) on the GPU: every design's head field
    is solved from its Table I geometry (pole, charge sheet, trailing shield, under-layer), its
    target and previous bits go through the critical-field searches, its adjacent-track bit
    through the NEB barrier, and EGO (maximin Latin hypercube, kriging, expected improvement)
    proposes the next design from log10(BER_tot); one JSON line."""
    import torch
    from paper_1603_09493_gb300 import api, model
    torch.cuda.set_device(0)
    ctx = api.Context(0, stream=torch.cuda.Stream())
    keys = ["trailing_shield_gap_nm", "trailing_edge_angle_deg", "side_edge_angle_deg", "pole_tip_width_nm",
            "shield_thickness_nm", "K1_hard_MJ_m3", "A_ex_int_pJ_m", "down_track_offset_nm"]
    t = time.perf_counter()
    init = model.evaluate(ctx, model.initial_design(), layout=args.loop_layout)
    t_init = time.perf_counter() - t
    print(json.dumps({"initial_design": init}), file=sys.stderr, flush=True)
    t = time.perf_counter()
    res = model.optimise(ctx, keys, args.loop_init, args.loop_iters, seed=1, layout=args.loop_layout,
                         log=lambda r: print(json.dumps({k: r[k] for k in ("ber_tot", "ber_targ", "ber_prev",
                                                                            "ber_adj", "unit")}),
                                             file=sys.stderr, flush=True))
    t_loop = time.perf_counter() - t
    y = res["log10_ber_tot"]
    best_so_far = np.minimum.accumulate(y).tolist()
    ctx.close()
    print(json.dumps({
        "workload": "paper loop: Table I design -> solved head field -> critical-field searches -> NEB -> BER_tot, "
                    f"EGO over {len(keys)} parameters, {args.loop_layout} layout",
        "free_parameters": keys, "initial_design": init, "initial_seconds": t_init,
        "lhs_designs": args.loop_init, "ego_iterations": args.loop_iters,
        "log10_ber_tot": [float(v) for v in y], "best_so_far": best_so_far,
        "best_design": res["best"], "best_log10_ber_tot": res["best_log10_ber_tot"],
        "max_ei": res["max_ei"], "space_filling_steps": res["space_filling_steps"],
        "designs_writing_the_target": int(sum(not r["aborted"] for r in res["evaluations"])),
        "seconds": t_loop, "seconds_per_design": t_loop / len(y)}))
    return 0


def main_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_1603_09493_gb300 import synth
    mesh, mats, hm, p = workload()
    k = oracle_step_count(p)        # the step count of the whole workload, as the GPU arm uses
    W = host_cores()
    isl = synth.jittered_islands(W, seed=1)
    pool = OraclePool(1, threads=W)
    m = None

    def step(s_):
        q = type(p)(**{**p.__dict__})
        q.substeps, q.t0_ps, q.t_end_ps = k, s_ * DT_PS, (s_ + 1) * DT_PS
        return pool.run([(isl, q, m)])[0]

    try:
        for w_ in range(args.warmup):
            step(0)
        t = time.perf_counter()
        for s_ in range(args.steps):
            m = step(s_)
        el = time.perf_counter() - t
    finally:
        pool.close()
    value = W * args.steps * DT_PS * 1e-3 / el
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(mesh, k, "fp64 (oracle)", W, 1), "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": W, "kind": "oracle",
                             "workers": f"one process, its BLAS pinned to {W} threads (one per host core)",
                             "sample": f"{W} islands per step in one oracle batch, one 0.1 ps interval ({k} Heun "
                                       "steps) each, the state carried from step to step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main_uneven(args):
    """The uneven workload: 16 design variants (518-3906 nodes), each with
    `realisations` jittered targets plus two adjacent-track islands (staggered
    layout), all in one batch (one graph: a grouped demag GEMM over all mesh
    groups and one stage launch per occupancy class per Heun stage)."""
    import torch
    from paper_1603_09493_gb300 import _lib as L
    from paper_1603_09493_gb300 import api, synth
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    ctx = api.Context(0, stream=stream)
    variants = synth.design_variants()
    mats = synth.ecc_materials()
    hm = synth.synthetic_head_map()
    mids = [ctx.mesh_upload(v["mesh"], mats) for v in variants]
    hid = ctx.headmap_upload(hm)
    isl, role = synth.uneven_batch(variants, mids, realisations=args.realisations, seed=2, layout="staggered")
    p = synth.RunParams(dt_ps=DT_PS, alpha=0.1, rise_ps=100.0, v_m_per_s=20.0, x0_nm=-10.0, use_map=True)
    p.substeps = stable_k(ctx, hid, isl, p)
    bt = ctx.batch(isl, p, precision=L.PREC_BF16X3, map_id=hid)
    for _ in range(max(args.warmup, 1)):
        bt.advance(1)
    torch.cuda.synchronize()
    proc, cf = sample_clocks_start(args.clock_log)
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        bt.advance(1)
    e1.record(stream)
    e1.synchronize()
    clocks = sample_clocks_stop(proc, cf, 0)
    ms = e0.elapsed_time(e1)
    ok = bool(np.all(bt.read()["status"] == 0))
    launches_per_interval = bt.graph_kernels()
    kt = bt.kernel_times(reps=4)
    flops = sum(6.0 * int(np.sum(isl.mesh_id == mid)) * (3 * v["mesh"].n_nodes) ** 2
                for mid, v in zip(mids, variants))
    pk = peaks()
    peak, peak_source = gemm_peak(pk)
    B = len(isl)
    line = {"metric": METRIC, "value": B * args.steps * DT_PS * 1e-3 / (ms * 1e-3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3+f32", "data": "synthetic",
            "config": {"workload": f"uneven batch: 16 design variants (d 6-10 nm, t_soft/t_hard 0.2/0.5, circular "
                                   f"or 1.5:1 elliptical, {min(v['mesh'].n_nodes for v in variants)}-"
                                   f"{max(v['mesh'].n_nodes for v in variants)} nodes), {args.realisations} "
                                   "jittered targets + 2 staggered adjacent-track islands each",
                       "islands": B, "heun_steps_per_interval": p.substeps, "dt_ps": DT_PS},
            "gpu_launches": args.steps * launches_per_interval,
            "roofline": {"bound": "tensor", "achieved": flops / (kt["gemm_ms"] * 1e-3) / 1e12, "peak": peak,
                         "unit": "TFLOP/s", "peak_source": peak_source,
                         "frac": flops / (kt["gemm_ms"] * 1e-3) / 1e12 / peak, "traffic": None,
                         "kernel": "grouped demag GEMM over the 16 mesh groups (one launch)"},
            "kernel_ms": kt, "clocks": clocks, "status_ok": ok}
    bt.destroy()
    ctx.close()
    print(json.dumps(line))
    return 0


def main_extras(args):
    """The NEXT-row measurements alone (band barriers and EGO steps on the census
    mesh, the surrogate-assisted design search on the 209-node mesh), one JSON
    line; used for their launch lists."""
    import torch
    from paper_1603_09493_gb300 import api
    torch.cuda.set_device(0)
    ctx = api.Context(0, stream=torch.cuda.Stream())
    mesh, mats, hm, p = workload()
    mid = ctx.mesh_upload(mesh, mats)
    hid = ctx.headmap_upload(hm)
    line = {"workload": "extras (census mesh)",
            "neb": measure_neb(ctx, mid, hm, hid, mesh=None if args.no_cpu else mesh,
                               mats=None if args.no_cpu else mats),
            "ego": measure_ego(ctx), "search": measure_search(ctx)}
    ctx.close()
    print(json.dumps(line))
    return 0


def main_surrogate(args):
    """The surrogate measurement alone (inference and training), one JSON line; used for its
    launch list."""
    import torch
    from paper_1603_09493_gb300 import api
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    ctx = api.Context(0, stream=stream)
    line = {"workload": "surrogate MLP 16-256x4-2", "surrogate": measure_surrogate(ctx, torch, stream)}
    ctx.close()
    print(json.dumps(line))
    return 0


def main(args):
    if args.impl == "reference":
        return main_reference(args)
    if args.workload == "surrogate":
        return main_surrogate(args)
    if args.workload == "uneven":
        return main_uneven(args)
    if args.workload == "extras":
        return main_extras(args)
    if args.workload == "surrogate-study":
        return main_surrogate_study(args)
    if args.workload == "paper-loop":
        return main_paper_loop(args)
    import torch
    from paper_1603_09493_gb300 import _lib as L
    from paper_1603_09493_gb300 import api, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    if not os.path.exists(L.LIB_PATH):
        from paper_1603_09493_gb300 import build
        build.build()
    prec = {"bf16x3": L.PREC_BF16X3, "fp32": L.PREC_FP32, "bf16": L.PREC_BF16}[args.precision]
    mesh, mats, hm, p = workload()
    B = args.islands
    from paper_1603_09493_gb300 import shard
    lo, _ = shard.island_range(B, rank)
    isl = synth.jittered_islands(B, seed=1, first_index=lo)
    stream = torch.cuda.Stream()
    ctx = api.Context(local if world > 1 else 0, stream=stream)
    mid = ctx.mesh_upload(mesh, mats)
    isl.mesh_id[:] = mid
    hid = ctx.headmap_upload(hm)
    k = stable_k(ctx, hid, isl, p)
    p.substeps = k
    bt = ctx.batch(isl, p, precision=prec, map_id=hid)
    tuning = None
    if args.gemm_pair:
        # the CTA-pair demag GEMM (256 x 256 tiles on two SMs), its fastest k-block
        bt.set_tuning(256, 256, L.RASTER_AUTO, 2, 64, gemm_pair=1)
        tuning = {"gemm_pair": 1, "gemm_k_block": 64, "cached": False}
    elif not args.no_autotune:
        tuning = bt.autotune_cached(os.path.expanduser("~/.cache/bpmllg/tuning.json"),
                                    torch.cuda.get_device_name(), reps=4)
        bt.set_state(None, 0.0)
    for _ in range(max(args.warmup, 1)):
        bt.advance(1)
    stream.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    proc, cf = sample_clocks_start(args.clock_log)
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        bt.advance(1)
    e1.record(stream)
    e1.synchronize()
    clocks = sample_clocks_stop(proc, cf, local)
    ms = shard.max_over_ranks(e0.elapsed_time(e1), dist, device="cuda")
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    out = bt.read()
    ok = bool(np.all(out["status"] == 0))
    value = world * B * args.steps * DT_PS * 1e-3 / (ms * 1e-3)
    # kernel durations (events on the launching stream, outside the graph)
    launches_per_interval = bt.graph_kernels()
    kt = bt.kernel_times(reps=max(4, min(2 * k, 40)))
    bt.destroy()
    n = mesh.n_nodes
    K3 = 3 * n
    products = {L.PREC_BF16X3: 3, L.PREC_BF16: 1, L.PREC_FP32: 1}[prec]
    gemm_flops = products * 2.0 * B * K3 * K3
    pk = peaks()
    if prec == L.PREC_FP32:
        roof = {"bound": "alu", "achieved": gemm_flops / (kt["gemm_ms"] * 1e-3) / 1e12,
                "peak": SM_FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz (derived)"}
    else:
        peak, peak_source = gemm_peak(pk)
        roof = {"bound": "tensor", "achieved": gemm_flops / (kt["gemm_ms"] * 1e-3) / 1e12, "peak": peak,
                "unit": "TFLOP/s", "peak_source": peak_source}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = gemm_traffic(prec, B, n)
    roof["kernel"] = "demag GEMM"
    # step kernels: algorithmic HBM bytes, 48 n (stage 1) and 60 n (stage 2) per island. Stage 1
    # reads m and B_d and writes k1 and the operand; stage 2 reads m, k1 and B_d and writes m and
    # the operand (m* is rebuilt from m and k1, not stored). The operand is 12 B a node: FP32, or
    # BF16 hi plus lo.
    hbm_peak = pk["hbm_gbs"] if pk else 6800.0
    s1_bytes = B * n * (12 + 12 + 12 + 12)
    s2_bytes = B * n * (12 * 3 + 12 + 12)
    roof_steps = {"bound": "hbm", "unit": "GB/s", "peak": hbm_peak,
                  "stage1_achieved": s1_bytes / (kt["stage1_ms"] * 1e-3) / 1e9,
                  "stage2_achieved": s2_bytes / (kt["stage2_ms"] * 1e-3) / 1e9}
    roof_steps["stage1_frac"] = roof_steps["stage1_achieved"] / hbm_peak
    roof_steps["stage2_frac"] = roof_steps["stage2_achieved"] / hbm_peak
    wi = NCU_STAGE_WARP_INSTR.get(n) if prec == L.PREC_BF16X3 else None
    if wi and clocks:
        # the bound these kernels meet first: instruction issue (4 warp instructions per cycle
        # per SM at the run's median SM clock)
        issue_peak = SM_COUNT * ISSUE_PER_SM_CLK * clocks["sm_mhz"] * 1e6
        roof_steps["issue"] = {"bound": "issue", "unit": "warp instructions/s", "peak": issue_peak,
                               "warp_instructions_per_island_node": list(wi),
                               "stage1_frac": B * n * wi[0] / (kt["stage1_ms"] * 1e-3) / issue_peak,
                               "stage2_frac": B * n * wi[1] / (kt["stage2_ms"] * 1e-3) / issue_peak,
                               "peak_source": "152 SMs x 4 schedulers x median SM clock of the run"}

    # end to end through the one-call public API with pinned host buffers
    e2e = None
    if not args.no_e2e:
        isl_arr = api.island_array(isl)
        pin = torch.empty(isl_arr.nbytes, dtype=torch.uint8).pin_memory()
        pin.numpy()[:] = isl_arr.view(np.uint8)
        m_h = torch.empty((B, 3, n), dtype=torch.float32).pin_memory()
        sw_h = torch.empty(B, dtype=torch.uint8).pin_memory()
        ts_h = torch.empty(B, dtype=torch.float32).pin_memory()
        st_h = torch.empty(B, dtype=torch.int32).pin_memory()
        q = api.run_params(p, prec, hid)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        L.check(ctx.lib.bpm_run_batch(ctx.h, L.ptr(pin), B, __import__("ctypes").byref(q), args.steps,
                                      L.ptr(m_h), n, L.ptr(sw_h), L.ptr(ts_h), L.ptr(st_h)))
        el = time.perf_counter() - t0
        el = shard.max_over_ranks(el, dist, device="cuda")
        e2e = {"value": world * B * args.steps * DT_PS * 1e-3 / el, "unit": UNIT,
               "h2d_bytes_per_step": int(isl_arr.nbytes) / args.steps,
               "d2h_bytes_per_step": int(m_h.numel() * 4 + B * 9) / args.steps,
               "note": "one bpm_run_batch call per run of K intervals: batch setup, graph capture, island-table "
                       "H2D, K intervals, m_final/flags D2H"}
    extras = {}
    if rank == 0:
        extras["parity"] = measure_parity(ctx, hid)
    if not args.no_extras and rank == 0:
        extras["plain"] = measure_plain(ctx, isl, p, hid, prec, n)
        extras["plain_fp64"] = measure_plain_f64(ctx, isl, p, hid, mesh, mats)
        extras["uneven"] = measure_uneven(ctx, hm, hid)
        extras["surrogate"] = measure_surrogate(ctx, torch, stream)
        extras["neb"] = measure_neb(ctx, mid, hm, hid, mesh=None if args.no_cpu else mesh,
                                    mats=None if args.no_cpu else mats)
        extras["ego"] = measure_ego(ctx)
        extras["head_field"] = measure_head_field(ctx)
        extras["model_evaluation"] = measure_model_evaluation(ctx)
        extras["search"] = measure_search(ctx)
    ctx.close()
    if rank != 0:
        return 0
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"bf16x3": "bf16x3+f32", "fp32": "f32", "bf16": "bf16+f32"}[args.precision],
            "data": "synthetic", "config": config_dict(mesh, k, args.precision, B, world),
            "e2e": e2e, "gpu_launches": args.steps * launches_per_interval, "roofline": roof, "roofline_step_kernels": roof_steps,
            "kernel_ms": kt, "tuning": tuning, "clocks": clocks, "status_ok": ok, **extras}
    if world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(p, k)
    print(json.dumps(line))
    return 0


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16x3", choices=["bf16x3", "fp32", "bf16"])
    ap.add_argument("--islands", type=int, default=B_ISLANDS)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--gemm-pair", action="store_true", help="run the demag GEMM on CTA pairs (no autotune)")
    ap.add_argument("--workload", default="census",
                    choices=["census", "uneven", "extras", "surrogate", "surrogate-study", "paper-loop"])
    ap.add_argument("--study-round", type=int, default=32768, help="labels per round of the surrogate study")
    ap.add_argument("--study-rounds", type=int, default=4)
    ap.add_argument("--loop-init", type=int, default=16, help="Latin-hypercube designs of the paper loop")
    ap.add_argument("--loop-iters", type=int, default=16, help="EGO iterations of the paper loop")
    ap.add_argument("--loop-layout", default="staggered", choices=["centered", "staggered", "shingled"])
    ap.add_argument("--realisations", type=int, default=512)
    ap.add_argument("--clock-log", default="", help="also write the raw nvidia-smi clock samples here")
    sys.exit(main(ap.parse_args()))
