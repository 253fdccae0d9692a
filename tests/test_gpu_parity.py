"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances (from the arithmetic, stated per check):
* assembly is FP64 on the GPU vs FP64 dense LU in the oracle: the batched CG
  stops at a 1e-12 relative residual, so N agrees to ~1e-9 of max|N|;
* FP32 field terms: single rounding of each stored operand and FP32
  accumulation, ~1e-6 relative to the term's scale;
* BF16 hi/lo split demag: operands carry ~16 mantissa bits, ~1e-5 relative;
* dynamics: max |dm| <= 1e-3 over the first 100 ps, identical switch outcome,
  |dt_sw| <= 2 ps (the acceptance bar of the batched mixed-precision path).
"""
import math
import os

import numpy as np
import pytest

from oracle import fem, llg
from paper_1603_09493_gb300 import _lib as L
from paper_1603_09493_gb300 import api, synth

pytestmark = pytest.mark.gpu

MU0 = 4e-7 * math.pi


@pytest.fixture(scope="module")
def ctx():
    if not os.path.exists(L.LIB_PATH):
        from paper_1603_09493_gb300 import build
        build.build()
    c = api.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def small(ctx):
    mesh = synth.small_island_mesh()
    mats = synth.ecc_materials()
    ops = fem.MeshOperators(mesh.xyz_nm, mesh.tets, mesh.tet_region, mats)
    mid = ctx.mesh_upload(mesh, mats, keep_f64=True)
    return mesh, mats, ops, mid


@pytest.fixture(scope="module")
def headmap(ctx):
    hm = synth.synthetic_head_map()
    return hm, ctx.headmap_upload(hm)


def _check_assembly(ctx, ops, mid):
    info = ctx.mesh_info(mid)
    assert info["n_nodes"] == ops.n
    V = ctx.get_operator(mid, L.OP_VOLUMES_F64)
    Ms = ctx.get_operator(mid, L.OP_NODAL_MS_F64)
    Ku = ctx.get_operator(mid, L.OP_NODAL_KU_F64)
    assert np.allclose(V, ops.V, rtol=1e-12, atol=0)
    assert np.allclose(Ms, ops.Ms, rtol=1e-12, atol=0)
    assert np.allclose(Ku, ops.Ku, rtol=1e-12, atol=1e-6)
    S = ctx.get_operator(mid, L.OP_EXCHANGE_F32).astype(np.float64)
    assert np.abs(S - ops.S).max() <= 2e-6 * np.abs(ops.S).max()
    N64 = ctx.get_operator(mid, L.OP_DEMAG_F64)
    assert np.abs(N64 - ops.demag).max() <= 1e-9 * np.abs(ops.demag).max()
    N32 = ctx.get_operator(mid, L.OP_DEMAG_F32).astype(np.float64)
    ref = -MU0 * 1e6 * ops.demag
    assert np.abs(N32 - ref).max() <= 1e-6 * np.abs(ref).max()
    lam = ops.exchange_lambda_max()
    assert abs(info["exchange_lambda_max_T"] - lam) <= 1e-3 * lam
    assert info["cg_residual_neumann"] < 1e-12 and info["cg_residual_dirichlet"] < 1e-12
    assert abs(info["volume_nm3"] - ops.V.sum()) < 1e-9 * ops.V.sum()


def test_assembly_small_mesh(ctx, small):
    _, _, ops, mid = small
    _check_assembly(ctx, ops, mid)


def test_assembly_census_mesh(ctx):
    mesh = synth.census_island_mesh()
    mats = synth.ecc_materials()
    ops = fem.MeshOperators(mesh.xyz_nm, mesh.tets, mesh.tet_region, mats)
    mid = ctx.mesh_upload(mesh, mats, keep_f64=True)
    _check_assembly(ctx, ops, mid)


def _smooth_state(xyz, B, seed):
    rng = np.random.default_rng(seed)
    m = np.zeros((B, xyz.shape[0], 3))
    for b in range(B):
        a = rng.uniform(-0.6, 0.6, size=(3, 3))
        m[b] = np.stack([a[0, 0] * np.sin(0.4 * xyz[:, 0] + a[0, 1]) + a[0, 2] * 0.1 * xyz[:, 2],
                         a[1, 0] * np.cos(0.3 * xyz[:, 1] + a[1, 1]),
                         np.ones(xyz.shape[0]) + a[2, 0] * 0.05 * xyz[:, 2]], 1)
    return m / np.linalg.norm(m, axis=2, keepdims=True)


@pytest.mark.parametrize("prec", [L.PREC_FP32, L.PREC_BF16X3_REF, L.PREC_BF16X3])
def test_field_terms(ctx, small, headmap, prec):
    mesh, mats, ops, mid = small
    hm, hid = headmap
    B = 100                                     # not a multiple of the 128-row tile
    isl = synth.jittered_islands(B, seed=21, mesh_id=mid)
    isl.Hext_T[:] = np.array([0.01, -0.02, 0.03], np.float32)
    p = synth.RunParams(dt_ps=0.1, substeps=1, alpha=0.1, rise_ps=80.0, use_map=True,
                        uniform_T=synth.uniform_field(0.4, 160.0))
    m = _smooth_state(ops.xyz, B, 3)
    ob = llg.Batch(ops, isl, p, head_map=hm)
    with ctx.batch(isl, p, precision=prec, map_id=hid) as bt:
        bt.set_state(m.transpose(0, 2, 1).astype(np.float32), 0.0)
        mf = bt.read()["m"].transpose(0, 2, 1).astype(np.float64)
        t = 37.5
        tol = {L.TERM_EXCHANGE: 2e-6, L.TERM_ANISOTROPY: 2e-6, L.TERM_HEAD: 2e-6, L.TERM_UNIFORM: 2e-6,
               L.TERM_DEMAG: 2e-6 if prec == L.PREC_FP32 else 2e-5}
        for term, rel in tol.items():
            g = bt.field(t, term).transpose(0, 2, 1)
            o = ob.field(mf, t, term)
            scale = max(np.abs(o).max(), 1e-3)
            err = np.abs(g - o).max()
            print(f"prec {prec} term {term}: max err {err:.3e} scale {scale:.3e}")
            assert err <= rel * scale * 10, (term, err, scale)


def _traj_parity(ctx, ops, mid, hm, hid, isl, p, prec, every, n_samples):
    ob = llg.Batch(ops, isl, p, head_map=hm)
    ref = ob.run(sample_every=every)
    worst = 0.0
    with ctx.batch(isl, p, precision=prec, map_id=hid) as bt:
        for s in range(n_samples):
            bt.advance(every)
            g = bt.read()["m"].transpose(0, 2, 1)
            worst = max(worst, float(np.abs(g - ref["samples"][s]).max()))
        out = bt.read()
    return worst, ref, out


@pytest.mark.parametrize("prec", [L.PREC_FP32, L.PREC_BF16X3_REF, L.PREC_BF16X3])
def test_dynamics_parity_first_100ps(ctx, small, headmap, prec):
    mesh, mats, ops, mid = small
    hm, hid = headmap
    B = 40
    isl = synth.jittered_islands(B, seed=31, mesh_id=mid)
    isl.pos_nm[:, 0] += 6.0                     # under the head centre mid-run
    p = synth.RunParams(dt_ps=0.1, t_end_ps=100.0, alpha=0.1, rise_ps=50.0, use_map=True, v_m_per_s=20.0,
                        x0_nm=-4.0, uniform_T=synth.uniform_field(0.5, 170.0))
    p.substeps = llg.stable_substeps(llg.Batch(ops, isl, p, head_map=hm))
    worst, ref, out = _traj_parity(ctx, ops, mid, hm, hid, isl, p, prec, every=20, n_samples=50)
    assert worst <= 1e-3, worst
    assert np.all(out["status"] == 0)
    assert np.abs(np.linalg.norm(out["m"], axis=1) - 1.0).max() < 1e-5


def test_switching_outcomes_and_times(ctx, small):
    mesh, mats, ops, mid = small
    B = 64
    isl = synth.jittered_islands(B, seed=41, mesh_id=mid)
    Bmag = 0.81
    isl.Hext_T[:] = np.array([math.sin(math.radians(170)) * Bmag, 0.0, math.cos(math.radians(170)) * Bmag],
                             np.float32)
    p = synth.RunParams(dt_ps=0.1, t_end_ps=200.0, alpha=0.1, rise_ps=0.0, use_map=False)
    ob = llg.Batch(ops, isl, p)
    p.substeps = llg.stable_substeps(ob)
    ref = ob.run()
    assert 0 < ref["switched"].sum() < B            # a mix of outcomes
    for prec in (L.PREC_FP32, L.PREC_BF16X3):
        out = ctx.run_batch(isl, p, p.n_intervals, precision=prec)
        assert np.array_equal(out["switched"], ref["switched"]), prec
        sw = ref["t_sw"] > 0
        assert np.array_equal(out["t_sw"] > 0, sw)
        assert np.abs(out["t_sw"][sw] - ref["t_sw"][sw]).max() <= 2.0


def test_census_size_sampled_islands(ctx, headmap):
    # the full-size workload shape (4096 islands, ~1500-node mesh, head map); the
    # oracle recomputes a sample of islands one by one
    hm, hid = headmap
    mesh = synth.census_island_mesh()
    mats = synth.ecc_materials()
    ops = fem.MeshOperators(mesh.xyz_nm, mesh.tets, mesh.tet_region, mats)
    mid = ctx.mesh_upload(mesh, mats)
    B = 4096
    isl = synth.jittered_islands(B, seed=1, mesh_id=mid)
    p = synth.RunParams(dt_ps=0.1, t_end_ps=1.0, alpha=0.1, rise_ps=100.0, use_map=True, x0_nm=-2.0)
    p.substeps = ctx.stable_substeps(isl, p, hid)[0]
    assert p.substeps == llg.stable_substeps(llg.Batch(ops, isl.subset(np.arange(B)), p, head_map=hm))
    out = ctx.run_batch(isl, p, p.n_intervals, precision=L.PREC_BF16X3, map_id=hid)
    assert np.all(out["status"] == 0)
    assert np.abs(np.linalg.norm(out["m"], axis=1) - 1.0).max() < 1e-5
    pick = np.array([0, 1234, 2047, 4095])
    ob = llg.Batch(ops, isl.subset(pick), p, head_map=hm)
    ref = ob.run()
    assert np.abs(out["m"][pick].transpose(0, 2, 1) - ref["m"]).max() <= 1e-3


def test_plain_one_island_form_matches_batch_and_oracle(ctx, small, headmap):
    # the one-island-per-launch baseline (FP32 GEMV demag) gives the same
    # outcomes as the batched path; only the demag summation order differs
    mesh, mats, ops, mid = small
    hm, hid = headmap
    isl = synth.jittered_islands(6, seed=61, mesh_id=mid)
    p = synth.RunParams(dt_ps=0.1, t_end_ps=20.0, alpha=0.1, rise_ps=10.0, use_map=True, x0_nm=0.0,
                        uniform_T=synth.uniform_field(0.6, 170.0))
    p.substeps = llg.stable_substeps(llg.Batch(ops, isl, p, head_map=hm))
    plain = ctx.run_plain(isl, p, p.n_intervals, map_id=hid)
    batch = ctx.run_batch(isl, p, p.n_intervals, precision=L.PREC_FP32, map_id=hid)
    ref = llg.Batch(ops, isl, p, head_map=hm).run()
    assert plain["device_ms"] > 0
    assert np.abs(plain["m"] - batch["m"]).max() <= 1e-5
    assert np.abs(plain["m"].transpose(0, 2, 1) - ref["m"]).max() <= 1e-3
    assert np.array_equal(plain["switched"], batch["switched"])


def test_autotuner_choices_do_not_change_results(ctx, small, headmap):
    # tile width and CTA size are launch shapes only: m is bitwise identical
    # for every tuning; <m_z> sums in a CTA-size dependent order (last bits)
    mesh, mats, ops, mid = small
    hm, hid = headmap
    isl = synth.jittered_islands(300, seed=71, mesh_id=mid)
    p = synth.RunParams(dt_ps=0.1, substeps=8, alpha=0.1, rise_ps=10.0, use_map=True,
                        uniform_T=synth.uniform_field(0.7, 170.0))
    outs = []
    # (tile width, stage CTA size, GEMM tile order, islands per stage CTA)
    for tn, nt, ras, ipb in [(256, 256, L.RASTER_AUTO, 1), (128, 128, L.RASTER_N, 1), (256, 512, L.RASTER_M, 1),
                             (128, 256, L.RASTER_AUTO, 1), (256, 256, L.RASTER_N, 2), (128, 256, L.RASTER_M, 2)]:
        with ctx.batch(isl, p, precision=L.PREC_BF16X3, map_id=hid) as bt:
            bt.set_tuning(tn, nt, ras, ipb)
            bt.advance(20)
            outs.append(bt.read())
    for o in outs[1:]:
        assert np.array_equal(o["m"], outs[0]["m"])
        assert np.abs(o["mz"] - outs[0]["mz"]).max() <= 1e-6
    with ctx.batch(isl, p, precision=L.PREC_BF16X3, map_id=hid) as bt:
        t = bt.autotune(reps=2)
        assert t["gemm_tile_n"] in (128, 256) and t["stage_threads"] in (128, 256, 512)
        assert t["gemm_raster"] in (0, 1, 2) and t["stage_islands"] in (1, 2)
        assert t["gemm_ms"] > 0 and t["stage_ms"] > 0
        bt.set_state(None, 0.0)
        bt.advance(20)
        assert np.array_equal(bt.read()["m"], outs[0]["m"])


def test_two_stream_intervals_give_the_same_states(ctx, small, headmap):
    # tuning streams = s integrates chunks of islands (multiples of 128) as chains on their own
    # streams; every island sees the same kernels, so m, the switch data and <m_z> are bitwise
    # those of one chain.  300 islands: 256 + 44 (s = 2), 128 + 128 + 44 (s = 3, 4); 512: 256 + 256
    # (s = 2, 3) or four chunks of 128; 255 islands: 128 + 127.  A real GEMM wait that runs
    # out inside the two-chain graph reports BPM_ERR_TIMEOUT like the one-chain graph.
    mesh, mats, ops, mid = small
    hm, hid = headmap
    p = synth.RunParams(dt_ps=0.1, substeps=8, alpha=0.1, rise_ps=10.0, use_map=True, x0_nm=-3.0,
                        uniform_T=synth.uniform_field(0.7, 170.0))
    for B in (300, 512, 255):
        isl = synth.jittered_islands(B, seed=B, mesh_id=mid)
        outs = []
        for streams in (1, 2, 3, 4):
            with ctx.batch(isl, p, precision=L.PREC_BF16X3, map_id=hid) as bt:
                bt.set_tuning(256, 256, L.RASTER_AUTO, 2, 32, streams=streams)
                bt.advance(30)
                outs.append(bt.read())
        for o in outs[1:]:
            for key in ("m", "switched", "t_sw", "mz", "status"):
                assert np.array_equal(o[key], outs[0][key]), (B, key)
            assert np.all(o["status"] == 0)
    isl = synth.jittered_islands(300, seed=5, mesh_id=mid)
    with ctx.batch(isl, p, precision=L.PREC_BF16X3, map_id=hid) as bt:
        bt.set_tuning(256, 256, L.RASTER_AUTO, 2, 32, streams=3)
        L.check(ctx.lib.bpm_debug_set_gemm_wait(bt.h, 1000.0))        # 1 us
        bt.advance(2)
        with pytest.raises(L.BpmError) as e:
            bt.read()
        assert e.value.code == L.BPM_ERR_TIMEOUT
        L.check(ctx.lib.bpm_debug_set_gemm_wait(bt.h, 0.0))
        L.check(ctx.lib.bpm_debug_set_gemm_error(bt.h, 0))
        bt.set_state(None, 0.0)
        bt.advance(2)
        assert np.all(bt.read()["status"] == 0)
    with ctx.batch(synth.jittered_islands(512, seed=7, mesh_id=mid), p, precision=L.PREC_BF16X3,
                   map_id=hid) as bt:
        t = bt.autotune(reps=2)
        assert t["streams"] in (1, 2, 3, 4)
    # a batch of three meshes: its groups dealt to two or three chains
    mid2 = ctx.mesh_upload(synth.layered_island_mesh(7.0, 6.0, 4.0, rings=2, hard_slabs=9, soft_slabs=6, seed=5),
                           mats)
    mid3 = ctx.mesh_upload(synth.layered_island_mesh(6.0, 5.0, 3.0, rings=2, hard_slabs=7, soft_slabs=4, seed=6),
                           mats)
    isl = synth.Islands.concat([synth.jittered_islands(101, seed=73, mesh_id=mid),
                                synth.jittered_islands(200, seed=74, mesh_id=mid2),
                                synth.jittered_islands(57, seed=75, mesh_id=mid3)])
    outs = []
    for streams in (1, 2, 4):
        with ctx.batch(isl, p, precision=L.PREC_BF16X3, map_id=hid) as bt:
            bt.set_tuning(256, 256, L.RASTER_AUTO, 2, 32, streams=streams)
            bt.advance(20)
            outs.append(bt.read())
    for o in outs[1:]:
        for key in ("m", "switched", "t_sw", "mz", "status"):
            assert np.array_equal(o[key], outs[0][key]), key


def test_two_islands_per_cta_odd_groups(ctx, small, headmap):
    # two islands per stage CTA over two mesh groups of odd sizes (the last CTA
    # of each group holds one island): the same m and switch data as one island
    # per CTA, for the one-group launch and the grouped launch
    mesh, mats, ops, mid = small
    hm, hid = headmap
    mid2 = ctx.mesh_upload(synth.layered_island_mesh(7.0, 6.0, 4.0, rings=2, hard_slabs=9, soft_slabs=6, seed=5),
                           mats)
    p = synth.RunParams(dt_ps=0.1, substeps=8, alpha=0.1, rise_ps=10.0, use_map=True,
                        uniform_T=synth.uniform_field(0.7, 170.0))
    one = synth.jittered_islands(101, seed=73, mesh_id=mid)
    two = synth.Islands.concat([one, synth.jittered_islands(57, seed=74, mesh_id=mid2)])
    for isl in (one, two):
        outs = []
        for ipb in (1, 2):
            with ctx.batch(isl, p, precision=L.PREC_BF16X3, map_id=hid) as bt:
                bt.set_tuning(256, 256, L.RASTER_AUTO, ipb)
                bt.advance(20)
                outs.append(bt.read())
        assert np.all(outs[1]["status"] == 0)
        assert np.array_equal(outs[1]["m"], outs[0]["m"])
        assert np.array_equal(outs[1]["switched"], outs[0]["switched"])
        assert np.abs(outs[1]["mz"] - outs[0]["mz"]).max() <= 1e-6


@pytest.mark.parametrize("prec,tol", [(L.PREC_FP32, 1e-6), (L.PREC_BF16X3, 1e-6)])
def test_energy_and_torque_match_oracle(ctx, small, headmap, prec, tol):
    # bpm_batch_energy on random states against the oracle's energy and |m x B|; the bar
    # is relative to the sum of the individual term energies' magnitudes (measured 5e-8,
    # torque 1e-7)
    mesh, mats, ops, mid = small
    hm, hid = headmap
    isl = synth.jittered_islands(5, seed=91, mesh_id=mid)
    p = synth.RunParams(dt_ps=0.1, substeps=4, alpha=0.1, rise_ps=10.0, use_map=True, x0_nm=-3.0,
                        uniform_T=synth.uniform_field(0.4, 160.0))
    rng = np.random.default_rng(17)
    m = rng.standard_normal((5, ops.n, 3)) * 0.5 + np.array([0.0, 0.0, 1.0])
    m /= np.linalg.norm(m, axis=-1, keepdims=True)
    with ctx.batch(isl, p, precision=prec, map_id=hid) as bt:
        bt.set_state(m.transpose(0, 2, 1).astype(np.float32), 4.0)
        E, T = bt.energy()
    pp = synth.RunParams(**{**p.__dict__})
    ob = llg.Batch(ops, isl, pp, head_map=hm)
    m32 = m.astype(np.float32).astype(np.float64)
    ref = ob.energy(m32, 4.0)
    scale = np.zeros(5)
    for term in (llg.T_EXCHANGE, llg.T_ANISOTROPY, llg.T_DEMAG, llg.T_HEAD, llg.T_UNIFORM):
        pt = synth.RunParams(**{**p.__dict__, "term_mask": term})
        scale += np.abs(llg.Batch(ops, isl, pt, head_map=hm).energy(m32, 4.0))
    B = ob.field(m32, 4.0)
    tref = np.linalg.norm(np.cross(m32, B), axis=-1).max(axis=1)
    print("energy rel err", np.abs(E - ref).max() / scale.min(), "torque rel err", np.abs(T - tref).max() / tref.max())
    assert np.all(np.abs(E - ref) <= tol * scale)
    assert np.allclose(T, tref, rtol=10 * tol)


def test_energy_decreases_under_damping(ctx, small):
    # a static uniform field (no ramp, no head): with damping the energy of every island
    # only decreases from interval to interval, and the torque falls as it settles
    mesh, mats, ops, mid = small
    isl = synth.jittered_islands(8, seed=92, mesh_id=mid)
    p = synth.RunParams(dt_ps=0.1, alpha=0.5, rise_ps=0.0, use_map=False, uniform_T=synth.uniform_field(0.6, 150.0))
    p.substeps = llg.stable_substeps(llg.Batch(ops, isl, p))
    with ctx.batch(isl, p, precision=L.PREC_BF16X3) as bt:
        Es, Ts = [], []
        for _ in range(6):
            E, T = bt.energy()
            Es.append(E)
            Ts.append(T)
            bt.advance(5)
    Es = np.array(Es)
    assert np.all(np.diff(Es, axis=0) <= 1e-6 * np.abs(Es).max())
    assert np.all(Ts[-1] < Ts[0])
