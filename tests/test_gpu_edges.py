"""Edge cases of the batched path: an empty batch, a single island (one valid
row of a 128-row GEMM tile) against the FP64 oracle, and the largest mesh the
library accepts (8192 nodes).

For the largest mesh the oracle's dense demag assembly (a 24000-unknown LU)
is out of reach, so the check there covers the assembly residuals, the
exchange, anisotropy and head terms against the oracle without its demag,
finite unit-norm states after a few intervals with every term on, and the
rejection of one node more than the limit."""
import os

import numpy as np
import pytest

from oracle import fem, llg
from paper_1603_09493_gb300 import _lib as L
from paper_1603_09493_gb300 import api, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not os.path.exists(L.LIB_PATH):
        from paper_1603_09493_gb300 import build
        build.build()
    c = api.Context(0)
    yield c
    c.close()


def test_empty_batch_is_rejected(ctx):
    # through the C ABI directly: a batch of zero islands is an argument error
    from ctypes import byref, c_void_p
    ctx.mesh_upload(synth.small_island_mesh(), synth.ecc_materials())
    q = api.run_params(synth.RunParams(dt_ps=0.1, substeps=2))
    h = c_void_p()
    assert ctx.lib.bpm_batch_create(ctx.h, None, 0, byref(q), byref(h)) == L.BPM_ERR_ARG
    assert not h.value
    assert ctx.lib.bpm_run_batch(ctx.h, None, 0, byref(q), 1, None, 0, None, None, None) == L.BPM_ERR_ARG


def test_single_island_matches_oracle(ctx):
    mesh = synth.small_island_mesh()
    mats = synth.ecc_materials()
    ops = fem.MeshOperators(mesh.xyz_nm, mesh.tets, mesh.tet_region, mats)
    mid = ctx.mesh_upload(mesh, mats)
    hm = synth.synthetic_head_map()
    hid = ctx.headmap_upload(hm)
    isl = synth.jittered_islands(1, seed=5, mesh_id=mid)
    p = synth.RunParams(dt_ps=0.1, t_end_ps=30.0, alpha=0.1, rise_ps=10.0, use_map=True, x0_nm=-2.0,
                        uniform_T=synth.uniform_field(0.6, 165.0))
    p.substeps = llg.stable_substeps(llg.Batch(ops, isl, p, head_map=hm))
    ref = llg.Batch(ops, isl, p, head_map=hm).run()
    for prec in (L.PREC_FP32, L.PREC_BF16X3):
        out = ctx.run_batch(isl, p, p.n_intervals, precision=prec, map_id=hid)
        err = np.abs(out["m"].transpose(0, 2, 1) - ref["m"]).max()
        print(f"single island, prec {prec}: max |dm| {err:.2e}")
        assert err <= 1e-3
        assert np.array_equal(out["switched"], ref["switched"])
        assert np.all(out["status"] == 0)


def _largest_mesh():
    # 10 hexagonal rings (331 nodes a plane) x 24 planes = 7944 nodes, 20 nm across
    return synth.layered_island_mesh(20.0, 7.0, 3.0, rings=10, hard_slabs=16, soft_slabs=7, seed=3)


def test_largest_mesh(ctx):
    mesh = _largest_mesh()
    assert 7900 <= mesh.n_nodes <= 8192
    mats = synth.ecc_materials()
    mid = ctx.mesh_upload(mesh, mats)
    info = ctx.mesh_info(mid)
    assert info["n_nodes"] == mesh.n_nodes
    assert info["cg_residual_neumann"] < 1e-12 and info["cg_residual_dirichlet"] < 1e-12
    ops = fem.MeshOperators(mesh.xyz_nm, mesh.tets, mesh.tet_region, mats, with_demag=False)
    hm = synth.synthetic_head_map()
    hid = ctx.headmap_upload(hm)
    B = 130                                                   # one full and one ragged row tile
    isl = synth.jittered_islands(B, seed=7, mesh_id=mid)
    p = synth.RunParams(dt_ps=0.1, substeps=2, alpha=0.1, rise_ps=10.0, use_map=True,
                        uniform_T=synth.uniform_field(0.5, 160.0))
    rng = np.random.default_rng(3)
    m = rng.standard_normal((2, mesh.n_nodes, 3)) * 0.3 + np.array([0.0, 0.0, 1.0])
    m /= np.linalg.norm(m, axis=-1, keepdims=True)
    two = isl.subset(np.arange(2))
    ob = llg.Batch(ops, two, p, head_map=hm)
    with ctx.batch(two, p, precision=L.PREC_BF16X3, map_id=hid) as bt:
        bt.set_state(m.transpose(0, 2, 1).astype(np.float32), 0.0)
        mf = bt.read()["m"].transpose(0, 2, 1).astype(np.float64)
        for term in (L.TERM_EXCHANGE, L.TERM_ANISOTROPY, L.TERM_HEAD):
            g = bt.field(4.0, term).transpose(0, 2, 1)
            o = ob.field(mf, 4.0, term)
            err = np.abs(g - o).max() / max(np.abs(o).max(), 1e-3)
            print(f"largest mesh, term {term}: rel err {err:.2e}")
            assert err <= 2e-5
    # every term on, a ragged batch of 130 islands, a few intervals
    p.substeps = ctx.stable_substeps(isl, p, hid)[0]
    out = ctx.run_batch(isl, p, 3, precision=L.PREC_BF16X3, map_id=hid)
    assert np.all(out["status"] == 0)
    nrm = np.linalg.norm(out["m"][:, :, :mesh.n_nodes], axis=1)
    assert np.abs(nrm - 1.0).max() < 1e-5


def test_one_node_past_the_limit_is_rejected(ctx):
    mesh = _largest_mesh()
    n = mesh.n_nodes
    # append isolated nodes up to 8193 (they belong to no tet): the size check comes first
    extra = 8193 - n
    xyz = np.concatenate([mesh.xyz_nm, mesh.xyz_nm[:extra] + np.array([0.0, 0.0, 50.0])])
    big = synth.IslandMesh(xyz_nm=xyz, tets=mesh.tets, tet_region=mesh.tet_region,
                           z_interface_nm=mesh.z_interface_nm, height_nm=mesh.height_nm)
    with pytest.raises(RuntimeError):
        ctx.mesh_upload(big, synth.ecc_materials())


def test_undamped_precession_in_a_uniform_field(ctx):
    # alpha = 0, a uniform 1 T field along z and no other term: every node precesses about z at
    # gamma B, m_z stays fixed.  Heun with renormalisation keeps |m| and errs in phase by about
    # N (omega h)^3 / 6 after N steps (omega h = 0.0088 here).
    mid = ctx.mesh_upload(synth.small_island_mesh(), synth.ecc_materials())
    isl = synth.jittered_islands(3, seed=2, mesh_id=mid)
    isl.Hext_T[:] = 0.0
    p = synth.RunParams(dt_ps=0.1, substeps=2, alpha=0.0, rise_ps=0.0, use_map=False, term_mask=L.TERM_UNIFORM,
                        uniform_T=(0.0, 0.0, 1.0))
    n = ctx.mesh_info(mid)["n_nodes"]
    th = np.deg2rad(30.0)
    m0 = np.zeros((3, 3, n), np.float32)
    m0[:, 0, :], m0[:, 2, :] = np.sin(th), np.cos(th)
    intervals = 200                                              # 20 ps, 400 Heun steps
    with ctx.batch(isl, p, precision=L.PREC_FP32) as bt:
        bt.set_state(m0, 0.0)
        bt.advance(intervals)
        m = bt.read()["m"]
    gamma = 1.76085963023e-1                                      # rad / (ps T)
    phi = gamma * 1.0 * intervals * p.dt_ps                       # dm/dt = -gamma m x B: phi' = +gamma B
    ref = np.array([np.sin(th) * np.cos(phi), np.sin(th) * np.sin(phi), np.cos(th)])
    steps = intervals * p.substeps
    wh = gamma * p.dt_ps / p.substeps
    tol = steps * wh ** 3 / 6.0 + 1e-4                            # phase error + FP32 rounding over 400 steps
    err = np.abs(m - ref[None, :, None]).max()
    print(f"precession: max |dm| {err:.2e}, bound {tol:.2e}")
    assert err <= tol
    assert np.abs(m[:, 2, :] - np.cos(th)).max() <= 1e-5


def test_no_field_leaves_the_state_unchanged(ctx):
    mid = ctx.mesh_upload(synth.small_island_mesh(), synth.ecc_materials())
    isl = synth.jittered_islands(4, seed=3, mesh_id=mid)
    p = synth.RunParams(dt_ps=0.1, substeps=3, alpha=0.1, use_map=False, term_mask=0)
    n = ctx.mesh_info(mid)["n_nodes"]
    rng = np.random.default_rng(9)
    m0 = rng.standard_normal((4, 3, n))
    m0 = (m0 / np.linalg.norm(m0, axis=1, keepdims=True)).astype(np.float32)
    for prec in (L.PREC_FP32, L.PREC_BF16X3):
        with ctx.batch(isl, p, precision=prec) as bt:
            bt.set_state(m0, 0.0)
            bt.advance(10)
            m = bt.read()["m"]
        assert np.abs(m - m0).max() <= 1e-6


def test_stoner_wohlfarth_switching_field_at_45_degrees(ctx):
    # a small homogeneous island (5 nm, hard material, no demag) reverses coherently: with the
    # field at 45 degrees to the easy axis (135 degrees from the initial +z) it switches above
    # h = B / B_K = 0.5 and stays below, B_K = 2 K / Ms (Stoner-Wohlfarth astroid)
    mesh = synth.layered_island_mesh(5.0, 4.0, 1.0, rings=2, hard_slabs=4, soft_slabs=1, seed=0)
    K, Ms = 0.9e6, 0.8e6
    mats = synth.ecc_materials(Ms_hard=Ms, Ku_hard=K, Ms_soft=Ms, Ku_soft=K, interlayer_scale=1.0)
    mid = ctx.mesh_upload(mesh, mats)
    BK = 2.0 * K / Ms
    hs = [0.47, 0.53]
    isl = synth.Islands(np.full(2, mid, np.int32), np.ones(2, np.float32), np.ones(2, np.float32),
                        np.tile(np.array([[0.0, 0.0, 1.0]], np.float32), (2, 1)), np.zeros((2, 2), np.float32),
                        np.array([[h * BK * np.sin(np.deg2rad(135.0)), 0.0, h * BK * np.cos(np.deg2rad(135.0))]
                                  for h in hs], np.float32))
    p = synth.RunParams(dt_ps=1.0, t_end_ps=600.0, alpha=1.0, rise_ps=0.0, use_map=False,
                        term_mask=L.TERM_EXCHANGE | L.TERM_ANISOTROPY | L.TERM_UNIFORM)
    p.substeps = ctx.stable_substeps(isl, p)[0]
    out = ctx.run_batch(isl, p, p.n_intervals, precision=L.PREC_FP32)
    print("switched", out["switched"], "t_sw", out["t_sw"])
    assert not out["switched"][0] and out["switched"][1]


def test_device_output_run_matches_the_host_run(ctx):
    # bpm_run_batch_dev writes the same results into device buffers
    mid = ctx.mesh_upload(synth.small_island_mesh(), synth.ecc_materials())
    hid = ctx.headmap_upload(synth.synthetic_head_map())
    isl = synth.jittered_islands(37, seed=8, mesh_id=mid)
    p = synth.RunParams(dt_ps=0.1, t_end_ps=20.0, alpha=0.1, rise_ps=10.0, use_map=True, x0_nm=-2.0,
                        uniform_T=synth.uniform_field(0.6, 165.0))
    p.substeps = ctx.stable_substeps(isl, p, hid)[0]
    host = ctx.run_batch(isl, p, p.n_intervals, map_id=hid)
    dev = ctx.run_batch_dev(isl, p, p.n_intervals, map_id=hid)
    assert dev["m"].is_cuda and dev["switched"].is_cuda
    assert np.array_equal(dev["m"].cpu().numpy(), host["m"])
    assert np.array_equal(dev["switched"].cpu().numpy(), host["switched"])
    assert np.array_equal(dev["t_sw"].cpu().numpy(), host["t_sw"])
    assert np.array_equal(dev["status"].cpu().numpy(), host["status"])
