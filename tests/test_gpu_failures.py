"""Failure detection without a GPU fault: every failure is made on the host
(bad inputs, a NaN state, the GEMM error flag raised from the host) and must
come back as an error code or a per-island status, with the context usable
afterwards."""
import ctypes
import os

import numpy as np
import pytest

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


@pytest.fixture(scope="module")
def mid(ctx):
    return ctx.mesh_upload(synth.small_island_mesh(), synth.ecc_materials())


def test_bad_meshes_are_rejected(ctx):
    m = synth.small_island_mesh()
    bad = synth.IslandMesh(m.xyz_nm.copy(), m.tets.copy(), m.tet_region, m.z_interface_nm, m.height_nm)
    bad.xyz_nm[bad.tets[0, 3]] = bad.xyz_nm[bad.tets[0, 0]]          # collapse tet 0
    with pytest.raises(L.BpmError) as e:
        ctx.mesh_upload(bad, synth.ecc_materials())
    assert e.value.code == -1 and "degenerate" in str(e.value)
    bad2 = synth.IslandMesh(m.xyz_nm, m.tets.copy(), m.tet_region, m.z_interface_nm, m.height_nm)
    bad2.tets[5, 1] = m.n_nodes + 3
    with pytest.raises(L.BpmError) as e:
        ctx.mesh_upload(bad2, synth.ecc_materials())
    assert e.value.code == -1
    # the context still works
    assert ctx.mesh_upload(m, synth.ecc_materials()) >= 0


def test_bad_island_parameters_are_rejected(ctx, mid):
    isl = synth.nominal_islands(4, mesh_id=mid)
    isl.Ms_scale[2] = 0.0
    with pytest.raises(L.BpmError) as e:
        ctx.batch(isl, synth.RunParams(substeps=2), precision=L.PREC_BF16X3)
    assert e.value.code == -1 and "Ms_scale" in str(e.value)
    isl = synth.nominal_islands(4, mesh_id=mid + 100)
    with pytest.raises(L.BpmError):
        ctx.batch(isl, synth.RunParams(substeps=2))


def test_nonfinite_island_is_flagged_alone(ctx, mid):
    isl = synth.jittered_islands(6, seed=3, mesh_id=mid)
    p = synth.RunParams(dt_ps=0.1, substeps=6, alpha=0.1, rise_ps=0.0, uniform_T=(0.0, 0.0, -0.5))
    n = ctx.mesh_info(mid)["n_nodes"]
    m0 = np.zeros((6, 3, n), np.float32)
    m0[:, 2, :] = 1.0
    m0[4, 0, 7] = np.nan
    with ctx.batch(isl, p, precision=L.PREC_BF16X3) as bt:
        bt.set_state(m0, 0.0)
        bt.advance(5)
        out = bt.read()
    assert out["status"][4] & L.ISLAND_NONFINITE
    assert np.all(out["status"][[0, 1, 2, 3, 5]] == 0)
    assert np.all(np.isfinite(out["m"][[0, 1, 2, 3, 5]]))


def test_gemm_error_flag_reports_timeout_and_clears(ctx, mid):
    isl = synth.jittered_islands(8, seed=4, mesh_id=mid)
    p = synth.RunParams(dt_ps=0.1, substeps=4, alpha=0.1)
    with ctx.batch(isl, p, precision=L.PREC_BF16X3) as bt:
        L.check(ctx.lib.bpm_debug_set_gemm_error(bt.h, 3))
        bt.advance(2)                           # the GEMMs return at entry
        with pytest.raises(L.BpmError) as e:
            bt.read()
        assert e.value.code == -4 and "gave up" in str(e.value)
        L.check(ctx.lib.bpm_debug_set_gemm_error(bt.h, 0))
        bt.set_state(None, 0.0)
        bt.advance(2)
        out = bt.read()
        assert np.all(out["status"] == 0)


def test_a_real_gemm_wait_runs_out_and_the_batch_recovers(ctx, mid):
    # a wait limit far below one output tile's MMAs: the first tile's accumulator is not full
    # in time, the wait gives up, the kernel lets its copies and MMAs land, frees TMEM and
    # returns; the batch reports BPM_ERR_TIMEOUT, and after the limit is restored and the
    # flag cleared the same run gives the same state as a batch that never timed out
    isl = synth.jittered_islands(300, seed=5, mesh_id=mid)
    p = synth.RunParams(dt_ps=0.1, substeps=4, alpha=0.1, rise_ps=10.0, uniform_T=(0.0, 0.0, -0.6))
    with ctx.batch(isl, p, precision=L.PREC_BF16X3) as bt:
        bt.advance(3)
        clean = bt.read()
    with ctx.batch(isl, p, precision=L.PREC_BF16X3) as bt:
        L.check(ctx.lib.bpm_debug_set_gemm_wait(bt.h, 1000.0))        # 1 us
        bt.advance(3)
        with pytest.raises(L.BpmError) as e:
            bt.read()
        assert e.value.code == L.BPM_ERR_TIMEOUT
        L.check(ctx.lib.bpm_debug_set_gemm_wait(bt.h, 0.0))
        L.check(ctx.lib.bpm_debug_set_gemm_error(bt.h, 0))
        bt.set_state(None, 0.0)
        bt.advance(3)
        out = bt.read()
    assert np.array_equal(out["m"], clean["m"])
    assert np.all(out["status"] == 0)
    with pytest.raises(L.BpmError):
        L.check(ctx.lib.bpm_debug_set_gemm_wait(None, 5.0))


def test_meshes_and_maps_are_released(ctx):
    # a released mesh or map is gone: runs naming it are refused; release is refused while a
    # live batch uses it, and a second release is refused
    mesh, mats = synth.small_island_mesh(), synth.ecc_materials()
    mid = ctx.mesh_upload(mesh, mats)
    hid = ctx.headmap_upload(synth.synthetic_head_map())
    isl = synth.jittered_islands(4, seed=2, mesh_id=mid)
    p = synth.RunParams(dt_ps=0.1, substeps=4, alpha=0.1, use_map=True)
    with ctx.batch(isl, p, precision=L.PREC_BF16X3, map_id=hid) as bt:
        for fn, i in ((ctx.mesh_release, mid), (ctx.headmap_release, hid)):
            with pytest.raises(L.BpmError) as e:
                fn(i)
            assert e.value.code == L.BPM_ERR_STATE
        bt.advance(1)
    ctx.headmap_release(hid)
    with pytest.raises(L.BpmError) as e:
        ctx.run_batch(isl, p, 1, map_id=hid)
    assert e.value.code == L.BPM_ERR_ARG
    ctx.mesh_release(mid)
    with pytest.raises(L.BpmError) as e:
        ctx.run_batch(isl, synth.RunParams(dt_ps=0.1, substeps=4, alpha=0.1), 1)
    assert e.value.code == L.BPM_ERR_ARG
    for fn, i in ((ctx.mesh_release, mid), (ctx.headmap_release, hid)):
        with pytest.raises(L.BpmError) as e:
            fn(i)
        assert e.value.code == L.BPM_ERR_ARG
    # the context still works: a new mesh gets a new id and runs
    mid2 = ctx.mesh_upload(mesh, mats)
    assert mid2 != mid
    out = ctx.run_batch(synth.jittered_islands(2, seed=3, mesh_id=mid2), synth.RunParams(dt_ps=0.1, substeps=4), 1)
    assert np.all(out["status"] == 0)
