"""The plain FP64 form (bpm_run_plain_f64: one island per launch, every step in
FP64) against the FP64 oracle.

Both sides evaluate the same readings in FP64; they differ only in the demag
matrix (the GPU's batched-CG assembly agrees with the oracle's dense LU to
about 1e-12 of max|N|, at most 1e-9 by the assembly test), the exchange
summation (difference form against the dense product) and the order of the
volume-weighted sums.  A field difference dB moves m by about gamma dB t; while
an island reverses, its state passes near the unstable equilibrium, where such
differences grow about as exp(gamma B_K t) (B_K ~ 2 T: e-folding in ~3 ps).
Without a reversal the states agree to rounding (1e-14 over 1 ps on the census
mesh); through one (the 20 ps run) to 1e-6, three orders below the
mixed-precision bar, while a dropped or mis-signed term moves m by more than
1e-2.  The switch flags and crossing times must agree to 1e-6 ps."""
import math
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


@pytest.fixture(scope="module")
def small(ctx):
    mesh = synth.small_island_mesh()
    mats = synth.ecc_materials()
    ops = fem.MeshOperators(mesh.xyz_nm, mesh.tets, mesh.tet_region, mats)
    return ops, ctx.mesh_upload(mesh, mats, keep_f64=True)


def test_plain_fp64_trajectory_matches_oracle(ctx, small):
    ops, mid = small
    hm = synth.synthetic_head_map()
    hid = ctx.headmap_upload(hm)
    isl = synth.jittered_islands(6, seed=61, mesh_id=mid)
    isl.Hext_T[:] = np.array([0.02, -0.01, 0.03], np.float32)
    p = synth.RunParams(dt_ps=0.1, t_end_ps=20.0, alpha=0.1, rise_ps=10.0, use_map=True, x0_nm=0.0,
                        uniform_T=synth.uniform_field(0.6, 170.0))
    p.substeps = ctx.stable_substeps(isl, p, hid)[0]
    got = ctx.run_plain_f64(isl, p, p.n_intervals, map_id=hid)
    ref = llg.Batch(ops, isl, p, head_map=hm).run()
    err = float(np.abs(got["m"].transpose(0, 2, 1) - ref["m"]).max())
    mz_err = float(np.abs(got["m"][:, 2, :] @ (ops.V / ops.V.sum()) - ref["mz"]).max())
    print(f"FP64 plain vs oracle over 20 ps: max |dm| {err:.2e}, <m_z> {mz_err:.2e}")
    assert err <= 1e-6 and mz_err <= 1e-6
    assert got["device_ms"] > 0 and np.all(got["status"] == 0)
    # the state moved well away from the start
    assert float(np.abs(got["m"][:, 2, :] - 1.0).max()) > 0.05


def test_plain_fp64_switching_matches_oracle(ctx, small):
    ops, mid = small
    B = 16
    isl = synth.jittered_islands(B, seed=41, mesh_id=mid)
    Bmag = 0.81
    isl.Hext_T[:] = np.array([math.sin(math.radians(170)) * Bmag, 0.0, math.cos(math.radians(170)) * Bmag],
                             np.float32)
    p = synth.RunParams(dt_ps=0.1, t_end_ps=200.0, alpha=0.1, rise_ps=0.0, use_map=False)
    ob = llg.Batch(ops, isl, p)
    p.substeps = llg.stable_substeps(ob)
    ref = ob.run()
    got = ctx.run_plain_f64(isl, p, p.n_intervals)
    assert 0 < ref["switched"].sum() < B                     # a mix of outcomes
    assert np.array_equal(got["switched"], ref["switched"])
    sw = ref["t_sw"] > 0
    assert np.array_equal(got["t_sw"] > 0, sw)
    print("max |dt_sw| (ps):", np.abs(got["t_sw"][sw] - ref["t_sw"][sw]).max())
    assert np.abs(got["t_sw"][sw] - ref["t_sw"][sw]).max() <= 1e-6


def test_plain_fp64_census_mesh_matches_oracle(ctx):
    mesh = synth.census_island_mesh()
    mats = synth.ecc_materials()
    ops = fem.MeshOperators(mesh.xyz_nm, mesh.tets, mesh.tet_region, mats)
    mid = ctx.mesh_upload(mesh, mats, keep_f64=True)
    hm = synth.synthetic_head_map()
    hid = ctx.headmap_upload(hm)
    isl = synth.jittered_islands(4096, seed=1, mesh_id=mid)
    p = synth.RunParams(dt_ps=0.1, t_end_ps=1.0, alpha=0.1, rise_ps=100.0, use_map=True, x0_nm=-2.0)
    p.substeps = ctx.stable_substeps(isl, p, hid)[0]            # the census workload's count
    pick = isl.subset(np.array([7, 3000]))
    got = ctx.run_plain_f64(pick, p, p.n_intervals, map_id=hid)
    ref = llg.Batch(ops, pick, p, head_map=hm).run()
    err = float(np.abs(got["m"].transpose(0, 2, 1) - ref["m"]).max())
    print(f"census mesh, FP64 plain vs oracle over 1 ps: max |dm| {err:.2e}")
    assert err <= 1e-10


def test_plain_fp64_needs_the_fp64_operator(ctx):
    mesh = synth.small_island_mesh()
    mid = ctx.mesh_upload(mesh, synth.ecc_materials())          # FP64 matrix not kept
    isl = synth.jittered_islands(2, seed=3, mesh_id=mid)
    p = synth.RunParams(dt_ps=0.1, substeps=4, alpha=0.1)
    with pytest.raises(L.BpmError) as ei:
        ctx.run_plain_f64(isl, p, 1)
    assert ei.value.code == L.BPM_ERR_STATE
