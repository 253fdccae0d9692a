"""Uneven batches: islands of several mesh variants in one batch.

Each island's result must equal the FP64 oracle run of its own mesh (same
bar as the single-mesh parity, max |dm| <= 1e-3), and must be identical to
the result of a single-mesh batch of the same islands (the grouping changes
which rows of which GEMM an island occupies, never its arithmetic)."""
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


def test_mixed_mesh_batch_matches_oracle_and_single_mesh_batches(ctx):
    meshes = [synth.small_island_mesh(seed=0),
              synth.layered_island_mesh(7.0, 6.0, 4.0, rings=2, hard_slabs=9, soft_slabs=6, seed=5),
              synth.layered_island_mesh(9.0, 7.0, 3.0, rings=2, hard_slabs=8, soft_slabs=3, aspect=1.5, seed=6)]
    mats = synth.ecc_materials()
    mids = [ctx.mesh_upload(m, mats) for m in meshes]
    hm = synth.synthetic_head_map()
    hid = ctx.headmap_upload(hm)
    per = 20
    parts = [synth.jittered_islands(per, seed=50 + k, mesh_id=mids[k]) for k in range(3)]
    # interleave the variants: island b belongs to mesh b % 3
    order = np.argsort(np.tile(np.arange(per), 3) * 3 + np.repeat(np.arange(3), per), kind="stable")
    isl = synth.Islands.concat(parts).subset(order)
    p = synth.RunParams(dt_ps=0.1, t_end_ps=30.0, alpha=0.1, rise_ps=20.0, use_map=True, x0_nm=-3.0,
                        uniform_T=synth.uniform_field(0.5, 165.0))
    ks = []
    ops = []
    for k, m in enumerate(meshes):
        o = fem.MeshOperators(m.xyz_nm, m.tets, m.tet_region, mats)
        ops.append(o)
        ks.append(llg.stable_substeps(llg.Batch(o, parts[k], p, head_map=hm)))
    p.substeps = max(ks)
    out = ctx.run_batch(isl, p, p.n_intervals, precision=L.PREC_BF16X3, map_id=hid)
    assert np.all(out["status"] == 0)
    for k in range(3):
        rows = np.where(isl.mesh_id == mids[k])[0]
        n = meshes[k].n_nodes
        ref = llg.Batch(ops[k], isl.subset(rows), p, head_map=hm).run()
        got = out["m"][rows][:, :, :n].transpose(0, 2, 1)
        err = float(np.abs(got - ref["m"]).max())
        print(f"mesh {k} (n={n}): max |dm| = {err:.2e}")
        assert err <= 1e-3
        assert np.all(out["m"][rows][:, :, n:] == 0)
        single = ctx.run_batch(isl.subset(rows), p, p.n_intervals, precision=L.PREC_BF16X3, map_id=hid)
        assert np.array_equal(single["m"][:, :, :n], out["m"][rows][:, :, :n])
        assert np.array_equal(single["t_sw"], out["t_sw"][rows])


def test_design_variants_assemble_and_step(ctx):
    # the 16 variants of the uneven workload (518..3906 nodes) in one batch with
    # adjacent-track islands; a few intervals, every island finite and unit-norm
    variants = synth.design_variants()
    mats = synth.ecc_materials()
    mids = [ctx.mesh_upload(v["mesh"], mats) for v in variants]
    for mid, v in zip(mids, variants):
        info = ctx.mesh_info(mid)
        assert info["cg_residual_neumann"] < 1e-12 and info["cg_residual_dirichlet"] < 1e-12
        assert abs(info["volume_nm3"] - synth.polygon_area_nm2(v["mesh"]) * v["mesh"].height_nm) < 1e-9 * info[
            "volume_nm3"]
    hid = ctx.headmap_upload(synth.synthetic_head_map())
    isl, role = synth.uneven_batch(variants, mids, realisations=16, seed=2, layout="staggered")
    p = synth.RunParams(dt_ps=0.1, alpha=0.1, rise_ps=100.0, use_map=True)
    p.substeps = 0                      # the library takes its stable step count
    out = ctx.run_batch(isl, p, 3, precision=L.PREC_BF16X3, map_id=hid)
    assert np.all(out["status"] == 0)
    for mid, v in zip(mids, variants):
        rows = np.where(isl.mesh_id == mid)[0]
        n = v["mesh"].n_nodes
        nrm = np.linalg.norm(out["m"][rows][:, :, :n], axis=1)
        assert np.abs(nrm - 1.0).max() < 1e-5
