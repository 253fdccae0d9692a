"""The integrator step count is computed by the library (bpm_stable_substeps):
for jittered islands on the 209-node, census and design-variant meshes, with
and without the head map, it equals the oracle's count (the same bound, with
lambda_max from eigvalsh in the oracle and power iteration on the GPU), and a
run with substeps = 0 is the run with that count.

Device tensors handed to the library are ordered against torch's current
stream by the binding: an input whose producer is still queued behind a long
kernel, and an output read right after the call, give the host result."""
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


def _meshes():
    v = synth.design_variants()
    # the smallest variant, a 1.5:1 ellipse and a mid-size circle, besides the two workload meshes
    picks = [v[0]] + [x for x in v if x["mesh"].n_nodes <= 2400][1::3]
    return [("209-node", synth.small_island_mesh()), ("census", synth.census_island_mesh())] + \
        [(f"variant {x['mesh'].n_nodes}", x["mesh"]) for x in picks]


def test_library_step_count_equals_the_oracle_count(ctx):
    mats = synth.ecc_materials()
    hm = synth.synthetic_head_map()
    hid = ctx.headmap_upload(hm)
    for name, mesh in _meshes():
        ops = fem.MeshOperators(mesh.xyz_nm, mesh.tets, mesh.tet_region, mats, with_demag=False)
        mid = ctx.mesh_upload(mesh, mats)
        for seed, use_map, alpha, Hext in ((1, True, 0.1, 0.0), (2, False, 0.02, 0.12)):
            isl = synth.jittered_islands(512, seed=seed, mesh_id=mid)
            isl.Hext_T[:, 2] = -Hext
            p = synth.RunParams(dt_ps=0.1, alpha=alpha, use_map=use_map, uniform_T=synth.uniform_field(0.3, 160.0))
            ob = llg.Batch(ops, isl, p, head_map=hm if use_map else None, demag=np.zeros((1, 1)))
            k, bound = ctx.stable_substeps(isl, p, hid)
            print(f"{name}: k {k} (oracle {llg.stable_substeps(ob)}), bound {bound:.6f} T "
                  f"(oracle {llg.field_bound(ob):.6f})")
            assert abs(bound - llg.field_bound(ob)) <= 1e-8 * bound
            assert k == llg.stable_substeps(ob)


def test_zero_substeps_runs_the_stable_count(ctx):
    mesh = synth.small_island_mesh()
    mats = synth.ecc_materials()
    mid = ctx.mesh_upload(mesh, mats)
    hid = ctx.headmap_upload(synth.synthetic_head_map())
    isl = synth.jittered_islands(40, seed=5, mesh_id=mid)
    p = synth.RunParams(dt_ps=0.1, alpha=0.1, rise_ps=10.0, use_map=True, x0_nm=-2.0,
                        uniform_T=synth.uniform_field(0.6, 170.0))
    k = ctx.stable_substeps(isl, p, hid)[0]
    p.substeps = 0
    auto = ctx.run_batch(isl, p, 30, precision=L.PREC_BF16X3, map_id=hid)
    p.substeps = k
    fixed = ctx.run_batch(isl, p, 30, precision=L.PREC_BF16X3, map_id=hid)
    assert np.array_equal(auto["m"], fixed["m"]) and np.array_equal(auto["t_sw"], fixed["t_sw"])
    p.substeps = k + 1                  # a different count moves the state: the comparison has teeth
    other = ctx.run_batch(isl, p, 30, precision=L.PREC_BF16X3, map_id=hid)
    assert not np.array_equal(other["m"], fixed["m"])
    p.substeps = -1
    with pytest.raises(L.BpmError):
        ctx.run_batch(isl, p, 1, precision=L.PREC_BF16X3, map_id=hid)


def test_device_inputs_are_ordered_after_torch_producers(ctx):
    torch = pytest.importorskip("torch")
    sizes = [16, 256, 256, 256, 256, 2]
    sur = ctx.surrogate((16, 256, 4, 2), synth.mlp_init_params(sizes, seed=9))
    try:
        X = (synth.unit_points(4096 * 16, 16, seed=9, stream=0).astype(np.float32) * 2.0 - 1.0)
        R_host = sur.screen(X, 4096, 16)
        P_host = sur.infer(X)
        Xp = torch.from_numpy(X).pin_memory()
        for _ in range(2):
            # the input's producer queued behind tens of milliseconds of work on torch's stream
            big = torch.ones((4096, 4096), device="cuda")
            for _ in range(40):
                big = big @ big * (1.0 / 4096.0)
            Xd = torch.empty_like(Xp, device="cuda")
            Xd.copy_(Xp, non_blocking=True)
            R = sur.screen(Xd, 4096, 16)
            P = sur.infer(Xd)
            assert np.array_equal(R.cpu().numpy(), R_host)
            assert np.array_equal(P.cpu().numpy(), P_host)
            del Xd, R, P, big
    finally:
        sur.destroy()
