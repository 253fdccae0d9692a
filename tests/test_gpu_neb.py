"""The GPU nudged elastic band (bpm_neb_run) against the FP64 oracle band
(Sec. II.C, adjacent-track barrier, Eq. 3).

Same band, same initial images, same step, spring and climbing schedule on
both sides: the update is a contraction, so FP32 kernels and the BF16-split
demag product stay close to the FP64 iterates.  Bars (about ten times the
measured gaps of 4e-7 / 1e-6 / 6e-7): energies of the final band within 1e-5 of
the energy scale, barriers within 1e-5 relative, images within 1e-5.  A homogeneous island small
against the exchange length reaches its coherent-rotation barrier E(x) - E(z),
computed by the oracle's energy of two uniform states."""
import os

import numpy as np
import pytest

from oracle import fem, llg, neb
from paper_1603_09493_gb300 import _lib as L
from paper_1603_09493_gb300 import adjacent, api, synth

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
    return mesh, mats, ops, ctx.mesh_upload(mesh, mats)


@pytest.mark.parametrize("prec", [L.PREC_FP32, L.PREC_BF16X3])
def test_band_matches_oracle_in_fringing_field(ctx, small, prec):
    mesh, mats, ops, mid = small
    hm = synth.synthetic_head_map()
    hid = ctx.headmap_upload(hm)
    isl = synth.jittered_islands(2, seed=81, mesh_id=mid)
    isl.pos_nm[:, 1] += 12.7                       # the adjacent track
    p = synth.RunParams(dt_ps=0.1, rise_ps=0.0, v_m_per_s=0.0, x0_nm=2.0, use_map=True)
    P, iters, spring, climb = 7, 300, 1.0, 100
    step = 0.4 / (float(ops.Ms.max()) * 1e-6 * float(np.max(isl.Ms_scale)) *
                  llg.field_bound(llg.Batch(ops, isl, p, head_map=hm)))
    band = np.repeat(neb.great_circle_path(ops.n, P)[None], 2, axis=0)
    ref = neb.island_band(ops, isl, p, hm, band, iters, step, spring, climb)
    got = ctx.neb(isl, P, iters, step, spring, climb, precision=prec, map_id=hid, head_x_nm=p.x0_nm,
                  uniform_T=p.uniform_T, want_path=True)
    assert got["iters"] == iters
    scale = np.abs(ref["E"]).max()
    e_err = np.abs(got["E"] - ref["E"]).max() / scale
    b_err = np.abs(got["E_B"] - ref["E_B"]).max() / np.abs(ref["E_B"]).max()
    m_err = np.abs(got["m"].transpose(0, 1, 3, 2) - ref["m"]).max()
    print(f"prec {prec}: E_B {got['E_B'] / (neb.KB * 300)} kT (oracle {ref['E_B'] / (neb.KB * 300)}), "
          f"|dE|/scale {e_err:.1e}, |dE_B|/E_B {b_err:.1e}, |dm| {m_err:.1e}")
    assert e_err <= 1e-5
    assert b_err <= 1e-5
    assert m_err <= 1e-5
    assert np.allclose(np.linalg.norm(got["m"], axis=2), 1.0, atol=1e-5)


def _homogeneous(ctx):
    mesh = synth.layered_island_mesh(5.0, 4.0, 1.0, rings=2, hard_slabs=4, soft_slabs=1, seed=0)
    mats = synth.ecc_materials(Ms_soft=0.8e6, Ku_soft=0.9e6, interlayer_scale=1.0)
    ops = fem.MeshOperators(mesh.xyz_nm, mesh.tets, mesh.tet_region, mats)
    mid = ctx.mesh_upload(mesh, mats)
    isl = synth.Islands(np.full(1, mid, np.int32), np.ones(1, np.float32), np.ones(1, np.float32),
                        np.array([[0.0, 0.0, 1.0]], np.float32), np.zeros((1, 2), np.float32),
                        np.zeros((1, 3), np.float32))
    return ops, isl


def test_homogeneous_island_reaches_coherent_barrier(ctx):
    ops, isl = _homogeneous(ctx)
    mask = llg.T_EXCHANGE | llg.T_ANISOTROPY | llg.T_DEMAG
    p = synth.RunParams(dt_ps=0.1, rise_ps=0.0, term_mask=mask)
    b = llg.Batch(ops, isl, p)
    mx = np.zeros((1, ops.n, 3)); mx[..., 0] = 1.0
    mz = np.zeros((1, ops.n, 3)); mz[..., 2] = 1.0
    coherent = b.energy(mx, 0.0)[0] - b.energy(mz, 0.0)[0]
    step = 0.4 / (0.8 * llg.field_bound(b))
    got = adjacent.barriers(ctx, isl, p, n_images=9, max_iters=1500, climb_after=300, spring=1.0, step=step,
                            precision=L.PREC_BF16X3)
    eb = got["E_B"][0]
    print(f"GPU E_B {got['E_B_kT'][0]:.3f} kT, coherent {coherent / (neb.KB * 300):.3f} kT, "
          f"max force {got['max_force']:.1e}")
    assert 0.85 * coherent <= eb <= coherent * (1 + 1e-3)
    # Eq. (3) on the computed barrier
    assert got["ber_adj"][0] == pytest.approx(130.0 * np.exp(-got["E_B_kT"][0]), rel=1e-12)


def test_force_tolerance_stops_early(ctx):
    ops, isl = _homogeneous(ctx)
    p = synth.RunParams(dt_ps=0.1, rise_ps=0.0, term_mask=L.TERM_EXCHANGE | L.TERM_ANISOTROPY | L.TERM_DEMAG)
    step = 0.4 / (0.8 * llg.field_bound(llg.Batch(ops, isl, p)))
    out = ctx.neb(isl, 9, 5000, step, 1.0, 300, term_mask=p.term_mask, force_tol=1e-3, check_every=25)
    assert out["iters"] < 5000 and out["iters"] % 25 == 0
    assert out["max_force"] < 1e-3


def test_band_arguments_are_checked(ctx, small):
    mesh, mats, ops, mid = small
    ops2, isl2 = _homogeneous(ctx)
    isl = synth.jittered_islands(1, seed=1, mesh_id=mid)
    with pytest.raises(RuntimeError):
        ctx.neb(isl, 2, 10, 1e-3, 1.0)                      # fewer than three images
    with pytest.raises(RuntimeError):
        ctx.neb(isl, 5, 10, 0.0, 1.0)                       # no step
    with pytest.raises(RuntimeError):
        ctx.neb(synth.Islands.concat([isl, isl2]), 5, 10, 1e-3, 1.0)   # two meshes
