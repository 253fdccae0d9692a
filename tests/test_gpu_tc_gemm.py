"""The tcgen05 demag GEMM against the CUDA-core evaluation of the same BF16
split products and against FP32, through the demag term of bpm_batch_field.

Same products, different summation: the tensor core adds each MMA's products
into the FP32 accumulator with its own alignment and rounding, not as a chain
of IEEE FMAs.  Bound: one relative rounding of 2^-23 of the accumulator per MMA
issue, (3 K / 16) * 2^-23 of the field scale (2.1e-5 at K = 960, 1.1e-4 at
K = 4736; measured 3.2e-6 and 1.6e-5).  Against FP32 the split operands add
~2^-17 relative each.  One BF16 product: ~2^-9 per operand (measured ~3e-3,
bound 2e-2)."""
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


def _state(xyz, B, seed):
    rng = np.random.default_rng(seed)
    m = rng.standard_normal((B, 3, xyz.shape[0])) * 0.3
    m[:, 2, :] += 1.0
    return (m / np.linalg.norm(m, axis=1, keepdims=True)).astype(np.float32)


def _demag(ctx, isl, p, prec, m, tile_n=None, raster=L.RASTER_AUTO, k_block=64, pair=0):
    with ctx.batch(isl, p, precision=prec) as bt:
        if tile_n is not None:
            bt.set_tuning(tile_n, 256, raster, gemm_k_block=k_block, gemm_pair=pair)
        bt.set_state(m, 0.0)
        return bt.field(0.0, L.TERM_DEMAG)


@pytest.mark.parametrize("tile_n", [256, 128])
@pytest.mark.parametrize("case", ["ragged_small", "census"])
def test_tc_gemm_matches_split_reference_and_fp32(ctx, case, tile_n):
    if case == "ragged_small":
        mesh = synth.layered_island_mesh(8.0, 7.0, 3.0, rings=2, hard_slabs=10, soft_slabs=5, seed=4)
        B = 200                           # two 128-row tiles, second one partly padding
    else:
        mesh = synth.census_island_mesh()
        B = 4096
    mid = ctx.mesh_upload(mesh, synth.ecc_materials())
    info = ctx.mesh_info(mid)
    if case == "ragged_small":
        assert info["k_pad"] % 256 != 0 and info["k_pad"] >= 3 * info["n_pad"]
    isl = synth.jittered_islands(B, seed=3, mesh_id=mid)
    p = synth.RunParams(dt_ps=0.1, substeps=1, term_mask=L.TERM_DEMAG)
    m = _state(mesh.xyz_nm, B, 5)
    f32 = _demag(ctx, isl, p, L.PREC_FP32, m)
    ref = _demag(ctx, isl, p, L.PREC_BF16X3_REF, m)
    tc3 = _demag(ctx, isl, p, L.PREC_BF16X3, m, tile_n)
    tc1 = _demag(ctx, isl, p, L.PREC_BF16, m, tile_n)
    assert np.array_equal(_demag(ctx, isl, p, L.PREC_BF16X3, m, tile_n, k_block=32), tc3)
    assert np.array_equal(_demag(ctx, isl, p, L.PREC_BF16, m, tile_n, k_block=32), tc1)
    scale = np.abs(f32).max()
    K = info["k_pad"]
    acc_bound = (3 * K / 16) * 2.0 ** -23
    e_ref = np.abs(tc3 - ref).max() / scale
    e_f32 = np.abs(tc3 - f32).max() / scale
    e_1 = np.abs(tc1 - f32).max() / scale
    print(f"{case} TN={tile_n}: |tc3-ref| {e_ref:.2e}  |tc3-f32| {e_f32:.2e}  |tc1-f32| {e_1:.2e}  scale {scale:.3f} T")
    assert np.all(np.isfinite(tc3)) and np.all(np.isfinite(tc1))
    assert e_ref <= acc_bound
    assert e_f32 <= acc_bound + 4 * 2.0 ** -17
    assert e_1 <= 2e-2


def test_grouped_gemm_over_mesh_groups(ctx):
    # one persistent launch covers the tiles of three mesh groups of different
    # K (and a group smaller than one 128-row tile); every group must meet the
    # single-group bound against its own FP32 product
    meshes = [synth.small_island_mesh(seed=0),
              synth.layered_island_mesh(8.0, 7.0, 3.0, rings=2, hard_slabs=10, soft_slabs=5, seed=4),
              synth.layered_island_mesh(9.0, 7.0, 3.0, rings=2, hard_slabs=8, soft_slabs=3, aspect=1.5, seed=6)]
    mids = [ctx.mesh_upload(msh, synth.ecc_materials()) for msh in meshes]
    sizes = [300, 40, 170]
    isl = synth.Islands.concat([synth.jittered_islands(b, seed=9 + k, mesh_id=mids[k])
                                for k, b in enumerate(sizes)])
    p = synth.RunParams(dt_ps=0.1, substeps=1, term_mask=L.TERM_DEMAG)
    nmax = max(msh.n_nodes for msh in meshes)
    rng = np.random.default_rng(7)
    m = rng.standard_normal((len(isl), 3, nmax)) * 0.3
    m[:, 2, :] += 1.0
    m = (m / np.linalg.norm(m, axis=1, keepdims=True)).astype(np.float32)
    for k, msh in enumerate(meshes):          # nodes past a mesh's own count are not read
        rows = np.where(isl.mesh_id == mids[k])[0]
        m[np.ix_(rows, [0, 1, 2], np.arange(msh.n_nodes, nmax))] = 0.0
    f32 = _demag(ctx, isl, p, L.PREC_FP32, m)
    for tile_n in (256, 128):
        tc3 = _demag(ctx, isl, p, L.PREC_BF16X3, m, tile_n)
        assert np.all(np.isfinite(tc3))
        # the tile order changes which CTA computes a tile, and the stage depth how the
        # k16 MMAs are grouped into pipeline stages, never the summation
        for raster in (L.RASTER_M, L.RASTER_N):
            assert np.array_equal(_demag(ctx, isl, p, L.PREC_BF16X3, m, tile_n, raster), tc3)
        assert np.array_equal(_demag(ctx, isl, p, L.PREC_BF16X3, m, tile_n, L.RASTER_AUTO, 32), tc3)
        for k, msh in enumerate(meshes):
            rows = np.where(isl.mesh_id == mids[k])[0]
            n = msh.n_nodes
            K = ctx.mesh_info(mids[k])["k_pad"]
            scale = np.abs(f32[rows][:, :, :n]).max()
            err = np.abs(tc3[rows][:, :, :n] - f32[rows][:, :, :n]).max() / scale
            print(f"group {k} (B={sizes[k]}, K={K}) TN={tile_n}: |tc3-f32| {err:.2e}")
            assert err <= (3 * K / 16) * 2.0 ** -23 + 4 * 2.0 ** -17


@pytest.mark.parametrize("case", ["one_pair_tile", "odd_half_past_the_rows", "census"])
def test_pair_gemm_matches_one_sm_gemm(ctx, case):
    # 256 x 256 tiles on CTA pairs (cta_group::2): the same split products and K order as the
    # one-SM kernel, so the same bound against the CUDA-core reference; rows past the batch
    # (the odd CTA's half of the last tile when the rows end on a 128 boundary) are zero
    # operands and are not stored
    if case == "census":
        mesh, B = synth.census_island_mesh(), 4096
    else:
        mesh = synth.layered_island_mesh(8.0, 7.0, 3.0, rings=2, hard_slabs=10, soft_slabs=5, seed=4)
        B = 200 if case == "one_pair_tile" else 300        # 256 rows: one pair tile; 384: 1.5
    mid = ctx.mesh_upload(mesh, synth.ecc_materials())
    K = ctx.mesh_info(mid)["k_pad"]
    isl = synth.jittered_islands(B, seed=3, mesh_id=mid)
    p = synth.RunParams(dt_ps=0.1, substeps=1, term_mask=L.TERM_DEMAG)
    m = _state(mesh.xyz_nm, B, 5)
    ref = _demag(ctx, isl, p, L.PREC_BF16X3_REF, m)
    one = _demag(ctx, isl, p, L.PREC_BF16X3, m, 256)
    scale = np.abs(ref).max()
    bound = (3 * K / 16) * 2.0 ** -23
    for k_block in (32, 64):
        for raster in (L.RASTER_AUTO, L.RASTER_M):
            two = _demag(ctx, isl, p, L.PREC_BF16X3, m, 256, raster, k_block, pair=1)
            e_ref = np.abs(two - ref).max() / scale
            print(f"{case} (B={B}, K={K}) pair kb={k_block} raster={raster}: |pair-ref| {e_ref:.2e}, "
                  f"bitwise equal to one SM: {np.array_equal(two, one)}")
            assert np.all(np.isfinite(two)) and e_ref <= bound
            assert np.abs(two - one).max() / scale <= bound
    one1 = _demag(ctx, isl, p, L.PREC_BF16, m, 256)
    two1 = _demag(ctx, isl, p, L.PREC_BF16, m, 256, L.RASTER_AUTO, 32, pair=1)
    assert np.abs(two1 - one1).max() / scale <= bound


def test_pair_gemm_over_mesh_groups_and_in_a_run(ctx):
    meshes = [synth.small_island_mesh(seed=0),
              synth.layered_island_mesh(8.0, 7.0, 3.0, rings=2, hard_slabs=10, soft_slabs=5, seed=4),
              synth.layered_island_mesh(9.0, 7.0, 3.0, rings=2, hard_slabs=8, soft_slabs=3, aspect=1.5, seed=6)]
    mids = [ctx.mesh_upload(msh, synth.ecc_materials()) for msh in meshes]
    sizes = [300, 40, 170]
    isl = synth.Islands.concat([synth.jittered_islands(b, seed=9 + k, mesh_id=mids[k])
                                for k, b in enumerate(sizes)])
    p = synth.RunParams(dt_ps=0.1, substeps=1, term_mask=L.TERM_DEMAG)
    nmax = max(msh.n_nodes for msh in meshes)
    rng = np.random.default_rng(7)
    m = rng.standard_normal((len(isl), 3, nmax)) * 0.3
    m[:, 2, :] += 1.0
    m = (m / np.linalg.norm(m, axis=1, keepdims=True)).astype(np.float32)
    for k, msh in enumerate(meshes):
        rows = np.where(isl.mesh_id == mids[k])[0]
        m[np.ix_(rows, [0, 1, 2], np.arange(msh.n_nodes, nmax))] = 0.0
    ref = _demag(ctx, isl, p, L.PREC_BF16X3_REF, m)
    two = _demag(ctx, isl, p, L.PREC_BF16X3, m, 256, L.RASTER_AUTO, 32, pair=1)
    for k, msh in enumerate(meshes):
        rows = np.where(isl.mesh_id == mids[k])[0]
        n = msh.n_nodes
        K = ctx.mesh_info(mids[k])["k_pad"]
        scale = np.abs(ref[rows][:, :, :n]).max()
        assert np.abs(two[rows][:, :, :n] - ref[rows][:, :, :n]).max() / scale <= (3 * K / 16) * 2.0 ** -23
    # a whole run on the pair kernel: the trajectory of the one-SM kernel within the bound's drift
    hm = synth.synthetic_head_map()
    hid = ctx.headmap_upload(hm)
    q = synth.RunParams(dt_ps=0.1, alpha=0.1, rise_ps=10.0, use_map=True, x0_nm=-2.0, substeps=0,
                        uniform_T=synth.uniform_field(0.6, 170.0))
    outs = []
    for pair in (0, 1):
        with ctx.batch(isl, q, precision=L.PREC_BF16X3, map_id=hid) as bt:
            bt.set_tuning(256, 256, L.RASTER_AUTO, 2, 32, gemm_pair=pair)
            bt.advance(50)
            outs.append(bt.read())
    assert np.all(outs[1]["status"] == 0)
    print("pair vs one-SM run, 5 ps: max |dm|", float(np.abs(outs[1]["m"] - outs[0]["m"]).max()))
    assert np.abs(outs[1]["m"] - outs[0]["m"]).max() <= 1e-4
