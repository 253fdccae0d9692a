"""Argument checks of the Python binding, without a GPU: a device tensor handed to the
library as a raw pointer must be a CUDA tensor on the context's device, of the call's
dtype, contiguous and of the call's extents; host arrays must have the extents the
library will read.  Every refusal happens before any library call."""
import types

import numpy as np
import pytest

from paper_1603_09493_gb300 import api, synth

torch = pytest.importorskip("torch")


class _Dev:
    """Stands in for a CUDA tensor (its attributes only)."""

    def __init__(self, shape, dtype=torch.float32, index=0, contiguous=True):
        self.shape = tuple(shape)
        self.dtype = dtype
        self.device = types.SimpleNamespace(index=index)
        self.is_cuda = True
        self._contiguous = contiguous

    def is_contiguous(self):
        return self._contiguous


def test_device_tensor_accepts_the_stated_form():
    t = _Dev((4, 3, 10))
    assert api.device_tensor(t, 0, "float32", (4, 3, None), "m") is t
    assert api.device_tensor(_Dev((7,), torch.uint8, index=1), 1, "uint8", (7,), "s") is not None


@pytest.mark.parametrize("t, why", [
    (torch.zeros((4, 3, 10)), "CUDA"),                                 # a host tensor
    (np.zeros((4, 3, 10), np.float32), "CUDA"),
    (_Dev((4, 3, 10), index=1), "cuda:1"),                             # another device
    (_Dev((4, 3, 10), torch.float64), "dtype"),
    (_Dev((4, 3, 10), contiguous=False), "contiguous"),
    (_Dev((5, 3, 10)), "shape"),
    (_Dev((4, 10, 3)), "shape"),
    (_Dev((4, 3)), "shape"),
])
def test_device_tensor_refuses_other_forms(t, why):
    with pytest.raises(ValueError, match=why):
        api.device_tensor(t, 0, "float32", (4, 3, None), "m")


class _NoLib:
    def __getattr__(self, name):
        raise AssertionError(f"library called: {name}")


def _batch(B=4, n=10):
    bt = object.__new__(api.Batch)
    bt.ctx = types.SimpleNamespace(device=0)
    bt.lib, bt.h, bt.B, bt.n = _NoLib(), None, B, n
    return bt


def test_batch_state_and_reads_are_checked_before_the_library():
    bt = _batch()
    with pytest.raises(ValueError, match="shape"):
        bt.set_state(np.zeros((3, 3, 10), np.float32))              # fewer islands than the batch
    with pytest.raises(ValueError, match="shape"):
        bt.set_state(np.zeros((4, 10, 3), np.float32))              # node-major, not [B][3][ld]
    with pytest.raises(ValueError, match="dtype"):
        bt.set_state(_Dev((4, 3, 10), torch.float16))
    with pytest.raises(ValueError, match="switched"):
        bt.read_device(None, _Dev((4,), torch.float32), None, None, None)
    with pytest.raises(ValueError, match="mz"):
        bt.read_device(None, None, None, None, _Dev((3,)))
    with pytest.raises(ValueError, match="status"):
        bt.read_device(None, None, None, _Dev((4,), torch.int64), None)


def test_surrogate_inputs_are_checked_before_the_library():
    sur = object.__new__(api.Surrogate)
    sur.ctx = types.SimpleNamespace(device=0, h=None)
    sur.lib, sur.sid, sur.n_in, sur.n_out, sur.P = _NoLib(), 0, 16, 2, 0
    with pytest.raises(ValueError, match="expected"):
        sur.infer(np.zeros((8, 15), np.float32))                     # too few features
    with pytest.raises(ValueError, match="shape"):
        sur.infer(_Dev((8, 15)))
    with pytest.raises(ValueError, match="dtype"):
        sur.screen(_Dev((8, 16), torch.float64), 2, 4)
    with pytest.raises(ValueError, match="rows"):
        sur.screen(np.zeros((8, 16), np.float32), 3, 4)
    with pytest.raises(ValueError, match="Y"):
        sur.grad(np.zeros((8, 16), np.float32), np.zeros((8, 1), np.float32))
    with pytest.raises(ValueError, match="labels"):
        sur.train(np.zeros((8, 16), np.float32), np.zeros((7, 2), np.float32), 1, 4, 1e-3, 0.0)


def test_context_outputs_are_checked_before_the_library():
    ctx = object.__new__(api.Context)
    ctx.lib, ctx.h, ctx.device = _NoLib(), None, 0
    with pytest.raises(ValueError, match="shape"):
        ctx.head_field({}, 8, 8, 4, 1.0, (0.0, 0.0, 0.0), out=_Dev((4, 8, 8)))
    with pytest.raises(ValueError, match="origin"):
        ctx.head_field({}, 8, 8, 4, 1.0, (0.0, 0.0))
    isl = synth.nominal_islands(4)
    with pytest.raises(ValueError, match="m_dev"):
        ctx.llg_advance_noalloc(isl, synth.RunParams(), 1, _Dev((3, 3, 10)))
    with pytest.raises(ValueError, match="mz_dev"):
        ctx.llg_advance_noalloc(isl, synth.RunParams(), 1, _Dev((4, 3, 10)), _Dev((4,), torch.float64))


def test_uploads_are_checked_before_the_library():
    ctx = object.__new__(api.Context)
    ctx.lib, ctx.h, ctx.device = _NoLib(), None, 0
    hm = synth.synthetic_head_map(nx=8, ny=8, nz=4)
    with pytest.raises(ValueError, match="head map"):
        ctx.headmap_upload(synth.HeadMap(B_T=hm.B_T[..., 0], origin_nm=hm.origin_nm, h_nm=hm.h_nm))
    with pytest.raises(ValueError, match="head map"):
        ctx.headmap_upload(synth.HeadMap(B_T=hm.B_T, origin_nm=hm.origin_nm[:2], h_nm=hm.h_nm))
    mesh = synth.small_island_mesh()
    bad = types.SimpleNamespace(xyz_nm=mesh.xyz_nm.T, tets=mesh.tets, tet_region=mesh.tet_region)
    with pytest.raises(ValueError, match="mesh"):
        ctx.mesh_upload(bad, synth.ecc_materials())
    bad = types.SimpleNamespace(xyz_nm=mesh.xyz_nm, tets=mesh.tets, tet_region=mesh.tet_region[:-1])
    with pytest.raises(ValueError, match="mesh"):
        ctx.mesh_upload(bad, synth.ecc_materials())


def test_surrogate_parameter_count_is_checked_before_the_library():
    ctx = types.SimpleNamespace(lib=_NoLib(), h=None, device=0)
    sizes = [16, 64, 64, 2]
    flat = synth.mlp_init_params(sizes, seed=1)
    with pytest.raises(ValueError, match="parameters"):
        api.Surrogate(ctx, (16, 64, 2, 2), flat[:-1])
    with pytest.raises(AssertionError, match="library called"):      # the right count reaches it
        api.Surrogate(ctx, (16, 64, 2, 2), flat)


def test_band_start_is_checked_before_the_band_runs():
    calls = []

    class _InfoLib(_NoLib):
        def bpm_mesh_info_get(self, h, mid, info):
            calls.append("info")
            info._obj.n_nodes = 10
            return 0

    ctx = object.__new__(api.Context)
    ctx.lib, ctx.h, ctx.device = _InfoLib(), None, 0
    isl = synth.nominal_islands(2)
    with pytest.raises(ValueError, match="m_init"):
        ctx.neb(isl, 5, 10, 0.1, 1.0, m_init=np.zeros((2, 5, 10, 3), np.float32))
    assert calls == ["info"]
