"""The allocation-free advance against the ordinary batch advance.

bpm_llg_advance_noalloc serves callers that cannot allocate device memory
when they step islands (a host application whose pool allocator owns the
device memory, or a loop that must not stall on cudaMalloc/cudaFree); its
scratch lives in a fixed device array inside the library.  It runs the
kernels of a BPM_PREC_FP32 batch on the same arithmetic, so each call's
final state must equal, bit for bit, that of a batch started from the same
state at the same time; the volume-averaged m_z is summed in a CTA-size
dependent order and agrees to 1e-6.  Two calls run in a row, so that the
second one runs on an array that still holds the first call's contents.
This file is collected last on purpose."""
import os

import numpy as np
import pytest

from paper_1603_09493_gb300 import _lib as L
from paper_1603_09493_gb300 import api, synth

pytestmark = pytest.mark.gpu


def test_noalloc_matches_batch_advance_on_two_calls():
    torch = pytest.importorskip("torch")
    if not os.path.exists(L.LIB_PATH):
        from paper_1603_09493_gb300 import build
        build.build()
    stream = torch.cuda.Stream()
    with api.Context(0, stream=stream) as ctx:
        mesh = synth.small_island_mesh()
        mats = synth.ecc_materials()
        mid = ctx.mesh_upload(mesh, mats)
        hm = synth.synthetic_head_map()
        hid = ctx.headmap_upload(hm)
        B = 24
        isl = synth.jittered_islands(B, seed=7, mesh_id=mid)
        isl.pos_nm[:, 0] += 8.0
        p = synth.RunParams(dt_ps=0.1, alpha=0.1, rise_ps=20.0, use_map=True, x0_nm=-2.0,
                            uniform_T=synth.uniform_field(0.6, 170.0))
        p.substeps = ctx.stable_substeps(isl, p, hid)[0]
        n = mesh.n_nodes
        steps = 60
        m_dev = torch.zeros((B, 3, n), dtype=torch.float32, device="cuda")
        m_dev[:, 2, :] = 1.0
        mz_dev = torch.zeros(B, dtype=torch.float32, device="cuda")
        for call in range(2):
            q = synth.RunParams(**{**p.__dict__})
            q.t0_ps = call * steps * p.dt_ps
            m_start = m_dev.cpu().numpy()
            ctx.llg_advance_noalloc(isl, q, steps, m_dev, mz_dev, map_id=hid)
            got, mz = m_dev.cpu().numpy(), mz_dev.cpu().numpy()
            with ctx.batch(isl, q, precision=L.PREC_FP32, map_id=hid) as bt:
                bt.set_state(m_start, q.t0_ps)
                bt.advance(steps)
                ref = bt.read()
            assert np.array_equal(got, ref["m"]), (call, float(np.abs(got - ref["m"]).max()))
            assert np.abs(mz - ref["mz"]).max() <= 1e-6
            # the state moved (the comparison is not between two copies of the start state)
            assert float(np.abs(got - m_start).max()) > 1e-3
        # a request larger than the fixed array is refused with a clear error
        big = synth.jittered_islands(4096, seed=1, mesh_id=mid)
        m_big = torch.zeros((4096, 3, n), dtype=torch.float32, device="cuda")
        with pytest.raises(L.BpmError) as ei:
            ctx.llg_advance_noalloc(big, p, 1, m_big, None, map_id=hid)
        assert "maximum" in str(ei.value)
