"""Critical-field search and BER (Sec. II.C, Eqs. 1-2) on the GPU path against
the same search with the FP64 oracle LLG: both take every decision from
switching outcomes, so the critical fields must coincide (up to one
finest-grid step sigma/8 if a borderline outcome differs)."""
import math
import os

import numpy as np
import pytest

from oracle import ber as oracle_ber
from oracle import fem, hcrit as ohcrit, llg
from paper_1603_09493_gb300 import _lib as L
from paper_1603_09493_gb300 import api, hcrit, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("role, drive_T", [("targ", 0.85), ("prev", 0.65)])
def test_critical_field_search_matches_oracle(role, drive_T):
    if not os.path.exists(L.LIB_PATH):
        from paper_1603_09493_gb300 import build
        build.build()
    mesh = synth.small_island_mesh()
    mats = synth.ecc_materials()
    ops = fem.MeshOperators(mesh.xyz_nm, mesh.tets, mesh.tet_region, mats)
    with api.Context(0) as ctx:
        mid = ctx.mesh_upload(mesh, mats)
        isl = synth.jittered_islands(2, seed=81, mesh_id=mid)
        isl.Ku_scale[:] = [0.95, 1.05]
        # the uniform ramped field stands in for the head field under the pole
        p = synth.RunParams(dt_ps=0.1, t_end_ps=80.0, alpha=0.1, rise_ps=20.0, use_map=False,
                            uniform_T=synth.uniform_field(drive_T, 160.0))
        p.substeps = llg.stable_substeps(llg.Batch(ops, isl, p))
        direction = np.tile(np.array(p.uniform_T) / np.linalg.norm(p.uniform_T), (2, 1))
        Js = 4e-7 * math.pi * 0.8e6
        sigma = np.array([hcrit.sfd_sigma_T(0.9e6 * float(k), Js) for k in isl.Ku_scale], np.float64)
        assert abs(oracle_ber.sfd_sigma_T(0.9e6, Js) - hcrit.sfd_sigma_T(0.9e6, Js)) < 1e-15
        res = hcrit.critical_field_search(hcrit.gpu_flag_runner(ctx, p, p.n_intervals), isl, direction, sigma, role)
        h_ref, ber_ref, ab_ref = ohcrit.search(ops, isl, p, direction, sigma, role)
    print(role, "gpu", res.h_crit_T / sigma, res.ber, "oracle", h_ref / sigma, ber_ref, "runs", res.n_runs)
    assert np.array_equal(res.aborted, ab_ref)
    assert np.all(np.abs(res.h_crit_T - h_ref) <= sigma / 8 + 1e-12)
    assert np.all(res.h_crit_T <= 4 * sigma + 1e-12) and np.any(res.h_crit_T < 4 * sigma)
    for h, b, s in zip(res.h_crit_T, res.ber, sigma):
        assert abs(b - oracle_ber.ber_from_hcrit(h, s)) <= 1e-15
