"""What the trained surrogate gains over LLG alone.

The batched LLG solver labels 4096 random designs (switched by 100 ps;
switched by 40 ps), the surrogate trains on those outcomes on the GPU, and on
2048 fresh candidates it screens: its top-256 picks are verified against fresh
LLG solves.  Gain: the hit rate of the screened picks against the base rate
of the candidate pool, at the cost of one inference batch instead of 2048 LLG
solves.  Screening error bound: accuracy >= 0.9 and AUC >= 0.95 against the
fresh LLG outcomes."""
import os

import numpy as np
import pytest

from paper_1603_09493_gb300 import _lib as L
from paper_1603_09493_gb300 import api, synth

pytestmark = pytest.mark.gpu


def auc(score, label):
    order = np.argsort(score)
    ranks = np.empty(len(score))
    ranks[order] = np.arange(1, len(score) + 1)
    pos = label > 0.5
    n1, n0 = pos.sum(), (~pos).sum()
    return (ranks[pos].sum() - n1 * (n1 + 1) / 2) / (n1 * n0)


def test_surrogate_screening_gain():
    if not os.path.exists(L.LIB_PATH):
        from paper_1603_09493_gb300 import build
        build.build()
    with api.Context(0) as ctx:
        mesh = synth.small_island_mesh()
        mid = ctx.mesh_upload(mesh, synth.ecc_materials())
        p = synth.RunParams(dt_ps=0.1, t_end_ps=100.0, alpha=0.1, rise_ps=0.0, use_map=False)

        def label(isl):
            p.substeps = ctx.stable_substeps(isl, p)[0]
            out = ctx.run_batch(isl, p, p.n_intervals, precision=L.PREC_BF16X3)
            assert np.all(out["status"] == 0)
            return np.stack([out["switched"], (out["t_sw"] > 0) & (out["t_sw"] <= 40.0)], 1).astype(np.float32)

        isl_tr, X_tr = synth.screening_designs(4096, seed=3, mesh_id=mid)
        Y_tr = label(isl_tr)
        base = Y_tr[:, 0].mean()
        assert 0.2 < base < 0.8, base
        sur = ctx.surrogate((16, 256, 4, 2), synth.mlp_init_params([16, 256, 256, 256, 256, 2], seed=4))
        sur.train(X_tr, Y_tr, epochs=60, batch=512, lr=2e-3, weight_decay=1e-4)

        isl_c, X_c = synth.screening_designs(2048, seed=3, mesh_id=mid, first_index=10 ** 6)
        P = sur.infer(X_c)
        Y_c = label(isl_c)                        # fresh LLG solves: the judge of the surrogate
        acc = float(np.mean((P[:, 0] > 0.5) == (Y_c[:, 0] > 0.5)))
        a0 = auc(P[:, 0], Y_c[:, 0])
        top = np.argsort(-P[:, 0])[:256]
        hit = float(Y_c[top, 0].mean())
        rate = float(Y_c[:, 0].mean())
        print(f"base rate {rate:.3f}, screened hit rate {hit:.3f}, accuracy {acc:.3f}, AUC {a0:.4f}")
        assert acc >= 0.9 and a0 >= 0.95
        assert hit >= 0.98 and hit > rate + 0.2
        sur.destroy()
