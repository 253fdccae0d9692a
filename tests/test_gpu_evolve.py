"""Surrogate-assisted design search on the GPU: the surrogate is trained on LLG
outcomes of random designs, screens each generation on fresh jitter samples
through bpm_surrogate_screen, and only its best-screened designs are solved
with the batched LLG path.  Checked against fresh LLG solves: the screened
error rates of the verified designs, the gain of the screened picks over
random designs, and the error rate of the best design found."""
import os

import numpy as np
import pytest

from paper_1603_09493_gb300 import _lib as L
from paper_1603_09493_gb300 import api, evolve, synth

pytestmark = pytest.mark.gpu


def test_surrogate_assisted_search():
    if not os.path.exists(L.LIB_PATH):
        from paper_1603_09493_gb300 import build
        build.build()
    with api.Context(0) as ctx:
        mid = ctx.mesh_upload(synth.small_island_mesh(), synth.ecc_materials())
        p = evolve.run_params(100.0)
        # training set: 4096 random designs, one jitter sample each, labelled by LLG
        Zt = synth.counter_uniform(21, 0, np.arange(4096 * 4)).reshape(4096, 4)
        tgt, adj, Xt = evolve.samples(Zt, 1, seed=22, first_index=0, mesh_id=mid)
        Yt = evolve.llg_outcomes(ctx, mid, p, tgt, adj)
        print("training labels: switched %.3f, adjacent flipped %.3f" % tuple(Yt.mean(0)))
        assert 0.2 < Yt[:, 0].mean() < 0.9 and 0.02 < Yt[:, 1].mean() < 0.6
        sur = ctx.surrogate((16, 256, 4, 2), synth.mlp_init_params([16, 256, 256, 256, 256, 2], seed=4))
        sur.train(Xt, Yt, epochs=60, batch=512, lr=2e-3, weight_decay=1e-4)

        cfg = evolve.SearchConfig(generations=3, population=256, top_k=16, n_jitter_screen=32,
                                  n_jitter_verify=32, seed=23)
        res = evolve.search(ctx, sur, mid, cfg, t_end_ps=100.0)
        s = np.concatenate([h["screened_of_verified"] for h in res.history])
        v = np.concatenate([h["verified"] for h in res.history])
        print("best per generation", [round(h["best_verified"], 4) for h in res.history],
              "best rates", res.best_rates, "design", evolve.design_values(res.best_Z[None]))
        print(f"screen {res.screen_s:.2f} s, verify {res.verify_s:.2f} s, LLG only {res.llg_only_s:.2f} s")
        # the surrogate's error rates of the verified designs against their LLG rates (32 samples each)
        assert np.abs(s - v).mean() <= 0.1
        # random designs of the same space, solved with LLG, fare far worse than the screened picks
        Zr = synth.counter_uniform(24, 0, np.arange(16 * 4)).reshape(16, 4)
        tr, ar, _ = evolve.samples(Zr, 32, seed=25, first_index=0, mesh_id=mid)
        rand = evolve.error_rates(evolve.llg_outcomes(ctx, mid, p, tr, ar), 16, 32).sum(1)
        picks0 = np.array(res.history[0]["verified"])
        print(f"generation-0 picks {picks0.mean():.3f} against random designs {rand.mean():.3f}")
        assert picks0.mean() <= 0.5 * rand.mean()
        assert res.best_rates.sum() <= 0.25 and res.best_rates.sum() <= rand.min() + 1e-12
        assert res.llg_only_s > res.verify_s
        sur.destroy()
