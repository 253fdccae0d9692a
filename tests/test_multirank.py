"""The N-GPU path of the benchmark on CPU: two gloo ranks shard the islands
(disjoint, contiguous, covering) and reduce the timed region with max."""
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1603_09493_gb300 import shard, synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    lo, hi = shard.island_range(64, rank)
    isl = synth.jittered_islands(hi - lo, seed=1, first_index=lo)
    t = shard.max_over_ranks(10.0 + rank, dist)
    q.put((rank, lo, hi, isl.Ms_scale.tolist(), t))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, lo0, hi0, ms0, t0), (r1, lo1, hi1, ms1, t1) = res
    assert (lo0, hi0, lo1, hi1) == (0, 64, 64, 128)
    # each rank's islands are exactly the corresponding slice of the 1-process draw
    ref = synth.jittered_islands(128, seed=1).Ms_scale
    assert np.array_equal(np.array(ms0 + ms1, np.float32), ref)
    assert t0 == t1 == 11.0
