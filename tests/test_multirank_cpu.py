"""The N > 1 path of the benchmark on CPU: two gloo ranks (codewords are independent, so
ranks are replicas with disjoint shards and only the timing is reduced across them)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r, w, _ = bench.dist_env()
    worst = bench.max_over_ranks(1.5 + rank)              # each rank's own step time
    wl = bench.make_inputs(2, r)
    out.put((r, w, worst, wl.info.copy(), bench.job_gbps(w, 3, 2, wl.K, worst)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=240) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, t0, info0, g0), (r1, w1, t1, info1, g1) = res
    assert (r0, r1, w0, w1) == (0, 1, 2, 2)
    assert t0 == t1 == 2.5                                   # max over ranks on both
    assert g0 == g1 == pytest.approx(2 * 3 * 2 * 8448 / 2.5 / 1e9)
    import bench
    whole = bench.make_inputs(4, 0)                          # the same codewords, one shard
    assert np.array_equal(np.concatenate([info0, info1]), whole.info)
    assert not np.array_equal(info0, info1)
