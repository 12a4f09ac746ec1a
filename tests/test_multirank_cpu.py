"""The N > 1 path on CPU: two gloo ranks run bench.py's distributed helpers
(barrier, max-over-ranks timing) and merge per-rank error statistics on the
host, as the GPU ranks do (no collective on the data path)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    from oracle import oracle as O
    from paper_2003_02633_gb300 import ivc, synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(dist)
        t = bench.max_over_ranks(dist, float(10 * (rank + 1)), torch.device("cpu"))
        # each rank owns its shard (its own seeds), as in the benchmark
        x = synth.random_vectors(2000, seed=2 * rank)
        xh = O.decompress(O.PRIMARY, O.compress(O.PRIMARY, x))
        s = O.error_stats(x, xh)
        acc = [s["n"], s["mean"] * s["n"], (s["sd"] ** 2) * (s["n"] - 1) + s["n"] * s["mean"] ** 2,
               s["max"], s["mean_rel"] * s["n"], s["max_rel"], s["rms_ang"] ** 2 * s["n"],
               s["max_ang"], s["rms_mag_rel"] ** 2 * s["n"], s["max_mag_rel"], 0.0]
        gathered = [None] * world
        dist.all_gather_object(gathered, acc)
        merged = ivc.merge_stats(gathered)
        q.put((rank, t, merged, x[:3].tolist()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    assert all(r[1] == 20.0 for r in res)          # max over ranks
    assert res[0][2] == res[1][2]                  # same merged stats everywhere
    merged = res[0][2]
    assert merged[0] == 4000
    assert res[0][3] != res[1][3]                  # distinct shards
    from oracle import oracle as O
    from paper_2003_02633_gb300 import synth
    x = np.concatenate([synth.random_vectors(2000, seed=0), synth.random_vectors(2000, seed=2)])
    s = O.error_stats(x, O.decompress(O.PRIMARY, O.compress(O.PRIMARY, x)))
    assert np.isclose(merged[1] / merged[0], s["mean"], rtol=1e-12)
    assert merged[3] == pytest.approx(s["max"], rel=1e-15)
