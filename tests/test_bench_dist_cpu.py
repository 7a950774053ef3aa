"""The benchmark's rank logic with 2 gloo ranks on the CPU.

Under torchrun every rank times its own steps; the job's time is the maximum
over ranks and, for the sharded batch workload, its pixels are the sum of
every rank's shard.  Here the same functions run over gloo
(IRP_DIST_BACKEND=gloo) in two spawned processes.
"""
import multiprocessing as mp
import os
import socket

import bench
from paper_2008_11486_gb300 import shard


def _rank_main(rank, world, port, q):
    os.environ.update(WORLD_SIZE=str(world), RANK=str(rank), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), IRP_DIST_BACKEND="gloo")
    w, r, _ = bench.dist_init()
    bench.barrier(w)
    t_max = bench.max_over_ranks(1.5 * (r + 1), w)
    # the batch workload's shards, as main() forms them
    shapes = bench.workload_shapes("batch")
    costs = [shard.set_cost(n, W, H) for (W, H, n) in shapes]
    mine = [shapes[i] for i in shard.rank_shard(costs, w, r)]
    px = bench.sum_over_ranks(float(sum(n * W * H for (W, H, n) in mine)), w)
    import torch.distributed as dist
    dist.destroy_process_group()
    q.put((r, w, t_max, px))


def test_two_gloo_ranks_time_by_the_slowest_and_count_every_pixel():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict((r, rest) for r, *rest in (q.get(timeout=120) for _ in procs))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    total = sum(n * W * H for (W, H, n) in bench.workload_shapes("batch"))
    for r in (0, 1):
        w, t_max, px = res[r]
        assert w == 2 and t_max == 3.0 and px == float(total)
    # one rank: no process group, the values pass through
    assert bench.max_over_ranks(2.5, 1) == 2.5 and bench.sum_over_ranks(7.0, 1) == 7.0
