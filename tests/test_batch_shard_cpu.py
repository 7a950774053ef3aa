"""Host-side logic of batching and multi-rank sharding (no GPU): the batch
signature, the autotuner cache, the cost-balanced shard assignment, and a
two-rank gloo run that checks every set is reduced by exactly one rank."""
import json
import os
import socket
import types

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2008_11486_gb300 import batch, shard


def _fake_sets(shapes):
    return [types.SimpleNamespace(n=n, W=W, H=H) for (n, W, H) in shapes]


def test_signature_is_order_free_and_bucketed():
    a = _fake_sets([(3, 512, 512), (17, 1024, 1024), (40, 4096, 4096)])
    b = _fake_sets([(40, 4096, 4096), (3, 512, 512), (17, 1024, 1024)])
    assert batch.signature(a, "bilinear") == batch.signature(b, "bilinear")
    c = _fake_sets([(4, 512, 512), (18, 1024, 1024), (40, 4096, 4096)])  # same buckets
    assert batch.signature(a, "bilinear") == batch.signature(c, "bilinear")
    assert batch.signature(a, "bilinear") != batch.signature(a, "spline3")


def test_autotuner_caches_per_signature(tmp_path, monkeypatch):
    path = str(tmp_path / "tune.json")
    calls = []

    def fake_tune(self, sets, interp="bilinear", clip=None, persistent=True, stream=None):
        calls.append(len(sets))
        return {"rows_per_warp": 2, "max_ctas": 304}, {}

    monkeypatch.setattr(batch.Autotuner, "tune", fake_tune)
    monkeypatch.setattr(batch.core, "reduce_params", lambda *a, **k: ("params", a, k))
    t = batch.Autotuner(path)
    sets = _fake_sets([(5, 64, 64), (9, 64, 64)])
    p1, cfg1 = t.params_for(sets)
    p2, cfg2 = t.params_for(sets)
    # a cached choice without the distribution knob keeps the caller's form
    assert calls == [2] and cfg1 == cfg2 == {"persistent": True, "rows_per_warp": 2, "max_ctas": 304}
    saved = json.load(open(path))
    assert len(saved) == 1
    t2 = batch.Autotuner(path)  # a new process reads the cache instead of tuning
    t2.params_for(sets)
    assert calls == [2]


def test_autotuner_candidates_offer_each_bucket_its_other_tile_height(monkeypatch):
    """Rows per warp: 0 (the library's default) and the bucket's other
    choice -- 2 up to 16 frames (default 4), 1 up to 40 frames (default 2),
    above 40 frames 2 (default 1) except for the Keys stencil (1, default 2);
    the persistent grid as 0, 1x, 2x and 4x the SM count, or plain launches."""
    monkeypatch.setattr(batch, "lib", lambda: types.SimpleNamespace(irp_device_sm_count=lambda: 152))
    cases = [((5,), "bilinear", [0, 2]), ((24,), "bilinear", [0, 1]), ((40,), "cubic", [0, 1]),
             ((48,), "bilinear", [0, 2]), ((64,), "spline3", [0, 2]), ((57,), "cubic", [0, 1]),
             ((3, 33, 60), "bilinear", [0, 1, 2])]
    for ns, interp, rows in cases:
        cands = batch.Autotuner.candidates(_fake_sets([(n, 64, 64) for n in ns]), True, interp)
        assert sorted({c["rows_per_warp"] for c in cands}) == rows, (ns, interp)
        grids = sorted({c["max_ctas"] for c in cands if c["persistent"]})
        assert grids == [0, 152, 304, 608]
        assert {c["rows_per_warp"] for c in cands if not c["persistent"]} == set(rows)


def test_autotuner_ignores_an_unreadable_cache(tmp_path):
    for text in ("{not json", "[1, 2]", ""):
        path = tmp_path / "tune.json"
        path.write_text(text)
        assert batch.Autotuner(str(path)).cache == {}


def test_shard_sets_partition_and_balance():
    shapes = batch_shapes = [(n, s, s) for n, s in
                             zip([3, 40, 17, 8, 25, 31, 5, 12, 39, 22, 6, 14],
                                 [512, 4096, 2048, 1024, 4096, 512, 2048, 1024, 2048, 4096, 512, 1024])]
    costs = [shard.set_cost(*t) for t in shapes]
    for world in (1, 2, 3, 4, 8):
        parts = shard.shard_sets(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        # LPT bound: no rank exceeds the mean by more than the largest set
        assert max(loads) <= sum(costs) / world + max(costs)
    assert shard.shard_sets(costs, 3) == shard.shard_sets(costs, 3)
    with pytest.raises(ValueError):
        shard.shard_sets(costs, 0)


def _rank_main(rank, world, port, costs, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = shard.rank_shard(costs, world, rank)
    got = [None] * world
    dist.all_gather_object(got, mine)
    dist.destroy_process_group()
    q.put((rank, got))


def test_two_rank_gloo_shards_cover_every_set_once():
    costs = [shard.set_cost(n, s, s) for n, s in [(3, 512), (40, 4096), (17, 2048), (8, 1024),
                                                  (25, 4096), (31, 512), (5, 2048)]]
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, costs, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0] == res[1]
    all_ids = sorted(res[0][0] + res[0][1])
    assert all_ids == list(range(len(costs)))
    assert not set(res[0][0]) & set(res[0][1])
