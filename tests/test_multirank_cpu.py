"""The multi-GPU path of bench.py on CPU: N independent replicas, timings reduced with a
maximum over ranks (gloo, world size 2, 127.0.0.1)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    got = bench.max_over_ranks([10.0 * (rank + 1), 5.0 - rank, 7.0])
    dist.barrier()
    out[rank] = got
    dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        assert out[0] == out[1] == [20.0, 5.0, 7.0]


def test_max_over_ranks_single_process_is_identity():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([1.5, 2.5]) == [1.5, 2.5]


def _shard_worker(rank, world, port, out):
    """One rank of a sharded batch: its share by the split rule, solved with the CPU oracle (the GPU
    path solves the same share with the batched kernel), the shares and residuals gathered."""
    import sys
    sys.path.insert(0, ROOT)
    import numpy as np
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle as O
    from paper_2206_05843_gb300 import shard, synth as S
    items = S.gen_batch(count=20, base_seed=31, n_lo=300, n_hi=3000, rhs_hi=4)
    costs = [shard.item_cost(it.matrix.nnz, it.nrhs) for it in items]
    mine = shard.shard_batch(costs, world)[rank]
    worst = 0.0
    for i in mine:
        it = items[i]
        x = O.forward_subst(it.matrix.rowptr, it.matrix.colidx, it.matrix.vals, it.b)
        rp = it.matrix.rowptr.astype(np.int64)
        rowid = np.repeat(np.arange(it.matrix.n), np.diff(rp))
        for k in range(it.nrhs):
            r = np.bincount(rowid, weights=it.matrix.vals * np.atleast_2d(x)[k][it.matrix.colidx],
                            minlength=it.matrix.n) - np.atleast_2d(it.b)[k]
            worst = max(worst, float(np.linalg.norm(r) / np.linalg.norm(np.atleast_2d(it.b)[k])))
    gathered = [None] * world
    dist.all_gather_object(gathered, {"items": mine, "residual": worst, "cost": sum(costs[i] for i in mine)})
    out[rank] = {"gathered": gathered, "costs": costs}
    dist.destroy_process_group()


def test_batch_shards_over_two_gloo_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_shard_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(300)
            assert p.exitcode == 0
        g0, g1 = out[0]["gathered"], out[1]["gathered"]
        assert g0 == g1  # every rank sees the same split
        costs = out[0]["costs"]
        shares = [set(g["items"]) for g in g0]
        assert not (shares[0] & shares[1]) and shares[0] | shares[1] == set(range(len(costs)))
        loads = [g["cost"] for g in g0]
        assert max(loads) - min(loads) <= max(costs)  # the longest-processing-time bound
        assert max(g["residual"] for g in g0) < 1e-12


def test_shard_batch_rule():
    import sys
    sys.path.insert(0, ROOT)
    from paper_2206_05843_gb300 import shard
    # 5 -> rank 0; 4 -> rank 1; 3 -> rank 1 (4 < 5); 3 -> rank 0 (5 < 7); 1 -> rank 1 (7 < 8): loads 8 and 8
    assert shard.shard_batch([5, 4, 3, 3, 1], 2) == [[0, 3], [1, 2, 4]]
    assert shard.shard_batch([7], 3) == [[0], [], []]
    assert shard.shard_batch([], 2) == [[], []]
    parts = shard.shard_batch(list(range(100, 0, -1)), 4)
    assert sorted(i for p in parts for i in p) == list(range(100))
