"""The multi-rank paths on the CPU (gloo, world size 2): the batch of independent
patches is sharded without a data-path collective, every rank computes the same
partition, and the results are combined as the maximum time and the summed counts
over ranks (the reductions bench.py makes under torchrun)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import paper_2102_11536_gb300 as iga
        import workloads as W
        ws = W.multipatch_batch()
        works = [iga.patch_work(w.ndof, w.p[0]) for w in ws]
        sh = iga.shard_patches(works, world)
        mine = [None] * world
        dist.all_gather_object(mine, sh[rank])
        mx, sm = bench.combine_over_ranks(torch, dist, torch.device("cpu"), [1.5 * (rank + 1), 10.0 - rank],
                                          [float(rank + 1), 2.0])
        q.put((rank, sh, mine, mx, sm, works))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_the_batch_and_combine_results():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    sh0 = res[0][1]
    works = res[0][5]
    for rank, sh, mine, mx, sm, _ in res:
        assert sh == sh0                    # every rank computes the same partition
        assert mine == sh0                  # and holds exactly its own shard
        assert mx == [3.0, 10.0]            # maximum time over ranks
        assert sm == [3.0, 4.0]             # summed counts
    flat = sorted(i for part in sh0 for i in part)
    assert flat == list(range(len(works)))  # disjoint cover of the 48 patches
    loads = [sum(works[i] for i in part) for part in sh0]
    assert max(loads) <= 1.05 * sum(loads) / world


def test_shard_patches_host_logic():
    import paper_2102_11536_gb300 as iga
    assert iga.shard_patches([5.0, 1.0, 1.0, 3.0], 1) == [[0, 1, 2, 3]]
    assert iga.shard_patches([5.0, 1.0, 1.0, 3.0], 2) == [[0], [1, 2, 3]]
    assert iga.shard_patches([1.0], 3) == [[0], [], []]
    with pytest.raises(ValueError):
        iga.shard_patches([1.0], 0)
    assert iga.patch_work(10, 3) == 10 * 343.0
