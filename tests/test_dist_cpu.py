"""Multi-rank host logic on CPU: two gloo ranks, no GPU.

Elements are independent units of the fill, so a multi-GPU run shards them across ranks
and exchanges no data on the fill's path.  These tests run that logic with the CPU oracle
standing in for each rank's fill: the shards' element matrices put together equal the
unsharded fill, the ranges cover the batch, and the timing reductions give the slowest
rank's time and the whole job's unit count."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_1703_09619_gb300 import dist as D
from paper_1703_09619_gb300 import workloads as W


def free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def small_c4(n=5):
    wl = W.make("c4", n).with_npts(4)
    wl.orders[:] = np.minimum(wl.orders, 3)
    return wl


def _worker(rank, world, port, outdir):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import torch.distributed as dist
    w, r, _ = D.init("gloo")
    assert (w, r) == (world, rank)
    wl = small_c4()
    # strong scaling: one batch cut into entry-balanced contiguous ranges
    n = wl.ndof()
    lo, hi = D.balanced_ranges(4 * n * n, world)[rank]
    sub = wl.subset(np.arange(lo, hi))
    out, _, rc = oracle.fill(sub.orders, sub.kind, sub.params, sub.nodes, sub.bulge, sub.npts, nthreads=1)
    parts = [None] * world
    dist.all_gather_object(parts, (lo, hi, out.tolist(), rc))
    # timing reductions: the job time is the slowest rank's, units add up
    t = D.max_over_ranks(1.0 + rank, world)
    u = D.sum_over_ranks(10 * (rank + 1), world)
    # weak scaling: every rank's own batch differs from the others'
    mine = W.make("c5", 3, shard=rank).params
    batches = [None] * world
    dist.all_gather_object(batches, mine.tolist())
    D.barrier(world)
    if rank == 0:
        np.savez(os.path.join(outdir, "result.npz"),
                 ranges=np.array([(p[0], p[1]) for p in parts]),
                 out=np.concatenate([np.asarray(p[2]) for p in parts]),
                 rcs=np.array([p[3] for p in parts]), t=t, u=u,
                 batches=np.array(batches))
    dist.destroy_process_group()


@pytest.fixture(scope="module")
def two_rank_result(tmp_path_factory):
    import torch.multiprocessing as mp
    outdir = str(tmp_path_factory.mktemp("dist"))
    mp.start_processes(_worker, args=(2, free_port(), outdir), nprocs=2, join=True, start_method="spawn")
    return np.load(os.path.join(outdir, "result.npz"))


def test_two_ranks_shards_equal_unsharded_fill(two_rank_result):
    wl = small_c4()
    ref, _, rc = oracle.fill(wl.orders, wl.kind, wl.params, wl.nodes, wl.bulge, wl.npts, nthreads=1)
    r = two_rank_result
    assert (r["rcs"] == 0).all() and rc == 0
    assert r["ranges"][0][0] == 0 and r["ranges"][-1][1] == wl.n_elem
    assert r["ranges"][0][1] == r["ranges"][1][0]
    assert np.array_equal(r["out"], ref)  # each entry is one element's own sum: bitwise equal


def test_two_ranks_reductions(two_rank_result):
    assert float(two_rank_result["t"]) == 2.0
    assert float(two_rank_result["u"]) == 30.0


def test_two_ranks_weak_scaling_batches_differ(two_rank_result):
    b = two_rank_result["batches"]
    assert b.shape[0] == 2 and not np.array_equal(b[0], b[1])
    assert np.array_equal(b[0], W.make("c5", 3).params)  # rank 0 fills the canonical batch


def test_balanced_ranges_cover_and_balance():
    rng = np.random.default_rng(3)
    for world in (1, 2, 3, 4, 8):
        for n in (0, 1, 5, 97):
            w = rng.integers(1, 50, n).astype(float)
            rs = D.balanced_ranges(w, world)
            assert len(rs) == world
            assert rs[0][0] == 0 and rs[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
            assert all(lo <= hi for lo, hi in rs)
            if n:
                share, heavy = w.sum() / world, w.max()
                assert all(w[lo:hi].sum() <= share + heavy for lo, hi in rs)


def test_balanced_ranges_uneven_orders_by_entries():
    wl = W.make("c4", 256)
    n = wl.ndof()
    e = 4.0 * n * n
    rs = D.balanced_ranges(e, 4)
    sums = np.array([e[lo:hi].sum() for lo, hi in rs])
    assert sums.max() - sums.min() <= 2 * e.max()
    with pytest.raises(ValueError):
        D.balanced_ranges([1.0, -1.0], 2)
    with pytest.raises(ValueError):
        D.balanced_ranges([1.0], 0)
