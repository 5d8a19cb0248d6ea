"""Multi-rank path on the CPU: event sharding and the cross-section merge,
run as two gloo ranks (world_size 2) that each reweight their shard with the
oracle and merge sigma'_p; the result must equal the single-process exact sum."""
import math
import os
import socket

import numpy as np
import pytest

from paper_2312_07440_gb300 import shard


def test_shard_ranges_cover_exactly():
    for n in (0, 1, 7, 1000, 1 << 20):
        for world in (1, 2, 3, 8):
            got = [shard.shard_range(n, r, world) for r in range(world)]
            assert got[0][0] == 0 and got[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(got, got[1:]))
            sizes = [b - a for a, b in got]
            assert max(sizes) - min(sizes) <= 1


def test_merge_sums_is_compensated():
    rng = np.random.default_rng(0)
    parts = rng.lognormal(size=(5, 3)) * np.array([1e16, 1.0, 1e-8])
    parts[:, 1] = [1e16, 1.0, -1e16, 1.0, 1e-3]
    got = shard.merge_sums(parts)
    for j in range(3):
        assert abs(got[j] - math.fsum(parts[:, j])) <= 2 * np.spacing(abs(math.fsum(parts[:, j])) + 1e-300)


def test_merge_pairs_keeps_each_shards_compensation():
    """A shard's compensation term can exceed the ulp of the total; merging
    the collapsed values loses it, merging the pairs keeps it."""
    sums = np.array([[1e16], [1.0], [-1e16]])
    comps = np.array([[0.75], [0.0], [0.5]])
    exact = math.fsum([1e16, 0.75, 1.0, -1e16, 0.5])
    assert shard.merge_pairs(sums, comps)[0] == exact
    assert shard.merge_sums(sums + comps)[0] != exact


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_path):
    import torch.distributed as dist

    import oracle
    from paper_2312_07440_gb300 import events as ev
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    oracle.set_threads(1)
    wl = ev.WORKLOADS["gg_tt_1m"]
    n_total = 3001
    a, b = shard.shard_range(n_total, rank, world)
    mom, w = ev.generate(wl, b - a, start=a)
    pts = ev.reweight_points("gg_tt_1m")
    res = oracle.reweight("gg_tt", ev.param_vector(), pts, mom, w)
    # each shard's sums as (sum, compensation) pairs, as the library returns them
    parts = list(res["wnew"]) + [w]
    s = [math.fsum(x) for x in parts]
    c = [math.fsum(list(x) + [-v]) for x, v in zip(parts, s)]
    merged = shard.allreduce_pairs(s, c)
    if rank == 0:
        np.save(out_path, merged)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_merge_to_the_single_process_sum(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    import oracle
    from paper_2312_07440_gb300 import events as ev
    out = str(tmp_path / "merged.npy")
    mp.start_processes(_rank_main, args=(2, _free_port(), out), nprocs=2, start_method="spawn")
    merged = np.load(out)
    mom, w = ev.generate(ev.WORKLOADS["gg_tt_1m"], 3001)
    ref = oracle.reweight("gg_tt", ev.param_vector(), ev.reweight_points("gg_tt_1m"), mom, w)
    # shard-wise exact sums merged with compensation: within 2 ulp of the exact total
    assert abs(merged[0] - ref["sigma"][0]) <= 2 * np.spacing(ref["sigma"][0])
    assert abs(merged[1] - ref["sigma_orig"]) <= 2 * np.spacing(ref["sigma_orig"])
    assert torch is not None
