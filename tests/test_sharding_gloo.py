"""Multi-rank host logic on CPU: world_size 2 over gloo.

Each rank transports its shard of the histories (the CPU oracle stands in for
the per-GPU engine, which needs a GPU), the int64 tallies are summed with an
all-reduce, and the result must equal the single-process run bit for bit."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1503_01722_gb300 import sharding


def test_split_covers_range_exactly():
    for n in (0, 1, 7, 1000, 10 ** 9 + 3):
        for w in (1, 2, 3, 8):
            parts = [sharding.split(n, r, w) for r in range(w)]
            assert parts[0][0] == 0
            assert sum(c for _, c, _ in parts) == n
            for (f0, c0, _), (f1, _, _) in zip(parts, parts[1:]):
                assert f0 + c0 == f1
    assert sharding.shard(3, 4, 100) == (300, 100, 400)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, n, out_dir, fail_rank):
    import torch
    import torch.distributed as dist
    import ocmc_inputs as I
    import oracle as O
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        if rank == fail_rank:
            raise RuntimeError("injected rank failure")
        ph = I.scaled(I.slab(), 6)
        beam = I.beam_on(ph, 0, I.spectrum_6mv(), (10, 10), 100.0)
        first, count, total = sharding.split(n, rank, world)
        r = O.run(ph, beam, total, first=first, count=count, seed=4, threads=2)
        t = torch.from_numpy(r.tally.copy())
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        if rank == 0:
            np.save(os.path.join(out_dir, "sum.npy"), t.numpy())
    finally:
        dist.destroy_process_group()


def test_two_rank_allreduce_equals_single_run(tmp_path):
    import ocmc_inputs as I
    import oracle as O
    n = 1500
    mp.start_processes(_worker, args=(2, _free_port(), n, str(tmp_path), -1), nprocs=2, start_method="spawn")
    got = np.load(tmp_path / "sum.npy")
    ph = I.scaled(I.slab(), 6)
    beam = I.beam_on(ph, 0, I.spectrum_6mv(), (10, 10), 100.0)
    ref = O.run(ph, beam, n, seed=4, threads=2).tally
    assert np.array_equal(got, ref)


def test_failed_rank_surfaces_on_host(tmp_path):
    """A rank that raises before the collective: the launcher reports the failure
    instead of hanging (the surviving rank's all-reduce ends with an error)."""
    os.environ["TORCH_DIST_INIT_BARRIER"] = "0"
    with pytest.raises(Exception):
        mp.start_processes(_worker, args=(2, _free_port(), 300, str(tmp_path), 1), nprocs=2,
                           start_method="spawn")
