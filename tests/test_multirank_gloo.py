"""The multi-GPU path's host logic on two CPU ranks (gloo): disjoint event
ranges per rank, the job time as the maximum over ranks, and the merged
histograms.  The ranks' union must equal one batch of all their events.
The showers here come from the oracle (no GPU)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

N_PER_RANK = 150
WORLD = 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist

    from oracle import oracle as O
    from paper_2403_08692_gb300 import sharding
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        first, n = sharding.shard(rank, world, N_PER_RANK, first_event=1000)
        p = O.make_params(seed=21)
        r = O.run(p, first, n, threads=1)
        hist = torch.from_numpy(r["hist"].copy())
        sharding.merge_histograms(hist, dist)
        t = sharding.job_time_ms(10.0 * (rank + 1), dist)
        hashes = [None] * world
        dist.all_gather_object(hashes, r["events"]["hash"].tolist())
        if rank == 0:
            np.save(os.path.join(out_dir, "hist.npy"), hist.numpy())
            np.save(os.path.join(out_dir, "hash.npy"), np.concatenate([np.array(h, dtype=np.uint64)
                                                                       for h in hashes]))
            np.save(os.path.join(out_dir, "time.npy"), np.array([t]))
    finally:
        dist.destroy_process_group()


def test_two_ranks_equal_one_batch(tmp_path, oracle_mod):
    import torch.multiprocessing as mp
    mp.start_processes(_worker, args=(WORLD, _free_port(), str(tmp_path)), nprocs=WORLD, join=True,
                       start_method="spawn")
    whole = oracle_mod.run(oracle_mod.make_params(seed=21), 1000, WORLD * N_PER_RANK, threads=1)
    assert np.array_equal(np.load(tmp_path / "hash.npy"), whole["events"]["hash"].astype(np.uint64))
    np.testing.assert_allclose(np.load(tmp_path / "hist.npy"), whole["hist"], rtol=1e-12, atol=1e-12)
    assert float(np.load(tmp_path / "time.npy")[0]) == 20.0


def test_shard_ranges():
    from paper_2403_08692_gb300 import sharding
    ranges = [sharding.shard(r, 4, 250, first_event=7) for r in range(4)]
    assert ranges == [(7, 250), (257, 250), (507, 250), (757, 250)]
    with pytest.raises(ValueError):
        sharding.shard(4, 4, 250)
