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


def _fixed_worker(rank, world, port, out_dir):
    import torch.distributed as dist

    from paper_2403_08692_gb300 import sharding
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        acc = torch.from_numpy(np.load(os.path.join(out_dir, f"acc{rank}.npy")).view(np.int64).copy())
        sharding.merge_hist_fixed(acc, dist)
        np.save(os.path.join(out_dir, f"merged{rank}.npy"), acc.numpy().view(np.uint64))
    finally:
        dist.destroy_process_group()


def _as_int128(words):
    w = words.reshape(-1, 5).astype(object)
    signed = lambda hi: hi - (1 << 64) if hi >= (1 << 63) else hi
    return [(signed(int(r[1])) << 64) + int(r[0]) for r in w], [(signed(int(r[3])) << 64) + int(r[2]) for r in w], \
        [int(r[4]) for r in w]


def _random_fixed(rng, cells):
    """Accumulators of random signed 128-bit sums, many near the 64-bit
    boundary of their low words (so the merge must carry)."""
    vals = []
    for _ in range(cells):
        a = int(rng.integers(-(1 << 62), 1 << 62)) * (1 << 3) + int(rng.integers(0, 1 << 63))
        b = int(rng.integers(0, 1 << 62)) * (1 << 2)
        vals.append((a, b, int(rng.integers(0, 1 << 40))))
    words = np.zeros((cells, 5), dtype=np.uint64)
    for c, (a, b, n) in enumerate(vals):
        for k, v in ((0, a), (2, b)):
            u = v % (1 << 128)
            words[c, k] = u & ((1 << 64) - 1)
            words[c, k + 1] = u >> 64
        words[c, 4] = n
    return words.reshape(-1)


def test_fixed_point_histograms_merge_exactly(tmp_path):
    """Two ranks' fixed-point accumulators merge to the exact 128-bit sums,
    the same bits on every rank, whatever the carries."""
    import torch.multiprocessing as mp
    from paper_2403_08692_gb300 import sharding
    rng = np.random.default_rng(3)
    parts = [_random_fixed(rng, 816) for _ in range(WORLD)]
    for r, p in enumerate(parts):
        np.save(tmp_path / f"acc{r}.npy", p)
    mp.start_processes(_fixed_worker, args=(WORLD, _free_port(), str(tmp_path)), nprocs=WORLD, join=True,
                       start_method="spawn")
    m0, m1 = np.load(tmp_path / "merged0.npy"), np.load(tmp_path / "merged1.npy")
    assert np.array_equal(m0, m1)
    got = _as_int128(m0)
    want = [[x + y for x, y in zip(a, b)] for a, b in zip(_as_int128(parts[0]), _as_int128(parts[1]))]
    assert got[0] == want[0] and got[1] == want[1] and got[2] == want[2]
    # the order of the terms does not matter
    assert np.array_equal(sharding.add_fixed(parts[1], parts[0]), m0)
