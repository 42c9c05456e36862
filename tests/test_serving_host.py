"""Host-side logic of the serving loop (no GPU): the first-fit range
allocator that admits jobs by pool room, and the latency summary."""
import random

import pytest

from paper_2403_08692_gb300.serving import RangeAllocator, ServeResult, latency_summary


def test_first_fit_and_coalescing():
    a = RangeAllocator(100)
    assert a.alloc(30) == 0
    assert a.alloc(30) == 30
    assert a.alloc(50) is None          # only 40 left
    assert a.alloc(40) == 60
    assert a.alloc(1) is None
    a.free(30, 30)
    assert a.alloc(31) is None          # hole of 30
    a.free(0, 30)                       # coalesces with [30, 60)
    assert a.alloc(60) == 0
    a.free(60, 40)
    a.free(0, 60)
    assert a.free_events() == 100 and a.alloc(100) == 0


def test_random_alloc_free_never_overlaps():
    rng = random.Random(3)
    size = 10_000
    a = RangeAllocator(size)
    owned = {}
    for _ in range(5000):
        if owned and rng.random() < 0.45:
            b = rng.choice(list(owned))
            a.free(b, owned.pop(b))
        else:
            n = rng.randint(1, 900)
            b = a.alloc(n)
            if b is None:
                assert n > max([0] + [a._len[x] for x in a._begin])
                continue
            assert 0 <= b and b + n <= size
            for c, m in owned.items():
                assert b + n <= c or c + m <= b
            owned[b] = n
        assert a.free_events() + sum(owned.values()) == size
        # free ranges never touch: coalescing is complete
        ends = [(x, x + a._len[x]) for x in a._begin]
        assert all(e0[1] < e1[0] for e0, e1 in zip(ends, ends[1:]))
    for b in list(owned):
        a.free(b, owned.pop(b))
    assert a._begin == [0] and a._len[0] == size


def test_latency_summary():
    import numpy as np
    rs = [ServeResult(k, 1000, np.zeros(1), 0.0, 0.0, 0.01 * (k + 1), 0, 0) for k in range(100)]
    s = latency_summary(rs, 2.0)
    assert s["events"] == 100_000 and s["events_per_s"] == pytest.approx(50_000.0)
    assert s["p50_latency_s"] == pytest.approx(0.505)
    assert s["p99_latency_s"] == pytest.approx(0.9901)
