"""The serving loop's schedule on the host, with a host-side stand-in for
the device pool: admission in arrival order as job slots and contiguous
ranges free up, ranges that never overlap, slots and ranges reused, a job
finalised once and only after all of its events finished, oversized jobs
rejected, and a pool that stops making progress ending in an error instead of
a hang.  The stand-in advances every live event by the round's cycles and
finishes each after a fixed, seeded number of cycles; the real pool is
exercised by tests/test_gpu_serving.py."""
import contextlib
import types

import numpy as np
import pytest
import torch

from paper_2403_08692_gb300 import serving


def _cycles_needed(seed, event_id):
    return 3 + (seed * 7919 + event_id * 104729) % 29


class FakePool:
    """The gaps_pool_* calls the server makes, on the host."""
    MAX_JOBS = 4
    HIST_DOUBLES = 4

    def __init__(self, stuck=False):
        self.stuck = stuck
        self.finished_jobs = []
        self.rounds_shared = []

    class _Workspace:
        def __init__(self, n, capacity, device="cpu"):
            self.n = n
            self.counters = torch.zeros(serving.COUNTER_WORDS, dtype=torch.int64)
            self.job_done = torch.zeros(FakePool.MAX_JOBS, dtype=torch.int64)
            self.remaining = {}   # batch event -> cycles left
            self.owner = {}       # batch event -> job slot
            self.jobs = {}        # slot -> (begin, n, first_event, seed)
            self.physics = {}     # slot -> the job's physics tag

        def view(self, name, dtype, shape):
            return {"counters": self.counters, "job_done": self.job_done}[name]

    def Workspace(self, n, capacity, device="cpu", layout=0):
        return FakePool._Workspace(n, capacity, device)

    @staticmethod
    def workspace_bytes(n, capacity):
        return 1000 * n

    def pool_reset(self, ws, stream=None):
        ws.counters.zero_()
        ws.job_done.zero_()
        ws.remaining.clear()
        ws.owner.clear()
        ws.jobs.clear()

    def pool_admit(self, params, slot, begin, n, first_event, ws, cycle, stream=None):
        assert slot not in ws.jobs, "job slot in use"
        assert 0 <= begin and begin + n <= ws.n
        for e in range(begin, begin + n):
            assert e not in ws.owner, "range overlaps a live job"
            ws.remaining[e] = _cycles_needed(params.seed, first_event + e - begin)
            ws.owner[e] = slot
        ws.jobs[slot] = (begin, n, first_event, params.seed)
        ws.physics[slot] = getattr(params, "physics", 0)
        ws.job_done[slot] = 0

    def _advance(self, ws, k, next_cycle):
        if not self.stuck:
            for e in list(ws.remaining):
                ws.remaining[e] -= k
                if ws.remaining[e] <= 0:
                    del ws.remaining[e]
                    ws.job_done[ws.owner[e]] += 1
        ws.counters[10 + next_cycle % 3] = len(ws.remaining)
        ws.counters[18 + next_cycle % 3] = 0

    @staticmethod
    def same_physics(a, b):
        return getattr(a, "physics", 0) == getattr(b, "physics", 0)

    def _check_shared(self, ws, shared):
        # the keyed form only when every live job has the shared physics
        live = {ws.owner[e] for e in ws.remaining}
        phys = {ws.physics[slot] for slot in live}
        self.rounds_shared.append(shared is not None)
        if shared is not None:
            assert phys <= {getattr(shared, "physics", 0)}, "keyed round over jobs of other physics"

    def pool_slice(self, ws, cycle, k, bound, cfg, shared=None, stream=None):
        assert bound >= len(ws.remaining), "the grid bound must cover every live event"
        self._check_shared(ws, shared)
        self._advance(ws, k, cycle + 1)

    def pool_cycles(self, ws, cycle, k, bound, shared=None, stream=None):
        assert bound >= len(ws.remaining), "the grid bound must cover every live event"
        self._check_shared(ws, shared)
        self._advance(ws, k, cycle + k)

    def pool_finish_jobs(self, slots, begins, counts, ws, hist, stream=None):
        assert len(set(slots)) == len(slots), "a slot finalised twice in one call"
        spans = sorted((b, b + n) for b, n in zip(begins, counts))
        assert all(a[1] <= b[0] for a, b in zip(spans, spans[1:])), "overlapping ranges"
        for slot, b, n in zip(slots, begins, counts):
            self.pool_finish(slot, b, n, ws, hist[slot], stream)

    def pool_finish(self, slot, begin, n, ws, hist, stream=None):
        assert ws.jobs[slot][:2] == (begin, n)
        assert int(ws.job_done[slot]) == n, "finalised before all of its events finished"
        assert not any(ws.owner[e] == slot for e in ws.remaining), "an event of the job is still live"
        _, _, first_event, seed = ws.jobs.pop(slot)
        for e in range(begin, begin + n):
            del ws.owner[e]
        hist[:] = torch.tensor([n, first_event, seed, 1.0], dtype=torch.float64)
        self.finished_jobs.append(first_event)


class _Event:
    def record(self, stream=None):
        pass

    def synchronize(self):
        pass

    def query(self):
        return True


class _Stream:
    def synchronize(self):
        pass

    def wait_stream(self, other):
        pass


_fake_torch = types.SimpleNamespace(
    zeros=torch.zeros, empty=torch.empty, tensor=torch.tensor, float64=torch.float64, int64=torch.int64,
    cuda=types.SimpleNamespace(Stream=lambda device=None: _Stream(), Event=_Event,
                               current_stream=lambda device=None: _Stream(),
                               stream=lambda s: contextlib.nullcontext()))


def _server(pool, pool_events, mode="slice", cycles=4):
    return serving.Server(pool_events=pool_events, capacity=8, cycles_per_round=cycles, clock="rounds",
                          device="cpu", mode=mode, device_layer=(pool, _fake_torch))


def _jobs(rng, count, max_events):
    jobs, first = [], 0
    for i in range(count):
        n = int(rng.integers(1, max_events + 1))
        jobs.append(serving.ServeJob(params=types.SimpleNamespace(seed=100 + i), n_events=n, first_event=first,
                                     arrival=float(rng.integers(0, 40)), tag=i))
        first += n
    return jobs


@pytest.mark.parametrize("mode", ["slice", "steps"])
def test_every_job_served_once_in_arrival_order(mode):
    rng = np.random.default_rng(3)
    jobs = _jobs(rng, 40, 120)
    pool = FakePool()
    srv = _server(pool, pool_events=300, mode=mode)
    results = srv.serve(jobs, max_rounds=10_000)
    assert sorted(r.tag for r in results) == list(range(len(jobs)))
    by_tag = {r.tag: r for r in results}
    for j in jobs:
        r = by_tag[j.tag]
        # each job's result is its own, whatever ran beside it
        assert np.array_equal(r.hist, np.array([j.n_events, j.first_event, j.params.seed, 1.0]))
        assert j.arrival <= r.admitted <= r.finished
        # it cannot finish before its longest event has had its cycles
        longest = max(_cycles_needed(j.params.seed, j.first_event + e) for e in range(j.n_events))
        assert r.finished - r.admitted >= np.ceil(longest / srv.cycles_per_round) - 1
    # strict arrival order: no job is admitted before one that arrived earlier
    order = sorted(jobs, key=lambda j: (j.arrival, j.tag))
    admitted = [by_tag[j.tag].admitted for j in order]
    assert all(a <= b for a, b in zip(admitted, admitted[1:]))
    # four job slots served forty jobs, and the pool held a few at a time
    assert len({r.slot for r in results}) == FakePool.MAX_JOBS
    assert srv.peak_live_jobs <= FakePool.MAX_JOBS
    assert sorted(pool.finished_jobs) == sorted(j.first_event for j in jobs)


def test_job_larger_than_the_pool_is_rejected():
    srv = _server(FakePool(), pool_events=50)
    job = serving.ServeJob(params=types.SimpleNamespace(seed=1), n_events=51, first_event=0, arrival=0.0, tag=0)
    with pytest.raises(ValueError):
        srv.serve([job])
    empty = serving.ServeJob(params=types.SimpleNamespace(seed=1), n_events=0, first_event=0, arrival=0.0, tag=0)
    with pytest.raises(ValueError):
        srv.serve([empty])


def test_a_pool_that_stops_progressing_ends_in_an_error():
    srv = _server(FakePool(stuck=True), pool_events=100)
    job = serving.ServeJob(params=types.SimpleNamespace(seed=1), n_events=10, first_event=0, arrival=0.0, tag=0)
    with pytest.raises(RuntimeError):
        srv.serve([job], max_rounds=50)


def test_memory_budget_sizes_the_pool():
    srv = serving.Server(memory_budget=123_456, capacity=8, clock="rounds", device="cpu",
                         device_layer=(FakePool(), _fake_torch))
    assert srv.pool_events == 123


def test_keyed_rounds_only_for_shared_physics():
    """Rounds run the keyed kernels (shared parameters passed) while every live
    job has the same physics, and the general ones once a job of other physics
    is live; the schedule and the results do not change."""
    rng = np.random.default_rng(3)
    jobs = _jobs(rng, 12, 40)
    pool = FakePool()
    srv = _server(pool, 200)
    srv.serve(jobs, max_rounds=10000)
    assert pool.rounds_shared and all(pool.rounds_shared)
    mixed = _jobs(rng, 12, 40)
    for i, j in enumerate(mixed):
        j.params.physics = i % 2
    pool2 = FakePool()
    srv2 = _server(pool2, 200)
    res = srv2.serve(mixed, max_rounds=10000)
    assert len(res) == len(mixed)
    assert not all(pool2.rounds_shared)
    off = _server(FakePool(), 200)
    off.keyed = False
    off.serve(_jobs(rng, 4, 40), max_rounds=10000)
    assert not any(off._gaps.rounds_shared)
