"""Serving loop: continuous batching of shower jobs on one GPU.

Shower jobs (physics parameters, an event count, the id of their first
event) arrive over time.  The server keeps one resident workspace, the pool,
sized by a device-memory budget.  A job is admitted as soon as a free job
slot and a free contiguous range of the pool can hold its events: its matrix
elements are generated in place and its events join the live active list.
Each round then advances the live events of all jobs at once, so jobs that
arrive while others shower share their launches: either one launch of the
persistent form that runs every live event for a slice of veto cycles in
per-block pools (mode "slice"), or a few launches of the plain form's step
over the active list (mode "steps").  A job whose events
have all reached the cutoff is finalised on its own range (validation,
observables, its own histograms), its histograms go back to the host, and its
range and slot are reused (the jobs that finish in the same round are
finalised together, in one sequence of launches).

All of the arithmetic runs in the library's kernels (gaps_pool_* in
include/gaps.h); this module only keeps the schedule: the arrival queue, the
first-fit range allocator, the job slots, the cycle count and an upper bound
on the live events that sizes the grids.  Progress is read back
asynchronously one round behind, so the GPU always has the next round of
cycles queued while the host inspects the last one.

Every event is the event a single-job batch of its job produces: its
draws are keyed by (seed, event id, its own cycle), never by where or when it
ran, so a job's results are the same alone and in any mix (the histograms
too: they are exact fixed-point sums).
"""
import bisect
import collections
import dataclasses
import time

import numpy as np

from . import gaps

COUNTER_WORDS = 32   # device counter words of a workspace (include/gaps.h)


@dataclasses.dataclass
class ServeJob:
    """A request: parameters (gaps.Params), its event count, the id of its
    first event, its arrival time (seconds from the start of serving, or
    rounds for the round clock) and a caller tag."""
    params: object
    n_events: int
    first_event: int = 0
    arrival: float = 0.0
    tag: object = None


@dataclasses.dataclass
class ServeResult:
    tag: object
    n_events: int
    hist: np.ndarray          # GAPS_HIST_DOUBLES doubles, this job only
    arrival: float            # seconds from the start
    admitted: float
    finished: float           # its histograms are on the host
    slot: int
    ev_begin: int

    @property
    def latency(self):
        return self.finished - self.arrival


class RangeAllocator:
    """First-fit allocator of contiguous event ranges in [0, size), with
    coalescing of freed neighbours."""

    def __init__(self, size):
        self.size = int(size)
        self._begin = [0]           # sorted free range starts
        self._len = {0: self.size}

    def alloc(self, n):
        for b in self._begin:
            ln = self._len[b]
            if ln >= n:
                i = bisect.bisect_left(self._begin, b)
                del self._begin[i]
                del self._len[b]
                if ln > n:
                    bisect.insort(self._begin, b + n)
                    self._len[b + n] = ln - n
                return b
        return None

    def free(self, b, n):
        i = bisect.bisect_left(self._begin, b)
        # merge with the following range
        if i < len(self._begin) and self._begin[i] == b + n:
            n += self._len.pop(self._begin[i])
            del self._begin[i]
        # merge with the preceding range
        if i > 0 and self._begin[i - 1] + self._len[self._begin[i - 1]] == b:
            p = self._begin[i - 1]
            self._len[p] += n
            return
        self._begin.insert(i, b)
        self._len[b] = n

    def free_events(self):
        return sum(self._len.values())


class Server:
    """Continuous-batching shower server over one resident pool.

    pool_events: pool size in events (None: from memory_budget bytes);
    capacity: parton slots per event; cycles_per_round: veto cycles per
    event and round; clock: "wall" (arrival times in seconds, served in real
    time) or "rounds" (arrival times in rounds, for deterministic tests);
    mode: "slice" (one persistent launch per round, launch shape cfg) or
    "steps" (cycles_per_round plain-form steps per round).  device_layer:
    (binding, torch) pair the server drives; None is this package's binding
    and PyTorch on a CUDA device (the host-logic tests pass a host-side
    stand-in and device "cpu")."""

    def __init__(self, pool_events=None, capacity=128, memory_budget=None, cycles_per_round=8, clock="wall",
                 device="cuda", mode="slice", cfg=None, device_layer=None, layout=0, keyed=True):
        if device_layer is None:
            import torch
            device_layer = (gaps, torch)
        self._gaps, torch = device_layer
        G = self._gaps
        if pool_events is None:
            if memory_budget is None:
                raise ValueError("give pool_events or memory_budget")
            per_event = G.workspace_bytes(1 << 20, capacity) / float(1 << 20)
            pool_events = int(memory_budget // per_event)
        self.pool_events = int(pool_events)
        self.capacity = int(capacity)
        self.cycles_per_round = int(cycles_per_round)
        if clock not in ("wall", "rounds"):
            raise ValueError("clock must be 'wall' or 'rounds'")
        if mode not in ("slice", "steps"):
            raise ValueError("mode must be 'slice' or 'steps'")
        self.clock = clock
        self.mode = mode
        self.cfg = cfg
        self.keyed = keyed
        pin = (lambda t: t) if device == "cpu" else (lambda t: t.pin_memory())
        self.ws = G.Workspace(self.pool_events, self.capacity, device=device, layout=layout)
        self.stream = torch.cuda.Stream(device=device)
        self.hist = torch.zeros((G.MAX_JOBS, G.HIST_DOUBLES), dtype=torch.float64, device=device)
        self.hist_host = pin(torch.empty((G.MAX_JOBS, G.HIST_DOUBLES), dtype=torch.float64))
        # the buffers were filled on the current stream: the server's stream
        # starts after those fills
        self.stream.wait_stream(torch.cuda.current_stream(device))
        self._counters = self.ws.view("counters", torch.int64, (COUNTER_WORDS,))
        self._job_done = self.ws.view("job_done", torch.int64, (G.MAX_JOBS,))
        self._progress_host = [pin(torch.empty(COUNTER_WORDS + G.MAX_JOBS, dtype=torch.int64)) for _ in range(2)]
        self._torch = torch
        self.reset()

    # ------------------------------------------------------------ state
    def reset(self):
        self.alloc = RangeAllocator(self.pool_events)
        self.free_slots = list(range(self._gaps.MAX_JOBS - 1, -1, -1))
        self.queue = collections.deque()
        self.live = {}                  # slot -> (job, ev_begin, admitted time, admitted round)
        self.cycle = 0
        self.rounds = 0
        self.admitted_events = 0        # running total, for the live bound
        self.bound = 0                  # upper bound on live events
        self.launched_cycles = 0
        self.peak_live_jobs = 0
        self._inflight = collections.deque()
        self._completions = []
        self._gaps.pool_reset(self.ws, stream=self.stream)

    def _now(self, t0):
        return time.perf_counter() - t0 if self.clock == "wall" else float(self.rounds)

    def _admit(self, now):
        while self.queue and self.free_slots:
            job = self.queue[0]
            begin = self.alloc.alloc(job.n_events)
            if begin is None:
                return  # first in, first admitted: wait for room
            self.queue.popleft()
            slot = self.free_slots.pop()
            self._gaps.pool_admit(job.params, slot, begin, job.n_events, job.first_event, self.ws, self.cycle,
                                  stream=self.stream)
            self.live[slot] = (job, begin, now, self.rounds)
            self.admitted_events += job.n_events
            self.bound += job.n_events
        self.peak_live_jobs = max(self.peak_live_jobs, len(self.live))

    def _shared_physics(self):
        """The live jobs' common parameters when they differ only in their
        seeds (the pool then runs its keyed kernels), else None."""
        if not self.keyed or not self.live:
            return None
        jobs = [job for job, _, _, _ in self.live.values()]
        first = jobs[0].params
        return first if all(self._gaps.same_physics(j.params, first) for j in jobs[1:]) else None

    def _launch_round(self):
        torch = self._torch
        k = self.cycles_per_round
        bound = min(self.bound, self.pool_events)
        shared = self._shared_physics()
        if self.mode == "slice":
            # self.cycle counts slices: the rotation index of the pool's lists
            self._gaps.pool_slice(self.ws, self.cycle, k, bound, self.cfg, shared=shared, stream=self.stream)
            self.cycle += 1
        else:
            self._gaps.pool_cycles(self.ws, self.cycle, k, bound, shared=shared, stream=self.stream)
            self.cycle += k
        self.launched_cycles += k
        buf = self._progress_host[self.rounds % 2]
        with torch.cuda.stream(self.stream):
            buf[:COUNTER_WORDS].copy_(self._counters, non_blocking=True)
            buf[COUNTER_WORDS:].copy_(self._job_done, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(self.stream)
        self._inflight.append((ev, buf, self.admitted_events, self.rounds, self.cycle))
        self.rounds += 1

    def _read_round(self, now, on_finish):
        torch = self._torch
        ev, buf, admitted_at_copy, read_round, cycle = self._inflight.popleft()
        ev.synchronize()
        # live events: the active list and the pending emissions of the next step
        active = int(buf[10 + cycle % 3]) + int(buf[18 + cycle % 3])
        self.bound = active + (self.admitted_events - admitted_at_copy)
        done = buf[COUNTER_WORDS:].numpy()
        # A job admitted after this read was enqueued would see the finished
        # count of its slot's previous job.
        finished = [slot for slot, (job, _, _, admitted_round) in self.live.items()
                    if admitted_round <= read_round and done[slot] >= job.n_events]
        if not finished:
            return
        with torch.cuda.stream(self.stream):
            for slot in finished:
                self.hist[slot].zero_()
            # every job finished this round, finalised in one sequence of launches
            self._gaps.pool_finish_jobs(finished, [self.live[k][1] for k in finished],
                                        [self.live[k][0].n_events for k in finished], self.ws, self.hist,
                                        stream=self.stream)
        for slot in finished:
            job, begin, admitted, _ = self.live[slot]
            with torch.cuda.stream(self.stream):
                if on_finish is not None:
                    on_finish(job, self.ws, begin, self.stream)
                self.hist_host[slot].copy_(self.hist[slot], non_blocking=True)
                fin = torch.cuda.Event()
                fin.record(self.stream)
            self._completions.append((fin, slot, job, begin, admitted))
            del self.live[slot]
            # The range and the slot are free for admissions queued after the
            # copies above (same stream).
            self.alloc.free(begin, job.n_events)

    def _collect(self, now, results, block=False):
        keep = []
        for fin, slot, job, begin, admitted in self._completions:
            if block:
                fin.synchronize()
            elif not fin.query():
                keep.append((fin, slot, job, begin, admitted))
                continue
            finished = self._now(self._t0)
            results.append(ServeResult(job.tag, job.n_events, self.hist_host[slot].numpy().copy(), job.arrival,
                                       admitted, finished, slot, begin))
            self.free_slots.append(slot)
        self._completions = keep

    # -------------------------------------------------------------- serve
    def serve(self, jobs, on_finish=None, max_rounds=None):
        """Serve the jobs (ServeJob, any order) to completion.  on_finish(job,
        workspace, ev_begin, stream), if given, runs when a job's range is
        final, before the range is reused (tests read the events there).
        Returns the list of ServeResult in completion order."""
        for j in jobs:
            if j.n_events < 1 or j.n_events > self.pool_events:
                raise ValueError(f"job of {j.n_events} events does not fit a pool of {self.pool_events}")
        pending = sorted(jobs, key=lambda j: j.arrival)
        results = []
        i = 0
        self._t0 = time.perf_counter()
        while i < len(pending) or self.queue or self.live or self._completions:
            now = self._now(self._t0)
            while i < len(pending) and pending[i].arrival <= now:
                self.queue.append(pending[i])
                i += 1
            self._admit(now)
            if self.bound > 0:
                self._launch_round()
            if self._inflight and (len(self._inflight) >= 2 or self.bound == 0):
                self._read_round(now, on_finish)
            self._collect(now, results)
            idle = self.bound == 0 and not self._inflight
            if idle and not self.live and not self.queue:
                if self._completions:
                    self._collect(now, results, block=True)
                elif i < len(pending):
                    if self.clock == "wall":
                        time.sleep(max(0.0, pending[i].arrival - self._now(self._t0)))
                    else:
                        self.rounds = max(self.rounds, int(np.ceil(pending[i].arrival)))
            if max_rounds is not None and self.rounds > max_rounds:
                raise RuntimeError("serving did not finish within max_rounds")
        self.stream.synchronize()
        return results


def latency_summary(results, wall_s):
    """p50/p99 job latency (s) and sustained events/s over wall_s seconds."""
    lat = np.array([r.latency for r in results]) if results else np.zeros(1)
    events = sum(r.n_events for r in results)
    return {"jobs": len(results), "events": events, "wall_s": wall_s,
            "events_per_s": events / wall_s if wall_s > 0 else 0.0,
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "max_latency_s": float(lat.max())}
