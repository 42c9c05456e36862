"""Serving loop (continuous batching over a resident pool): jobs that arrive
while others shower share the veto-cycle launches, wait for pool room when
the pool is full, and every job's results are the same alone and in the mix.
Requires a GB300."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2403_08692_gb300 as g
    g.load()
    return g


SCALARS = ("hash", "n_partons", "status", "n_steps", "n_trials", "n_winners", "n_emissions", "t", "weight",
           "me_flavour", "valid")


def _capture(ws, begin, n):
    sc = {k: v[begin:begin + n].cpu().numpy() for k, v in ws.scalars().items()}
    obs = ws.obs()[:, begin:begin + n].cpu().numpy()
    mom = {c: v[:, begin:begin + n].cpu().numpy() for c, v in ws.momenta().items()}
    return sc, obs, mom


def _alone(g, p, n, first_event, capacity):
    import torch
    ws = g.Workspace(n, capacity, first_event)
    g.generate_me(p, ws)
    g.shower(p, ws)
    g.validate(p, ws)
    g.observables(p, ws)
    hist = torch.zeros(g.HIST_DOUBLES, dtype=torch.float64, device="cuda")
    g.histograms(p, ws, hist)
    torch.cuda.synchronize()
    return _capture(ws, 0, n), hist.cpu().numpy()


def _assert_same_events(a, b, tag):
    sa, oa, ma = a
    sb, ob, mb = b
    for k in SCALARS:
        assert np.array_equal(sa[k], sb[k]), (tag, k)
    assert np.array_equal(oa, ob), tag
    n_partons = sa["n_partons"]
    live = np.arange(ma["e"].shape[0])[:, None] < n_partons[None, :]
    for c in ("e", "px", "py", "pz"):
        assert np.array_equal(ma[c][live], mb[c][live]), (tag, c)


@pytest.mark.parametrize("mode", ["slice", "steps"])
def test_pool_allocator_and_slots_reuse(g, mode):
    """Jobs admitted at different rounds into a pool too small for all of
    them at once: later jobs wait for room, ranges are reused, and each job
    equals the same job run alone, whether the pool advances by persistent
    slices or by plain-form steps."""
    cap = 128
    specs = [  # (sqrt_s, t_cutoff, seed, n_events, first_event, arrival round)
        (91.2, 1.0, 11, 20000, 0, 0),
        (200.0, 0.5, 12, 3000, 0, 0),
        (91.2, 1.0, 13, 1, 0, 2),
        (133.0, 2.0, 14, 15000, 777777, 3),
        (91.2, 1.0, 15, 777, 0, 5),
        (91.2, 1.0, 16, 25000, 0, 6),   # does not fit until the first jobs finish
        (200.0, 1.0, 17, 5000, 0, 40),
    ]
    jobs = []
    for k, (rs, tc, seed, n, first, arr) in enumerate(specs):
        p = g.make_params(sqrt_s=rs, t_cutoff=tc, seed=seed)
        jobs.append(g.ServeJob(p, n, first, float(arr), tag=k))
    srv = g.Server(pool_events=40000, capacity=cap, cycles_per_round=3, clock="rounds", mode=mode)
    seen = {}
    tag_of = {}

    def on_finish(job, ws, begin, stream):
        seen[job.tag] = _capture(ws, begin, job.n_events)
        tag_of[job.tag] = begin

    results = srv.serve(jobs, on_finish=on_finish, max_rounds=100000)
    assert sorted(r.tag for r in results) == list(range(len(specs)))
    assert srv.peak_live_jobs >= 3
    by_tag = {r.tag: r for r in results}
    # the 25000-event job had to wait for room
    assert by_tag[5].admitted > by_tag[5].arrival
    assert srv.alloc.free_events() == srv.pool_events
    for k, (rs, tc, seed, n, first, arr) in enumerate(specs):
        p = g.make_params(sqrt_s=rs, t_cutoff=tc, seed=seed)
        ev_alone, hist_alone = _alone(g, p, n, first, cap)
        _assert_same_events(seen[k], ev_alone, k)
        # exact fixed-point sums: the same events give the same bits
        assert np.array_equal(by_tag[k].hist, hist_alone), k
        # thrust and heavy-jet mass count every finished valid event once
        sc = seen[k][0]
        good = int(((sc["status"] == g.DONE) & (sc["valid"] == 0)).sum())
        counts = by_tag[k].hist.reshape(g.N_OBS, g.HIST_ROW, 3)[:, :, 2].sum(axis=1)
        assert np.all(counts[4:] == good)  # 1-T, rho_H, B_T, B_W: every finished valid event


@pytest.mark.parametrize("mode", ["slice", "steps"])
def test_wall_clock_poisson(g, mode):
    """Real-time Poisson arrivals: every job completes with its events all
    counted, latencies are positive, and the pool ends empty."""
    from paper_2403_08692_gb300 import workloads
    arrivals = workloads.poisson_arrivals(rate_per_s=100.0, duration_s=0.5, seed=9, n_min=1000, n_max=30000)
    jobs = [g.ServeJob(g.make_params(seed=s), n, 0, t, tag=k) for k, (t, n, s) in enumerate(arrivals)]
    srv = g.Server(pool_events=60000, capacity=128, cycles_per_round=8, clock="wall", mode=mode)
    results = srv.serve(jobs)
    assert len(results) == len(jobs)
    for r in results:
        assert r.latency > 0.0
        h = r.hist.reshape(g.N_OBS, g.HIST_ROW, 3)
        # thrust counts every finished valid event once (under/overflow included)
        assert 0.99 * r.n_events <= h[4, :, 2].sum() <= r.n_events
    assert srv.alloc.free_events() == srv.pool_events
    s = g.latency_summary(results, max(r.finished for r in results))
    assert s["jobs"] == len(jobs) and s["p99_latency_s"] >= s["p50_latency_s"] > 0.0


@pytest.mark.parametrize("trial_mode", [0, 1])
@pytest.mark.parametrize("mode", ["slice", "steps"])
def test_keyed_rounds_equal_general_rounds(g, mode, trial_mode):
    """Jobs that differ only in seed and first event: the pool runs its keyed
    kernels (physics from the launch, key and id offset per job), and every
    event and histogram is bitwise the one the general multi-job kernels give
    and the job gives alone, for both trial modes."""
    specs = [(21, 9000, 0, 0), (22, 4000, 123456, 0), (23, 1, 0, 1), (24, 7000, 0, 2)]

    def serve(keyed):
        jobs = [g.ServeJob(g.make_params(seed=s, trial_mode=trial_mode), n, first, float(arr), tag=k)
                for k, (s, n, first, arr) in enumerate(specs)]
        srv = g.Server(pool_events=16000, capacity=128, cycles_per_round=5, clock="rounds", mode=mode, keyed=keyed)
        seen = {}
        res = srv.serve(jobs, on_finish=lambda job, ws, b, st: seen.__setitem__(job.tag, _capture(ws, b, job.n_events)),
                        max_rounds=100000)
        return {r.tag: r.hist for r in res}, seen

    hk, ek = serve(True)
    hg, eg = serve(False)
    for k, (s, n, first, arr) in enumerate(specs):
        _assert_same_events(ek[k], eg[k], k)
        assert np.array_equal(hk[k], hg[k]), k
    s, n, first, _ = specs[1]
    ev_alone, hist_alone = _alone(g, g.make_params(seed=s, trial_mode=trial_mode), n, first, 128)
    _assert_same_events(ek[1], ev_alone, 1)
    assert np.array_equal(hk[1], hist_alone)


def test_finish_jobs_equals_finish_one_by_one(g):
    """gaps_pool_finish_jobs over several finished jobs (disjoint ranges,
    other live ranges between them) gives bitwise the validation bits,
    observables and per-slot histograms of one gaps_pool_finish per job."""
    import torch
    specs = [(91.2, 1.0, 31, 3000, 0, 5), (200.0, 0.5, 32, 2500, 3500, 2), (133.0, 2.0, 33, 1, 7000, 9),
             (91.2, 1.0, 34, 4000, 8000, 0)]  # (sqrt_s, t_C, seed, n, begin, slot)
    ws = g.Workspace(20000, 128)
    g.pool_reset(ws)
    for rs, tc, seed, n, b, slot in specs:
        g.pool_admit(g.make_params(sqrt_s=rs, t_cutoff=tc, seed=seed), slot, b, n, 0, ws, 0)
    total = sum(sp[3] for sp in specs)
    r = 0
    while True:
        g.pool_slice(ws, r, 16, total)
        r += 1
        if g.pool_progress(ws, r) == 0:
            break
    one = torch.zeros((g.MAX_JOBS, g.HIST_DOUBLES), dtype=torch.float64, device="cuda")
    for rs, tc, seed, n, b, slot in specs:
        g.pool_finish(slot, b, n, ws, one[slot])
    torch.cuda.synchronize()
    sc = ws.scalars()
    valid1 = sc["valid"].clone()
    obs1 = ws.obs().clone()
    sc["valid"].fill_(-7)
    ws.obs().fill_(-7.0)
    both = torch.zeros_like(one)
    g.pool_finish_jobs([sp[5] for sp in specs], [sp[4] for sp in specs], [sp[3] for sp in specs], ws, both)
    torch.cuda.synchronize()
    for rs, tc, seed, n, b, slot in specs:
        assert torch.equal(sc["valid"][b:b + n], valid1[b:b + n]), slot
        assert torch.equal(ws.obs()[:, b:b + n], obs1[:, b:b + n]), slot
        assert torch.equal(both[slot], one[slot]), slot
        assert float(both[slot].reshape(g.N_OBS, g.HIST_ROW, 3)[4, :, 2].sum()) > 0.0 or n == 1
    untouched = [k for k in range(g.MAX_JOBS) if k not in {sp[5] for sp in specs}]
    assert float(both[untouched].abs().sum()) == 0.0
    # the events between the ranges were not visited
    gap = sc["valid"][3000:3500]
    assert bool((gap == -7).all())


def test_observables_thread_and_group_forms_agree(g):
    """The observables of events of up to 16 partons run one thread per event
    in large batches and in groups of lanes in small ones (a finished serving
    round, one job): the same events give bitwise the same observables either
    way (one finalisation over two 30 000-event ranges, against one per
    range)."""
    import torch
    ws = g.Workspace(70000, 128)
    g.pool_reset(ws)
    specs = [(41, 30000, 0, 0), (42, 30000, 35000, 1)]  # seed, n, begin, slot
    for seed, n, b, slot in specs:
        g.pool_admit(g.make_params(seed=seed), slot, b, n, 0, ws, 0)
    r = 0
    while True:
        g.pool_slice(ws, r, 32, 60000, None, shared=g.make_params(seed=41))
        r += 1
        if g.pool_progress(ws, r) == 0:
            break
    hist = torch.zeros((g.MAX_JOBS, g.HIST_DOUBLES), dtype=torch.float64, device="cuda")
    g.pool_finish_jobs([sp[3] for sp in specs], [sp[2] for sp in specs], [sp[1] for sp in specs], ws, hist)
    torch.cuda.synchronize()
    together = ws.obs().clone()
    ws.obs().fill_(-7.0)
    for seed, n, b, slot in specs:
        g.pool_finish_jobs([slot], [b], [n], ws, hist)  # 30 000 events: the lane-group form
    torch.cuda.synchronize()
    for seed, n, b, slot in specs:
        assert torch.equal(ws.obs()[:, b:b + n], together[:, b:b + n]), slot
    assert bool((ws.obs()[:, 30000:35000] == -7.0).all())
