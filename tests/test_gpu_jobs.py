"""Uneven multi-job batches: many jobs with their own sqrt(s), cutoff and
seed showered in one launch, with per-job histograms.  Every event must be
the event a single-job batch of its job produces, and agree with the oracle.
Requires a GB300."""
import numpy as np
import pytest

from paper_2403_08692_gb300 import workloads
from tests import gpu_harness as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2403_08692_gb300 as g
    g.load()
    return g


def _params(g, job):
    return g.make_params(sqrt_s=job["sqrt_s"], t_cutoff=job["t_cutoff"], alphas_mz=job["alphas_mz"],
                         seed=job["seed"])


def _multi(g, jobs, persistent, capacity=128):
    import torch
    n = sum(j["n_events"] for j in jobs)
    ws = g.Workspace(n, capacity)
    g.set_jobs([(_params(g, j), j["n_events"], j["first_event"]) for j in jobs], ws)
    g.generate_me(None, ws)
    if persistent:
        g.shower_persistent(None, ws)
    else:
        g.shower(None, ws)
    g.validate(None, ws)
    g.observables(None, ws)
    hist = torch.zeros(len(jobs) * g.HIST_DOUBLES, dtype=torch.float64, device="cuda")
    g.histograms(None, ws, hist)
    torch.cuda.synchronize()
    return ws, hist.cpu().numpy().reshape(len(jobs), g.N_OBS, g.HIST_ROW, 3)


def _single(g, job, capacity=128):
    import torch
    ws = g.Workspace(job["n_events"], capacity, job["first_event"])
    p = _params(g, job)
    g.generate_me(p, ws)
    g.shower(p, ws)
    g.validate(p, ws)
    g.observables(p, ws)
    hist = torch.zeros(g.HIST_DOUBLES, dtype=torch.float64, device="cuda")
    g.histograms(p, ws, hist)
    torch.cuda.synchronize()
    return ws, hist.cpu().numpy().reshape(g.N_OBS, g.HIST_ROW, 3)


def _slice(ws, lo, hi):
    sc = {k: v.cpu().numpy()[lo:hi] for k, v in ws.scalars().items()}
    return sc, ws.obs().cpu().numpy()[:, lo:hi]


@pytest.mark.parametrize("persistent", [False, True])
def test_small_mix_equals_single_jobs(g, persistent):
    jobs = workloads.uneven_batch(n_jobs=12, seed=40, n_min=100, n_max=20000)
    jobs[3]["first_event"] = 123456  # a job whose event ids do not start at 0
    ws, hist = _multi(g, jobs, persistent)
    lo = 0
    for j, job in enumerate(jobs):
        hi = lo + job["n_events"]
        ws1, h1 = _single(g, job)
        a, oa = _slice(ws, lo, hi)
        b, ob = _slice(ws1, 0, job["n_events"])
        for k in ("hash", "n_partons", "status", "n_steps", "n_trials", "weight", "me_flavour", "valid"):
            assert np.array_equal(a[k], b[k]), (j, k)
        assert np.array_equal(oa, ob)
        # exact fixed-point sums: the same events give the same bits
        assert np.array_equal(hist[j], h1), j
        lo = hi


def test_config4_uneven_batch_against_oracle(g, oracle_mod):
    """64 jobs, event counts log-uniform in [10^3, 10^6], sqrt(s) from
    {91.2, 133, 200} GeV, cutoffs from {0.5, 1, 2} GeV^2, one key per job, all
    in one persistent launch: every job's sampled events match the oracle."""
    jobs = workloads.uneven_batch()
    ws, hist = _multi(g, jobs, persistent=True)
    sc = {k: v.cpu().numpy() for k, v in ws.scalars().items()}
    sc["hash"] = sc["hash"].view(np.uint64)
    assert np.all(sc["status"] == g.DONE) and np.all(sc["valid"] == 0)
    rng = np.random.default_rng(11)
    lo, same, total = 0, 0, 0
    for j, job in enumerate(jobs):
        n = job["n_events"]
        picks = rng.choice(n, size=min(n, 40), replace=False)
        op = oracle_mod.make_params(sqrt_s=job["sqrt_s"], t_cutoff=job["t_cutoff"], seed=job["seed"], capacity=128)
        for k in picks:
            ev = oracle_mod.run(op, int(k), 1, want_obs=False, want_hist=False)["events"][0]
            total += 1
            same += int(ev["hash"] == sc["hash"][lo + k] and ev["n_partons"] == sc["n_partons"][lo + k])
        # the job's histogram holds exactly its finished events with y23
        assert hist[j, 0, :, 2].sum() == np.sum(sc["n_partons"][lo:lo + n] >= 3)
        lo += n
    assert same / total >= H.AGREE_MIN, (same, total)


def test_job_table_validation(g):
    p = g.make_params()
    ws = g.Workspace(100, 128)
    with pytest.raises(g.GapsError):
        g.set_jobs([(p, 60, 0), (p, 30, 0)], ws)  # counts do not add up
    with pytest.raises(g.GapsError):
        g.set_jobs([(g.make_params(t_cutoff=0.0), 100, 0)], ws)
    with pytest.raises(g.GapsError):
        g.set_jobs([(p, 100, 0xFFFFFFF0)], ws)  # ids would wrap
    g.set_jobs([(p, 0, 0), (p, 100, 7), (p, 0, 0)], ws)  # empty jobs are fine
