"""The seeded workload generators (inputs only): the uneven 64-job batch and
the serving loop's Poisson arrivals are reproducible, stay in their stated
ranges and follow their stated distributions (log-uniform job sizes,
exponential gaps at the stated rate, the stated sqrt(s) and cutoff sets)."""
import math

import numpy as np

from paper_2403_08692_gb300 import workloads as W


def test_uneven_batch():
    jobs = W.uneven_batch()
    assert jobs == W.uneven_batch()  # same seed, same jobs
    assert len(jobs) == 64
    assert len({j["seed"] for j in jobs}) == 64  # one Philox key per job
    n = np.array([j["n_events"] for j in jobs])
    assert n.min() >= 1_000 and n.max() <= 1_000_000
    assert {j["sqrt_s"] for j in jobs} <= {91.2, 133.0, 200.0} and len({j["sqrt_s"] for j in jobs}) == 3
    assert {j["t_cutoff"] for j in jobs} <= {0.5, 1.0, 2.0} and len({j["t_cutoff"] for j in jobs}) == 3
    # log-uniform sizes over many draws: ln n uniform on [ln 1e3, ln 1e6]
    big = W.uneven_batch(n_jobs=20_000, seed=11)
    u = (np.log([j["n_events"] for j in big]) - math.log(1e3)) / (math.log(1e6) - math.log(1e3))
    hist, _ = np.histogram(u, bins=10, range=(0.0, 1.0))
    expect = len(u) / 10
    chi2 = float(((hist - expect) ** 2 / expect).sum())
    assert chi2 < 30.0, chi2  # 9 degrees of freedom; p ~ 4e-4 at 30
    assert W.uneven_batch(seed=5) != jobs


def test_poisson_arrivals():
    arr = W.poisson_arrivals()
    assert arr == W.poisson_arrivals()
    t = np.array([a[0] for a in arr])
    assert np.all(np.diff(t) > 0) and t[0] > 0 and t[-1] < 60.0
    # 50 jobs/s for 60 s: 3000 expected, Poisson spread sqrt(3000) ~ 55
    assert abs(len(arr) - 3000) < 5 * math.sqrt(3000)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 1 / 50) < 5 * (1 / 50) / math.sqrt(len(gaps))
    # exponential gaps: the fraction above the mean is 1/e
    assert abs((gaps > 1 / 50).mean() - math.exp(-1)) < 0.03
    n = np.array([a[1] for a in arr])
    assert n.min() >= 1_000 and n.max() <= 1_000_000
    assert len({a[2] for a in arr}) == len(arr)  # distinct job keys
