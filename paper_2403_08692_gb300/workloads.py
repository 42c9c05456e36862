"""Seeded synthetic workloads (inputs only, no physics): the job mixes and
arrival schedules the tests, the benchmark and the serving loop use.

The paper's workload is itself generated, so a workload is a list of jobs:
physics parameters, an event count and a seed.  Every draw here comes from a
numpy Generator with a fixed seed, so the same call always returns the same
jobs.
"""
import math

import numpy as np

LEP_SQRT_S = 91.2
ALPHAS_MZ = 0.118


def uneven_batch(n_jobs=64, seed=4, n_min=1_000, n_max=1_000_000, sqrt_s_choices=(91.2, 133.0, 200.0),
                 t_cutoff_choices=(0.5, 1.0, 2.0)):
    """Uneven multi-job batch: event counts log-uniform in [n_min, n_max],
    sqrt(s) and cutoff drawn from the given sets, one Philox key per job
    (seed * 1000 + job index).  Returns a list of dicts."""
    rng = np.random.default_rng(seed)
    jobs = []
    for j in range(n_jobs):
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        jobs.append({"sqrt_s": float(rng.choice(sqrt_s_choices)), "t_cutoff": float(rng.choice(t_cutoff_choices)),
                     "alphas_mz": ALPHAS_MZ, "seed": seed * 1000 + j, "n_events": n, "first_event": 0})
    return jobs


def poisson_arrivals(rate_per_s=50.0, duration_s=60.0, seed=5, n_min=1_000, n_max=1_000_000):
    """Serving workload: Poisson arrivals at rate_per_s for duration_s, each
    job of log-uniform size at LEP energy.  Returns (arrival time in s,
    event count, job seed) per job, sorted by time."""
    rng = np.random.default_rng(seed)
    t, out, j = 0.0, [], 0
    while True:
        t += rng.exponential(1.0 / rate_per_s)
        if t >= duration_s:
            break
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        out.append((t, n, seed * 100000 + j))
        j += 1
    return out
