"""GPU parity of the per-dipole trial mode (one trial per dipole with the
summed overestimate, the kernel drawn by its share) against the oracle's
same mode, in every shower form.  Requires a GB300."""
import numpy as np
import pytest

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


def _both(g, O, n, seed, **kw):
    gp = g.make_params(seed=seed, trial_mode=g.TRIALS_PER_DIPOLE, **kw)
    op = H.oracle_params(O, 128, seed=seed, trial_mode=O.TRIALS_PER_DIPOLE, **kw)
    gpu = H.run_gpu(g, gp, n, 128)
    orc = O.run(op, 0, n, threads=O.threads_available(), want_momenta=True)
    return gpu, orc


@pytest.mark.parametrize("kw", [dict(), dict(sqrt_s=200.0, t_cutoff=0.5), dict(n_flavours=3, fixed_alphas=1)])
def test_per_dipole_plain_matches_oracle(g, oracle_mod, kw):
    gpu, orc = _both(g, oracle_mod, 10000, seed=51, **kw)
    res = H.compare_events(gpu, orc)
    assert res["agree"] >= H.AGREE_MIN, res
    sc = gpu["scalars"]
    assert np.all(sc["status"] == g.DONE) and np.all(sc["valid"] == 0)
    assert np.array_equal(sc["n_trials"], sc["n_dipoles"])  # one trial per dipole


def test_per_dipole_persistent_equals_plain(g):
    import torch
    p = g.make_params(seed=52, trial_mode=g.TRIALS_PER_DIPOLE)
    out = []
    for persistent in (False, True):
        ws = g.Workspace(30000, 128)
        g.generate_me(p, ws)
        if persistent:
            g.shower_persistent(p, ws)
        else:
            g.shower(p, ws)
        torch.cuda.synchronize()
        sc = ws.scalars()
        out.append({k: sc[k].cpu().numpy() for k in ("hash", "n_partons", "n_steps", "n_trials")})
    for k in out[0]:
        assert np.array_equal(out[0][k], out[1][k]), k


def test_modes_mix_in_one_batch(g):
    """A multi-job batch with one job per mode: each job's events equal the
    same job run alone."""
    import torch
    jobs = [(g.make_params(seed=61), 3000, 0), (g.make_params(seed=62, trial_mode=g.TRIALS_PER_DIPOLE), 4000, 0)]
    ws = g.Workspace(7000, 128)
    g.set_jobs(jobs, ws)
    g.generate_me(None, ws)
    g.shower_persistent(None, ws)
    torch.cuda.synchronize()
    mix = ws.scalars()["hash"].cpu().numpy()
    lo = 0
    for p, n, first in jobs:
        w1 = g.Workspace(n, 128, first)
        g.generate_me(p, w1)
        g.shower(p, w1)
        torch.cuda.synchronize()
        assert np.array_equal(mix[lo:lo + n], w1.scalars()["hash"].cpu().numpy())
        lo += n


def test_per_dipole_paper_scale(g, oracle_mod):
    """10^6 events in the per-dipole mode: sampled events against the oracle
    one by one and every histogram against the oracle's (the same events,
    so chi^2/ndf near zero)."""
    import torch
    n = 1_000_000
    p = g.make_params(seed=53, trial_mode=g.TRIALS_PER_DIPOLE)
    ws = g.Workspace(n, 128)
    host = torch.zeros(g.HIST_DOUBLES, dtype=torch.float64).pin_memory()
    rc, st = g.run(p, ws, host)
    assert rc == 0 and st.n_done == n and st.n_invalid == 0
    assert st.sum_trials == st.sum_dipoles
    sc = {k: v.cpu().numpy() for k, v in ws.scalars().items()}
    sc["hash"] = sc["hash"].view(np.uint64)
    op = H.oracle_params(oracle_mod, 128, seed=53, trial_mode=oracle_mod.TRIALS_PER_DIPOLE)
    ids = np.sort(np.random.default_rng(7).choice(n, size=2000, replace=False))
    same = sum(1 for j in ids if oracle_mod.run(op, int(j), 1, want_obs=False, want_hist=False)["events"][0]["hash"]
               == sc["hash"][j])
    assert same / len(ids) >= H.AGREE_MIN
    orc = oracle_mod.run(op, 0, n, threads=oracle_mod.threads_available(), want_obs=False)
    chi2, ndf = H.hist_chi2(host.numpy().reshape(g.N_OBS, g.HIST_ROW, 3), orc["hist"])
    assert chi2 < 0.05, (chi2, ndf)
