"""The C serving scheduler (gaps_server_create, gaps_submit, gaps_poll):
three jobs of different physics, sizes and first event ids submitted to a
pool too small for all of them at once (one waits for room), driven only
through the C ABI.  Each job's histograms are bitwise those of the same job
run alone and those the Python server gives for the same jobs, in both round
modes.  Requires a GB300."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

JOBS = [dict(sqrt_s=91.2, t_cutoff=1.0, seed=101, n=20000, first=0),
        dict(sqrt_s=133.0, t_cutoff=0.5, seed=102, n=35000, first=5000),
        dict(sqrt_s=200.0, t_cutoff=2.0, seed=103, n=8000, first=0)]
POOL = 50000


@pytest.fixture(scope="module")
def g():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2403_08692_gb300 as g
    g.load()
    return g


def _params(g, j):
    return g.make_params(sqrt_s=j["sqrt_s"], t_cutoff=j["t_cutoff"], seed=j["seed"])


def _alone(g, j):
    import torch
    p = _params(g, j)
    ws = g.Workspace(j["n"], 128, j["first"])
    g.generate_me(p, ws)
    g.shower(p, ws)
    g.validate(p, ws)
    g.observables(p, ws)
    hist = torch.zeros(g.HIST_DOUBLES, dtype=torch.float64, device="cuda")
    g.histograms(p, ws, hist)
    return hist.cpu().numpy()


def _serve_c(g, mode):
    srv = g.CServer(POOL, 128, max_jobs=8, cycles_per_round=8, mode=mode)
    ids = [srv.submit(_params(g, j), j["n"], j["first"]) for j in JOBS]
    out, waited, polls = {}, False, 0
    while len(out) < len(ids):
        for k, jid in enumerate(ids):
            if k in out:
                continue
            h = srv.poll(jid)
            polls += 1
            if h is not None:
                out[k] = h
        q, live, _ = srv.counts()
        waited |= q > 0 and live > 0
        assert polls < 200000, "serving did not finish"
    assert waited  # the second job had to wait for room
    with pytest.raises(g.GapsError):
        srv.poll(ids[0])  # already reported
    with pytest.raises(g.GapsError):
        srv.submit(_params(g, JOBS[0]), POOL + 1)  # larger than the pool
    srv.close()
    return out


@pytest.mark.parametrize("mode", ["slice", "steps"])
def test_c_scheduler_equals_alone_and_python_server(g, mode):
    cmode = g.SERVE_SLICE if mode == "slice" else g.SERVE_STEPS
    got = _serve_c(g, cmode)
    for k, j in enumerate(JOBS):
        assert np.array_equal(got[k], _alone(g, j)), k
        assert got[k].reshape(g.N_OBS, g.HIST_ROW, 3)[4, :, 2].sum() > 0.99 * j["n"]
    srv = g.Server(pool_events=POOL, capacity=128, cycles_per_round=8, clock="rounds", mode=mode)
    res = srv.serve([g.ServeJob(_params(g, j), j["n"], j["first"], 0.0, tag=k) for k, j in enumerate(JOBS)])
    for r in res:
        assert np.array_equal(r.hist, got[r.tag]), r.tag
