"""The batched persistent form at its paper-scale workload: 10^7 LEP events,
seed 3, the autotuned launch shape, the whole pass (ME, shower, validation,
observables, histograms) captured in one CUDA graph and replayed.  Sampled
events against the oracle one by one, every histogram against the oracle's
10^7-event histograms.  Requires a GB300 (133 GB workspace)."""
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


def test_config3_persistent_graph_1e7(g, oracle_mod):
    import torch
    n = 10_000_000
    p = g.make_params(seed=3)
    ws = g.Workspace(n, 128)
    cfg, _ = g.autotune_persistent(p, ws)
    hist = torch.zeros(g.HIST_DOUBLES, dtype=torch.float64, device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph, stream=side):
            hist.zero_()
            g.generate_me(p, ws, side)
            g.shower_persistent(p, ws, cfg, side)
            g.validate(p, ws, side)
            g.observables(p, ws, side)
            g.histograms(p, ws, hist, side)
    torch.cuda.synchronize()
    ws.buffer.zero_()
    graph.replay()
    torch.cuda.synchronize()
    stats = torch.zeros(16, dtype=torch.int64, device="cuda")
    g.reduce_stats(ws, stats)
    st = g.Stats.from_buffer_copy(stats.cpu().numpy().tobytes()[:len(bytes(g.Stats()))])
    assert st.n_events == n and st.n_done == n and st.n_invalid == 0 and st.n_overflow == 0

    sc = {k: v.cpu().numpy() for k, v in ws.scalars().items()}
    sc["hash"] = sc["hash"].view(np.uint64)
    rng = np.random.default_rng(2025)
    ids = np.sort(rng.choice(n, size=3000, replace=False))
    idx = torch.from_numpy(ids).cuda()
    e = ws.momenta()["e"][:, idx].cpu().numpy()      # sampled columns only
    obs = ws.obs()[:, idx].cpu().numpy()
    op = H.oracle_params(oracle_mod, 128, seed=3)
    same = 0
    for c, j in enumerate(ids):
        one = oracle_mod.run(op, int(j), 1, want_momenta=True)
        ev = one["events"][0]
        if ev["hash"] == sc["hash"][j] and ev["n_partons"] == sc["n_partons"][j]:
            same += 1
            k = ev["n_partons"]
            ref = one["mom"][0, :k, 0]
            assert np.all(np.abs(e[:k, c] - ref) <= H.MOM_REL * ref + H.MOM_ABS)
            o = one["obs"][0]
            assert np.all(np.abs(obs[:, c] - o) <= H.OBS_REL * np.abs(o) + H.OBS_ABS)
    assert same / len(ids) >= H.AGREE_MIN
    del e, obs
    orc = oracle_mod.run(op, 0, n, threads=oracle_mod.threads_available(), want_obs=False)
    chi2, ndf = H.hist_chi2(hist.cpu().numpy().reshape(g.N_OBS, g.HIST_ROW, 3), orc["hist"])
    assert chi2 < 1.5, (chi2, ndf)
    # the same events on both sides: only bin-edge rounding could still differ
    assert chi2 < 0.05, (chi2, ndf)
    print("config3", cfg.as_dict(), "max steps", st.max_steps, "chi2/ndf", chi2)
    del graph, ws
    torch.cuda.empty_cache()
