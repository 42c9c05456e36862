"""Record layouts of the per-parton arrays (structure of arrays, tiles of 8
and of 32 events): the layout changes where the library keeps each element,
never what it computes.  The plain form, a multi-job batch and the serving
pool give bitwise the same events, observables and histograms in every
layout, and the autotuner's pick is one of them.  Requires a GB300."""
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


def _pass(g, p, n, layout, first_event=0, persistent=False):
    import torch
    ws = g.Workspace(n, 128, first_event, layout=layout)
    g.generate_me(p, ws)
    if persistent:
        g.shower_persistent(p, ws, {"block_threads": 128, "compact_period": 4, "layout": layout})
    else:
        g.shower(p, ws)
    g.validate(p, ws)
    g.observables(p, ws)
    hist = torch.zeros(g.HIST_DOUBLES, dtype=torch.float64, device="cuda")
    g.histograms(p, ws, hist)
    torch.cuda.synchronize()
    out = {k: v.cpu().numpy() for k, v in ws.scalars().items()}
    out.update({"m_" + k: v.cpu().numpy() for k, v in ws.momenta().items()})
    out.update({"c_" + k: v.cpu().numpy() for k, v in ws.colours().items()})
    out["obs"] = ws.obs().cpu().numpy()
    out["hist"] = hist.cpu().numpy()
    return out


def _same(a, b):
    n = a["n_partons"]
    kmax = int(n.max())
    live = np.arange(kmax)[:, None] < n[None, :]
    for k, v in a.items():
        if k.startswith("m_") or (k.startswith("c_") and k != "c_link"):
            assert np.array_equal(v[:kmax][live], b[k][:kmax][live]), k
        elif k == "c_link":
            assert np.array_equal(v[:, :kmax][:, live], b[k][:, :kmax][:, live]), k
        else:
            assert np.array_equal(v, b[k]), k


@pytest.mark.parametrize("persistent", [False, True])
def test_layouts_give_the_same_events(g, persistent):
    p = g.make_params(seed=23)
    n = 12347  # not a multiple of any tile
    ref = _pass(g, p, n, g.LAYOUT_SOA, first_event=99, persistent=persistent)
    for layout in (g.LAYOUT_TILE8, g.LAYOUT_TILE32):
        _same(ref, _pass(g, p, n, layout, first_event=99, persistent=persistent))


def test_layouts_in_multi_job_batches_and_the_pool(g):
    import torch
    from paper_2403_08692_gb300 import workloads
    jobs = workloads.uneven_batch(n_jobs=6, seed=41, n_min=100, n_max=5000)
    n = sum(j["n_events"] for j in jobs)
    hists = []
    for layout in (g.LAYOUT_SOA, g.LAYOUT_TILE8, g.LAYOUT_TILE32):
        ws = g.Workspace(n, 128, layout=layout)
        g.set_jobs([(g.make_params(sqrt_s=j["sqrt_s"], t_cutoff=j["t_cutoff"], seed=j["seed"]), j["n_events"],
                     j["first_event"]) for j in jobs], ws)
        g.generate_me(None, ws)
        g.shower_persistent(None, ws)
        g.validate(None, ws)
        g.observables(None, ws)
        h = torch.zeros(len(jobs) * g.HIST_DOUBLES, dtype=torch.float64, device="cuda")
        g.histograms(None, ws, h)
        hists.append((ws.scalars()["hash"].cpu().numpy(), ws.obs().cpu().numpy(), h.cpu().numpy()))
    for other in hists[1:]:
        for a, b in zip(hists[0], other):
            assert np.array_equal(a, b)
    # serving pool: jobs admitted at arbitrary pool offsets (sub-ranges of a tiled record)
    specs = [(g.make_params(seed=51), 3001, 7), (g.make_params(seed=52, sqrt_s=133.0), 1999, 0),
             (g.make_params(seed=53), 2500, 100)]
    results = []
    for layout in (g.LAYOUT_SOA, g.LAYOUT_TILE8):
        srv = g.Server(pool_events=5003, capacity=128, cycles_per_round=8, clock="rounds", layout=layout)
        res = srv.serve([g.ServeJob(p, nn, first, 0.0, tag=k) for k, (p, nn, first) in enumerate(specs)])
        results.append({r.tag: r.hist for r in res})
    for k in range(len(specs)):
        assert np.array_equal(results[0][k], results[1][k]), k


def test_autotuner_picks_a_layout(g):
    p = g.make_params(seed=29)
    ws = g.Workspace(30000, 128)
    cfg, ms = g.autotune_persistent(p, ws)
    assert cfg.layout in (g.LAYOUT_SOA, g.LAYOUT_TILE8, g.LAYOUT_TILE32) and ms > 0
    ref = _pass(g, p, 30000, g.LAYOUT_SOA)
    _same(ref, _pass(g, p, 30000, cfg.layout, persistent=True))
