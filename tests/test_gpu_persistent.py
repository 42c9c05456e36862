"""The persistent shower form (one launch, per-block event pools with
compaction and refill) against the plain per-cycle form and the oracle.
Both forms draw the same random numbers per (seed, event, cycle), so every
event must come out bit-identical.  Requires a GB300."""
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


def _run(g, p, n, persistent, cfg=None, capacity=128, first_event=0, layout=0):
    import torch
    ws = g.Workspace(n, capacity, first_event, layout=layout)
    g.generate_me(p, ws)
    if persistent:
        g.shower_persistent(p, ws, cfg)
    else:
        g.shower(p, ws)
    g.validate(p, ws)
    g.observables(p, ws)
    torch.cuda.synchronize()
    sc = {k: v.cpu().numpy() for k, v in ws.scalars().items()}
    mom = {k: v.cpu().numpy() for k, v in ws.momenta().items()}
    return ws, sc, mom, ws.obs().cpu().numpy(), ws.view("counters", torch.int64, (16,)).cpu().numpy()


def _assert_same(a, b):
    _, sa, ma, oa, _ = a
    _, sb, mb, ob, _ = b
    for k in ("hash", "n_partons", "status", "n_steps", "n_emissions", "n_winners", "n_trials", "n_dipoles",
              "me_flavour", "valid", "t", "weight"):
        assert np.array_equal(sa[k], sb[k]), k
    kmax = int(sa["n_partons"].max())
    slot = np.arange(kmax)[:, None]
    live = slot < sa["n_partons"][None, :]
    for c in ("e", "px", "py", "pz"):
        assert np.array_equal(ma[c][:kmax][live], mb[c][:kmax][live]), c
    assert np.array_equal(oa, ob)


def test_persistent_equals_plain(g):
    p = g.make_params(seed=5)
    plain = _run(g, p, 20011, persistent=False)
    pers = _run(g, p, 20011, persistent=True)
    _assert_same(plain, pers)
    # every event finished, counted once
    assert pers[4][0] == 20011 and pers[4][6] >= 20011


@pytest.mark.parametrize("layout", [0, 1, 2])
@pytest.mark.parametrize("threads,period,per_sm", [(64, 1, 0), (128, 2, 0), (256, 4, 1), (512, 3, 0), (128, 8, 0),
                                                  (256, 16, 0), (512, 7, 1)])
def test_persistent_launch_shapes(g, threads, period, per_sm, layout):
    """Every launch shape, in every record layout (structure of arrays,
    tiles of 8 and of 32 events), gives the plain form's events."""
    p = g.make_params(seed=6)
    plain = _run(g, p, 7001, persistent=False)
    cfg = {"block_threads": threads, "compact_period": period, "blocks_per_sm": per_sm, "layout": layout}
    _assert_same(plain, _run(g, p, 7001, persistent=True, cfg=cfg, layout=layout))


def test_persistent_matches_oracle(g, oracle_mod):
    """Config 1 (10^4 events, seed 1) through the persistent form."""
    p = g.make_params(seed=1)
    ws = g.Workspace(10000, 128)
    g.generate_me(p, ws)
    g.shower_persistent(p, ws)
    g.validate(p, ws)
    g.observables(p, ws)
    import torch
    torch.cuda.synchronize()
    sc = {k: v.cpu().numpy() for k, v in ws.scalars().items()}
    sc["hash"] = sc["hash"].view(np.uint64)
    mom = ws.momenta()
    col = ws.colours()
    gpu = {"scalars": sc,
           "mom": np.stack([mom[c].cpu().numpy() for c in ("e", "px", "py", "pz")], axis=-1).transpose(1, 0, 2),
           "info": np.stack([col["flav"].cpu().numpy().astype(np.int32), col["col"].cpu().numpy().astype(np.int32),
                             col["acol"].cpu().numpy().astype(np.int32)], axis=-1).transpose(1, 0, 2),
           "obs": ws.obs().cpu().numpy().T.copy()}
    orc = oracle_mod.run(H.oracle_params(oracle_mod, 128, seed=1), 0, 10000,
                         threads=oracle_mod.threads_available(), want_momenta=True)
    res = H.compare_events(gpu, orc)
    assert res["agree"] >= H.AGREE_MIN, res


def test_persistent_step_limit_and_overflow(g, oracle_mod):
    for kw, cap in ((dict(seed=3, max_steps=6), 128), (dict(seed=3), 4)):
        p = g.make_params(**kw)
        pers = _run(g, p, 3000, persistent=True, capacity=cap)
        plain = _run(g, p, 3000, persistent=False, capacity=cap)
        _assert_same(plain, pers)
        orc = oracle_mod.run(H.oracle_params(oracle_mod, cap, **kw), 0, 3000, want_obs=False, want_hist=False)
        assert np.array_equal(pers[1]["status"], orc["events"]["status"])


def test_empty_and_tiny_batches(g):
    p = g.make_params(seed=8)
    for n in (0, 1, 63, 257):
        ws = g.Workspace(n, 128)
        g.generate_me(p, ws)
        g.shower_persistent(p, ws)
    with pytest.raises(g.GapsError):
        g.shower_persistent(p, g.Workspace(10, 128), {"block_threads": 96, "compact_period": 1})
    with pytest.raises(g.GapsError):
        g.shower_persistent(p, g.Workspace(10, 128), {"block_threads": 128, "compact_period": 0})


def test_autotuner_picks_a_valid_shape(g):
    p = g.make_params(seed=9)
    ws = g.Workspace(100000, 128)
    cfg, ms = g.autotune_persistent(p, ws)
    assert cfg.block_threads in (128, 256, 512) and cfg.compact_period in (2, 4, 8, 16) and ms > 0
    # the tuned shape gives the same events as the plain form
    plain = _run(g, p, 20000, persistent=False)
    _assert_same(plain, _run(g, p, 20000, persistent=True, cfg=cfg.as_dict()))


def test_run_with_persistent_form(g):
    import torch
    p = g.make_params(seed=10)
    h1 = torch.zeros(g.HIST_DOUBLES, dtype=torch.float64).pin_memory()
    h2 = torch.zeros(g.HIST_DOUBLES, dtype=torch.float64).pin_memory()
    rc1, st1 = g.run(p, g.Workspace(30000, 128), h1, g.SHOWER_PLAIN)
    rc2, st2 = g.run(p, g.Workspace(30000, 128), h2, g.SHOWER_PERSISTENT)
    assert rc1 == rc2 == 0
    assert st2.launches == 1 and st1.max_steps <= st1.launches <= 2 * st1.max_steps
    for f in ("n_done", "sum_steps", "sum_trials", "sum_emissions", "max_steps"):
        assert getattr(st1, f) == getattr(st2, f), f
    np.testing.assert_allclose(h1.numpy(), h2.numpy(), rtol=1e-12, atol=1e-9)


def test_cuda_graph_replay_of_the_pass(g):
    """The asynchronous pass (matrix element, persistent shower, validation,
    observables) captured in a CUDA graph and replayed gives the events of a
    direct plain-form run."""
    import torch
    p = g.make_params(seed=12)
    n = 50000
    plain = _run(g, p, n, persistent=False)
    ws = g.Workspace(n, 128)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph, stream=side):
            g.generate_me(p, ws, side)
            g.shower_persistent(p, ws, None, side)
            g.validate(p, ws, side)
            g.observables(p, ws, side)
    for _ in range(2):
        ws.buffer.zero_()
        graph.replay()
        torch.cuda.synchronize()
        sc = {k: v.cpu().numpy() for k, v in ws.scalars().items()}
        for k in ("hash", "n_partons", "n_steps", "status"):
            assert np.array_equal(sc[k], plain[1][k]), k
        assert np.array_equal(ws.obs().cpu().numpy(), plain[3])


def test_paper_scale_persistent(g):
    """10^6 events: the persistent form reproduces the plain form event by
    event (decision hashes and multiplicities)."""
    import torch
    p = g.make_params(seed=2)
    res = []
    for persistent in (False, True):
        ws = g.Workspace(1_000_000, 128)
        g.generate_me(p, ws)
        if persistent:
            g.shower_persistent(p, ws)
        else:
            g.shower(p, ws)
        torch.cuda.synchronize()
        sc = ws.scalars()
        res.append((sc["hash"].cpu().numpy(), sc["n_partons"].cpu().numpy(), sc["n_steps"].cpu().numpy()))
        del ws
    for a, b in zip(*res):
        assert np.array_equal(a, b)
