"""GPU histograms (Sec. 3.2, atomic histogramming) in exact fixed point: the
same events give the same bits whatever the order of the fills -- two runs,
the plain and the persistent forms, and two half-batches merged by 128-bit
addition -- and the double histograms are the fixed-point sums converted
once.  Requires a GB300."""
import math

import numpy as np
import pytest

from paper_2403_08692_gb300 import sharding

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2403_08692_gb300 as g
    g.load()
    return g


def _pass(g, p, n, first=0, persistent=False):
    import torch
    ws = g.Workspace(n, 128, first)
    g.generate_me(p, ws)
    if persistent:
        g.shower_persistent(p, ws, {"block_threads": 256, "compact_period": 4})
    else:
        g.shower(p, ws)
    g.validate(p, ws)
    g.observables(p, ws)
    hist = torch.zeros(g.HIST_DOUBLES, dtype=torch.float64, device="cuda")
    g.histograms(p, ws, hist)
    acc = torch.zeros(g.HIST_FIXED_WORDS, dtype=torch.int64, device="cuda")
    g.histograms_fixed(p, ws, acc)
    torch.cuda.synchronize()
    return hist.cpu().numpy(), acc.cpu().numpy().view(np.uint64)


def test_histograms_are_order_free_and_exact(g):
    p = g.make_params(seed=17)
    n = 60001
    h1, a1 = _pass(g, p, n)
    h2, a2 = _pass(g, p, n)
    h3, a3 = _pass(g, p, n, persistent=True)
    assert np.array_equal(h1, h2) and np.array_equal(a1, a2)
    # the persistent form fills the same events in another order
    assert np.array_equal(h1, h3) and np.array_equal(a1, a3)
    # two halves (event ids continue) merge exactly into the whole
    half = n // 2
    _, b1 = _pass(g, p, half, 0)
    _, b2 = _pass(g, p, n - half, half)
    assert np.array_equal(sharding.add_fixed(b1, b2), a1)
    assert np.array_equal(sharding.add_fixed(b2, b1), a1)
    # the double histograms are the fixed-point sums converted once
    assert np.array_equal(g.hist_fixed_to_double(p, a1), h1)
    # and agree with a plain float64 sum of the same weights
    k_w, k_w2 = g.hist_fixed_scales(p)
    w = a1.reshape(-1, 5)
    entries = w[:, 4].astype(np.float64)
    assert np.array_equal(entries, h1.reshape(-1, 3)[:, 2])
    assert entries.sum() > 3 * n  # most events fill most observables
    assert 30 < k_w < 62 and 0 < k_w2 < k_w


def _host_bins(x, h):
    """The FP64 bin formula (underflow 0, overflow 101, -1 undefined)."""
    if h < 4:
        ok = x > 0
        v, lo, hi = np.log10(np.where(ok, x, 1.0)), -4.3, -0.3
    else:
        ok = np.ones_like(x, dtype=bool)
        v, lo, hi = np.maximum(np.nan_to_num(x, nan=0.0, posinf=np.inf, neginf=0.0), 0.0), 0.0, (0.5 if h < 6 else 0.4)
    f = (v - lo) / (hi - lo) * 100
    b = np.where(f < 0, 0, np.where(f >= 100, 101, 1 + np.floor(np.clip(f, 0, 99.999999)).astype(int)))
    return np.where(ok, b, -1)


def test_bins_near_edges(g):
    """Values placed just off every bin edge (1e-5 bins: decided by the FP64
    formula; 3e-4 and 5e-4 bins: by the FP32 position) and the special
    values (zero, negative, NaN, above the range) land in the FP64 formula's
    bins; signed weights sum exactly."""
    import torch
    offsets = np.array([-5e-4, -3e-4, -1e-5, 1e-5, 3e-4, 5e-4])
    pos = (np.arange(1, 100)[:, None] + offsets[None, :]).ravel()
    special = np.array([0.0, -0.0, -1e-3, np.nan, 1e3, 0.25])
    n = len(pos) + len(special)
    p = g.make_params(seed=3)
    ws = g.Workspace(n, 128)
    sc = ws.scalars()
    sc["status"].fill_(g.DONE)
    sc["valid"].zero_()
    rng = np.random.default_rng(2)
    w = rng.uniform(-2.0, 2.0, n)  # negative weights too: the fixed-point sums are signed
    sc["weight"].copy_(torch.from_numpy(w))
    obs = np.empty((g.N_OBS, n))
    for h in range(g.N_OBS):
        if h < 4:
            x = 10.0 ** (pos / 25.0 - 4.3)
        else:
            x = pos / (200.0 if h < 6 else 250.0)
        obs[h] = np.concatenate([x, special])
    ws.obs().copy_(torch.from_numpy(obs))
    hist = torch.zeros(g.HIST_DOUBLES, dtype=torch.float64, device="cuda")
    g.histograms(p, ws, hist)
    torch.cuda.synchronize()
    hh = hist.cpu().numpy().reshape(g.N_OBS, g.HIST_ROW, 3)
    # the exact expectation: every fill w 2^k_w (and w^2 2^k_w2) rounded to
    # an integer (nearest, ties to even), summed exactly, converted once
    k_w, k_w2 = g.hist_fixed_scales(p)
    q1 = [int(v) for v in np.rint(w * 2.0 ** k_w)]
    q2 = [int(v) for v in np.rint((w * w) * 2.0 ** k_w2)]
    for h in range(g.N_OBS):
        b = _host_bins(obs[h], h)
        ok = b >= 0
        assert np.array_equal(hh[h, :, 2], np.bincount(b[ok], minlength=g.HIST_ROW).astype(float)), h
        s1 = [0] * g.HIST_ROW
        s2 = [0] * g.HIST_ROW
        for i in np.nonzero(ok)[0]:
            s1[b[i]] += q1[i]
            s2[b[i]] += q2[i]
        want1 = np.array([math.ldexp(float(v), -k_w) for v in s1])
        want2 = np.array([math.ldexp(float(v), -k_w2) for v in s2])
        assert np.array_equal(hh[h, :, 0], want1), (h, np.nonzero(hh[h, :, 0] != want1)[0][:5])
        assert np.array_equal(hh[h, :, 1], want2), h
        np.testing.assert_allclose(hh[h, :, 0], np.bincount(b[ok], weights=w[ok], minlength=g.HIST_ROW),
                                   rtol=1e-9, atol=64 * 2.0 ** -k_w)
