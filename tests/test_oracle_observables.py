"""Oracle pins for the observables (Sec. 3.1): Durham jet resolutions against
an independent re-clustering, thrust against exhaustive subset enumeration,
3-parton closed forms, rotation invariance, and the histogram binning.
Planted mistakes must fail.  CPU only."""
import itertools
import math

import numpy as np
import pytest


def _random_event(rng, n, sqrt_s=91.2):
    """n massless momenta with total (sqrt_s, 0, 0, 0): random directions and
    energies, boosted to rest and rescaled (RAMBO-like, built in the test)."""
    while True:
        q = rng.normal(size=(n, 3))
        e = np.linalg.norm(q, axis=1) * rng.uniform(0.2, 1.0, size=n)[:, None].ravel()
        dirs = q / np.linalg.norm(q, axis=1)[:, None]
        p = np.concatenate([e[:, None], e[:, None] * dirs], axis=1)
        tot = p.sum(axis=0)
        m = math.sqrt(tot[0] ** 2 - tot[1:] @ tot[1:])
        b = -tot[1:] / tot[0]
        g = tot[0] / m
        bp = p[:, 1:] @ b
        b2 = b @ b
        g2 = (g - 1) / b2 if b2 > 0 else 0.0
        pe = g * (p[:, 0] + bp)
        pv = p[:, 1:] + (g2 * bp + g * p[:, 0])[:, None] * b[None, :]
        out = np.concatenate([pe[:, None], pv], axis=1) * (sqrt_s / m)
        if np.all(out[:, 0] > 1e-3):
            return out


def _durham_reference(p, s):
    """Independent E-scheme Durham re-clustering: rebuild the full distance
    matrix each round, merge the closest pair, append the merged jet."""
    jets = [row.copy() for row in p]
    ys = {}
    while len(jets) > 1:
        n = len(jets)
        best = None
        for i in range(n):
            for j in range(i + 1, n):
                a, b = jets[i], jets[j]
                cosij = a[1:] @ b[1:] / (np.linalg.norm(a[1:]) * np.linalg.norm(b[1:]))
                y = 2 * min(a[0] ** 2, b[0] ** 2) * (1 - cosij) / s
                if best is None or y < best[0]:
                    best = (y, i, j)
        y, i, j = best
        ys[n - 1] = y  # y_{n-1, n}
        merged = jets[i] + jets[j]
        jets = [jj for k, jj in enumerate(jets) if k not in (i, j)] + [merged]
    return np.array([ys.get(m, -1.0) for m in (2, 3, 4, 5)])


def _thrust_enumeration(p):
    """T = max over subsets S of 2 |sum_S p| / sum |p|, and rho_H of that
    split."""
    n = len(p)
    mag = np.linalg.norm(p[:, 1:], axis=1).sum()
    best, best_mask = -1.0, None
    for mask in range(1 << (n - 1)):  # the last parton fixed on the '-' side
        sel = np.array([(mask >> i) & 1 for i in range(n)], dtype=bool)
        v = p[sel, 1:].sum(axis=0)
        val = 2 * np.linalg.norm(v)
        if val > best:
            best, best_mask = val, sel
    def m2(q):
        return q[0] ** 2 - q[1:] @ q[1:]
    heavy = max(m2(p[best_mask].sum(axis=0)), m2(p[~best_mask].sum(axis=0)))
    return best / mag, heavy


@pytest.mark.parametrize("n", [3, 4, 5, 7, 9])
def test_durham_matches_reclustering(oracle_mod, n):
    rng = np.random.default_rng(100 + n)
    s = 91.2 ** 2
    for _ in range(40):
        p = _random_event(rng, n)
        ours = oracle_mod.durham(p, s)
        ref = _durham_reference(p, s)
        assert np.allclose(ours, ref, rtol=1e-10, atol=0)
        bad = oracle_mod.durham(p, s, 1 << 6)
        if n >= 3:
            assert not np.allclose(bad, ref, rtol=1e-6, atol=0)


@pytest.mark.parametrize("n", [3, 4, 5, 6, 8, 10, 12])
def test_thrust_matches_enumeration(oracle_mod, n):
    rng = np.random.default_rng(200 + n)
    s = 91.2 ** 2
    fails_nosign = 0
    for _ in range(25 if n < 10 else 6):
        p = _random_event(rng, n)
        t_ref, heavy_ref = _thrust_enumeration(p)
        t = oracle_mod.thrust(p)
        assert t[0] == pytest.approx(t_ref, rel=1e-12)
        assert np.linalg.norm(t[1:]) == pytest.approx(1.0, rel=1e-13)
        shapes = oracle_mod.event_shapes(p, s)
        assert shapes[4] == pytest.approx(1 - t_ref, rel=1e-9, abs=1e-13)
        assert shapes[5] == pytest.approx(heavy_ref / s, rel=1e-9, abs=1e-13)
        if oracle_mod.thrust(p, 1 << 7)[0] < t_ref * (1 - 1e-9):
            fails_nosign += 1
    assert fails_nosign > 0


def test_three_parton_closed_forms(oracle_mod):
    """Three massless partons: T = max x_i (x = 2E/sqrt s), rho_H = 1 - T, and
    y23 = the smallest pair measure."""
    rng = np.random.default_rng(3)
    s = 91.2 ** 2
    for _ in range(200):
        p = _random_event(rng, 3)
        x = 2 * p[:, 0] / 91.2
        out = oracle_mod.event_shapes(p, s)
        assert 1 - out[4] == pytest.approx(x.max(), rel=1e-12)
        assert out[5] == pytest.approx(1 - x.max(), rel=1e-9, abs=1e-13)
        ys = []
        for i, j in itertools.combinations(range(3), 2):
            c = p[i, 1:] @ p[j, 1:] / (np.linalg.norm(p[i, 1:]) * np.linalg.norm(p[j, 1:]))
            ys.append(2 * min(p[i, 0], p[j, 0]) ** 2 * (1 - c) / s)
        assert out[0] == pytest.approx(min(ys), rel=1e-10)
        assert np.all(out[1:4] == -1.0)
    light = oracle_mod.event_shapes(p, s, 1 << 10)
    assert light[5] != pytest.approx(1 - x.max(), rel=1e-6)


def test_three_parton_broadening(oracle_mod):
    """Three massless partons: the thrust axis lies along the hardest one, so
    its hemisphere has no transverse momentum and the other holds two equal
    and opposite p_T; B_T = B_W = p_T / sqrt s = sqrt((1-x1)(1-x2)(1-x3)) / x1
    with x1 the largest x = 2E/sqrt s.  Broadening from |p . n_T| instead of
    |p x n_T| (planted) fails."""
    rng = np.random.default_rng(8)
    s = 91.2 ** 2
    for _ in range(200):
        p = _random_event(rng, 3)
        x = np.sort(2 * p[:, 0] / 91.2)[::-1]
        b = math.sqrt((1 - x[0]) * (1 - x[1]) * (1 - x[2])) / x[0]
        out = oracle_mod.event_shapes(p, s)
        assert out[6] == pytest.approx(b, rel=1e-9, abs=1e-13)
        assert out[7] == pytest.approx(b, rel=1e-9, abs=1e-13)
        bad = oracle_mod.event_shapes(p, s, oracle_mod.MUT_BROAD_DOT)
        assert bad[6] != pytest.approx(b, rel=1e-6)


@pytest.mark.parametrize("n", [4, 6, 9])
def test_broadening_against_enumerated_axis(oracle_mod, n):
    """B_T and B_W from the definition about the axis of the exhaustive
    thrust enumeration: sum |p_i x n| over each hemisphere / (2 sum |p_i|)."""
    rng = np.random.default_rng(20 + n)
    s = 91.2 ** 2
    for _ in range(20):
        p = _random_event(rng, n)
        best, axis = -1.0, None
        for mask in range(1 << (n - 1)):
            sel = np.array([(mask >> i) & 1 for i in range(n)], dtype=bool)
            v = p[sel, 1:].sum(axis=0) - p[~sel, 1:].sum(axis=0)
            if np.linalg.norm(v) > best:
                best, axis = np.linalg.norm(v), v / np.linalg.norm(v)
        pt = np.linalg.norm(np.cross(p[:, 1:], axis), axis=1)
        side = p[:, 1:] @ axis >= 0
        denom = 2 * np.linalg.norm(p[:, 1:], axis=1).sum()
        bp, bm = pt[side].sum() / denom, pt[~side].sum() / denom
        out = oracle_mod.event_shapes(p, s)
        assert out[6] == pytest.approx(bp + bm, rel=1e-9)
        assert out[7] == pytest.approx(max(bp, bm), rel=1e-9)


def test_two_partons(oracle_mod):
    p = np.array([[45.6, 0, 0, 45.6], [45.6, 0, 0, -45.6]])
    out = oracle_mod.event_shapes(p, 91.2 ** 2)
    assert out[6] == 0.0 and out[7] == 0.0
    assert out[4] == 0.0 and out[5] == 0.0
    assert np.all(out[:4] == -1.0)


def test_rotation_invariance(oracle_mod):
    rng = np.random.default_rng(4)
    s = 91.2 ** 2
    for n in (4, 6, 9):
        p = _random_event(rng, n)
        a = rng.normal(size=(3, 3))
        q, _ = np.linalg.qr(a)
        pr = p.copy()
        pr[:, 1:] = p[:, 1:] @ q.T
        assert np.allclose(oracle_mod.event_shapes(p, s), oracle_mod.event_shapes(pr, s), rtol=1e-9, atol=1e-14)


def test_histograms_are_the_binned_observables(oracle_mod):
    """The run's histogram equals re-binning the per-event observables with
    the stated edges (log10 y on [-4.3, -0.3], 1-T and rho_H on [0, 0.5],
    B_T and B_W on [0, 0.4])."""
    p = oracle_mod.make_params(seed=6)
    r = oracle_mod.run(p, 0, 3000, threads=oracle_mod.threads_available())
    obs, ev, hist = r["obs"], r["events"], r["hist"]
    w = ev["weight"]
    for h in range(oracle_mod.N_OBS):
        x = obs[:, h]
        ok = (ev["status"] == oracle_mod.DONE)
        if h < 4:
            ok &= x > 0
            v, lo, hi = np.log10(np.where(ok, x, 1.0)), -4.3, -0.3
        else:
            v, lo, hi = np.maximum(x, 0.0), 0.0, (0.5 if h < 6 else 0.4)   # non-negative by definition
        f = (v - lo) / (hi - lo) * 100
        b = np.where(f < 0, 0, np.where(f >= 100, 101, 1 + np.floor(np.clip(f, 0, 99.999999)).astype(int)))
        sw = np.bincount(b[ok], weights=w[ok], minlength=102)
        n = np.bincount(b[ok], minlength=102)
        assert np.allclose(hist[h, :, 0], sw, rtol=1e-12)
        assert np.array_equal(hist[h, :, 2], n.astype(float))
    # y23 is defined for every event with >= 3 partons
    assert hist[0, :, 2].sum() == np.sum(ev["n_partons"] >= 3)


def test_two_parton_shapes_bin_as_zero(oracle_mod):
    """Events without an emission (the cutoff just below s/4 leaves no phase
    space) have 1-T = rho_H = 0 up to FP64 rounding in either direction; the
    histogram puts every one of them in the first bin of [0, 0.5], never in
    the underflow, whatever the sign of the rounding."""
    s = 91.2 ** 2
    p = oracle_mod.make_params(seed=8, t_cutoff=0.2499 * s)
    r = oracle_mod.run(p, 0, 2000, threads=1)
    assert np.all(r["events"]["n_partons"] == 2)
    obs, hist = r["obs"], r["hist"]
    assert np.all(np.abs(obs[:, 4:6]) < 1e-12)
    for h in (4, 5, 6, 7):
        assert hist[h, 0, 2] == 0.0 and hist[h, 1, 2] == 2000.0
