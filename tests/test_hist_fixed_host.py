"""The conversion of the exact fixed-point histogram sums (signed 128-bit
integers in units of 2^-k) to doubles, through the library's host entry
gaps_hist_fixed_to_double (the device finalisation runs the same code):
each cell converts with one rounding to nearest even, checked against
Python's exact integer-to-float conversion on small negative sums (which
must not cancel against 2^64), sums beyond 64 bits, and exact ties at and
above 2^64.  No GPU needed."""
import math

import numpy as np
import pytest


@pytest.fixture(scope="module")
def g():
    import paper_2403_08692_gb300 as g
    g.load()
    return g


def _words(v):
    """Two's-complement (low, high) words of a signed 128-bit integer."""
    u = v % (1 << 128)
    return u & ((1 << 64) - 1), u >> 64


def test_conversion_rounds_once(g):
    p = g.make_params(seed=1)
    k_w, k_w2 = g.hist_fixed_scales(p)
    rng = np.random.default_rng(3)
    values = [0, 1, -1, -12345, 12345, (1 << 53) + 1, -((1 << 53) + 1), (1 << 64) - 1, -((1 << 64) - 1),
              1 << 64, -(1 << 64), (1 << 64) + 1, -((1 << 64) + 1),
              # exact ties above 2^64: 53 significant bits, then a one and zeros
              ((1 << 53) + 1) * (1 << 13) + (1 << 12), -(((1 << 53) + 1) * (1 << 13) + (1 << 12)),
              ((1 << 53) + 2) * (1 << 13) + (1 << 12),
              # one above a tie, the extra bit far below the rounding position
              ((1 << 53) + 2) * (1 << 70) + (1 << 69) + 1, -(((1 << 53) + 2) * (1 << 70) + (1 << 69) + 1)]
    values += [int(x) for x in rng.integers(-(1 << 62), 1 << 62, 40)]
    values += [int(a) * (1 << 40) + int(b) for a, b in zip(rng.integers(-(1 << 60), 1 << 60, 40),
                                                          rng.integers(0, 1 << 40, 40))]
    cells = g.N_OBS * g.HIST_ROW
    assert len(values) <= cells
    acc = np.zeros(g.HIST_FIXED_WORDS, dtype=np.uint64)
    for c, v in enumerate(values):
        lo, hi = _words(v)
        acc[5 * c + 0] = lo
        acc[5 * c + 1] = hi
        acc[5 * c + 2] = lo  # sum of w^2 words: the same value, in units of 2^-k_w2
        acc[5 * c + 3] = hi
        acc[5 * c + 4] = 1
    out = g.hist_fixed_to_double(p, acc).reshape(-1, 3)
    for c, v in enumerate(values):
        assert out[c, 0] == math.ldexp(float(v), -k_w), (c, v, out[c, 0])
        assert out[c, 1] == math.ldexp(float(v), -k_w2), (c, v)
        assert out[c, 2] == 1.0


def test_rank_merge_is_exact_for_signed_sums(g):
    """sharding.add_fixed (the ranks' merge) adds the words as 128-bit
    two's-complement integers, so signed partial sums combine exactly and in
    any order; the merged set converts like the exact sum."""
    from paper_2403_08692_gb300 import sharding
    p = g.make_params(seed=1)
    k_w, _ = g.hist_fixed_scales(p)
    rng = np.random.default_rng(9)
    cells = g.N_OBS * g.HIST_ROW
    a_vals = [int(x) * (1 << 30) + int(y) for x, y in zip(rng.integers(-(1 << 62), 1 << 62, cells),
                                                          rng.integers(0, 1 << 30, cells))]
    b_vals = [-v + int(d) for v, d in zip(a_vals, rng.integers(-1000, 1000, cells))]  # near cancellation
    acc_a = np.zeros(g.HIST_FIXED_WORDS, dtype=np.uint64)
    acc_b = np.zeros(g.HIST_FIXED_WORDS, dtype=np.uint64)
    for c in range(cells):
        for acc, v in ((acc_a, a_vals[c]), (acc_b, b_vals[c])):
            lo, hi = _words(v)
            acc[5 * c], acc[5 * c + 1], acc[5 * c + 2], acc[5 * c + 3], acc[5 * c + 4] = lo, hi, lo, hi, 1
    ab = sharding.add_fixed(acc_a, acc_b)
    assert np.array_equal(ab, sharding.add_fixed(acc_b, acc_a))
    out = g.hist_fixed_to_double(p, ab).reshape(-1, 3)
    for c in range(cells):
        lo, hi = _words(a_vals[c] + b_vals[c])
        assert int(ab[5 * c]) == lo and int(ab[5 * c + 1]) == hi and int(ab[5 * c + 4]) == 2
        assert out[c, 0] == math.ldexp(float(a_vals[c] + b_vals[c]), -k_w)
