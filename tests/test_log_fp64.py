"""The shower's FP64 logarithm (table-driven, after Tang, ACM TOMS 16 (1990)
378), host build: error below one ulp against a 50-digit decimal reference on
the inputs the shower feeds it (uniforms in (0, 1) built from two 32-bit
draws, ratios z+/z- from just above 1 up to 1e12, scales t/m_Z^2) and on the
method's hard spots (the table breakpoints' edges, the sqrt(2) split, values
next to 1, powers of two); special inputs follow the library's log."""
import math
from decimal import Decimal, getcontext

import numpy as np
import pytest

getcontext().prec = 50


@pytest.fixture(scope="module")
def g():
    import paper_2403_08692_gb300 as g
    g.load()
    return g


def _ulp_errors(x, y):
    out = []
    for xi, yi in zip(x, y):
        ref = Decimal(float(xi)).ln()
        ulp = math.ulp(float(ref)) if float(ref) != 0.0 else math.ulp(0.0)
        out.append(float(abs(Decimal(float(yi)) - ref) / Decimal(ulp)))
    return np.array(out)


def _inputs():
    rng = np.random.default_rng(20240313)
    hi = rng.integers(0, 2**32, 3000, dtype=np.uint64)
    lo = rng.integers(0, 2**32, 3000, dtype=np.uint64)
    uniforms = ((hi >> 5).astype(np.float64) * 2.0**26 + (lo >> 6).astype(np.float64) + 0.5) * 2.0**-53
    j = np.arange(90, 182, dtype=np.float64)
    edges = np.concatenate([(j + 0.5) / 128, (j - 0.5) / 128, j / 128])
    parts = [
        uniforms,
        1.0 + np.exp(rng.uniform(np.log(1e-12), np.log(1e12), 3000)),  # z+/z- ratios
        np.exp(rng.uniform(-745.0, 709.0, 3000)),                       # the whole normal range
        1.0 + rng.uniform(-2e-2, 2e-2, 3000),                           # around 1
        1.0 + rng.uniform(-1e-9, 1e-9, 500),
        np.concatenate([np.nextafter(edges, 0.0), edges, np.nextafter(edges, 2.0)]),
        np.sqrt(2.0) * np.array([1.0, 1.0 + 2.0**-52, 1.0 - 2.0**-53]),
        np.ldexp(1.0, np.arange(-1022, 1024)),
        np.array([np.nextafter(1.0, 0.0), np.nextafter(1.0, 2.0), 2.2250738585072014e-308, 1.7976931348623157e308]),
    ]
    return np.concatenate(parts)


def test_below_one_ulp(g):
    x = _inputs()
    y = g.log_fp64_host(x)
    err = _ulp_errors(x, y)
    worst = int(np.argmax(err))
    assert err.max() < 1.0, (x[worst], y[worst], err.max())
    # and nearly always the correctly rounded value
    assert (err <= 0.5).mean() > 0.97


def test_exact_values(g):
    y = g.log_fp64_host(np.array([1.0, 2.0, 0.5, 4.0]))
    assert y[0] == 0.0
    assert y[1] == math.log(2.0) and y[2] == -math.log(2.0) and y[3] == 2.0 * math.log(2.0)


def test_special_inputs(g):
    y = g.log_fp64_host(np.array([0.0, -1.0, np.inf, np.nan, 5e-324, 1e-310]))
    assert y[0] == -np.inf
    assert np.isnan(y[1]) and np.isnan(y[3])
    assert y[2] == np.inf
    assert abs(y[4] - math.log(5e-324)) <= 1e-13 * abs(math.log(5e-324))
    assert abs(y[5] - math.log(1e-310)) <= 1e-13 * abs(math.log(1e-310))


def test_bad_arguments(g):
    lib = g.gaps.load_probe()
    assert lib.gaps_log_fp64_host(None, None, -1) != 0
    assert lib.gaps_log_fp64_host(None, None, 5) != 0
    assert lib.gaps_log_fp64_host(None, None, 0) == 0


def test_f32_from_f64_is_round_to_nearest_even(g):
    """The kernels' integer double -> float conversion equals numpy's (IEEE
    round to nearest even) on random doubles of every magnitude, on ties
    (the dropped 29 bits exactly one half), on values that round up into
    the next binade or to infinity, and on the special values."""
    rng = np.random.default_rng(11)
    x = np.concatenate([
        rng.standard_normal(100_000) * np.exp(rng.uniform(-100.0, 100.0, 100_000)),
        np.exp(rng.uniform(-745.0, 709.0, 20_000)) * rng.choice([-1.0, 1.0], 20_000),
    ])
    f = rng.standard_normal(20_000).astype(np.float32).astype(np.float64)
    ties = np.abs(f) * (1.0 + 2.0**-24)                         # exactly half an FP32 ulp above
    ties2 = np.nextafter(np.abs(f).astype(np.float32), np.float32(np.inf)).astype(np.float64) * (1.0 - 2.0**-25)
    edge = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 5e-324, 1e-40, 1.1754942e-38, 1.1754944e-38,
                     3.4028234e38, 3.4028235e38, 3.40282357e38, 1e39, -1e39, 2.0**-126, 2.0**-127,
                     np.nextafter(2.0, 0.0), 1.0 - 2.0**-25, 1.0 - 2.0**-26])
    x = np.concatenate([x, ties, ties2, edge])
    with np.errstate(over="ignore"):
        want = x.astype(np.float32)
    got = g.f32_from_f64_host(x)
    assert np.array_equal(got.view(np.uint32)[~np.isnan(want)], want.view(np.uint32)[~np.isnan(want)])
    assert np.isnan(got[np.isnan(want)]).all()
