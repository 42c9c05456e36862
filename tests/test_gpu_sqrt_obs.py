"""The observables' square root on the GPU (the FP32 reciprocal square root
refined by one Newton step in FP64): within 1.5e-13 relative of the
correctly rounded square root over a million inputs from 2^-120 to 2^121
and over the range the event shapes take (squared lengths of momenta up to
(200 GeV)^2), and the library's value outside that range."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2403_08692_gb300 as g
    g.load()
    return g


def test_relative_error_bound(g):
    rng = np.random.default_rng(11)
    x = np.concatenate([np.exp2(rng.uniform(-120.0, 121.0, 600_000)),   # the refined range, log-uniform
                        rng.uniform(0.0, 4.0e4, 300_000),                 # |p|^2 of partons up to 200 GeV
                        rng.uniform(1e-8, 1e-2, 100_000)])                # soft and collinear |p x n|^2
    x = x[(x >= 2.0 ** -120) & (x < 2.0 ** 121)]
    y = g.sqrt_obs_device(torch.from_numpy(x).cuda()).cpu().numpy()
    want = np.sqrt(x)  # correctly rounded
    rel = np.abs(y - want) / want
    assert rel.max() <= 1.5e-13, rel.max()
    # the refinement does the work: a plain FP32 square root is 1e-7 off
    assert np.median(rel) < 3e-14


def test_outside_the_refined_range(g):
    x = np.array([0.0, -0.0, -4.0, np.inf, np.nan, 5e-324, 1e-300, 2.0 ** -121, 2.0 ** 122, 1e300])
    y = g.sqrt_obs_device(torch.from_numpy(x).cuda()).cpu().numpy()
    with np.errstate(invalid="ignore"):
        want = np.sqrt(x)  # NaN for the negative input, as on the GPU
    same = (y == want) | (np.isnan(y) & np.isnan(want))
    assert np.all(same), (y, want)
    assert np.signbit(y[1])  # sqrt(-0) = -0
