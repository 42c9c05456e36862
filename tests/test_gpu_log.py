"""The shower's FP64 logarithm on the GPU: bitwise the host build (whose
accuracy test_log_fp64 pins below one ulp), and within one ulp of the CUDA
library's log, over a million inputs spanning the shower's uses."""
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


def test_device_equals_host(g):
    rng = np.random.default_rng(7)
    x = np.concatenate([rng.random(400_000), 1.0 + np.exp(rng.uniform(-28.0, 28.0, 300_000)),
                        np.exp(rng.uniform(-745.0, 709.0, 300_000)), 1.0 + rng.uniform(-0.02, 0.02, 100_000)])
    x = x[x > 2.3e-308]
    host = g.log_fp64_host(x)
    xd = torch.from_numpy(x).cuda()
    dev = g.log_fp64_device(xd)
    torch.cuda.synchronize()
    assert np.array_equal(dev.cpu().numpy(), host)
    lib = torch.log(xd).cpu().numpy()
    ulps = np.abs(host - lib) / np.spacing(np.abs(lib))
    assert ulps.max() <= 1.0


def test_special_inputs_device(g):
    x = torch.tensor([0.0, -1.0, float("inf"), float("nan"), 5e-324, 1.0], dtype=torch.float64, device="cuda")
    y = g.log_fp64_device(x).cpu().numpy()
    assert y[0] == -np.inf and np.isnan(y[1]) and y[2] == np.inf and np.isnan(y[3]) and y[5] == 0.0
    assert abs(y[4] - np.log(5e-324)) <= 1e-13 * abs(np.log(5e-324))
