"""gaps_event_shapes_noalloc: the observables stage for callers that cannot
allocate device memory (code confined to another framework's memory pool,
plug-ins whose host forbids allocation calls, processes that hand out all
device memory up front).  Its working arrays live in a fixed device array
inside the library.  Checked through the C ABI against gaps_observables on
the same showered events, on two calls in a row.  Requires a GB300; kept in
its own file, collected last."""
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


def test_noalloc_matches_observables_twice(g):
    import torch
    n, cap = 30011, 128  # a ragged batch size
    p = g.make_params(seed=77)
    ws = g.Workspace(n, cap)
    g.generate_me(p, ws)
    g.shower(p, ws)
    g.observables(p, ws)
    ref = ws.obs().clone()
    mom = ws.momenta()
    sc = ws.scalars()
    torch.cuda.synchronize()
    ref_np = ref.cpu().numpy()
    for _ in range(2):
        out = torch.full((g.N_OBS, n), 123.0, dtype=torch.float64, device="cuda")
        g.event_shapes_noalloc(mom["px"], mom["py"], mom["pz"], mom["e"], sc["n_partons"], sc["status"],
                               n, cap, p.sqrt_s, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.abs(got - ref_np) <= H.OBS_REL * np.abs(ref_np) + H.OBS_ABS)
    # the events have real structure: most have y23, some reach y56
    assert np.mean(ref_np[0] > 0) > 0.7 and np.any(ref_np[3] > 0)


def test_noalloc_rejects_oversized_batches(g):
    import torch
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    ints = torch.zeros(8, dtype=torch.int32, device="cuda")
    with pytest.raises(g.GapsError) as e:
        g.event_shapes_noalloc(dummy, dummy, dummy, dummy, ints, ints, g.gaps.NOALLOC_MAX_EVENTS + 1, 128, 91.2,
                               dummy)
    assert e.value.code == -1
