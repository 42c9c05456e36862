"""gaps_event_shapes_noalloc: the observables stage for callers that cannot
allocate device memory (code confined to another framework's memory pool,
plug-ins whose host forbids allocation calls, processes that hand out all
device memory up front).  Its working arrays live in a fixed device array
inside the library.  Checked through the C ABI against gaps_observables on
the same events, on two calls in a row: showered events at capacity 128, and
synthetic events at capacity 24 (multiplicity classes above the capacity are
skipped) with a mix of statuses and parton counts outside 2..capacity.
Requires a GB300; kept in its own file, collected last."""
import ctypes as C

import numpy as np
import pytest

from tests import gpu_harness as H
from tests import synthetic_events as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2403_08692_gb300 as g
    g.load()
    return g


def _call_twice_and_compare(g, mom, sc, n, cap, sqrt_s, ref_np):
    import torch
    outs = []
    for _ in range(2):
        out = torch.full((g.N_OBS, n), 123.0, dtype=torch.float64, device="cuda")
        g.event_shapes_noalloc(mom["px"], mom["py"], mom["pz"], mom["e"], sc["n_partons"], sc["status"],
                               n, cap, sqrt_s, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.abs(got - ref_np) <= H.OBS_REL * np.abs(ref_np) + H.OBS_ABS)
        outs.append(got)
    return outs


def test_noalloc_set_up_call(g):
    """n_events = 0 runs only the per-device set-up and needs no arrays."""
    g.event_shapes_noalloc(None, None, None, None, None, None, 0, 128, 91.2, None)


def test_noalloc_matches_observables_twice(g):
    import torch
    n, cap = 30011, 128  # a ragged batch size
    p = g.make_params(seed=77)
    ws = g.Workspace(n, cap)
    g.generate_me(p, ws)
    g.shower(p, ws)
    g.observables(p, ws)
    ref = ws.obs().clone()
    torch.cuda.synchronize()
    ref_np = ref.cpu().numpy()
    _call_twice_and_compare(g, ws.momenta(), ws.scalars(), n, cap, p.sqrt_s, ref_np)
    # the events have real structure: most have y23, some reach y56
    assert np.mean(ref_np[0] > 0) > 0.7 and np.any(ref_np[3] > 0)


def test_noalloc_small_capacity_mixed_statuses(g):
    """Capacity 24 (only the 16- and 32-parton classes run, the latter on
    events of 17..24 partons), some events not finished, and finished events
    whose parton count is outside 2..24 (above the capacity, 255, negative,
    one): those get -1 observables and no slot past the capacity is read."""
    import torch
    cap, n, sqrt_s = 24, 3001, 91.2
    rng = np.random.default_rng(11)
    counts = rng.integers(2, cap + 1, size=n)
    arrays, npart = S.pack_slot_major(S.events_with_multiplicities(12, counts, sqrt_s), cap)
    status = np.full(n, g.DONE, dtype=np.int32)
    status[rng.random(n) < 0.1] = g.OVERFLOW
    status[rng.random(n) < 0.05] = g.STEP_LIMIT
    bad = rng.choice(np.nonzero(status == g.DONE)[0], size=40, replace=False)
    npart[bad[:10]] = cap + 1
    npart[bad[10:20]] = 255
    npart[bad[20:30]] = -7
    npart[bad[30:]] = 1
    ws = g.Workspace(n, cap)
    mom = ws.momenta()
    for c in ("e", "px", "py", "pz"):
        mom[c].copy_(torch.from_numpy(arrays[c]))
    sc = ws.scalars()
    sc["n_partons"].copy_(torch.from_numpy(npart))
    sc["status"].copy_(torch.from_numpy(status))
    g.observables(g.make_params(sqrt_s=sqrt_s), ws)
    ref_np = ws.obs().cpu().numpy()
    counters = ws.view("counters", torch.int64, (32,)).cpu().numpy()
    assert counters[8] == len(bad)
    outs = _call_twice_and_compare(g, mom, sc, n, cap, sqrt_s, ref_np)
    for got in outs:
        assert np.all(got[:, bad] == -1.0)
        assert np.all(got[:, status != g.DONE] == -1.0)
        good = (status == g.DONE) & (npart >= 2) & (npart <= cap)
        assert np.all(got[4, good] >= -1e-15)  # 1-T defined for every good event
    assert np.any((counts > 16) & (status == g.DONE))


def test_noalloc_rejects_bad_arguments(g):
    """Through the C ABI: a batch above the fixed maximum, a capacity below 4,
    a non-positive sqrt(s) and a null array are rejected before any work."""
    import torch
    L = g.load()
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    ints = torch.zeros(8, dtype=torch.int32, device="cuda")
    d, i = C.c_void_p(dummy.data_ptr()), C.c_void_p(ints.data_ptr())
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert L.gaps_event_shapes_noalloc(d, d, d, d, i, i, g.gaps.NOALLOC_MAX_EVENTS + 1, 128, 91.2, d, stream) == -1
    assert L.gaps_event_shapes_noalloc(d, d, d, d, i, i, 2, 3, 91.2, d, stream) == -1
    assert L.gaps_event_shapes_noalloc(d, d, d, d, i, i, 2, 128, 0.0, d, stream) == -1
    assert L.gaps_event_shapes_noalloc(d, d, d, d, i, None, 2, 128, 91.2, d, stream) == -1
    with pytest.raises(ValueError):
        g.event_shapes_noalloc(dummy, dummy, dummy, dummy, ints, ints, 100, 128, 91.2, dummy)
