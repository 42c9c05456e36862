"""The C-ABI library builds, loads and exports every symbol include/gaps.h
declares; host-only calls (sizing, layout, parameter checks) behave.  No GPU
needed, no compute calls."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions(header=None):
    names = []
    for hdr in os.listdir(os.path.join(ROOT, "include")):
        if not hdr.endswith(".h") or (header is not None and hdr != header):
            continue
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s+\**(gaps_[a-z0-9_]+)\s*\(", text, re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def g():
    import paper_2403_08692_gb300 as g
    g.load()
    return g


def test_every_declared_symbol_is_exported(g):
    """gaps.h: the product library libgaps.so; gaps_probe.h: the measurement
    and test library libgaps_probe.so, whose symbols the product library
    does not carry."""
    names = _declared_functions("gaps.h")
    assert len(names) >= 14, names
    lib = C.CDLL(g.gaps.library_path())
    for n in names:
        assert hasattr(lib, n), n
    # and the binding knows every one of them, with the same names
    assert set(names) <= set(g.gaps.SIGNATURES), set(names) - set(g.gaps.SIGNATURES)
    probe_names = _declared_functions("gaps_probe.h")
    assert "gaps_probe_fp64_rates" in probe_names and "gaps_log_fp64_host" in probe_names
    probe = C.CDLL(g.gaps.probe_library_path())
    for n in probe_names:
        assert hasattr(probe, n), n
        assert not hasattr(lib, n), n
    assert set(probe_names) <= set(g.gaps.PROBE_SIGNATURES)
    assert not set(names) & set(probe_names)


def test_header_constants_match_binding(g):
    text = open(os.path.join(ROOT, "include", "gaps.h")).read()
    assert f"GAPS_N_OBS = {g.N_OBS}, GAPS_N_BINS = 100, GAPS_HIST_ROW = 102" in text
    assert g.N_OBS == 8 and g.HIST_DOUBLES == 8 * 102 * 3
    assert C.sizeof(g.gaps.Params) == 48
    assert C.sizeof(g.gaps.Batch) == 32
    assert C.sizeof(g.gaps.Stats) == 15 * 8


def test_workspace_layout(g):
    for n, cap in ((0, 4), (1, 128), (10000, 128), (12345, 50), (1000000, 255)):
        L = g.layout(n, cap)
        total = g.workspace_bytes(n, cap)
        assert total == L.total_bytes
        offs = [getattr(L, f) for f, _ in L._fields_ if f != "total_bytes"]
        assert all(o % 256 == 0 for o in offs)
        assert offs == sorted(offs)
        if n > 0:
            assert len(set(offs)) == len(offs)
        assert L.py - L.px >= 8 * n * cap and L.flav - L.e >= 8 * n * cap
        assert L.obs + 48 * n <= L.counters
    assert g.workspace_bytes(10, 3) == 0
    assert g.workspace_bytes(10, 256) == 0
    assert g.workspace_bytes(-1, 128) == 0
    with pytest.raises(g.GapsError):
        g.layout(10, 300)


def test_param_checks(g):
    assert g.check_params(g.make_params()) == 0
    assert g.check_params(g.make_params(t_cutoff=0.0)) == -1
    assert g.check_params(g.make_params(t_cutoff=91.2 ** 2 / 4)) == -1
    assert g.check_params(g.make_params(n_flavours=6)) == -1
    assert g.check_params(g.make_params(max_steps=0)) == -1
    assert g.check_params(g.make_params(t_cutoff=1e-4)) == -1
    assert g.check_params(g.make_params(trial_mode=g.TRIALS_PER_DIPOLE)) == 0
    p = g.make_params()
    p.trial_mode = 2
    assert g.check_params(p) == -1


def test_status_strings(g):
    L = g.load()
    assert L.gaps_strerror(0) == b"ok"
    assert b"invalid" in L.gaps_strerror(-1)
    assert L.gaps_version() >= 100


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2403_08692_gb300 import gaps as G
    monkeypatch.setattr(G, "_lib", None)
    monkeypatch.setattr(G._build, "LIB", str(tmp_path / "nope.so"))
    with pytest.raises(RuntimeError):
        G.load(build_if_missing=False)


def test_pool_calls_reject_bad_arguments_before_any_device_work(g):
    """gaps_pool_finish_jobs checks its job list (slots in range and distinct,
    ranges inside the pool and disjoint, array pointers) and gaps_pool_slice /
    gaps_pool_cycles their shared parameters on the host, before any device
    call: a bad list or bad parameters give GAPS_ERR_INVALID here, without a
    GPU (the workspace pointer is never dereferenced)."""
    L = g.load()
    n, cap = 1000, 128
    batch = g.gaps.Batch(C.c_void_p(1 << 20), n, cap, 0, 0, 0)  # aligned, never touched
    hist = C.c_void_p(1 << 21)

    def finish(slots, begins, counts, k=None):
        S = (C.c_int32 * max(1, len(slots)))(*slots)
        B = (C.c_int64 * max(1, len(begins)))(*begins)
        N = (C.c_int64 * max(1, len(counts)))(*counts)
        k = len(slots) if k is None else k
        return L.gaps_pool_finish_jobs(C.cast(S, C.c_void_p), C.cast(B, C.c_void_p), C.cast(N, C.c_void_p), k,
                                       C.byref(batch), hist, None)

    INVALID = -1
    assert finish([0, 0], [0, 100], [10, 10]) == INVALID            # one slot twice
    assert finish([0, 1], [0, 5], [10, 10]) == INVALID              # overlapping ranges
    assert finish([0], [995], [10]) == INVALID                      # past the pool's end
    assert finish([0], [-1], [10]) == INVALID                       # negative begin
    assert finish([0], [0], [-3]) == INVALID                        # negative count
    assert finish([g.MAX_JOBS], [0], [10]) == INVALID               # slot out of range
    assert finish([0], [0], [10], k=g.MAX_JOBS + 1) == INVALID      # too many jobs
    assert L.gaps_pool_finish_jobs(None, None, None, 1, C.byref(batch), hist, None) == INVALID
    assert finish([], [], [], k=0) == 0                             # nothing to do
    bad = g.make_params(t_cutoff=0.0)
    assert L.gaps_pool_slice(C.byref(batch), 0, 8, 10, None, C.byref(bad), None) == INVALID
    assert L.gaps_pool_cycles(C.byref(batch), 0, 8, 10, C.byref(bad), None) == INVALID
