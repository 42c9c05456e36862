"""Python binding of the C ABI in include/gaps.h (ctypes, argument marshalling
only).  Every step of the hot path runs in the CUDA library; PyTorch supplies
the device workspace and the stream.  There is no CPU fallback: loading the
library fails loudly if it has not been built or no GPU is present.
"""
import ctypes as C
import os

from . import build as _build

GAPS_OK, GAPS_ERR_INVALID, GAPS_ERR_CUDA, GAPS_ERR_STEP_LIMIT, GAPS_ERR_NO_DEVICE = 0, -1, -2, -3, -4
ACTIVE, DONE, OVERFLOW, STEP_LIMIT, PENDING = 0, 1, 2, 3, 4
SHOWER_PLAIN, SHOWER_PERSISTENT = 0, 1
N_OBS, N_BINS, HIST_ROW = 8, 100, 102
HIST_DOUBLES = N_OBS * HIST_ROW * 3
HIST_FIXED_WORDS = N_OBS * HIST_ROW * 5


class Params(C.Structure):
    _fields_ = [("sqrt_s", C.c_double), ("alphas_mz", C.c_double), ("t_cutoff", C.c_double),
                ("seed", C.c_uint64), ("n_flavours", C.c_int32), ("fixed_alphas", C.c_int32),
                ("max_steps", C.c_int32), ("trial_mode", C.c_int32)]


LAYOUT_SOA, LAYOUT_TILE8, LAYOUT_TILE32 = 0, 1, 2
LAYOUT_NAMES = {LAYOUT_SOA: "structure of arrays", LAYOUT_TILE8: "tiles of 8 events", LAYOUT_TILE32: "tiles of 32 events"}
_TILE = {LAYOUT_TILE8: 8, LAYOUT_TILE32: 32}


class PersistentConfig(C.Structure):
    _fields_ = [("block_threads", C.c_int32), ("compact_period", C.c_int32), ("blocks_per_sm", C.c_int32),
                ("layout", C.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def persistent_config(cfg):
    """A PersistentConfig from a PersistentConfig, a dict of its fields or None."""
    if isinstance(cfg, dict):
        return PersistentConfig(int(cfg["block_threads"]), int(cfg["compact_period"]),
                                int(cfg.get("blocks_per_sm", 0)), int(cfg.get("layout", LAYOUT_SOA)))
    return cfg


class Batch(C.Structure):
    _fields_ = [("workspace", C.c_void_p), ("n_events", C.c_int64), ("capacity", C.c_int32),
                ("first_event", C.c_uint32), ("layout", C.c_int32), ("reserved", C.c_int32)]


_LAYOUT_FIELDS = ["px", "py", "pz", "e", "flav", "col", "acol", "link", "dip", "dq2", "dzp", "dinv", "t", "lnt",
                  "weight", "hash",
                  "n_partons", "status", "n_steps", "n_emissions", "n_winners", "n_trials",
                  "n_dipoles", "next_colour", "me_flavour", "valid", "obs", "buckets", "order", "active", "tasks",
                  "counters",
                  "hist", "hist_fixed",
                  "stats", "jobs", "job_begin", "job_of", "job_done", "finish", "total_bytes"]


MAX_JOBS = 1024


class Job(C.Structure):
    _fields_ = [("params", Params), ("n_events", C.c_int64), ("first_event", C.c_uint32), ("reserved", C.c_int32)]


class Layout(C.Structure):
    _fields_ = [(f, C.c_int64) for f in _LAYOUT_FIELDS]


class Stats(C.Structure):
    _fields_ = [("n_events", C.c_int64), ("n_done", C.c_int64), ("n_overflow", C.c_int64),
                ("n_step_limit", C.c_int64), ("n_invalid", C.c_int64), ("sum_steps", C.c_int64),
                ("max_steps", C.c_int64), ("sum_trials", C.c_int64), ("sum_winners", C.c_int64),
                ("sum_emissions", C.c_int64), ("sum_partons", C.c_int64), ("sum_dipoles", C.c_int64),
                ("launches", C.c_int64),
                ("sum_weight", C.c_double), ("sum_weight2", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


# Every symbol include/gaps.h declares, with its ctypes signature.
_P = C.POINTER
SIGNATURES = {
    "gaps_workspace_bytes": (C.c_size_t, [C.c_int64, C.c_int32]),
    "gaps_workspace_layout": (C.c_int, [C.c_int64, C.c_int32, _P(Layout)]),
    "gaps_check_params": (C.c_int, [_P(Params)]),
    "gaps_generate_me": (C.c_int, [_P(Params), _P(Batch), C.c_void_p]),
    "gaps_shower": (C.c_int, [_P(Params), _P(Batch), C.c_int, _P(C.c_int64), C.c_void_p]),
    "gaps_shower_timed": (C.c_int, [_P(Params), _P(Batch), C.c_int, _P(C.c_int64), _P(C.c_double),
                                    C.c_void_p]),
    "gaps_set_jobs": (C.c_int, [_P(Job), C.c_int32, _P(Batch), C.c_void_p]),
    "gaps_shower_persistent": (C.c_int, [_P(Params), _P(Batch), _P(PersistentConfig), C.c_void_p]),
    "gaps_autotune_persistent": (C.c_int, [_P(Params), _P(Batch), _P(PersistentConfig), _P(C.c_double),
                                           C.c_void_p]),
    "gaps_shower_step": (C.c_int, [_P(Params), _P(Batch), C.c_void_p]),
    "gaps_validate": (C.c_int, [_P(Params), _P(Batch), C.c_void_p]),
    "gaps_observables": (C.c_int, [_P(Params), _P(Batch), C.c_void_p]),
    "gaps_histograms": (C.c_int, [_P(Params), _P(Batch), C.c_void_p, C.c_void_p]),
    "gaps_reduce_stats": (C.c_int, [_P(Batch), C.c_void_p, C.c_void_p]),
    "gaps_histograms_fixed": (C.c_int, [_P(Params), _P(Batch), C.c_void_p, C.c_void_p]),
    "gaps_hist_fixed_scales": (C.c_int, [_P(Params), _P(C.c_int32), _P(C.c_int32)]),
    "gaps_hist_fixed_to_double": (C.c_int, [_P(Params), C.c_void_p, C.c_void_p]),
    "gaps_run": (C.c_int, [_P(Params), _P(Batch), C.c_int, _P(C.c_double), _P(Stats), C.c_void_p]),
    "gaps_event_shapes_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                            C.c_void_p, C.c_int64, C.c_int32, C.c_double, C.c_void_p,
                                            C.c_void_p]),
    "gaps_pool_reset": (C.c_int, [_P(Batch), C.c_void_p]),
    "gaps_pool_admit": (C.c_int, [_P(Params), C.c_int32, C.c_int64, C.c_int64, C.c_uint32, _P(Batch), C.c_int64,
                                  C.c_void_p]),
    "gaps_pool_cycles": (C.c_int, [_P(Batch), C.c_int64, C.c_int32, C.c_int64, _P(Params), C.c_void_p]),
    "gaps_pool_slice": (C.c_int, [_P(Batch), C.c_int64, C.c_int32, C.c_int64, _P(PersistentConfig), _P(Params),
                                  C.c_void_p]),
    "gaps_pool_finish_jobs": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, _P(Batch), C.c_void_p,
                                        C.c_void_p]),
    "gaps_pool_progress": (C.c_int, [_P(Batch), C.c_int64, _P(C.c_int64), C.c_void_p, C.c_void_p]),
    "gaps_pool_finish": (C.c_int, [C.c_int32, C.c_int64, C.c_int64, _P(Batch), C.c_void_p, C.c_void_p]),
    "gaps_server_create": (C.c_int, [_P(Batch), C.c_void_p, C.c_int32, C.c_int32, C.c_int32, _P(PersistentConfig),
                                     C.c_void_p, _P(C.c_void_p)]),
    "gaps_submit": (C.c_int, [C.c_void_p, _P(Params), C.c_int64, C.c_uint32, _P(C.c_uint64)]),
    "gaps_poll": (C.c_int, [C.c_void_p, C.c_uint64, C.c_void_p, _P(C.c_int32)]),
    "gaps_server_step": (C.c_int, [C.c_void_p, _P(C.c_uint64), C.c_int32, _P(C.c_int32)]),
    "gaps_server_counts": (C.c_int, [C.c_void_p, _P(C.c_int64), _P(C.c_int64), _P(C.c_int64)]),
    "gaps_server_destroy": (None, [C.c_void_p]),
    "gaps_strerror": (C.c_char_p, [C.c_int]),
    "gaps_last_cuda_error": (C.c_char_p, []),
    "gaps_version": (C.c_int, []),
}

# The measurement and test library (include/gaps_probe.h), separate from the
# product library.
PROBE_SIGNATURES = {
    "gaps_probe_fp64_rates": (C.c_int, [C.c_void_p, _P(C.c_double), C.c_void_p]),
    "gaps_log_fp64_host": (C.c_int, [_P(C.c_double), _P(C.c_double), C.c_int64]),
    "gaps_f32_from_f64_host": (C.c_int, [_P(C.c_double), _P(C.c_float), C.c_int64]),
    "gaps_log_fp64_device": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    "gaps_sqrt_obs_device": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    "gaps_probe_last_cuda_error": (C.c_char_p, []),
}

_lib = None
_probe = None


def library_path() -> str:
    return _build.LIB


def probe_library_path() -> str:
    return _build.PROBE_LIB


def load_probe(build_if_missing: bool = True):
    """Load libgaps_probe.so (the FP64 probe and the accuracy-test exports)."""
    global _probe
    if _probe is None:
        if build_if_missing:
            _build.build()
        path = _build.PROBE_LIB
        if not os.path.exists(path):
            raise RuntimeError(f"probe library {path} is missing; build it with paper_2403_08692_gb300.build")
        L = C.CDLL(path)
        for name, (res, args) in PROBE_SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _probe = L
    return _probe


def _check_probe(code, where):
    if code != GAPS_OK:
        msg = f"{where}: status {code}"
        if code == GAPS_ERR_CUDA:
            msg += ": " + load_probe().gaps_probe_last_cuda_error().decode()
        raise RuntimeError(msg)
    return code


def load(build_if_missing: bool = True):
    """Load libgaps.so (building it first if needed) and bind every symbol."""
    global _lib
    if _lib is None:
        path = _build.build() if build_if_missing else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is missing; build it with paper_2403_08692_gb300.build")
        L = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class GapsError(RuntimeError):
    def __init__(self, code, where):
        L = load()
        msg = L.gaps_strerror(code).decode()
        if code == GAPS_ERR_CUDA:
            msg += ": " + L.gaps_last_cuda_error().decode()
        super().__init__(f"{where}: {msg} ({code})")
        self.code = code


def _check(code, where, allow=()):
    if code != GAPS_OK and code not in allow:
        raise GapsError(code, where)
    return code


TRIALS_PER_KERNEL, TRIALS_PER_DIPOLE = 0, 1


def make_params(sqrt_s=91.2, alphas_mz=0.118, t_cutoff=1.0, seed=1, n_flavours=5, fixed_alphas=0,
                max_steps=100000, trial_mode=TRIALS_PER_KERNEL):
    return Params(float(sqrt_s), float(alphas_mz), float(t_cutoff), int(seed), int(n_flavours),
                  int(fixed_alphas), int(max_steps), int(trial_mode))


def workspace_bytes(n_events, capacity):
    return int(load().gaps_workspace_bytes(int(n_events), int(capacity)))


def layout(n_events, capacity) -> Layout:
    L = Layout()
    _check(load().gaps_workspace_layout(int(n_events), int(capacity), C.byref(L)), "gaps_workspace_layout")
    return L


_workspace_layout = layout


def check_params(p: Params) -> int:
    return load().gaps_check_params(C.byref(p))


def _stream_handle(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _pp(p):
    """Parameters of a single-job call, or NULL for a multi-job batch."""
    return C.byref(p) if p is not None else None


def _batch(ws) -> Batch:
    return Batch(C.c_void_p(ws.buffer.data_ptr()), ws.n_events, ws.capacity, ws.first_event, ws.record_layout, 0)


def generate_me(p, ws, stream=None):
    _check(load().gaps_generate_me(_pp(p), C.byref(_batch(ws)), _stream_handle(stream)), "gaps_generate_me")


def shower(p, ws, mode=SHOWER_PLAIN, stream=None):
    """Returns (status code, launches); GAPS_ERR_STEP_LIMIT is not raised."""
    n = C.c_int64(0)
    rc = _check(load().gaps_shower(_pp(p), C.byref(_batch(ws)), int(mode), C.byref(n), _stream_handle(stream)),
                "gaps_shower", allow=(GAPS_ERR_STEP_LIMIT,))
    return rc, n.value


def shower_timed(p, ws, mode=SHOWER_PLAIN, stream=None):
    """gaps_shower_timed: returns (status code, launches, summed kernel ms)."""
    n = C.c_int64(0)
    ms = C.c_double(0.0)
    rc = _check(load().gaps_shower_timed(_pp(p), C.byref(_batch(ws)), int(mode), C.byref(n), C.byref(ms),
                                         _stream_handle(stream)), "gaps_shower_timed", allow=(GAPS_ERR_STEP_LIMIT,))
    return rc, n.value, ms.value


def set_jobs(jobs, ws, stream=None):
    """gaps_set_jobs: jobs is a list of (Params, n_events, first_event); the
    batch's events are split into consecutive ranges in that order."""
    arr = (Job * len(jobs))()
    for k, (p, n, first) in enumerate(jobs):
        arr[k] = Job(p, int(n), int(first), 0)
    _check(load().gaps_set_jobs(arr, len(jobs), C.byref(_batch(ws)), _stream_handle(stream)), "gaps_set_jobs")


def shower_persistent(p, ws, cfg=None, stream=None):
    """gaps_shower_persistent: asynchronous, one launch.  cfg: PersistentConfig,
    a dict of its fields, or None for the library default."""
    cfg = persistent_config(cfg)
    ptr = C.byref(cfg) if cfg is not None else None
    _check(load().gaps_shower_persistent(_pp(p), C.byref(_batch(ws)), ptr, _stream_handle(stream)),
           "gaps_shower_persistent")


def autotune_persistent(p, ws, stream=None):
    """gaps_autotune_persistent: returns (PersistentConfig, best ms)."""
    cfg = PersistentConfig()
    ms = C.c_double(0.0)
    _check(load().gaps_autotune_persistent(_pp(p), C.byref(_batch(ws)), C.byref(cfg), C.byref(ms),
                                           _stream_handle(stream)), "gaps_autotune_persistent")
    return cfg, ms.value


def shower_step(p, ws, stream=None):
    _check(load().gaps_shower_step(_pp(p), C.byref(_batch(ws)), _stream_handle(stream)), "gaps_shower_step")


def validate(p, ws, stream=None):
    _check(load().gaps_validate(_pp(p), C.byref(_batch(ws)), _stream_handle(stream)), "gaps_validate")


def observables(p, ws, stream=None):
    _check(load().gaps_observables(_pp(p), C.byref(_batch(ws)), _stream_handle(stream)), "gaps_observables")


def histograms(p, ws, hist_device, stream=None):
    _check(load().gaps_histograms(_pp(p), C.byref(_batch(ws)), C.c_void_p(hist_device.data_ptr()),
                                  _stream_handle(stream)), "gaps_histograms")


def histograms_fixed(p, ws, acc_device, stream=None):
    """gaps_histograms_fixed: add the batch's exact fixed-point fills to
    acc_device (a CUDA int64 tensor of HIST_FIXED_WORDS per set)."""
    _check(load().gaps_histograms_fixed(_pp(p), C.byref(_batch(ws)), C.c_void_p(acc_device.data_ptr()),
                                        _stream_handle(stream)), "gaps_histograms_fixed")


def hist_fixed_scales(p):
    """(k_w, k_w2): the fixed-point exponents of a job's accumulators."""
    a, b = C.c_int32(0), C.c_int32(0)
    _check(load().gaps_hist_fixed_scales(C.byref(p), C.byref(a), C.byref(b)), "gaps_hist_fixed_scales")
    return a.value, b.value


def hist_fixed_to_double(p, acc):
    """One fixed-point set (host int64/uint64 numpy array of HIST_FIXED_WORDS)
    as a float64 numpy array of HIST_DOUBLES."""
    import numpy as np
    a = np.ascontiguousarray(acc).view(np.uint64)
    out = np.empty(HIST_DOUBLES, dtype=np.float64)
    _check(load().gaps_hist_fixed_to_double(C.byref(p), C.c_void_p(a.ctypes.data), C.c_void_p(out.ctypes.data)),
           "gaps_hist_fixed_to_double")
    return out


def reduce_stats(ws, stats_device, stream=None):
    _check(load().gaps_reduce_stats(C.byref(_batch(ws)), C.c_void_p(stats_device.data_ptr()),
                                    _stream_handle(stream)), "gaps_reduce_stats")


def probe_fp64_rates(stream=None):
    """FP64 results per second of this GPU: dict of dfma, log, exp, div, sqrt,
    sincospi and log_fp64 (the shower's table-driven log)."""
    import torch
    sink = torch.zeros(1, dtype=torch.float64, device="cuda")
    rates = (C.c_double * 7)()
    _check_probe(load_probe().gaps_probe_fp64_rates(C.c_void_p(sink.data_ptr()), rates, _stream_handle(stream)),
                 "gaps_probe_fp64_rates")
    return dict(zip(("dfma", "log", "exp", "div", "sqrt", "sincospi", "log_fp64"), list(rates)))


def log_fp64_host(x):
    """The shower's FP64 logarithm on a float64 numpy array (host code)."""
    import numpy as np
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty_like(x)
    _check_probe(load_probe().gaps_log_fp64_host(x.ctypes.data_as(_P(C.c_double)),
                                                 y.ctypes.data_as(_P(C.c_double)), int(x.size)),
                 "gaps_log_fp64_host")
    return y


def f32_from_f64_host(x):
    """The kernels' integer double -> float conversion on a float64 numpy
    array (host code)."""
    import numpy as np
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(x.shape, dtype=np.float32)
    _check_probe(load_probe().gaps_f32_from_f64_host(x.ctypes.data_as(_P(C.c_double)),
                                                     y.ctypes.data_as(_P(C.c_float)), int(x.size)),
                 "gaps_f32_from_f64_host")
    return y


def log_fp64_device(x, stream=None):
    """The shower's FP64 logarithm on a contiguous float64 CUDA tensor."""
    import torch
    x = x.contiguous()
    y = torch.empty_like(x)
    _check_probe(load_probe().gaps_log_fp64_device(C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                                                   int(x.numel()), _stream_handle(stream)), "gaps_log_fp64_device")
    return y


def sqrt_obs_device(x, stream=None):
    """The observables' Newton-refined square root on a contiguous float64
    CUDA tensor."""
    import torch
    x = x.contiguous()
    y = torch.empty_like(x)
    _check_probe(load_probe().gaps_sqrt_obs_device(C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                                                   int(x.numel()), _stream_handle(stream)), "gaps_sqrt_obs_device")
    return y


NOALLOC_MAX_EVENTS = 1 << 20


def event_shapes_noalloc(px, py, pz, e, n_partons, status, n_events, capacity, sqrt_s, obs, stream=None):
    """gaps_event_shapes_noalloc on caller-owned device tensors (no workspace,
    no allocation): momenta [capacity][n_events] float64, n_partons and
    status int32 [n_events]; writes obs [N_OBS][n_events] float64.  The
    tensors are checked (dtype, device, contiguity, length) before the call,
    since the library only sees raw pointers.  n_events = 0 (tensors may be
    None) runs only the per-device set-up."""
    import torch
    n, cap = int(n_events), int(capacity)
    if n > 0:
        need = {"px": (px, torch.float64, cap * n), "py": (py, torch.float64, cap * n),
                "pz": (pz, torch.float64, cap * n), "e": (e, torch.float64, cap * n),
                "n_partons": (n_partons, torch.int32, n), "status": (status, torch.int32, n),
                "obs": (obs, torch.float64, N_OBS * n)}
        for name, (t, dtype, count) in need.items():
            if t is None or t.dtype != dtype or not t.is_cuda or not t.is_contiguous() or t.numel() < count:
                raise ValueError(f"event_shapes_noalloc: {name} must be a contiguous CUDA {dtype} tensor "
                                 f"of at least {count} elements")
    ptr = lambda t: C.c_void_p(t.data_ptr() if t is not None else 0)
    _check(load().gaps_event_shapes_noalloc(ptr(px), ptr(py), ptr(pz), ptr(e), ptr(n_partons), ptr(status),
                                            n, cap, float(sqrt_s), ptr(obs),
                                            _stream_handle(stream)), "gaps_event_shapes_noalloc")


def pool_reset(ws, stream=None):
    _check(load().gaps_pool_reset(C.byref(_batch(ws)), _stream_handle(stream)), "gaps_pool_reset")


def pool_admit(p, job_slot, ev_begin, n_events, first_event, ws, cycle, stream=None):
    _check(load().gaps_pool_admit(C.byref(p), int(job_slot), int(ev_begin), int(n_events), int(first_event),
                                  C.byref(_batch(ws)), int(cycle), _stream_handle(stream)), "gaps_pool_admit")


def pool_cycles(ws, first_cycle, n_cycles, max_active, shared=None, stream=None):
    """gaps_pool_cycles.  shared: Params every live job has apart from its
    seed (the keyed kernels), or None."""
    _check(load().gaps_pool_cycles(C.byref(_batch(ws)), int(first_cycle), int(n_cycles), int(max_active),
                                   _pp(shared), _stream_handle(stream)), "gaps_pool_cycles")


def pool_slice(ws, round_index, cycles, max_active, cfg=None, shared=None, stream=None):
    """gaps_pool_slice: every live event runs up to `cycles` more cycles in one
    persistent launch.  cfg: PersistentConfig, a dict of its fields, or None;
    shared as for pool_cycles."""
    cfg = persistent_config(cfg)
    ptr = C.byref(cfg) if cfg is not None else None
    _check(load().gaps_pool_slice(C.byref(_batch(ws)), int(round_index), int(cycles), int(max_active), ptr,
                                  _pp(shared), _stream_handle(stream)), "gaps_pool_slice")


PHYSICS_FIELDS = ("sqrt_s", "alphas_mz", "t_cutoff", "n_flavours", "fixed_alphas", "max_steps", "trial_mode")


def same_physics(a, b):
    """Whether two Params differ at most in their seed."""
    return all(getattr(a, f) == getattr(b, f) for f in PHYSICS_FIELDS)


def pool_progress(ws, cycle, job_done=None, stream=None):
    """Live events before cycle `cycle`; fills job_done (a host uint64 array
    of MAX_JOBS elements) when given.  Synchronises the stream."""
    active = C.c_int64(0)
    ptr = None if job_done is None else C.c_void_p(job_done.ctypes.data)
    _check(load().gaps_pool_progress(C.byref(_batch(ws)), int(cycle), C.byref(active), ptr,
                                     _stream_handle(stream)), "gaps_pool_progress")
    return active.value


def pool_finish_jobs(job_slots, ev_begins, n_events, ws, hist_device, stream=None):
    """gaps_pool_finish_jobs: finalise several finished jobs at once; job i's
    histograms are added to hist_device[job_slots[i]] (hist_device: MAX_JOBS x
    HIST_DOUBLES or at least as many rows as the largest slot + 1)."""
    import numpy as np
    k = len(job_slots)
    slots = np.ascontiguousarray(job_slots, dtype=np.int32)
    begins = np.ascontiguousarray(ev_begins, dtype=np.int64)
    counts = np.ascontiguousarray(n_events, dtype=np.int64)
    if len(begins) != k or len(counts) != k:
        raise ValueError("one begin and one count per job")
    if k and int(slots.max()) >= hist_device.shape[0]:
        raise ValueError("hist_device has no row for a job slot")
    _check(load().gaps_pool_finish_jobs(C.c_void_p(slots.ctypes.data), C.c_void_p(begins.ctypes.data),
                                        C.c_void_p(counts.ctypes.data), int(k), C.byref(_batch(ws)),
                                        C.c_void_p(hist_device.data_ptr()), _stream_handle(stream)),
           "gaps_pool_finish_jobs")


def pool_finish(job_slot, ev_begin, n_events, ws, hist_device, stream=None):
    _check(load().gaps_pool_finish(int(job_slot), int(ev_begin), int(n_events), C.byref(_batch(ws)),
                                   C.c_void_p(hist_device.data_ptr()), _stream_handle(stream)), "gaps_pool_finish")


SERVE_SLICE, SERVE_STEPS = 0, 1


class CServer:
    """The library's C serving scheduler (gaps_server_*, gaps_submit,
    gaps_poll) over a pool workspace and a device histogram buffer this object
    allocates with PyTorch (the library allocates no device memory)."""

    def __init__(self, pool_events, capacity=128, max_jobs=64, cycles_per_round=8, mode=SERVE_SLICE, cfg=None,
                 stream=None):
        import torch
        self.ws = Workspace(pool_events, capacity)
        self.hist = torch.zeros((max_jobs, HIST_DOUBLES), dtype=torch.float64, device="cuda")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.stream.wait_stream(torch.cuda.current_stream())  # the buffers' fills come first
        cfg = persistent_config(cfg)
        self._batch = _batch(self.ws)
        h = C.c_void_p()
        _check(load().gaps_server_create(C.byref(self._batch), C.c_void_p(self.hist.data_ptr()), int(max_jobs),
                                         int(cycles_per_round), int(mode), C.byref(cfg) if cfg is not None else None,
                                         _stream_handle(self.stream), C.byref(h)), "gaps_server_create")
        self._h = h

    def submit(self, p, n_events, first_event=0):
        jid = C.c_uint64(0)
        _check(load().gaps_submit(self._h, C.byref(p), int(n_events), int(first_event), C.byref(jid)), "gaps_submit")
        return jid.value

    def poll(self, job_id):
        """None while the job runs, else its histograms (numpy, HIST_DOUBLES)."""
        import numpy as np
        out = np.empty(HIST_DOUBLES, dtype=np.float64)
        done = C.c_int32(0)
        _check(load().gaps_poll(self._h, C.c_uint64(job_id), C.c_void_p(out.ctypes.data), C.byref(done)), "gaps_poll")
        return out if done.value else None

    def step(self, max_ids=1024):
        """One step of the schedule; returns the ids of the finished jobs not
        yet reported by poll."""
        ids = (C.c_uint64 * max_ids)()
        n = C.c_int32(0)
        _check(load().gaps_server_step(self._h, ids, int(max_ids), C.byref(n)), "gaps_server_step")
        return list(ids[:min(n.value, max_ids)])

    def counts(self):
        q, l, f = C.c_int64(0), C.c_int64(0), C.c_int64(0)
        _check(load().gaps_server_counts(self._h, C.byref(q), C.byref(l), C.byref(f)), "gaps_server_counts")
        return q.value, l.value, f.value

    def close(self):
        if self._h:
            load().gaps_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def run(p, ws, host_hist, mode=SHOWER_PLAIN, stream=None):
    """The whole pipeline through host buffers.  host_hist: a CPU float64
    tensor/array of HIST_DOUBLES elements (pinned for asynchronous copies).
    Returns (status code, Stats)."""
    st = Stats()
    ptr = host_hist.data_ptr() if hasattr(host_hist, "data_ptr") else host_hist.ctypes.data
    rc = _check(load().gaps_run(_pp(p), C.byref(_batch(ws)), int(mode), C.cast(ptr, C.POINTER(C.c_double)),
                                C.byref(st), _stream_handle(stream)), "gaps_run", allow=(GAPS_ERR_STEP_LIMIT,))
    return rc, st


class Workspace:
    """A device workspace for one batch, allocated by PyTorch, with typed
    views of every array in the layout."""

    def __init__(self, n_events, capacity=128, first_event=0, device="cuda", layout=LAYOUT_SOA):
        import torch
        self.n_events = int(n_events)
        self.capacity = int(capacity)
        self.first_event = int(first_event)
        # the record layout the library reads and writes this workspace in
        # (gaps_batch::layout); a workspace holds any layout, so it may change
        # between passes (the events must then be generated again)
        self.record_layout = int(layout)
        nbytes = workspace_bytes(self.n_events, self.capacity)
        if nbytes == 0:
            raise ValueError("batch sizes out of range")
        # 256 extra bytes so the base can be aligned to 256
        self._raw = torch.zeros(nbytes + 256, dtype=torch.uint8, device=device)
        if self._raw.is_cuda:
            # The fill ran on the current stream; library calls may come on
            # any stream, so it must be complete before the first of them.
            torch.cuda.current_stream(self._raw.device).synchronize()
        off = (-self._raw.data_ptr()) % 256
        self.buffer = self._raw[off:off + nbytes]
        self.layout = _workspace_layout(self.n_events, self.capacity)  # byte offsets of every array

    def view(self, name, dtype, shape):
        import torch
        off = getattr(self.layout, name)
        nbytes = 1
        for d in shape:
            nbytes *= d
        nbytes *= torch.empty((), dtype=dtype).element_size()
        return self.buffer[off:off + nbytes].view(dtype).view(*shape)

    def slot_view(self, name, dtype, sides=0):
        """A per-parton array as [capacity][n_events] ([2][capacity][n_events]
        with sides=2): a view for the structure-of-arrays layout, a copy
        (read only) for the tiled layouts."""
        import torch
        n, cap = self.n_events, self.capacity
        shape = (cap, n) if not sides else (2, cap, n)
        if self.record_layout == LAYOUT_SOA:
            return self.view(name, dtype, shape)
        T = _TILE[self.record_layout]
        n_pad = (n + 31) // 32 * 32
        tiles = n_pad // T
        inner = (tiles, cap, T) if not sides else (tiles, 2, cap, T)
        raw = self.view(name, dtype, inner)
        if not sides:
            return raw.permute(1, 0, 2).reshape(cap, n_pad)[:, :n]
        return raw.permute(1, 2, 0, 3).reshape(2, cap, n_pad)[:, :, :n]

    def momenta(self):
        import torch
        return {c: self.slot_view(c, torch.float64) for c in ("e", "px", "py", "pz")}

    def scalars(self):
        import torch
        n = self.n_events
        out = {k: self.view(k, torch.int32, (n,)) for k in ("n_partons", "status", "n_steps", "n_emissions",
                                                            "n_winners", "n_trials", "n_dipoles", "next_colour",
                                                            "me_flavour", "valid")}
        out["t"] = self.view("t", torch.float64, (n,))
        out["weight"] = self.view("weight", torch.float64, (n,))
        out["hash"] = self.view("hash", torch.int64, (n,))
        return out

    def obs(self):
        import torch
        return self.view("obs", torch.float64, (N_OBS, self.n_events))

    def colours(self):
        import torch
        return {"flav": self.slot_view("flav", torch.int8), "col": self.slot_view("col", torch.int16),
                "acol": self.slot_view("acol", torch.int16), "link": self.slot_view("link", torch.uint8, sides=2)}
