"""ctypes binding of the oracle (test infrastructure only).

The oracle is the plain serial FP64 CPU implementation of the paper's event
generator that the CUDA path is checked against.  Only the tests, the smoke
check and the benchmark's CPU-baseline leg may import this module.
"""
import ctypes as C
import os

import numpy as np

from . import build_oracle

N_OBS = 8
HIST_ROW = 102
DONE, OVERFLOW, STEP_LIMIT = 1, 2, 3

MUT_NO_JACOBIAN = 1 << 0
MUT_Z_UNIFORM = 1 << 1
MUT_NO_RECOIL = 1 << 2
MUT_COLOUR_SWAP = 1 << 3
MUT_ALPHAS_OVER = 1 << 4
MUT_ME_NO_INTERF = 1 << 5
MUT_DURHAM_MAX = 1 << 6
MUT_THRUST_NOSIGNS = 1 << 7
MUT_KT_SIGN = 1 << 8
MUT_Z_SWAP = 1 << 9
MUT_HJM_LIGHT = 1 << 10
MUT_TRIAL_RESTART = 1 << 11
MUT_KERNEL_UNIFORM = 1 << 12
MUT_BROAD_DOT = 1 << 13
MUT_NF_MINUS_ONE = 1 << 14
MUT_PAIR_UNIFORM = 1 << 15
MUT_GG_FULL = 1 << 16
TRIALS_PER_KERNEL, TRIALS_PER_DIPOLE = 0, 1


class Params(C.Structure):
    _fields_ = [
        ("sqrt_s", C.c_double),
        ("alphas_mz", C.c_double),
        ("t_cutoff", C.c_double),
        ("seed", C.c_uint64),
        ("n_flavours", C.c_int32),
        ("fixed_alphas", C.c_int32),
        ("capacity", C.c_int32),
        ("max_steps", C.c_int32),
        ("max_emissions", C.c_int32),
        ("mutation", C.c_int32),
        ("trial_mode", C.c_int32),
    ]


EVENT_DTYPE = np.dtype([
    ("weight", "f8"), ("t_first", "f8"), ("t_final", "f8"), ("hash", "u8"), ("n_trials", "i8"),
    ("me_flavour", "i4"), ("n_partons", "i4"), ("status", "i4"), ("n_steps", "i4"),
    ("n_emissions", "i4"), ("n_winners", "i4"), ("valid", "i4"), ("n_dipoles", "i4"),
])
assert EVENT_DTYPE.itemsize == 72

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = build_oracle.build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int32)
        up = C.POINTER(C.c_uint32)
        L.oracle_check_params.argtypes = [C.POINTER(Params)]
        L.oracle_run.argtypes = [C.POINTER(Params), C.c_uint32, C.c_int64, C.c_int, C.c_void_p,
                                 dp, ip, dp, dp]
        L.oracle_run_from_state.argtypes = [C.POINTER(Params), C.c_int, dp, ip, C.c_uint32, C.c_int64, C.c_int,
                                            C.c_void_p, dp, ip]
        L.oracle_philox4x32_10.argtypes = [up, up, up]
        L.oracle_philox4x32_10.restype = None
        L.oracle_uniform_pair.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, dp]
        L.oracle_uniform_pair.restype = None
        for name in ("oracle_dsigma_dcos",):
            getattr(L, name).argtypes = [C.POINTER(Params), C.c_int, C.c_double]
            getattr(L, name).restype = C.c_double
        L.oracle_alphas.argtypes = [C.POINTER(Params), C.c_double]
        L.oracle_alphas.restype = C.c_double
        L.oracle_alphas_over.argtypes = [C.POINTER(Params)]
        L.oracle_alphas_over.restype = C.c_double
        L.oracle_kernel_value.argtypes = [C.c_int, C.c_double, C.c_double]
        L.oracle_kernel_value.restype = C.c_double
        L.oracle_kernel_estimate.argtypes = [C.c_int, C.c_double]
        L.oracle_kernel_estimate.restype = C.c_double
        L.oracle_kernel_integral.argtypes = [C.c_int, C.c_double, C.c_double]
        L.oracle_kernel_integral.restype = C.c_double
        L.oracle_kernel_generate_z.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_int]
        L.oracle_kernel_generate_z.restype = C.c_double
        L.oracle_splitting_map.argtypes = [dp, dp, C.c_double, C.c_double, C.c_double, C.c_int, dp, dp, dp]
        L.oracle_durham.argtypes = [C.c_int, dp, C.c_double, C.c_int, dp]
        L.oracle_thrust.argtypes = [C.c_int, dp, C.c_int, dp]
        L.oracle_event_shapes.argtypes = [C.c_int, dp, C.c_double, C.c_int, dp]
        L.oracle_validate.argtypes = [C.c_int, dp, ip, C.c_double]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else None


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32)) if a is not None else None


def make_params(sqrt_s=91.2, alphas_mz=0.118, t_cutoff=1.0, seed=1, n_flavours=5, fixed_alphas=0,
                capacity=128, max_steps=100000, max_emissions=0, mutation=0, trial_mode=0):
    return Params(float(sqrt_s), float(alphas_mz), float(t_cutoff), int(seed), int(n_flavours),
                  int(fixed_alphas), int(capacity), int(max_steps), int(max_emissions), int(mutation),
                  int(trial_mode))


def check_params(p: Params) -> int:
    return lib().oracle_check_params(C.byref(p))


def run(p: Params, first_event: int, n_events: int, threads: int = 1, want_momenta=False,
        want_obs=True, want_hist=True):
    """Shower events first_event .. first_event+n_events-1.  Returns a dict with
    'events' (structured array), and optionally 'mom' [n, cap, 4] (E, px, py,
    pz), 'info' [n, cap, 3] (flavour, colour, anticolour), 'obs' [n, 8] and
    'hist' [8, 102, 3]."""
    n = int(n_events)
    ev = np.zeros(n, dtype=EVENT_DTYPE)
    mom = np.zeros((n, p.capacity, 4)) if want_momenta else None
    info = np.zeros((n, p.capacity, 3), dtype=np.int32) if want_momenta else None
    obs = np.zeros((n, N_OBS)) if want_obs else None
    hist = np.zeros((N_OBS, HIST_ROW, 3)) if want_hist else None
    rc = lib().oracle_run(C.byref(p), first_event, n, threads, ev.ctypes.data_as(C.c_void_p),
                          _dp(mom), _ip(info), _dp(obs), _dp(hist))
    if rc != 0:
        raise ValueError("oracle_run rejected its arguments")
    out = {"events": ev}
    if want_momenta:
        out["mom"] = mom
        out["info"] = info
    if want_obs:
        out["obs"] = obs
    if want_hist:
        out["hist"] = hist
    return out


def run_from_state(p: Params, mom, info, first_event: int, n_events: int, threads: int = 1, want_momenta=False):
    """Shower events first_event .. first_event+n_events-1 from the given
    parton state (mom [n][4] as (E, px, py, pz), info [n][3] as (flavour,
    colour, anticolour)) instead of the matrix element.  Returns 'events' and,
    with want_momenta, 'mom' [n_events, cap, 4] and 'info' [n_events, cap, 3]."""
    m = np.ascontiguousarray(mom, dtype=np.float64)
    i = np.ascontiguousarray(info, dtype=np.int32)
    n = int(n_events)
    ev = np.zeros(n, dtype=EVENT_DTYPE)
    mo = np.zeros((n, p.capacity, 4)) if want_momenta else None
    io = np.zeros((n, p.capacity, 3), dtype=np.int32) if want_momenta else None
    rc = lib().oracle_run_from_state(C.byref(p), len(m), _dp(m), _ip(i), first_event, n, threads,
                                     ev.ctypes.data_as(C.c_void_p), _dp(mo), _ip(io))
    if rc != 0:
        raise ValueError("oracle_run_from_state rejected its arguments")
    out = {"events": ev}
    if want_momenta:
        out["mom"] = mo
        out["info"] = io
    return out


def philox(ctr, key):
    c = (C.c_uint32 * 4)(*ctr)
    k = (C.c_uint32 * 2)(*key)
    o = (C.c_uint32 * 4)()
    lib().oracle_philox4x32_10(c, k, o)
    return list(o)


def uniform_pair(seed, event, step, slot, purpose):
    o = np.zeros(2)
    lib().oracle_uniform_pair(seed, event, step, slot, purpose, _dp(o))
    return o


def dsigma_dcos(p, flavour, cth):
    return lib().oracle_dsigma_dcos(C.byref(p), flavour, cth)


def alphas(p, t):
    return lib().oracle_alphas(C.byref(p), t)


def alphas_over(p):
    return lib().oracle_alphas_over(C.byref(p))


def kernel_value(kind, z, y):
    return lib().oracle_kernel_value(kind, z, y)


def kernel_estimate(kind, z):
    return lib().oracle_kernel_estimate(kind, z)


def kernel_integral(kind, zm, zp):
    return lib().oracle_kernel_integral(kind, zm, zp)


def kernel_generate_z(kind, zm, zp, u, mutation=0):
    return lib().oracle_kernel_generate_z(kind, zm, zp, u, mutation)


def splitting_map(pij, pk, z, y, phi, mutation=0):
    a = np.ascontiguousarray(pij, dtype=np.float64)
    b = np.ascontiguousarray(pk, dtype=np.float64)
    oi, oj, ok = np.zeros(4), np.zeros(4), np.zeros(4)
    lib().oracle_splitting_map(_dp(a), _dp(b), z, y, phi, mutation, _dp(oi), _dp(oj), _dp(ok))
    return oi, oj, ok


def durham(mom, s, mutation=0):
    m = np.ascontiguousarray(mom, dtype=np.float64)
    o = np.zeros(4)
    if lib().oracle_durham(len(m), _dp(m), s, mutation, _dp(o)) != 0:
        raise ValueError("bad durham input")
    return o


def thrust(mom, mutation=0):
    m = np.ascontiguousarray(mom, dtype=np.float64)
    o = np.zeros(4)
    if lib().oracle_thrust(len(m), _dp(m), mutation, _dp(o)) != 0:
        raise ValueError("bad thrust input")
    return o


def event_shapes(mom, s, mutation=0):
    m = np.ascontiguousarray(mom, dtype=np.float64)
    o = np.zeros(N_OBS)
    if lib().oracle_event_shapes(len(m), _dp(m), s, mutation, _dp(o)) != 0:
        raise ValueError("bad event-shape input")
    return o


def validate(mom, info, sqrt_s):
    m = np.ascontiguousarray(mom, dtype=np.float64)
    i = np.ascontiguousarray(info, dtype=np.int32)
    return lib().oracle_validate(len(m), _dp(m), _ip(i), sqrt_s)


def threads_available() -> int:
    return max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count() or 1)
