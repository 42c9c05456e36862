"""Event-parallel parton shower on GB300 (sm_103a).

A from-scratch implementation of the event-parallel Sudakov veto algorithm of
Seymour & Sule, "An Algorithm to Parallelise Parton Showers on a GPU": the LO
e+e- -> q qbar matrix element, the final-state dipole shower run for millions
of events at once, and the Durham / thrust / heavy-jet-mass observables with
their histograms.  The compute path is the CUDA library libgaps.so (C ABI in
include/gaps.h); this package is its thin Python binding.
"""
from .gaps import (  # noqa: F401
    ACTIVE, DONE, OVERFLOW, STEP_LIMIT, SHOWER_PLAIN, SHOWER_PERSISTENT, HIST_DOUBLES, N_OBS, HIST_ROW,
    PersistentConfig, shower_persistent, autotune_persistent, Job, set_jobs, MAX_JOBS,
    GapsError, Params, Stats, Workspace, check_params, generate_me, histograms, layout, load, shower_timed,
    make_params, observables, reduce_stats, run, shower, shower_step, validate, workspace_bytes,
    event_shapes_noalloc, probe_fp64_rates, log_fp64_host, log_fp64_device, sqrt_obs_device, f32_from_f64_host, TRIALS_PER_KERNEL, TRIALS_PER_DIPOLE, pool_reset, pool_admit, pool_cycles, pool_slice, pool_progress,
    pool_finish, pool_finish_jobs, same_physics, LAYOUT_SOA, LAYOUT_TILE8, LAYOUT_TILE32, LAYOUT_NAMES, persistent_config, CServer, SERVE_SLICE, SERVE_STEPS, HIST_FIXED_WORDS, histograms_fixed, hist_fixed_scales, hist_fixed_to_double,
)
from .serving import RangeAllocator, ServeJob, ServeResult, Server, latency_summary  # noqa: F401
