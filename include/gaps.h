/* gaps.h -- C ABI of the event-parallel parton-shower library (sm_103a).
 *
 * The library implements the event-parallel Sudakov veto algorithm of
 * Seymour & Sule, "An Algorithm to Parallelise Parton Showers on a GPU"
 * (Sec. 2, Fig. 2, App. C): many independent e+e- -> q qbar events are
 * showered at once, every veto cycle running for all events in lock-step.
 * Around it sit the LO matrix element that creates the events (App. B) and
 * the observables computed on the finished events (Sec. 3.1: Durham jet
 * rates, thrust, heavy-jet mass; and the jet broadenings B_T, B_W of
 * Table 1) with their histograms.
 *
 * Memory model.  The caller owns all device memory: one workspace of
 * gaps_workspace_bytes(n_events, capacity) bytes, 256-byte aligned, holds the
 * structure-of-arrays event records and every per-event scalar, laid out as
 * gaps_workspace_layout() reports.  No compute entry point allocates, frees
 * or keeps device memory between calls, so the workspace may come from any
 * allocator (PyTorch's caching allocator in the Python binding).  Host
 * pointers are only read or written during the call.
 *
 * Streams.  `stream` is a cudaStream_t passed as void* (NULL = legacy
 * default stream).  Compute calls are asynchronous on that stream unless
 * stated otherwise; their host arguments may be reused as soon as the call
 * returns.
 *
 * Errors.  Every call returns GAPS_OK (0) or a negative gaps_status code;
 * gaps_strerror() names it.  Invalid arguments are reported before any work
 * is enqueued.  A CUDA launch or copy failure returns GAPS_ERR_CUDA and the
 * CUDA error string is available from gaps_last_cuda_error().
 *
 * Random numbers.  Every draw is Philox4x32-10 (Salmon et al., SC'11) keyed
 * by the 64-bit seed, with counter (event id, veto cycle, slot, purpose), so
 * an event's history depends only on (seed, event id) and never on the
 * launch configuration, the shower form, or the other events in the batch.
 */
#ifndef GAPS_H
#define GAPS_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gaps_status {
  GAPS_OK = 0,
  GAPS_ERR_INVALID = -1,    /* bad parameters, sizes or pointers */
  GAPS_ERR_CUDA = -2,       /* a CUDA call failed */
  GAPS_ERR_STEP_LIMIT = -3, /* some event hit max_steps veto cycles */
  GAPS_ERR_NO_DEVICE = -4   /* no usable sm_103 device */
} gaps_status;

/* Physics parameters as the paper states them: sqrt(s) = 91.2 GeV for LEP
 * (Sec. 1, Sec. 3), alpha_s(m_Z) = 0.118 and t_C = 1 (Fig. 4 caption; t_C in
 * GeV^2), the number of quark flavours drawn by the matrix element (App. B,
 * random(1, 5)), and the Philox seed. */
typedef struct gaps_params {
  double sqrt_s;        /* centre-of-mass energy in GeV, > 0 */
  double alphas_mz;     /* strong coupling at the Z mass, > 0 */
  double t_cutoff;      /* shower cutoff t_C in GeV^2, 0 < t_C < s/4, alpha_s(t_C) finite */
  uint64_t seed;        /* Philox key */
  int32_t n_flavours;   /* 1..5 */
  int32_t fixed_alphas; /* 0: one-loop running alpha_s(t); 1: alpha_s fixed at alpha_s(m_Z) */
  int32_t max_steps;    /* veto cycles allowed per event (>= 1); more sets the step-limit status */
  int32_t trial_mode;   /* GAPS_TRIALS_PER_KERNEL or GAPS_TRIALS_PER_DIPOLE */
} gaps_params;

/* Trial generation (App. A).  Per kernel: one trial scale for every
 * (dipole, matching kernel), as App. A generates them.  Per dipole: one
 * trial per dipole with the sum of its kernels' overestimates, the kernel
 * then drawn with probability proportional to its share.  The first of
 * independent exponential trials is distributed as one trial with the
 * summed rate whose kind has probability rate / sum, so this is the same
 * distribution with fewer trials (a gluon's six kernels need one trial, not
 * six), but other random numbers, so other events. */
enum { GAPS_TRIALS_PER_KERNEL = 0, GAPS_TRIALS_PER_DIPOLE = 1 };

/* Record layouts of the per-parton arrays of a workspace.  Structure of
 * arrays: slot-major [capacity][n_events], element (slot i, event e) at index
 * i * n_events + e.  Tiles of T = 8 or 32 events (array of structures of
 * arrays): [ceil(n_events / T)][capacity][T], element (i, e) at
 * (e / T) * capacity * T + i * T + e % T, so all slots of an event lie within
 * capacity * T elements while a warp of consecutive events still reads
 * contiguous segments.  The [2][capacity] arrays (link, dip, dq2, dzp, dinv)
 * are [2][capacity][n_events] and [ceil(n_events / T)][2][capacity][T]. */
enum { GAPS_LAYOUT_SOA = 0, GAPS_LAYOUT_TILE8 = 1, GAPS_LAYOUT_TILE32 = 2 };

/* One batch of events inside a caller-owned device workspace.  Event j of
 * the batch has id first_event + j (the Philox counter's event word).  The
 * layout is a property of the workspace's contents: every call on the same
 * events must give the layout gaps_generate_me (or gaps_pool_admit) wrote
 * them with.  A workspace sized by gaps_workspace_bytes holds any layout. */
typedef struct gaps_batch {
  void* workspace;      /* device pointer, 256-byte aligned, gaps_workspace_bytes() long */
  int64_t n_events;     /* 0 .. 2^31-1 */
  int32_t capacity;     /* parton slots per event, 4..255; the paper uses 50 (App. C) */
  uint32_t first_event; /* id of the batch's first event */
  int32_t layout;       /* GAPS_LAYOUT_SOA (0), GAPS_LAYOUT_TILE8 or GAPS_LAYOUT_TILE32 */
  int32_t reserved;     /* must be 0 */
} gaps_batch;

/* Byte offsets, from the workspace base, of every array in the workspace.
 * Each per-parton array has room for capacity * n_events events rounded up
 * to a multiple of 32, in the batch's layout (above); with the default
 * structure-of-arrays layout element (slot i, event e) is at index
 * i * n_events + e, so a warp of consecutive events reads one contiguous
 * segment per slot. */
typedef struct gaps_layout {
  int64_t px, py, pz, e;  /* double [capacity][n_events] (in the batch's layout), GeV */
  int64_t flav;           /* int8   [capacity][n_events]: PDG id, 21 = gluon */
  int64_t col, acol;      /* int16  [capacity][n_events]: colour / anticolour line, 0 = none */
  int64_t link;           /* uint8  [2][capacity][n_events]: colour partner slot on side 0
                             (colour line) and side 1 (anticolour line), 255 = none */
  int64_t dip;            /* float2 [2][capacity][n_events]: per-dipole cache of the trial
                             densities (library-internal contents) */
  int64_t dq2, dzp, dinv; /* double [2][capacity][n_events]: FP64 part of the dipole cache
                             (Q^2, z+, 1/ln(z+/z-); library-internal contents) */
  int64_t t;              /* double [n_events]: evolution scale t (GeV^2) at which the event
                             finished: t_C at the cutoff, the last winner's scale otherwise */
  int64_t lnt;            /* double [n_events]: ln t while the event is showering */
  int64_t weight;         /* double [n_events]: matrix-element weight (pb) */
  int64_t hash;           /* uint64 [n_events]: FNV-1a of the veto decisions */
  int64_t n_partons;      /* int32  [n_events] */
  int64_t status;         /* int32  [n_events]: 0 active, 1 done, 2 overflow, 3 step limit */
  int64_t n_steps;        /* int32  [n_events]: veto cycles run */
  int64_t n_emissions;    /* int32  [n_events] */
  int64_t n_winners;      /* int32  [n_events]: cycles with a trial above t_C */
  int64_t n_trials;       /* int32  [n_events]: trial emissions generated */
  int64_t n_dipoles;      /* int32  [n_events]: dipoles evaluated (Q^2 >= 4 t_C), over all cycles */
  int64_t next_colour;    /* int32  [n_events] */
  int64_t me_flavour;     /* int32  [n_events] */
  int64_t valid;          /* int32  [n_events]: validation bits, 0 = valid */
  int64_t obs;            /* double [GAPS_N_OBS][n_events]: y23, y34, y45, y56, 1-T, rho_H, B_T, B_W
                             (-1 = undefined) */
  int64_t buckets;        /* int32 [769]: scratch of gaps_observables (multiplicity buckets) */
  int64_t order;          /* int32 [n_events]: scratch of gaps_observables (events by multiplicity) */
  int64_t active;         /* int32 [2][n_events]: scratch of the plain shower (active-event lists) */
  int64_t tasks;          /* [2][n_events] 56-byte records: scratch of the plain shower (the accepted
                             emissions deferred to the next launch) */
  int64_t counters;       /* uint64 [32]: device counters of the last shower call: 0 finished events,
                             1 step-limited events, 2 cycles decided in full FP64, 3 vetoes decided in FP64;
                             of the last gaps_observables call: 4 thrust searches run in FP64, 5 Durham
                             merges with several FP64 candidates, 8 finished events left without
                             observables for a parton count outside 2..capacity; 6 the persistent
                             form's event cursor; 9 the job count of a multi-job batch;
                             7 scratch of the plain form's list rebuild; 21..23 the plain form's
                             active-list lengths and 24..26 its deferred-emission counts, rotating
                             over three launches; 10..12 and 18..20 the same for the serving pool;
                             27 the plain form's list rebuilds; 28 the pool slices' event cursor;
                             29..31 and 13..15 the emission-task cursors of the plain form's and the
                             pool's step launches */
  int64_t hist;           /* double [GAPS_HIST_DOUBLES]: histogram accumulator of gaps_run */
  int64_t hist_fixed;     /* uint64 [GAPS_MAX_JOBS][GAPS_HIST_FIXED_WORDS]: fixed-point scratch of
                             gaps_histograms */
  int64_t stats;          /* gaps_stats: statistics accumulator of gaps_run */
  int64_t jobs;           /* job table of a multi-job batch (library-internal, GAPS_MAX_JOBS entries) */
  int64_t job_begin;      /* int64 [GAPS_MAX_JOBS + 1]: first batch event of every job */
  int64_t job_of;         /* uint16 [n_events]: job of every event of a multi-job batch */
  int64_t job_done;       /* uint64 [GAPS_MAX_JOBS]: finished events per job slot */
  int64_t finish;         /* int64 [2][GAPS_MAX_JOBS + 1]: scratch of gaps_pool_finish_jobs (the
                             position prefix and first event of every range) */
  int64_t total_bytes;
} gaps_layout;

/* Largest number of jobs in one multi-job batch. */
#define GAPS_MAX_JOBS 1024

/* One job of a multi-job batch: its own physics parameters and seed, and a
 * contiguous range of the batch's events. */
typedef struct gaps_job {
  gaps_params params;
  int64_t n_events;     /* events of this job (>= 0) */
  uint32_t first_event; /* Philox event id of the job's first event */
  int32_t reserved;     /* must be 0 */
} gaps_job;

/* Event status values.  GAPS_PENDING marks an active event whose accepted
 * emission waits for the next launch of the plain form; it is seen only
 * between the launches of a shower call, never after one returns. */
enum { GAPS_ACTIVE = 0, GAPS_DONE = 1, GAPS_OVERFLOW = 2, GAPS_STEP_LIMIT = 3, GAPS_PENDING = 4 };

/* Histograms: GAPS_N_OBS observables x GAPS_HIST_ROW bins (underflow, 100
 * bins, overflow) x (sum w, sum w^2, entries), double.  Binning: log10 y23,
 * y34, y45, y56 on [-4.3, -0.3]; 1-T and rho_H on [0, 0.5]; B_T and B_W on
 * [0, 0.4]. */
enum { GAPS_N_OBS = 8, GAPS_N_BINS = 100, GAPS_HIST_ROW = 102 };
#define GAPS_HIST_DOUBLES (GAPS_N_OBS * GAPS_HIST_ROW * 3)

/* Exact histogram accumulators (gaps_histograms_fixed): per cell (observable
 * h, bin b: cell = h * GAPS_HIST_ROW + b) five uint64 words -- sum w as a
 * two's-complement 128-bit integer in units of 2^-k_w pb (words 5 cell, 5
 * cell + 1: low, high), sum w^2 likewise in units of 2^-k_w2 pb^2 (words
 * 5 cell + 2, 5 cell + 3) and the entries (word 5 cell + 4).  Every weight is
 * rounded once to its unit; the sums are then exact, so they do not depend on
 * the order of the fills and two accumulators of the same job merge exactly
 * by 128-bit addition.  gaps_hist_fixed_scales gives k_w and k_w2 (chosen so
 * that every weight the job's matrix element can give stays below 2^62
 * units). */
#define GAPS_HIST_FIXED_WORDS (GAPS_N_OBS * GAPS_HIST_ROW * 5)

/* Totals over a batch, reduced on the device. */
typedef struct gaps_stats {
  int64_t n_events;
  int64_t n_done, n_overflow, n_step_limit, n_invalid;
  int64_t sum_steps, max_steps, sum_trials, sum_winners, sum_emissions, sum_partons, sum_dipoles;
  int64_t launches;  /* shower launches made by the shower call of gaps_run */
  double sum_weight;
  double sum_weight2;
} gaps_stats;

/* Shower forms for gaps_shower() and gaps_run(). */
enum {
  GAPS_SHOWER_PLAIN = 0,     /* one launch per shower step over the active events, host all-done check
                                (App. C); a step runs the select/veto phase and the splittings the
                                previous step accepted */
  GAPS_SHOWER_PERSISTENT = 1 /* one launch; per-block event pools, compaction and refill (no host loop) */
};

/* Launch shape of the persistent form.  block_threads: 64, 128, 256 or 512
 * events per block pool; compact_period: veto cycles between compactions
 * and refills of a pool (>= 1); blocks_per_sm: resident blocks per SM (0 =
 * as many as fit); layout: the record layout the autotuner found fastest
 * with this shape (gaps_autotune_persistent's output, to be used as the
 * batch's layout; launches take the layout from the batch and ignore this
 * field, which must be a valid layout). */
typedef struct gaps_persistent_config {
  int32_t block_threads;
  int32_t compact_period;
  int32_t blocks_per_sm;
  int32_t layout;
} gaps_persistent_config;

/* ---------------------------------------------------------------- sizing */

/* Bytes of workspace for a batch; 0 if the sizes are out of range. */
size_t gaps_workspace_bytes(int64_t n_events, int32_t capacity);
/* Fill *out with the layout of a workspace for these sizes. */
int gaps_workspace_layout(int64_t n_events, int32_t capacity, gaps_layout* out);
/* GAPS_OK if the parameters are physical (see gaps_params). */
int gaps_check_params(const gaps_params* params);

/* ------------------------------------------------------- multi-job batches */

/* Make the batch a multi-job batch: jobs[0..n_jobs) take consecutive ranges
 * of the batch's events in order (their n_events must add up to the batch's).
 * Each job keeps its own sqrt(s), alpha_s, cutoff, flavours and seed, and its
 * events their own ids (first_event + k), so every event is the one a
 * single-job batch of that job would produce.  After this call pass
 * params = NULL to gaps_generate_me, gaps_shower, gaps_shower_persistent,
 * gaps_validate, gaps_observables and gaps_histograms; gaps_histograms then
 * fills one histogram set per job (hist_device holds n_jobs *
 * GAPS_HIST_DOUBLES doubles).  Synchronous. */
int gaps_set_jobs(const gaps_job* jobs, int32_t n_jobs, const gaps_batch* batch, void* stream);

/* ------------------------------------------------ serving: the event pool */

/* Continuous batching over one resident workspace (the pool).  Jobs arrive
 * while others shower: each is admitted into a free range of the pool and a
 * free job slot, its events join the live active list, and every veto cycle
 * advances all live events of all jobs (the plain cycle over the active
 * list, Sec. 2).  A job whose events have all finished is finalised on its
 * own range and its range and slot are reused.  The caller keeps the
 * schedule: the number of cycles launched so far (`cycle`), the free ranges
 * and slots, and an upper bound on the live events.  Every event equals the
 * event a single-job batch of its job produces. */

/* Clear the pool's active lists and per-job counters.  Asynchronous. */
int gaps_pool_reset(const gaps_batch* pool, void* stream);

/* Admit a job: n_events events in pool range [ev_begin, ev_begin +
 * n_events), job slot job_slot (0 .. GAPS_MAX_JOBS-1), event ids
 * first_event + k; generates their matrix elements and appends them to the
 * active list read by the next cycle (cycle = cycles launched so far).
 * Asynchronous. */
int gaps_pool_admit(const gaps_params* params, int32_t job_slot, int64_t ev_begin, int64_t n_events,
                    uint32_t first_event, const gaps_batch* pool, int64_t cycle, void* stream);

/* Enqueue n_cycles shower steps, numbered first_cycle.., over the live
 * events: each step runs the select/veto phase of the events in the active
 * list and the splittings the previous step accepted (gaps_shower's plain
 * form).  max_active bounds the live events (it sizes the grids).
 * shared: NULL, or parameters that every live job of the pool was admitted
 * with apart from its seed; the kernels then take the physics from `shared`
 * and only each job's Philox key and event-id offset from the job table
 * (the same events, faster).  A job whose other parameters differ from
 * `shared` is showered with `shared`'s physics: pass NULL for a mix.  No host
 * synchronisation. */
int gaps_pool_cycles(const gaps_batch* pool, int64_t first_cycle, int32_t n_cycles, int64_t max_active,
                     const gaps_params* shared, void* stream);

/* The same advance by the persistent form (time-sliced): one launch runs
 * every live event for up to `cycles` (1..255) more veto cycles in per-block
 * pools (cfg as for gaps_shower_persistent, NULL for the default), and the
 * events still active afterwards make up the next active list.  `round`
 * numbers the slices (the `cycle` of gaps_pool_admit and
 * gaps_pool_progress); shared as for gaps_pool_cycles.  A pool is driven
 * either by gaps_pool_cycles or by gaps_pool_slice.  No host
 * synchronisation. */
int gaps_pool_slice(const gaps_batch* pool, int64_t round, int32_t cycles, int64_t max_active,
                    const gaps_persistent_config* cfg, const gaps_params* shared, void* stream);

/* Read the number of live events before step `cycle` and, if job_done_out
 * is not NULL, the finished-event count of every job slot
 * (GAPS_MAX_JOBS values).  Synchronises the stream. */
int gaps_pool_progress(const gaps_batch* pool, int64_t cycle, int64_t* active_out, uint64_t* job_done_out,
                       void* stream);

/* Validation, observables and histograms of a finished job's range; adds
 * its histograms to hist_device (one set, GAPS_HIST_DOUBLES doubles, not
 * cleared).  Asynchronous. */
int gaps_pool_finish(int32_t job_slot, int64_t ev_begin, int64_t n_events, const gaps_batch* pool,
                     double* hist_device, void* stream);

/* Validation, observables and histograms of n_jobs finished jobs at once
 * (0 <= n_jobs <= GAPS_MAX_JOBS): job i holds pool range [ev_begins[i],
 * ev_begins[i] + n_events[i]) and job slot job_slots[i]; the ranges are
 * disjoint and the slots distinct.  The same results as one gaps_pool_finish
 * per job, in one sequence of launches over all of their events: a launch
 * lasts as long as its slowest event, so finalising the jobs of a round
 * together pays that latency once.  Job i's histograms are added to
 * hist_device + job_slots[i] * GAPS_HIST_DOUBLES (not cleared).  job_slots,
 * ev_begins and n_events are host arrays, read before the call returns.
 * The list goes to a small table in the pool's workspace, so calls on one
 * pool must be ordered (one stream), as all pool calls are.  Asynchronous. */
int gaps_pool_finish_jobs(const int32_t* job_slots, const int64_t* ev_begins, const int64_t* n_events,
                          int32_t n_jobs, const gaps_batch* pool, double* hist_device, void* stream);

/* ------------------------------------------- serving: the C scheduler */

/* The serving loop as a C API: continuous batching over one pool, with the
 * schedule kept by the library (Sec. 2 / App. C's host driver turned into a
 * request loop).  The caller owns the pool workspace (gaps_batch, first_event
 * 0) and hist_device (device memory, max_jobs * GAPS_HIST_DOUBLES doubles,
 * one set per job slot); the server keeps host state and a little pinned
 * host memory, never device memory.  Jobs are submitted as they arrive;
 * every step (gaps_server_step, or gaps_poll of a job not yet finished)
 * advances the schedule:
 *  - admission in submission order: a job takes a free slot (< max_jobs) and
 *    the first free contiguous range of the pool that holds its events (first
 *    fit, freed neighbours coalesced), its matrix elements are generated in
 *    place and its events join the live list (gaps_pool_admit);
 *  - one round: every live event runs up to cycles_per_round more veto
 *    cycles, by one time-sliced persistent launch (GAPS_SERVE_SLICE,
 *    gaps_pool_slice with cfg, NULL = default shape) or by that many
 *    plain-form steps (GAPS_SERVE_STEPS, gaps_pool_cycles);
 *  - progress read one round behind (the GPU keeps a round queued);
 *  - a job whose events have all finished is finalised on its range
 *    (gaps_pool_finish) and its histograms copied to the host; its range is
 *    reused at once, its slot once the copy has landed.
 * Every event equals the event a single-job batch of its job produces, and
 * the histograms are exact fixed-point sums converted once, so a job's
 * histograms are bitwise those of the same job run alone.  All calls on one
 * server must come from one host thread, on its stream. */
enum { GAPS_SERVE_SLICE = 0, GAPS_SERVE_STEPS = 1 };
typedef struct gaps_server gaps_server;

/* Create a server over the pool (resets its lists and counters).  max_jobs
 * 1..GAPS_MAX_JOBS, cycles_per_round 1..255, mode GAPS_SERVE_SLICE or
 * GAPS_SERVE_STEPS; cfg may be NULL.  *out = NULL on failure. */
int gaps_server_create(const gaps_batch* pool, double* hist_device, int32_t max_jobs, int32_t cycles_per_round,
                       int32_t mode, const gaps_persistent_config* cfg, void* stream, gaps_server** out);
/* Queue a job (params as for gaps_generate_me; 1 <= n_events <= the pool's
 * events; event ids first_event + k).  *job_id identifies it in gaps_poll.
 * Host only: the GPU work starts at the next poll. */
int gaps_submit(gaps_server* server, const gaps_params* params, int64_t n_events, uint32_t first_event,
                uint64_t* job_id);
/* One step of the schedule.  Then the ids of the finished jobs not yet
 * reported by gaps_poll go to finished_ids[0 .. min(count, max_ids)) and
 * their count to *n_finished (may be NULL).  May wait for the round before
 * the last to finish on the GPU. */
int gaps_server_step(gaps_server* server, uint64_t* finished_ids, int32_t max_ids, int32_t* n_finished);
/* Report job job_id: if it has not finished yet, one step of the schedule
 * first.  *done = 1 if it has finished, with its histograms copied to
 * host_hist (GAPS_HIST_DOUBLES doubles, may be NULL; the job is then
 * forgotten), else *done = 0.  GAPS_ERR_INVALID for a job id that was never
 * submitted or was already reported finished. */
int gaps_poll(gaps_server* server, uint64_t job_id, double* host_hist, int32_t* done);
/* Jobs waiting for admission, jobs live or being finalised, and finished jobs
 * not yet reported by gaps_poll (each may be NULL). */
int gaps_server_counts(const gaps_server* server, int64_t* queued, int64_t* live, int64_t* finished_unread);
/* Wait for the server's work on its stream and free it. */
void gaps_server_destroy(gaps_server* server);

/* ------------------------------------------------------------- hot path */

/* App. B: draw each event's flavour, cos(theta) and phi, set the quark and
 * antiquark back to back at E = sqrt(s)/2, and the weight w = n_f * 2 *
 * d sigma / d cos(theta) in pb (LO gamma/Z with interference).  Also the
 * shower's initial state (App. C listing, main program): t = s, two partons
 * on one colour line, status active.  Asynchronous. */
int gaps_generate_me(const gaps_params* params, const gaps_batch* batch, void* stream);

/* Sec. 2 / App. C: run the veto algorithm until every event has reached the
 * cutoff (or overflowed its capacity, or hit max_steps).  Each cycle selects,
 * per event, the winning trial emission over every colour-connected dipole
 * and matching splitting kernel (Eq. A.6), checks the cutoff, applies the
 * veto (Eq. A.8, A.9) and performs the accepted splitting.  mode =
 * GAPS_SHOWER_PLAIN: one launch per step (a step runs the select/veto phase
 * of the listed events and the splittings the previous step accepted); the
 * host checks the live count after every launch (the all-done check), read
 * from host-mapped memory that the next launch writes as it starts, and
 * keeps one launch queued ahead.  mode = GAPS_SHOWER_PERSISTENT: one
 * persistent launch (gaps_shower_persistent with the default shape).  The
 * stream is synchronised before returning.  *launches_out (may be NULL)
 * receives the number of step launches that had work.  Returns
 * GAPS_ERR_STEP_LIMIT if any event stopped at max_steps (the other events
 * are complete). */
int gaps_shower(const gaps_params* params, const gaps_batch* batch, int mode, int64_t* launches_out,
                void* stream);

/* gaps_shower that also measures the shower kernels: *kernel_ms_out (may be
 * NULL) receives the summed device time of the cycle launches, timed with
 * CUDA events recorded on `stream` around every launch. */
int gaps_shower_timed(const gaps_params* params, const gaps_batch* batch, int mode, int64_t* launches_out,
                      double* kernel_ms_out, void* stream);

/* The persistent form (Sec. 2, without the cutoff wait of Fig. 3): one
 * launch runs every event to the cutoff.  Each block keeps a pool of events,
 * two per thread for pools of up to 256 threads, runs cfg->compact_period
 * veto cycles on it (each warp on its own events, no block barrier; a
 * thread runs whichever of its events can run), generates the period's
 * accepted emissions together, packs the still-active events to the front
 * (warp ballot) and refills the free slots from a global event cursor.  An
 * event with a queued emission skips its selects until the end of the
 * period.  Events are identical to the plain form's (same draws, same cycle
 * code).  cfg = NULL uses {128, 8, 0}.  Fully asynchronous: no host synchronisation; the
 * workspace counters record finished and step-limited events. */
int gaps_shower_persistent(const gaps_params* params, const gaps_batch* batch,
                           const gaps_persistent_config* cfg, void* stream);

/* Autotuner of the persistent form (batching): times every record layout
 * (structure of arrays, tiles of 8 and of 32 events), block size {128, 256,
 * 512} and compaction period {2, 4, 8, 16} on this batch's workspace, the
 * better of two timings each (matrix element + shower each time, CUDA events
 * on `stream`), and returns the fastest in *best (layout included; its time
 * in *best_ms, may be NULL).  Overwrites the batch's events: regenerate them
 * with the chosen layout as the batch's layout.  Synchronous. */
int gaps_autotune_persistent(const gaps_params* params, const gaps_batch* batch, gaps_persistent_config* best,
                             double* best_ms, void* stream);

/* One veto cycle of the plain form for every active event (one launch). */
int gaps_shower_step(const gaps_params* params, const gaps_batch* batch, void* stream);

/* Validation of the finished record (the paper's "Validate Events" stage):
 * sets valid bits 1 momentum not conserved to 1e-10 GeV, 2 a parton off
 * shell (|p^2| > 1e-10 E sqrt(s)), 4 non-positive energy, 8 broken colour flow,
 * 16 flavour imbalance, 32 non-finite momentum, for every event of the
 * batch (whatever its status).  A parton count outside 0..capacity (a record
 * edited through the workspace) is read as its nearest bound, so no slot
 * beyond the capacity is touched.  Asynchronous. */
int gaps_validate(const gaps_params* params, const gaps_batch* batch, void* stream);

/* Sec. 3.1: Durham y23..y56 (E-scheme), thrust 1-T (exact), heavy-jet mass
 * rho_H, and the total and wide jet broadenings B_T, B_W (Table 1's
 * observable list: sum |p x n_T| / (2 sum |p|) per thrust hemisphere; B_T
 * their sum, B_W the larger) for every event that reached the cutoff; -1
 * where undefined.  Asynchronous. */
int gaps_observables(const gaps_params* params, const gaps_batch* batch, void* stream);

/* Sec. 3.2 (atomic histogramming): add the batch's observables, weighted by
 * the ME weight, to hist_device (GAPS_HIST_DOUBLES doubles, device memory,
 * not cleared by this call; n_jobs sets for a multi-job batch).  Only events
 * with status GAPS_DONE and valid == 0 are filled.  The fills are summed
 * exactly in fixed point (gaps_histograms_fixed) and converted once, so the
 * result does not depend on the order of the fills.  Asynchronous. */
int gaps_histograms(const gaps_params* params, const gaps_batch* batch, double* hist_device,
                    void* stream);

/* gaps_histograms' exact fixed-point form: add the batch's fills to
 * acc_device (device memory, GAPS_HIST_FIXED_WORDS uint64 per set, not
 * cleared; one set per job for a multi-job batch).  Only events with status
 * GAPS_DONE and valid == 0 are filled.  gaps_histograms accumulates this way
 * in the workspace and adds the converted sums to its double histograms, so
 * its results are bitwise reproducible too.  Asynchronous. */
int gaps_histograms_fixed(const gaps_params* params, const gaps_batch* batch, uint64_t* acc_device, void* stream);

/* The fixed-point exponents k_w, k_w2 of a job's accumulators (host only). */
int gaps_hist_fixed_scales(const gaps_params* params, int32_t* k_w, int32_t* k_w2);

/* One fixed-point set (host memory) as double histograms (host memory,
 * GAPS_HIST_DOUBLES, overwritten): sum w, sum w^2, entries per cell, each
 * converted with one rounding.  Host only. */
int gaps_hist_fixed_to_double(const gaps_params* params, const uint64_t* acc_host, double* hist_host);

/* Reduce the batch's per-event counters into *stats_device (device memory,
 * one gaps_stats).  Asynchronous. */
int gaps_reduce_stats(const gaps_batch* batch, gaps_stats* stats_device, void* stream);

/* The whole pipeline through host buffers: ME, shower (mode), validation,
 * observables, histograms and statistics, then copies the histograms into
 * host_hist (GAPS_HIST_DOUBLES doubles) and the statistics into
 * *host_stats (may be NULL), and synchronises the stream.  The histogram
 * and statistics accumulators live in the workspace and are cleared first. */
int gaps_run(const gaps_params* params, const gaps_batch* batch, int mode, double* host_hist,
             gaps_stats* host_stats, void* stream);

/* ------------------------------------------------- allocation-free entry */

/* Largest batch gaps_event_shapes_noalloc accepts. */
#define GAPS_NOALLOC_MAX_EVENTS (1 << 20)

/* The observables stage of gaps_observables (Durham y23..y56, 1-T, rho_H,
 * B_T, B_W) for callers that cannot allocate device memory -- code that must
 * stay inside another framework's memory pool, plug-ins whose host forbids
 * allocation calls, or processes that hand out all device memory up front.
 * The paper has no counterpart; it is a deployment variant.  The caller
 * passes only inputs and outputs: momenta px, py, pz, e as slot-major
 * [capacity][n_events] doubles (the workspace layout), n_partons and status
 * (int32 [n_events]), and obs (double [GAPS_N_OBS][n_events], written).  All
 * are device pointers.  The working arrays live in one fixed device array
 * inside the library, so the call allocates nothing and calls no allocating
 * routine.
 * Limits and behaviour:
 *  - n_events <= GAPS_NOALLOC_MAX_EVENTS, 4 <= capacity <= 255, sqrt_s > 0,
 *    and non-null arrays when n_events > 0, else GAPS_ERR_INVALID before any
 *    work.
 *  - obs gets -1 for events whose status is not GAPS_DONE, for events whose
 *    n_partons is outside 2 .. capacity (no slot beyond the capacity is
 *    read), and for undefined y values.
 *  - Set-up: the first call on a device looks up the array's device address
 *    (once per device, with that device current) and makes CUDA load the
 *    library code that holds the array and the observables' kernels.  CUDA
 *    loads that code lazily by default, so this first call is when the array
 *    (about 4.2 MB) and the kernels take their device memory, held until the
 *    process exits.  A call with n_events = 0 does only this set-up: make it
 *    before handing out all device memory and before any stream capture on
 *    the device.  The looked-up address is not valid after a
 *    cudaDeviceReset of the device; do not call this entry point after one.
 *  - All calls share the array and it keeps the last call's contents; each
 *    call clears what must start at zero on its own stream.  Calls whose
 *    work overlaps on the GPU race on the array: order them on one stream or
 *    synchronise between them.
 *  - Asynchronous on `stream`; results equal gaps_observables' for the same
 *    events. */
int gaps_event_shapes_noalloc(const double* px, const double* py, const double* pz, const double* e,
                              const int32_t* n_partons, const int32_t* status, int64_t n_events,
                              int32_t capacity, double sqrt_s, double* obs, void* stream);

/* --------------------------------------------------------------- misc */

const char* gaps_strerror(int status);
const char* gaps_last_cuda_error(void);
/* Library version as major * 10000 + minor * 100 + patch. */
int gaps_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GAPS_H */
