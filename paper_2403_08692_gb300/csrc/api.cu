// C ABI entry points (include/gaps.h): argument checks, workspace layout,
// launch sequencing and the host all-done loop of the plain shower form.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "gaps_launch.hpp"

namespace gaps {

namespace {

thread_local char g_cuda_error[256] = "";

int cuda_fail(cudaError_t e) {
  std::snprintf(g_cuda_error, sizeof(g_cuda_error), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
  return GAPS_ERR_CUDA;
}

constexpr int64_t kAlign = 256;
int64_t align_up(int64_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

bool sizes_ok(int64_t n_events, int32_t capacity) {
  return n_events >= 0 && n_events <= 0x7fffffffLL && capacity >= 4 && capacity <= 255;
}

void compute_layout(int64_t n, int32_t cap, gaps_layout* L) {
  int64_t off = 0;
  auto take = [&](int64_t bytes) {
    const int64_t at = off;
    off = align_up(off + bytes);
    return at;
  };
  // per-parton arrays: room for the events rounded up to whole tiles of 32,
  // so that every record layout fits
  const int64_t pc = static_cast<int64_t>(cap) * ((n + 31) / 32 * 32);
  L->px = take(8 * pc);
  L->py = take(8 * pc);
  L->pz = take(8 * pc);
  L->e = take(8 * pc);
  L->flav = take(pc);
  L->col = take(2 * pc);
  L->acol = take(2 * pc);
  L->link = take(2 * pc);
  L->dip = take(16 * pc);
  L->dq2 = take(16 * pc);
  L->dzp = take(16 * pc);
  L->dinv = take(16 * pc);
  L->t = take(8 * n);
  L->lnt = take(8 * n);
  L->weight = take(8 * n);
  L->hash = take(8 * n);
  L->n_partons = take(4 * n);
  L->status = take(4 * n);
  L->n_steps = take(4 * n);
  L->n_emissions = take(4 * n);
  L->n_winners = take(4 * n);
  L->n_trials = take(4 * n);
  L->n_dipoles = take(4 * n);
  L->next_colour = take(4 * n);
  L->me_flavour = take(4 * n);
  L->valid = take(4 * n);
  L->obs = take(8 * GAPS_N_OBS * n);
  L->buckets = take(4 * 769);
  L->order = take(4 * n);
  L->active = take(8 * n);
  L->tasks = take(2 * static_cast<int64_t>(kEmitTaskBytes) * n);
  L->counters = take(8 * kCounterWords);
  L->hist = take(8 * GAPS_HIST_DOUBLES);
  L->hist_fixed = take(8 * static_cast<int64_t>(GAPS_MAX_JOBS) * GAPS_HIST_FIXED_WORDS);
  L->stats = take(sizeof(gaps_stats));
  L->jobs = take(static_cast<int64_t>(sizeof(DevParams)) * GAPS_MAX_JOBS);
  L->job_begin = take(8 * (GAPS_MAX_JOBS + 1));
  L->job_of = take(2 * n);
  L->job_done = take(8 * GAPS_MAX_JOBS);
  L->finish = take(8 * 2 * (GAPS_MAX_JOBS + 1));
  L->total_bytes = off;
}

bool layout_ok(int layout) {
  return layout == GAPS_LAYOUT_SOA || layout == GAPS_LAYOUT_TILE8 || layout == GAPS_LAYOUT_TILE32;
}

int check_batch(const gaps_batch* b) {
  if (!b || !sizes_ok(b->n_events, b->capacity)) return GAPS_ERR_INVALID;
  if (!layout_ok(b->layout) || b->reserved != 0) return GAPS_ERR_INVALID;
  if (!b->workspace || (reinterpret_cast<uintptr_t>(b->workspace) % kAlign) != 0) return GAPS_ERR_INVALID;
  if (static_cast<uint64_t>(b->first_event) + static_cast<uint64_t>(b->n_events) > 0x100000000ull)
    return GAPS_ERR_INVALID;
  return GAPS_OK;
}

}  // namespace

int record_cuda_error(cudaError_t e) { return cuda_fail(e); }

// Fixed-point histogram exponents of a job: every weight its matrix element
// can give, w = a (1 + cos^2) + b cos, has |w| <= 2 |a| + |b| < 2^e, so
// |w| 2^(62 - e) and w^2 2^(62 - 2 e) stay below 2^62.
void hist_scales(const DevParams& d, int* k_w, int* k_w2) {
  double bound = 0.0;
  for (int f = 0; f < 5; ++f) bound = std::max(bound, 2.0 * std::fabs(d.me_a[f]) + std::fabs(d.me_b[f]));
  int e = 0;
  std::frexp(bound, &e);
  *k_w = 62 - e;
  *k_w2 = 62 - 2 * e;
}

DevParams make_dev_params(const gaps_params& p, int64_t id_offset) {
  DevParams d{};
  d.id_offset = id_offset;
  d.sqrt_s = p.sqrt_s;
  d.s = p.sqrt_s * p.sqrt_s;
  d.tc = p.t_cutoff;
  d.inv_4tc = 1.0 / (4.0 * p.t_cutoff);
  d.inv_s = 1.0 / d.s;
  for (int f = 1; f <= 5; ++f) {
    double a = 0.0, b = 0.0;
    dsigma_parts(d.s, f, &a, &b);
    d.me_a[f - 1] = p.n_flavours * 2.0 * a;
    d.me_b[f - 1] = p.n_flavours * 2.0 * b;
  }
  d.alphas_mz = p.alphas_mz;
  d.nf = p.n_flavours;
  d.fixed = p.fixed_alphas ? 1 : 0;
  d.max_steps = p.max_steps;
  d.trial_mode = p.trial_mode;
  d.b0 = (33.0 - 2.0 * p.n_flavours) / (12.0 * kPi);
  d.as_over = d.fixed ? p.alphas_mz
                      : p.alphas_mz / (1.0 + p.alphas_mz * d.b0 * std::log(p.t_cutoff / (kMZ * kMZ)));
  d.ln_tc = std::log(p.t_cutoff);
  d.ln_s = std::log(d.s);
  d.inv_as2pi_2cf = 1.0 / ((d.as_over / (2.0 * kPi)) * (2.0 * kCF));
  d.inv_as2pi_ca = 1.0 / ((d.as_over / (2.0 * kPi)) * kCA);
  d.tcf = static_cast<float>(p.t_cutoff);
  d.as2pi_f = static_cast<float>(d.as_over / (2.0 * kPi));
  d.lg2_tc_f = static_cast<float>(std::log2(p.t_cutoff));
  d.as_mz_over_f = static_cast<float>(p.alphas_mz / d.as_over);
  d.as_b0_f = static_cast<float>(p.alphas_mz * d.b0);
  d.ln_mz2_f = static_cast<float>(std::log(kMZ * kMZ));
  d.seed_lo = static_cast<uint32_t>(p.seed);
  d.seed_hi = static_cast<uint32_t>(p.seed >> 32);
  for (int r = 0; r < 10; ++r) {
    d.rk[2 * r] = d.seed_lo + static_cast<uint32_t>(r) * 0x9E3779B9u;
    d.rk[2 * r + 1] = d.seed_hi + static_cast<uint32_t>(r) * 0xBB67AE85u;
  }
  int k_w = 0, k_w2 = 0;
  hist_scales(d, &k_w, &k_w2);
  d.hist_sw = std::ldexp(1.0, k_w);
  d.hist_sw2 = std::ldexp(1.0, k_w2);
  d.hist_sw_inv = std::ldexp(1.0, -k_w);
  d.hist_sw2_inv = std::ldexp(1.0, -k_w2);
  return d;
}

Events make_events(const gaps_batch& b) {
  gaps_layout L;
  compute_layout(b.n_events, b.capacity, &L);
  char* base = static_cast<char*>(b.workspace);
  Events E{};
  E.px = reinterpret_cast<double*>(base + L.px);
  E.py = reinterpret_cast<double*>(base + L.py);
  E.pz = reinterpret_cast<double*>(base + L.pz);
  E.e = reinterpret_cast<double*>(base + L.e);
  E.flav = reinterpret_cast<int8_t*>(base + L.flav);
  E.col = reinterpret_cast<int16_t*>(base + L.col);
  E.acol = reinterpret_cast<int16_t*>(base + L.acol);
  E.link = reinterpret_cast<uint8_t*>(base + L.link);
  E.dip = reinterpret_cast<float2*>(base + L.dip);
  E.dq2 = reinterpret_cast<double*>(base + L.dq2);
  E.dzp = reinterpret_cast<double*>(base + L.dzp);
  E.dinv = reinterpret_cast<double*>(base + L.dinv);
  E.lnt = reinterpret_cast<double*>(base + L.lnt);
  E.t = reinterpret_cast<double*>(base + L.t);
  E.weight = reinterpret_cast<double*>(base + L.weight);
  E.hash = reinterpret_cast<unsigned long long*>(base + L.hash);
  E.n_partons = reinterpret_cast<int32_t*>(base + L.n_partons);
  E.status = reinterpret_cast<int32_t*>(base + L.status);
  E.n_steps = reinterpret_cast<int32_t*>(base + L.n_steps);
  E.n_emissions = reinterpret_cast<int32_t*>(base + L.n_emissions);
  E.n_winners = reinterpret_cast<int32_t*>(base + L.n_winners);
  E.n_trials = reinterpret_cast<int32_t*>(base + L.n_trials);
  E.n_dipoles = reinterpret_cast<int32_t*>(base + L.n_dipoles);
  E.next_colour = reinterpret_cast<int32_t*>(base + L.next_colour);
  E.me_flavour = reinterpret_cast<int32_t*>(base + L.me_flavour);
  E.valid = reinterpret_cast<int32_t*>(base + L.valid);
  E.obs = reinterpret_cast<double*>(base + L.obs);
  E.buckets = reinterpret_cast<int*>(base + L.buckets);
  E.order = reinterpret_cast<int*>(base + L.order);
  E.active = reinterpret_cast<int*>(base + L.active);
  E.tasks = reinterpret_cast<EmitTask*>(base + L.tasks);
  E.counters = reinterpret_cast<unsigned long long*>(base + L.counters);
  E.hist = reinterpret_cast<double*>(base + L.hist);
  E.hist_fixed = reinterpret_cast<unsigned long long*>(base + L.hist_fixed);
  E.stats = reinterpret_cast<gaps_stats*>(base + L.stats);
  E.n = b.n_events;
  E.stride = b.n_events;
  E.base = 0;
  E.cap = b.capacity;
  set_layout(E, b.layout, b.n_events, b.capacity);
  return E;
}

// The view of workspace events [a, a + count) of E: same arrays, every
// per-event pointer moved to event a; the per-parton arrays keep their base
// and the view's events are offset by a in their layout.
Events sub_view(const Events& E, int64_t a, int64_t count) {
  Events V = E;
  V.slot_off = E.slot_off + static_cast<int>(a);
  V.lnt += a;
  V.t += a;
  V.weight += a;
  V.hash += a;
  V.n_partons += a;
  V.status += a;
  V.n_steps += a;
  V.n_emissions += a;
  V.n_winners += a;
  V.n_trials += a;
  V.n_dipoles += a;
  V.next_colour += a;
  V.me_flavour += a;
  V.valid += a;
  V.obs += a;
  if (V.job_of) V.job_of += a;
  V.n = count;
  V.base = E.base + a;
  return V;
}

// The launch parameters and event view of a call.  With params, a single-job
// batch whose event j has id first_event + j.  Without, a multi-job batch
// prepared by gaps_set_jobs: every event takes its job's parameters from the
// workspace's job table; the host-side step bound is then only a guard.
int prepare(const gaps_params* params, const gaps_batch* batch, DevParams* P, Events* E, bool pool = false) {
  if (check_batch(batch) != GAPS_OK) return GAPS_ERR_INVALID;
  *E = make_events(*batch);
  if (params) {
    if (gaps_check_params(params) != GAPS_OK) return GAPS_ERR_INVALID;
    *P = make_dev_params(*params, batch->first_event);
    return GAPS_OK;
  }
  gaps_layout L;
  compute_layout(batch->n_events, batch->capacity, &L);
  char* base = static_cast<char*>(batch->workspace);
  E->jobs = reinterpret_cast<const DevParams*>(base + L.jobs);
  E->job_of = reinterpret_cast<const uint16_t*>(base + L.job_of);
  // only the serving pool tracks its jobs' finished events
  E->job_done = pool ? reinterpret_cast<unsigned long long*>(base + L.job_done) : nullptr;
  *P = DevParams{};
  P->max_steps = 0x7fffffff;
  return GAPS_OK;
}

}  // namespace gaps

using namespace gaps;

extern "C" {

size_t gaps_workspace_bytes(int64_t n_events, int32_t capacity) {
  if (!sizes_ok(n_events, capacity)) return 0;
  gaps_layout L;
  compute_layout(n_events, capacity, &L);
  return static_cast<size_t>(L.total_bytes);
}

int gaps_workspace_layout(int64_t n_events, int32_t capacity, gaps_layout* out) {
  if (!out || !sizes_ok(n_events, capacity)) return GAPS_ERR_INVALID;
  compute_layout(n_events, capacity, out);
  return GAPS_OK;
}

int gaps_check_params(const gaps_params* p) {
  if (!p) return GAPS_ERR_INVALID;
  if (!(p->sqrt_s > 0.0) || !std::isfinite(p->sqrt_s)) return GAPS_ERR_INVALID;
  if (!(p->alphas_mz > 0.0) || !std::isfinite(p->alphas_mz)) return GAPS_ERR_INVALID;
  if (!(p->t_cutoff > 0.0) || !(p->t_cutoff < 0.25 * p->sqrt_s * p->sqrt_s)) return GAPS_ERR_INVALID;
  if (p->n_flavours < 1 || p->n_flavours > 5) return GAPS_ERR_INVALID;
  if (p->max_steps < 1) return GAPS_ERR_INVALID;
  if (p->trial_mode != GAPS_TRIALS_PER_KERNEL && p->trial_mode != GAPS_TRIALS_PER_DIPOLE) return GAPS_ERR_INVALID;
  if (!p->fixed_alphas) {
    const double b0 = (33.0 - 2.0 * p->n_flavours) / (12.0 * kPi);
    if (!(1.0 + p->alphas_mz * b0 * std::log(p->t_cutoff / (kMZ * kMZ)) > 0.0)) return GAPS_ERR_INVALID;
  }
  return GAPS_OK;
}

int gaps_generate_me(const gaps_params* params, const gaps_batch* batch, void* stream) {
  DevParams P;
  Events E;
  if (prepare(params, batch, &P, &E) != GAPS_OK) return GAPS_ERR_INVALID;
  const cudaError_t e = launch_me(P, E, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? GAPS_OK : cuda_fail(e);
}

int gaps_shower_step(const gaps_params* params, const gaps_batch* batch, void* stream) {
  DevParams P;
  Events E;
  if (prepare(params, batch, &P, &E) != GAPS_OK) return GAPS_ERR_INVALID;
  const cudaError_t e =
      launch_step_plain(P, E, nullptr, batch->n_events, nullptr, nullptr, nullptr, nullptr,
                        static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? GAPS_OK : cuda_fail(e);
}

int gaps_set_jobs(const gaps_job* jobs, int32_t n_jobs, const gaps_batch* batch, void* stream) {
  if (!jobs || n_jobs < 1 || n_jobs > GAPS_MAX_JOBS || check_batch(batch) != GAPS_OK) return GAPS_ERR_INVALID;
  DevParams table[GAPS_MAX_JOBS];
  int64_t begin[GAPS_MAX_JOBS + 1];
  int64_t at = 0;
  for (int j = 0; j < n_jobs; ++j) {
    const gaps_job& job = jobs[j];
    if (gaps_check_params(&job.params) != GAPS_OK || job.n_events < 0 || job.reserved != 0) return GAPS_ERR_INVALID;
    if (static_cast<uint64_t>(job.first_event) + static_cast<uint64_t>(job.n_events) > 0x100000000ull)
      return GAPS_ERR_INVALID;
    table[j] = make_dev_params(job.params, static_cast<int64_t>(job.first_event) - at);
    begin[j] = at;
    at += job.n_events;
  }
  begin[n_jobs] = at;
  if (at != batch->n_events) return GAPS_ERR_INVALID;
  gaps_layout L;
  compute_layout(batch->n_events, batch->capacity, &L);
  char* base = static_cast<char*>(batch->workspace);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(base + L.jobs, table, sizeof(DevParams) * n_jobs, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(base + L.job_begin, begin, sizeof(int64_t) * (n_jobs + 1), cudaMemcpyHostToDevice, s);
  const unsigned long long count = static_cast<unsigned long long>(n_jobs);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(reinterpret_cast<unsigned long long*>(base + L.counters) + kJobCountWord, &count,
                        sizeof(count), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = launch_fill_job_of(reinterpret_cast<uint16_t*>(base + L.job_of),
                           reinterpret_cast<const int64_t*>(base + L.job_begin), n_jobs, batch->n_events, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the host tables live on this stack
  return e == cudaSuccess ? GAPS_OK : cuda_fail(e);
}

namespace {

constexpr gaps_persistent_config kDefaultPersistent = {128, 8, 0, GAPS_LAYOUT_SOA};

bool config_ok(const gaps_persistent_config& c) {
  const bool threads_ok = c.block_threads == 64 || c.block_threads == 128 || c.block_threads == 256 ||
                          c.block_threads == 512;
  return threads_ok && c.compact_period >= 1 && c.compact_period <= 64 && c.blocks_per_sm >= 0 &&
         c.blocks_per_sm <= 32 && layout_ok(c.layout);
}

// Clear the shower's counters (finished, step-limited, FP64 fallbacks, the
// persistent form's event cursor).
cudaError_t clear_shower_counters(const Events& E, cudaStream_t s) {
  // words 0..8 (word 9 keeps the job count) and the plain form's list and
  // task counts and emission cursors
  cudaError_t e = cudaMemsetAsync(E.counters, 0, 9 * sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(E.counters + kPlainListWord, 0, 7 * sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(E.counters + kPlainEmitCursorWord, 0, 3 * sizeof(unsigned long long), s);
  return e;
}

// Host memory of the plain form's host loop, per host thread: the final
// counters, the host-mapped slots the step launches publish their input
// lengths to ({list, tasks, sequence number}, kSlots of them in rotation),
// and the timing events.  Sequence numbers grow across calls (`next_seq`),
// so a slot never shows a value of an earlier call as current.
struct HostCounters {
  static constexpr int kSlots = 8;
  static constexpr int kSlotWords = 4;
  unsigned long long* words = nullptr;
  unsigned long long* pub = nullptr;      // host view
  unsigned long long* pub_dev = nullptr;  // device view of the same memory
  unsigned long long next_seq = 1;
  std::vector<cudaEvent_t> timing;
  bool ok = false;
  cudaError_t err = cudaSuccess;
};

HostCounters& host_counters() {
  thread_local HostCounters hc;
  if (!hc.ok) {
    hc.err = cudaSuccess;
    if (!hc.words) hc.err = cudaMallocHost(&hc.words, kCounterWords * sizeof(unsigned long long));
    if (hc.err == cudaSuccess && !hc.pub) {
      hc.err = cudaHostAlloc(&hc.pub, HostCounters::kSlots * HostCounters::kSlotWords * sizeof(unsigned long long),
                             cudaHostAllocMapped);
      if (hc.err == cudaSuccess) {
        std::memset(hc.pub, 0, HostCounters::kSlots * HostCounters::kSlotWords * sizeof(unsigned long long));
        void* d = nullptr;
        hc.err = cudaHostGetDevicePointer(&d, hc.pub, 0);
        hc.pub_dev = static_cast<unsigned long long*>(d);
      }
    }
    hc.ok = hc.err == cudaSuccess;
  }
  return hc;
}

// The plain form rebuilds its active list in event order after a launch
// while the list holds at least 1/GAPS_REBUILD_DIV of the batch.
#ifndef GAPS_REBUILD_DIV
#define GAPS_REBUILD_DIV 16
#endif

// Launches the plain form's host loop queues ahead of the one it reads back.
#ifndef GAPS_PLAIN_LOOKAHEAD
#define GAPS_PLAIN_LOOKAHEAD 1
#endif
constexpr int64_t kLookahead = GAPS_PLAIN_LOOKAHEAD;
static_assert(kLookahead >= 1 && kLookahead + 2 <= 8, "lookahead and readback slots");

int shower_impl(const gaps_params* params, const gaps_batch* batch, int mode, int64_t* launches_out,
                double* kernel_ms_out, void* stream) {
  DevParams P;
  Events E;
  if (prepare(params, batch, &P, &E) != GAPS_OK) return GAPS_ERR_INVALID;
  if (mode != GAPS_SHOWER_PLAIN && mode != GAPS_SHOWER_PERSISTENT) return GAPS_ERR_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (launches_out) *launches_out = 0;
  if (kernel_ms_out) *kernel_ms_out = 0.0;
  if (E.n == 0) return GAPS_OK;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cudaError_t e = cudaSuccess;
  if (kernel_ms_out) {
    e = cudaEventCreate(&ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&ev1);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  struct EventGuard {
    cudaEvent_t a, b;
    ~EventGuard() {
      if (a) cudaEventDestroy(a);
      if (b) cudaEventDestroy(b);
    }
  } guard{ev0, ev1};
  e = clear_shower_counters(E, s);
  if (e != cudaSuccess) return cuda_fail(e);
  unsigned long long cnt[2] = {0, 0};  // finished events, events stopped at max_steps
  if (mode == GAPS_SHOWER_PERSISTENT) {
    if (ev0 && (e = cudaEventRecord(ev0, s)) != cudaSuccess) return cuda_fail(e);
    e = launch_shower_persistent(P, E, kDefaultPersistent, s);
    if (e != cudaSuccess) return cuda_fail(e);
    if (ev1 && (e = cudaEventRecord(ev1, s)) != cudaSuccess) return cuda_fail(e);
    e = cudaMemcpyAsync(cnt, E.counters, sizeof(cnt), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e);
    if (ev0) {
      float ms = 0.0f;
      if ((e = cudaEventElapsedTime(&ms, ev0, ev1)) != cudaSuccess) return cuda_fail(e);
      *kernel_ms_out = ms;
    }
    if (launches_out) *launches_out = 1;
    return cnt[1] > 0 ? GAPS_ERR_STEP_LIMIT : GAPS_OK;
  }
  // The host loop of App. C: one step for every active event per launch,
  // and the host checks how many events are still active.  A step runs the
  // select/veto phase of the listed events and the splittings the previous
  // step accepted; each launch writes its vetoed and emitted events to the
  // other half of the active-list double buffer and its accepted emissions
  // to the other half of the task double buffer, and reads its own input
  // lengths on the device.  The host therefore never waits for a launch
  // before queueing the next: it sizes the grids from a count one or two
  // launches old (the number of live events only falls, so that count
  // bounds them).  It learns the counts without a copy on the stream: each
  // launch writes the lengths the previous one left to host-mapped memory
  // as it starts.  An event stops after max_steps cycles and each cycle
  // takes at most two launches, so at most 2 max_steps + 1 launches have
  // work.
  HostCounters& hc = host_counters();
  if (!hc.ok) return cuda_fail(hc.err);
  std::vector<cudaEvent_t>& tev = hc.timing;
  int64_t bound = E.n;  // upper bound on the live events entering the next launch
  int64_t queued = 0;   // launches queued
  int64_t worked = 0;   // launches whose input held events
  const int64_t max_launches = 2 * static_cast<int64_t>(P.max_steps) + 2;
  const unsigned long long seq0 = hc.next_seq;  // launch c publishes launch c - 1's lengths as seq0 + c
  hc.next_seq += static_cast<unsigned long long>(max_launches) + 1;
  auto pub_slot = [&](int64_t c, bool device) {
    const size_t at = static_cast<size_t>(c % HostCounters::kSlots) * HostCounters::kSlotWords;
    return (device ? hc.pub_dev : hc.pub) + at;
  };
  auto enqueue = [&](int64_t c) -> cudaError_t {
    const int in_half = static_cast<int>(c & 1), out_half = 1 - in_half;
    const int* list_in = c == 0 ? nullptr : E.active + static_cast<size_t>(in_half) * E.n;
    int* list_out = E.active + static_cast<size_t>(out_half) * E.n;
    const EmitTask* tasks_in = E.tasks + static_cast<size_t>(in_half) * E.n;
    EmitTask* tasks_out = E.tasks + static_cast<size_t>(out_half) * E.n;
    cudaError_t err = cudaSuccess;
    if (kernel_ms_out) {
      while (static_cast<int64_t>(tev.size()) < 2 * (c + 1)) {
        cudaEvent_t x = nullptr;
        if ((err = cudaEventCreate(&x)) != cudaSuccess) return err;
        tev.push_back(x);
      }
      if ((err = cudaEventRecord(tev[2 * c], s)) != cudaSuccess) return err;
    }
    // Counter words rotate over three launches: launch c reads its input
    // lengths from words c%3, writes its outputs' to (c+1)%3 and clears
    // (c+2)%3 for launch c+1 (never a word that it or a neighbour reads).
    unsigned long long* lw = &E.counters[kPlainListWord];
    unsigned long long* tw = &E.counters[kPlainTaskWord];
    unsigned long long* cw = &E.counters[kPlainEmitCursorWord];
    const int r0 = static_cast<int>(c % 3), r1 = static_cast<int>((c + 1) % 3), r2 = static_cast<int>((c + 2) % 3);
    const StepPublish pub{c == 0 ? nullptr : pub_slot(c - 1, true), seq0 + static_cast<unsigned long long>(c)};
    err = launch_step_deferred(P, E, list_in, c == 0 ? E.n : bound, c == 0 ? nullptr : lw + r0, tasks_in,
                               c == 0 ? 0 : bound, c == 0 ? nullptr : tw + r0, list_out, lw + r1, tasks_out, tw + r1,
                               lw + r2, tw + r2, cw + r0, cw + r2, pub, s);
    if (err != cudaSuccess) return err;
    if (kernel_ms_out && (err = cudaEventRecord(tev[2 * c + 1], s)) != cudaSuccess) return err;
    // While the list is long, put it back in event order (appends scatter
    // it); the same events, so its length stands.
    if (bound * GAPS_REBUILD_DIV >= E.n &&
        (err = launch_list_active(E, list_out, &E.counters[kListScratchWord], s)) != cudaSuccess)
      return err;
    return cudaSuccess;
  };
  // The live events launch c leaves, once launch c + 1 has published them
  // (or, for the last queued launch, once the stream has drained).
  auto live_after = [&](int64_t c) -> cudaError_t {
    if (c + 1 >= queued) {
      cudaError_t err = cudaMemcpyAsync(hc.words, E.counters, kCounterWords * sizeof(unsigned long long),
                                        cudaMemcpyDeviceToHost, s);
      if (err == cudaSuccess) err = cudaStreamSynchronize(s);
      const int r1 = static_cast<int>((c + 1) % 3);
      bound = static_cast<int64_t>(hc.words[kPlainListWord + r1] + hc.words[kPlainTaskWord + r1]);
      return err;
    }
    volatile unsigned long long* w = pub_slot(c, false);
    const unsigned long long want = seq0 + static_cast<unsigned long long>(c) + 1;
    for (uint64_t spin = 1; w[2] != want; ++spin) {
      if ((spin & 1023) != 0) continue;
      // every 1024 polls: has the stream failed, or drained without it?
      const cudaError_t q = cudaStreamQuery(s);
      if (q == cudaSuccess && w[2] != want) return cudaErrorUnknown;
      if (q != cudaSuccess && q != cudaErrorNotReady) return q;
    }
    std::atomic_thread_fence(std::memory_order_acquire);
    bound = static_cast<int64_t>(w[0] + w[1]);
    return cudaSuccess;
  };
  if ((e = enqueue(queued++)) != cudaSuccess) return cuda_fail(e);
  for (int64_t c = 0;; ++c) {
    // c: the oldest launch not yet read back; keep kLookahead more queued
    // behind it, so the GPU has work while the host waits for the counts
    while (queued < max_launches && queued <= c + kLookahead)
      if ((e = enqueue(queued++)) != cudaSuccess) return cuda_fail(e);
    if ((e = live_after(c)) != cudaSuccess) return cuda_fail(e);
    worked = c + 1;
    if (bound == 0 || queued >= max_launches) break;
  }
  // The launches queued after the last one with work have empty inputs; the
  // counters after the last queued launch are final.
  e = cudaMemcpyAsync(hc.words, E.counters, kCounterWords * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e);
  cnt[0] = hc.words[0];
  cnt[1] = hc.words[1];
  double total_ms = 0.0;
  if (kernel_ms_out) {
    for (int64_t c = 0; c < worked; ++c) {
      float ms = 0.0f;
      if ((e = cudaEventElapsedTime(&ms, tev[2 * c], tev[2 * c + 1])) != cudaSuccess) return cuda_fail(e);
      total_ms += ms;
    }
  }
  if (launches_out) *launches_out = worked;
  if (kernel_ms_out) *kernel_ms_out = total_ms;
  return cnt[1] > 0 ? GAPS_ERR_STEP_LIMIT : GAPS_OK;
}

}  // namespace

int gaps_shower(const gaps_params* params, const gaps_batch* batch, int mode, int64_t* launches_out,
                void* stream) {
  return shower_impl(params, batch, mode, launches_out, nullptr, stream);
}

int gaps_shower_timed(const gaps_params* params, const gaps_batch* batch, int mode, int64_t* launches_out,
                      double* kernel_ms_out, void* stream) {
  return shower_impl(params, batch, mode, launches_out, kernel_ms_out, stream);
}

int gaps_shower_persistent(const gaps_params* params, const gaps_batch* batch,
                           const gaps_persistent_config* cfg, void* stream) {
  DevParams P;
  Events E;
  if (prepare(params, batch, &P, &E) != GAPS_OK) return GAPS_ERR_INVALID;
  const gaps_persistent_config c = cfg ? *cfg : kDefaultPersistent;
  if (!config_ok(c)) return GAPS_ERR_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (E.n == 0) return GAPS_OK;
  cudaError_t e = clear_shower_counters(E, s);
  if (e == cudaSuccess) e = launch_shower_persistent(P, E, c, s);
  return e == cudaSuccess ? GAPS_OK : cuda_fail(e);
}

int gaps_autotune_persistent(const gaps_params* params, const gaps_batch* batch, gaps_persistent_config* best,
                             double* best_ms, void* stream) {
  DevParams P;
  Events E;
  if (!best || prepare(params, batch, &P, &E) != GAPS_OK) return GAPS_ERR_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  *best = kDefaultPersistent;
  best->layout = batch->layout;
  if (best_ms) *best_ms = 0.0;
  if (E.n == 0) return GAPS_OK;
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  double best_time = -1.0;
  const int layouts[3] = {GAPS_LAYOUT_SOA, GAPS_LAYOUT_TILE8, GAPS_LAYOUT_TILE32};
  const int threads[3] = {128, 256, 512};
  const int periods[4] = {2, 4, 8, 16};
  for (int li = 0; li < 3 && e == cudaSuccess; ++li) {
    // the same workspace read in another record layout (sized for all)
    gaps_batch bl = *batch;
    bl.layout = layouts[li];
    if (prepare(params, &bl, &P, &E) != GAPS_OK) {
      e = cudaErrorInvalidValue;
      break;
    }
    for (int ti = 0; ti < 3 && e == cudaSuccess; ++ti) {
      for (int pi = 0; pi < 4 && e == cudaSuccess; ++pi) {
        const gaps_persistent_config c = {threads[ti], periods[pi], 0, layouts[li]};
        float shape_ms = -1.0f;  // the better of two timings of the shape
        for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
          e = launch_me(P, E, s);
          if (e == cudaSuccess) e = clear_shower_counters(E, s);
          if (e == cudaSuccess) e = cudaEventRecord(a, s);
          if (e == cudaSuccess) e = launch_shower_persistent(P, E, c, s);
          if (e == cudaSuccess) e = cudaEventRecord(b, s);
          if (e == cudaSuccess) e = cudaEventSynchronize(b);
          float ms = 0.0f;
          if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
          if (e == cudaSuccess && (shape_ms < 0.0f || ms < shape_ms)) shape_ms = ms;
        }
        if (e == cudaSuccess && (best_time < 0.0 || shape_ms < best_time)) {
          best_time = shape_ms;
          *best = c;
        }
      }
    }
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (e != cudaSuccess) return cuda_fail(e);
  if (best_ms) *best_ms = best_time;
  return GAPS_OK;
}

int gaps_validate(const gaps_params* params, const gaps_batch* batch, void* stream) {
  DevParams P;
  Events E;
  if (prepare(params, batch, &P, &E) != GAPS_OK) return GAPS_ERR_INVALID;
  const cudaError_t e = launch_validate(P, E, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? GAPS_OK : cuda_fail(e);
}

int gaps_observables(const gaps_params* params, const gaps_batch* batch, void* stream) {
  DevParams P;
  Events E;
  if (prepare(params, batch, &P, &E) != GAPS_OK) return GAPS_ERR_INVALID;
  const cudaError_t e = launch_observables(P, E, E.buckets, E.order, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? GAPS_OK : cuda_fail(e);
}

int gaps_histograms(const gaps_params* params, const gaps_batch* batch, double* hist_device, void* stream) {
  DevParams P;
  Events E;
  if (!hist_device || prepare(params, batch, &P, &E) != GAPS_OK) return GAPS_ERR_INVALID;
  const cudaError_t e = launch_histograms(P, nullptr, E, hist_device, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? GAPS_OK : cuda_fail(e);
}

int gaps_histograms_fixed(const gaps_params* params, const gaps_batch* batch, uint64_t* acc_device, void* stream) {
  DevParams P;
  Events E;
  if (!acc_device || prepare(params, batch, &P, &E) != GAPS_OK) return GAPS_ERR_INVALID;
  const cudaError_t e = launch_hist_fixed(P, nullptr, E, reinterpret_cast<unsigned long long*>(acc_device),
                                          static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? GAPS_OK : cuda_fail(e);
}

int gaps_hist_fixed_scales(const gaps_params* params, int32_t* k_w, int32_t* k_w2) {
  if (!params || !k_w || !k_w2 || gaps_check_params(params) != GAPS_OK) return GAPS_ERR_INVALID;
  int a = 0, b = 0;
  hist_scales(make_dev_params(*params, 0), &a, &b);
  *k_w = a;
  *k_w2 = b;
  return GAPS_OK;
}

int gaps_hist_fixed_to_double(const gaps_params* params, const uint64_t* acc_host, double* hist_host) {
  if (!params || !acc_host || !hist_host || gaps_check_params(params) != GAPS_OK) return GAPS_ERR_INVALID;
  const DevParams d = make_dev_params(*params, 0);
  for (int cell = 0; cell < GAPS_N_OBS * GAPS_HIST_ROW; ++cell) {
    const uint64_t* c = acc_host + 5 * cell;
    hist_host[3 * cell + 0] = fixed128_to_double(c[0], c[1], d.hist_sw_inv);
    hist_host[3 * cell + 1] = fixed128_to_double(c[2], c[3], d.hist_sw2_inv);
    hist_host[3 * cell + 2] = static_cast<double>(c[4]);
  }
  return GAPS_OK;
}

int gaps_reduce_stats(const gaps_batch* batch, gaps_stats* stats_device, void* stream) {
  if (check_batch(batch) != GAPS_OK || !stats_device) return GAPS_ERR_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(stats_device, 0, sizeof(gaps_stats), s);
  if (e != cudaSuccess) return cuda_fail(e);
  e = launch_stats(make_events(*batch), stats_device, s);
  return e == cudaSuccess ? GAPS_OK : cuda_fail(e);
}

int gaps_run(const gaps_params* params, const gaps_batch* batch, int mode, double* host_hist,
             gaps_stats* host_stats, void* stream) {
  // single-job batches only: the workspace holds one histogram accumulator
  if (!params || gaps_check_params(params) != GAPS_OK || check_batch(batch) != GAPS_OK || !host_hist)
    return GAPS_ERR_INVALID;
  if (mode != GAPS_SHOWER_PLAIN && mode != GAPS_SHOWER_PERSISTENT) return GAPS_ERR_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Events E = make_events(*batch);
  cudaError_t e = cudaMemsetAsync(E.hist, 0, sizeof(double) * GAPS_HIST_DOUBLES, s);
  if (e != cudaSuccess) return cuda_fail(e);
  int rc = gaps_generate_me(params, batch, stream);
  if (rc != GAPS_OK) return rc;
  int64_t launches = 1;
  if (mode == GAPS_SHOWER_PERSISTENT) {
    rc = gaps_shower_persistent(params, batch, nullptr, stream);  // no host synchronisation
  } else {
    rc = gaps_shower(params, batch, mode, &launches, stream);
  }
  if (rc != GAPS_OK && rc != GAPS_ERR_STEP_LIMIT) return rc;
  rc = gaps_validate(params, batch, stream);
  if (rc != GAPS_OK) return rc;
  rc = gaps_observables(params, batch, stream);
  if (rc != GAPS_OK) return rc;
  rc = gaps_histograms(params, batch, E.hist, stream);
  if (rc != GAPS_OK) return rc;
  rc = gaps_reduce_stats(batch, E.stats, stream);
  if (rc != GAPS_OK) return rc;
  e = cudaMemcpyAsync(host_hist, E.hist, sizeof(double) * GAPS_HIST_DOUBLES, cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_fail(e);
  gaps_stats st{};
  e = cudaMemcpyAsync(&st, E.stats, sizeof(gaps_stats), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_fail(e);
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e);
  st.launches = launches;
  if (host_stats) *host_stats = st;
  return st.n_step_limit > 0 ? GAPS_ERR_STEP_LIMIT : GAPS_OK;
}

// ---------------------------------------------------------- serving pool
// Counter words 10..12 hold the pool's active-list lengths and 18..20 its
// deferred-emission counts: step c reads words 10 + c%3 and 18 + c%3, writes
// its outputs' counts to 10 + (c+1)%3 and 18 + (c+1)%3 and clears
// 10 + (c+2)%3 and 18 + (c+2)%3 for the step after it; the lists are
// active[c%2] and tasks[c%2].  A live event is in one of them.

int gaps_pool_reset(const gaps_batch* pool, void* stream) {
  DevParams P;
  Events E;
  if (prepare(nullptr, pool, &P, &E, true) != GAPS_OK) return GAPS_ERR_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(E.counters, 0, kCounterWords * sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(E.job_done, 0, GAPS_MAX_JOBS * sizeof(unsigned long long), s);
  return e == cudaSuccess ? GAPS_OK : cuda_fail(e);
}

int gaps_pool_admit(const gaps_params* params, int32_t job_slot, int64_t ev_begin, int64_t n_events,
                    uint32_t first_event, const gaps_batch* pool, int64_t cycle, void* stream) {
  DevParams P;
  Events E;
  if (!params || gaps_check_params(params) != GAPS_OK || prepare(nullptr, pool, &P, &E, true) != GAPS_OK)
    return GAPS_ERR_INVALID;
  if (job_slot < 0 || job_slot >= GAPS_MAX_JOBS || ev_begin < 0 || n_events < 0 || cycle < 0 ||
      ev_begin + n_events > pool->n_events ||
      static_cast<uint64_t>(first_event) + static_cast<uint64_t>(n_events) > 0x100000000ull)
    return GAPS_ERR_INVALID;
  if (n_events == 0) return GAPS_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const DevParams job = make_dev_params(*params, static_cast<int64_t>(first_event) - ev_begin);
  // A pageable host-to-device copy returns once the source has been staged.
  cudaError_t e = cudaMemcpyAsync(const_cast<DevParams*>(E.jobs) + job_slot, &job, sizeof(job),
                                  cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(E.job_done + job_slot, 0, sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = launch_set_job(const_cast<uint16_t*>(E.job_of), ev_begin, n_events, job_slot, s);
  if (e == cudaSuccess) e = launch_me(P, sub_view(E, ev_begin, n_events), s);
  if (e == cudaSuccess)
    e = launch_append_range(E.active + static_cast<size_t>(cycle % 2) * E.stride, &E.counters[10 + cycle % 3],
                            ev_begin, n_events, s);
  return e == cudaSuccess ? GAPS_OK : cuda_fail(e);
}

// The launch parameters of a pool call: the live jobs' shared parameters
// (the keyed modes) or none (every parameter from the job table).
int pool_params(const gaps_params* shared, DevParams* P) {
  if (!shared) return GAPS_OK;
  if (gaps_check_params(shared) != GAPS_OK) return GAPS_ERR_INVALID;
  *P = make_dev_params(*shared, 0);
  P->shared_physics = 1;
  return GAPS_OK;
}

int gaps_pool_cycles(const gaps_batch* pool, int64_t first_cycle, int32_t n_cycles, int64_t max_active,
                     const gaps_params* shared, void* stream) {
  DevParams P;
  Events E;
  if (prepare(nullptr, pool, &P, &E, true) != GAPS_OK || pool_params(shared, &P) != GAPS_OK || first_cycle < 0 ||
      n_cycles < 0 || max_active < 0 || max_active > pool->n_events)
    return GAPS_ERR_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (int64_t c = first_cycle; c < first_cycle + n_cycles; ++c) {
    const size_t in = static_cast<size_t>(c % 2) * E.stride, out = static_cast<size_t>((c + 1) % 2) * E.stride;
    const cudaError_t e = launch_step_deferred(
        P, E, E.active + in, max_active, &E.counters[10 + c % 3], E.tasks + in, max_active,
        &E.counters[18 + c % 3], E.active + out, &E.counters[10 + (c + 1) % 3], E.tasks + out,
        &E.counters[18 + (c + 1) % 3], &E.counters[10 + (c + 2) % 3], &E.counters[18 + (c + 2) % 3],
        &E.counters[kPoolEmitCursorWord + c % 3], &E.counters[kPoolEmitCursorWord + (c + 2) % 3],
        StepPublish{nullptr, 0ull}, s);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  return GAPS_OK;
}

int gaps_pool_slice(const gaps_batch* pool, int64_t round, int32_t cycles, int64_t max_active,
                    const gaps_persistent_config* cfg, const gaps_params* shared, void* stream) {
  DevParams P;
  Events E;
  if (prepare(nullptr, pool, &P, &E, true) != GAPS_OK || pool_params(shared, &P) != GAPS_OK || round < 0 ||
      cycles < 1 || cycles > 255 || max_active < 0 || max_active > pool->n_events)
    return GAPS_ERR_INVALID;
  const gaps_persistent_config c = cfg ? *cfg : kDefaultPersistent;
  if (c.compact_period < 1 || !layout_ok(c.layout) || c.blocks_per_sm < 0) return GAPS_ERR_INVALID;
  if (c.block_threads != 64 && c.block_threads != 128 && c.block_threads != 256 && c.block_threads != 512)
    return GAPS_ERR_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t in = static_cast<size_t>(round % 2) * E.stride, out = static_cast<size_t>((round + 1) % 2) * E.stride;
  unsigned long long* out_count = &E.counters[10 + (round + 1) % 3];
  cudaError_t e = cudaMemsetAsync(out_count, 0, sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(&E.counters[kSliceCursorWord], 0, sizeof(unsigned long long), s);
  if (e == cudaSuccess)
    e = launch_shower_slice(P, E, c, E.active + in, max_active, &E.counters[10 + round % 3],
                            &E.counters[kSliceCursorWord], cycles, E.active + out, out_count, s);
  return e == cudaSuccess ? GAPS_OK : cuda_fail(e);
}

int gaps_pool_progress(const gaps_batch* pool, int64_t cycle, int64_t* active_out, uint64_t* job_done_out,
                       void* stream) {
  DevParams P;
  Events E;
  if (prepare(nullptr, pool, &P, &E, true) != GAPS_OK || cycle < 0 || !active_out) return GAPS_ERR_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned long long counts[kCounterWords] = {0};
  cudaError_t e = cudaMemcpyAsync(counts, E.counters, sizeof(counts), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && job_done_out)
    e = cudaMemcpyAsync(job_done_out, E.job_done, GAPS_MAX_JOBS * sizeof(uint64_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e);
  *active_out = static_cast<int64_t>(counts[10 + cycle % 3] + counts[18 + cycle % 3]);
  return GAPS_OK;
}

int gaps_pool_finish(int32_t job_slot, int64_t ev_begin, int64_t n_events, const gaps_batch* pool,
                     double* hist_device, void* stream) {
  DevParams P;
  Events E;
  if (prepare(nullptr, pool, &P, &E, true) != GAPS_OK || !hist_device || job_slot < 0 || job_slot >= GAPS_MAX_JOBS ||
      ev_begin < 0 || n_events < 0 || ev_begin + n_events > pool->n_events)
    return GAPS_ERR_INVALID;
  if (n_events == 0) return GAPS_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Events V = sub_view(E, ev_begin, n_events);
  cudaError_t e = launch_validate(P, V, s);
  if (e == cudaSuccess) e = launch_observables(P, V, E.buckets, E.order, s);
  Events H = V;  // one histogram set: the range is one job, at its scales
  H.jobs = nullptr;
  H.job_of = nullptr;
  if (e == cudaSuccess) e = launch_histograms(P, E.jobs + job_slot, H, hist_device, s);
  return e == cudaSuccess ? GAPS_OK : cuda_fail(e);
}

int gaps_pool_finish_jobs(const int32_t* job_slots, const int64_t* ev_begins, const int64_t* n_events,
                          int32_t n_jobs, const gaps_batch* pool, double* hist_device, void* stream) {
  DevParams P;
  Events E;
  if (prepare(nullptr, pool, &P, &E, true) != GAPS_OK || !hist_device || n_jobs < 0 || n_jobs > GAPS_MAX_JOBS ||
      (n_jobs > 0 && (!job_slots || !ev_begins || !n_events)))
    return GAPS_ERR_INVALID;
  // The position prefix and the first events, checked: slots in range and
  // distinct, ranges inside the pool and disjoint.
  std::vector<int64_t> table(2 * (static_cast<size_t>(n_jobs) + 1), 0);
  int64_t* prefix = table.data();
  int64_t* begin = prefix + n_jobs + 1;
  std::vector<std::pair<int64_t, int64_t>> spans;
  std::vector<char> slot_used(GAPS_MAX_JOBS, 0);
  for (int j = 0; j < n_jobs; ++j) {
    const int32_t slot = job_slots[j];
    const int64_t b = ev_begins[j], n = n_events[j];
    if (slot < 0 || slot >= GAPS_MAX_JOBS || slot_used[slot] || b < 0 || n < 0 || b + n > pool->n_events)
      return GAPS_ERR_INVALID;
    slot_used[slot] = 1;
    prefix[j + 1] = prefix[j] + n;
    begin[j] = b;
    if (n > 0) spans.emplace_back(b, b + n);
  }
  std::sort(spans.begin(), spans.end());
  for (size_t k = 1; k < spans.size(); ++k)
    if (spans[k].first < spans[k - 1].second) return GAPS_ERR_INVALID;
  const int64_t total = prefix[n_jobs];
  if (total == 0) return GAPS_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  gaps_layout L;
  compute_layout(pool->n_events, pool->capacity, &L);
  int64_t* dev = reinterpret_cast<int64_t*>(static_cast<char*>(pool->workspace) + L.finish);
  // a pageable host-to-device copy returns once the source has been staged
  cudaError_t e = cudaMemcpyAsync(dev, table.data(), table.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s);
  const Ranges R{dev, dev + n_jobs + 1, n_jobs};
  Events U = E;  // positions 0 .. total - 1 over the ranges, pool events
  U.n = total;
  if (e == cudaSuccess) e = launch_validate(P, U, s, R);
  if (e == cudaSuccess) e = launch_observables(P, U, E.buckets, E.order, s, R);
  // every job's histograms in its slot's set, at its own scales
  if (e == cudaSuccess)
    e = cudaMemsetAsync(E.hist_fixed, 0, static_cast<size_t>(GAPS_MAX_JOBS) * GAPS_HIST_FIXED_WORDS * sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = launch_hist_fixed(P, nullptr, U, E.hist_fixed, s, R);
  if (e == cudaSuccess) e = launch_hist_finalize(P, nullptr, E.jobs, GAPS_MAX_JOBS, nullptr, E.hist_fixed, hist_device, s);
  return e == cudaSuccess ? GAPS_OK : cuda_fail(e);
}

const char* gaps_strerror(int status) {
  switch (status) {
    case GAPS_OK: return "ok";
    case GAPS_ERR_INVALID: return "invalid argument";
    case GAPS_ERR_CUDA: return "CUDA error";
    case GAPS_ERR_STEP_LIMIT: return "an event reached the veto-cycle limit";
    case GAPS_ERR_NO_DEVICE: return "no usable device";
    default: return "unknown status";
  }
}

const char* gaps_last_cuda_error(void) { return g_cuda_error; }

int gaps_version(void) { return 100; }

}  // extern "C"
