// C-ABI serving scheduler: continuous batching of shower jobs over one
// resident pool (the paper's host driver, Sec. 2 and App. C, turned into a
// request loop).  Jobs are submitted as they arrive; every step (an explicit
// gaps_server_step, or a gaps_poll of an unfinished job) advances the
// schedule:
//   1. admission, in submission order: a job takes a free job slot and the
//      first free contiguous range of the pool that holds its events (first
//      fit, freed neighbours coalesced); its matrix elements are generated in
//      place and its events join the live active list;
//   2. one round: every live event of every job runs up to cycles_per_round
//      more veto cycles (one persistent launch of the time-sliced form, or
//      that many plain-form steps), in the keyed form when every live job has
//      the same parameters apart from its seed;
//   3. progress, read one round behind from pinned host memory (the live
//      count and every job's finished-event count), so the GPU always has the
//      next round queued while the host looks at the last one;
//   4. the jobs whose events have all finished are finalised together on
//      their ranges (validation, observables, each job's own histograms,
//      copied to the host), and their ranges are reused at once, their slots
//      once the copies have landed.
// All arithmetic runs in the pool entry points (gaps_pool_*); this file keeps
// only the schedule.  Every event equals the event a single-job batch of its
// job produces (draws keyed by seed, event id and the event's own cycle), and
// the histograms are exact fixed-point sums, so a job's results are bitwise
// the same alone and in any mix.
#include <algorithm>
#include <cstring>
#include <deque>
#include <iterator>
#include <map>
#include <set>
#include <unordered_map>
#include <vector>

#include "gaps_launch.hpp"

namespace {

struct Pending {
  gaps_params params;
  int64_t n_events;
  uint32_t first_event;
  uint64_t id;
};

struct Live {
  Pending job;
  int64_t begin;
  int64_t admitted_round;
};

struct Inflight {
  cudaEvent_t done;
  int buf;
  int64_t admitted_at_copy, read_round, cycle;
};

struct Completion {
  cudaEvent_t done;
  int slot;
  uint64_t id;
};

}  // namespace

struct gaps_server {
  gaps_batch pool{};
  gaps_layout layout{};
  double* hist_device = nullptr;  // caller's, max_jobs * GAPS_HIST_DOUBLES
  int max_jobs = 0;
  int cycles_per_round = 8;
  int mode = GAPS_SERVE_SLICE;
  bool has_cfg = false;
  gaps_persistent_config cfg{};
  cudaStream_t stream = nullptr;
  // schedule
  std::map<int64_t, int64_t> free_ranges;  // begin -> length
  std::vector<int> free_slots;
  std::deque<Pending> queue;
  std::map<int, Live> live;
  int64_t cycle = 0, rounds = 0, admitted_events = 0, bound = 0;
  std::deque<Inflight> inflight;
  std::vector<Completion> completions;
  std::unordered_map<uint64_t, std::vector<double>> results;
  std::set<uint64_t> open;  // submitted, not yet reported finished
  uint64_t next_id = 1;
  // pinned host memory: two progress buffers (counters + per-slot finished
  // counts) and one histogram staging set per slot, made on first use
  unsigned long long* progress[2] = {nullptr, nullptr};
  std::vector<double*> staging;
  std::vector<cudaEvent_t> spare_events;
};

namespace {

constexpr int kProgressWords = gaps::kCounterWords + GAPS_MAX_JOBS;

int fail(cudaError_t e) { return gaps::record_cuda_error(e); }

cudaError_t take_event(gaps_server* s, cudaEvent_t* out) {
  if (!s->spare_events.empty()) {
    *out = s->spare_events.back();
    s->spare_events.pop_back();
    return cudaSuccess;
  }
  return cudaEventCreateWithFlags(out, cudaEventDisableTiming);
}

// First fit: the lowest free range that holds n events; -1 if none.
int64_t alloc_range(gaps_server* s, int64_t n) {
  for (auto it = s->free_ranges.begin(); it != s->free_ranges.end(); ++it) {
    if (it->second < n) continue;
    const int64_t b = it->first, len = it->second;
    s->free_ranges.erase(it);
    if (len > n) s->free_ranges[b + n] = len - n;
    return b;
  }
  return -1;
}

void free_range(gaps_server* s, int64_t b, int64_t n) {
  auto next = s->free_ranges.lower_bound(b);
  if (next != s->free_ranges.end() && next->first == b + n) {
    n += next->second;
    s->free_ranges.erase(next);
  }
  auto it = s->free_ranges.lower_bound(b);
  if (it != s->free_ranges.begin()) {
    auto prev = std::prev(it);
    if (prev->first + prev->second == b) {
      prev->second += n;
      return;
    }
  }
  s->free_ranges[b] = n;
}

int admit(gaps_server* s) {
  while (!s->queue.empty() && !s->free_slots.empty()) {
    const Pending& job = s->queue.front();
    const int64_t begin = alloc_range(s, job.n_events);
    if (begin < 0) return GAPS_OK;  // first in, first admitted: wait for room
    const int slot = s->free_slots.back();
    s->free_slots.pop_back();
    const int rc = gaps_pool_admit(&job.params, slot, begin, job.n_events, job.first_event, &s->pool, s->cycle,
                                   s->stream);
    if (rc != GAPS_OK) return rc;
    s->live[slot] = Live{job, begin, s->rounds};
    s->admitted_events += job.n_events;
    s->bound += job.n_events;
    s->queue.pop_front();
  }
  return GAPS_OK;
}

// Whether two jobs shower with the same physics (every parameter but the
// seed).
bool same_physics(const gaps_params& a, const gaps_params& b) {
  return a.sqrt_s == b.sqrt_s && a.alphas_mz == b.alphas_mz && a.t_cutoff == b.t_cutoff &&
         a.n_flavours == b.n_flavours && a.fixed_alphas == b.fixed_alphas && a.max_steps == b.max_steps &&
         a.trial_mode == b.trial_mode;
}

// The live jobs' common parameters, if they share their physics (the pool
// kernels then read only each job's key), else NULL.
const gaps_params* shared_physics(const gaps_server* s) {
  if (s->live.empty()) return nullptr;
  const gaps_params& first = s->live.begin()->second.job.params;
  for (const auto& kv : s->live)
    if (!same_physics(kv.second.job.params, first)) return nullptr;
  return &first;
}

int launch_round(gaps_server* s) {
  const int64_t bound = std::min(s->bound, s->pool.n_events);
  const gaps_params* shared = shared_physics(s);
  int rc;
  if (s->mode == GAPS_SERVE_SLICE) {
    rc = gaps_pool_slice(&s->pool, s->cycle, s->cycles_per_round, bound, s->has_cfg ? &s->cfg : nullptr, shared,
                         s->stream);
    s->cycle += 1;  // slices number the rotation of the pool's lists
  } else {
    rc = gaps_pool_cycles(&s->pool, s->cycle, s->cycles_per_round, bound, shared, s->stream);
    s->cycle += s->cycles_per_round;
  }
  if (rc != GAPS_OK) return rc;
  const int buf = static_cast<int>(s->rounds % 2);
  const char* base = static_cast<const char*>(s->pool.workspace);
  cudaError_t e = cudaMemcpyAsync(s->progress[buf], base + s->layout.counters,
                                  gaps::kCounterWords * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->progress[buf] + gaps::kCounterWords, base + s->layout.job_done,
                        GAPS_MAX_JOBS * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s->stream);
  Inflight f{nullptr, buf, s->admitted_events, s->rounds, s->cycle};
  if (e == cudaSuccess) e = take_event(s, &f.done);
  if (e == cudaSuccess) e = cudaEventRecord(f.done, s->stream);
  if (e != cudaSuccess) return fail(e);
  s->inflight.push_back(f);
  s->rounds += 1;
  return GAPS_OK;
}

int read_round(gaps_server* s) {
  const Inflight f = s->inflight.front();
  s->inflight.pop_front();
  cudaError_t e = cudaEventSynchronize(f.done);
  s->spare_events.push_back(f.done);
  if (e != cudaSuccess) return fail(e);
  const unsigned long long* w = s->progress[f.buf];
  // live events: the active list and the pending emissions of the next step
  const int64_t active = static_cast<int64_t>(w[10 + f.cycle % 3] + w[18 + f.cycle % 3]);
  s->bound = active + (s->admitted_events - f.admitted_at_copy);
  const unsigned long long* done = w + gaps::kCounterWords;
  // the jobs whose events have all finished, finalised together
  std::vector<int32_t> slots;
  std::vector<int64_t> begins, counts;
  for (const auto& kv : s->live) {
    const Live& L = kv.second;
    // a job admitted after this read was enqueued would see the finished
    // count of its slot's previous job
    if (L.admitted_round > f.read_round || done[kv.first] < static_cast<unsigned long long>(L.job.n_events)) continue;
    slots.push_back(kv.first);
    begins.push_back(L.begin);
    counts.push_back(L.job.n_events);
  }
  if (slots.empty()) return GAPS_OK;
  for (int32_t slot : slots) {
    e = cudaMemsetAsync(s->hist_device + static_cast<size_t>(slot) * GAPS_HIST_DOUBLES, 0,
                        GAPS_HIST_DOUBLES * sizeof(double), s->stream);
    if (e != cudaSuccess) return fail(e);
  }
  const int rc = gaps_pool_finish_jobs(slots.data(), begins.data(), counts.data(), static_cast<int32_t>(slots.size()),
                                       &s->pool, s->hist_device, s->stream);
  if (rc != GAPS_OK) return rc;
  for (int32_t slot : slots) {
    const Live& L = s->live.at(slot);
    const double* h = s->hist_device + static_cast<size_t>(slot) * GAPS_HIST_DOUBLES;
    if (!s->staging[slot] && (e = cudaMallocHost(&s->staging[slot], GAPS_HIST_DOUBLES * sizeof(double))) != cudaSuccess)
      return fail(e);
    Completion c{nullptr, slot, L.job.id};
    e = cudaMemcpyAsync(s->staging[slot], h, GAPS_HIST_DOUBLES * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = take_event(s, &c.done);
    if (e == cudaSuccess) e = cudaEventRecord(c.done, s->stream);
    if (e != cudaSuccess) return fail(e);
    s->completions.push_back(c);
    // the range is free for admissions queued after the calls above (same
    // stream); the slot once its histograms are on the host
    free_range(s, L.begin, L.job.n_events);
    s->live.erase(slot);
  }
  return GAPS_OK;
}

int collect(gaps_server* s, bool block) {
  std::vector<Completion> keep;
  for (const Completion& c : s->completions) {
    cudaError_t e = block ? cudaEventSynchronize(c.done) : cudaEventQuery(c.done);
    if (e == cudaErrorNotReady) {
      keep.push_back(c);
      continue;
    }
    if (e != cudaSuccess) return fail(e);
    s->results[c.id].assign(s->staging[c.slot], s->staging[c.slot] + GAPS_HIST_DOUBLES);
    s->free_slots.push_back(c.slot);
    s->spare_events.push_back(c.done);
  }
  s->completions.swap(keep);
  return GAPS_OK;
}

// One step of the schedule.
int step(gaps_server* s) {
  int rc = admit(s);
  if (rc == GAPS_OK && s->bound > 0) rc = launch_round(s);
  if (rc == GAPS_OK && !s->inflight.empty() && (s->inflight.size() >= 2 || s->bound == 0)) rc = read_round(s);
  if (rc == GAPS_OK) rc = collect(s, false);
  // nothing left on the GPU but copies: wait for them
  if (rc == GAPS_OK && s->bound == 0 && s->inflight.empty() && s->live.empty() && !s->completions.empty())
    rc = collect(s, true);
  return rc;
}

}  // namespace

extern "C" {

int gaps_server_create(const gaps_batch* pool, double* hist_device, int32_t max_jobs, int32_t cycles_per_round,
                       int32_t mode, const gaps_persistent_config* cfg, void* stream, gaps_server** out) {
  if (!out) return GAPS_ERR_INVALID;
  *out = nullptr;
  if (!pool || !hist_device || max_jobs < 1 || max_jobs > GAPS_MAX_JOBS || cycles_per_round < 1 ||
      cycles_per_round > 255 || (mode != GAPS_SERVE_SLICE && mode != GAPS_SERVE_STEPS) || pool->n_events < 1 ||
      pool->first_event != 0)
    return GAPS_ERR_INVALID;
  gaps_server* s = new gaps_server();
  s->pool = *pool;
  if (gaps_workspace_layout(pool->n_events, pool->capacity, &s->layout) != GAPS_OK || !pool->workspace ||
      reinterpret_cast<uintptr_t>(pool->workspace) % 256 != 0) {
    delete s;
    return GAPS_ERR_INVALID;
  }
  s->hist_device = hist_device;
  s->max_jobs = max_jobs;
  s->cycles_per_round = cycles_per_round;
  s->mode = mode;
  if (cfg) {
    s->cfg = *cfg;
    s->has_cfg = true;
  }
  s->stream = static_cast<cudaStream_t>(stream);
  s->free_ranges[0] = pool->n_events;
  for (int k = max_jobs - 1; k >= 0; --k) s->free_slots.push_back(k);
  s->staging.assign(max_jobs, nullptr);
  cudaError_t e = cudaSuccess;
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) e = cudaMallocHost(&s->progress[b], kProgressWords * sizeof(unsigned long long));
  if (e != cudaSuccess) {
    gaps_server_destroy(s);
    return fail(e);
  }
  const int rc = gaps_pool_reset(pool, stream);
  if (rc != GAPS_OK) {
    gaps_server_destroy(s);
    return rc;
  }
  *out = s;
  return GAPS_OK;
}

int gaps_submit(gaps_server* s, const gaps_params* params, int64_t n_events, uint32_t first_event, uint64_t* job_id) {
  if (!s || !params || !job_id || gaps_check_params(params) != GAPS_OK || n_events < 1 ||
      n_events > s->pool.n_events || static_cast<uint64_t>(first_event) + static_cast<uint64_t>(n_events) > 0x100000000ull)
    return GAPS_ERR_INVALID;
  const uint64_t id = s->next_id++;
  s->queue.push_back(Pending{*params, n_events, first_event, id});
  s->open.insert(id);
  *job_id = id;
  return GAPS_OK;
}

int gaps_server_step(gaps_server* s, uint64_t* finished_ids, int32_t max_ids, int32_t* n_finished) {
  if (!s || max_ids < 0 || (max_ids > 0 && !finished_ids)) return GAPS_ERR_INVALID;
  const int rc = step(s);
  if (rc != GAPS_OK) return rc;
  int32_t k = 0;
  for (const auto& r : s->results) {
    if (k < max_ids) finished_ids[k] = r.first;
    ++k;
  }
  if (n_finished) *n_finished = k;
  return GAPS_OK;
}

int gaps_poll(gaps_server* s, uint64_t job_id, double* host_hist, int32_t* done) {
  if (!s || !done || s->open.count(job_id) == 0) return GAPS_ERR_INVALID;
  *done = 0;
  auto it = s->results.find(job_id);
  if (it == s->results.end()) {
    const int rc = step(s);
    if (rc != GAPS_OK) return rc;
    it = s->results.find(job_id);
  }
  if (it == s->results.end()) return GAPS_OK;
  if (host_hist) std::memcpy(host_hist, it->second.data(), GAPS_HIST_DOUBLES * sizeof(double));
  s->results.erase(it);
  s->open.erase(job_id);
  *done = 1;
  return GAPS_OK;
}

int gaps_server_counts(const gaps_server* s, int64_t* queued, int64_t* live, int64_t* finished_unread) {
  if (!s) return GAPS_ERR_INVALID;
  if (queued) *queued = static_cast<int64_t>(s->queue.size());
  if (live) *live = static_cast<int64_t>(s->live.size() + s->completions.size());
  if (finished_unread) *finished_unread = static_cast<int64_t>(s->results.size());
  return GAPS_OK;
}

void gaps_server_destroy(gaps_server* s) {
  if (!s) return;
  cudaStreamSynchronize(s->stream);
  for (auto& f : s->inflight) cudaEventDestroy(f.done);
  for (auto& c : s->completions) cudaEventDestroy(c.done);
  for (cudaEvent_t e : s->spare_events) cudaEventDestroy(e);
  for (double* p : s->staging)
    if (p) cudaFreeHost(p);
  for (auto* p : s->progress)
    if (p) cudaFreeHost(p);
  delete s;
}

}  // extern "C"
