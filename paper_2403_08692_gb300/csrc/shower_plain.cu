// Matrix element + shower initial state (App. B; App. C main program) and the
// plain event-parallel veto cycle (Sec. 2, Fig. 2, App. C).
//
// Plain form: one launch per step with a host all-done check.  A step
// (k_step_deferred) runs SelectWinnerEmission, CheckCutoff and AcceptOrVeto
// (the paper's first three per-cycle kernels and its alpha_s kernel, fused)
// for the events of the active list, one event per group of L lanes, and
// GenerateEmission for the emissions the previous step accepted, in full
// warps; the lists live on the device and the host only sizes the grids and
// reads the live count.  Finished events leave at once (the paper's
// endShower early exit).  k_step_plain, one fused cycle of every event with
// its emissions in the same launch, serves gaps_shower_step.
#include <algorithm>

#include "gaps_launch.hpp"
#include "shower_cycle.cuh"

namespace gaps {

namespace {

template <bool kMulti>
__global__ void __launch_bounds__(256) k_me(DevParams P0, Events E) {
  const int64_t ev = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (ev >= E.n) return;
  const DevParams& P = params_of<kMulti>(P0, E, ev);
  const uint32_t id = event_id(P, E, ev);
  const Uniforms r0 = draw2(P, id, 0, 0, kDrawME);
  const Uniforms r1 = draw2(P, id, 0, 1, kDrawME);
  int fl = 1 + static_cast<int>(r0.a * P.nf);
  fl = fl > P.nf ? P.nf : fl;
  const double cth = 2.0 * r0.b - 1.0;
  double sphi, cphi;
  sincospi(2.0 * r1.a, &sphi, &cphi);
  const double sth = sqrt(1.0 - cth * cth);
  const double en = 0.5 * P.sqrt_s;
  const V4 q{en, en * sth * cphi, en * sth * sphi, en * cth};
  const V4 qbar{en, -q.x, -q.y, -q.z};
  store_p(E, 0, ev, q);
  store_p(E, 1, ev, qbar);
  E.flav[E.at(0, ev)] = static_cast<int8_t>(fl);
  E.flav[E.at(1, ev)] = static_cast<int8_t>(-fl);
  E.col[E.at(0, ev)] = 1;
  E.acol[E.at(0, ev)] = 0;
  E.col[E.at(1, ev)] = 0;
  E.acol[E.at(1, ev)] = 1;
  E.link[E.link_at(0, 0, ev)] = 1;
  E.link[E.link_at(1, 0, ev)] = kNoLink;
  E.link[E.link_at(0, 1, ev)] = kNoLink;
  E.link[E.link_at(1, 1, ev)] = 0;
  const DipoleEntry d = make_dipole(P, 2.0 * mdot(q, qbar));
  store_dipole(E, ev, 0, 0, d);
  store_dipole(E, ev, 1, 1, d);
  E.weight[ev] = fma(P.me_a[fl - 1], fma(cth, cth, 1.0), P.me_b[fl - 1] * cth);
  E.me_flavour[ev] = fl;
  E.t[ev] = P.s;  // starting scale t0 = s
  E.lnt[ev] = P.ln_s;
  E.hash[ev] = kFnvBasis;
  E.n_partons[ev] = 2;
  E.status[ev] = GAPS_ACTIVE;
  E.n_steps[ev] = 0;
  E.n_emissions[ev] = 0;
  E.n_winners[ev] = 0;
  E.n_trials[ev] = 0;
  E.n_dipoles[ev] = 0;
  E.next_colour[ev] = 2;
  E.valid[ev] = 0;
}

// Launch shape of the veto-cycle kernels (compile-time tuning knobs): 64
// threads per block measured fastest for the deferred step at 10^6 events
// (256: +3 %, 128: +0.5 %, 32: +1 %).
#ifndef GAPS_STEP_THREADS
#define GAPS_STEP_THREADS 64
#endif
#ifndef GAPS_STEP_MIN_BLOCKS
#define GAPS_STEP_MIN_BLOCKS (1024 / GAPS_STEP_THREADS)
#endif
// Emission warps of a deferred step launch per SM, at most.
#ifndef GAPS_EMIT_WARPS_PER_SM
#define GAPS_EMIT_WARPS_PER_SM 4
#endif
constexpr int kStepThreads = GAPS_STEP_THREADS;


// One veto cycle over the events list_in[0 .. n_in): the list holds the
// active events only (the previous launch wrote it), so every thread of a
// full block has an event to shower.  Without a list (the first cycle, or a
// single step over the whole batch) the thread of event idx runs it if it is
// still active.  The select/veto phase runs per thread; the accepted
// emissions (about one in ten) are packed into the block's leading threads
// for the emission phase and their dipole refreshes spread over the whole
// block, so the FP64-heavy work runs in full warps.  Surviving events are
// appended to list_out with one atomic per warp (the list order does not
// matter: every draw is keyed by event and cycle).  The host reads
// *out_count to size the next launch and to end the loop; this launch zeroes
// *reset_count, the output counter of the next launch.  Counter word 0 counts
// finished events (the paper's completedEventsCounter), word 1 those stopped
// by the veto-cycle limit.
template <int kMode>
__global__ void __launch_bounds__(kStepThreads, GAPS_STEP_MIN_BLOCKS)
    k_step_plain(DevParams P, Events E, const int* list_in, int64_t n_in, const unsigned long long* n_in_dev,
                 int* list_out, unsigned long long* out_count, unsigned long long* reset_count) {
  __shared__ EmitTask s_task[kStepThreads];
  __shared__ uint32_t s_jobs[kMaxRefresh * kStepThreads];
  __shared__ int s_naccept, s_njobs;
  const int tid = threadIdx.x, lane = tid & 31;
  if (blockIdx.x == 0 && tid == 0 && reset_count) *reset_count = 0ull;
  if (tid == 0) {
    s_naccept = 0;
    s_njobs = 0;
  }
  const int64_t idx = static_cast<int64_t>(blockIdx.x) * kStepThreads + tid;
  // The list length comes from the previous launch when it is on the device
  // (n_in is then only the bound the grid was sized for).
  const int64_t len = n_in_dev ? min(n_in, static_cast<int64_t>(*n_in_dev)) : n_in;
  int64_t ev = -1;
  if (idx < len) ev = list_in ? static_cast<int64_t>(list_in[idx]) : idx;
  const bool active = ev >= 0 && E.status[ev] == GAPS_ACTIVE;
  __syncthreads();
  bool survive = false, finished = false;
  if (active) {
    EmitTask task;
    const int r = cycle_select_veto<kMode>(P, E, ev, task);
    if (r == kCycleAccepted) {
      s_task[atomicAdd(&s_naccept, 1)] = task;
    } else if (r == kCycleFinished) {
      atomicAdd(&E.counters[0], 1ull);
      if (E.status[ev] == GAPS_STEP_LIMIT) atomicAdd(&E.counters[1], 1ull);
      finished = true;
    }
    survive = r != kCycleFinished;
  }
  count_job_done(E, ev, finished);
  if (list_out) {
    const unsigned mask = __ballot_sync(0xffffffffu, survive);
    if (mask != 0u) {
      const int leader = __ffs(mask) - 1;
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(out_count, static_cast<unsigned long long>(__popc(mask)));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (survive) list_out[base + __popc(mask & ((1u << lane) - 1u))] = static_cast<int>(ev);
    }
  }
  __syncthreads();
  if (tid < s_naccept) cycle_emit<kMode>(P, E, s_task[tid], tid, s_jobs, &s_njobs);
  __syncthreads();
  for (int j = tid; j < s_njobs; j += kStepThreads) refresh_dipole<kJobPhysics<kMode>>(P, E, s_task, s_jobs[j]);
}

// Slot of this thread's item in an output list shared by the grid: one
// atomic per warp.  Every lane of the warp must call it; returns -1 where
// flag is false.
__device__ __forceinline__ int64_t warp_append_slot(bool flag, unsigned long long* count) {
  const unsigned mask = __ballot_sync(0xffffffffu, flag);
  if (mask == 0u) return -1;
  const int lane = threadIdx.x & 31, leader = __ffs(mask) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(count, static_cast<unsigned long long>(__popc(mask)));
  base = __shfl_sync(0xffffffffu, base, leader);
  return flag ? static_cast<int64_t>(base + __popc(mask & ((1u << lane) - 1u))) : -1;
}

// One step of the plain form with the emissions deferred by one launch.
// The last select_blocks blocks run SelectWinnerEmission, CheckCutoff and
// AcceptOrVeto for the events list_in[0 .. n_list) (no list: events
// 0 .. n_list), one event per group of L lanes and without a block barrier:
// the group's lanes screen every L-th parton's trials and merge their
// screens exactly (the same winner and bounds as one thread's loop), its
// first lane decides.  A vetoed event goes back to list_out, an accepted
// one leaves its emission in tasks_out, a finished one leaves.  The host
// widens L as the batch thins out, so the last, longest showers do not run
// their whole trial loop in one thread.  The first blocks run
// GenerateEmission for the accepted emissions of the previous launch,
// tasks_in[0 .. n_tasks), one per thread in rounds of a block's worth taken
// from a shared cursor (an SM whose other blocks run slower takes fewer
// rounds), refresh the dipoles they moved block-wide, and put their events
// back in list_out.  They come first so that their long FP64 work starts
// with the launch, beside the select blocks, instead of forming its tail.  Blocks are small (GAPS_STEP_THREADS = 64): a block holds its slot on
// the SM until its slowest warp is done, and the select warps' lengths vary
// with their events' parton counts.  An event
// with a pending emission is in no list, so it never runs two phases in one
// launch, and its history is the one the fused cycle gives (every draw is
// keyed by event and cycle).  Lengths given on the device (n_list_dev,
// n_tasks_dev) replace the host ones, which then only bound them.  The
// launch zeroes *reset_list and *reset_tasks, the output counters of the
// next launch, and publishes its input lengths to the host (pub).
template <int kMode, int L>
__device__ __forceinline__ void select_role(const DevParams& P0, const Events& E, int64_t block,
                                            const int* list_in, int64_t len, int* list_out,
                                            unsigned long long* list_count, EmitTask* tasks_out,
                                            unsigned long long* task_count) {
  const int tid = threadIdx.x;
  constexpr int kGroups = kStepThreads / L;
  const int sub = tid & (L - 1);
  // the host sizes the grid for any lanes choice: one pass
  {
    const int64_t idx = block * kGroups + tid / L;
    int64_t ev = -1;
    if (idx < len) ev = list_in ? static_cast<int64_t>(list_in[idx]) : idx;
    // The event's status, size, cycle and (one lane per event) first parton
    // are loaded together, not one after another: every listed event has
    // slot 0.
    // A multi-job batch's job index is loaded with them.
    constexpr bool kMulti = kJobPhysics<kMode>;
    int status = -1, n = 0, step = 0, job = 0;
    PartonScreen first{};
    if (ev >= 0) {
      status = E.status[ev];
      n = E.n_partons[ev];
      step = E.n_steps[ev];
      if (kJobKey<kMode>) job = E.job_of[ev];
      if (L == 1) first = load_parton_screen(E, ev, 0);
    }
    const bool active = status == GAPS_ACTIVE;
    Screen sc;
    screen_none(sc);
    bool limited = false;
    if (active) {
      const DevParams& P = job_params<kMulti>(P0, E, job);
      limited = step >= P.max_steps;
      if (!limited)
        screen_partons<kMode>(P, E, ev, event_key<kMode>(P, E, ev, job), step, n, sub, L, sc, L == 1 ? &first : nullptr);
    } else {
      n = step = 0;
    }
    screen_group_reduce<L>(sc);  // every lane of the warp, one call site
    const bool lead = active && sub == 0;
    int r = kCycleFinished;
    EmitTask task;
    // The screen's verdict; a cycle it leaves undecided gets the exact FP64
    // selection from the whole warp.
    int verdict = kScreenNone;
    double lnt = 0.0;
    EventKey key{0u, 0u, 0u};
    if (lead && !limited) {
      const DevParams& P = job_params<kMulti>(P0, E, job);
      lnt = E.lnt[ev];
      key = event_key<kMode>(P, E, ev, job);
      verdict = cycle_screen<kMode>(P, E, ev, step, lnt, sc, task);
      if (verdict == kScreenUndecided) atomicAdd(&E.counters[2], 1ull);  // full FP64 cycle
    }
    bool have = verdict == kScreenWinner;
    if (__any_sync(0xffffffffu, verdict == kScreenUndecided))
      fallback_warp<kMode>(P0, E, verdict == kScreenUndecided, ev, job, key, step, n, lnt, have, task);
    if (lead) {
      const DevParams& P = job_params<kMulti>(P0, E, job);
      if (limited) {
        finish_event(E, ev, GAPS_STEP_LIMIT, exp(E.lnt[ev]));
      } else {
        r = cycle_conclude<kMode>(P, E, ev, key, step, n, have, task);
      }
      if (r == kCycleFinished) {
        atomicAdd(&E.counters[0], 1ull);
        if (E.status[ev] == GAPS_STEP_LIMIT) atomicAdd(&E.counters[1], 1ull);
      }
    }
    count_job_done(E, ev, lead && r == kCycleFinished);
    const int64_t at_task = warp_append_slot(lead && r == kCycleAccepted, task_count);
    if (at_task >= 0) {
      tasks_out[at_task] = task;
      E.status[ev] = GAPS_PENDING;
    }
    const int64_t at_list = warp_append_slot(lead && r == kCycleVetoed, list_count);
    if (at_list >= 0) list_out[at_list] = static_cast<int>(ev);
  }
}

// Lanes per event for a list of len events: doubled, up to 32, while
// len x 2 x lanes fits the device's resident threads (so len x lanes stays
// within them).
__host__ __device__ __forceinline__ int lanes_for(int64_t len, int64_t resident) {
  int lanes = 1;
  while (lanes < 32 && len * 2 * lanes <= resident) lanes *= 2;
  return lanes;
}

template <int kMode, int L>
__global__ void __launch_bounds__(kStepThreads, GAPS_STEP_MIN_BLOCKS)
    k_step_deferred(DevParams P0, Events E, int64_t select_blocks, const int* list_in,
                    int64_t n_list, const unsigned long long* n_list_dev, const EmitTask* tasks_in, int64_t n_tasks,
                    const unsigned long long* n_tasks_dev, int* list_out, unsigned long long* list_count,
                    EmitTask* tasks_out, unsigned long long* task_count, unsigned long long* reset_list,
                    unsigned long long* reset_tasks, unsigned long long* emit_cursor,
                    unsigned long long* reset_cursor, StepPublish pub) {
  __shared__ EmitTask s_task[kStepThreads];
  __shared__ uint32_t s_jobs[kMaxRefresh * kStepThreads];
  __shared__ int s_njobs;
  __shared__ unsigned long long s_base;
  const int tid = threadIdx.x;
  if (blockIdx.x == 0 && tid == 0) {
    E.counters[kListScratchWord] = 0ull;  // the cursor of a list rebuild after this launch
    if (reset_list) *reset_list = 0ull;
    if (reset_tasks) *reset_tasks = 0ull;
    if (reset_cursor) *reset_cursor = 0ull;
    if (pub.slot) {
      // the lengths are final: the launch that wrote them has finished
      volatile unsigned long long* w = pub.slot;
      w[0] = n_list_dev ? *n_list_dev : static_cast<unsigned long long>(n_list);
      w[1] = n_tasks_dev ? *n_tasks_dev : static_cast<unsigned long long>(n_tasks);
      __threadfence_system();
      w[2] = pub.seq;
    }
  }
  const int64_t emit_blocks = static_cast<int64_t>(gridDim.x) - select_blocks;
  if (static_cast<int64_t>(blockIdx.x) >= emit_blocks) {
    const int64_t len = n_list_dev ? min(n_list, static_cast<int64_t>(*n_list_dev)) : n_list;
    select_role<kMode, L>(P0, E, static_cast<int64_t>(blockIdx.x) - emit_blocks, list_in, len, list_out, list_count,
                          tasks_out, task_count);
    return;
  }
  const int64_t len = n_tasks_dev ? min(n_tasks, static_cast<int64_t>(*n_tasks_dev)) : n_tasks;
  for (;;) {
    __syncthreads();  // the previous round is done with s_task, s_jobs and s_base
    if (tid == 0) {
      s_njobs = 0;
      s_base = atomicAdd(emit_cursor, static_cast<unsigned long long>(kStepThreads));
    }
    __syncthreads();
    const int64_t base = static_cast<int64_t>(s_base);
    if (base >= len) break;
    const int64_t k = base + tid;
    const bool has = k < len;
    if (has) s_task[tid] = tasks_in[k];
    __syncthreads();
    if (has) cycle_emit<kMode>(P0, E, s_task[tid], tid, s_jobs, &s_njobs);
    __syncthreads();
    for (int j = tid; j < s_njobs; j += kStepThreads) refresh_dipole<kJobPhysics<kMode>>(P0, E, s_task, s_jobs[j]);
    if (has) E.status[s_task[tid].ev] = GAPS_ACTIVE;
    const int64_t at_list = warp_append_slot(has, list_count);
    if (at_list >= 0) list_out[at_list] = s_task[tid].ev;
  }
}

// The active list rebuilt in event order: the events of [0, n) with status
// GAPS_ACTIVE (live and without a pending emission), each block's in order,
// one atomic per block.  Appends scatter a warp's events over the batch as
// the cycles go by; in event order a warp's events sit in one window of a
// block's events, so its loads of the slot-major record coalesce again.
// Each thread takes four consecutive events (one 16-byte load of their
// statuses where the array allows it), a block of 256 threads 1024 events.
__global__ void __launch_bounds__(256) k_list_active(Events E, int64_t n, int* list, unsigned long long* count) {
  __shared__ int s_warp[8];
  __shared__ unsigned long long s_base;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t ev0 = (static_cast<int64_t>(blockIdx.x) * 256 + tid) * 4;
  int st[4] = {-1, -1, -1, -1};
  if (ev0 + 3 < n && (reinterpret_cast<uintptr_t>(E.status) & 15u) == 0u) {
    const int4 v = *reinterpret_cast<const int4*>(E.status + ev0);
    st[0] = v.x;
    st[1] = v.y;
    st[2] = v.z;
    st[3] = v.w;
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (ev0 + k < n) st[k] = E.status[ev0 + k];
  }
  if (blockIdx.x == 0 && tid == 0) atomicAdd(&E.counters[kRebuildWord], 1ull);  // launches of this kernel
  int mine = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) mine += st[k] == GAPS_ACTIVE ? 1 : 0;
  int incl = mine;  // inclusive scan of the live counts over the warp
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (tid == 0) {
    int run = 0;
    for (int w = 0; w < 8; ++w) {
      const int c = s_warp[w];
      s_warp[w] = run;
      run += c;
    }
    s_base = run ? atomicAdd(count, static_cast<unsigned long long>(run)) : 0ull;
  }
  __syncthreads();
  unsigned long long at = s_base + static_cast<unsigned long long>(s_warp[warp] + incl - mine);
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if (st[k] == GAPS_ACTIVE) list[at++] = static_cast<int>(ev0 + k);
}

}  // namespace

cudaError_t launch_me(const DevParams& P, const Events& E, cudaStream_t s) {
  if (E.n == 0) return cudaSuccess;
  const int threads = 256;
  const unsigned blocks = static_cast<unsigned>((E.n + threads - 1) / threads);
  if (E.jobs)
    k_me<true><<<blocks, threads, 0, s>>>(P, E);
  else
    k_me<false><<<blocks, threads, 0, s>>>(P, E);
  return cudaGetLastError();
}

cudaError_t launch_step_plain(const DevParams& P, const Events& E, const int* list_in, int64_t n_in,
                              const unsigned long long* n_in_dev, int* list_out, unsigned long long* out_count,
                              unsigned long long* reset_count, cudaStream_t s) {
  if (n_in <= 0) return cudaSuccess;
  const unsigned blocks = static_cast<unsigned>((n_in + kStepThreads - 1) / kStepThreads);
  switch (launch_mode(P, E)) {
    case kModeMulti:
    case kModeKeyed:
    case kModeKeyedDipole:  // the job table holds the same parameters
      k_step_plain<kModeMulti>
          <<<blocks, kStepThreads, 0, s>>>(P, E, list_in, n_in, n_in_dev, list_out, out_count, reset_count);
      break;
    case kModeSingleDipole:
      k_step_plain<kModeSingleDipole>
          <<<blocks, kStepThreads, 0, s>>>(P, E, list_in, n_in, n_in_dev, list_out, out_count, reset_count);
      break;
    default:
      k_step_plain<kModeSingleKernel>
          <<<blocks, kStepThreads, 0, s>>>(P, E, list_in, n_in, n_in_dev, list_out, out_count, reset_count);
  }
  return cudaGetLastError();
}

namespace {

// Resident threads the device runs at once (SMs x 1024), queried once per
// device.
int64_t resident_threads() {
  static int64_t cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152 * 1024;
  if (cached[dev] == 0) {
    int sms = 152;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) sms = 152;
    cached[dev] = static_cast<int64_t>(sms) * 1024;
  }
  return cached[dev];
}

}  // namespace

cudaError_t launch_step_deferred(const DevParams& P, const Events& E, const int* list_in, int64_t n_list,
                                 const unsigned long long* n_list_dev, const EmitTask* tasks_in, int64_t n_tasks,
                                 const unsigned long long* n_tasks_dev, int* list_out, unsigned long long* list_count,
                                 EmitTask* tasks_out, unsigned long long* task_count, unsigned long long* reset_list,
                                 unsigned long long* reset_tasks, unsigned long long* emit_cursor,
                                 unsigned long long* reset_cursor, StepPublish pub, cudaStream_t s) {
  // The list length may be read on the device; n_list then bounds it, and
  // the lanes per event follow from the bound (at most one step narrower
  // than the exact length would give, since the bound is one or two launches
  // old).  The select grid covers n_list x lanes threads in one pass; the
  // emission blocks take the tasks in rounds from a cursor, at most
  // GAPS_EMIT_WARPS_PER_SM warps per SM, so that every SM starts with about
  // the same FP64 load and the rest goes to the SMs that free up first.
  const int64_t resident = resident_threads();
  const int lanes = lanes_for(n_list, resident);
  const int64_t select_blocks = (n_list * lanes + kStepThreads - 1) / kStepThreads;
  const int64_t emit_per_sm = std::max(1, 32 * GAPS_EMIT_WARPS_PER_SM / kStepThreads);
  const int64_t emit_blocks = std::min((n_tasks + kStepThreads - 1) / kStepThreads, resident / 1024 * emit_per_sm);
  if (select_blocks + emit_blocks == 0) return cudaSuccess;
  const unsigned grid = static_cast<unsigned>(select_blocks + emit_blocks);
#define GAPS_DEFERRED_CASE(MULTI, LN)                                                                     \
  case LN:                                                                                                \
    k_step_deferred<MULTI, LN><<<grid, kStepThreads, 0, s>>>(P, E, select_blocks, list_in, n_list, n_list_dev, \
                                                             tasks_in, n_tasks, n_tasks_dev, list_out,         \
                                                             list_count, tasks_out, task_count, reset_list,    \
                                                             reset_tasks, emit_cursor, reset_cursor, pub);     \
    break;
#define GAPS_DEFERRED_SWITCH(MULTI)  \
  switch (lanes) {                   \
    GAPS_DEFERRED_CASE(MULTI, 1)     \
    GAPS_DEFERRED_CASE(MULTI, 2)     \
    GAPS_DEFERRED_CASE(MULTI, 4)     \
    GAPS_DEFERRED_CASE(MULTI, 8)     \
    GAPS_DEFERRED_CASE(MULTI, 16)    \
    default:                         \
      GAPS_DEFERRED_CASE(MULTI, 32)  \
  }
  switch (launch_mode(P, E)) {
    case kModeMulti:
      GAPS_DEFERRED_SWITCH(kModeMulti)
      break;
    case kModeKeyed:
      GAPS_DEFERRED_SWITCH(kModeKeyed)
      break;
    case kModeKeyedDipole:
      GAPS_DEFERRED_SWITCH(kModeKeyedDipole)
      break;
    case kModeSingleDipole:
      GAPS_DEFERRED_SWITCH(kModeSingleDipole)
      break;
    default:
      GAPS_DEFERRED_SWITCH(kModeSingleKernel)
  }
#undef GAPS_DEFERRED_SWITCH
#undef GAPS_DEFERRED_CASE
  return cudaGetLastError();
}

namespace {

// Append events base .. base + n of the workspace to an active list.
__global__ void __launch_bounds__(256) k_append_range(int* list, unsigned long long* count, int64_t base, int64_t n) {
  __shared__ unsigned long long s_pos;
  const int64_t first = static_cast<int64_t>(blockIdx.x) * blockDim.x;
  const int64_t take = min(static_cast<int64_t>(blockDim.x), n - first);
  if (take <= 0) return;
  if (threadIdx.x == 0) s_pos = atomicAdd(count, static_cast<unsigned long long>(take));
  __syncthreads();
  if (threadIdx.x < take) list[s_pos + threadIdx.x] = static_cast<int>(base + first + threadIdx.x);
}

// Job index of events base .. base + n of the workspace.
__global__ void __launch_bounds__(256) k_set_job(uint16_t* job_of, int64_t base, int64_t n, int job) {
  const int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k < n) job_of[base + k] = static_cast<uint16_t>(job);
}

}  // namespace

cudaError_t launch_list_active(const Events& E, int* list, unsigned long long* count, cudaStream_t s) {
  if (E.n <= 0) return cudaSuccess;
  k_list_active<<<static_cast<unsigned>((E.n + 1023) / 1024), 256, 0, s>>>(E, E.n, list, count);
  return cudaGetLastError();
}

cudaError_t launch_append_range(int* list, unsigned long long* count, int64_t base, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_append_range<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(list, count, base, n);
  return cudaGetLastError();
}

cudaError_t launch_set_job(uint16_t* job_of, int64_t base, int64_t n, int job, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_set_job<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(job_of, base, n, job);
  return cudaGetLastError();
}

}  // namespace gaps
