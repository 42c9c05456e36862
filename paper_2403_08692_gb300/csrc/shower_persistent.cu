// Persistent shower form: one launch runs every event to the cutoff.
//
// Each block keeps a pool of events, two per thread (one for 512-thread
// blocks).  It runs `period` veto cycles on the pool (select/veto for a
// runnable event of every thread, each warp on its own events with no block
// barrier), generates the period's accepted emissions in packed threads,
// then compacts the still-active events to the front of the pool with warp
// ballots and refills the freed slots from a global event cursor (one
// atomic per block per round).  Events therefore
// leave as soon as they finish -- the paper's cutoff inefficiency (Sec. 2,
// Fig. 3: finished events wait for the last one) disappears -- and no
// lane is spent on a finished event for more than `period` cycles.
//
// Nothing waits on another block: a block exits when its pool is empty and
// the cursor has passed the last event.  Every event stops after at most
// max_steps cycles (step-limit status), so the launch always terminates.
// The per-event cycle is the same code as the plain form's, and every draw
// is keyed by (seed, event, cycle), so both forms give identical events.
#include "gaps_launch.hpp"
#include "shower_cycle.cuh"

namespace gaps {

namespace {

// Butterfly merge of the screens of each aligned group of `lanes` lanes
// (block-uniform; every lane of the warp must call it).
__device__ __forceinline__ void screen_group_reduce_n(Screen& sc, int lanes) {
  for (int off = 1; off < lanes; off <<= 1) {
    Screen o;
    o.best_key = __shfl_xor_sync(0xffffffffu, sc.best_key, off);
    o.best_m = __shfl_xor_sync(0xffffffffu, sc.best_m, off);
    o.others_hi = __shfl_xor_sync(0xffffffffu, sc.others_hi, off);
    o.best_code = __shfl_xor_sync(0xffffffffu, sc.best_code, off);
    o.best_hi = __shfl_xor_sync(0xffffffffu, sc.best_hi, off);
    o.best_lo = __shfl_xor_sync(0xffffffffu, sc.best_lo, off);
    o.best_aux = __shfl_xor_sync(0xffffffffu, sc.best_aux, off);
    o.trials = __shfl_xor_sync(0xffffffffu, sc.trials, off);
    o.dipoles = __shfl_xor_sync(0xffffffffu, sc.dipoles, off);
    screen_merge(sc, o);
  }
}

// Launch shape knob: resident threads per SM the register budget is set for
// (0: no bound).
#ifndef GAPS_PERSIST_THREADS_PER_SM
#define GAPS_PERSIST_THREADS_PER_SM 1024
#endif
constexpr int persist_min_blocks(int t) {
  return GAPS_PERSIST_THREADS_PER_SM > 0 && GAPS_PERSIST_THREADS_PER_SM / t > 0 ? GAPS_PERSIST_THREADS_PER_SM / t : 1;
}

// Slot states of a pool: dead, live, live with an emission waiting in the
// block's queue.
enum : uint8_t { kSlotDead = 0, kSlotLive = 1, kSlotPending = 2 };

// Where a launch takes its events from and how far it runs them.  Whole
// batch (kSlice false): events 0 .. E.n - 1 to the cutoff, cursor in counter
// word 6.  Slice (kSlice true): the events of list_in (length *n_in_dev, at
// most n_in), each for at most `cycles` veto cycles; those still active then
// go to list_out (one atomic per warp).
struct SliceArgs {
  const int* list_in;
  const unsigned long long* n_in_dev;
  int64_t n_in;
  unsigned long long* cursor;
  int cycles;
  int* list_out;
  unsigned long long* out_count;
};

// Pool slots per thread.  With two, a thread runs whichever of its events
// can run this cycle, so a lane idles only when both of its events have
// finished or wait for their emission (with one, finished and waiting
// events hold their lanes until the next compaction).  Shared memory bounds
// a block's pool at 512 events.
#ifndef GAPS_PERSIST_SLOTS
#define GAPS_PERSIST_SLOTS 2
#endif
constexpr int persist_slots(int t) { return t * GAPS_PERSIST_SLOTS <= 512 ? GAPS_PERSIST_SLOTS : 1; }

template <int T, int kMode, bool kSlice>
__global__ void __launch_bounds__(T, persist_min_blocks(T))
    k_shower_persistent(DevParams P0, Events E, int period, SliceArgs sl) {
  // A slice gives every event a fixed number of cycles: with two events per
  // thread each would get about half of them per slice (serving latency
  // measured 30 % higher), so slices keep one.
  constexpr int S = kSlice ? 1 : persist_slots(T);
  constexpr int kPool = S * T;  // events of the block's pool
  __shared__ int32_t s_pool[kPool];
  __shared__ uint8_t s_alive[kPool];
  __shared__ uint8_t s_cyc[kSlice ? kPool : 1];  // cycles run in this slice, per slot
  __shared__ EmitTask s_task[kPool];
  __shared__ uint32_t s_jobs[kMaxRefresh * kPool];
  __shared__ int s_count[6];  // pool size, accepted emissions, lanes per event, refill count, refresh jobs, tail
  __shared__ unsigned long long s_base;
  const int tid = threadIdx.x;
  unsigned long long* cursor = kSlice ? sl.cursor : &E.counters[6];
  const int64_t total = kSlice ? (sl.n_in_dev ? min(sl.n_in, static_cast<int64_t>(*sl.n_in_dev)) : sl.n_in) : E.n;
  int pool = 0;
  bool first = true;
  if (tid == 0) s_count[5] = 0;
  for (;;) {
    // Refill the free slots from the global cursor: one event per thread at
    // first, so that a batch of fewer than two events per resident thread
    // spreads over every block, then up to the whole pool.  Once the cursor
    // has passed the last event the pool only shrinks, and once it fits in
    // half the threads its events get several lanes each (the last, longest
    // showers).
    if (tid == 0) {
      const int want = (first ? T : kPool) - pool;
      unsigned long long base = 0;
      int take = 0;
      if (want > 0 && s_count[5] == 0) {
        base = atomicAdd(cursor, static_cast<unsigned long long>(want));
        const long long left = static_cast<long long>(total) - static_cast<long long>(base);
        take = left <= 0 ? 0 : (left < want ? static_cast<int>(left) : want);
        if (take < want) s_count[5] = 1;
      }
      int lanes = 1;
      if (s_count[5])
        while (lanes < 32 && (pool + take) * 2 * lanes <= T) lanes *= 2;
      s_base = base;
      s_count[3] = take;
      s_count[2] = lanes;
    }
    __syncthreads();
    const int take = s_count[3];
    for (int q = tid; q < kPool; q += T) {
      if (q >= pool && q < pool + take) {
        const int64_t k = static_cast<int64_t>(s_base) + (q - pool);
        s_pool[q] = kSlice ? (sl.list_in ? sl.list_in[k] : static_cast<int32_t>(k)) : static_cast<int32_t>(k);
        if constexpr (kSlice) s_cyc[q] = 0;
      }
    }
    pool += take;
    first = false;
    for (int q = tid; q < kPool; q += T) s_alive[q] = q < pool ? kSlotLive : kSlotDead;
    __syncthreads();
    if (pool == 0) break;
    const int lanes = s_count[2];
    const int g = tid / lanes, sub = tid - g * lanes;

    if (tid == 0) {
      s_count[1] = 0;
      s_count[4] = 0;
    }
    __syncthreads();
    // `period` veto cycles with no block barrier: each warp runs its own
    // events, and a cycle's cost is the warp's, not the slowest warp's.  An
    // event whose emission waits in the queue skips its remaining selects of
    // the period (its draws are keyed by its own cycle).  With one lane per
    // event a thread owns slots tid, tid + T, ... and runs the first that can
    // run, starting from another slot each cycle; with several lanes (then
    // pool <= T / 2 lanes) a group owns slot g.
    for (int c = 0; c < period; ++c) {
      __syncwarp();  // the group's first lane wrote s_alive / s_cyc last cycle
      int slot = -1;
      if (lanes == 1) {
#pragma unroll
        for (int o = 0; o < S; ++o) {
          const int q = tid + ((c + o) % S) * T;
          bool ok = slot < 0 && q < pool && s_alive[q] == kSlotLive;
          if constexpr (kSlice) ok = ok && s_cyc[q] < sl.cycles;
          if (ok) slot = q;
        }
      } else {
        bool ok = g < pool && s_alive[g] == kSlotLive;
        if constexpr (kSlice) ok = ok && s_cyc[g] < sl.cycles;
        if (ok) slot = g;
      }
      const bool live = slot >= 0;
      const int64_t ev = live ? s_pool[slot] : -1;
      Screen sc;
      screen_none(sc);
      int n = 0, step = 0;
      bool limited = false;
      int job = 0;
      if (live) {
        if (kJobKey<kMode>) job = E.job_of[ev];
        const DevParams& P = job_params<kJobPhysics<kMode>>(P0, E, job);
        n = E.n_partons[ev];
        step = E.n_steps[ev];
        limited = step >= P.max_steps;
        if (!limited) screen_partons<kMode>(P, E, ev, event_key<kMode>(P, E, ev, job), step, n, sub, lanes, sc);
      }
      screen_group_reduce_n(sc, lanes);  // every lane of the block, one call site
      bool finished = false;
      if (live && sub == 0) {
        if constexpr (kSlice) s_cyc[slot] = static_cast<uint8_t>(s_cyc[slot] + 1);
        const DevParams& P = job_params<kJobPhysics<kMode>>(P0, E, job);
        EmitTask task;
        int r = kCycleFinished;
        if (limited) {
          finish_event(E, ev, GAPS_STEP_LIMIT, exp(E.lnt[ev]));
        } else {
          // the rare undecided cycle takes its exact selection serially here:
          // the warp-wide form (fallback_warp) measured slower in this kernel
          // (its spills cost more than the waits it saves)
          r = cycle_decide<kMode>(P, E, ev, event_key<kMode>(P, E, ev, job), step, n, E.lnt[ev], sc, task);
        }
        if (r == kCycleAccepted) {
          task.pad0 = static_cast<uint8_t>(slot & 255);  // pool slot, to release it after the emission
          task.pad1 = static_cast<uint8_t>(slot >> 8);
          s_alive[slot] = kSlotPending;
          s_task[atomicAdd(&s_count[1], 1)] = task;
        } else if (r == kCycleFinished) {
          s_alive[slot] = kSlotDead;
          atomicAdd(&E.counters[0], 1ull);
          if (E.status[ev] == GAPS_STEP_LIMIT) atomicAdd(&E.counters[1], 1ull);
          finished = true;
        }
      }
      count_job_done(E, ev, finished);
    }
    __syncthreads();
    // GenerateEmission for the period's accepted emissions, in full warps,
    // before the pool is compacted (at most one per event: queued <= kPool).
    const int queued = s_count[1];
    if (queued > 0) {
      for (int q = tid; q < queued; q += T) cycle_emit<kMode>(P0, E, s_task[q], q, s_jobs, &s_count[4]);
      __syncthreads();
      for (int j = tid; j < s_count[4]; j += T) refresh_dipole<kJobPhysics<kMode>>(P0, E, s_task, s_jobs[j]);
      for (int q = tid; q < queued; q += T) s_alive[s_task[q].pad0 | (s_task[q].pad1 << 8)] = kSlotLive;
      __syncthreads();
    }

    // Compact: the still-active events move to the front of the pool; in a
    // slice, those that have run their cycles leave for list_out.  Every
    // slot is read before any is written.
    bool alive[S];
    int32_t mine[S];
    uint8_t my_cyc[S];
#pragma unroll
    for (int o = 0; o < S; ++o) {
      const int q = tid + o * T;
      alive[o] = q < pool && s_alive[q] == kSlotLive;
      mine[o] = alive[o] ? s_pool[q] : 0;
      my_cyc[o] = 0;
      if constexpr (kSlice) {
        my_cyc[o] = q < pool ? s_cyc[q] : 0;
        const bool done = alive[o] && my_cyc[o] >= sl.cycles;
        const unsigned dmask = __ballot_sync(0xffffffffu, done);
        if (dmask) {
          const int lane = tid & 31, leader = __ffs(dmask) - 1;
          unsigned long long at = 0;
          if (lane == leader) at = atomicAdd(sl.out_count, static_cast<unsigned long long>(__popc(dmask)));
          at = __shfl_sync(0xffffffffu, at, leader);
          if (done) sl.list_out[at + __popc(dmask & ((1u << lane) - 1u))] = mine[o];
        }
        alive[o] = alive[o] && !done;
      }
    }
    if (tid == 0) s_count[0] = 0;
    __syncthreads();
    int at[S];
#pragma unroll
    for (int o = 0; o < S; ++o) {
      const unsigned mask = __ballot_sync(0xffffffffu, alive[o]);
      int base = 0;
      if ((tid & 31) == 0 && mask) base = atomicAdd(&s_count[0], __popc(mask));
      base = __shfl_sync(0xffffffffu, base, 0);
      at[o] = base + __popc(mask & ((1u << (tid & 31)) - 1u));
    }
    __syncthreads();
#pragma unroll
    for (int o = 0; o < S; ++o) {
      if (alive[o]) {
        s_pool[at[o]] = mine[o];
        if constexpr (kSlice) s_cyc[at[o]] = my_cyc[o];
      }
    }
    pool = s_count[0];
    __syncthreads();
  }
}

template <int T, int kMode, bool kSlice>
cudaError_t launch_t(const DevParams& P, const Events& E, int period, int blocks_per_sm, const SliceArgs& sl,
                     cudaStream_t s) {
  int dev = 0, sms = 0, fit = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, k_shower_persistent<T, kMode, kSlice>, T, 0);
  if (e != cudaSuccess) return e;
  if (fit < 1) fit = 1;
  const int per_sm = blocks_per_sm > 0 && blocks_per_sm < fit ? blocks_per_sm : fit;
  int64_t blocks = static_cast<int64_t>(sms) * per_sm;
  const int64_t needed = ((kSlice ? sl.n_in : E.n) + T - 1) / T;  // one event per thread to start
  if (blocks > needed) blocks = needed;
  if (blocks == 0) return cudaSuccess;
  k_shower_persistent<T, kMode, kSlice><<<static_cast<unsigned>(blocks), T, 0, s>>>(P, E, period, sl);
  return cudaGetLastError();
}

template <int kMode, bool kSlice>
cudaError_t launch_shape_m(const DevParams& P, const Events& E, const gaps_persistent_config& cfg, const SliceArgs& sl,
                           cudaStream_t s) {
  const int k = cfg.compact_period, b = cfg.blocks_per_sm;
  switch (cfg.block_threads) {
    case 64: return launch_t<64, kMode, kSlice>(P, E, k, b, sl, s);
    case 128: return launch_t<128, kMode, kSlice>(P, E, k, b, sl, s);
    case 256: return launch_t<256, kMode, kSlice>(P, E, k, b, sl, s);
    case 512: return launch_t<512, kMode, kSlice>(P, E, k, b, sl, s);
    default: return cudaErrorInvalidValue;
  }
}

template <bool kSlice>
cudaError_t launch_shape(const DevParams& P, const Events& E, const gaps_persistent_config& cfg, const SliceArgs& sl,
                         cudaStream_t s) {
  switch (launch_mode(P, E)) {
    case kModeKeyed:
      if constexpr (kSlice) return launch_shape_m<kModeKeyed, kSlice>(P, E, cfg, sl, s);
      return launch_shape_m<kModeMulti, kSlice>(P, E, cfg, sl, s);  // the job table holds the same parameters
    case kModeKeyedDipole:
      if constexpr (kSlice) return launch_shape_m<kModeKeyedDipole, kSlice>(P, E, cfg, sl, s);
      return launch_shape_m<kModeMulti, kSlice>(P, E, cfg, sl, s);
    case kModeMulti: return launch_shape_m<kModeMulti, kSlice>(P, E, cfg, sl, s);
    case kModeSingleDipole: return launch_shape_m<kModeSingleDipole, kSlice>(P, E, cfg, sl, s);
    default: return launch_shape_m<kModeSingleKernel, kSlice>(P, E, cfg, sl, s);
  }
}

}  // namespace

cudaError_t launch_shower_persistent(const DevParams& P, const Events& E, const gaps_persistent_config& cfg,
                                     cudaStream_t s) {
  if (E.n == 0) return cudaSuccess;
  return launch_shape<false>(P, E, cfg, SliceArgs{}, s);
}

cudaError_t launch_shower_slice(const DevParams& P, const Events& E, const gaps_persistent_config& cfg,
                                const int* list_in, int64_t n_in, const unsigned long long* n_in_dev,
                                unsigned long long* cursor, int cycles, int* list_out, unsigned long long* out_count,
                                cudaStream_t s) {
  if (n_in == 0 || cycles < 1 || cycles > 255) return n_in == 0 ? cudaSuccess : cudaErrorInvalidValue;
  gaps_persistent_config c = cfg;
  if (c.compact_period > cycles) c.compact_period = cycles;  // no slot idles past its last cycle
  const SliceArgs sl{list_in, n_in_dev, n_in, cursor, cycles, list_out, out_count};
  return launch_shape<true>(P, E, c, sl, s);
}

}  // namespace gaps
