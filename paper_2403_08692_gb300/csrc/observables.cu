// Event validation, atomic histogramming of the observables (Sec. 3.2) and
// batch statistics.
#include <algorithm>

#include "gaps_launch.hpp"

namespace gaps {

namespace {

// ------------------------------------------------------------ validation
// Finite / positive tests on the bits of a double: on this part the FP64
// pipe's compares cost as much as its FMAs, the ALU's tests a fraction.
__device__ __forceinline__ bool finite_bits(double x) {
  return ((static_cast<unsigned long long>(__double_as_longlong(x)) >> 52) & 0x7ffull) != 0x7ffull;
}
// x > 0 for a finite x
__device__ __forceinline__ bool positive_finite_bits(double x) { return __double_as_longlong(x) > 0; }
// Unbiased binary exponent of |x| read from its exponent field (-1023 for
// zero and subnormals, 1024 for inf and NaN).
__device__ __forceinline__ int exponent_bits(double x) {
  return static_cast<int>((static_cast<unsigned long long>(__double_as_longlong(x)) >> 52) & 0x7ffull) - 1023;
}

// The on-shell test |m2| > 1e-10 e sqrt(s), decided from exponents where
// they settle it.  For normal e > 0 and sqrt(s) > 0 with unbiased exponents
// u_e, u_s (1e-10 > 2^-34): while both rounded products stay normal
// (u_e >= -988 and u_e + u_s >= -987), the bound (1e-10 e) sqrt(s) is at
// least 2^(-34 + u_e + u_s) (1 - 2^-53)^2 > 2^(-35 + u_e + u_s); and
// |m2| < 2^(u_m + 1).  So u_m <= u_e + u_s - 36 puts |m2| below the bound
// (zero and subnormal m2 included; inf and NaN never pass).  An on-shell
// massless parton has |m2| at rounding level, 2^(2 u_e - 50) or less, and
// u_e <= u_s, so it passes; the rest take the FP64 test.  Saves two
// multiplies and a compare on the FP64 pipe.  u_s is kNoExponent when
// sqrt(s) is not a positive normal number: then every parton takes the FP64
// test.
constexpr int kNoExponent = -4096;
__device__ __forceinline__ int normal_exponent(double x) {
  const int u = exponent_bits(x);
  return positive_finite_bits(x) && u > -1023 && u < 1024 ? u : kNoExponent;
}
__device__ __forceinline__ bool off_shell(double m2, double e, double sqrt_s, int u_s) {
  const int u_e = normal_exponent(e);
  if (u_e >= -988 && u_e + u_s >= -987 && exponent_bits(m2) <= u_e + u_s - 36) return false;
  return fabs(m2) > 1e-10 * e * sqrt_s;
}

// The validation bits of one event: 1 momentum not conserved to 1e-10 GeV, 2 a
// parton off shell (|p^2| > 1e-10 E sqrt(s): every component is formed from
// momenta of the event's scale, so FP64 masslessness holds to ~eps E
// sqrt(s)), 4 non-positive energy, 8 broken colour flow, 16 flavour
// imbalance, 32 non-finite momentum.
__device__ __forceinline__ void validate_event(const DevParams& P0, const Events& E, int64_t ev) {
  const DevParams& P = params_of_event(P0, E, ev);
  // the record holds at most cap partons: a count outside 0..cap (a record
  // written by hand through the workspace views) reads no slot beyond it
  const int n = min(max(E.n_partons[ev], 0), E.cap);
  int bits = 0;
  double se = 0, sx = 0, sy = 0, sz = 0;
  // quark minus antiquark count of flavour f at weight 256^f in one integer:
  // with at most 255 partons every count is below 256 in magnitude, so the
  // sum is zero exactly when every count is (a register, not an indexed
  // array in local memory)
  long long fsum = 0;
  bool colour_ok = true;
  const int u_s = normal_exponent(P.sqrt_s);
  for (int i = 0; i < n; ++i) {
    const size_t a = E.at(i, ev);
    const double e = E.e[a], x = E.px[a], y = E.py[a], z = E.pz[a];
    const bool finite = finite_bits(e) && finite_bits(x) && finite_bits(y) && finite_bits(z);
    if (!finite) bits |= 32;
    se += e;
    sx += x;
    sy += y;
    sz += z;
    if (!(finite_bits(e) ? positive_finite_bits(e) : e > 0.0)) bits |= 4;
    if (off_shell(fma(-z, z, fma(-y, y, fma(-x, x, e * e))), e, P.sqrt_s, u_s)) bits |= 2;
    const int fl = E.flav[a];
    const int c = E.col[a], ac = E.acol[a];
    const int l0 = E.link[E.link_at(0, i, ev)], l1 = E.link[E.link_at(1, i, ev)];
    if (fl == kGluon) {
      colour_ok &= c > 0 && ac > 0;
    } else if (fl >= 1 && fl <= 5) {
      colour_ok &= c > 0 && ac == 0;
      fsum += 1ll << (8 * fl);
    } else if (fl <= -1 && fl >= -5) {
      colour_ok &= c == 0 && ac > 0;
      fsum -= 1ll << (-8 * fl);
    } else {
      colour_ok = false;
    }
    // Colour line c must continue on the partner's anticolour side and back.
    if (c > 0) {
      colour_ok &= l0 != kNoLink && l0 < n;
      if (l0 != kNoLink && l0 < n) {
        colour_ok &= E.acol[E.at(l0, ev)] == c;
        colour_ok &= E.link[E.link_at(1, l0, ev)] == i;
      }
    } else {
      colour_ok &= l0 == kNoLink;
    }
    if (ac > 0) {
      colour_ok &= l1 != kNoLink && l1 < n;
      if (l1 != kNoLink && l1 < n) {
        colour_ok &= E.col[E.at(l1, ev)] == ac;
        colour_ok &= E.link[E.link_at(0, l1, ev)] == i;
      }
    } else {
      colour_ok &= l1 == kNoLink;
    }
  }
  // Every chain runs from a quark to an antiquark; together they visit all
  // partons (no closed gluon loops).
  if (colour_ok) {
    int visited = 0;
    for (int i = 0; i < n && colour_ok; ++i) {
      const int fl = E.flav[E.at(i, ev)];
      if (!(fl >= 1 && fl <= 5)) continue;
      int cur = i;
      for (int guard = 0; guard <= n; ++guard) {
        ++visited;
        const int nxt = E.link[E.link_at(0, cur, ev)];
        if (nxt == kNoLink) break;
        cur = nxt;
      }
      const int fl_end = E.flav[E.at(cur, ev)];
      colour_ok &= fl_end <= -1 && fl_end >= -5;
    }
    colour_ok &= visited == n;
  }
  if (!colour_ok) bits |= 8;
  if (fabs(se - P.sqrt_s) > 1e-10 || fabs(sx) > 1e-10 || fabs(sy) > 1e-10 || fabs(sz) > 1e-10) bits |= 1;
  if (fsum != 0) bits |= 16;
  E.valid[ev] = bits;
}

// One thread per event.  A block first sorts its events by parton count
// (a counting sort in shared memory), so that each warp holds events of
// about one size: a warp's loop over partons lasts as long as its largest
// event's, and on this part an FP64 instruction costs a warp the same issue
// time with one lane active as with 32.  Every event is validated alone, so
// the order changes nothing in the results.  At 10^6 events: 0.200 ms with
// blocks of 128, 0.221 with 256, 0.275 with 512, against 0.249 ms unsorted.
#ifndef GAPS_VALIDATE_THREADS
#define GAPS_VALIDATE_THREADS 128
#endif
constexpr int kValidateThreads = GAPS_VALIDATE_THREADS;

__global__ void __launch_bounds__(kValidateThreads) k_validate(DevParams P0, Events E, Ranges R) {
  __shared__ int s_bin[256];  // counts per parton count, then the first slot of each
  __shared__ int s_pos[kValidateThreads];
  const int tid = threadIdx.x;
  const int64_t first = static_cast<int64_t>(blockIdx.x) * kValidateThreads;
  const int64_t t = first + tid;
  for (int b = tid; b < 256; b += kValidateThreads) s_bin[b] = 0;
  __syncthreads();
  int key = -1, rank = 0;
  if (t < E.n) {
    key = min(max(E.n_partons[R.event(t)], 0), 255);
    rank = atomicAdd(&s_bin[key], 1);
  }
  __syncthreads();
  if (tid < 32) {  // exclusive scan of the 256 counts: 8 per lane, then across the warp
    int c[8], sum = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      c[k] = s_bin[tid * 8 + k];
      sum += c[k];
    }
    int incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (tid >= o) incl += y;
    }
    int run = incl - sum;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      s_bin[tid * 8 + k] = run;
      run += c[k];
    }
  }
  __syncthreads();
  if (key >= 0) s_pos[s_bin[key] + rank] = tid;
  __syncthreads();
  if (first + tid < E.n) validate_event(P0, E, R.event(first + s_pos[tid]));
}

// ---------------------------------------------------------- histograms
// Bin of observable h with value o (log10 y23..y56 on [-4.3, -0.3], 1-T and
// rho_H on [0, 0.5]; 100 bins plus underflow 0 and overflow 101), or -1 when
// the value is undefined.  1-T and rho_H cannot be negative (Sec. 3.1): a
// negative value is an exact zero after rounding and is binned as zero.
// The oracle's FP64 formula.
__device__ __noinline__ int hist_bin_fp64(int h, double o) {
  double x, lo, hi;
  if (h < 4) {
    if (!(o > 0.0)) return -1;
    x = log10(o);
    lo = -4.3;
    hi = -0.3;
  } else {
    x = o > 0.0 ? o : 0.0;
    lo = 0.0;
    hi = h < 6 ? 0.5 : 0.4;
  }
  const double f = (x - lo) / (hi - lo) * GAPS_N_BINS;
  return f < 0.0 ? 0 : (f >= GAPS_N_BINS ? GAPS_N_BINS + 1 : 1 + static_cast<int>(f));
}

// o > 0.0 from the bits of o (false for NaN, true for +inf): the FP64
// pipe's compare costs as much as an FMA on this part.
__device__ __forceinline__ bool positive_bits(double o) {
  const long long b = __double_as_longlong(o);
  return b > 0 && b <= 0x7ff0000000000000ll;
}

// The same bin from an FP32 position: MUFU log2 and the FP32 conversion put
// the position within 1e-4 bins of the FP64 one (|log10 y| <= 10 at 2e-6
// absolute, times 25 bins per decade, plus the FP32 roundings of the
// position, each at most 4e-6 bins; the event shapes at 6e-8 relative, times
// 250 bins per unit at most), so a position more than 2.5e-4 bins from every
// edge is in the FP64 formula's bin; the others (about one value in 2000)
// take the FP64 formula, and with it the whole warp, whose FP64 instructions
// cost the same with one lane active as with 32.
__device__ __forceinline__ int hist_bin(int h, double o) {
  float f;
  const bool pos = positive_bits(o);
  if (h < 4) {
    if (!pos) return -1;
    f = (__log2f(f32_from_f64(o)) * 0.30102999566f + 4.3f) * 25.0f;
  } else {
    // zero (2-parton events) and negative values are the first bin's: the
    // FP64 formula takes x = 0 to position 0 exactly, an edge the screen
    // below would send to the FP64 formula for every such event
    if (!pos) return 1;
    f = f32_from_f64(o) * (h < 6 ? 200.0f : 250.0f);
  }
  const float fr = f - floorf(f);
  if (!(fr > 2.5e-4f && fr < 1.0f - 2.5e-4f) || !(fabsf(f) < 1e6f)) return hist_bin_fp64(h, o);
  return f < 0.0f ? 0 : (f >= GAPS_N_BINS ? GAPS_N_BINS + 1 : 1 + static_cast<int>(f));
}

// ------------------------------------------- fixed-point accumulation
// Weighted fills (sum w, sum w^2, entries) in exact integer arithmetic, so
// the histograms do not depend on the order of the fills (and merge exactly
// across batches or ranks): w is taken in units of 2^-k_w (w 2^k_w rounded
// to an integer, |w 2^k_w| <= 2^62 for every weight the job's matrix element
// can give) and w^2 in units of 2^-k_w2; each cell of acc sums them as
// 128-bit two's-complement integers (low word, high word) and counts its
// entries.
constexpr int kCells = GAPS_N_OBS * GAPS_HIST_ROW;

// Add the signed 128-bit value (lo, hi) to the accumulator at acc[0..1]:
// the low words add atomically, and the carry out of this addition (read
// from the value the low word held) goes to the high word.
__device__ __forceinline__ void add128(unsigned long long* acc, unsigned long long lo, long long hi) {
  const unsigned long long old = atomicAdd(acc, lo);
  const long long up = hi + (old + lo < old ? 1 : 0);
  if (up != 0) atomicAdd(acc + 1, static_cast<unsigned long long>(up));
}

// A block's partial sums of one cell in shared memory take a fill value v
// (|v| <= 2^62) as its low 32 bits (unsigned) and its high part v >> 32
// (signed), summed in separate 64-bit words: v = hi 2^32 + lo, and neither
// sum can overflow for fewer than 2^31 fills, so the adds need no carry and
// no returned value (fire-and-forget shared-memory atomics).  The sum is put
// back together as a 128-bit integer when the block merges into acc.
__device__ __forceinline__ void split_sum_to128(unsigned long long lo_sum, long long hi_sum, unsigned long long* lo,
                                                long long* hi) {
  // hi_sum 2^32 = (hi_sum >> 32) 2^64 + (hi_sum mod 2^32) 2^32
  const unsigned long long low = (static_cast<unsigned long long>(hi_sum) << 32) + lo_sum;
  *hi = (hi_sum >> 32) + (low < lo_sum ? 1 : 0);
  *lo = low;
}

// Every finished valid event fills each observable's bin.  The lanes of a
// warp that fill the same cell are merged first (match on the cell; the
// first lane sums its peers' split fixed-point weights from shared memory),
// so a crowded bin costs one set of atomics per warp, not one per event.
// Each block takes a contiguous chunk of events and accumulates the fills of
// its first event's job (the home job) in shared memory (split form, above),
// merged into that job's set of acc (acc + job * GAPS_HIST_FIXED_WORDS) once
// per block.  Single-job batch (kJobs false): every fill is the home job's,
// at the scales of P, or of *scale_src (a job-table entry on the device) when
// it is given.  Multi-job batch: a job's events lie together, so nearly
// every fill is the home job's; the others go to acc directly as 128-bit
// adds; every event at its own job's scales.
template <bool kJobs>
__global__ void __launch_bounds__(256) k_hist_fixed(DevParams P, const DevParams* scale_src, Events E,
                                                    unsigned long long* acc, Ranges R) {
  // per cell: sum lo(w), sum hi(w), sum lo(w^2), sum hi(w^2), entries
  __shared__ unsigned long long sh[GAPS_HIST_FIXED_WORDS];
  __shared__ long long s_w[256], s_w2[256];
  const int tid = threadIdx.x, lane = tid & 31, warp0 = tid & ~31;
  for (int i = tid; i < GAPS_HIST_FIXED_WORDS; i += blockDim.x) sh[i] = 0ull;
  __syncthreads();
  const int64_t N = E.n;
  const int64_t chunk = ((N + gridDim.x - 1) / gridDim.x + 31) & ~static_cast<int64_t>(31);
  const int64_t b0 = static_cast<int64_t>(blockIdx.x) * chunk;
  const int64_t b1 = b0 + chunk < N ? b0 + chunk : N;
  const int home = kJobs && b0 < N ? static_cast<int>(E.job_of[R.event(b0)]) : 0;
  double sc_w = P.hist_sw, sc_w2 = P.hist_sw2;
  if (!kJobs && scale_src) {
    sc_w = scale_src->hist_sw;
    sc_w2 = scale_src->hist_sw2;
  }
  // every lane of a warp runs the same iterations (the match needs them all)
  for (int64_t base = b0 + warp0; base < b1; base += blockDim.x) {
    const int64_t t = base + lane;
    const int64_t ev = t < b1 ? R.event(t) : 0;
    const bool fill = t < b1 && E.status[ev] == GAPS_DONE && E.valid[ev] == 0;
    const int job = kJobs && fill ? static_cast<int>(E.job_of[ev]) : home;
    if (kJobs && fill) {
      sc_w = E.jobs[job].hist_sw;
      sc_w2 = E.jobs[job].hist_sw2;
    }
    // the event's observables, all loads in flight at once
    double o[GAPS_N_OBS];
#pragma unroll
    for (int h = 0; h < GAPS_N_OBS; ++h) o[h] = fill ? E.obs[h * E.stride + ev] : -1.0;
    const double w = fill ? E.weight[ev] : 0.0;
    // exact scalings by powers of two, then one rounding to an integer
    s_w[tid] = __double2ll_rn(w * sc_w);
    s_w2[tid] = __double2ll_rn((w * w) * sc_w2);
    __syncwarp();
#pragma unroll 1
    for (int h = 0; h < GAPS_N_OBS; ++h) {
      const int bin = fill ? hist_bin(h, o[h]) : -1;
      const int cell = bin < 0 ? -1 : job * kCells + h * GAPS_HIST_ROW + bin;
      const unsigned peers = __match_any_sync(0xffffffffu, cell);
      if (cell >= 0 && lane == __ffs(peers) - 1) {
        unsigned long long lo1 = 0, lo2 = 0;
        long long hi1 = 0, hi2 = 0;
        for (unsigned m = peers; m; m &= m - 1) {
          const int l = __ffs(m) - 1;
          const long long a = s_w[warp0 + l], b = s_w2[warp0 + l];
          lo1 += static_cast<unsigned long long>(a) & 0xffffffffull;
          hi1 += a >> 32;
          lo2 += static_cast<unsigned long long>(b) & 0xffffffffull;
          hi2 += b >> 32;
        }
        if (job == home) {
          unsigned long long* c = sh + static_cast<size_t>(cell - home * kCells) * 5;
          atomicAdd(c + 0, lo1);
          atomicAdd(c + 1, static_cast<unsigned long long>(hi1));
          atomicAdd(c + 2, lo2);
          atomicAdd(c + 3, static_cast<unsigned long long>(hi2));
          atomicAdd(c + 4, static_cast<unsigned long long>(__popc(peers)));
        } else {
          unsigned long long* c = acc + static_cast<size_t>(cell) * 5;
          unsigned long long l128;
          long long h128;
          split_sum_to128(lo1, hi1, &l128, &h128);
          add128(c + 0, l128, h128);
          split_sum_to128(lo2, hi2, &l128, &h128);
          add128(c + 2, l128, h128);
          atomicAdd(c + 4, static_cast<unsigned long long>(__popc(peers)));
        }
      }
    }
    __syncwarp();
  }
  __syncthreads();
  unsigned long long* g_home = acc + static_cast<size_t>(home) * GAPS_HIST_FIXED_WORDS;
  for (int cell = tid; cell < kCells; cell += blockDim.x) {
    const unsigned long long* c = sh + cell * 5;
    if (c[4] == 0ull) continue;
    unsigned long long* g = g_home + cell * 5;
    unsigned long long l128;
    long long h128;
    split_sum_to128(c[0], static_cast<long long>(c[1]), &l128, &h128);
    add128(g + 0, l128, h128);
    split_sum_to128(c[2], static_cast<long long>(c[3]), &l128, &h128);
    add128(g + 2, l128, h128);
    atomicAdd(g + 4, c[4]);
  }
}

// Add the accumulators of sets 0 .. n_sets - 1 (n_sets: *n_sets_dev when
// given) to hist as doubles, set j at hist + j * GAPS_HIST_DOUBLES.  Scales:
// P, or *scale_src, or the job table (multi-job sets).
__global__ void __launch_bounds__(256) k_hist_finalize(DevParams P, const DevParams* scale_src, const DevParams* jobs,
                                                       int n_sets, const unsigned long long* n_sets_dev,
                                                       unsigned long long* acc, double* hist) {
  const int sets = n_sets_dev ? static_cast<int>(*n_sets_dev) : n_sets;
  for (int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; k < static_cast<int64_t>(sets) * kCells;
       k += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int job = static_cast<int>(k / kCells), cell = static_cast<int>(k % kCells);
    const DevParams& S = jobs ? jobs[job] : (scale_src ? *scale_src : P);
    unsigned long long* c = acc + k * 5;
    double* h = hist + static_cast<size_t>(job) * GAPS_HIST_DOUBLES + static_cast<size_t>(cell) * 3;
    if (c[4] != 0ull) {
      h[0] += fixed128_to_double(c[0], c[1], S.hist_sw_inv);
      h[1] += fixed128_to_double(c[2], c[3], S.hist_sw2_inv);
      h[2] += static_cast<double>(c[4]);
    }
  }
}

// Job index of every event of a multi-job batch: job j covers
// [begin[j], begin[j + 1]).
__global__ void __launch_bounds__(256) k_fill_job_of(uint16_t* job_of, const int64_t* begin, int n_jobs, int64_t n) {
  const int64_t ev = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (ev >= n) return;
  int lo = 0, hi = n_jobs - 1;  // last job whose begin <= ev
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (begin[mid] <= ev) lo = mid;
    else hi = mid - 1;
  }
  job_of[ev] = static_cast<uint16_t>(lo);
}

// -------------------------------------------------------------- stats
__global__ void __launch_bounds__(256) k_stats(Events E, gaps_stats* st) {
  long long done = 0, over = 0, lim = 0, inval = 0, steps = 0, mx = 0, trials = 0, wins = 0, ems = 0,
            parts = 0, dips = 0;
  double sw = 0.0, sw2 = 0.0;
  for (int64_t ev = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; ev < E.n;
       ev += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int stt = E.status[ev];
    done += stt == GAPS_DONE;
    over += stt == GAPS_OVERFLOW;
    lim += stt == GAPS_STEP_LIMIT;
    inval += E.valid[ev] != 0;
    const int ns = E.n_steps[ev];
    steps += ns;
    mx = ns > mx ? ns : mx;
    trials += E.n_trials[ev];
    wins += E.n_winners[ev];
    ems += E.n_emissions[ev];
    parts += E.n_partons[ev];
    dips += E.n_dipoles[ev];
    const double w = E.weight[ev];
    sw += w;
    sw2 += w * w;
  }
  // warp reduction, then one atomic per warp
  for (int o = 16; o > 0; o >>= 1) {
    done += __shfl_down_sync(0xffffffffu, done, o);
    over += __shfl_down_sync(0xffffffffu, over, o);
    lim += __shfl_down_sync(0xffffffffu, lim, o);
    inval += __shfl_down_sync(0xffffffffu, inval, o);
    steps += __shfl_down_sync(0xffffffffu, steps, o);
    const long long om = __shfl_down_sync(0xffffffffu, mx, o);
    mx = om > mx ? om : mx;
    trials += __shfl_down_sync(0xffffffffu, trials, o);
    wins += __shfl_down_sync(0xffffffffu, wins, o);
    ems += __shfl_down_sync(0xffffffffu, ems, o);
    parts += __shfl_down_sync(0xffffffffu, parts, o);
    dips += __shfl_down_sync(0xffffffffu, dips, o);
    sw += __shfl_down_sync(0xffffffffu, sw, o);
    sw2 += __shfl_down_sync(0xffffffffu, sw2, o);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0)
    atomicAdd(reinterpret_cast<unsigned long long*>(&st->n_events), static_cast<unsigned long long>(E.n));
  if ((threadIdx.x & 31) == 0) {
    auto add = [](int64_t* p, long long v) {
      if (v) atomicAdd(reinterpret_cast<unsigned long long*>(p), static_cast<unsigned long long>(v));
    };
    add(&st->n_done, done);
    add(&st->n_overflow, over);
    add(&st->n_step_limit, lim);
    add(&st->n_invalid, inval);
    add(&st->sum_steps, steps);
    atomicMax(reinterpret_cast<unsigned long long*>(&st->max_steps), static_cast<unsigned long long>(mx));
    add(&st->sum_trials, trials);
    add(&st->sum_winners, wins);
    add(&st->sum_emissions, ems);
    add(&st->sum_partons, parts);
    add(&st->sum_dipoles, dips);
    atomicAdd(&st->sum_weight, sw);
    atomicAdd(&st->sum_weight2, sw2);
  }
}

}  // namespace

cudaError_t launch_validate(const DevParams& P, const Events& E, cudaStream_t s, const Ranges& R) {
  if (E.n == 0) return cudaSuccess;
  const unsigned blocks = static_cast<unsigned>((E.n + kValidateThreads - 1) / kValidateThreads);
  k_validate<<<blocks, kValidateThreads, 0, s>>>(P, E, R);
  return cudaGetLastError();
}

// Blocks per SM of the single-job histogram kernel: each block merges its
// shared-memory histograms into the global ones at the end.
#ifndef GAPS_HIST_BLOCKS_PER_SM
#define GAPS_HIST_BLOCKS_PER_SM 4
#endif

cudaError_t launch_hist_fixed(const DevParams& P, const DevParams* scale_src, const Events& E, unsigned long long* acc,
                              cudaStream_t s, const Ranges& R) {
  if (E.n == 0) return cudaSuccess;
  int sms = 152;
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (E.n + 255) / 256;
  const int64_t most = static_cast<int64_t>(GAPS_HIST_BLOCKS_PER_SM) * sms;
  if (E.jobs && E.job_of) {
    k_hist_fixed<true><<<static_cast<unsigned>(want < most ? want : most), 256, 0, s>>>(P, nullptr, E, acc, R);
  } else {
    k_hist_fixed<false><<<static_cast<unsigned>(want < most ? want : most), 256, 0, s>>>(P, scale_src, E, acc, R);
  }
  return cudaGetLastError();
}

cudaError_t launch_hist_finalize(const DevParams& P, const DevParams* scale_src, const DevParams* jobs, int n_sets,
                                 const unsigned long long* n_sets_dev, unsigned long long* acc, double* hist,
                                 cudaStream_t s) {
  const int64_t cells = static_cast<int64_t>(n_sets) * kCells;
  const unsigned blocks = static_cast<unsigned>(std::min<int64_t>((cells + 255) / 256, 1024));
  k_hist_finalize<<<blocks, 256, 0, s>>>(P, scale_src, jobs, n_sets, n_sets_dev, acc, hist);
  return cudaGetLastError();
}

cudaError_t launch_histograms(const DevParams& P, const DevParams* scale_src, const Events& E, double* hist,
                              cudaStream_t s) {
  if (E.n == 0) return cudaSuccess;
  const bool multi = E.jobs && E.job_of;
  // every job slot of a multi-job batch (the job count is on the device)
  const size_t sets = multi ? GAPS_MAX_JOBS : 1;
  cudaError_t e = cudaMemsetAsync(E.hist_fixed, 0, sets * GAPS_HIST_FIXED_WORDS * sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = launch_hist_fixed(P, scale_src, E, E.hist_fixed, s);
  if (e == cudaSuccess)
    e = launch_hist_finalize(P, scale_src, multi ? E.jobs : nullptr, multi ? GAPS_MAX_JOBS : 1,
                             multi ? E.counters + kJobCountWord : nullptr, E.hist_fixed, hist, s);
  return e;
}

cudaError_t launch_fill_job_of(uint16_t* job_of, const int64_t* begin, int n_jobs, int64_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_fill_job_of<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(job_of, begin, n_jobs, n);
  return cudaGetLastError();
}

cudaError_t launch_stats(const Events& E, gaps_stats* stats, cudaStream_t s) {
  if (E.n == 0) return cudaSuccess;
  int sms = 152;
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (E.n + 255) / 256;
  const unsigned blocks = static_cast<unsigned>(want < 4 * sms ? want : 4 * sms);
  k_stats<<<blocks, 256, 0, s>>>(E, stats);
  return cudaGetLastError();
}

}  // namespace gaps
