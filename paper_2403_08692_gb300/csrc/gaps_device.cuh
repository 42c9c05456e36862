// Device-side building blocks of the shower library (sm_103a): the Philox
// counter generator, the event-record view over the workspace, physics
// constants, the LO matrix element, the running coupling, the splitting
// kernels and the final-final dipole map.
#pragma once
#include <cstdint>

#include "gaps.h"
#include "log_fp64.cuh"

namespace gaps {

// ------------------------------------------------------------ constants
constexpr double kPi = 3.14159265358979323846;
constexpr double kCF = 4.0 / 3.0;
constexpr double kCA = 3.0;
constexpr double kTR = 0.5;
constexpr double kNc = 3.0;
// Electroweak inputs of the LO matrix element; the paper names none, these
// are the values this library adopts.
constexpr double kMZ = 91.1876;
constexpr double kGammaZ = 2.4952;
constexpr double kAlphaQED = 1.0 / 128.802;
constexpr double kSin2W = 0.222;
constexpr double kGeV2ToPb = 0.389379e9;
constexpr int kGluon = 21;
constexpr uint8_t kNoLink = 255;

enum : uint32_t { kDrawME = 1, kDrawTrial = 2, kDrawWinner = 3 };
enum : int { kQtoQG = 0, kGtoGG = 1, kGtoQQ = 2 };
// A gluon dipole's per-dipole trial won; its kernel is drawn afterwards.
constexpr int kKindUnchosen = 7;

// Parameters of one launch, derived once on the host from gaps_params.
struct DevParams {
  double sqrt_s, s, tc;
  double alphas_mz, as_over;  // alpha_s(m_Z) and the overestimate alpha_s(t_C)
  double b0;                  // one-loop beta_0 = (33 - 2 n_f) / (12 pi)
  uint32_t seed_lo, seed_hi;
  // Philox key schedule (Weyl sequence of the seed), rounds 0..9: key words
  // rk[2r], rk[2r+1].  It depends on the seed only, so the host forms it once
  // and every round reads its key words from the launch parameters.
  uint32_t rk[20];
  int nf, fixed, max_steps;
  int trial_mode;  // GAPS_TRIALS_PER_KERNEL or GAPS_TRIALS_PER_DIPOLE
  // Set on a pool launch whose live jobs all have these parameters apart
  // from their seeds (and first events): the kernels then read only each
  // job's Philox key and event-id offset from the job table.
  int shared_physics;
  double ln_tc;                       // ln t_C
  double ln_s;                        // ln s, the starting scale of the evolution variable
  double inv_4tc;                     // 1 / (4 t_C)
  double inv_s;                       // 1 / s
  // event weight n_f 2 dsigma/dcos of flavour f: me_a[f-1] (1 + cos^2) + me_b[f-1] cos
  double me_a[5], me_b[5];
  double inv_as2pi_2cf, inv_as2pi_ca;  // 1 / (alpha_s^over/(2 pi) K) of q->qg and g->gg
  // FP32 copies used by the screens
  float tcf, as2pi_f, lg2_tc_f, as_mz_over_f, as_b0_f, ln_mz2_f;
  // Philox event id of batch event ev: ev + id_offset (mod 2^32)
  int64_t id_offset;
  // Fixed-point histogram units: w and w^2 are accumulated as integers
  // w 2^k_w and w^2 2^k_w2 (hist_sw = 2^k_w, hist_sw2 = 2^k_w2, and their
  // inverses), with k chosen so that every weight the job can give stays
  // within 2^62.
  double hist_sw, hist_sw2, hist_sw_inv, hist_sw2_inv;
};

// Everything GenerateEmission needs about an accepted winner (56 bytes:
// workspaces hold fewer than 2^31 events and at most 255 partons each).
struct EmitTask {
  double lnt, q2, zp, inv_ls;
  uint32_t rz_hi, rz_lo;
  int32_t ev, step;
  uint8_t i, k, n, side, kappa, kind, pad0, pad1;
};
constexpr int kEmitTaskBytes = 56;
static_assert(sizeof(EmitTask) == kEmitTaskBytes, "EmitTask layout");
// Device counter words in the workspace; the plain form's active-list and
// deferred-emission lengths rotate over three words each.
constexpr int kCounterWords = 32;
constexpr int kPlainListWord = 21;
constexpr int kPlainTaskWord = 24;
constexpr int kRebuildWord = 27;
// The plain form's list rebuild cursor (cleared by every step launch).
constexpr int kListScratchWord = 7;
constexpr int kSliceCursorWord = 28;
// The deferred step's emission-task cursor, rotating like the lengths:
// plain form words 29..31, serving pool words 13..15.
constexpr int kPlainEmitCursorWord = 29;
constexpr int kPoolEmitCursorWord = 13;
// The number of jobs of a multi-job batch (written by gaps_set_jobs).
constexpr int kJobCountWord = 9;

// The signed 128-bit fixed-point value (lo, hi) times scale_inv (= 2^-k) as
// a double, rounded once to nearest even (the power-of-two scalings are
// exact).  The magnitude is taken first (two's complement), so a small
// negative sum does not cancel against 2^64; a magnitude of 64 bits or
// fewer converts directly, a larger one as its leading 64 bits with every
// lower bit folded into the last (a sticky bit: the conversion rounds 11
// bits above it, so the rounding is that of the whole value).  Host and
// device run the same code.
__host__ __device__ inline double fixed128_to_double(unsigned long long lo, unsigned long long hi, double scale_inv) {
  const bool neg = static_cast<long long>(hi) < 0;
  if (neg) {
    lo = ~lo + 1ull;
    hi = ~hi + (lo == 0ull ? 1ull : 0ull);
  }
  double mag;
  if (hi == 0ull) {
    mag = static_cast<double>(lo);
  } else {
#ifdef __CUDA_ARCH__
    const int bits = 64 - __clzll(static_cast<long long>(hi));  // 1 .. 63
#else
    const int bits = 64 - __builtin_clzll(hi);
#endif
    const unsigned long long top = (hi << (64 - bits)) | (lo >> bits);
    const unsigned long long sticky = (lo << (64 - bits)) != 0ull ? 1ull : 0ull;
    mag = static_cast<double>(top | sticky) * static_cast<double>(1ull << bits);
  }
  return (neg ? -mag : mag) * scale_inv;
}

// Pointers into the workspace (gaps_layout) for one batch.
struct Events {
  double *px, *py, *pz, *e;
  int8_t* flav;
  int16_t *col, *acol;
  uint8_t* link;  // [2][cap][n]
  float2* dip;    // [2][cap][n] dipole cache (see shower_cycle.cuh)
  double *dq2, *dzp, *dinv;  // [2][cap][n] FP64 part of the dipole cache
  double* lnt;               // [n] ln t of the active events
  double *t, *weight;
  unsigned long long* hash;
  int32_t *n_partons, *status, *n_steps, *n_emissions, *n_winners, *n_trials, *n_dipoles, *next_colour,
      *me_flavour, *valid;
  double* obs;  // [GAPS_N_OBS][n]
  int* buckets;  // [769] scratch of the observables' multiplicity buckets
  int* order;    // [n] scratch: finished events ordered by multiplicity
  int* active;   // [2][n] scratch: the plain form's active-event lists
  EmitTask* tasks;  // [2][n] scratch: the plain form's deferred emissions
  unsigned long long* counters;
  double* hist;
  unsigned long long* hist_fixed;  // [GAPS_MAX_JOBS][GAPS_HIST_FIXED_WORDS] fixed-point histogram scratch
  gaps_stats* stats;
  // Multi-job batches: parameters per job and the job of every event
  // (NULL for a single-job batch, whose parameters come with the launch).
  const DevParams* jobs;
  const uint16_t* job_of;
  unsigned long long* job_done;  // [GAPS_MAX_JOBS] finished events per job (multi-job batches)
  int64_t n;       // events in this view
  int64_t stride;  // events in the whole workspace (the row length of the per-event arrays)
  int64_t base;    // workspace index of this view's event 0
  int cap;
  // Record layout of the per-parton arrays (gaps_batch::layout): element
  // (slot, workspace event e) of a [cap] array is at
  //   (e >> tile_shift) * tile_stride + slot * slot_stride + (e & ev_mask),
  // and of a [2][cap] array at the same with 2 tile_stride and slot side * cap
  // + slot.  Structure of arrays: tile_shift 31 (a single tile), slot_stride
  // = the workspace's events, ev_mask all ones.  Tiles of T events: tile_shift
  // log2 T, tile_stride cap T, slot_stride T, ev_mask T - 1.  slot_off is the
  // workspace index of this view's event 0 (the per-parton arrays are never
  // shifted; the per-event ones are).
  // Workspace events number fewer than 2^31, and strides fit 32 bits, so
  // each term is one 32 x 32 -> 64-bit multiply.
  int tile_shift, ev_mask, tile_stride, slot_stride, slot_off;

  // The part of an element's index that depends on the event only.
  __device__ __forceinline__ int64_t event_base(int64_t ev, int tiles) const {
    const int e = static_cast<int>(ev) + slot_off;
    return static_cast<int64_t>(e >> tile_shift) * (tiles * tile_stride) + (e & ev_mask);
  }
  __device__ __forceinline__ size_t at(int slot, int64_t ev) const {
    return static_cast<size_t>(event_base(ev, 1) + static_cast<int64_t>(slot) * slot_stride);
  }
  __device__ __forceinline__ size_t link_at(int side, int slot, int64_t ev) const {
    return static_cast<size_t>(event_base(ev, 2) + static_cast<int64_t>(side * cap + slot) * slot_stride);
  }
};

// The layout fields of a view of n_events events (the workspace's row
// length) with `capacity` slots.
inline void set_layout(Events& E, int layout, int64_t n_events, int capacity) {
  E.slot_off = 0;
  if (layout == GAPS_LAYOUT_TILE8 || layout == GAPS_LAYOUT_TILE32) {
    const int T = layout == GAPS_LAYOUT_TILE8 ? 8 : 32;
    E.tile_shift = layout == GAPS_LAYOUT_TILE8 ? 3 : 5;
    E.tile_stride = capacity * T;
    E.slot_stride = T;
    E.ev_mask = T - 1;
  } else {
    E.tile_shift = 31;  // events < 2^31: one tile
    E.tile_stride = 0;
    E.slot_stride = static_cast<int>(n_events);
    E.ev_mask = 0x7fffffff;
  }
}

// The events a finalisation kernel visits: positions t = 0 .. E.n - 1 of a
// view, or of a list of disjoint event ranges (several finished jobs of a
// serving pool at once): range j holds positions prefix[j] ..
// prefix[j + 1] - 1, events begin[j] .. begin[j] + prefix[j + 1] - prefix[j]
// - 1.  n = 0: the identity.
struct Ranges {
  const int64_t* prefix;  // [n + 1], prefix[0] = 0
  const int64_t* begin;   // [n]
  int n;
  __device__ __forceinline__ int64_t event(int64_t t) const {
    if (n == 0) return t;
    int lo = 0, hi = n - 1;  // the last range whose first position is <= t
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (prefix[mid] <= t) {
        lo = mid;
      } else {
        hi = mid - 1;
      }
    }
    return begin[lo] + (t - prefix[lo]);
  }
};

// The parameters of event ev: its job's in a multi-job batch (kMulti), else
// the launch's.  A compile-time choice, so that single-job kernels read
// their parameters from the kernel-argument bank.
template <bool kMulti>
__device__ __forceinline__ const DevParams& params_of(const DevParams& launch, const Events& E, int64_t ev) {
  if constexpr (kMulti) {
    return E.jobs[E.job_of[ev]];
  } else {
    return launch;
  }
}

// The parameters of a job: the multi-job table's entry `job` (kMulti), else
// the launch's.  For kernels that already hold an event's job index.
template <bool kMulti>
__device__ __forceinline__ const DevParams& job_params(const DevParams& launch, const Events& E, int job) {
  if constexpr (kMulti) {
    return E.jobs[job];
  } else {
    return launch;
  }
}

// Compile-time policy of the shower kernels: a single job with one trial per
// (dipole, kernel), a single job with one trial per dipole, a multi-job
// batch (parameters and trial mode read per event), or a multi-job batch
// whose jobs share their parameters apart from the seed (keyed: the physics
// from the launch, each event's Philox key and id offset from its job, with
// one trial per kernel or per dipole).  Single-job kernels then carry no
// code of the mode they do not run.
enum : int { kModeSingleKernel = 0, kModeSingleDipole = 1, kModeMulti = 2, kModeKeyed = 3, kModeKeyedDipole = 4 };
// Physics parameters from the job table (else from the launch).
template <int kMode>
constexpr bool kJobPhysics = kMode == kModeMulti;
// Philox key and event-id offset from the job table (else from the launch).
template <int kMode>
constexpr bool kJobKey = kMode >= kModeMulti;
template <int kMode>
__device__ __forceinline__ bool per_dipole(const DevParams& P) {
  if constexpr (kMode == kModeMulti) {
    return P.trial_mode == GAPS_TRIALS_PER_DIPOLE;
  } else {
    return kMode == kModeSingleDipole || kMode == kModeKeyedDipole;
  }
}
// The mode of a launch.
inline int launch_mode(const DevParams& P, const Events& E) {
  const bool dipole = P.trial_mode == GAPS_TRIALS_PER_DIPOLE;
  if (!E.jobs) return dipole ? kModeSingleDipole : kModeSingleKernel;
  if (!P.shared_physics) return kModeMulti;
  return dipole ? kModeKeyedDipole : kModeKeyed;
}

// The same choice at run time, for kernels that read the parameters once per
// event.
__device__ __forceinline__ const DevParams& params_of_event(const DevParams& launch, const Events& E, int64_t ev) {
  return E.jobs ? params_of<true>(launch, E, ev) : launch;
}

// The Philox event id (first counter word) of view event ev.
__device__ __forceinline__ uint32_t event_id(const DevParams& P, const Events& E, int64_t ev) {
  return static_cast<uint32_t>(E.base + ev + P.id_offset);
}

// --------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64-bit multiplies with a Weyl-sequence key schedule.
struct U4 {
  uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, const uint32_t* rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c0;
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
    c0 = hi1 ^ c1 ^ rk[2 * r];
    c1 = lo1;
    c2 = hi0 ^ c3 ^ rk[2 * r + 1];
    c3 = lo0;
  }
  return U4{c0, c1, c2, c3};
}

// The same generator with the key schedule formed on the fly from the seed
// words (two additions per round).  Multi-job kernels take their parameters
// from the job table in global memory, where reading twenty round keys per
// call would put a load into every round of the dependent chain.
__device__ __forceinline__ U4 philox10_seed(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                            uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c0;
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
    c0 = hi1 ^ c1 ^ k0;
    c1 = lo1;
    c2 = hi0 ^ c3 ^ k1;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return U4{c0, c1, c2, c3};
}

// An event's random stream: its Philox event id (the first counter word)
// and key.  Single-job kernels take the round keys from the launch (P.rk)
// and leave k0, k1 unused.
struct EventKey {
  uint32_t id, k0, k1;
};

// The stream of view event ev of job `job` (the job is read only in the
// job-keyed modes; P: the event's physics parameters).
template <int kMode>
__device__ __forceinline__ EventKey event_key(const DevParams& P, const Events& E, int64_t ev, int job) {
  if constexpr (kMode == kModeKeyed || kMode == kModeKeyedDipole) {
    const DevParams& K = E.jobs[job];
    return EventKey{static_cast<uint32_t>(E.base + ev + K.id_offset), K.seed_lo, K.seed_hi};
  } else {
    return EventKey{static_cast<uint32_t>(E.base + ev + P.id_offset), P.seed_lo, P.seed_hi};
  }
}

// A draw of counter (event id, c1, c2, c3): round keys from the parameter
// bank (single-job launches), or formed from the seed for keys read from the
// job table.
template <int kMode>
__device__ __forceinline__ U4 philox_draw(const DevParams& P, const EventKey& key, uint32_t c1, uint32_t c2,
                                          uint32_t c3) {
  if constexpr (kJobKey<kMode>) {
    return philox10_seed(key.id, c1, c2, c3, key.k0, key.k1);
  } else {
    return philox10(key.id, c1, c2, c3, P.rk);
  }
}

// 52-bit uniform strictly inside (0, 1): the top 26 bits of each word, plus
// one half, times 2^-52, i.e. (2m + 1) 2^-53 -- exact in binary64, so its
// bits are assembled with integer instructions (the FP64 pipe's conversions
// and adds cost as much as its FMAs on this part).
__device__ __forceinline__ double to_unit(uint32_t hi, uint32_t lo) {
  const unsigned long long m = (static_cast<unsigned long long>(hi >> 6) << 26) | (lo >> 6);
  const unsigned long long odd = (m << 1) | 1ull;  // < 2^53
  const int top = 63 - __clzll(static_cast<long long>(odd));
  const unsigned long long bits = (static_cast<unsigned long long>(top - 53 + 1023) << 52) |
                                  ((odd << (52 - top)) & ((1ull << 52) - 1ull));
  return __longlong_as_double(static_cast<long long>(bits));
}

struct Uniforms {
  double a, b;
};

__device__ __forceinline__ Uniforms draw2(const DevParams& P, uint32_t ev, uint32_t step, uint32_t slot,
                                          uint32_t purpose) {
  const U4 r = philox10(ev, step, slot, purpose, P.rk);
  return Uniforms{to_unit(r.x, r.y), to_unit(r.z, r.w)};
}

// FNV-1a, 64 bit, over the eight little-endian bytes of a decision word.
__device__ __forceinline__ unsigned long long fnv1a64(unsigned long long h, unsigned long long word) {
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    h ^= (word >> (8 * b)) & 0xFFull;
    h *= 1099511628211ull;
  }
  return h;
}
constexpr unsigned long long kFnvBasis = 14695981039346656037ull;

// ------------------------------------------------------------- physics
// One-loop running coupling alpha_s(t); the fixed mode returns alpha_s(m_Z).
__device__ __forceinline__ double alpha_s(const DevParams& P, double t) {
  if (P.fixed) return P.alphas_mz;
  return P.alphas_mz / (1.0 + P.alphas_mz * P.b0 * log_fp64(t / (kMZ * kMZ)));
}

// Splitting kernel P(z, y) and its overestimate P^over(z).
__device__ __forceinline__ double kernel_p(int kind, double z, double y) {
  if (kind == kQtoQG) return kCF * (2.0 / (1.0 - z * (1.0 - y)) - (1.0 + z));
  if (kind == kGtoGG) return 0.5 * kCA * (2.0 / (1.0 - z * (1.0 - y)) - 2.0 + z * (1.0 - z));
  return 0.5 * kTR * (1.0 - 2.0 * z * (1.0 - z));
}
__device__ __forceinline__ double kernel_over(int kind, double z) {
  if (kind == kQtoQG) return 2.0 * kCF / (1.0 - z);
  if (kind == kGtoGG) return kCA / (1.0 - z);
  return 0.5 * kTR;
}
// Coefficient K of the kernel's overestimate: P^over = K / (1 - z) for the
// soft kernels, K for g -> q qbar.
__device__ __forceinline__ double kernel_k(int kind) {
  return kind == kQtoQG ? 2.0 * kCF : (kind == kGtoGG ? kCA : 0.5 * kTR);
}

// Minkowski product.
// Products and sums below are fused only where written as fma: the library
// is compiled without automatic contraction, so each expression rounds the
// same way wherever it is inlined.
__device__ __forceinline__ double mdot(double ae, double ax, double ay, double az, double be, double bx,
                                       double by, double bz) {
  return fma(-az, bz, fma(-ay, by, fma(-ax, bx, ae * be)));
}

struct V4 {
  double e, x, y, z;
};

__device__ __forceinline__ double mdot(const V4& a, const V4& b) {
  return fma(-a.z, b.z, fma(-a.y, b.y, fma(-a.x, b.x, a.e * b.e)));
}

__device__ __forceinline__ double det3(double a1, double a2, double a3, double b1, double b2, double b3,
                                       double c1, double c2, double c3) {
  const double m1 = fma(b2, c3, -(b3 * c2)), m2 = fma(b1, c3, -(b3 * c1)), m3 = fma(b1, c2, -(b2 * c1));
  return fma(a3, m3, fma(-a2, m2, a1 * m1));
}

// Catani-Seymour final-final map for massless splitter a and spectator b:
// p_i = z a + (1-z) y b + k, p_j = (1-z) a + z y b - k, p_b' = (1-y) b,
// k = sqrt(z(1-z) y Q^2) (cos phi n1 + sin phi n2), with n1, n2 unit
// spacelike vectors orthogonal to a, b and each other: n1 projects the
// first of the references (1,1,0,0), (1,0,1,0), (1,0,0,1) whose projection
// has |n1^2| >= 1e-4, n2 is the Minkowski-orthogonal complement of (a, b,
// n1) (cofactor expansion of det[X; a; b; n1]).  n1 is formed scaled by a.b
// (no division) and both normalisations take the library's rsqrt (one ulp):
// the oracle's vectors up to rounding.
__device__ __forceinline__ void dipole_map(const V4& a, const V4& b, double z, double y, double cphi,
                                           double sphi, V4& pi, V4& pj, V4& pb) {
  const double ab = mdot(a, b);
  const double q2 = 2.0 * ab;
  // n1 scaled by a.b (a.b > 0): ab ref - (ref.b) a - (ref.a) b, so no
  // division; the reference test |n1^2| >= 1e-4 becomes |(ab n1)^2| >=
  // 1e-4 ab^2, and the normalisation below removes the scale.
  const double lim = 1e-4 * ab * ab;
  V4 n1{0, 0, 0, 0};
  for (int r = 0; r < 3; ++r) {
    const V4 ref{1.0, r == 0 ? 1.0 : 0.0, r == 1 ? 1.0 : 0.0, r == 2 ? 1.0 : 0.0};
    const double cb = mdot(ref, b);
    const double ca = mdot(ref, a);
    n1 = V4{fma(-ca, b.e, fma(-cb, a.e, ab)), fma(-ca, b.x, fma(-cb, a.x, r == 0 ? ab : 0.0)),
            fma(-ca, b.y, fma(-cb, a.y, r == 1 ? ab : 0.0)), fma(-ca, b.z, fma(-cb, a.z, r == 2 ? ab : 0.0))};
    if (fabs(mdot(n1, n1)) >= lim) break;
  }
  const double s1 = rsqrt(-mdot(n1, n1));
  n1 = V4{n1.e * s1, n1.x * s1, n1.y * s1, n1.z * s1};
  const double c0 = det3(a.x, a.y, a.z, b.x, b.y, b.z, n1.x, n1.y, n1.z);
  const double c1 = -det3(a.e, a.y, a.z, b.e, b.y, b.z, n1.e, n1.y, n1.z);
  const double c2 = det3(a.e, a.x, a.z, b.e, b.x, b.z, n1.e, n1.x, n1.z);
  const double c3 = -det3(a.e, a.x, a.y, b.e, b.x, b.y, n1.e, n1.x, n1.y);
  V4 n2{c0, -c1, -c2, -c3};
  const double s2 = rsqrt(-mdot(n2, n2));
  n2 = V4{n2.e * s2, n2.x * s2, n2.y * s2, n2.z * s2};
  const double kt = sqrt(z * (1.0 - z) * y * q2);
  const double kc = kt * cphi, ks = kt * sphi;
  const V4 k{fma(ks, n2.e, kc * n1.e), fma(ks, n2.x, kc * n1.x), fma(ks, n2.y, kc * n1.y), fma(ks, n2.z, kc * n1.z)};
  const double fa_i = z, fb_i = (1.0 - z) * y, fa_j = 1.0 - z, fb_j = z * y;
  pi = V4{fma(fb_i, b.e, fa_i * a.e) + k.e, fma(fb_i, b.x, fa_i * a.x) + k.x, fma(fb_i, b.y, fa_i * a.y) + k.y,
          fma(fb_i, b.z, fa_i * a.z) + k.z};
  pj = V4{fma(fb_j, b.e, fa_j * a.e) - k.e, fma(fb_j, b.x, fa_j * a.x) - k.x, fma(fb_j, b.y, fa_j * a.y) - k.y,
          fma(fb_j, b.z, fa_j * a.z) - k.z};
  const double r = 1.0 - y;
  pb = V4{r * b.e, r * b.x, r * b.y, r * b.z};
}

// d sigma / d cos(theta) for e+e- -> q qbar (flavour f, PDG 1..5) at LO with
// photon and Z exchange and their interference, in pb; theta is the quark's
// angle to the electron beam.  It is a (1 + cos^2) + b cos: dsigma_parts gives
// a and b (the host tabulates them per job and flavour, the matrix-element
// kernel evaluates the quadratic).
__host__ __device__ inline void dsigma_parts(double s, int f, double* a, double* b) {
  const bool up = (f == 2 || f == 4);
  const double qf = up ? 2.0 / 3.0 : -1.0 / 3.0;
  const double af = up ? 0.5 : -0.5;
  const double vf = af - 2.0 * qf * kSin2W;
  const double qe = -1.0, ae = -0.5, ve = -0.5 + 2.0 * kSin2W;
  const double kappa = 1.0 / (4.0 * kSin2W * (1.0 - kSin2W));
  const double mz2 = kMZ * kMZ;
  const double den = (s - mz2) * (s - mz2) + kGammaZ * kGammaZ * mz2;
  const double chi1 = kappa * s * (s - mz2) / den;
  const double chi2 = kappa * kappa * s * s / den;
  const double even = qe * qe * qf * qf + 2.0 * qe * qf * ve * vf * chi1 + (ae * ae + ve * ve) * (af * af + vf * vf) * chi2;
  const double odd = 2.0 * qe * qf * ae * af * chi1 + 4.0 * ae * ve * af * vf * chi2;
  const double pref = kPi * kAlphaQED * kAlphaQED / (2.0 * s) * kNc * kGeV2ToPb;
  *a = pref * even;
  *b = pref * 2.0 * odd;
}

}  // namespace gaps
