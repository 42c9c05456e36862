// One veto cycle of one event (Sec. 2, App. A, App. C), split in two phases
// and shared by every shower form:
//   cycle_select_veto  SelectWinnerEmission + CheckCutoff + AcceptOrVeto
//   cycle_emit         GenerateEmission for an accepted winner
// The caller runs the first phase for a dense set of active events, queues
// the accepted ones (about one in ten) and runs the second phase on the
// queue, so the FP64-heavy splitting never executes in a warp whose other
// lanes idle.
//
// GB300 runs FP64 at about 1/74 of its FP32 rate, so the cycle spends FP64
// only where the result must be FP64:
//  * Trial screening.  Every trial's scale is ranked by its key
//    log2(t'/t) = log2(r) / c in FP32, from a per-dipole cache of 1/c; each
//    key carries a bound on its FP32 error.  When one trial's key beats every
//    other trial's and the cutoff by more than the bounds, it is the winner
//    the exact FP64 comparison would pick, and only its scale is evaluated in
//    FP64.  Otherwise (about 1e-4 of cycles) the whole cycle is redone with
//    every trial in FP64, exactly as the oracle does it.
//  * Log-space evolution.  The event carries L = ln t; a winner moves it to
//    L + ln(r)/c (Eq. A.6 in logarithms), so a cycle needs one FP64 log and
//    no exp; t itself is formed only for an accepted emission.
//  * Veto.  z, y and the acceptance ratio are formed in FP32 with an error
//    bound; only a veto number within the bound of the ratio is decided in
//    FP64.  z and y are recomputed in FP64 for the accepted emissions.
//  * Dipole cache.  A dipole's trial density depends only on its invariant
//    mass, which changes only when an emission moves one of its partons, so
//    Q^2, z+ and 1/ln(z+/z-) (FP64) and 1/c (FP32) are stored per dipole and
//    recomputed once per dipole an emission touches.
#pragma once
#include "gaps_device.cuh"

namespace gaps {

// Error allowances of the FP32 screens, several times the worst-case error of
// the FP32 operations involved.  Trial key = log2(r) * (1/c): the 24-bit
// uniform is within 2^-22 relative of r (3.4e-7 absolute in log2 r), MUFU
// log2 adds at most 2e-6 (1 + |log2 r|), the cached 1/c is within 1e-6
// relative, the product rounds once; so |key error| <= 2e-6/c + 7e-6 |key|,
// allowed as 4e-6/c + 1.6e-5 |key|.  Veto ratio: z, 1 - z and y from MUFU
// exp/log and ~20 FP32 operations carry <= 1e-5 relative error and (1 - y)
// <= 5e-6 absolute, allowed as 5e-5 (ratio + r) + 2e-5.
constexpr float kKeyRelInvc = 4e-6f;
constexpr float kKeyRelKey = 1.6e-5f;
constexpr float kVetoRel = 5e-5f;
constexpr float kVetoAbs = 2e-5f;

__device__ __forceinline__ V4 load_p(const Events& E, int slot, int64_t ev) {
  const size_t a = E.at(slot, ev);
  return V4{E.e[a], E.px[a], E.py[a], E.pz[a]};
}
__device__ __forceinline__ void store_p(const Events& E, int slot, int64_t ev, const V4& p) {
  const size_t a = E.at(slot, ev);
  E.e[a] = p.e;
  E.px[a] = p.x;
  E.py[a] = p.y;
  E.pz[a] = p.z;
}

__device__ __forceinline__ size_t dip_at(const Events& E, int side, int slot, int64_t ev) {
  return E.link_at(side, slot, ev);
}

// Cache entry of a dipole of invariant mass q2: FP64 Q^2, z+ = (1 + b)/2
// with b = sqrt(1 - 4 t_C/Q^2) (the oracle's formula) and 1/ln(z+/z-) with
// z- = 1 - z+, and the FP32 screen entry x = 1/(a ln(z+/z-)), y = 1/(a T_R/2
// (z+ - z-)), a = alpha_s^over/(2 pi).  x = -1 marks a dipole without phase
// space (Q^2 < 4 t_C, the oracle's FP64 test).  z+/z- = (1 + b)/(1 - b)
// equals (1 + b)^2 Q^2 / (4 t_C) since 1 - b^2 = 4 t_C/Q^2: no division, and
// none of the cancellation in 1 - z+ (the values agree with the oracle's two
// logarithms to about 1e-13 relative at LEP energies).
struct DipoleEntry {
  double q2, zp, inv_ls;
  float2 screen;
};

__device__ __forceinline__ DipoleEntry make_dipole(const DevParams& P, double q2) {
  DipoleEntry d;
  d.q2 = q2;
  if (q2 < 4.0 * P.tc) {
    d.zp = d.inv_ls = 0.0;
    d.screen = make_float2(-1.0f, -1.0f);
    return d;
  }
  // b = sqrt(1 - 4 t_C/Q^2) = a / sqrt(Q^2 a) with a = Q^2 - 4 t_C: one
  // reciprocal square root instead of a division and a square root
  const double a = q2 - 4.0 * P.tc;
  const double b = __double_as_longlong(a) > 0 ? a * rsqrt(q2 * a) : 0.0;  // a > 0, tested on the bits
  const double b1 = 1.0 + b;
  d.zp = 0.5 * b1;
  const double ls = log_fp64((b1 * b1) * (q2 * P.inv_4tc));
  d.inv_ls = 1.0 / ls;
  d.screen = make_float2(1.0f / (P.as2pi_f * f32_from_f64(ls)),
                         1.0f / (P.as2pi_f * 0.5f * static_cast<float>(kTR) * f32_from_f64(b)));
  return d;
}

__device__ __forceinline__ void store_dipole(const Events& E, int64_t ev, int slot, int side, const DipoleEntry& d) {
  const size_t a = dip_at(E, side, slot, ev);
  E.dip[a] = d.screen;
  if (d.screen.x < 0.0f) return;
  E.dq2[a] = d.q2;
  E.dzp[a] = d.zp;
  E.dinv[a] = d.inv_ls;
}

// 32-bit float close to the 52-bit uniform built from (hi, lo): relative
// error below 2^-22 for every value.
__device__ __forceinline__ float unit_float(uint32_t hi, uint32_t lo) {
  const float a = __uint2float_rn(hi >> 6);
  const float b = __uint2float_rn(lo >> 6);
  return fmaf(a, 0x1p-26f, fmaf(b, 0x1p-52f, 0x1p-53f));
}


// A dipole whose cache entry an emission invalidated: parton slots x and k,
// partners on x's side `side`, of the event of task t in the block's queue.
// An emission invalidates at most kMaxRefresh dipoles: (i, j), (j, k) and
// the other partners of the splitter and of the spectator.
constexpr int kMaxRefresh = 4;
__device__ __forceinline__ uint32_t pack_refresh(int t, int x, int side, int k) {
  return static_cast<uint32_t>(t) | (static_cast<uint32_t>(x) << 10) | (static_cast<uint32_t>(k) << 18) |
         (static_cast<uint32_t>(side) << 26);
}

// 1/c of a kernel for a dipole, c = alpha_s^over/(2 pi) * integral of
// P^over over [z-, z+].
__device__ __forceinline__ double inv_c_fp64(const DevParams& P, int kind, double zp, double inv_ls) {
  if (kind == kGtoQQ) return 1.0 / ((P.as_over / (2.0 * kPi)) * (0.5 * kTR) * (zp - (1.0 - zp)));
  return inv_ls * (kind == kQtoQG ? P.inv_as2pi_2cf : P.inv_as2pi_ca);
}

// 1/c of a gluon's kernels together (the per-dipole trial): c summed over
// the kernels in their order, as the oracle sums it.
__device__ __forceinline__ double inv_c_sum_fp64(const DevParams& P, double zp, double inv_ls) {
  const double c_gg = 1.0 / (inv_ls * P.inv_as2pi_ca);
  const double c_qq = (P.as_over / (2.0 * kPi)) * (0.5 * kTR) * (zp - (1.0 - zp));
  double c = c_gg;
  for (int f = 0; f < P.nf; ++f) c += c_qq;
  return 1.0 / c;
}

// The kernel of a winning gluon dipole in the per-dipole mode: kappa with
// probability c_kappa / c_sum, by the running sum against v c_sum.
__device__ __forceinline__ int choose_kernel(const DevParams& P, double zp, double inv_ls, double v) {
  const double c_gg = 1.0 / (inv_ls * P.inv_as2pi_ca);
  const double c_qq = (P.as_over / (2.0 * kPi)) * (0.5 * kTR) * (zp - (1.0 - zp));
  double c_sum = c_gg;
  for (int f = 0; f < P.nf; ++f) c_sum += c_qq;
  const double target = v * c_sum;
  double cum = c_gg;
  if (target < cum) return 0;
  for (int q = 1; q <= P.nf; ++q) {
    cum += c_qq;
    if (target < cum) return q;
  }
  return P.nf;
}

// The full FP64 SelectWinnerEmission (every trial exact, recomputed from the
// momenta); the fallback of the FP32 screen.  The log-space scale of trial
// j is L + ln(r_j)/c_j; the highest above ln t_C wins, the first on ties.
// This form covers partons first, first + stride, ... and keeps, in *best,
// *code and w, the best of those trials above the incoming *best (the first
// in loop order on ties; code = (2 i + side) * 8 + kappa orders the trials
// as the loop does); returns whether one was found.
template <int kMode>
__device__ inline bool select_winner_fp64_range(const DevParams& P, const Events& E, int64_t ev, const EventKey& key,
                                                int step, int n, double lnt, int first, int stride, EmitTask& w,
                                                double& best, int& code) {
  bool found = false;
  for (int i = first; i < n; i += stride) {
    const bool gluon = E.flav[E.at(i, ev)] == kGluon;
    const bool combined = gluon && per_dipole<kMode>(P);
    const int nk = gluon && !combined ? 1 + P.nf : 1;
    const V4 pi = load_p(E, i, ev);
    for (int side = 0; side < 2; ++side) {
      const int k = E.link[E.link_at(side, i, ev)];
      if (k == kNoLink) continue;
      const DipoleEntry d = make_dipole(P, 2.0 * mdot(pi, load_p(E, k, ev)));
      if (d.screen.x < 0.0f) continue;
      for (int kp = 0; kp < nk; kp += 2) {
        const U4 r = philox_draw<kMode>(P, key, static_cast<uint32_t>(step),
                                        static_cast<uint32_t>((2 * i + side) * 4 + kp / 2), kDrawTrial);
        for (int h = 0; h < 2 && kp + h < nk; ++h) {
          const int kappa = kp + h;
          const int kind = combined ? kKindUnchosen : (gluon ? (kappa == 0 ? kGtoGG : kGtoQQ) : kQtoQG);
          const double u = h ? to_unit(r.z, r.w) : to_unit(r.x, r.y);
          const double inv_c = combined ? inv_c_sum_fp64(P, d.zp, d.inv_ls) : inv_c_fp64(P, kind, d.zp, d.inv_ls);
          const double lt = fma(log_fp64(u), inv_c, lnt);
          if (lt > best) {
            best = lt;
            code = (2 * i + side) * 8 + kappa;
            found = true;
            w.lnt = lt;
            w.q2 = d.q2;
            w.zp = d.zp;
            w.inv_ls = d.inv_ls;
            w.i = i;
            w.k = k;
            w.side = side;
            w.kappa = kappa;
            w.kind = kind;
          }
        }
      }
    }
  }
  return found;
}

// The serial form: every parton in one thread.  Returns false if no trial
// is above t_C.
template <int kMode>
__device__ inline bool select_winner_fp64(const DevParams& P, const Events& E, int64_t ev, const EventKey& key, int step,
                                   int n, double lnt, EmitTask& w) {
  double best = P.ln_tc;
  int code = 0;
  return select_winner_fp64_range<kMode>(P, E, ev, key, step, n, lnt, 0, 1, w, best, code);
}

// Exact FP64 acceptance ratio of Eq. (A.9) with the (1 - y) factor, for a
// given z.  Returns -1 when y >= 1.
__device__ __forceinline__ double veto_ratio_fp64(const DevParams& P, int kind, double t, double q2, double z) {
  const double y = t / (q2 * z * (1.0 - z));
  if (!(y < 1.0)) return -1.0;
  const double f = (1.0 - y) * alpha_s(P, t) * kernel_p(kind, z, y);
  const double g = P.as_over * kernel_over(kind, z);
  return f / g;
}

// z from Eq. (A.8) in FP64, in a cancellation-free form: for the 1/(1-z)
// kernels 1 - z = z+ (z-/z+)^r, i.e. z = z- - z+ expm1(-r ln(z+/z-)).
__device__ __forceinline__ double z_fp64(int kind, double zp, double lsoft, double r) {
  const double zm = 1.0 - zp;
  if (kind == kGtoQQ) return fma(zp - zm, r, zm);
  return fma(-zp, expm1(-r * lsoft), zm);
}

enum : int { kCycleVetoed = 0, kCycleFinished = 1, kCycleAccepted = 2 };

// The serving pool counts every job's finished events (E.job_done, set only
// for the pool): the lanes of a warp that finished events of the same job
// add them with one atomic.  Every lane of the warp must call it.
__device__ __forceinline__ void count_job_done(const Events& E, int64_t ev, bool finished) {
  if (!E.job_done) return;  // the same for every lane (a launch argument)
  const int job = finished ? static_cast<int>(E.job_of[ev]) : -1;
  const unsigned peers = __match_any_sync(0xffffffffu, job);
  if (finished && static_cast<int>(threadIdx.x & 31) == __ffs(peers) - 1)
    atomicAdd(&E.job_done[job], static_cast<unsigned long long>(__popc(peers)));
}

// Leave the active state with `status`, recording the final scale.
__device__ __forceinline__ void finish_event(const Events& E, int64_t ev, int status, double t) {
  E.status[ev] = status;
  E.t[ev] = t;
}

// The FP32 screen of SelectWinnerEmission over the trials of partons
// first, first + stride, ... of an event: the best key (ties go to the
// smallest code, i.e. the first trial in the loop order of the exact
// selection), its error bound, the largest upper bound of every other
// trial, and the work counts.
struct Screen {
  float best_key, best_m, others_hi;
  int best_code;  // (2 i + side) * 8 + kappa, -1: no trial
  uint32_t best_hi, best_lo;
  uint32_t best_aux;  // the best trial's partner slot (bits 0-7) and gluon splitter (bit 8), as screened
  int trials, dipoles;
};

__device__ __forceinline__ void screen_none(Screen& sc) {
  sc.best_key = -INFINITY;
  sc.best_m = 0.0f;
  sc.others_hi = -INFINITY;
  sc.best_code = -1;
  sc.best_hi = sc.best_lo = 0;
  sc.best_aux = 0;
  sc.trials = sc.dipoles = 0;
}

// What the screen reads of one parton: flavour, colour partners and the
// FP32 cache entries of its two dipoles (read whether or not a partner
// exists; the entry is then ignored).
struct PartonScreen {
  int8_t flav;
  uint8_t link0, link1;
  float2 d0, d1;
};

__device__ __forceinline__ PartonScreen load_parton_screen(const Events& E, int64_t ev, int i) {
  PartonScreen q;
  q.flav = E.flav[E.at(i, ev)];
  q.link0 = E.link[E.link_at(0, i, ev)];
  q.link1 = E.link[E.link_at(1, i, ev)];
  q.d0 = E.dip[dip_at(E, 0, i, ev)];
  q.d1 = E.dip[dip_at(E, 1, i, ev)];
  return q;
}

// The loads of the next parton are issued before the trials of the current
// one are generated, so their latency hides behind the Philox rounds.
template <int kMode>
__device__ __forceinline__ void screen_partons(const DevParams& P, const Events& E, int64_t ev, const EventKey& key,
                                               int step, int n, int first, int stride, Screen& sc,
                                               const PartonScreen* first_loaded = nullptr) {
  screen_none(sc);
  if (first >= n) return;
  constexpr float kInvCF2 = static_cast<float>(1.0 / (2.0 * kCF));
  constexpr float kInvCA = static_cast<float>(1.0 / kCA);
  PartonScreen cur = first_loaded ? *first_loaded : load_parton_screen(E, ev, first);
  for (int i = first; i < n; i += stride) {
    PartonScreen nxt = cur;
    if (i + stride < n) nxt = load_parton_screen(E, ev, i + stride);
    const bool gluon = cur.flav == kGluon;
    const bool combined = gluon && per_dipole<kMode>(P);
    const int nk = gluon && !combined ? 1 + P.nf : 1;
    for (int side = 0; side < 2; ++side) {
      if ((side ? cur.link1 : cur.link0) == kNoLink) continue;
      const float2 d = side ? cur.d1 : cur.d0;
      if (d.x < 0.0f) continue;
      ++sc.dipoles;
      // per-dipole trial of a gluon: 1/c of all its kernels (a few ulp)
      const float inv_sum = combined ? 1.0f / (static_cast<float>(kCA) / d.x + static_cast<float>(P.nf) / d.y) : 0.0f;
      for (int kp = 0; kp < nk; kp += 2) {
        const U4 r = philox_draw<kMode>(P, key, static_cast<uint32_t>(step),
                                        static_cast<uint32_t>((2 * i + side) * 4 + kp / 2), kDrawTrial);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int kappa = kp + h;
          if (kappa >= nk) break;
          const uint32_t whi = h ? r.z : r.x, wlo = h ? r.w : r.y;
          const float lg2u = __log2f(unit_float(whi, wlo));
          const float invc = combined ? inv_sum : (!gluon ? d.x * kInvCF2 : (kappa == 0 ? d.x * kInvCA : d.y));
          const float key = lg2u * invc;
          const float m = fmaf(kKeyRelKey, fabsf(key), kKeyRelInvc * invc);
          ++sc.trials;
          if (key > sc.best_key) {
            sc.others_hi = fmaxf(sc.others_hi, sc.best_key + sc.best_m);
            sc.best_key = key;
            sc.best_m = m;
            sc.best_code = (2 * i + side) * 8 + kappa;
            sc.best_hi = whi;
            sc.best_lo = wlo;
            sc.best_aux = static_cast<uint32_t>(side ? cur.link1 : cur.link0) | (gluon ? 256u : 0u);
          } else {
            sc.others_hi = fmaxf(sc.others_hi, key + m);
          }
        }
      }
    }
    cur = nxt;
  }
}

// Merge the screen of other trials into sc: the same result as one screen
// over both sets in loop order (commutative and associative, so a butterfly
// over lanes gives every lane the whole event's screen).
__device__ __forceinline__ void screen_merge(Screen& sc, const Screen& o) {
  const bool o_wins = o.best_code >= 0 &&
                      (sc.best_code < 0 || o.best_key > sc.best_key ||
                       (o.best_key == sc.best_key && o.best_code < sc.best_code));
  const float lose = o_wins ? sc.best_key + sc.best_m : o.best_key + o.best_m;
  sc.others_hi = fmaxf(fmaxf(sc.others_hi, o.others_hi), lose);
  if (o_wins) {
    sc.best_key = o.best_key;
    sc.best_m = o.best_m;
    sc.best_code = o.best_code;
    sc.best_hi = o.best_hi;
    sc.best_lo = o.best_lo;
    sc.best_aux = o.best_aux;
  }
  sc.trials += o.trials;
  sc.dipoles += o.dipoles;
}

// Butterfly merge of the screens of the L lanes of each aligned lane group
// (every lane of the warp must call it).
template <int L>
__device__ __forceinline__ void screen_group_reduce(Screen& sc) {
#pragma unroll
  for (int off = 1; off < L; off <<= 1) {
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

// What the FP32 screen settles about a cycle: no trial above the cutoff, a
// certain winner (its exact scale computed), or neither -- then the exact
// FP64 selection decides (select_winner_fp64 / fallback_warp).
enum : int { kScreenNone = 0, kScreenWinner = 1, kScreenUndecided = 2 };

// The first part of the cycle once the screen is known: the cycle and work
// counts, and the screen's verdict; for a certain winner its exact scale
// (from the FP64 cache) and the winner's data in `task`.
template <int kMode>
__device__ inline int cycle_screen(const DevParams& P, const Events& E, int64_t ev, int step, double lnt,
                                   const Screen& sc, EmitTask& task) {
  const float best_key = sc.best_key, best_m = sc.best_m, others_hi = sc.others_hi;
  const int best_code = sc.best_code;
  const uint32_t best_hi = sc.best_hi, best_lo = sc.best_lo;
  E.n_steps[ev] = step + 1;
  E.n_trials[ev] += sc.trials;
  E.n_dipoles[ev] += sc.dipoles;

  // Cutoff threshold in key units: t' > t_C  <=>  key > log2(t_C / t).
  const float lt2 = f32_from_f64(lnt) * 1.44269504f;
  const float thr = P.lg2_tc_f - lt2;
  const float thr_m = 2e-6f * (1.0f + fabsf(lt2) + fabsf(P.lg2_tc_f));

  if (best_code < 0 || fmaxf(best_key + best_m, others_hi) < thr - thr_m) {
    return kScreenNone;  // certainly no trial above the cutoff
  }
  if (best_key - best_m > thr + thr_m && others_hi < best_key - best_m) {
    // Certain winner: its scale exactly, from the FP64 cache.
    const int dcode = best_code >> 3, kappa = best_code & 7;
    const int i = dcode >> 1, side = dcode & 1;
    const size_t a = dip_at(E, side, i, ev);
    const bool gluon = (sc.best_aux & 256u) != 0u;  // as the screen read them: no second load
    const bool combined = gluon && per_dipole<kMode>(P);
    const int kind = combined ? kKindUnchosen : (gluon ? (kappa == 0 ? kGtoGG : kGtoQQ) : kQtoQG);
    const double zp = E.dzp[a], inv_ls = E.dinv[a];
    const double inv_c = combined ? inv_c_sum_fp64(P, zp, inv_ls) : inv_c_fp64(P, kind, zp, inv_ls);
    const double lt = fma(log_fp64(to_unit(best_hi, best_lo)), inv_c, lnt);
    if (lt > P.ln_tc) {
      task.lnt = lt;
      task.q2 = E.dq2[a];
      task.zp = zp;
      task.inv_ls = inv_ls;
      task.i = i;
      task.k = static_cast<uint8_t>(sc.best_aux & 255u);
      task.side = side;
      task.kappa = kappa;
      task.kind = kind;
      return kScreenWinner;
    }
  }
  return kScreenUndecided;
}

// The exact FP64 selection for the undecided events of a warp, each computed
// by the whole warp: for every lane whose `need` is set, in turn, lane l takes
// partons l, l + 32, ... of that lane's event and the warp keeps the highest
// scale (the first trial in loop order on ties), the serial selection's
// winner.  The rare undecided cycle of an event with many partons thus takes
// a thirty-second of the dependent loads and FP64 work on its lane, which a
// whole launch or pool would otherwise wait for.  Sets have / task on the
// needing lanes.  Every lane of the warp must call it.
template <int kMode>
__device__ __noinline__ void fallback_warp(const DevParams& P0, const Events& E, bool need, int64_t ev, int job,
                                           const EventKey& key, int step, int n, double lnt, bool& have,
                                           EmitTask& task) {
  const int lane = static_cast<int>(threadIdx.x & 31);
  unsigned pending = __ballot_sync(0xffffffffu, need);
  while (pending) {
    const int src = __ffs(pending) - 1;
    pending &= pending - 1;
    const long long sev = __shfl_sync(0xffffffffu, static_cast<long long>(ev), src);
    EventKey skey;
    skey.id = __shfl_sync(0xffffffffu, key.id, src);
    skey.k0 = kJobKey<kMode> ? __shfl_sync(0xffffffffu, key.k0, src) : 0u;
    skey.k1 = kJobKey<kMode> ? __shfl_sync(0xffffffffu, key.k1, src) : 0u;
    const int sjob = kJobPhysics<kMode> ? __shfl_sync(0xffffffffu, job, src) : 0;
    const int sstep = __shfl_sync(0xffffffffu, step, src);
    const int sn = __shfl_sync(0xffffffffu, n, src);
    const double slnt = __shfl_sync(0xffffffffu, lnt, src);
    const DevParams& P = job_params<kJobPhysics<kMode>>(P0, E, sjob);
    EmitTask w;
    double best = P.ln_tc;
    int code = 0x7fffffff;
    const bool found = select_winner_fp64_range<kMode>(P, E, sev, skey, sstep, sn, slnt, lane, 32, w, best, code);
    // the highest scale; equal scales go to the smallest code
    double wb = best;
    int wc = code;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, wb, off);
      const int oc = __shfl_xor_sync(0xffffffffu, wc, off);
      if (ob > wb || (ob == wb && oc < wc)) {
        wb = ob;
        wc = oc;
      }
    }
    const unsigned own = __ballot_sync(0xffffffffu, found && code == wc);
    if (own) {
      const int ol = __ffs(own) - 1;
      const double t_lnt = __shfl_sync(0xffffffffu, w.lnt, ol), t_q2 = __shfl_sync(0xffffffffu, w.q2, ol);
      const double t_zp = __shfl_sync(0xffffffffu, w.zp, ol), t_inv = __shfl_sync(0xffffffffu, w.inv_ls, ol);
      const uint32_t packed = __shfl_sync(0xffffffffu,
                                          static_cast<uint32_t>(w.i) | (static_cast<uint32_t>(w.k) << 8) |
                                              (static_cast<uint32_t>(w.side) << 16) |
                                              (static_cast<uint32_t>(w.kappa) << 20) |
                                              (static_cast<uint32_t>(w.kind) << 24),
                                          ol);
      if (lane == src) {
        task.lnt = t_lnt;
        task.q2 = t_q2;
        task.zp = t_zp;
        task.inv_ls = t_inv;
        task.i = static_cast<uint8_t>(packed & 255u);
        task.k = static_cast<uint8_t>((packed >> 8) & 255u);
        task.side = static_cast<uint8_t>((packed >> 16) & 15u);
        task.kappa = static_cast<uint8_t>((packed >> 20) & 15u);
        task.kind = static_cast<uint8_t>(packed >> 24);
      }
    }
    if (lane == src) have = own != 0u;
  }
}

// The rest of the cycle once the winner is known (have: a trial above t_C,
// with its data in task): CheckCutoff, AcceptOrVeto and the decision hash.
// Returns kCycleFinished when the event left the active state (status
// written), kCycleAccepted with `task` filled when an emission must be
// generated, kCycleVetoed otherwise.
template <int kMode>
__device__ inline int cycle_conclude(const DevParams& P, const Events& E, int64_t ev, const EventKey& key, int step,
                                     int n, bool have, EmitTask& task) {
  // ---- CheckCutoff.
  if (!have) {
    finish_event(E, ev, GAPS_DONE, P.tc);
    return kCycleFinished;
  }
  E.lnt[ev] = task.lnt;
  E.n_winners[ev] += 1;
  if (task.kind == kKindUnchosen) {
    // per-dipole trial of a gluon: its kernel from the winner's second draw
    const U4 rk = philox_draw<kMode>(P, key, static_cast<uint32_t>(step), 1u, kDrawWinner);
    const int kappa = choose_kernel(P, task.zp, task.inv_ls, to_unit(rk.z, rk.w));
    task.kappa = static_cast<uint8_t>(kappa);
    task.kind = static_cast<uint8_t>(kappa == 0 ? kGtoGG : kGtoQQ);
  }

  // ---- AcceptOrVeto: FP32 screen of Eq. (A.8)-(A.9), FP64 near the edge.
  const U4 rw = philox_draw<kMode>(P, key, static_cast<uint32_t>(step), 0u, kDrawWinner);
  bool accept;
  {
    const float zpf = f32_from_f64(task.zp);
    const float zmf = f32_from_f64(1.0 - task.zp);
    const float lf = 1.0f / f32_from_f64(task.inv_ls);
    const float rzf = unit_float(rw.x, rw.y);
    float z, e;  // z and 1 - z
    if (task.kind == kGtoQQ) {
      z = fmaf(zpf - zmf, rzf, zmf);
      e = fmaf(-(zpf - zmf), rzf, zpf);
    } else {
      z = zmf - zpf * expm1f(-rzf * lf);
      e = zpf * __expf(-rzf * lf);
    }
    const float lnt_f = f32_from_f64(task.lnt);
    const float y = __expf(lnt_f) / (f32_from_f64(task.q2) * z * e);
    const float as_ratio = P.fixed ? 1.0f : P.as_mz_over_f / (1.0f + P.as_b0_f * (lnt_f - P.ln_mz2_f));
    float pr;  // P(z, y) / P^over(z)
    if (task.kind == kQtoQG) {
      pr = e / (e + z * y) - 0.5f * (1.0f + z) * e;
    } else if (task.kind == kGtoGG) {
      pr = e / (e + z * y) - e + 0.5f * z * e * e;
    } else {
      pr = 1.0f - 2.0f * z * e;
    }
    const float ratio = (1.0f - y) * as_ratio * pr;
    const float rvf = unit_float(rw.z, rw.w);
    const float margin = kVetoRel * (fabsf(ratio) + rvf) + kVetoAbs;
    if (fabsf(y - 1.0f) <= 1e-4f || fabsf(rvf - ratio) <= margin) {
      atomicAdd(&E.counters[3], 1ull);  // veto decided in FP64
      const double zz = z_fp64(task.kind, task.zp, 1.0 / task.inv_ls, to_unit(rw.x, rw.y));
      const double ratio64 = veto_ratio_fp64(P, task.kind, exp(task.lnt), task.q2, zz);
      accept = ratio64 >= 0.0 && to_unit(rw.z, rw.w) < ratio64;
    } else {
      accept = y < 1.0f && rvf < ratio;
    }
  }
  const unsigned long long word = static_cast<unsigned long long>(step) |
                                  (static_cast<unsigned long long>(task.i) << 32) |
                                  (static_cast<unsigned long long>(task.side) << 40) |
                                  (static_cast<unsigned long long>(task.kappa) << 48) |
                                  (static_cast<unsigned long long>(accept ? 1 : 0) << 56);
  E.hash[ev] = fnv1a64(E.hash[ev], word);
  if (!accept) return kCycleVetoed;
  if (n >= E.cap) {
    finish_event(E, ev, GAPS_OVERFLOW, exp(task.lnt));
    return kCycleFinished;
  }
  task.ev = static_cast<int32_t>(ev);
  task.rz_hi = rw.x;
  task.rz_lo = rw.y;
  task.n = n;
  task.step = step;
  return kCycleAccepted;
}

// The whole decision of a cycle in one thread, the exact selection serial.
template <int kMode>
__device__ inline int cycle_decide(const DevParams& P, const Events& E, int64_t ev, const EventKey& key, int step,
                                   int n, double lnt, const Screen& sc, EmitTask& task) {
  const int s = cycle_screen<kMode>(P, E, ev, step, lnt, sc, task);
  bool have = s == kScreenWinner;
  if (s == kScreenUndecided) {
    atomicAdd(&E.counters[2], 1ull);  // screen undecided: full FP64 cycle
    have = select_winner_fp64<kMode>(P, E, ev, key, step, n, lnt, task);
  }
  return cycle_conclude<kMode>(P, E, ev, key, step, n, have, task);
}

// Phase 1 of a cycle for active event ev, one thread: SelectWinnerEmission
// (the FP32 screen over every trial), then cycle_decide.
template <int kMode>
__device__ inline int cycle_select_veto(const DevParams& P0, const Events& E, int64_t ev, EmitTask& task) {
  const int job = kJobKey<kMode> ? static_cast<int>(E.job_of[ev]) : 0;
  const DevParams& P = job_params<kJobPhysics<kMode>>(P0, E, job);
  const EventKey key = event_key<kMode>(P, E, ev, job);
  const int n = E.n_partons[ev];
  const int step = E.n_steps[ev];
  const double lnt = E.lnt[ev];
  if (step >= P.max_steps) {
    finish_event(E, ev, GAPS_STEP_LIMIT, exp(lnt));
    return kCycleFinished;
  }
  Screen sc;
  screen_partons<kMode>(P, E, ev, key, step, n, 0, 1, sc);
  return cycle_decide<kMode>(P, E, ev, key, step, n, lnt, sc, task);
}

// Phase 2: GenerateEmission -- azimuth, the final-final dipole map, colours
// and the new parton in slot n.  The dipoles whose invariant mass moved are
// appended to the block's refresh list (jobs, *n_jobs) under task_index; the
// caller recomputes them with refresh_dipole after a block barrier, spread
// over all of its threads, so that this FP64-heavy step runs in full warps.
template <int kMode>
__device__ inline void cycle_emit(const DevParams& P0, const Events& E, const EmitTask& w, int task_index,
                                  uint32_t* jobs, int* n_jobs) {
  const int64_t ev = w.ev;
  const int job = kJobKey<kMode> ? static_cast<int>(E.job_of[ev]) : 0;
  const DevParams& P = job_params<kJobPhysics<kMode>>(P0, E, job);
  const EventKey key = event_key<kMode>(P, E, ev, job);
  const double t = exp(w.lnt);
  const double z = z_fp64(w.kind, w.zp, 1.0 / w.inv_ls, to_unit(w.rz_hi, w.rz_lo));
  const double y = t / (w.q2 * z * (1.0 - z));
  const U4 rphi = philox_draw<kMode>(P, key, static_cast<uint32_t>(w.step), 1u, kDrawWinner);
  double sphi, cphi;
  sincospi(2.0 * to_unit(rphi.x, rphi.y), &sphi, &cphi);
  const V4 a = load_p(E, w.i, ev);
  const V4 b = load_p(E, w.k, ev);
  V4 pi, pj, pb;
  dipole_map(a, b, z, y, cphi, sphi, pi, pj, pb);
  const int j = w.n;
  store_p(E, w.i, ev, pi);
  store_p(E, j, ev, pj);
  store_p(E, w.k, ev, pb);
  const size_t ai = E.at(w.i, ev), aj = E.at(j, ev);
  if (w.kind == kGtoQQ) {
    // g(c, a) -> q(c, 0) + qbar(0, a); the parton holding colour a now
    // connects to the antiquark.
    const int q = E.link[E.link_at(1, w.i, ev)];
    E.flav[ai] = static_cast<int8_t>(w.kappa);
    E.flav[aj] = static_cast<int8_t>(-w.kappa);
    E.col[aj] = 0;
    E.acol[aj] = E.acol[ai];
    E.acol[ai] = 0;
    E.link[E.link_at(1, w.i, ev)] = kNoLink;
    E.link[E.link_at(0, j, ev)] = kNoLink;
    E.link[E.link_at(1, j, ev)] = static_cast<uint8_t>(q);
    E.link[E.link_at(0, q, ev)] = static_cast<uint8_t>(j);
  } else {
    // A gluon enters the shared colour line between splitter and spectator;
    // the splitter takes the new line m.
    const int m = E.next_colour[ev];
    E.next_colour[ev] = m + 1;
    E.flav[aj] = static_cast<int8_t>(kGluon);
    if (w.side == 0) {
      E.col[aj] = E.col[ai];
      E.acol[aj] = static_cast<int16_t>(m);
      E.col[ai] = static_cast<int16_t>(m);
      E.link[E.link_at(0, w.i, ev)] = static_cast<uint8_t>(j);
      E.link[E.link_at(0, j, ev)] = static_cast<uint8_t>(w.k);
      E.link[E.link_at(1, j, ev)] = static_cast<uint8_t>(w.i);
      E.link[E.link_at(1, w.k, ev)] = static_cast<uint8_t>(j);
    } else {
      E.col[aj] = static_cast<int16_t>(m);
      E.acol[aj] = E.acol[ai];
      E.acol[ai] = static_cast<int16_t>(m);
      E.link[E.link_at(1, w.i, ev)] = static_cast<uint8_t>(j);
      E.link[E.link_at(1, j, ev)] = static_cast<uint8_t>(w.k);
      E.link[E.link_at(0, j, ev)] = static_cast<uint8_t>(w.i);
      E.link[E.link_at(0, w.k, ev)] = static_cast<uint8_t>(j);
    }
  }
  // Every dipole with a moved parton, once: dipole (x, side) and its
  // partner's opposite side share Q^2; a pair whose partner is a moved parton
  // listed earlier was already taken from that side.
  const int moved[3] = {w.i, j, w.k};
  uint32_t mine[kMaxRefresh];
  int count = 0;
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    const int x = moved[m];
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const int k = E.link[E.link_at(side, x, ev)];
      if (k == kNoLink) continue;
      bool seen = false;
#pragma unroll
      for (int m2 = 0; m2 < m; ++m2) seen |= (k == moved[m2]);
      if (seen || count == kMaxRefresh) continue;
      mine[count++] = pack_refresh(task_index, x, side, k);
    }
  }
  const int at = atomicAdd(n_jobs, count);
  for (int c = 0; c < count; ++c) jobs[at + c] = mine[c];
  E.n_partons[ev] = j + 1;
  E.n_emissions[ev] += 1;
}

// Recompute one dipole of the refresh list from the stored momenta of its
// two partons (the oracle's formulas, in the oracle's operand order).
template <bool kMulti>
__device__ inline void refresh_dipole(const DevParams& P0, const Events& E, const EmitTask* tasks, uint32_t job) {
  const int t = static_cast<int>(job & 1023u), x = static_cast<int>((job >> 10) & 255u);
  const int k = static_cast<int>((job >> 18) & 255u), side = static_cast<int>((job >> 26) & 1u);
  const int64_t ev = tasks[t].ev;
  const DevParams& P = params_of<kMulti>(P0, E, ev);
  const DipoleEntry d = make_dipole(P, 2.0 * mdot(load_p(E, x, ev), load_p(E, k, ev)));
  store_dipole(E, ev, x, side, d);
  store_dipole(E, ev, k, 1 - side, d);
}

}  // namespace gaps
