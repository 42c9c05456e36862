// Oracle: LO matrix element and the serial Sudakov veto-algorithm shower.
// Test infrastructure only (see oracle_api.h).
#include <algorithm>
#include <cmath>

#include "oracle_internal.hpp"
#include "philox.hpp"

namespace oracle {

// ------------------------------------------------------------------ App. B
// One event of e+e- -> q qbar: a uniformly chosen flavour (App. B draws
// flavour = random(1, n_f)), cos(theta) uniform in [-1, 1] and phi uniform in
// [0, 2 pi).  The weight is the Monte Carlo estimate of the total cross
// section: w = n_f * 2 * d sigma / d cos(theta), in pb.
void generate_me(const oracle_params& p, uint32_t event_id, Event& ev) {
  const UniformPair r0 = uniform_pair(p.seed, event_id, 0, 0, kPurposeME);
  const UniformPair r1 = uniform_pair(p.seed, event_id, 0, 1, kPurposeME);
  int fl = 1 + static_cast<int>(r0.u0 * p.n_flavours);
  if (fl > p.n_flavours) fl = p.n_flavours;
  const double cth = 2.0 * r0.u1 - 1.0;
  const double phi = 2.0 * kPi * r1.u0;
  const double s = p.sqrt_s * p.sqrt_s;
  const double sth = std::sqrt(1.0 - cth * cth);
  const double e = 0.5 * p.sqrt_s;
  const Vec4 pq{e, e * sth * std::cos(phi), e * sth * std::sin(phi), e * cth};
  const Vec4 pqbar{e, -pq.x, -pq.y, -pq.z};
  ev.partons.clear();
  ev.partons.push_back(Parton{pq, fl, 1, 0});
  ev.partons.push_back(Parton{pqbar, -fl, 0, 1});
  ev.next_colour = 2;
  ev.me_flavour = fl;
  ev.weight = p.n_flavours * 2.0 *
              dsigma_dcos(s, fl, cth, (p.mutation & ORACLE_MUT_ME_NO_INTERF) != 0);
}

namespace {

// FNV-1a (64-bit) over the eight little-endian bytes of one decision word.
uint64_t fnv1a_word(uint64_t h, uint64_t word) {
  for (int b = 0; b < 8; ++b) {
    h ^= (word >> (8 * b)) & 0xFFu;
    h *= 1099511628211ull;
  }
  return h;
}
constexpr uint64_t kFnvOffset = 14695981039346656037ull;

// Colour-connected partner of parton i: side 0 follows i's colour line
// (i.col == k.acol), side 1 its anticolour line (i.acol == k.col).  -1 if none.
int colour_partner(const std::vector<Parton>& ps, int i, int side) {
  const int line = side == 0 ? ps[i].col : ps[i].acol;
  if (line == 0) return -1;
  for (int k = 0; k < static_cast<int>(ps.size()); ++k) {
    if (k == i) continue;
    if ((side == 0 ? ps[k].acol : ps[k].col) == line) return k;
  }
  return -1;
}

struct KernelRef {
  int kind;
  int flavour;  // flavour of the produced quark for g -> q qbar
};

// The splitting kernels whose splitter flavour matches (App. A listing: "P(u
// -> ug) may not be same as P(d -> dg)").  Quark or antiquark: one q -> qg
// kernel.  Gluon: g -> gg, then g -> q qbar for flavours 1..n_f.
int kernels_for(int flav, int nf, KernelRef out[8], int mutation) {
  if (flav != kGluon) {
    out[0] = {kQtoQG, 0};
    return 1;
  }
  out[0] = {kGtoGG, 0};
  const int nq = (mutation & ORACLE_MUT_NF_MINUS_ONE) ? nf - 1 : nf;
  for (int f = 1; f <= nq; ++f) out[f] = {kGtoQQ, f};
  return 1 + nq;
}

// c = alpha_s^over / (2 pi) times the integral of the kernel's overestimate
// over [z-, z+] (Eq. A.4).
double trial_density(int kind, double as_over, double zm, double zp, int mutation) {
  const double c = as_over / (2.0 * kPi) * kernel_integral(kind, zm, zp);
  // planted: g -> gg at the full C_A instead of half of it per dipole
  return (kind == kGtoGG && (mutation & ORACLE_MUT_GG_FULL)) ? 2.0 * c : c;
}

struct Winner {
  bool found = false;
  int i = -1, k = -1, side = 0, kappa = 0;
  KernelRef kernel{0, 0};
  double q2 = 0, zm = 0, zp = 0;
  // per-dipole trials: the dipole's kernels and their overestimate integrals
  int nk = 0;
  KernelRef kernels[8];
  double c[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  double c_sum = 0;
};

}  // namespace

// ---------------------------------------------------- Sec. 2, App. A, App. C
// The serial veto algorithm with competing emissions.  Every cycle:
//  (1) SelectWinnerEmission: for every colour-connected (splitter, spectator)
//      pair and every matching kernel, a trial scale t' = t r^(1/c) (Eq. A.6)
//      with c = alpha_s^over / (2 pi) * integral of P^over over [z-, z+]
//      (Eq. A.4); the highest t' above t_C wins, the first one on ties.
//  (2) CheckCutoff: no trial above t_C ends the event.
//  (3) The winner's scale becomes the evolution scale whatever the outcome
//      of the veto (App. A: all emissions were offered the chance above it).
//  (4) AcceptOrVeto: z from Eq. (A.8), y = t / (Q^2 z (1-z)); accept with
//      probability (1-y) alpha_s(t) P(z,y) / (alpha_s^over P^over(z)) when
//      y < 1 (Eq. A.9; y < 1 is the Theta(z- < z < z+) at scale t).
//  (5) GenerateEmission: azimuth, the final-final dipole map, colours, and
//      the new parton appended to the record.
void shower(const oracle_params& p, uint32_t event_id, Event& ev) {
  const double tc = p.t_cutoff;
  const bool fixed = p.fixed_alphas != 0;
  const bool running_over_bug = (p.mutation & ORACLE_MUT_ALPHAS_OVER) != 0 && !fixed;
  const double as_over = running_over_bug ? p.alphas_mz
                                          : alphas_at(tc, p.alphas_mz, p.n_flavours, fixed);
  const MapMutations mmut{(p.mutation & ORACLE_MUT_NO_RECOIL) != 0,
                          (p.mutation & ORACLE_MUT_KT_SIGN) != 0,
                          (p.mutation & ORACLE_MUT_Z_SWAP) != 0};
  ev.t = p.sqrt_s * p.sqrt_s;  // starting scale t0 = s
  ev.hash = kFnvOffset;
  ev.status = 0;
  ev.n_steps = ev.n_emissions = ev.n_winners = 0;
  ev.n_trials = 0;
  ev.n_dipoles = 0;
  ev.t_first = 0.0;

  while (ev.status == 0) {
    if (ev.n_steps >= p.max_steps) {
      ev.status = ORACLE_STEP_LIMIT;
      break;
    }
    const uint32_t step = static_cast<uint32_t>(ev.n_steps);
    const int n = static_cast<int>(ev.partons.size());

    // (1) SelectWinnerEmission.
    double t_win = tc;
    Winner w;
    for (int i = 0; i < n; ++i) {
      for (int side = 0; side < 2; ++side) {
        const int k = colour_partner(ev.partons, i, side);
        if (k < 0) continue;
        const double q2 = 2.0 * dot(ev.partons[i].p, ev.partons[k].p);
        if (q2 < 4.0 * tc) continue;  // no phase space above the cutoff
        const double zp = 0.5 * (1.0 + std::sqrt(1.0 - 4.0 * tc / q2));
        const double zm = 1.0 - zp;
        ++ev.n_dipoles;
        KernelRef kernels[8];
        const int nk = kernels_for(ev.partons[i].flav, p.n_flavours, kernels, p.mutation);
        if (p.trial_mode == 1) {
          // One trial for the dipole with c = sum of its kernels' c
          // (competing exponentials: the first of independent trials is one
          // trial with the summed rate, its kernel drawn by share).
          double c[8], c_sum = 0.0;
          for (int kappa = 0; kappa < nk; ++kappa) {
            c[kappa] = trial_density(kernels[kappa].kind, as_over, zm, zp, p.mutation);
            c_sum += c[kappa];
          }
          const uint32_t slot = static_cast<uint32_t>((2 * i + side) * 4);
          const double u = uniform_pair(p.seed, event_id, step, slot, kPurposeTrial).u0;
          const double t_trial = ev.t * std::pow(u, 1.0 / c_sum);
          ++ev.n_trials;
          if (t_trial > t_win) {
            t_win = t_trial;
            w.found = true;
            w.i = i;
            w.k = k;
            w.side = side;
            w.q2 = q2;
            w.zm = zm;
            w.zp = zp;
            w.nk = nk;
            for (int kappa = 0; kappa < nk; ++kappa) {
              w.kernels[kappa] = kernels[kappa];
              w.c[kappa] = c[kappa];
            }
            w.c_sum = c_sum;
          }
          continue;
        }
        for (int kappa = 0; kappa < nk; ++kappa) {
          const double c = trial_density(kernels[kappa].kind, as_over, zm, zp, p.mutation);
          const uint32_t slot = static_cast<uint32_t>((2 * i + side) * 4 + kappa / 2);
          const UniformPair r = uniform_pair(p.seed, event_id, step, slot, kPurposeTrial);
          const double u = ((kappa & 1) && !(p.mutation & ORACLE_MUT_PAIR_UNIFORM)) ? r.u1 : r.u0;
          const double t_trial = ev.t * std::pow(u, 1.0 / c);
          ++ev.n_trials;
          if (t_trial > t_win) {
            t_win = t_trial;
            w.found = true;
            w.i = i;
            w.k = k;
            w.side = side;
            w.kappa = kappa;
            w.kernel = kernels[kappa];
            w.q2 = q2;
            w.zm = zm;
            w.zp = zp;
          }
        }
      }
    }
    ++ev.n_steps;

    // (2) CheckCutoff.
    if (!w.found) {
      ev.t = tc;
      ev.status = ORACLE_DONE;
      break;
    }
    // (3) The winner's scale is the new upper scale for every parton.
    const double t_old = ev.t;
    ev.t = t_win;
    ++ev.n_winners;
    if (p.trial_mode == 1) {
      // The winning dipole's kernel, with probability c_kappa / c_sum.
      const double v = uniform_pair(p.seed, event_id, step, 1, kPurposeWinner).u1;
      int kappa = w.nk - 1;
      if (p.mutation & ORACLE_MUT_KERNEL_UNIFORM) {
        kappa = std::min(static_cast<int>(v * w.nk), w.nk - 1);
      } else {
        double cum = 0.0;
        for (int q = 0; q < w.nk; ++q) {
          cum += w.c[q];
          if (v * w.c_sum < cum) {
            kappa = q;
            break;
          }
        }
      }
      w.kappa = kappa;
      w.kernel = w.kernels[kappa];
    }

    // (4) AcceptOrVeto.
    const UniformPair rw = uniform_pair(p.seed, event_id, step, 0, kPurposeWinner);
    const int kind = w.kernel.kind;
    const double z = kernel_generate_z(kind, w.zm, w.zp, rw.u0,
                                       (p.mutation & ORACLE_MUT_Z_UNIFORM) != 0);
    const double y = ev.t / (w.q2 * z * (1.0 - z));
    bool accept = false;
    if (y < 1.0) {
      const double jac = (p.mutation & ORACLE_MUT_NO_JACOBIAN) ? 1.0 : (1.0 - y);
      const double f = jac * alphas_at(ev.t, p.alphas_mz, p.n_flavours, fixed) *
                       kernel_value(kind, z, y);
      const double g = as_over * kernel_estimate(kind, z);
      accept = rw.u1 < f / g;
    }
    const uint64_t word = static_cast<uint64_t>(step) | (static_cast<uint64_t>(w.i) << 32) |
                          (static_cast<uint64_t>(w.side) << 40) |
                          (static_cast<uint64_t>(w.kappa) << 48) |
                          (static_cast<uint64_t>(accept ? 1 : 0) << 56);
    ev.hash = fnv1a_word(ev.hash, word);
    if (!accept) {
      if (p.mutation & ORACLE_MUT_TRIAL_RESTART) ev.t = t_old;
      continue;
    }

    // (5) GenerateEmission.
    if (n >= p.capacity) {
      ev.status = ORACLE_OVERFLOW;
      break;
    }
    const double phi = 2.0 * kPi * uniform_pair(p.seed, event_id, step, 1, kPurposeWinner).u0;
    Parton& pi = ev.partons[w.i];
    Parton& pk = ev.partons[w.k];
    Vec4 mi, mj, mk;
    splitting_map(pi.p, pk.p, z, y, phi, mmut, mi, mj, mk);
    Parton pj{mj, 0, 0, 0};
    if (kind == kGtoQQ) {
      // g(c, a) -> q(c, 0) + qbar(0, a), whichever side the spectator is on.
      const int f = w.kernel.flavour;
      pj.flav = -f;
      pj.col = 0;
      pj.acol = pi.acol;
      pi.flav = f;
      pi.acol = 0;
    } else {
      // Gluon emission: the new gluon sits between splitter and spectator on
      // the colour line they shared; the splitter takes a new line m.
      const int m = ev.next_colour++;
      pj.flav = kGluon;
      const bool swap = (p.mutation & ORACLE_MUT_COLOUR_SWAP) != 0;
      if (w.side == 0) {
        pj.col = swap ? m : pi.col;
        pj.acol = swap ? pi.col : m;
        pi.col = m;
      } else {
        pj.col = swap ? pi.acol : m;
        pj.acol = swap ? m : pi.acol;
        pi.acol = m;
      }
    }
    pi.p = mi;
    pk.p = mk;
    ev.partons.push_back(pj);
    ++ev.n_emissions;
    if (ev.n_emissions == 1) ev.t_first = ev.t;
    if (p.max_emissions > 0 && ev.n_emissions >= p.max_emissions) {
      ev.status = ORACLE_DONE;
      break;
    }
  }
}

}  // namespace oracle
