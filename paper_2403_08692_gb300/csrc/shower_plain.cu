// Matrix element + shower initial state (App. B; App. C main program) and the
// plain event-parallel veto cycle (Sec. 2, Fig. 2, App. C).
//
// Plain form: one launch per veto cycle over every event of the batch, one
// thread per event.  The paper's four per-cycle kernels (SelectWinnerEmission,
// CheckCutoff, AcceptOrVeto, GenerateEmission) and its alpha_s kernel are
// fused into one launch, so an event's state stays in registers for the
// whole cycle instead of making four round trips through HBM.  Finished
// events leave at once (the paper's endShower early exit) and bump the
// finished-event counter that the host polls between cycles.
#include "gaps_launch.hpp"

namespace gaps {

namespace {

__global__ void __launch_bounds__(256) k_me(DevParams P, Events E) {
  const int64_t ev = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (ev >= E.n) return;
  const uint32_t id = E.first + static_cast<uint32_t>(ev);
  const Uniforms r0 = draw2(P, id, 0, 0, kDrawME);
  const Uniforms r1 = draw2(P, id, 0, 1, kDrawME);
  int fl = 1 + static_cast<int>(r0.a * P.nf);
  fl = fl > P.nf ? P.nf : fl;
  const double cth = 2.0 * r0.b - 1.0;
  double sphi, cphi;
  sincospi(2.0 * r1.a, &sphi, &cphi);
  const double sth = sqrt(1.0 - cth * cth);
  const double en = 0.5 * P.sqrt_s;
  const double x = en * sth * cphi, y = en * sth * sphi, z = en * cth;
  E.e[E.at(0, ev)] = en;
  E.px[E.at(0, ev)] = x;
  E.py[E.at(0, ev)] = y;
  E.pz[E.at(0, ev)] = z;
  E.e[E.at(1, ev)] = en;
  E.px[E.at(1, ev)] = -x;
  E.py[E.at(1, ev)] = -y;
  E.pz[E.at(1, ev)] = -z;
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
  E.weight[ev] = P.nf * 2.0 * dsigma_dcos(P.s, fl, cth);
  E.me_flavour[ev] = fl;
  E.t[ev] = P.s;  // starting scale t0 = s
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

// Counter word 0 counts finished events (the paper's completedEventsCounter),
// word 1 those stopped by the veto-cycle limit.
__device__ __forceinline__ void finish(const Events& E, int64_t ev, int status) {
  E.status[ev] = status;
  atomicAdd(&E.counters[0], 1ull);
  if (status == GAPS_STEP_LIMIT) atomicAdd(&E.counters[1], 1ull);
}

__global__ void __launch_bounds__(128) k_step_plain(DevParams P, Events E) {
  const int64_t ev = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (ev >= E.n) return;
  if (E.status[ev] != GAPS_ACTIVE) return;  // finished events idle (App. C)
  const uint32_t id = E.first + static_cast<uint32_t>(ev);
  const int n = E.n_partons[ev];
  const int step = E.n_steps[ev];
  if (step >= P.max_steps) {
    finish(E, ev, GAPS_STEP_LIMIT);
    return;
  }
  const double t = E.t[ev];
  const double tc = P.tc;
  const double as2pi = P.as_over / (2.0 * kPi);

  // SelectWinnerEmission: every colour-connected (splitter, side) dipole and
  // every kernel matching the splitter; trial t' = t r^(1/c) (Eq. A.6).
  double t_win = tc;
  int wi = -1, wk = 0, wside = 0, wkappa = 0, wkind = 0;
  double wq2 = 0.0, wzm = 0.0, wzp = 0.0;
  int trials = 0, dipoles = 0;
  for (int i = 0; i < n; ++i) {
    const bool gluon = E.flav[E.at(i, ev)] == kGluon;
    const int nk = gluon ? 1 + P.nf : 1;
    const V4 pi = load_p(E, i, ev);
    for (int side = 0; side < 2; ++side) {
      const int k = E.link[E.link_at(side, i, ev)];
      if (k == kNoLink) continue;
      const V4 pk = load_p(E, k, ev);
      const double q2 = 2.0 * mdot(pi, pk);
      if (q2 < 4.0 * tc) continue;
      const double zp = 0.5 * (1.0 + sqrt(1.0 - 4.0 * tc / q2));
      const double zm = 1.0 - zp;
      ++dipoles;
      const double lsoft = log(zp / zm);  // = ln((1 - zm) / (1 - zp))
      for (int kp = 0; kp < nk; kp += 2) {
        const Uniforms u = draw2(P, id, step, static_cast<uint32_t>((2 * i + side) * 4 + kp / 2), kDrawTrial);
        for (int h = 0; h < 2; ++h) {
          const int kappa = kp + h;
          if (kappa >= nk) break;
          const int kind = gluon ? (kappa == 0 ? kGtoGG : kGtoQQ) : kQtoQG;
          const double integral = kind == kGtoQQ ? 0.5 * kTR * (zp - zm) : kernel_k(kind) * lsoft;
          const double c = as2pi * integral;
          const double tt = t * exp(log(h ? u.b : u.a) / c);
          ++trials;
          if (tt > t_win) {
            t_win = tt;
            wi = i;
            wk = k;
            wside = side;
            wkappa = kappa;
            wkind = kind;
            wq2 = q2;
            wzm = zm;
            wzp = zp;
          }
        }
      }
    }
  }
  E.n_steps[ev] = step + 1;
  E.n_trials[ev] += trials;
  E.n_dipoles[ev] += dipoles;

  // CheckCutoff.
  if (wi < 0) {
    E.t[ev] = tc;
    finish(E, ev, GAPS_DONE);
    return;
  }
  E.t[ev] = t_win;
  E.n_winners[ev] += 1;

  // AcceptOrVeto: z from Eq. (A.8), then the ratio of Eq. (A.9) with the
  // (1 - y) phase-space factor; y < 1 is the physical z range at scale t.
  const Uniforms uw = draw2(P, id, step, 0, kDrawWinner);
  double z;
  if (wkind == kGtoQQ) {
    z = wzm + (wzp - wzm) * uw.a;
  } else {
    const double l1 = log(1.0 - wzm), l2 = log(1.0 - wzp);
    z = 1.0 - exp(l1 + (l2 - l1) * uw.a);
  }
  const double y = t_win / (wq2 * z * (1.0 - z));
  bool accept = false;
  if (y < 1.0) {
    const double f = (1.0 - y) * alpha_s(P, t_win) * kernel_p(wkind, z, y);
    const double g = P.as_over * kernel_over(wkind, z);
    accept = uw.b < f / g;
  }
  const unsigned long long word = static_cast<unsigned long long>(step) |
                                  (static_cast<unsigned long long>(wi) << 32) |
                                  (static_cast<unsigned long long>(wside) << 40) |
                                  (static_cast<unsigned long long>(wkappa) << 48) |
                                  (static_cast<unsigned long long>(accept ? 1 : 0) << 56);
  E.hash[ev] = fnv1a64(E.hash[ev], word);
  if (!accept) return;

  // GenerateEmission.
  if (n >= E.cap) {
    finish(E, ev, GAPS_OVERFLOW);
    return;
  }
  const double uphi = draw2(P, id, step, 1, kDrawWinner).a;
  double sphi, cphi;
  sincospi(2.0 * uphi, &sphi, &cphi);
  const V4 a = load_p(E, wi, ev);
  const V4 b = load_p(E, wk, ev);
  V4 pi, pj, pb;
  dipole_map(a, b, z, y, cphi, sphi, pi, pj, pb);
  const int j = n;
  store_p(E, wi, ev, pi);
  store_p(E, j, ev, pj);
  store_p(E, wk, ev, pb);
  const size_t ai = E.at(wi, ev), aj = E.at(j, ev);
  if (wkind == kGtoQQ) {
    // g(c, a) -> q(c, 0) + qbar(0, a); the parton holding colour a now
    // connects to the antiquark.
    const int q = E.link[E.link_at(1, wi, ev)];
    E.flav[ai] = static_cast<int8_t>(wkappa);
    E.flav[aj] = static_cast<int8_t>(-wkappa);
    E.col[aj] = 0;
    E.acol[aj] = E.acol[ai];
    E.acol[ai] = 0;
    E.link[E.link_at(1, wi, ev)] = kNoLink;
    E.link[E.link_at(0, j, ev)] = kNoLink;
    E.link[E.link_at(1, j, ev)] = static_cast<uint8_t>(q);
    E.link[E.link_at(0, q, ev)] = static_cast<uint8_t>(j);
  } else {
    // A gluon enters the shared colour line between splitter and spectator;
    // the splitter takes the new line m.
    const int m = E.next_colour[ev];
    E.next_colour[ev] = m + 1;
    E.flav[aj] = static_cast<int8_t>(kGluon);
    if (wside == 0) {
      E.col[aj] = E.col[ai];
      E.acol[aj] = static_cast<int16_t>(m);
      E.col[ai] = static_cast<int16_t>(m);
      E.link[E.link_at(0, wi, ev)] = static_cast<uint8_t>(j);
      E.link[E.link_at(0, j, ev)] = static_cast<uint8_t>(wk);
      E.link[E.link_at(1, j, ev)] = static_cast<uint8_t>(wi);
      E.link[E.link_at(1, wk, ev)] = static_cast<uint8_t>(j);
    } else {
      E.col[aj] = static_cast<int16_t>(m);
      E.acol[aj] = E.acol[ai];
      E.acol[ai] = static_cast<int16_t>(m);
      E.link[E.link_at(1, wi, ev)] = static_cast<uint8_t>(j);
      E.link[E.link_at(1, j, ev)] = static_cast<uint8_t>(wk);
      E.link[E.link_at(0, j, ev)] = static_cast<uint8_t>(wi);
      E.link[E.link_at(0, wk, ev)] = static_cast<uint8_t>(j);
    }
  }
  E.n_partons[ev] = n + 1;
  E.n_emissions[ev] += 1;
}

}  // namespace

cudaError_t launch_me(const DevParams& P, const Events& E, cudaStream_t s) {
  if (E.n == 0) return cudaSuccess;
  const int threads = 256;
  const unsigned blocks = static_cast<unsigned>((E.n + threads - 1) / threads);
  k_me<<<blocks, threads, 0, s>>>(P, E);
  return cudaGetLastError();
}

cudaError_t launch_step_plain(const DevParams& P, const Events& E, cudaStream_t s) {
  if (E.n == 0) return cudaSuccess;
  const int threads = 128;
  const unsigned blocks = static_cast<unsigned>((E.n + threads - 1) / threads);
  k_step_plain<<<blocks, threads, 0, s>>>(P, E);
  return cudaGetLastError();
}

}  // namespace gaps
