// Oracle C interface (test infrastructure only; see oracle_api.h).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <thread>
#include <vector>

#include "oracle_internal.hpp"
#include "philox.hpp"

using namespace oracle;

namespace {

std::vector<Vec4> momenta_of(const Event& ev) {
  std::vector<Vec4> m;
  m.reserve(ev.partons.size());
  for (const Parton& q : ev.partons) m.push_back(q.p);
  return m;
}

// A given starting state (oracle_run_from_state) in place of the matrix
// element: its partons and the next free colour line.
struct StartState {
  std::vector<Parton> partons;
  int next_colour = 0;
};

void run_range(const oracle_params& p, uint32_t first_event, int64_t begin, int64_t end,
               oracle_event_out* out, double* mom, int32_t* info, double* obs, double* hist,
               const StartState* start) {
  const double s = p.sqrt_s * p.sqrt_s;
  Event ev;
  ev.partons.reserve(static_cast<size_t>(p.capacity) + 1);
  for (int64_t j = begin; j < end; ++j) {
    const uint32_t id = first_event + static_cast<uint32_t>(j);
    if (start) {
      ev.partons = start->partons;
      ev.next_colour = start->next_colour;
      ev.me_flavour = 0;
      ev.weight = 1.0;
    } else {
      generate_me(p, id, ev);
    }
    shower(p, id, ev);
    const int valid = validate(ev.partons, p.sqrt_s);
    double o[kNObs] = {-1, -1, -1, -1, -1, -1, -1, -1};
    if (ev.status == ORACLE_DONE) event_shapes(momenta_of(ev), s, p.mutation, o);
    if (out) {
      oracle_event_out& r = out[j];
      r.weight = ev.weight;
      r.t_first = ev.t_first;
      r.t_final = ev.t;
      r.hash = ev.hash;
      r.n_trials = ev.n_trials;
      r.me_flavour = ev.me_flavour;
      r.n_partons = static_cast<int32_t>(ev.partons.size());
      r.status = ev.status;
      r.n_steps = ev.n_steps;
      r.n_emissions = ev.n_emissions;
      r.n_winners = ev.n_winners;
      r.valid = valid;
      r.n_dipoles = ev.n_dipoles;
    }
    if (mom) {
      double* dst = mom + j * p.capacity * 4;
      for (size_t i = 0; i < ev.partons.size() && i < static_cast<size_t>(p.capacity); ++i) {
        dst[4 * i + 0] = ev.partons[i].p.e;
        dst[4 * i + 1] = ev.partons[i].p.x;
        dst[4 * i + 2] = ev.partons[i].p.y;
        dst[4 * i + 3] = ev.partons[i].p.z;
      }
    }
    if (info) {
      int32_t* dst = info + j * p.capacity * 3;
      for (size_t i = 0; i < ev.partons.size() && i < static_cast<size_t>(p.capacity); ++i) {
        dst[3 * i + 0] = ev.partons[i].flav;
        dst[3 * i + 1] = ev.partons[i].col;
        dst[3 * i + 2] = ev.partons[i].acol;
      }
    }
    if (obs) std::memcpy(obs + j * kNObs, o, sizeof(o));
    if (hist && ev.status == ORACLE_DONE) histogram_fill(hist, o, ev.weight);
  }
}

std::vector<Vec4> unpack(int n, const double* mom) {
  std::vector<Vec4> v(n);
  for (int i = 0; i < n; ++i) v[i] = Vec4{mom[4 * i], mom[4 * i + 1], mom[4 * i + 2], mom[4 * i + 3]};
  return v;
}

void pack(const Vec4& v, double* out) {
  out[0] = v.e;
  out[1] = v.x;
  out[2] = v.y;
  out[3] = v.z;
}

}  // namespace

extern "C" {

int oracle_check_params(const oracle_params* p) {
  if (!p) return -1;
  if (!(p->sqrt_s > 0.0) || !(p->t_cutoff > 0.0) || !(p->alphas_mz > 0.0)) return -1;
  if (!(p->t_cutoff < 0.25 * p->sqrt_s * p->sqrt_s)) return -1;
  if (p->n_flavours < 1 || p->n_flavours > 5) return -1;
  if (p->capacity < 2 || p->capacity > 1024 || p->max_steps < 1) return -1;
  if (p->trial_mode != 0 && p->trial_mode != 1) return -1;
  // The one-loop coupling must stay finite and positive down to the cutoff.
  if (!p->fixed_alphas) {
    const double b0 = (33.0 - 2.0 * p->n_flavours) / (12.0 * kPi);
    if (!(1.0 + p->alphas_mz * b0 * std::log(p->t_cutoff / (kMZ * kMZ)) > 0.0)) return -1;
  }
  return 0;
}

int oracle_run(const oracle_params* p, uint32_t first_event, int64_t n_events, int n_threads,
               oracle_event_out* out, double* mom, int32_t* info, double* obs, double* hist) {
  if (oracle_check_params(p) != 0 || n_events < 0) return -1;
  if (mom) std::memset(mom, 0, sizeof(double) * n_events * p->capacity * 4);
  if (info) std::memset(info, 0, sizeof(int32_t) * n_events * p->capacity * 3);
  const size_t hsize = static_cast<size_t>(kNObs) * kRow * 3;
  if (n_threads <= 1 || n_events < 2 * n_threads) {
    run_range(*p, first_event, 0, n_events, out, mom, info, obs, hist, nullptr);
    return 0;
  }
  std::vector<std::vector<double>> partial(n_threads, std::vector<double>(hist ? hsize : 0, 0.0));
  std::vector<std::thread> pool;
  for (int t = 0; t < n_threads; ++t) {
    const int64_t b = n_events * t / n_threads;
    const int64_t e = n_events * (t + 1) / n_threads;
    double* h = hist ? partial[t].data() : nullptr;
    pool.emplace_back(run_range, std::cref(*p), first_event, b, e, out, mom, info, obs, h,
                      static_cast<const StartState*>(nullptr));
  }
  for (auto& th : pool) th.join();
  if (hist)
    for (int t = 0; t < n_threads; ++t)
      for (size_t i = 0; i < hsize; ++i) hist[i] += partial[t][i];
  return 0;
}

int oracle_run_from_state(const oracle_params* p, int n_init, const double* mom, const int32_t* info,
                          uint32_t first_event, int64_t n_events, int n_threads, oracle_event_out* out,
                          double* mom_out, int32_t* info_out) {
  if (oracle_check_params(p) != 0 || n_events < 0 || !mom || !info || n_init < 2 || n_init > p->capacity)
    return -1;
  StartState st;
  int top = 0;
  for (int i = 0; i < n_init; ++i) {
    const Parton q{Vec4{mom[4 * i], mom[4 * i + 1], mom[4 * i + 2], mom[4 * i + 3]}, info[3 * i], info[3 * i + 1],
                   info[3 * i + 2]};
    if (q.col < 0 || q.acol < 0 || q.col >= 1000 || q.acol >= 1000) return -1;
    top = std::max(top, std::max(q.col, q.acol));
    st.partons.push_back(q);
  }
  st.next_colour = top + 1;
  if (mom_out) std::memset(mom_out, 0, sizeof(double) * n_events * p->capacity * 4);
  if (info_out) std::memset(info_out, 0, sizeof(int32_t) * n_events * p->capacity * 3);
  if (n_threads <= 1 || n_events < 2 * n_threads) {
    run_range(*p, first_event, 0, n_events, out, mom_out, info_out, nullptr, nullptr, &st);
    return 0;
  }
  std::vector<std::thread> pool;
  for (int t = 0; t < n_threads; ++t) {
    const int64_t b = n_events * t / n_threads;
    const int64_t e = n_events * (t + 1) / n_threads;
    pool.emplace_back(run_range, std::cref(*p), first_event, b, e, out, mom_out, info_out,
                      static_cast<double*>(nullptr), static_cast<double*>(nullptr),
                      static_cast<const StartState*>(&st));
  }
  for (auto& th : pool) th.join();
  return 0;
}

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const Draw4 d = philox4x32_10(ctr[0], ctr[1], ctr[2], ctr[3], key[0], key[1]);
  for (int i = 0; i < 4; ++i) out[i] = d.w[i];
}

void oracle_uniform_pair(uint64_t seed, uint32_t event, uint32_t step, uint32_t slot,
                         uint32_t purpose, double out[2]) {
  const UniformPair u = uniform_pair(seed, event, step, slot, purpose);
  out[0] = u.u0;
  out[1] = u.u1;
}

double oracle_dsigma_dcos(const oracle_params* p, int flavour, double cos_theta) {
  return dsigma_dcos(p->sqrt_s * p->sqrt_s, flavour, cos_theta,
                     (p->mutation & ORACLE_MUT_ME_NO_INTERF) != 0);
}

double oracle_alphas(const oracle_params* p, double t) {
  return alphas_at(t, p->alphas_mz, p->n_flavours, p->fixed_alphas != 0);
}

double oracle_alphas_over(const oracle_params* p) {
  return alphas_at(p->t_cutoff, p->alphas_mz, p->n_flavours, p->fixed_alphas != 0);
}

double oracle_kernel_value(int kind, double z, double y) { return kernel_value(kind, z, y); }
double oracle_kernel_estimate(int kind, double z) { return kernel_estimate(kind, z); }
double oracle_kernel_integral(int kind, double zm, double zp) { return kernel_integral(kind, zm, zp); }
double oracle_kernel_generate_z(int kind, double zm, double zp, double u, int mutation) {
  return kernel_generate_z(kind, zm, zp, u, (mutation & ORACLE_MUT_Z_UNIFORM) != 0);
}

int oracle_splitting_map(const double pij[4], const double pk[4], double z, double y, double phi,
                         int mutation, double pi_out[4], double pj_out[4], double pk_out[4]) {
  const Vec4 a{pij[0], pij[1], pij[2], pij[3]};
  const Vec4 b{pk[0], pk[1], pk[2], pk[3]};
  const MapMutations mut{(mutation & ORACLE_MUT_NO_RECOIL) != 0, (mutation & ORACLE_MUT_KT_SIGN) != 0,
                         (mutation & ORACLE_MUT_Z_SWAP) != 0};
  Vec4 mi, mj, mk;
  splitting_map(a, b, z, y, phi, mut, mi, mj, mk);
  pack(mi, pi_out);
  pack(mj, pj_out);
  pack(mk, pk_out);
  return 0;
}

int oracle_durham(int n, const double* mom, double s, int mutation, double y_out[4]) {
  if (n < 1 || !mom) return -1;
  durham(unpack(n, mom), s, mutation, y_out);
  return 0;
}

int oracle_thrust(int n, const double* mom, int mutation, double out[4]) {
  if (n < 2 || !mom) return -1;
  Vec4 axis{};
  out[0] = thrust(unpack(n, mom), mutation, &axis);
  out[1] = axis.x;
  out[2] = axis.y;
  out[3] = axis.z;
  return 0;
}

int oracle_event_shapes(int n, const double* mom, double s, int mutation, double out[8]) {
  if (n < 2 || !mom) return -1;
  event_shapes(unpack(n, mom), s, mutation, out);
  return 0;
}

int oracle_validate(int n, const double* mom, const int32_t* info, double sqrt_s) {
  if (n < 0 || !mom || !info) return -1;
  std::vector<Parton> ps(n);
  for (int i = 0; i < n; ++i)
    ps[i] = Parton{Vec4{mom[4 * i], mom[4 * i + 1], mom[4 * i + 2], mom[4 * i + 3]}, info[3 * i],
                   info[3 * i + 1], info[3 * i + 2]};
  return validate(ps, sqrt_s);
}

}  // extern "C"
