// Observables of the finished events (Sec. 3.1): exact thrust and the
// heavy-jet mass, and the Durham jet resolutions y23..y56.
//
// Layout of the work.  The finished events are first bucketed by parton
// multiplicity (count, scan, scatter into an index list), so the threads of
// a warp handle events of the same size: the O(n^3) loops of thrust and
// Durham then run with no lane waiting on a larger neighbour.  Events of up
// to 16 partons take one thread each, with per-thread arrays (in batches of
// fewer than 50 000 events, groups of 4 lanes).  Larger events take a warp
// each: the event's momenta sit in shared memory, the lanes split the O(n^2)
// pairs of each search and reduce their partial results in the serial
// loop's order (the first pair wins ties, as in the oracle), and the O(n)
// FP64 steps run on every lane alike.  A single thread takes about 0.2 ms
// for one 16-parton event and 64 times that for 64 partons, and a launch
// waits for its largest event; the groups cut that wait by their width.
//
// Precision.  As in the shower, the searches run in FP32 and the answers in
// FP64:
//  * Thrust.  Every candidate partition P = sum s_i p_i of the exact
//    algorithm (planes through every pair, both signs of the pair) is scored
//    |P|^2 in FP32 and identified by its bitmask; the two best distinct
//    partitions are tracked.  When the best beats the runner-up by more than
//    the FP32 error bound, its |P| and axis are recomputed in FP64; otherwise
//    (or for more than 64 partons) the whole search runs in FP64.
//  * Durham.  Pair distances min(E_i^2, E_j^2) |u_i - u_j|^2 (u = unit
//    momentum, free of the 1 - cos cancellation) are compared in FP32 with a
//    per-pair error bound; every pair that could be the minimum is evaluated
//    with the FP64 formula 2 min(E_i^2, E_j^2)(1 - cos theta_ij)/s, and the
//    smallest of those is merged, ties to the first pair as in the oracle.
//  * Final scalings take reciprocals (1/s, 1/|P|, 1/(2 sum |p|)): the
//    oracle's divisions up to an ulp.  The cosine inside Durham's 1 - cos
//    keeps the oracle's division, since 1 - cos magnifies its rounding.
#include "gaps_launch.hpp"
#include "sqrt_obs.cuh"

namespace gaps {

namespace {

constexpr int kShapeThreads = 128;
constexpr int kMaskMax = 64;

// The products and sums of this file in fused form (the library is built
// without automatic contraction): both the per-thread and the lane-group
// forms below call these, so they round alike.
__device__ __forceinline__ float dot3f(float ax, float ay, float az, float bx, float by, float bz) {
  return fmaf(az, bz, fmaf(ay, by, ax * bx));
}
__device__ __forceinline__ float crossf(float a, float b, float c, float d) { return fmaf(a, b, -(c * d)); }
__device__ __forceinline__ double dot3(double ax, double ay, double az, double bx, double by, double bz) {
  return fma(az, bz, fma(ay, by, ax * bx));
}
__device__ __forceinline__ double cross(double a, double b, double c, double d) { return fma(a, b, -(c * d)); }
// The squared mass of a four-vector (e, x, y, z).
__device__ __forceinline__ double mass2(const double* h) {
  return fma(-h[3], h[3], fma(-h[2], h[2], fma(-h[1], h[1], h[0] * h[0])));
}

// Exact FP64 thrust search (the fallback): planes through every pair with a
// non-zero cross product, other momenta signed by their side, the pair tried
// with both signs; the longest P is the thrust axis.
template <int MAXJ>
__device__ double thrust_fp64(int n, const double* jx, const double* jy, const double* jz, double sum_abs,
                              double& ax, double& ay, double& az) {
  double best2 = -1.0, bx = 0.0, by = 0.0, bz = 0.0;
  for (int j = 0; j < n; ++j) {
    for (int k = j + 1; k < n; ++k) {
      const double nx = cross(jy[j], jz[k], jz[j], jy[k]);
      const double ny = cross(jz[j], jx[k], jx[j], jz[k]);
      const double nz = cross(jx[j], jy[k], jy[j], jx[k]);
      if (nx == 0.0 && ny == 0.0 && nz == 0.0) continue;
      double px = 0.0, py = 0.0, pz = 0.0;
      for (int i = 0; i < n; ++i) {
        if (i == j || i == k) continue;
        const double sg = dot3(jx[i], jy[i], jz[i], nx, ny, nz) >= 0.0 ? 1.0 : -1.0;
        px = fma(sg, jx[i], px);
        py = fma(sg, jy[i], py);
        pz = fma(sg, jz[i], pz);
      }
      for (int c = 0; c < 4; ++c) {
        const double fj = (c & 2) ? -1.0 : 1.0, fk = (c & 1) ? -1.0 : 1.0;
        const double cx = fma(fk, jx[k], fma(fj, jx[j], px));
        const double cy = fma(fk, jy[k], fma(fj, jy[j], py));
        const double cz = fma(fk, jz[k], fma(fj, jz[j], pz));
        const double c2 = dot3(cx, cy, cz, cx, cy, cz);
        if (c2 > best2) {
          best2 = c2;
          bx = cx;
          by = cy;
          bz = cz;
        }
      }
    }
  }
  if (best2 < 0.0) {  // collinear: T = 1 along the first momentum
    const double l = sqrt_obs(dot3(jx[0], jy[0], jz[0], jx[0], jy[0], jz[0]));
    ax = jx[0] / l;
    ay = jy[0] / l;
    az = jz[0] / l;
    return 1.0;
  }
  const double l = sqrt_obs(best2), inv_l = 1.0 / l;
  ax = bx * inv_l;
  ay = by * inv_l;
  az = bz * inv_l;
  return l / sum_abs;
}

// Top two distinct partitions by score.
struct Top2 {
  float s1 = -1.0f, s2 = -1.0f;
  unsigned long long m1 = 0ull, m2 = ~0ull;
  __device__ __forceinline__ void add(float s, unsigned long long m) {
    if (m == m1) {
      s1 = fmaxf(s1, s);
    } else if (s > s1) {
      s2 = s1;
      m2 = m1;
      s1 = s;
      m1 = m;
    } else if (m == m2) {
      s2 = fmaxf(s2, s);
    } else if (s > s2) {
      s2 = s;
      m2 = m;
    }
  }
};

template <int MAXJ>
__device__ void event_shapes(const DevParams& P0, const Events& E, int64_t ev, int n) {
  const DevParams& P = params_of_event(P0, E, ev);
  double je[MAXJ], jx[MAXJ], jy[MAXJ], jz[MAXJ], ja[MAXJ];  // ja: |p| of every jet
  float fx[MAXJ], fy[MAXJ], fz[MAXJ];
  double sum_abs = 0.0;
  float sum_absf = 0.0f;
  for (int i = 0; i < n; ++i) {
    const size_t a = E.at(i, ev);
    je[i] = E.e[a];
    jx[i] = E.px[a];
    jy[i] = E.py[a];
    jz[i] = E.pz[a];
    fx[i] = f32_from_f64(jx[i]);
    fy[i] = f32_from_f64(jy[i]);
    fz[i] = f32_from_f64(jz[i]);
    ja[i] = sqrt_obs(dot3(jx[i], jy[i], jz[i], jx[i], jy[i], jz[i]));
    sum_abs += ja[i];
  }
  sum_absf = f32_from_f64(sum_abs);

  // ---- thrust
  double thrust = 1.0, ax = 0.0, ay = 0.0, az = 0.0;
  bool decided = false;
  if (n == 2) {
    // no emission: the pair is back to back, T = 1 along the quark
    const double inv_l = 1.0 / ja[0];
    ax = jx[0] * inv_l;
    ay = jy[0] * inv_l;
    az = jz[0] * inv_l;
    decided = true;
  } else if (n <= kMaskMax) {
    Top2 top;
    const unsigned long long full = n == 64 ? ~0ull : ((1ull << n) - 1ull);
    for (int j = 0; j < n; ++j) {
      for (int k = j + 1; k < n; ++k) {
        const float nx = crossf(fy[j], fz[k], fz[j], fy[k]);
        const float ny = crossf(fz[j], fx[k], fx[j], fz[k]);
        const float nz = crossf(fx[j], fy[k], fy[j], fx[k]);
        if (nx == 0.0f && ny == 0.0f && nz == 0.0f) continue;
        float px = 0.0f, py = 0.0f, pz = 0.0f;
        unsigned long long mask = 0ull;
        for (int i = 0; i < n; ++i) {
          if (i == j || i == k) continue;
          if (dot3f(fx[i], fy[i], fz[i], nx, ny, nz) >= 0.0f) {
            px += fx[i];
            py += fy[i];
            pz += fz[i];
            mask |= 1ull << i;
          } else {
            px -= fx[i];
            py -= fy[i];
            pz -= fz[i];
          }
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const bool pj = !(c & 2), pk = !(c & 1);
          const float cx = px + (pj ? fx[j] : -fx[j]) + (pk ? fx[k] : -fx[k]);
          const float cy = py + (pj ? fy[j] : -fy[j]) + (pk ? fy[k] : -fy[k]);
          const float cz = pz + (pj ? fz[j] : -fz[j]) + (pk ? fz[k] : -fz[k]);
          unsigned long long m = mask | (pj ? 1ull << j : 0ull) | (pk ? 1ull << k : 0ull);
          if (m & 1ull) m = ~m & full;  // a partition and its complement are one candidate
          top.add(dot3f(cx, cy, cz, cx, cy, cz), m);
        }
      }
    }
    // FP32 error of |P|^2: n rounded terms of size <= sum |p| per component.
    const float margin = 8.0f * static_cast<float>(n + 2) * 6.0e-8f * sum_absf * sum_absf;
    if (top.s1 < 0.0f) {
      decided = false;  // no pair spans a plane: let the exact search decide
    } else if (top.s2 < top.s1 - margin) {
      double px = 0.0, py = 0.0, pz = 0.0;
      for (int i = 0; i < n; ++i) {
        const double sg = ((top.m1 >> i) & 1ull) ? 1.0 : -1.0;
        px = fma(sg, jx[i], px);
        py = fma(sg, jy[i], py);
        pz = fma(sg, jz[i], pz);
      }
      const double l = sqrt_obs(dot3(px, py, pz, px, py, pz)), inv_l = 1.0 / l;
      thrust = l / sum_abs;
      ax = px * inv_l;
      ay = py * inv_l;
      az = pz * inv_l;
      decided = true;
    }
  }
  if (!decided) {
    atomicAdd(&E.counters[4], 1ull);  // thrust decided by the exact FP64 search
    thrust = thrust_fp64<MAXJ>(n, jx, jy, jz, sum_abs, ax, ay, az);
  }
  // Hemispheres by the sign of p . n_T: heavy-jet mass, and the jet
  // broadenings B_+- = sum |p x n_T| / (2 sum |p|), B_T = B_+ + B_-,
  // B_W = max(B_+, B_-).
  double hp[4] = {0, 0, 0, 0}, hm[4] = {0, 0, 0, 0};
  double bp = 0.0, bm = 0.0;
  for (int i = 0; i < n; ++i) {
    // p . n >= 0 on the bits (-0 counts as 0; the FP64 pipe's compares cost
    // as much as its FMAs on this part)
    const long long pn = __double_as_longlong(dot3(jx[i], jy[i], jz[i], ax, ay, az));
    const bool plus = pn >= 0 || pn == static_cast<long long>(0x8000000000000000ull);
    double* h = plus ? hp : hm;
    h[0] += je[i];
    h[1] += jx[i];
    h[2] += jy[i];
    h[3] += jz[i];
    const double cx = cross(jy[i], az, jz[i], ay), cy = cross(jz[i], ax, jx[i], az), cz = cross(jx[i], ay, jy[i], ax);
    const double pt = sqrt_obs(dot3(cx, cy, cz, cx, cy, cz));
    if (plus) {
      bp += pt;
    } else {
      bm += pt;
    }
  }
  const double mp = mass2(hp);
  const double mm = mass2(hm);
  E.obs[4 * E.stride + ev] = 1.0 - thrust;
  E.obs[5 * E.stride + ev] = fmax(mp, mm) * P.inv_s;
  const double inv_2sum = 0.5 / sum_abs;
  bp *= inv_2sum;
  bm *= inv_2sum;
  E.obs[6 * E.stride + ev] = bp + bm;
  E.obs[7 * E.stride + ev] = fmax(bp, bm);

  // ---- Durham (E-scheme)
  float fe2[MAXJ];
  for (int i = 0; i < n; ++i) {
    const float e = f32_from_f64(je[i]);
    fe2[i] = e * e;
    const float r = rsqrtf(dot3f(fx[i], fy[i], fz[i], fx[i], fy[i], fz[i]));
    fx[i] *= r;  // from here on fx, fy, fz hold unit directions
    fy[i] *= r;
    fz[i] *= r;
  }
  double yres[4] = {-1.0, -1.0, -1.0, -1.0};
  // y of jets i, j with the oracle's FP64 formula (|p| cached per jet).
  auto y_exact = [&](int i, int j) {
    const double cosij = dot3(jx[i], jy[i], jz[i], jx[j], jy[j], jz[j]) / (ja[i] * ja[j]);
    return 2.0 * fmin(je[i] * je[i], je[j] * je[j]) * (1.0 - cosij) * P.inv_s;
  };
  for (int m = n; m > 1; --m) {
    // pass 1: the smallest upper bound of the FP32 distances, and its pair
    float ubest = INFINITY;
    int ui = 0, uj = 1;
    for (int i = 0; i < m; ++i) {
      for (int j = i + 1; j < m; ++j) {
        const float dx = fx[i] - fx[j], dy = fy[i] - fy[j], dz = fz[i] - fz[j];
        const float d = dot3f(dx, dy, dz, dx, dy, dz);
        const float y = fminf(fe2[i], fe2[j]) * d;
        const float rel = 4.0e-6f + 1.0e-6f * rsqrtf(fmaxf(d, 1e-30f));
        const float ub = fmaf(y, 1.0f + rel, 1e-30f);
        if (ub < ubest) {
          ubest = ub;
          ui = i;
          uj = j;
        }
      }
    }
    // pass 2: how many pairs have a lower bound that reaches it
    int n_cand = 0;
    for (int i = 0; i < m; ++i) {
      for (int j = i + 1; j < m; ++j) {
        const float dx = fx[i] - fx[j], dy = fy[i] - fy[j], dz = fz[i] - fz[j];
        const float d = dot3f(dx, dy, dz, dx, dy, dz);
        const float y = fminf(fe2[i], fe2[j]) * d;
        const float rel = 4.0e-6f + 1.0e-6f * rsqrtf(fmaxf(d, 1e-30f));
        n_cand += y * (1.0f - rel) <= ubest ? 1 : 0;
      }
    }
    // One candidate (nearly every merge): it is the pair of the smallest
    // upper bound and the exact minimum, evaluated once, in step with the
    // other lanes.  Otherwise every candidate in FP64, ties to the first
    // pair as in the oracle.
    double ymin = 0.0;
    int bi = ui, bj = uj;
    if (n_cand == 1) {
      ymin = y_exact(ui, uj);
    } else {
      atomicAdd(&E.counters[5], 1ull);  // merges with several FP64 candidates
      bi = -1;
      for (int i = 0; i < m; ++i) {
        for (int j = i + 1; j < m; ++j) {
          const float dx = fx[i] - fx[j], dy = fy[i] - fy[j], dz = fz[i] - fz[j];
          const float d = dot3f(dx, dy, dz, dx, dy, dz);
          const float y = fminf(fe2[i], fe2[j]) * d;
          const float rel = 4.0e-6f + 1.0e-6f * rsqrtf(fmaxf(d, 1e-30f));
          if (y * (1.0f - rel) > ubest) continue;
          const double yy = y_exact(i, j);
          if (bi < 0 || yy < ymin) {
            ymin = yy;
            bi = i;
            bj = j;
          }
        }
      }
    }
    const int idx = m - 3;
    if (idx >= 0 && idx < 4) yres[idx] = ymin;
    je[bi] += je[bj];
    jx[bi] += jx[bj];
    jy[bi] += jy[bj];
    jz[bi] += jz[bj];
    je[bj] = je[m - 1];
    jx[bj] = jx[m - 1];
    jy[bj] = jy[m - 1];
    jz[bj] = jz[m - 1];
    ja[bj] = ja[m - 1];
    ja[bi] = sqrt_obs(dot3(jx[bi], jy[bi], jz[bi], jx[bi], jy[bi], jz[bi]));
    fe2[bj] = fe2[m - 1];
    fx[bj] = fx[m - 1];
    fy[bj] = fy[m - 1];
    fz[bj] = fz[m - 1];
    {
      const float e = f32_from_f64(je[bi]);
      fe2[bi] = e * e;
      const float x = f32_from_f64(jx[bi]), y = f32_from_f64(jy[bi]), z = f32_from_f64(jz[bi]);
      const float r = rsqrtf(dot3f(x, y, z, x, y, z));
      fx[bi] = x * r;
      fy[bi] = y * r;
      fz[bi] = z * r;
    }
  }
  for (int h = 0; h < 4; ++h) E.obs[h * E.stride + ev] = yres[h];
}

// ------------------------------------------------------- lane groups
// Lanes of this thread's aligned group of L (L a power of two, <= 32).
template <int L>
__device__ __forceinline__ unsigned group_lanes() {
  if constexpr (L == 32) {
    return 0xffffffffu;
  } else {
    return ((1u << L) - 1u) << ((threadIdx.x & 31u) & ~static_cast<unsigned>(L - 1));
  }
}

// The pairs (j, k), j < k < n, of one lane: positions sub, sub + L, ... of
// the serial loop (j outer, k inner); p is the position.
struct PairWalk {
  int j, off, row, p;
  __device__ __forceinline__ void start(int n, int sub) {
    j = 0;
    off = sub;
    row = n - 1;
    p = sub;
    settle(n);
  }
  __device__ __forceinline__ void settle(int n) {
    while (j < n - 1 && off >= row) {
      off -= row;
      ++j;
      row = n - 1 - j;
    }
  }
  __device__ __forceinline__ bool valid(int n) const { return j < n - 1; }
  __device__ __forceinline__ int k() const { return j + 1 + off; }
  template <int L>
  __device__ __forceinline__ void next(int n) {
    off += L;
    p += L;
    settle(n);
  }
};

// The event's arrays in shared memory, one set per group.
template <int MAXJ>
struct GroupArrays {
  double je[MAXJ], jx[MAXJ], jy[MAXJ], jz[MAXJ], ja[MAXJ];
  float fx[MAXJ], fy[MAXJ], fz[MAXJ], fe2[MAXJ];
};

// thrust_fp64 over the group: each lane takes its pairs, the group keeps the
// longest P and, on equal lengths, the first candidate in the serial loop's
// order (pair position x 4 + sign choice), so the result is the serial one.
template <int MAXJ, int L>
__device__ double thrust_fp64_group(int n, const GroupArrays<MAXJ>& a, double sum_abs, int sub, unsigned gm,
                                    double& ax, double& ay, double& az) {
  double best2 = -1.0, bx = 0.0, by = 0.0, bz = 0.0;
  int bidx = 0x7fffffff;
  PairWalk w;
  for (w.start(n, sub); w.valid(n); w.next<L>(n)) {
    const int j = w.j, k = w.k();
    const double nx = cross(a.jy[j], a.jz[k], a.jz[j], a.jy[k]);
    const double ny = cross(a.jz[j], a.jx[k], a.jx[j], a.jz[k]);
    const double nz = cross(a.jx[j], a.jy[k], a.jy[j], a.jx[k]);
    if (nx == 0.0 && ny == 0.0 && nz == 0.0) continue;
    double px = 0.0, py = 0.0, pz = 0.0;
    for (int i = 0; i < n; ++i) {
      if (i == j || i == k) continue;
      const double sg = dot3(a.jx[i], a.jy[i], a.jz[i], nx, ny, nz) >= 0.0 ? 1.0 : -1.0;
      px = fma(sg, a.jx[i], px);
      py = fma(sg, a.jy[i], py);
      pz = fma(sg, a.jz[i], pz);
    }
    for (int c = 0; c < 4; ++c) {
      const double fj = (c & 2) ? -1.0 : 1.0, fk = (c & 1) ? -1.0 : 1.0;
      const double cx = fma(fk, a.jx[k], fma(fj, a.jx[j], px));
      const double cy = fma(fk, a.jy[k], fma(fj, a.jy[j], py));
      const double cz = fma(fk, a.jz[k], fma(fj, a.jz[j], pz));
      const double c2 = dot3(cx, cy, cz, cx, cy, cz);
      if (c2 > best2) {  // within a lane the positions rise: the first wins ties
        best2 = c2;
        bidx = 4 * w.p + c;
        bx = cx;
        by = cy;
        bz = cz;
      }
    }
  }
#pragma unroll
  for (int off = 1; off < L; off <<= 1) {
    const double o2 = __shfl_xor_sync(gm, best2, off);
    const int oi = __shfl_xor_sync(gm, bidx, off);
    const double ox = __shfl_xor_sync(gm, bx, off), oy = __shfl_xor_sync(gm, by, off);
    const double oz = __shfl_xor_sync(gm, bz, off);
    if (o2 > best2 || (o2 == best2 && oi < bidx)) {
      best2 = o2;
      bidx = oi;
      bx = ox;
      by = oy;
      bz = oz;
    }
  }
  if (best2 < 0.0) {  // collinear: T = 1 along the first momentum
    const double l = sqrt_obs(dot3(a.jx[0], a.jy[0], a.jz[0], a.jx[0], a.jy[0], a.jz[0]));
    ax = a.jx[0] / l;
    ay = a.jy[0] / l;
    az = a.jz[0] / l;
    return 1.0;
  }
  const double l = sqrt_obs(best2), inv_l = 1.0 / l;
  ax = bx * inv_l;
  ay = by * inv_l;
  az = bz * inv_l;
  return l / sum_abs;
}

// event_shapes for one event by a group of L lanes (every lane of the group
// calls it for the same event).  The searches give exactly the serial
// results: each lane screens its pairs in the serial order, the group merges
// the lanes' bests with the serial tie rule, and the O(n) FP64 steps (the
// thrust sum, hemispheres, broadenings, the merged jets) run on every lane in
// the serial order.  Lane 0 of the group writes the observables.
template <int MAXJ, int L>
__device__ void event_shapes_group(const DevParams& P0, const Events& E, int64_t ev, int n, GroupArrays<MAXJ>& a,
                                   int sub, unsigned gm) {
  const DevParams& P = params_of_event(P0, E, ev);
  for (int i = sub; i < n; i += L) {
    const size_t at = E.at(i, ev);
    const double x = E.px[at], y = E.py[at], z = E.pz[at];
    a.je[i] = E.e[at];
    a.jx[i] = x;
    a.jy[i] = y;
    a.jz[i] = z;
    a.fx[i] = f32_from_f64(x);
    a.fy[i] = f32_from_f64(y);
    a.fz[i] = f32_from_f64(z);
    a.ja[i] = sqrt_obs(dot3(x, y, z, x, y, z));
  }
  __syncwarp(gm);
  double sum_abs = 0.0;
  for (int i = 0; i < n; ++i) sum_abs += a.ja[i];
  const float sum_absf = f32_from_f64(sum_abs);

  // ---- thrust
  double thrust = 1.0, ax = 0.0, ay = 0.0, az = 0.0;
  bool decided = false;
  if (n == 2) {
    const double inv_l = 1.0 / a.ja[0];
    ax = a.jx[0] * inv_l;
    ay = a.jy[0] * inv_l;
    az = a.jz[0] * inv_l;
    decided = true;
  } else if (n <= kMaskMax) {
    Top2 top;
    const unsigned long long full = n == 64 ? ~0ull : ((1ull << n) - 1ull);
    PairWalk w;
    for (w.start(n, sub); w.valid(n); w.next<L>(n)) {
      const int j = w.j, k = w.k();
      const float nx = crossf(a.fy[j], a.fz[k], a.fz[j], a.fy[k]);
      const float ny = crossf(a.fz[j], a.fx[k], a.fx[j], a.fz[k]);
      const float nz = crossf(a.fx[j], a.fy[k], a.fy[j], a.fx[k]);
      if (nx == 0.0f && ny == 0.0f && nz == 0.0f) continue;
      float px = 0.0f, py = 0.0f, pz = 0.0f;
      unsigned long long mask = 0ull;
      for (int i = 0; i < n; ++i) {
        if (i == j || i == k) continue;
        if (dot3f(a.fx[i], a.fy[i], a.fz[i], nx, ny, nz) >= 0.0f) {
          px += a.fx[i];
          py += a.fy[i];
          pz += a.fz[i];
          mask |= 1ull << i;
        } else {
          px -= a.fx[i];
          py -= a.fy[i];
          pz -= a.fz[i];
        }
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const bool pj = !(c & 2), pk = !(c & 1);
        const float cx = px + (pj ? a.fx[j] : -a.fx[j]) + (pk ? a.fx[k] : -a.fx[k]);
        const float cy = py + (pj ? a.fy[j] : -a.fy[j]) + (pk ? a.fy[k] : -a.fy[k]);
        const float cz = pz + (pj ? a.fz[j] : -a.fz[j]) + (pk ? a.fz[k] : -a.fz[k]);
        unsigned long long m = mask | (pj ? 1ull << j : 0ull) | (pk ? 1ull << k : 0ull);
        if (m & 1ull) m = ~m & full;
        top.add(dot3f(cx, cy, cz, cx, cy, cz), m);
      }
    }
    // The top two distinct partitions of the union: each lane's two entries
    // added to the other's (the best score of every partition reaches the
    // merged pair; only which of two equal scores is first can depend on
    // the order, and equal scores leave the search to the exact FP64 pass).
#pragma unroll
    for (int off = 1; off < L; off <<= 1) {
      const float s1 = __shfl_xor_sync(gm, top.s1, off), s2 = __shfl_xor_sync(gm, top.s2, off);
      const unsigned long long m1 = __shfl_xor_sync(gm, top.m1, off), m2 = __shfl_xor_sync(gm, top.m2, off);
      top.add(s1, m1);
      top.add(s2, m2);
    }
    const float margin = 8.0f * static_cast<float>(n + 2) * 6.0e-8f * sum_absf * sum_absf;
    if (top.s1 >= 0.0f && top.s2 < top.s1 - margin) {
      double px = 0.0, py = 0.0, pz = 0.0;
      for (int i = 0; i < n; ++i) {
        const double sg = ((top.m1 >> i) & 1ull) ? 1.0 : -1.0;
        px = fma(sg, a.jx[i], px);
        py = fma(sg, a.jy[i], py);
        pz = fma(sg, a.jz[i], pz);
      }
      const double l = sqrt_obs(dot3(px, py, pz, px, py, pz)), inv_l = 1.0 / l;
      thrust = l / sum_abs;
      ax = px * inv_l;
      ay = py * inv_l;
      az = pz * inv_l;
      decided = true;
    }
  }
  if (!decided) {
    if (sub == 0) atomicAdd(&E.counters[4], 1ull);  // thrust decided by the exact FP64 search
    thrust = thrust_fp64_group<MAXJ, L>(n, a, sum_abs, sub, gm, ax, ay, az);
  }
  double hp[4] = {0, 0, 0, 0}, hm[4] = {0, 0, 0, 0};
  double bp = 0.0, bm = 0.0;
  for (int i = 0; i < n; ++i) {
    const double x = a.jx[i], y = a.jy[i], z = a.jz[i];
    const long long pn = __double_as_longlong(dot3(x, y, z, ax, ay, az));
    const bool plus = pn >= 0 || pn == static_cast<long long>(0x8000000000000000ull);
    double* h = plus ? hp : hm;
    h[0] += a.je[i];
    h[1] += x;
    h[2] += y;
    h[3] += z;
    const double cx = cross(y, az, z, ay), cy = cross(z, ax, x, az), cz = cross(x, ay, y, ax);
    const double pt = sqrt_obs(dot3(cx, cy, cz, cx, cy, cz));
    if (plus) {
      bp += pt;
    } else {
      bm += pt;
    }
  }
  if (sub == 0) {
    const double mp = mass2(hp);
    const double mm = mass2(hm);
    E.obs[4 * E.stride + ev] = 1.0 - thrust;
    E.obs[5 * E.stride + ev] = fmax(mp, mm) * P.inv_s;
    const double inv_2sum = 0.5 / sum_abs;
    bp *= inv_2sum;
    bm *= inv_2sum;
    E.obs[6 * E.stride + ev] = bp + bm;
    E.obs[7 * E.stride + ev] = fmax(bp, bm);
  }

  // ---- Durham (E-scheme)
  __syncwarp(gm);  // every lane has read the FP32 momenta
  for (int i = sub; i < n; i += L) {
    const float e = f32_from_f64(a.je[i]);
    a.fe2[i] = e * e;
    const float r = rsqrtf(dot3f(a.fx[i], a.fy[i], a.fz[i], a.fx[i], a.fy[i], a.fz[i]));
    a.fx[i] *= r;
    a.fy[i] *= r;
    a.fz[i] *= r;
  }
  __syncwarp(gm);
  double yres[4] = {-1.0, -1.0, -1.0, -1.0};
  auto y_exact = [&](int i, int j) {
    const double cosij = dot3(a.jx[i], a.jy[i], a.jz[i], a.jx[j], a.jy[j], a.jz[j]) / (a.ja[i] * a.ja[j]);
    return 2.0 * fmin(a.je[i] * a.je[i], a.je[j] * a.je[j]) * (1.0 - cosij) * P.inv_s;
  };
  auto bounds = [&](int i, int j, float& y, float& rel) {
    const float dx = a.fx[i] - a.fx[j], dy = a.fy[i] - a.fy[j], dz = a.fz[i] - a.fz[j];
    const float d = dot3f(dx, dy, dz, dx, dy, dz);
    y = fminf(a.fe2[i], a.fe2[j]) * d;
    rel = 4.0e-6f + 1.0e-6f * rsqrtf(fmaxf(d, 1e-30f));
  };
  for (int m = n; m > 1; --m) {
    // pass 1: the smallest FP32 upper bound, the first pair on ties
    float ubest = INFINITY;
    int up = 0x7fffffff, ui = 0, uj = 1;
    PairWalk w;
    for (w.start(m, sub); w.valid(m); w.next<L>(m)) {
      float y, rel;
      bounds(w.j, w.k(), y, rel);
      const float ub = fmaf(y, 1.0f + rel, 1e-30f);
      if (ub < ubest) {
        ubest = ub;
        up = w.p;
        ui = w.j;
        uj = w.k();
      }
    }
#pragma unroll
    for (int off = 1; off < L; off <<= 1) {
      const float ou = __shfl_xor_sync(gm, ubest, off);
      const int op = __shfl_xor_sync(gm, up, off), oi = __shfl_xor_sync(gm, ui, off);
      const int oj = __shfl_xor_sync(gm, uj, off);
      if (ou < ubest || (ou == ubest && op < up)) {
        ubest = ou;
        up = op;
        ui = oi;
        uj = oj;
      }
    }
    // pass 2: the pairs whose lower bound reaches it
    int n_cand = 0;
    for (w.start(m, sub); w.valid(m); w.next<L>(m)) {
      float y, rel;
      bounds(w.j, w.k(), y, rel);
      n_cand += y * (1.0f - rel) <= ubest ? 1 : 0;
    }
#pragma unroll
    for (int off = 1; off < L; off <<= 1) n_cand += __shfl_xor_sync(gm, n_cand, off);
    double ymin = 0.0;
    int bi = ui, bj = uj;
    if (n_cand == 1) {
      ymin = y_exact(ui, uj);
    } else {
      if (sub == 0) atomicAdd(&E.counters[5], 1ull);  // merges with several FP64 candidates
      int bp_ = 0x7fffffff;
      ymin = INFINITY;
      for (w.start(m, sub); w.valid(m); w.next<L>(m)) {
        float y, rel;
        bounds(w.j, w.k(), y, rel);
        if (y * (1.0f - rel) > ubest) continue;
        const double yy = y_exact(w.j, w.k());
        if (bp_ == 0x7fffffff || yy < ymin) {
          ymin = yy;
          bp_ = w.p;
          bi = w.j;
          bj = w.k();
        }
      }
#pragma unroll
      for (int off = 1; off < L; off <<= 1) {
        const double oy = __shfl_xor_sync(gm, ymin, off);
        const int op = __shfl_xor_sync(gm, bp_, off), oi = __shfl_xor_sync(gm, bi, off);
        const int oj = __shfl_xor_sync(gm, bj, off);
        // lanes without a candidate hold position 0x7fffffff
        if (op != 0x7fffffff && (bp_ == 0x7fffffff || oy < ymin || (oy == ymin && op < bp_))) {
          ymin = oy;
          bp_ = op;
          bi = oi;
          bj = oj;
        }
      }
    }
    const int idx = m - 3;
    if (idx >= 0 && idx < 4) yres[idx] = ymin;
    __syncwarp(gm);  // every lane is done reading the jets of this merge
    if (sub == 0) {
      a.je[bi] += a.je[bj];
      a.jx[bi] += a.jx[bj];
      a.jy[bi] += a.jy[bj];
      a.jz[bi] += a.jz[bj];
      a.je[bj] = a.je[m - 1];
      a.jx[bj] = a.jx[m - 1];
      a.jy[bj] = a.jy[m - 1];
      a.jz[bj] = a.jz[m - 1];
      a.ja[bj] = a.ja[m - 1];
      a.ja[bi] = sqrt_obs(dot3(a.jx[bi], a.jy[bi], a.jz[bi], a.jx[bi], a.jy[bi], a.jz[bi]));
      a.fe2[bj] = a.fe2[m - 1];
      a.fx[bj] = a.fx[m - 1];
      a.fy[bj] = a.fy[m - 1];
      a.fz[bj] = a.fz[m - 1];
      const float e = f32_from_f64(a.je[bi]);
      a.fe2[bi] = e * e;
      const float x = f32_from_f64(a.jx[bi]), y = f32_from_f64(a.jy[bi]), z = f32_from_f64(a.jz[bi]);
      const float r = rsqrtf(dot3f(x, y, z, x, y, z));
      a.fx[bi] = x * r;
      a.fy[bi] = y * r;
      a.fz[bi] = z * r;
    }
    __syncwarp(gm);
  }
  if (sub == 0)
    for (int h = 0; h < 4; ++h) E.obs[h * E.stride + ev] = yres[h];
}

// ------------------------------------------------------------- buckets
// Parton count of event ev if it gets observables: finished, with 2 ..
// capacity partons (the shower never writes another count; callers that pass
// their own arrays may), else -1.
__device__ __forceinline__ int shape_partons(const Events& E, int64_t ev) {
  if (E.status[ev] != GAPS_DONE) return -1;
  const int n = E.n_partons[ev];
  return n >= 2 && n <= E.cap ? n : -1;
}

// counts[n] = finished events with n partons (2 <= n <= capacity <= 255).
__global__ void __launch_bounds__(256) k_bucket_count(Events E, int* counts, Ranges R) {
  __shared__ int sh[256];
  sh[threadIdx.x] = 0;
  __syncthreads();
  for (int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < E.n;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int n = shape_partons(E, R.event(t));
    if (n >= 0) atomicAdd(&sh[n], 1);
  }
  __syncthreads();
  if (sh[threadIdx.x]) atomicAdd(&counts[threadIdx.x], sh[threadIdx.x]);
}

// offsets[n] = first position of bucket n; cursor[n] = offsets[n];
// offsets[256] = number of finished events.
__global__ void __launch_bounds__(256) k_bucket_scan(const int* counts, int* offsets, int* cursor) {
  __shared__ int sh[256];
  const int t = threadIdx.x;
  sh[t] = counts[t];
  __syncthreads();
  for (int d = 1; d < 256; d <<= 1) {
    const int v = t >= d ? sh[t - d] : 0;
    __syncthreads();
    sh[t] += v;
    __syncthreads();
  }
  const int excl = t ? sh[t - 1] : 0;
  offsets[t] = excl;
  cursor[t] = excl;
  if (t == 255) offsets[256] = sh[255];
}

// Finished events go to their bucket; the others get undefined observables,
// and so do finished events with a parton count outside 2 .. capacity
// (counted in counter word 8).
// A warp's lanes of one bucket take their places with one shared-memory
// atomic, a block's with one global atomic per bucket and round, so the
// few hot buckets (a handful of multiplicities hold most events) see a
// thousand times fewer global atomics than with one per event.
__global__ void __launch_bounds__(256) k_bucket_scatter(Events E, int* cursor, int* order, Ranges R) {
  __shared__ int s_cnt[256];
  __shared__ int s_base[256];
  const int tid = threadIdx.x, lane = tid & 31;
  for (int64_t first = static_cast<int64_t>(blockIdx.x) * 256; first < E.n;
       first += static_cast<int64_t>(gridDim.x) * 256) {
    s_cnt[tid] = 0;
    __syncthreads();
    const int64_t t = first + tid;
    const int64_t ev = t < E.n ? R.event(t) : 0;
    int n = -1;
    if (t < E.n) {
      n = shape_partons(E, ev);
      if (n < 0) {
        if (E.status[ev] == GAPS_DONE) atomicAdd(&E.counters[8], 1ull);
        for (int h = 0; h < GAPS_N_OBS; ++h) E.obs[h * E.stride + ev] = -1.0;
      }
    }
    const unsigned peers = __match_any_sync(0xffffffffu, n);
    const int leader = __ffs(peers) - 1;
    int at = 0;
    if (n >= 0 && lane == leader) at = atomicAdd(&s_cnt[n], __popc(peers));
    at = __shfl_sync(0xffffffffu, at, leader) + __popc(peers & ((1u << lane) - 1u));
    __syncthreads();
    if (s_cnt[tid]) s_base[tid] = atomicAdd(&cursor[tid], s_cnt[tid]);
    __syncthreads();
    if (n >= 0) order[s_base[n] + at] = static_cast<int>(ev);
    __syncthreads();  // s_cnt and s_base are reused by the next round
  }
}

// Events of buckets n_lo..n_hi (all with n <= MAXJ), the largest first: the
// order list holds the buckets by rising multiplicity, and the threads take
// it from its end, so the blocks with the costliest events start first and
// the cheap ones fill the SMs that free up (a launch otherwise waits for the
// blocks of its largest events, dealt out last).
template <int MAXJ>
__global__ void __launch_bounds__(kShapeThreads) k_event_shapes(DevParams P, Events E, const int* order,
                                                                const int* offsets, int n_lo, int n_hi) {
  const int begin = offsets[n_lo], end = offsets[n_hi + 1 > 256 ? 256 : n_hi + 1];
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < end - begin; j += gridDim.x * blockDim.x) {
    const int64_t ev = order[end - 1 - j];
    event_shapes<MAXJ>(P, E, ev, E.n_partons[ev]);
  }
}

// Events of buckets n_lo..n_hi (all with n <= MAXJ), L lanes per event, T
// threads per block.
template <int MAXJ, int L, int T>
__global__ void __launch_bounds__(T) k_event_shapes_group(DevParams P, Events E, const int* order,
                                                          const int* offsets, int n_lo, int n_hi) {
  constexpr int G = T / L;
  __shared__ GroupArrays<MAXJ> s_ev[G];
  const int g = threadIdx.x / L, sub = threadIdx.x % L;
  const unsigned gm = group_lanes<L>();
  const int begin = offsets[n_lo], end = offsets[n_hi + 1 > 256 ? 256 : n_hi + 1];
  for (int k = begin + blockIdx.x * G + g; k < end; k += gridDim.x * G) {
    const int64_t ev = order[k];
    event_shapes_group<MAXJ, L>(P, E, ev, E.n_partons[ev], s_ev[g], sub, gm);
    __syncwarp(gm);  // the group's arrays are free for its next event
  }
}

// Events of up to 16 partons take one thread each in batches of at least
// GAPS_SHAPES_GROUP_BELOW events (throughput), groups of
// GAPS_SHAPES_SMALL_LANES lanes in smaller ones (a launch then waits for its
// slowest event, not for the SMs).  At 10^6 LEP events one thread per event
// up to 16 partons measured 1.04 ms for the observables, against 1.47 ms with
// 9..16-parton events in groups of 8 and 1.36 ms with the per-thread events
// in two launches (up to 8 partons, 9..16).  The per-thread grid holds one
// thread per event up to GAPS_SHAPES_BLOCKS_PER_SM blocks per SM (largest
// events first, above): 0.919 ms at 10^6 events and 0.623 ms at 5x10^5,
// against 0.967 and 0.702 ms for 16 blocks per SM striding over the events
// in rising size, and 1.168 and 0.726 ms for a grid of the resident blocks
// only.
#ifndef GAPS_SHAPES_BLOCKS_PER_SM
#define GAPS_SHAPES_BLOCKS_PER_SM 64
#endif
#ifndef GAPS_SHAPES_GROUP_BELOW
#define GAPS_SHAPES_GROUP_BELOW 50000
#endif
#ifndef GAPS_SHAPES_SMALL_LANES
#define GAPS_SHAPES_SMALL_LANES 4
#endif
constexpr int kSmallLanes = GAPS_SHAPES_SMALL_LANES;

}  // namespace

cudaError_t preload_observables() {
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, k_bucket_count);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_bucket_scan);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_bucket_scatter);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_event_shapes<16>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_event_shapes_group<16, kSmallLanes, 128>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_event_shapes_group<32, 32, 128>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_event_shapes_group<64, 32, 128>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_event_shapes_group<128, 32, 128>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_event_shapes_group<256, 32, 64>);
  return e;
}

cudaError_t launch_observables(const DevParams& P, const Events& E, int* buckets, int* order, cudaStream_t s,
                               const Ranges& R) {
  if (E.n == 0) return cudaSuccess;
  int sms = 152, dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int* counts = buckets;
  int* offsets = buckets + 256;
  int* cursor = buckets + 256 + 257;
  cudaError_t e = cudaMemsetAsync(counts, 0, 256 * sizeof(int), s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(E.counters + 4, 0, 2 * sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(E.counters + 8, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  const int64_t want = (E.n + 255) / 256;
  const unsigned grid_count = static_cast<unsigned>(want < 4 * sms ? want : 4 * sms);
  k_bucket_count<<<grid_count, 256, 0, s>>>(E, counts, R);
  k_bucket_scan<<<1, 256, 0, s>>>(counts, offsets, cursor);
  k_bucket_scatter<<<grid_count, 256, 0, s>>>(E, cursor, order, R);
  // One launch per multiplicity class; grids cover the largest possible
  // class (blocks of one event per thread or per group) and stride over the
  // actual one.
  auto grid = [&](int per_block, int per_sm) {
    const int64_t want = (E.n + per_block - 1) / per_block;
    return static_cast<unsigned>(want < static_cast<int64_t>(per_sm) * sms ? want : static_cast<int64_t>(per_sm) * sms);
  };
  if (E.n < GAPS_SHAPES_GROUP_BELOW) {
    k_event_shapes_group<16, kSmallLanes, 128><<<grid(128 / kSmallLanes, 8), 128, 0, s>>>(P, E, order, offsets, 0, 16);
  } else {
    k_event_shapes<16><<<grid(kShapeThreads, GAPS_SHAPES_BLOCKS_PER_SM), kShapeThreads, 0, s>>>(P, E, order, offsets, 0, 16);
  }
  if (E.cap > 16) k_event_shapes_group<32, 32, 128><<<grid(4, 2), 128, 0, s>>>(P, E, order, offsets, 17, 32);
  if (E.cap > 32) k_event_shapes_group<64, 32, 128><<<grid(4, 2), 128, 0, s>>>(P, E, order, offsets, 33, 64);
  if (E.cap > 64) k_event_shapes_group<128, 32, 128><<<grid(4, 2), 128, 0, s>>>(P, E, order, offsets, 65, 128);
  if (E.cap > 128) k_event_shapes_group<256, 32, 64><<<grid(2, 2), 64, 0, s>>>(P, E, order, offsets, 129, 255);
  return cudaGetLastError();
}

}  // namespace gaps
