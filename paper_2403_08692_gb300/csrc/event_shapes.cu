// Observables of the finished events (Sec. 3.1): exact thrust and the
// heavy-jet mass, and the Durham jet resolutions y23..y56.
//
// Layout of the work.  The finished events are first bucketed by parton
// multiplicity (count, scan, scatter into an index list), so the threads of
// a warp handle events of the same size: the O(n^3) loops of thrust and
// Durham then run with no lane waiting on a larger neighbour.  One thread
// handles one event, with per-thread arrays sized by the bucket (16, 32, 64,
// 128 or 256 partons).
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

namespace gaps {

namespace {

constexpr int kShapeThreads = 128;
constexpr int kMaskMax = 64;

// Exact FP64 thrust search (the fallback): planes through every pair with a
// non-zero cross product, other momenta signed by their side, the pair tried
// with both signs; the longest P is the thrust axis.
template <int MAXJ>
__device__ double thrust_fp64(int n, const double* jx, const double* jy, const double* jz, double sum_abs,
                              double& ax, double& ay, double& az) {
  double best2 = -1.0, bx = 0.0, by = 0.0, bz = 0.0;
  for (int j = 0; j < n; ++j) {
    for (int k = j + 1; k < n; ++k) {
      const double nx = jy[j] * jz[k] - jz[j] * jy[k];
      const double ny = jz[j] * jx[k] - jx[j] * jz[k];
      const double nz = jx[j] * jy[k] - jy[j] * jx[k];
      if (nx == 0.0 && ny == 0.0 && nz == 0.0) continue;
      double px = 0.0, py = 0.0, pz = 0.0;
      for (int i = 0; i < n; ++i) {
        if (i == j || i == k) continue;
        const double sg = (jx[i] * nx + jy[i] * ny + jz[i] * nz) >= 0.0 ? 1.0 : -1.0;
        px += sg * jx[i];
        py += sg * jy[i];
        pz += sg * jz[i];
      }
      for (int c = 0; c < 4; ++c) {
        const double fj = (c & 2) ? -1.0 : 1.0, fk = (c & 1) ? -1.0 : 1.0;
        const double cx = px + fj * jx[j] + fk * jx[k];
        const double cy = py + fj * jy[j] + fk * jy[k];
        const double cz = pz + fj * jz[j] + fk * jz[k];
        const double c2 = cx * cx + cy * cy + cz * cz;
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
    const double l = sqrt(jx[0] * jx[0] + jy[0] * jy[0] + jz[0] * jz[0]);
    ax = jx[0] / l;
    ay = jy[0] / l;
    az = jz[0] / l;
    return 1.0;
  }
  const double l = sqrt(best2), inv_l = 1.0 / l;
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
    ja[i] = sqrt(jx[i] * jx[i] + jy[i] * jy[i] + jz[i] * jz[i]);
    sum_abs += ja[i];
  }
  sum_absf = f32_from_f64(sum_abs);

  // ---- thrust
  double thrust = 1.0, ax = 0.0, ay = 0.0, az = 0.0;
  bool decided = false;
  if (n == 2) {
    // no emission: the pair is back to back, T = 1 along the quark
    const double l = sqrt(jx[0] * jx[0] + jy[0] * jy[0] + jz[0] * jz[0]);
    ax = jx[0] / l;
    ay = jy[0] / l;
    az = jz[0] / l;
    decided = true;
  } else if (n <= kMaskMax) {
    Top2 top;
    const unsigned long long full = n == 64 ? ~0ull : ((1ull << n) - 1ull);
    for (int j = 0; j < n; ++j) {
      for (int k = j + 1; k < n; ++k) {
        const float nx = fy[j] * fz[k] - fz[j] * fy[k];
        const float ny = fz[j] * fx[k] - fx[j] * fz[k];
        const float nz = fx[j] * fy[k] - fy[j] * fx[k];
        if (nx == 0.0f && ny == 0.0f && nz == 0.0f) continue;
        float px = 0.0f, py = 0.0f, pz = 0.0f;
        unsigned long long mask = 0ull;
        for (int i = 0; i < n; ++i) {
          if (i == j || i == k) continue;
          if (fx[i] * nx + fy[i] * ny + fz[i] * nz >= 0.0f) {
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
          top.add(cx * cx + cy * cy + cz * cz, m);
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
        px += sg * jx[i];
        py += sg * jy[i];
        pz += sg * jz[i];
      }
      const double l = sqrt(px * px + py * py + pz * pz), inv_l = 1.0 / l;
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
    const long long pn = __double_as_longlong(jx[i] * ax + jy[i] * ay + jz[i] * az);
    const bool plus = pn >= 0 || pn == static_cast<long long>(0x8000000000000000ull);
    double* h = plus ? hp : hm;
    h[0] += je[i];
    h[1] += jx[i];
    h[2] += jy[i];
    h[3] += jz[i];
    const double cx = jy[i] * az - jz[i] * ay, cy = jz[i] * ax - jx[i] * az, cz = jx[i] * ay - jy[i] * ax;
    const double pt = sqrt(cx * cx + cy * cy + cz * cz);
    if (plus) {
      bp += pt;
    } else {
      bm += pt;
    }
  }
  const double mp = hp[0] * hp[0] - hp[1] * hp[1] - hp[2] * hp[2] - hp[3] * hp[3];
  const double mm = hm[0] * hm[0] - hm[1] * hm[1] - hm[2] * hm[2] - hm[3] * hm[3];
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
    const float r = rsqrtf(fx[i] * fx[i] + fy[i] * fy[i] + fz[i] * fz[i]);
    fx[i] *= r;  // from here on fx, fy, fz hold unit directions
    fy[i] *= r;
    fz[i] *= r;
  }
  double yres[4] = {-1.0, -1.0, -1.0, -1.0};
  // y of jets i, j with the oracle's FP64 formula (|p| cached per jet).
  auto y_exact = [&](int i, int j) {
    const double cosij = (jx[i] * jx[j] + jy[i] * jy[j] + jz[i] * jz[j]) / (ja[i] * ja[j]);
    return 2.0 * fmin(je[i] * je[i], je[j] * je[j]) * (1.0 - cosij) * P.inv_s;
  };
  for (int m = n; m > 1; --m) {
    // pass 1: the smallest upper bound of the FP32 distances, and its pair
    float ubest = INFINITY;
    int ui = 0, uj = 1;
    for (int i = 0; i < m; ++i) {
      for (int j = i + 1; j < m; ++j) {
        const float dx = fx[i] - fx[j], dy = fy[i] - fy[j], dz = fz[i] - fz[j];
        const float d = dx * dx + dy * dy + dz * dz;
        const float y = fminf(fe2[i], fe2[j]) * d;
        const float rel = 4.0e-6f + 1.0e-6f * rsqrtf(fmaxf(d, 1e-30f));
        const float ub = y * (1.0f + rel) + 1e-30f;
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
        const float d = dx * dx + dy * dy + dz * dz;
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
          const float d = dx * dx + dy * dy + dz * dz;
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
    ja[bi] = sqrt(jx[bi] * jx[bi] + jy[bi] * jy[bi] + jz[bi] * jz[bi]);
    fe2[bj] = fe2[m - 1];
    fx[bj] = fx[m - 1];
    fy[bj] = fy[m - 1];
    fz[bj] = fz[m - 1];
    {
      const float e = f32_from_f64(je[bi]);
      fe2[bi] = e * e;
      const float x = f32_from_f64(jx[bi]), y = f32_from_f64(jy[bi]), z = f32_from_f64(jz[bi]);
      const float r = rsqrtf(x * x + y * y + z * z);
      fx[bi] = x * r;
      fy[bi] = y * r;
      fz[bi] = z * r;
    }
  }
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
__global__ void __launch_bounds__(256) k_bucket_count(Events E, int* counts) {
  __shared__ int sh[256];
  sh[threadIdx.x] = 0;
  __syncthreads();
  for (int64_t ev = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; ev < E.n;
       ev += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int n = shape_partons(E, ev);
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
__global__ void __launch_bounds__(256) k_bucket_scatter(Events E, int* cursor, int* order) {
  __shared__ int s_cnt[256];
  __shared__ int s_base[256];
  const int tid = threadIdx.x, lane = tid & 31;
  for (int64_t first = static_cast<int64_t>(blockIdx.x) * 256; first < E.n;
       first += static_cast<int64_t>(gridDim.x) * 256) {
    s_cnt[tid] = 0;
    __syncthreads();
    const int64_t ev = first + tid;
    int n = -1;
    if (ev < E.n) {
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

// Events of buckets n_lo..n_hi (all with n <= MAXJ).
template <int MAXJ>
__global__ void __launch_bounds__(kShapeThreads) k_event_shapes(DevParams P, Events E, const int* order,
                                                                const int* offsets, int n_lo, int n_hi) {
  const int begin = offsets[n_lo], end = offsets[n_hi + 1 > 256 ? 256 : n_hi + 1];
  for (int k = begin + blockIdx.x * blockDim.x + threadIdx.x; k < end; k += gridDim.x * blockDim.x) {
    const int64_t ev = order[k];
    event_shapes<MAXJ>(P, E, ev, E.n_partons[ev]);
  }
}

}  // namespace

cudaError_t preload_observables() {
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, k_bucket_count);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_bucket_scan);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_bucket_scatter);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_event_shapes<16>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_event_shapes<32>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_event_shapes<64>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_event_shapes<128>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_event_shapes<256>);
  return e;
}

cudaError_t launch_observables(const DevParams& P, const Events& E, int* buckets, int* order, cudaStream_t s) {
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
  k_bucket_count<<<grid_count, 256, 0, s>>>(E, counts);
  k_bucket_scan<<<1, 256, 0, s>>>(counts, offsets, cursor);
  k_bucket_scatter<<<grid_count, 256, 0, s>>>(E, cursor, order);
  // One launch per multiplicity class; grids cover the largest possible
  // class and stride over the actual one.
  const int64_t all = (E.n + kShapeThreads - 1) / kShapeThreads;
  const unsigned big = static_cast<unsigned>(all < 16 * sms ? all : 16 * sms);
  const unsigned small = static_cast<unsigned>(all < 2 * sms ? all : 2 * sms);
  k_event_shapes<16><<<big, kShapeThreads, 0, s>>>(P, E, order, offsets, 0, 16);
  if (E.cap > 16) k_event_shapes<32><<<small, kShapeThreads, 0, s>>>(P, E, order, offsets, 17, 32);
  if (E.cap > 32) k_event_shapes<64><<<small, kShapeThreads, 0, s>>>(P, E, order, offsets, 33, 64);
  if (E.cap > 64) k_event_shapes<128><<<small, kShapeThreads, 0, s>>>(P, E, order, offsets, 65, 128);
  if (E.cap > 128) k_event_shapes<256><<<small, kShapeThreads, 0, s>>>(P, E, order, offsets, 129, 255);
  return cudaGetLastError();
}

}  // namespace gaps
