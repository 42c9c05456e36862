// Measurement and test library (libgaps_probe.so, include/gaps_probe.h),
// kept out of the product library libgaps.so.
//
// FP64 throughput probe: how many DFMA, log, exp, division, square root,
// sincospi and table-driven log (log_fp64) results per second this GPU
// delivers, with every SM busy.  The benchmark uses it to express the
// shower's required FP64 work in DFMA-equivalents measured on the same device
// in the same run.  Also the shower's log_fp64 and its double -> float
// conversion, host and device builds of the same source, for the accuracy
// tests.
#include <cstdio>

#include <cuda_runtime.h>

#include "gaps.h"
#include "gaps_probe.h"
#include "log_fp64.cuh"
#include "sqrt_obs.cuh"

namespace gaps {

namespace {

thread_local char g_probe_error[256] = "";

int record_cuda_error(cudaError_t e) {
  std::snprintf(g_probe_error, sizeof(g_probe_error), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
  return GAPS_ERR_CUDA;
}

constexpr int kProbeThreads = 256;
constexpr int kChains = 4;
constexpr int kProbeOps = 7;

// One of seven operations, iterated on independent chains; the result is
// stored only under a condition no input meets, so nothing is written and
// nothing can be optimised away.
template <int OP>
__global__ void __launch_bounds__(kProbeThreads) k_probe(double* sink, int iters, double seed) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  double x[kChains], acc[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) {
    x[c] = 1.25 + 1e-9 * tid + 0.125 * c;
    acc[c] = seed;
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      if (OP == 0) {
        acc[c] = fma(acc[c], 0.999999999, x[c]);
        x[c] = fma(x[c], 1.000000001, -1e-12);
      } else if (OP == 1) {
        acc[c] += log(x[c]);
        x[c] += 0.25;
      } else if (OP == 2) {
        acc[c] += exp(-x[c]);
        x[c] += 0.25;
      } else if (OP == 3) {
        acc[c] += 1.0 / x[c];
        x[c] += 0.25;
      } else if (OP == 4) {
        acc[c] += sqrt(x[c]);
        x[c] += 0.25;
      } else if (OP == 5) {
        double s, co;
        sincospi(x[c], &s, &co);
        acc[c] += s + co;
        x[c] += 0.25;
      } else {
        acc[c] += log_fp64(x[c]);
        x[c] += 0.25;
      }
    }
  }
  double total = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) total += acc[c];
  if (total == -1.0e300) sink[0] = total;
}

template <int OP>
cudaError_t time_op(double* sink, int blocks, int iters, cudaStream_t s, float* ms) {
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  if (e == cudaSuccess) k_probe<OP><<<blocks, kProbeThreads, 0, s>>>(sink, iters / 8, 0.5);  // warm up
  if (e == cudaSuccess) e = cudaEventRecord(a, s);
  if (e == cudaSuccess) k_probe<OP><<<blocks, kProbeThreads, 0, s>>>(sink, iters, 0.5);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventRecord(b, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  return e;
}

}  // namespace

}  // namespace gaps

using namespace gaps;

extern "C" int gaps_probe_fp64_rates(double* device_sink, double* host_rates, void* stream) {
  if (!device_sink || !host_rates) return GAPS_ERR_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return record_cuda_error(e);
  const int blocks = sms * 8;
  const double threads = static_cast<double>(blocks) * kProbeThreads;
  // iterations per thread, sized for a few milliseconds per operation
  const int iters[kProbeOps] = {2048, 256, 256, 512, 512, 256, 512};
  // results per iteration and chain: the FMA loop issues two DFMA
  const double per_iter[kProbeOps] = {2.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0};
  float ms[kProbeOps] = {0, 0, 0, 0, 0, 0, 0};
  e = time_op<0>(device_sink, blocks, iters[0], s, &ms[0]);
  if (e == cudaSuccess) e = time_op<1>(device_sink, blocks, iters[1], s, &ms[1]);
  if (e == cudaSuccess) e = time_op<2>(device_sink, blocks, iters[2], s, &ms[2]);
  if (e == cudaSuccess) e = time_op<3>(device_sink, blocks, iters[3], s, &ms[3]);
  if (e == cudaSuccess) e = time_op<4>(device_sink, blocks, iters[4], s, &ms[4]);
  if (e == cudaSuccess) e = time_op<5>(device_sink, blocks, iters[5], s, &ms[5]);
  if (e == cudaSuccess) e = time_op<6>(device_sink, blocks, iters[6], s, &ms[6]);
  if (e != cudaSuccess) return record_cuda_error(e);
  for (int i = 0; i < kProbeOps; ++i)
    host_rates[i] = ms[i] > 0.0f ? threads * kChains * iters[i] * per_iter[i] / (ms[i] * 1e-3) : 0.0;
  return GAPS_OK;
}

namespace gaps {
namespace {

__global__ void __launch_bounds__(256) k_log_fp64(const double* x, double* y, int64_t n) {
  const int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k < n) y[k] = log_fp64(x[k]);
}

__global__ void __launch_bounds__(256) k_sqrt_obs(const double* x, double* y, int64_t n) {
  const int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k < n) y[k] = sqrt_obs(x[k]);
}

}  // namespace
}  // namespace gaps

extern "C" int gaps_log_fp64_host(const double* x, double* y, int64_t n) {
  if (n < 0 || (n > 0 && (!x || !y))) return GAPS_ERR_INVALID;
  for (int64_t k = 0; k < n; ++k) y[k] = log_fp64(x[k]);
  return GAPS_OK;
}

extern "C" int gaps_f32_from_f64_host(const double* x, float* y, int64_t n) {
  if (n < 0 || (n > 0 && (!x || !y))) return GAPS_ERR_INVALID;
  for (int64_t k = 0; k < n; ++k) y[k] = f32_from_f64(x[k]);
  return GAPS_OK;
}

extern "C" int gaps_log_fp64_device(const double* x, double* y, int64_t n, void* stream) {
  if (n < 0 || (n > 0 && (!x || !y))) return GAPS_ERR_INVALID;
  if (n == 0) return GAPS_OK;
  k_log_fp64<<<static_cast<unsigned>((n + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(x, y, n);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GAPS_OK : record_cuda_error(e);
}

extern "C" const char* gaps_probe_last_cuda_error(void) { return g_probe_error; }

extern "C" int gaps_sqrt_obs_device(const double* x, double* y, int64_t n, void* stream) {
  if (n < 0 || (n > 0 && (!x || !y))) return GAPS_ERR_INVALID;
  if (n == 0) return GAPS_OK;
  k_sqrt_obs<<<static_cast<unsigned>((n + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(x, y, n);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GAPS_OK : record_cuda_error(e);
}
