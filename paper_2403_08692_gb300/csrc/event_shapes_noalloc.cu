// gaps_event_shapes_noalloc: the observables stage for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc or any allocating routine: code
// running inside another framework's memory pool that must not be bypassed,
// a plug-in whose host forbids allocation calls, or a process that has
// handed out all device memory ahead of time.  They own the event arrays and
// the output, but have nowhere to put the observables' working arrays
// (multiplicity buckets, event order, debug counters).  This entry point
// keeps those in one file-scope device array of fixed size instead, so it
// allocates nothing.
//
// The array belongs to this file's module of the library image.  CUDA loads
// a module on a device when it is first used there (lazily, by default), and
// reserves the array's device memory (about 4.2 MB) then, until the process
// exits.  The first call on a device is that use: it looks up the array's
// address and loads the observables' kernels, so a call with n_events = 0
// does exactly this set-up and nothing else.  All calls share the array and
// it keeps the last call's contents; the parts that must start at zero are
// cleared by every call on its stream.  Two calls whose work overlaps on the
// GPU (different streams, or different host threads without ordering) race
// on it and give wrong results: serialise them.
#include <mutex>

#include "gaps_launch.hpp"

namespace gaps {

namespace {

// Working arrays of one call: debug counters, the multiplicity buckets
// (counts, offsets, cursors) and the event order.
struct NoAllocScratch {
  unsigned long long counters[16];
  int buckets[769];
  int pad[63];
  int order[GAPS_NOALLOC_MAX_EVENTS];
};

static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
NoAllocScratch* g_scratch_on_device[kMaxDevices] = {};

// Set-up on the current device, once: the device address of the static
// array (in host code `g_noalloc_scratch` only names a host-side stand-in, so
// the address is looked up with the device current, which also loads the
// module that holds the array) and the observables' kernels.  The address is
// cached per device ordinal; it belongs to the device's primary context, so
// it is not valid after a cudaDeviceReset of that device.
cudaError_t scratch_address(NoAllocScratch** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_on_device[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    e = preload_observables();
    if (e != cudaSuccess) return e;
    g_scratch_on_device[dev] = static_cast<NoAllocScratch*>(p);
  }
  *out = g_scratch_on_device[dev];
  return cudaSuccess;
}

}  // namespace

}  // namespace gaps

using namespace gaps;

extern "C" int gaps_event_shapes_noalloc(const double* px, const double* py, const double* pz, const double* e,
                                         const int32_t* n_partons, const int32_t* status, int64_t n_events,
                                         int32_t capacity, double sqrt_s, double* obs, void* stream) {
  if (n_events < 0 || n_events > GAPS_NOALLOC_MAX_EVENTS) return GAPS_ERR_INVALID;
  if (capacity < 4 || capacity > 255 || !(sqrt_s > 0.0)) return GAPS_ERR_INVALID;
  if (n_events > 0 && (!px || !py || !pz || !e || !n_partons || !status || !obs)) return GAPS_ERR_INVALID;
  NoAllocScratch* scratch = nullptr;
  cudaError_t err = scratch_address(&scratch);
  if (err != cudaSuccess) return record_cuda_error(err);
  if (n_events == 0) return GAPS_OK;
  Events E{};
  E.px = const_cast<double*>(px);
  E.py = const_cast<double*>(py);
  E.pz = const_cast<double*>(pz);
  E.e = const_cast<double*>(e);
  E.n_partons = const_cast<int32_t*>(n_partons);
  E.status = const_cast<int32_t*>(status);
  E.obs = obs;
  E.counters = scratch->counters;
  E.n = n_events;
  E.stride = n_events;
  E.base = 0;
  E.cap = capacity;
  set_layout(E, GAPS_LAYOUT_SOA, n_events, capacity);
  DevParams P{};
  P.sqrt_s = sqrt_s;
  P.s = sqrt_s * sqrt_s;
  P.inv_s = 1.0 / P.s;
  err = launch_observables(P, E, scratch->buckets, scratch->order, static_cast<cudaStream_t>(stream));
  return err == cudaSuccess ? GAPS_OK : record_cuda_error(err);
}
