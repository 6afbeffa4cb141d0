// Allocation-free entry point: velo_reconstruct_static.
//
// Some callers cannot allocate device memory at the moment they reconstruct:
// a trigger node whose device-memory budget is fixed when the process starts
// and must not move while data flows, or code that runs inside another
// framework's callbacks, where a cudaMalloc could block on the device or
// re-enter that framework's own allocator.  For them this entry point takes
// its scratch from a file-scope __device__ array compiled into the library
// (VELO_STATIC_SCRATCH_BYTES, 64 MiB), so it calls no cudaMalloc, cudaFree or
// allocating library routine.  The caller still passes inputs and outputs.
// The paper has no counterpart of this entry point.
//
// The array exists once on every device that loads the library and stays
// allocated until the process exits.  In host code its name is only a
// host-side stand-in, so its device address is looked up with
// cudaGetSymbolAddress, once per device, with that device current, during
// the first call made on that device (make that first call before any
// stream capture).  Every call shares the array, and the array keeps what the
// previous call left in it; the kernels initialise every scratch word before
// they read it, so nothing has to be cleared between calls.  Calls whose work
// overlaps on the GPU (two streams, or two host threads) race on the array:
// serialise them.
#include <cuda_runtime.h>

#include <mutex>

#include "velo_internal.cuh"

namespace {

static __device__ __align__(256) unsigned char g_static_scratch[VELO_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_static_scratch on the current device; the lookup runs
// once per device.  Returns VELO_OK or an error code.
int static_scratch(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return VELO_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return VELO_EINVAL;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return VELO_ECUDA;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return VELO_OK;
}

}  // namespace

extern "C" int velo_reconstruct_static(const velo_events_t* events, const velo_geometry_t* geometry,
                                       const velo_params_t* params, const velo_output_t* out, void* stream) {
  if (!events) return VELO_EINVAL;
  if (events->n_events >= (1ull << 31) || events->n_pixels >= (1ull << 40)) return VELO_EINVAL;
  if (velo::workspace_bytes(events->n_events, events->n_pixels) > VELO_STATIC_SCRATCH_BYTES) return VELO_ECAPACITY;
  void* scratch = nullptr;
  const int rc = static_scratch(&scratch);
  if (rc != VELO_OK) return rc;
  return velo_reconstruct_into(events, geometry, params, out, scratch, VELO_STATIC_SCRATCH_BYTES, stream);
}
