// wasabi_superpose_static: superposition for callers that cannot allocate
// device memory.  The binning scratch that wasabi_superpose takes from its
// caller lives here instead, in one file-scope device array of fixed size
// (WASABI_STATIC_SCRATCH_BYTES) that every device loading the library holds
// until the process exits.
#include <mutex>

#include "internal.cuh"

static __device__ __align__(256) unsigned char g_static_scratch[WASABI_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDev = 64;
std::mutex g_static_mu;
void* g_static_ptr[kMaxDev] = {nullptr};

// Device address of the array on the current device.  In host code the
// symbol itself is only a host-side stand-in, so the address is looked up
// once per device, with that device current, and cached.
wasabi_status static_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    wsb::set_error("superpose_static: cudaGetDevice: %s", cudaGetErrorString(e));
    return WASABI_E_CUDA;
  }
  if (dev < 0 || dev >= kMaxDev) {
    wsb::set_error("superpose_static: device ordinal %d out of range", dev);
    return WASABI_E_INVALID;
  }
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) {
      wsb::set_error("superpose_static: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
      return WASABI_E_CUDA;
    }
    g_static_ptr[dev] = p;
  }
  *out = g_static_ptr[dev];
  return WASABI_OK;
}

}  // namespace

extern "C" wasabi_status wasabi_superpose_static(const wasabi_lut* lut, const wasabi_point* points_dev,
                                                 int64_t n, int holo_w, int holo_h, int rule,
                                                 void* wbuf_dev, void* stream) {
  size_t need = 0;
  wasabi_status st = wasabi_scratch_bytes(lut, n, holo_w, holo_h, &need);
  if (st != WASABI_OK) return st;
  if (need > (size_t)WASABI_STATIC_SCRATCH_BYTES) {
    wsb::set_error("superpose_static: this problem needs %zu bytes of scratch, more than the %d-byte "
                   "static array; call wasabi_superpose with caller-owned scratch instead",
                   need, WASABI_STATIC_SCRATCH_BYTES);
    return WASABI_E_NOMEM;
  }
  void* scratch = nullptr;
  st = static_scratch(&scratch);
  if (st != WASABI_OK) return st;
  return wasabi_superpose(lut, points_dev, n, holo_w, holo_h, rule, wbuf_dev, scratch,
                          (size_t)WASABI_STATIC_SCRATCH_BYTES, stream);
}
