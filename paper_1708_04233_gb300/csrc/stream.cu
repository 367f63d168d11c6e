// Sub-hologram streaming (Sec. 1, large-scale calculation, steps 2-4): a
// hologram computed band by band -- each band a sub-hologram of band_h rows
// at its own origin -- with the band's outputs copied to host memory while
// the next band is computed, so the device holds two bands at a time and the
// hologram's size is bounded by host memory, not device memory.
//
// Two band slots (output buffers + binning scratch) alternate between two
// streams: band k runs on stream k % 2 (fused superposition + inverse +
// binarisation, then its device-to-host copies), so the copies of band k
// overlap the computation of band k + 1, and a slot is reused only after its
// previous copies completed (stream order).
#include <algorithm>
#include <cstring>

#include "lut_object.h"

using namespace wsb;

namespace {

struct Slot {
  void* scratch = nullptr;
  size_t scratch_bytes = 0;
  uint8_t* bits = nullptr;
  float2* u = nullptr;
};

}  // namespace

extern "C" {

wasabi_status wasabi_hologram_stream(const wasabi_lut* lut, const wasabi_point* points_dev, int64_t n, int holo_w,
                                     int holo_h, int band_h, int rule, const wasabi_frame* frame,
                                     uint8_t* bits_host, void* u_host, void* stream) {
  if (!lut || n < 0 || (n > 0 && !points_dev) || (!bits_host && !u_host)) {
    set_error("hologram_stream: need the LUT, the points (if n > 0) and a host output");
    return WASABI_E_INVALID;
  }
  const int ts = 1 << lut->L;
  if (lut->L < 2 || band_h < ts || band_h % ts || holo_w < ts || holo_h < ts || holo_w % ts || holo_h % ts ||
      (bits_host && holo_w % 8) || holo_w > (1 << 29) || holo_h > (1 << 29)) {
    set_error("hologram_stream: sizes must be multiples of 2^L = %d (levels >= 2; holo_w %% 8 == 0 for bits)", ts);
    return WASABI_E_INVALID;
  }
  int ox, oy;
  RefDev ref;
  const char* why = "";
  if (!frame_to_dev(frame, &ox, &oy, &ref, &why)) { set_error("hologram_stream: %s", why); return WASABI_E_INVALID; }
  if ((long long)oy + holo_h > 0x7fffffffll) { set_error("hologram_stream: bands leave the int32 plane"); return WASABI_E_INVALID; }
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != lut->device) { set_error("hologram_stream: LUT lives on another device"); return WASABI_E_INVALID; }
  const int bh = std::min(band_h, holo_h);
  const int nbands = (holo_h + bh - 1) / bh;
  size_t scratch = 0;
  wasabi_status st = wasabi_scratch_bytes(lut, n, holo_w, bh, &scratch);
  if (st != WASABI_OK) return st;
  const size_t band_bits = (size_t)holo_w * bh / 8, band_u = (size_t)holo_w * bh * sizeof(float2);

  Slot slot[2];
  cudaStream_t ss[2] = {nullptr, nullptr};
  cudaEvent_t start = nullptr;
  cudaError_t e = cudaEventCreateWithFlags(&start, cudaEventDisableTiming);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
    e = cudaStreamCreateWithFlags(&ss[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&slot[i].scratch, scratch);
    slot[i].scratch_bytes = scratch;
    if (e == cudaSuccess && bits_host) e = cudaMalloc(reinterpret_cast<void**>(&slot[i].bits), band_bits);
    if (e == cudaSuccess && u_host) e = cudaMalloc(reinterpret_cast<void**>(&slot[i].u), band_u);
  }
  // Both streams start after the work already queued on the caller's stream.
  if (e == cudaSuccess) e = cudaEventRecord(start, (cudaStream_t)stream);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(ss[i], start, 0);
  if (e != cudaSuccess) st = cuda_fail("hologram_stream: setup", e);

  int cell, threads;
  superpose_config(lut, holo_w, bh, superpose_config_kind(false, u_host, bits_host, frame), &cell, &threads);
  for (int k = 0; k < nbands && st == WASABI_OK; ++k) {
    Slot& sl = slot[k & 1];
    const cudaStream_t s = ss[k & 1];
    const int y0 = k * bh, hk = std::min(bh, holo_h - y0);
    wasabi_frame fk;
    std::memset(&fk, 0, sizeof fk);
    if (frame) fk = *frame;
    fk.origin_y = oy + y0;  // the band is the sub-hologram at (origin_x, origin_y + y0)
    st = superpose_impl(lut, points_dev, n, holo_w, hk, rule, nullptr, sl.u, sl.bits, sl.scratch, sl.scratch_bytes,
                        s, cell, threads, &fk);
    if (st != WASABI_OK) break;
    if (bits_host)
      e = cudaMemcpyAsync(bits_host + (size_t)y0 * holo_w / 8, sl.bits, (size_t)hk * holo_w / 8,
                          cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && u_host)
      e = cudaMemcpyAsync(static_cast<float2*>(u_host) + (size_t)y0 * holo_w, sl.u,
                          (size_t)hk * holo_w * sizeof(float2), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) st = cuda_fail("hologram_stream: copy", e);
  }
  // Wait for both streams (also on failure: nothing may still use the
  // buffers when they are freed), then release everything.
  for (int i = 0; i < 2; ++i) {
    if (!ss[i]) continue;
    const cudaError_t e2 = cudaStreamSynchronize(ss[i]);
    if (e2 != cudaSuccess && st == WASABI_OK) st = cuda_fail("hologram_stream: run", e2);
    cudaFree(slot[i].scratch);
    cudaFree(slot[i].bits);
    cudaFree(slot[i].u);
    cudaStreamDestroy(ss[i]);
  }
  if (start) cudaEventDestroy(start);
  return st;
}

}  // extern "C"
