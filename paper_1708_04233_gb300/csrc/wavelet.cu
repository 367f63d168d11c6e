// The order-1 coiflet (Sec. 1 uses coiflets at level 3; the order is not
// stated): its filters, and the inverse transformation (Sec. 1, step 3) of a
// hologram superposed from a coiflet LUT.
//
// The coiflet transform is periodic over the whole hologram and its filters
// overlap 2^L x 2^L tiles, so the inverse is not tile-local as Haar's is: the
// tile-major buffer is permuted into the Mallat layout, then each level runs
// two separable synthesis passes over the level's low-pass region (along y
// into a second buffer, then along x back), and a last pass writes the field
// and/or the binary hologram against the frame's reference wave.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "dbf.cuh"
#include "lut_object.h"

namespace wsb {

// h_k, k = -2 .. 3, solves sum h = sqrt 2, sum_k h_k h_{k+2m} = delta_m
// (m = 0, 1, 2), sum (-1)^k k h_k = 0 and sum k h_k = 0; of the two real
// solutions, the one with the largest tap at k = 0:
//   h / sqrt 2 = ((1 - r)/32, (5 + r)/32, (7 + r)/16, (7 - r)/16,
//                (1 - r)/32, (r - 3)/32),  r = sqrt 7.
// g_k = (-1)^k h_{1-k}.
void coif1_filters(double lo[6], double hi[6]) {
  const double r = std::sqrt(7.0), s2 = std::sqrt(2.0);
  lo[0] = s2 * (1.0 - r) / 32.0;
  lo[1] = s2 * (5.0 + r) / 32.0;
  lo[2] = s2 * (7.0 + r) / 16.0;
  lo[3] = s2 * (7.0 - r) / 16.0;
  lo[4] = s2 * (1.0 - r) / 32.0;
  lo[5] = s2 * (r - 3.0) / 32.0;
  for (int k = -2; k <= 3; ++k) hi[k + 2] = ((k & 1) ? -1.0 : 1.0) * lo[(1 - k) + 2];
}

namespace {

struct CoifTaps {
  float lo[6], hi[6];
};

// One synthesis output: sample j of a line of S samples receives
// h_k s[m] + g_k d[m] for every k = j - 2m (mod S), k = -2 .. 3; s and d are
// the line's low and high halves (S / 2 each), `step` apart in memory.
// The taps with k = j - 2m of j's parity pair with m = j/2 + 1, j/2, j/2 - 1
// (k = -2, 0, 2 for even j; -1, 1, 3 for odd j), taken in that order, each
// m wrapped once (h = 1: every m is 0).
__device__ __forceinline__ float2 coif_synth(const CoifTaps& t, const float2* line, long long step, int S, int j) {
  const int h = S / 2, m0 = j >> 1, par = j & 1;
  int mp = m0 + 1, mm = m0 - 1;
  if (mp >= h) mp -= h;
  if (mm < 0) mm += h;
  const int ms[3] = {mp, m0, mm};
  float2 acc = make_float2(0.f, 0.f);
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const int i = 2 * q + par;  // tap slot of k = 2q - 2 + par
    const float2 sv = line[(long long)ms[q] * step], dv = line[(long long)(h + ms[q]) * step];
    acc.x = __fmaf_rn(t.lo[i], sv.x, acc.x);
    acc.y = __fmaf_rn(t.lo[i], sv.y, acc.y);
    acc.x = __fmaf_rn(t.hi[i], dv.x, acc.x);
    acc.y = __fmaf_rn(t.hi[i], dv.y, acc.y);
  }
  return acc;
}

// Along y over the Sx x Sy low-pass region: a -> b (consecutive threads take
// consecutive columns).
__global__ void coif_syn_cols_kernel(const float2* __restrict__ a, float2* __restrict__ b, int w, int Sx, int Sy,
                                     CoifTaps t) {
  const long long n = (long long)Sx * Sy;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(i / Sx), col = (int)(i - (long long)j * Sx);
    b[(long long)j * w + col] = coif_synth(t, a + col, w, Sy, j);
  }
}

// Along x over the region: b -> a.
__global__ void coif_syn_rows_kernel(const float2* __restrict__ b, float2* __restrict__ a, int w, int Sx, int Sy,
                                     CoifTaps t) {
  const long long n = (long long)Sx * Sy;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i / Sx), j = (int)(i - (long long)r * Sx);
    a[(long long)r * w + j] = coif_synth(t, b + (long long)r * w, 1, Sx, j);
  }
}

// Re(u conj R) for the frame's reference (R = 1 for the plane wave), phase
// in double-float per pixel.
__device__ __forceinline__ float ref_re(const RefDbf& ref, float2 u, long long X, long long Y) {
  if (ref.kind == 0) return u.x;
  float sn, cs;
  sincospif(2.0f * ref_frac(ref, (float)X, (float)Y), &sn, &cs);
  return fmaf(u.x, cs, ref.sgn * u.y * sn);
}

// Field and/or bits (eight pixels of a row per thread when bits are wanted).
__global__ void coif_out_kernel(const float2* __restrict__ a, int w, int h, float2* __restrict__ u,
                                uint8_t* __restrict__ bits, int ox, int oy, RefDbf ref) {
  const int per = bits ? 8 : 1;
  const long long n = (long long)w * h / per;
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (long long)gridDim.x * blockDim.x) {
    const long long i0 = g * per;
    const long long y = i0 / w, x0 = i0 - y * w;
    unsigned byte = 0;
    for (int q = 0; q < per; ++q) {
      const float2 v = a[i0 + q];
      if (u) u[i0 + q] = v;
      if (bits && ref_re(ref, v, ox + x0 + q, oy + y) > 0.f) byte |= 1u << q;
    }
    if (bits) bits[g] = (uint8_t)byte;
  }
}

unsigned grid_for(long long n) { return (unsigned)std::max<long long>(1, std::min<long long>((n + 255) / 256, 8192)); }

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

cudaError_t launch_coif_inverse(const float2* wbuf, int w, int h, int L, float2* a, float2* b, cudaStream_t s,
                                float2* out) {
  double lo[6], hi[6];
  coif1_filters(lo, hi);
  CoifTaps t;
  for (int i = 0; i < 6; ++i) { t.lo[i] = (float)lo[i]; t.hi[i] = (float)hi[i]; }
  cudaError_t e = launch_wbuf_to_mallat(wbuf, w, h, L, a, s);
  for (int l = L; l >= 1 && e == cudaSuccess; --l) {
    const int Sx = w >> (l - 1), Sy = h >> (l - 1);
    const long long n = (long long)Sx * Sy;
    coif_syn_cols_kernel<<<grid_for(n), 256, 0, s>>>(a, b, w, Sx, Sy, t);
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    // The last level writes the field straight into `out` when given.
    coif_syn_rows_kernel<<<grid_for(n), 256, 0, s>>>(b, (l == 1 && out) ? out : a, w, Sx, Sy, t);
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace wsb

using namespace wsb;

extern "C" {

wasabi_status wasabi_inverse_wavelet_scratch_bytes(int holo_w, int holo_h, size_t* bytes_out) {
  if (holo_w <= 0 || holo_h <= 0 || !bytes_out) { set_error("inverse_wavelet_scratch_bytes: bad arguments"); return WASABI_E_INVALID; }
  *bytes_out = 2 * align256((size_t)holo_w * holo_h * sizeof(float2));
  return WASABI_OK;
}

wasabi_status wasabi_inverse_wavelet(const void* wbuf_dev, int holo_w, int holo_h, int levels, int wavelet,
                                     const wasabi_frame* frame, void* u_dev, uint8_t* bits_dev, void* scratch_dev,
                                     size_t scratch_bytes, void* stream) {
  if (wavelet == WASABI_HAAR)
    return wasabi_inverse_haar_frame(wbuf_dev, holo_w, holo_h, levels, frame, u_dev, bits_dev, stream);
  if (wavelet != WASABI_COIF1) { set_error("inverse_wavelet: unknown wavelet %d", wavelet); return WASABI_E_INVALID; }
  if (!wbuf_dev || (!u_dev && !bits_dev) || !scratch_dev) {
    set_error("inverse_wavelet: need the buffer, an output and scratch");
    return WASABI_E_INVALID;
  }
  if (levels < 1 || levels > kMaxLevels) { set_error("inverse_wavelet: levels must be in [1, %d]", kMaxLevels); return WASABI_E_INVALID; }
  const int ts = 1 << levels;
  if (holo_w != holo_h || holo_w < ts || holo_w % ts || (bits_dev && holo_w % 8)) {
    set_error("inverse_wavelet: the coiflet inverse needs a square hologram, side a multiple of 2^levels "
              "(and of 8 for bits)");
    return WASABI_E_INVALID;
  }
  if (((uintptr_t)wbuf_dev & 15) || ((uintptr_t)u_dev & 15) || ((uintptr_t)scratch_dev & 255)) {
    set_error("inverse_wavelet: misaligned buffer");
    return WASABI_E_INVALID;
  }
  int ox, oy;
  RefDev ref;
  const char* why = "";
  if (!frame_to_dev(frame, &ox, &oy, &ref, &why)) { set_error("inverse_wavelet: %s", why); return WASABI_E_INVALID; }
  // Plane pixel coordinates are exact in FP32 below 2^24.
  if (std::abs((long long)ox) + holo_w >= (1LL << 24) || std::abs((long long)oy) + holo_h >= (1LL << 24)) {
    set_error("inverse_wavelet: plane pixels must stay below 2^24 in magnitude");
    return WASABI_E_INVALID;
  }
  size_t need = 0;
  wasabi_inverse_wavelet_scratch_bytes(holo_w, holo_h, &need);
  if (scratch_bytes < need) {
    set_error("inverse_wavelet: scratch too small (%zu < %zu bytes)", scratch_bytes, need);
    return WASABI_E_NOMEM;
  }
  const cudaStream_t s = (cudaStream_t)stream;
  float2* a = static_cast<float2*>(scratch_dev);
  float2* b = reinterpret_cast<float2*>(static_cast<char*>(scratch_dev) + need / 2);
  float2* u = static_cast<float2*>(u_dev);
  cudaError_t e = launch_coif_inverse(static_cast<const float2*>(wbuf_dev), holo_w, holo_h, levels, a, b, s, u);
  if (e == cudaSuccess && bits_dev) {  // the field is in u when it was asked for, else in a
    const long long groups = (long long)holo_w * holo_h / 8;
    coif_out_kernel<<<grid_for(groups), 256, 0, s>>>(u ? u : a, holo_w, holo_h, nullptr, bits_dev, ox, oy,
                                                     ref_dbf(ref));
    e = cudaGetLastError();
  }
  return e == cudaSuccess ? WASABI_OK : cuda_fail("inverse_wavelet", e);
}

}  // extern "C"
