// Numerical reconstruction of a hologram by the angular spectrum method: the
// field in a plane at signed distance d is IFFT2(FFT2(U_0) H) with the
// transfer function H = exp(i 2 pi d sqrt(1/lambda^2 - fx^2 - fy^2)) of free
// space (evanescent frequencies dropped).  Three element-wise kernels around
// two cuFFT C2C transforms: the input (a complex field, or a binary
// hologram's transmittance times the reference wave), the transfer function
// (phase reduced in FP64, then FP32 sine and cosine), the outputs.
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "lut_object.h"

using namespace wsb;

namespace {

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// U_0 = field, or t R with t the hologram's bit (reference R of the frame).
__global__ void recon_input_kernel(const float2* __restrict__ field, const uint8_t* __restrict__ bits, int w,
                                   long long n, int ox, int oy, RefDev ref, float2* __restrict__ buf) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    if (field) {
      buf[i] = field[i];
      continue;
    }
    const float t = (float)((bits[i >> 3] >> (i & 7)) & 1);
    float2 r = make_float2(1.f, 0.f);
    if (ref.kind != 0) {
      const long long y = i / w, x = i - y * w;
      const double ex = (double)(ox + x) - ref.x, ey = (double)(oy + y) - ref.y;
      const double tr = sqrt(fma(ref.a2, fma(ex, ex, ey * ey), ref.c));
      float sn, cs;
      sincospif(2.0f * (float)(tr - floor(tr)), &sn, &cs);
      r = make_float2(cs, ref.sgn * sn);
    }
    buf[i] = make_float2(t * r.x, t * r.y);
  }
}

// Spectrum times H / (w h) (the inverse transform is unnormalised).
__global__ void recon_transfer_kernel(float2* __restrict__ buf, int w, int h, double lambda, double pitch, double d) {
  const long long n = (long long)w * h;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const float norm = (float)(1.0 / (double)n);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int ky = (int)(i / w), kx = (int)(i - (long long)ky * w);
    const int sx = kx <= (w - 1) / 2 ? kx : kx - w;  // FFT frequency order
    const int sy = ky <= (h - 1) / 2 ? ky : ky - h;
    const double ax = lambda * sx / (w * pitch), ay = lambda * sy / (h * pitch);  // lambda fx, lambda fy
    const double s = 1.0 - ax * ax - ay * ay;
    float2 v = make_float2(0.f, 0.f);
    if (s > 0.0) {
      const double ph = d / lambda * sqrt(s);  // cycles
      float sn, cs;
      sincospif(2.0f * (float)(ph - floor(ph)), &sn, &cs);
      const float2 u = buf[i];
      v = make_float2((u.x * cs - u.y * sn) * norm, (u.x * sn + u.y * cs) * norm);
    }
    buf[i] = v;
  }
}

__global__ void recon_output_kernel(const float2* __restrict__ buf, long long n, float2* __restrict__ field,
                                    float* __restrict__ inten) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const float2 u = buf[i];
    if (field) field[i] = u;
    if (inten) inten[i] = u.x * u.x + u.y * u.y;
  }
}

bool make_plan(int w, int h, cufftHandle* plan, size_t* work) {
  if (cufftCreate(plan) != CUFFT_SUCCESS) return false;
  long long dims[2] = {h, w};
  if (cufftSetAutoAllocation(*plan, 0) != CUFFT_SUCCESS ||
      cufftMakePlanMany64(*plan, 2, dims, nullptr, 1, 0, nullptr, 1, 0, CUFFT_C2C, 1, work) != CUFFT_SUCCESS) {
    cufftDestroy(*plan);
    return false;
  }
  return true;
}

}  // namespace

extern "C" {

wasabi_status wasabi_reconstruct_scratch_bytes(int w, int h, size_t* bytes_out) {
  if (w <= 0 || h <= 0 || !bytes_out) { set_error("reconstruct_scratch_bytes: bad arguments"); return WASABI_E_INVALID; }
  cufftHandle plan;
  size_t work = 0;
  if (cufftCreate(&plan) != CUFFT_SUCCESS) { set_error("reconstruct: cufftCreate failed"); return WASABI_E_CUDA; }
  long long dims[2] = {h, w};
  const cufftResult r = cufftGetSizeMany64(plan, 2, dims, nullptr, 1, 0, nullptr, 1, 0, CUFFT_C2C, 1, &work);
  cufftDestroy(plan);
  if (r != CUFFT_SUCCESS) { set_error("reconstruct: cufftGetSizeMany64 failed (%d)", (int)r); return WASABI_E_CUDA; }
  *bytes_out = align256((size_t)w * h * sizeof(float2)) + align256(work);
  return WASABI_OK;
}

wasabi_status wasabi_reconstruct(const void* input_dev, int input_kind, int w, int h, double lambda, double pitch,
                                 double d, const wasabi_frame* frame, void* field_out_dev, float* intensity_out_dev,
                                 void* scratch_dev, size_t scratch_bytes, void* stream) {
  if (!input_dev || (!field_out_dev && !intensity_out_dev) || !scratch_dev || w <= 0 || h <= 0) {
    set_error("reconstruct: need an input, an output and scratch");
    return WASABI_E_INVALID;
  }
  if (input_kind != WASABI_RECON_FIELD && input_kind != WASABI_RECON_BITS) {
    set_error("reconstruct: unknown input kind %d", input_kind);
    return WASABI_E_INVALID;
  }
  if (input_kind == WASABI_RECON_BITS && w % 8) { set_error("reconstruct: bits input needs w %% 8 == 0"); return WASABI_E_INVALID; }
  if (!(std::isfinite(lambda) && lambda > 0 && std::isfinite(pitch) && pitch > 0 && std::isfinite(d))) {
    set_error("reconstruct: need finite lambda > 0, pitch > 0 and a finite distance");
    return WASABI_E_INVALID;
  }
  if (((uintptr_t)input_dev & 7) || ((uintptr_t)field_out_dev & 7) || ((uintptr_t)intensity_out_dev & 3) ||
      ((uintptr_t)scratch_dev & 255)) {
    set_error("reconstruct: misaligned buffer");
    return WASABI_E_INVALID;
  }
  int ox, oy;
  RefDev ref;
  const char* why = "";
  if (!frame_to_dev(frame, &ox, &oy, &ref, &why)) { set_error("reconstruct: %s", why); return WASABI_E_INVALID; }
  int* status;
  int sms;
  if (!device_info(&status, &sms)) return WASABI_E_CUDA;
  const cudaStream_t s = (cudaStream_t)stream;
  const long long n = (long long)w * h;
  cufftHandle plan;
  size_t work = 0;
  if (!make_plan(w, h, &plan, &work)) { set_error("reconstruct: cuFFT plan failed for %d x %d", w, h); return WASABI_E_CUDA; }
  const size_t need = align256((size_t)n * sizeof(float2)) + align256(work);
  if (scratch_bytes < need) {
    cufftDestroy(plan);
    set_error("reconstruct: scratch too small (%zu < %zu bytes)", scratch_bytes, need);
    return WASABI_E_NOMEM;
  }
  float2* buf = static_cast<float2*>(scratch_dev);
  void* workarea = static_cast<char*>(scratch_dev) + align256((size_t)n * sizeof(float2));
  wasabi_status st = WASABI_OK;
  const unsigned grid = (unsigned)std::max(1, sms * 8);
  cufftResult fr = cufftSetWorkArea(plan, workarea);
  if (fr == CUFFT_SUCCESS) fr = cufftSetStream(plan, s);
  if (fr == CUFFT_SUCCESS) {
    recon_input_kernel<<<grid, 256, 0, s>>>(input_kind == WASABI_RECON_FIELD ? static_cast<const float2*>(input_dev)
                                                                             : nullptr,
                                            static_cast<const uint8_t*>(input_dev), w, n, ox, oy, ref, buf);
    fr = cufftExecC2C(plan, reinterpret_cast<cufftComplex*>(buf), reinterpret_cast<cufftComplex*>(buf),
                      CUFFT_FORWARD);
  }
  if (fr == CUFFT_SUCCESS) {
    recon_transfer_kernel<<<grid, 256, 0, s>>>(buf, w, h, lambda, pitch, d);
    fr = cufftExecC2C(plan, reinterpret_cast<cufftComplex*>(buf), reinterpret_cast<cufftComplex*>(buf),
                      CUFFT_INVERSE);
  }
  if (fr == CUFFT_SUCCESS) {
    recon_output_kernel<<<grid, 256, 0, s>>>(buf, n, static_cast<float2*>(field_out_dev), intensity_out_dev);
  } else {
    set_error("reconstruct: cuFFT failed (%d)", (int)fr);
    st = WASABI_E_CUDA;
  }
  const cudaError_t e = cudaStreamSynchronize(s);  // the plan is destroyed below
  cufftDestroy(plan);
  if (st == WASABI_OK && e != cudaSuccess) st = cuda_fail("reconstruct", e);
  if (st == WASABI_OK) {
    const cudaError_t e2 = cudaGetLastError();
    if (e2 != cudaSuccess) st = cuda_fail("reconstruct: launch", e2);
  }
  return st;
}

}  // extern "C"
