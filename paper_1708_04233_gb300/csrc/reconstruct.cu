// Numerical reconstruction of a hologram by the angular spectrum method: the
// field in a plane at signed distance d is IFFT2(FFT2(U_0) H) with the
// transfer function H = exp(i 2 pi d sqrt(1/lambda^2 - fx^2 - fy^2)) of free
// space (evanescent frequencies dropped).  Three element-wise kernels around
// two cuFFT C2C transforms: the input (a complex field, or a binary
// hologram's transmittance times the reference wave), the transfer function
// (phase in double-float FP32 pairs, then FP32 sine and cosine), the outputs.
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "dbf.cuh"
#include "lut_object.h"

using namespace wsb;

namespace {

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// U_0 = field, or t R with t the hologram's bit (reference R of the frame).
__global__ void recon_input_kernel(const float2* __restrict__ field, const uint8_t* __restrict__ bits, int w,
                                   long long n, int ox, int oy, RefDbf ref, float2* __restrict__ buf) {
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
      float sn, cs;
      sincospif(2.0f * ref_frac(ref, (float)(ox + x), (float)(oy + y)), &sn, &cs);
      r = make_float2(cs, ref.sgn * sn);
    }
    buf[i] = make_float2(t * r.x, t * r.y);
  }
}

// Spectrum times H / (w h) (the inverse transform is unnormalised).  The
// phase d/lambda sqrt(1 - (lambda fx)^2 - (lambda fy)^2) reaches 10^4 cycles
// and more, so it is carried in double-float to about 2^-44 relative (the
// square root is one Newton step from the FP32 root), then reduced to
// [0, 1): FP32 arithmetic only.  ax, ay: lambda / (w pitch) and
// lambda / (h pitch); cyc: d / lambda.
__global__ void recon_transfer_kernel(float2* __restrict__ buf, int w, int h, Dbf ax, Dbf ay, Dbf cyc, float norm) {
  const long long n = (long long)w * h;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int ky = (int)(i / w), kx = (int)(i - (long long)ky * w);
    const int sx = kx <= (w - 1) / 2 ? kx : kx - w;  // FFT frequency order
    const int sy = ky <= (h - 1) / 2 ? ky : ky - h;
    // q = (lambda fx)^2 + (lambda fy)^2, s = 1 - q.
    const Dbf px = dbf_sqr(dbf_mul_f(ax, (float)sx)), py = dbf_sqr(dbf_mul_f(ay, (float)sy));
    const Dbf q = two_sum(px.hi, py.hi);
    const float ql = __fadd_rn(q.lo, __fadd_rn(px.lo, py.lo));
    const Dbf s0 = two_sum(1.0f, -q.hi);
    const Dbf sv = two_sum(s0.hi, __fsub_rn(s0.lo, ql));
    float2 v = make_float2(0.f, 0.f);
    if (sv.hi > 0.f) {
      // sqrt(s) = y + r: y the FP32 root, r = (s - y^2) / (2 y) with y^2
      // split exactly (s.hi - y^2 is exact: y^2 lies within a factor 2 of s.hi).
      const float y = __fsqrt_rn(sv.hi);
      const float yy = __fmul_rn(y, y), ye = __fmaf_rn(y, y, -yy);
      const float r = __fmul_rn(__fadd_rn(__fsub_rn(__fsub_rn(sv.hi, yy), ye), sv.lo), __fdividef(0.5f, y));
      // Phase in cycles: cyc (y + r); p - floor(p) is exact in FP32.
      const float p = __fmul_rn(cyc.hi, y);
      const float pe = __fmaf_rn(cyc.hi, y, -p) + (cyc.hi * r + cyc.lo * y);
      float f = __fadd_rn(__fsub_rn(p, floorf(p)), pe);
      f -= floorf(f);
      float sn, cs;
      sincospif(2.0f * f, &sn, &cs);
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

// Plans of the first kPlanCache (device, w, h) shapes live for the process;
// one mutex serialises every use of them (stream and work area are set per
// call, then the transforms are enqueued).  Other shapes get a plan for the
// call only.
constexpr int kPlanCache = 8;
struct PlanEntry {
  int dev, w, h;
  cufftHandle plan;
  size_t work;
};
PlanEntry g_plans[kPlanCache];
int g_nplans = 0;
std::mutex g_plan_mu;

// With g_plan_mu held: the plan of (current device, w, h); *owned is true
// when the caller must destroy it (the cache is full).
bool get_plan(int w, int h, cufftHandle* plan, size_t* work, bool* owned) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  for (int i = 0; i < g_nplans; ++i)
    if (g_plans[i].dev == dev && g_plans[i].w == w && g_plans[i].h == h) {
      *plan = g_plans[i].plan;
      *work = g_plans[i].work;
      *owned = false;
      return true;
    }
  if (!make_plan(w, h, plan, work)) return false;
  *owned = g_nplans == kPlanCache;
  if (!*owned) g_plans[g_nplans++] = PlanEntry{dev, w, h, *plan, *work};
  return true;
}

}  // namespace

extern "C" {

wasabi_status wasabi_reconstruct_scratch_bytes(int w, int h, size_t* bytes_out) {
  if (w <= 0 || h <= 0 || !bytes_out) { set_error("reconstruct_scratch_bytes: bad arguments"); return WASABI_E_INVALID; }
  std::lock_guard<std::mutex> lock(g_plan_mu);
  cufftHandle plan;
  size_t work = 0;
  bool owned = false;
  if (!get_plan(w, h, &plan, &work, &owned)) { set_error("reconstruct: cuFFT plan failed for %d x %d", w, h); return WASABI_E_CUDA; }
  if (owned) cufftDestroy(plan);  // never executed
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
  // Plane pixel coordinates are exact in FP32 below 2^24.
  if (std::abs((long long)ox) + w >= (1LL << 24) || std::abs((long long)oy) + h >= (1LL << 24)) {
    set_error("reconstruct: plane pixels must stay below 2^24 in magnitude");
    return WASABI_E_INVALID;
  }
  const RefDbf rd = ref_dbf(ref);
  int* status;
  int sms;
  if (!device_info(&status, &sms)) return WASABI_E_CUDA;
  const cudaStream_t s = (cudaStream_t)stream;
  const long long n = (long long)w * h;
  std::lock_guard<std::mutex> lock(g_plan_mu);
  cufftHandle plan;
  size_t work = 0;
  bool owned = false;
  if (!get_plan(w, h, &plan, &work, &owned)) { set_error("reconstruct: cuFFT plan failed for %d x %d", w, h); return WASABI_E_CUDA; }
  const size_t need = align256((size_t)n * sizeof(float2)) + align256(work);
  if (scratch_bytes < need) {
    if (owned) cufftDestroy(plan);
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
                                            static_cast<const uint8_t*>(input_dev), w, n, ox, oy, rd, buf);
    fr = cufftExecC2C(plan, reinterpret_cast<cufftComplex*>(buf), reinterpret_cast<cufftComplex*>(buf),
                      CUFFT_FORWARD);
  }
  if (fr == CUFFT_SUCCESS) {
    recon_transfer_kernel<<<grid, 256, 0, s>>>(buf, w, h, split(lambda / (w * pitch)), split(lambda / (h * pitch)),
                                               split(d / lambda), (float)(1.0 / (double)n));
    fr = cufftExecC2C(plan, reinterpret_cast<cufftComplex*>(buf), reinterpret_cast<cufftComplex*>(buf),
                      CUFFT_INVERSE);
  }
  if (fr == CUFFT_SUCCESS) {
    recon_output_kernel<<<grid, 256, 0, s>>>(buf, n, static_cast<float2*>(field_out_dev), intensity_out_dev);
  } else {
    set_error("reconstruct: cuFFT failed (%d)", (int)fr);
    st = WASABI_E_CUDA;
  }
  if (owned) {  // a plan for this call only: wait for its transforms before destroying it
    const cudaError_t e = cudaStreamSynchronize(s);
    cufftDestroy(plan);
    if (st == WASABI_OK && e != cudaSuccess) st = cuda_fail("reconstruct", e);
  }
  if (st == WASABI_OK) {
    const cudaError_t e2 = cudaGetLastError();
    if (e2 != cudaSuccess) st = cuda_fail("reconstruct: launch", e2);
  }
  return st;
}

}  // extern "C"
