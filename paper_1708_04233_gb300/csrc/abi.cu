// libwasabi C ABI: argument checks, LUT ownership, scratch layout and the
// launches of the kernels in the other translation units.  See
// include/wasabi.h for the contract of each entry point.
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_fp16.h>

#include "internal.cuh"
#include "lut_object.h"

namespace wsb {
int direct_max_cell_rows();
}  // namespace wsb

// ------------------------------------------------------------ device status
// One word per device (a file-scope device variable: no allocation needed).
__device__ int g_wasabi_status = 0;

namespace wsb {
namespace {

thread_local std::string t_err;
std::mutex g_mu;
constexpr int kMaxDev = 64;
int* g_status_ptr[kMaxDev] = {nullptr};
int g_num_sms[kMaxDev] = {0};
cudaMemPool_t g_pool[kMaxDev] = {nullptr};

constexpr double kPi = 3.14159265358979323846264338327950288;

int current_device() {
  int dev = 0;
  cudaGetDevice(&dev);
  return dev;
}

}  // namespace

// Status word address and SM count of the current device (looked up once).
bool device_info(int** status, int* sms) {
  const int dev = current_device();
  if (dev < 0 || dev >= kMaxDev) { set_error("device ordinal %d out of range", dev); return false; }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_status_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_wasabi_status);
    if (e != cudaSuccess) { set_error("cudaGetSymbolAddress(status): %s", cudaGetErrorString(e)); return false; }
    int n = 0;
    e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) { set_error("cudaDeviceGetAttribute: %s", cudaGetErrorString(e)); return false; }
    // The library's own stream-ordered pool (LUT blocks and build scratch):
    // memory freed to it stays mapped for the next build instead of being
    // released at every synchronisation.  A pool of its own, so that the
    // device's default pool, which the host application may use, keeps its
    // settings.
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof props);
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    e = cudaMemPoolCreate(&pool, &props);
    if (e != cudaSuccess) { set_error("cudaMemPoolCreate: %s", cudaGetErrorString(e)); return false; }
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    g_pool[dev] = pool;
    g_status_ptr[dev] = static_cast<int*>(p);
    g_num_sms[dev] = n;
  }
  if (status) *status = g_status_ptr[dev];
  if (sms) *sms = g_num_sms[dev];
  // Every entry point that launches passes through here first; its launch
  // errors are read with cudaGetLastError, so an earlier, unrelated
  // (non-sticky) error is cleared now.
  cudaGetLastError();
  return true;
}

cudaError_t pool_alloc(void** p, size_t bytes, cudaStream_t s) {
  const int dev = current_device();
  if (dev < 0 || dev >= kMaxDev || !g_pool[dev]) return cudaErrorInitializationError;
  return cudaMallocFromPoolAsync(p, bytes, g_pool[dev], s);
}

wasabi_status cuda_fail(const char* what, cudaError_t e) {
  set_error("%s: %s", what, cudaGetErrorString(e));
  return WASABI_E_CUDA;
}

namespace {

// Support radius in pixels: z tan(asin(lambda / 2p)) / p.
double support_radius(double lambda, double pitch, double z) {
  const double s = lambda / (2.0 * pitch);
  const double t = s / std::sqrt(1.0 - s * s);
  return (std::fabs(z) * t) / pitch;
}

// Pinned staging for the small per-depth tables a LUT build uploads: one
// buffer per device, reused by later builds once the previous upload has
// completed.  Uploads from pinned memory do not wait for other work on the
// device, as copies from pageable memory can.
struct Staging {
  std::mutex mu;
  char* host = nullptr;
  size_t cap = 0;
  cudaEvent_t done = nullptr;
};
Staging g_staging[kMaxDev];

struct Upload {
  void* dst;
  const void* src;
  size_t bytes;
};

cudaError_t staged_upload(int dev, cudaStream_t s, const Upload* ups, int n) {
  Staging& st = g_staging[dev];
  std::lock_guard<std::mutex> lk(st.mu);
  size_t total = 0;
  for (int i = 0; i < n; ++i) total += align_up(ups[i].bytes, 16);
  cudaError_t e = cudaSuccess;
  if (st.done) e = cudaEventSynchronize(st.done);  // the previous build's upload has left the buffer
  if (e == cudaSuccess && st.cap < total) {
    if (st.host) cudaFreeHost(st.host);
    st.host = nullptr;
    st.cap = 0;
    const size_t want = std::max<size_t>(total, 64 * 1024);
    e = cudaMallocHost(&st.host, want);
    if (e == cudaSuccess) st.cap = want;
  }
  if (e == cudaSuccess && !st.done) e = cudaEventCreateWithFlags(&st.done, cudaEventDisableTiming);
  size_t off = 0;
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    std::memcpy(st.host + off, ups[i].src, ups[i].bytes);
    e = cudaMemcpyAsync(ups[i].dst, st.host + off, ups[i].bytes, cudaMemcpyHostToDevice, s);
    off += align_up(ups[i].bytes, 16);
  }
  if (e == cudaSuccess) e = cudaEventRecord(st.done, s);
  return e;
}

// A pinned host word per device that a one-thread kernel writes: small
// results come back without a device-to-host copy, so they never queue
// behind a large copy in flight on another stream.
struct HostWord {
  std::mutex mu;
  unsigned* word = nullptr;
};
HostWord g_hostword[kMaxDev];

__global__ void word_to_host_kernel(const unsigned* src, unsigned* dst) { *(volatile unsigned*)dst = *src; }

// Reads *src_dev after the work already on s; synchronises s.
cudaError_t read_word(int dev, const unsigned* src_dev, cudaStream_t s, unsigned* out) {
  HostWord& hw = g_hostword[dev];
  std::lock_guard<std::mutex> lk(hw.mu);
  cudaError_t e = cudaSuccess;
  if (!hw.word) e = cudaMallocHost(&hw.word, sizeof(unsigned));
  if (e != cudaSuccess) return e;
  word_to_host_kernel<<<1, 1, 0, s>>>(src_dev, hw.word);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) *out = *(volatile unsigned*)hw.word;
  return e;
}

int env_int(const char* name, int dflt) {
  const char* v = std::getenv(name);
  return v && *v ? std::atoi(v) : dflt;
}

}  // namespace

void set_error(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  t_err = buf;
}

int* device_status_ptr() {
  int* p = nullptr;
  device_info(&p, nullptr);
  return p;
}

}  // namespace wsb

using namespace wsb;

namespace wsb {

void superpose_config(const wasabi_lut* lut, int w, int h, int kind, int* cell, int* threads) {
  int T, nt;
  if (std::max(w, h) < kConfigLargeSide) kind = kConfigShared;
  superpose_default_config(lut->L, lut->lmin, lut->D, kind, &T, &nt);
  {
    std::lock_guard<std::mutex> lk(lut->tune_mu);
    const auto it = lut->tuned.find(size_class(w, h));
    if (it != lut->tuned.end()) { T = it->second.first; nt = it->second.second; }
  }
  T = env_int("WASABI_SUPERPOSE_T", T);
  nt = env_int("WASABI_SUPERPOSE_THREADS", nt);
  T = std::min(T, kMaxSuperTile);
  T = std::max(T, std::max(1 << lut->L, 32));
  // A multiple of 32 pixels (one word of the packed binary output) and of 2^L.
  const int unit = std::max(1 << lut->L, 32);
  T = std::max(unit, T / unit * unit);
  while (T > unit && superpose_smem_bytes(T, lut->L, lut->lmin, lut->D, false, superpose_min_range_cap()) > 220 * 1024)
    T = std::max(unit, T / 2 / unit * unit);
  nt = std::max(superpose_min_threads(), std::min(1024, nt / 32 * 32));
  *cell = T;
  *threads = nt;
}

}  // namespace wsb

namespace {

// Scratch of a one-job call: the job table, the batch totals, the cell
// arrays and the binned points.
struct BinLayout {
  int cell, ncx, ncy;
  size_t bytes;
  JobDev* jobs;
  BatchDev* batch;
  int *cnt, *off, *cursor;
  wasabi_point* sorted;
};

BinLayout bin_layout(int64_t n, int w, int h, int cell, void* base) {
  BinLayout b;
  b.cell = cell;
  b.ncx = (w + cell - 1) / cell;
  b.ncy = (h + cell - 1) / cell;
  const size_t ncells = (size_t)b.ncx * b.ncy;
  Carver c;
  c.base = static_cast<char*>(base);
  b.jobs = c.take<JobDev>(1);
  b.batch = c.take<BatchDev>(1);
  b.cnt = c.take<int>(ncells + 1);
  b.off = c.take<int>(ncells + 1);
  b.cursor = c.take<int>(ncells);
  b.sorted = c.take<wasabi_point>((size_t)std::max<int64_t>(n, 1));
  b.bytes = align_up(c.off, 256);
  return b;
}

// Device address of a field of the device-resident batch totals.
template <typename T>
T* batch_field(BatchDev* b, size_t offset) {
  return reinterpret_cast<T*>(reinterpret_cast<char*>(b) + offset);
}

JobDev make_job(const wasabi_lut* lut, const wasabi_point* pts, int64_t n, int w, int h, int rule,
                int cell, float2* wbuf, float2* u, uint8_t* bits) {
  JobDev J;
  std::memset(&J, 0, sizeof J);
  J.pts = pts;
  J.wbuf = wbuf;
  J.u = u;
  J.bits = bits;
  J.n = n;
  J.w = w;
  J.h = h;
  J.ntx = w >> lut->L;
  J.nty = h >> lut->L;
  J.ncx = (w + cell - 1) / cell;
  J.ncy = (h + cell - 1) / cell;
  J.ncells = J.ncx * J.ncy;
  J.rule = rule;
  return J;
}

int super_tiles(int ntx, int nty, int k) { return ((ntx + k - 1) / k) * ((nty + k - 1) / k); }

}  // namespace

extern "C" {

const char* wasabi_last_error(void) { return t_err.c_str(); }

wasabi_status wasabi_depth_grid(double zmin, double zmax, int n_depths, double* depths_host) {
  if (n_depths < 1 || !(zmax > zmin) || !depths_host) {
    set_error("depth_grid: need n_depths >= 1, zmax > zmin and an output array");
    return WASABI_E_INVALID;
  }
  const double dz = (zmax - zmin) / (double)n_depths;
  for (int d = 0; d < n_depths; ++d) depths_host[d] = zmin + ((double)d + 0.5) * dz;
  return WASABI_OK;
}

wasabi_status wasabi_quantize_points(const int32_t* x_dev, const int32_t* y_dev, const double* z_dev,
                                     const float* a_dev, int64_t n, double zmin, double zmax,
                                     int n_depths, wasabi_point* out_dev, void* stream) {
  if (n < 0 || n_depths < 1 || !(zmax > zmin) || (n > 0 && (!x_dev || !y_dev || !z_dev || !a_dev || !out_dev))) {
    set_error("quantize_points: bad arguments");
    return WASABI_E_INVALID;
  }
  int* status;
  if (!device_info(&status, nullptr)) return WASABI_E_CUDA;
  const double dz = (zmax - zmin) / (double)n_depths;
  const cudaError_t e = launch_quantize(x_dev, y_dev, z_dev, a_dev, n, zmin, zmax, dz, n_depths,
                                        out_dev, status, (cudaStream_t)stream);
  return e == cudaSuccess ? WASABI_OK : cuda_fail("quantize launch", e);
}

wasabi_status wasabi_build_lut(double lambda, double pitch, const double* depths_host, int n_depths,
                               int window, int levels, double keep_ratio, int dtype, void* stream,
                               wasabi_lut** out) {
  return wasabi_build_lut_wavelet(lambda, pitch, depths_host, n_depths, window, levels, keep_ratio, dtype,
                                  WASABI_HAAR, stream, out);
}

wasabi_status wasabi_build_lut_wavelet(double lambda, double pitch, const double* depths_host, int n_depths,
                                       int window, int levels, double keep_ratio, int dtype, int wavelet,
                                       void* stream, wasabi_lut** out) {
  if (!out) { set_error("build_lut: out is NULL"); return WASABI_E_INVALID; }
  if (wavelet != WASABI_HAAR && wavelet != WASABI_COIF1) { set_error("build_lut: unknown wavelet %d", wavelet); return WASABI_E_INVALID; }
  const bool coif = wavelet == WASABI_COIF1;
  *out = nullptr;
  if (!(lambda > 0) || !(pitch > 0) || !(lambda / (2.0 * pitch) < 1.0)) {
    set_error("build_lut: need lambda > 0, pitch > 0 and lambda / (2 pitch) < 1");
    return WASABI_E_INVALID;
  }
  if (n_depths < 1 || n_depths > kMaxDepths || !depths_host) {
    set_error("build_lut: n_depths must be in [1, %d]", kMaxDepths);
    return WASABI_E_INVALID;
  }
  if (levels < 1 || levels > kMaxLevels) {
    set_error("build_lut: levels must be in [1, %d]", kMaxLevels);
    return WASABI_E_INVALID;
  }
  if (window <= 0 || window % (2 << levels) != 0 || window > kMaxWindow || (window >> levels) > kMaxWindowTiles ||
      (long long)n_depths * ((long long)(window >> levels) * (window >> levels) + 1) > INT_MAX) {
    set_error("build_lut: window must be a positive multiple of 2^(levels+1), at most %d, with "
              "window/2^levels <= %d and n_depths * (window/2^levels)^2 < 2^31", kMaxWindow, kMaxWindowTiles);
    return WASABI_E_INVALID;
  }
  if (!(keep_ratio > 0)) { set_error("build_lut: keep_ratio must be > 0"); return WASABI_E_INVALID; }
  if (dtype != WASABI_F32 && dtype != WASABI_F16S && dtype != WASABI_BF16S) {
    set_error("build_lut: unknown dtype %d", dtype);
    return WASABI_E_INVALID;
  }
  wasabi_lut* lut = new wasabi_lut;
  lut->stream = (cudaStream_t)stream;
  lut->lambda = lambda; lut->pitch = pitch; lut->gamma = keep_ratio;
  lut->D = n_depths; lut->W = window; lut->L = levels; lut->nwt = window >> levels; lut->dtype = dtype;
  const int TSL = 1 << (2 * levels);
  std::vector<double> R2(n_depths);
  std::vector<long long> target(n_depths);
  lut->z.assign(depths_host, depths_host + n_depths);
  lut->R.resize(n_depths);
  lut->meta.resize(n_depths);
  int max_nb = 1, max_fr = 0;
  long long max_cap = 0, base = 0;
  for (int d = 0; d < n_depths; ++d) {
    const double z = depths_host[d];
    if (!std::isfinite(z)) { delete lut; set_error("build_lut: depth %d is not finite", d); return WASABI_E_INVALID; }
    const double R = support_radius(lambda, pitch, z);
    if (2.0 * R + 1.0 > (double)window) {
      delete lut;
      set_error("build_lut: PSF of depth %d has radius %.2f px, needs a window >= %d", d, R,
                (int)std::ceil(2.0 * R + 1.0));
      return WASABI_E_INVALID;
    }
    lut->R[d] = R;
    R2[d] = R * R;
    const int fr = (int)std::floor(R);
    max_fr = std::max(max_fr, fr);
    DepthMeta m;
    // Haar coefficients stay in the tiles the disk meets; coiflet filters
    // spread over the periodic window, so every tile is searched.
    m.tlo = coif ? 0 : std::max(0, (window / 2 - fr) >> levels);
    m.thi = coif ? lut->nwt - 1 : std::min(lut->nwt - 1, (window / 2 + fr) >> levels);
    const int nb = m.thi - m.tlo + 1;
    max_nb = std::max(max_nb, nb);
    const long long box = (long long)nb * nb * TSL;
    long long cap = box;
    if (keep_ratio < 1.0 && R > 1.0) {  // R <= 1: a delta, all its coefficients kept
      target[d] = (long long)std::ceil(keep_ratio * (kPi * (R * R)) - 1e-9);
      cap = std::min(cap, std::max(0ll, target[d]));
    } else {
      target[d] = LLONG_MAX;
    }
    cap = (long long)align_up((size_t)std::max(cap, 1ll), 32);
    m.base = (int)base;
    m.cap = (int)cap;
    base += cap;
    max_cap = std::max(max_cap, cap);
    lut->meta[d] = m;
  }
  if (base > INT_MAX) { delete lut; set_error("build_lut: table too large"); return WASABI_E_INVALID; }
  lut->total_cap = base;
  lut->reach = (coif ? window / 2 : max_fr) + (2 << levels);
  lut->wavelet = wavelet;
  const int ntpd = 2 * lut->nwt * (lut->nwt + 1);  // per depth: rows x segments x (tiles + 1)
  const cudaStream_t s = (cudaStream_t)stream;
  int* status;
  int sms;
  if (!device_info(&status, &sms)) { delete lut; return WASABI_E_CUDA; }
  lut->device = current_device();

  // Persistent arrays.
  Carver c;
  c.take<uint32_t>((size_t)base);                                    // pos
  c.take<float2>((size_t)base);                                      // val
  if (dtype != WASABI_F32) { c.take<uint32_t>((size_t)base); c.take<float>((size_t)base / 32 + 1); }
  c.take<int32_t>((size_t)n_depths * ntpd);                          // tile_off
  c.take<DepthMeta>((size_t)n_depths);
  c.take<long long>((size_t)n_depths);                               // nr
  c.take<float>(1);                                                  // cmax
  c.take<unsigned>(1);                                               // levels
  {
    const int unit = std::max(1 << levels, 32);  // super-tile sides: multiples of 32 and of 2^L
    for (int T = unit; T <= kMaxSuperTile && lut->ncode < kMaxCodes; T += unit) lut->code_k[lut->ncode++] = T >> levels;
  }
  c.take<uint2>((size_t)lut->ncode * (size_t)base + kCodePad);      // plane-code records
  const size_t persist_bytes = align_up(c.off, 256);
  cudaError_t e = pool_alloc(&lut->block, persist_bytes, s);
  if (e != cudaSuccess) { delete lut; set_error("build_lut: cudaMallocAsync: %s", cudaGetErrorString(e)); return WASABI_E_NOMEM; }
  c = Carver();
  c.base = static_cast<char*>(lut->block);
  lut->pos = c.take<uint32_t>((size_t)base);
  lut->val = c.take<float2>((size_t)base);
  if (dtype != WASABI_F32) {
    lut->val16 = c.take<uint32_t>((size_t)base);
    lut->scale = c.take<float>((size_t)base / 32 + 1);
  }
  lut->tile_off = c.take<int32_t>((size_t)n_depths * ntpd);
  lut->meta_dev = c.take<DepthMeta>((size_t)n_depths);
  lut->nr_dev = c.take<long long>((size_t)n_depths);
  lut->cmax = c.take<float>(1);
  lut->levels = c.take<unsigned>(1);
  lut->code = c.take<uint2>((size_t)lut->ncode * (size_t)base + kCodePad);
  e = cudaMemsetAsync(lut->code + (size_t)lut->ncode * (size_t)base, 0, kCodePad * sizeof(uint2), s);
  if (e != cudaSuccess) {
    cudaFreeAsync(lut->block, s);
    delete lut;
    set_error("build_lut: %s", cudaGetErrorString(e));
    return WASABI_E_CUDA;
  }

  // Build scratch.
  Carver sc;
  sc.take<float2>((size_t)n_depths * window * window);
  sc.take<unsigned long long>((size_t)n_depths * window * window);
  sc.take<unsigned long long>((size_t)n_depths);
  sc.take<unsigned long long>((size_t)2 * n_depths);
  sc.take<int>((size_t)n_depths * 2 * lut->nwt * lut->nwt);
  sc.take<double>((size_t)n_depths);
  sc.take<double>((size_t)n_depths);
  sc.take<double>((size_t)n_depths);
  sc.take<int>((size_t)n_depths + 1);
  sc.take<long long>((size_t)n_depths);
  if (coif) sc.take<float2>((size_t)n_depths * window * window);  // coiflet image
  // The PSF's octant table: (floor(R) + 1)(floor(R) + 2) / 2 values per depth.
  std::vector<long long> tri_off(n_depths + 1, 0);
  std::vector<int> tri_rd(n_depths);
  for (int d = 0; d < n_depths; ++d) {
    tri_rd[d] = (int)std::floor(lut->R[d]);
    const long long r1 = tri_rd[d] + 1;
    tri_off[d + 1] = tri_off[d] + r1 * (r1 + 1) / 2;
  }
  sc.take<float2>((size_t)tri_off[n_depths]);
  sc.take<long long>((size_t)n_depths + 1);
  sc.take<int>((size_t)n_depths);
  void* scratch = nullptr;
  e = pool_alloc(&scratch, align_up(sc.off, 256), s);
  if (e != cudaSuccess) {
    cudaFreeAsync(lut->block, s);
    delete lut;
    set_error("build_lut: scratch cudaMallocAsync: %s", cudaGetErrorString(e));
    return WASABI_E_NOMEM;
  }
  sc = Carver();
  sc.base = static_cast<char*>(scratch);
  LutBuildArgs a;
  a.D = n_depths; a.W = window; a.L = levels; a.nwt = lut->nwt; a.dtype = dtype;
  a.max_nb = max_nb; a.max_cap = max_cap;
  a.lambda = lambda; a.pitch = pitch;
  a.coef = sc.take<float2>((size_t)n_depths * window * window);
  a.keys = sc.take<unsigned long long>((size_t)n_depths * window * window);
  a.nnz = sc.take<unsigned long long>((size_t)n_depths);
  a.thr = sc.take<unsigned long long>((size_t)2 * n_depths);
  a.tile_cnt = sc.take<int>((size_t)n_depths * 2 * lut->nwt * lut->nwt);
  double* z_dev = sc.take<double>((size_t)n_depths);
  double* R2_dev = sc.take<double>((size_t)n_depths);
  double* c_dev = sc.take<double>((size_t)n_depths);
  int* blk0_dev = sc.take<int>((size_t)n_depths + 1);
  long long* target_dev = sc.take<long long>((size_t)n_depths);
  a.wavelet = wavelet;
  a.img = coif ? sc.take<float2>((size_t)n_depths * window * window) : nullptr;
  a.tri = sc.take<float2>((size_t)tri_off[n_depths]);
  long long* tri_off_dev = sc.take<long long>((size_t)n_depths + 1);
  int* tri_rd_dev = sc.take<int>((size_t)n_depths);
  a.tri_off = tri_off_dev;
  a.tri_rd = tri_rd_dev;
  {
    double lo[6], hi[6];
    coif1_filters(lo, hi);
    for (int i = 0; i < 6; ++i) { a.ctap_lo[i] = (float)lo[i]; a.ctap_hi[i] = (float)hi[i]; }
  }
  a.z_dev = z_dev; a.R2_dev = R2_dev; a.target_dev = target_dev; a.c_dev = c_dev;
  // Phase constants (pitch / lambda)^2 and (z / lambda)^2, plain IEEE double operations.
  const double pl = pitch / lambda;
  a.q = pl * pl;
  std::vector<double> cz(n_depths);
  for (int d = 0; d < n_depths; ++d) {
    const double zl = std::fabs(depths_host[d]) / lambda;
    cz[d] = zl * zl;
  }
  // PSF blocks: each depth's box tiles, psf_tiles_per_block(L) to a block.
  std::vector<int> blk0(n_depths + 1, 0);
  {
    const int tpb = psf_tiles_per_block(levels);
    long long acc = 0;
    for (int d = 0; d < n_depths; ++d) {
      blk0[d] = (int)acc;
      const long long nbd = lut->meta[d].thi - lut->meta[d].tlo + 1;
      acc += (nbd * nbd + tpb - 1) / tpb;
    }
    blk0[n_depths] = (int)acc;
  }
  a.psf_blk0 = blk0_dev;
  a.psf_blocks = blk0[n_depths];
  a.nr_dev = lut->nr_dev; a.pos = lut->pos; a.val = lut->val; a.val16 = lut->val16; a.scale = lut->scale;
  a.tile_off = lut->tile_off; a.meta = lut->meta_dev; a.cmax = lut->cmax; a.levels = lut->levels;
  a.code = lut->code; a.ncode = lut->ncode; a.total = base;
  for (int i = 0; i < kMaxCodes; ++i) a.code_k[i] = lut->code_k[i];
  a.status = status;

  const Upload ups[] = {
      {z_dev, depths_host, sizeof(double) * n_depths},
      {R2_dev, R2.data(), sizeof(double) * n_depths},
      {c_dev, cz.data(), sizeof(double) * n_depths},
      {blk0_dev, blk0.data(), sizeof(int) * (n_depths + 1)},
      {target_dev, target.data(), sizeof(long long) * n_depths},
      {tri_off_dev, tri_off.data(), sizeof(long long) * (n_depths + 1)},
      {tri_rd_dev, tri_rd.data(), sizeof(int) * n_depths},
      {lut->meta_dev, lut->meta.data(), sizeof(DepthMeta) * n_depths},
  };
  bool okc = staged_upload(lut->device, s, ups, (int)(sizeof ups / sizeof ups[0])) == cudaSuccess;
  okc = okc && cudaMemsetAsync(a.nnz, 0, sizeof(unsigned long long) * n_depths, s) == cudaSuccess;
  okc = okc && cudaMemsetAsync(lut->cmax, 0, sizeof(float), s) == cudaSuccess;
  okc = okc && cudaMemsetAsync(lut->levels, 0, sizeof(unsigned), s) == cudaSuccess;
  if (!okc) {
    cudaFreeAsync(scratch, s);
    cudaFreeAsync(lut->block, s);
    delete lut;
    return cuda_fail("build_lut: upload", cudaGetLastError());
  }
  e = launch_lut_build(a, s);
  cudaFreeAsync(scratch, s);
  if (e != cudaSuccess) {
    cudaFreeAsync(lut->block, s);
    delete lut;
    return cuda_fail("build_lut: launch", e);
  }
  // The finest kept level sizes the superposition's accumulator: wait for the
  // build and read it back.
  unsigned lvmask = 0;
  e = read_word(lut->device, lut->levels, s, &lvmask);
  if (e != cudaSuccess) {
    cudaFreeAsync(lut->block, s);
    delete lut;
    return cuda_fail("build_lut: readback", e);
  }
  lut->lmin = lut->L;  // an empty table needs only the coarsest slots
  for (int l = 1; l <= lut->L; ++l) {
    if (lvmask & (1u << l)) { lut->lmin = l; break; }
  }
  *out = lut;
  return WASABI_OK;
}

wasabi_status wasabi_lut_destroy(wasabi_lut* lut) {
  if (!lut) return WASABI_OK;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(lut->device);
  cudaFreeAsync(lut->block, lut->stream);
  cudaSetDevice(prev);
  delete lut;
  return WASABI_OK;
}

wasabi_status wasabi_lut_counts(const wasabi_lut* lut, int64_t* nr_host) {
  if (!lut || !nr_host) { set_error("lut_counts: NULL argument"); return WASABI_E_INVALID; }
  cudaError_t e = cudaStreamSynchronize(lut->stream);
  if (e != cudaSuccess) return cuda_fail("lut_counts: sync", e);
  std::vector<long long> nr(lut->D);
  e = cudaMemcpy(nr.data(), lut->nr_dev, sizeof(long long) * lut->D, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail("lut_counts: copy", e);
  for (int d = 0; d < lut->D; ++d) nr_host[d] = nr[d];
  return WASABI_OK;
}

namespace {
wasabi_status read_depth(const wasabi_lut* lut, int depth, std::vector<uint32_t>* pos,
                         std::vector<float2>* val) {
  if (!lut || depth < 0 || depth >= lut->D) { set_error("lut: bad depth"); return WASABI_E_INVALID; }
  cudaError_t e = cudaStreamSynchronize(lut->stream);
  if (e != cudaSuccess) return cuda_fail("lut: sync", e);
  long long nr = 0;
  e = cudaMemcpy(&nr, lut->nr_dev + depth, sizeof nr, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail("lut: copy", e);
  const size_t b = (size_t)lut->meta[depth].base;
  pos->resize((size_t)nr);
  val->resize((size_t)nr);
  if (nr == 0) return WASABI_OK;
  e = cudaMemcpy(pos->data(), lut->pos + b, sizeof(uint32_t) * nr, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail("lut: copy", e);
  if (lut->dtype == WASABI_F32) {
    e = cudaMemcpy(val->data(), lut->val + b, sizeof(float2) * nr, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail("lut: copy", e);
  } else {
    std::vector<uint32_t> q((size_t)nr);
    std::vector<float> sc((size_t)(nr + 31) / 32);
    e = cudaMemcpy(q.data(), lut->val16 + b, sizeof(uint32_t) * nr, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
      e = cudaMemcpy(sc.data(), lut->scale + b / 32, sizeof(float) * sc.size(), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail("lut: copy", e);
    for (size_t i = 0; i < (size_t)nr; ++i) {
      float re, im;
      const uint16_t lo = (uint16_t)(q[i] & 0xffff), hi = (uint16_t)(q[i] >> 16);
      if (lut->dtype == WASABI_BF16S) {
        uint32_t a = (uint32_t)lo << 16, c = (uint32_t)hi << 16;
        std::memcpy(&re, &a, 4);
        std::memcpy(&im, &c, 4);
      } else {
        re = __half2float(__ushort_as_half(lo));
        im = __half2float(__ushort_as_half(hi));
      }
      (*val)[i] = make_float2(re * sc[i / 32], im * sc[i / 32]);
    }
  }
  return WASABI_OK;
}

int32_t pos_to_mallat(const wasabi_lut* lut, uint32_t p) {
  int P, Q, lev, band;
  unpack_pos(p, &P, &Q, &lev, &band);
  const int S = lut->W >> lev;
  const int row = Q + ((band == 2 || band == 3) ? S : 0);
  const int col = P + ((band == 1 || band == 3) ? S : 0);
  return row * lut->W + col;
}
}  // namespace

wasabi_status wasabi_lut_selection(const wasabi_lut* lut, int depth, int32_t* idx_host, int64_t* n_inout) {
  if (!n_inout) { set_error("lut_selection: NULL count"); return WASABI_E_INVALID; }
  std::vector<uint32_t> pos;
  std::vector<float2> val;
  const wasabi_status st = read_depth(lut, depth, &pos, &val);
  if (st != WASABI_OK) return st;
  const int64_t cap = *n_inout;
  *n_inout = (int64_t)pos.size();
  if ((int64_t)pos.size() > cap || (!idx_host && !pos.empty())) { set_error("lut_selection: capacity too small"); return WASABI_E_NOMEM; }
  std::vector<int32_t> idx(pos.size());
  for (size_t i = 0; i < pos.size(); ++i) idx[i] = pos_to_mallat(lut, pos[i]);
  std::sort(idx.begin(), idx.end());
  std::copy(idx.begin(), idx.end(), idx_host);
  return WASABI_OK;
}

wasabi_status wasabi_lut_entries(const wasabi_lut* lut, int depth, int32_t* idx_host, float* val_host,
                                 int64_t* n_inout) {
  if (!n_inout) { set_error("lut_entries: NULL count"); return WASABI_E_INVALID; }
  std::vector<uint32_t> pos;
  std::vector<float2> val;
  const wasabi_status st = read_depth(lut, depth, &pos, &val);
  if (st != WASABI_OK) return st;
  const int64_t cap = *n_inout;
  *n_inout = (int64_t)pos.size();
  if ((int64_t)pos.size() > cap || ((!idx_host || !val_host) && !pos.empty())) { set_error("lut_entries: capacity too small"); return WASABI_E_NOMEM; }
  for (size_t i = 0; i < pos.size(); ++i) {
    idx_host[i] = pos_to_mallat(lut, pos[i]);
    val_host[2 * i] = val[i].x;
    val_host[2 * i + 1] = val[i].y;
  }
  return WASABI_OK;
}

wasabi_status wasabi_scratch_bytes(const wasabi_lut* lut, int64_t n, int holo_w, int holo_h, size_t* bytes_out) {
  if (!lut || !bytes_out || n < 0 || holo_w <= 0 || holo_h <= 0) {
    set_error("scratch_bytes: bad arguments");
    return WASABI_E_INVALID;
  }
  // The smallest cell the configuration can pick bounds every layout.
  const int cell = std::max(1 << lut->L, 32);
  *bytes_out = bin_layout(n, holo_w, holo_h, cell, nullptr).bytes;
  return WASABI_OK;
}

wasabi_status wasabi_superpose(const wasabi_lut* lut, const wasabi_point* points_dev, int64_t n, int holo_w,
                               int holo_h, int rule, void* wbuf_dev, void* scratch_dev, size_t scratch_bytes,
                               void* stream) {
  if (!lut) { set_error("superpose: NULL argument"); return WASABI_E_INVALID; }
  int cell, threads;
  superpose_config(lut, holo_w, holo_h, kConfigComplex, &cell, &threads);
  if (!wbuf_dev) { set_error("superpose: NULL wavelet buffer"); return WASABI_E_INVALID; }
  return superpose_impl(lut, points_dev, n, holo_w, holo_h, rule, wbuf_dev, nullptr, nullptr, scratch_dev,
                        scratch_bytes, (cudaStream_t)stream, cell, threads);
}

wasabi_status wasabi_hologram(const wasabi_lut* lut, const wasabi_point* points_dev, int64_t n, int holo_w,
                              int holo_h, int rule, void* wbuf_dev, void* u_dev, uint8_t* bits_dev,
                              void* scratch_dev, size_t scratch_bytes, void* stream) {
  if (!lut) { set_error("hologram: NULL argument"); return WASABI_E_INVALID; }
  if (!u_dev && !bits_dev) { set_error("hologram: need u_dev or bits_dev"); return WASABI_E_INVALID; }
  int cell, threads;
  superpose_config(lut, holo_w, holo_h, superpose_config_kind(wbuf_dev, u_dev, bits_dev, nullptr), &cell, &threads);
  return superpose_impl(lut, points_dev, n, holo_w, holo_h, rule, wbuf_dev, u_dev, bits_dev, scratch_dev,
                        scratch_bytes, (cudaStream_t)stream, cell, threads);
}

wasabi_status wasabi_hologram_frame(const wasabi_lut* lut, const wasabi_point* points_dev, int64_t n, int holo_w,
                                    int holo_h, int rule, const wasabi_frame* frame, void* wbuf_dev, void* u_dev,
                                    uint8_t* bits_dev, void* scratch_dev, size_t scratch_bytes, void* stream) {
  if (!lut) { set_error("hologram_frame: NULL argument"); return WASABI_E_INVALID; }
  int cell, threads;
  superpose_config(lut, holo_w, holo_h, superpose_config_kind(wbuf_dev, u_dev, bits_dev, frame), &cell, &threads);
  return superpose_impl(lut, points_dev, n, holo_w, holo_h, rule, wbuf_dev, u_dev, bits_dev, scratch_dev,
                        scratch_bytes, (cudaStream_t)stream, cell, threads, frame);
}

}  // extern "C"

bool wsb::frame_to_dev(const wasabi_frame* f, int* ox, int* oy, RefDev* ref, const char** why) {
  *ox = *oy = 0;
  std::memset(ref, 0, sizeof *ref);
  if (!f) return true;
  const wasabi_reference& r = f->ref;
  if (r.reserved != 0 || (r.kind != WASABI_REF_PLANE && r.kind != WASABI_REF_SPHERICAL)) {
    *why = "unknown reference kind";
    return false;
  }
  if (r.kind == WASABI_REF_SPHERICAL) {
    if (!(std::isfinite(r.lambda) && r.lambda > 0 && std::isfinite(r.pitch) && r.pitch > 0 &&
          std::isfinite(r.x) && std::isfinite(r.y) && std::isfinite(r.z) && r.z != 0)) {
      *why = "spherical reference needs finite lambda, pitch > 0, finite x, y and a finite nonzero z";
      return false;
    }
    const double a = r.pitch / r.lambda, c = r.z / r.lambda;
    ref->kind = 1;
    ref->sgn = r.z < 0 ? -1.f : 1.f;
    ref->a2 = a * a;
    ref->a2f = (float)(a * a);
    ref->c = c * c;
    ref->x = r.x;
    ref->y = r.y;
  }
  *ox = f->origin_x;
  *oy = f->origin_y;
  return true;
}

wasabi_status wsb::superpose_impl(const wasabi_lut* lut, const wasabi_point* points_dev, int64_t n, int holo_w,
                                  int holo_h, int rule, void* wbuf_dev, void* u_dev, uint8_t* bits_dev,
                                  void* scratch_dev, size_t scratch_bytes, cudaStream_t stream, int cell,
                                  int threads, const wasabi_frame* frame) {
  if (!lut || n < 0 || (n > 0 && !points_dev) || (!wbuf_dev && !u_dev && !bits_dev) || !scratch_dev) {
    set_error("superpose: NULL argument");
    return WASABI_E_INVALID;
  }
  int fox, foy;
  RefDev fref;
  const char* why = "";
  if (!frame_to_dev(frame, &fox, &foy, &fref, &why)) { set_error("hologram: %s", why); return WASABI_E_INVALID; }
  if ((u_dev || bits_dev) && lut->L < 2) {
    set_error("hologram: the fused inverse needs levels >= 2");
    return WASABI_E_INVALID;
  }
  if ((u_dev || bits_dev) && lut->wavelet != WASABI_HAAR) {
    set_error("hologram: the fused inverse is Haar's; use wasabi_superpose + wasabi_inverse_wavelet");
    return WASABI_E_INVALID;
  }
  if (bits_dev && holo_w % 8) { set_error("hologram: bits output needs holo_w %% 8 == 0"); return WASABI_E_INVALID; }
  if (((uintptr_t)u_dev & 15) || ((uintptr_t)bits_dev & 3)) { set_error("hologram: misaligned output"); return WASABI_E_INVALID; }
  const int ts = 1 << lut->L;
  if (holo_w < ts || holo_h < ts || holo_w % ts || holo_h % ts || holo_w > (1 << 29) || holo_h > (1 << 29)) {
    set_error("superpose: holo_w and holo_h must be multiples of 2^L = %d", ts);
    return WASABI_E_INVALID;
  }
  if (rule != WASABI_SHIFT_FLOOR && rule != WASABI_SHIFT_NEAREST) { set_error("superpose: unknown rule"); return WASABI_E_INVALID; }
  if (((uintptr_t)scratch_dev | (uintptr_t)wbuf_dev) & 255) { set_error("superpose: buffers must be 256-byte aligned"); return WASABI_E_INVALID; }
  if (current_device() != lut->device) { set_error("superpose: LUT lives on another device"); return WASABI_E_INVALID; }
  int* status;
  int sms;
  if (!device_info(&status, &sms)) return WASABI_E_CUDA;
  if (cell < std::max(1 << lut->L, 32) || cell > kMaxSuperTile || cell % std::max(1 << lut->L, 32) ||
      threads < superpose_min_threads() || threads > 1024 || threads % 32) {
    set_error("superpose: bad configuration (super-tile %d, %d threads)", cell, threads);
    return WASABI_E_INVALID;
  }
  BinLayout b = bin_layout(n, holo_w, holo_h, cell, scratch_dev);
  size_t need = 0;
  wasabi_scratch_bytes(lut, n, holo_w, holo_h, &need);
  if (scratch_bytes < need || scratch_bytes < b.bytes) {
    set_error("superpose: scratch too small (%zu < %zu bytes)", scratch_bytes, std::max(need, b.bytes));
    return WASABI_E_NOMEM;
  }
  const int rows = (cell + 2 * lut->reach) / cell + 2;
  if (rows > superpose_max_cell_rows()) { set_error("superpose: window too large for the super-tile"); return WASABI_E_INVALID; }
  const bool re_only = !wbuf_dev && !u_dev && bits_dev && !frame_needs_complex(frame);
  const int rcap = superpose_range_cap(cell, lut->L, lut->lmin, lut->D, re_only, threads);
  const size_t smem = superpose_smem_bytes(cell, lut->L, lut->lmin, lut->D, re_only, rcap);
  if (smem > 220 * 1024) { set_error("superpose: super-tile %d needs %zu B of shared memory", cell, smem); return WASABI_E_INVALID; }
  const cudaStream_t s = (cudaStream_t)stream;
  JobDev J = make_job(lut, points_dev, n, holo_w, holo_h, rule, cell, static_cast<float2*>(wbuf_dev),
                      static_cast<float2*>(u_dev), bits_dev);
  J.sorted = b.sorted; J.cnt = b.cnt; J.off = b.off; J.cursor = b.cursor;
  J.ox = fox; J.oy = foy; J.ref = fref;
  cudaError_t e = launch_init_single(J, b.jobs, b.batch, super_tiles(J.ntx, J.nty, cell >> lut->L), s);
  if (e != cudaSuccess) return cuda_fail("superpose: init", e);
  BinArgs ba;
  ba.jobs = b.jobs; ba.batch = b.batch; ba.D = lut->D; ba.cell = cell; ba.reach = lut->reach;
  ba.track_amax = 1; ba.status = status;
  ba.grid = sms * 4;
  e = launch_binning(ba, s);
  if (e != cudaSuccess) return cuda_fail("superpose: binning", e);
  SuperposeArgs sa;
  sa.lut = lut->view(cell >> lut->L);
  sa.jobs = b.jobs; sa.batch = b.batch; sa.cell = cell; sa.reach = lut->reach;
  sa.acc_float = env_int("WASABI_ACC_FLOAT", 0) != 0;
  sa.re_only = re_only ? 1 : 0;
  sa.has_ref = (fref.kind != 0 && bits_dev) ? 1 : 0;
  sa.rcap = rcap;
  sa.status = status; sa.threads = threads; sa.grid = sms;
  e = launch_superpose(sa, s);
  return e == cudaSuccess ? WASABI_OK : cuda_fail("superpose: launch", e);
}

extern "C" {

wasabi_status wasabi_inverse_haar(const void* wbuf_dev, int holo_w, int holo_h, int levels, void* u_dev,
                                  uint8_t* bits_dev, void* stream) {
  return wasabi_inverse_haar_frame(wbuf_dev, holo_w, holo_h, levels, nullptr, u_dev, bits_dev, stream);
}

namespace {
wasabi_status inverse_haar_impl(const void* wbuf_dev, int holo_w, int holo_h, int levels, const wasabi_frame* frame,
                                void* u_dev, uint8_t* bits_dev, long long wait_limit, long long skip_item,
                                void* stream);
}  // namespace

wasabi_status wasabi_inverse_haar_frame(const void* wbuf_dev, int holo_w, int holo_h, int levels,
                                        const wasabi_frame* frame, void* u_dev, uint8_t* bits_dev, void* stream) {
  return inverse_haar_impl(wbuf_dev, holo_w, holo_h, levels, frame, u_dev, bits_dev, kInverseWaitCycles, -1, stream);
}

wasabi_status wasabi_test_inverse_stall(const void* wbuf_dev, int holo_w, int holo_h, int levels, uint8_t* bits_dev,
                                        int64_t skip_strip, int64_t wait_cycles, void* stream) {
  if (wait_cycles < 1 || wait_cycles > kInverseWaitCycles || skip_strip < 0) {
    set_error("test_inverse_stall: need 0 <= skip_strip and 1 <= wait_cycles <= %lld", kInverseWaitCycles);
    return WASABI_E_INVALID;
  }
  return inverse_haar_impl(wbuf_dev, holo_w, holo_h, levels, nullptr, nullptr, bits_dev, wait_cycles, skip_strip,
                           stream);
}

}  // extern "C"

namespace {
wasabi_status inverse_haar_impl(const void* wbuf_dev, int holo_w, int holo_h, int levels, const wasabi_frame* frame,
                                void* u_dev, uint8_t* bits_dev, long long wait_limit, long long skip_item,
                                void* stream) {
  int fox, foy;
  RefDev fref;
  const char* why = "";
  if (!frame_to_dev(frame, &fox, &foy, &fref, &why)) { set_error("inverse_haar: %s", why); return WASABI_E_INVALID; }
  if (!wbuf_dev || (!u_dev && !bits_dev)) { set_error("inverse_haar: need the buffer and an output"); return WASABI_E_INVALID; }
  if (levels < 2 || levels > kMaxLevels) { set_error("inverse_haar: levels must be in [2, %d]", kMaxLevels); return WASABI_E_INVALID; }
  const int ts = 1 << levels;
  if (holo_w < ts || holo_h < ts || holo_w % ts || holo_h % ts) {
    set_error("inverse_haar: holo_w and holo_h must be multiples of 2^levels");
    return WASABI_E_INVALID;
  }
  if (bits_dev && holo_w % 8) { set_error("inverse_haar: bits output needs holo_w % 8 == 0"); return WASABI_E_INVALID; }
  if (((uintptr_t)wbuf_dev & 15) || ((uintptr_t)u_dev & 15) || ((uintptr_t)bits_dev & 3)) {
    set_error("inverse_haar: misaligned buffer");
    return WASABI_E_INVALID;
  }
  int* status;
  int sms;
  if (!device_info(&status, &sms)) return WASABI_E_CUDA;
  InverseArgs ia;
  std::memset(&ia, 0, sizeof ia);
  ia.wbuf = static_cast<const float2*>(wbuf_dev);
  ia.u = static_cast<float2*>(u_dev);
  ia.bits = bits_dev;
  ia.w = holo_w;
  ia.h = holo_h;
  ia.ntx = holo_w >> levels;
  ia.nstrips = inverse_strips(holo_w, holo_h, levels);
  ia.L = levels;
  ia.status = status;
  ia.num_sms = sms;
  ia.ox = fox;
  ia.oy = foy;
  ia.ref = fref;
  ia.wait_limit = wait_limit;
  ia.skip_item = skip_item;
  const cudaError_t e = launch_inverse(ia, (cudaStream_t)stream);
  return e == cudaSuccess ? WASABI_OK : cuda_fail("inverse_haar: launch", e);
}
}  // namespace

extern "C" {

namespace {
int direct_cell(int w, int h, bool aperture) {
  int cell = 64;
  if (!aperture) {
    const int maxdim = std::max(w, h);
    while ((maxdim + cell - 1) / cell + 2 > direct_max_cell_rows()) cell *= 2;
  }
  return cell;
}
}  // namespace

wasabi_status cgh_direct_scratch_bytes(int64_t n, int holo_w, int holo_h, size_t* bytes_out) {
  if (!bytes_out || n < 0 || holo_w <= 0 || holo_h <= 0) { set_error("cgh_direct_scratch_bytes: bad arguments"); return WASABI_E_INVALID; }
  const size_t b = bin_layout(n, holo_w, holo_h, 64, nullptr).bytes;
  *bytes_out = b + align_up(sizeof(double) * kMaxDepths, 256) + align_up(sizeof(long long) * kMaxDepths, 256);
  return WASABI_OK;
}

wasabi_status cgh_direct(double lambda, double pitch, const double* depths_host, int n_depths,
                         const wasabi_point* points_dev, int64_t n, int holo_w, int holo_h, int aperture,
                         void* u_dev, void* scratch_dev, size_t scratch_bytes, void* stream) {
  if (!(lambda > 0) || !(pitch > 0) || !(lambda / (2.0 * pitch) < 1.0) || n_depths < 1 ||
      n_depths > kMaxDepths || !depths_host || n < 0 || (n > 0 && !points_dev) || !u_dev || !scratch_dev ||
      holo_w <= 0 || holo_h <= 0 || holo_w > (1 << 29) || holo_h > (1 << 29)) {
    set_error("cgh_direct: bad arguments");
    return WASABI_E_INVALID;
  }
  if (((uintptr_t)scratch_dev & 255) || ((uintptr_t)u_dev & 7)) { set_error("cgh_direct: misaligned buffer"); return WASABI_E_INVALID; }
  size_t need = 0;
  cgh_direct_scratch_bytes(n, holo_w, holo_h, &need);
  if (scratch_bytes < need) { set_error("cgh_direct: scratch too small (%zu < %zu)", scratch_bytes, need); return WASABI_E_NOMEM; }
  int* status;
  int sms;
  if (!device_info(&status, &sms)) return WASABI_E_CUDA;
  const int cell = direct_cell(holo_w, holo_h, aperture != 0);
  BinLayout b = bin_layout(n, holo_w, holo_h, cell, scratch_dev);
  Carver c;
  c.base = static_cast<char*>(scratch_dev);
  c.off = b.bytes;
  double* beta_dev = c.take<double>(kMaxDepths);
  long long* nlim_dev = c.take<long long>(kMaxDepths);
  std::vector<double> beta(n_depths);
  std::vector<long long> nlim(n_depths);
  double Rmax = 0;
  for (int d = 0; d < n_depths; ++d) {
    const double z = depths_host[d];
    if (!std::isfinite(z)) { set_error("cgh_direct: depth %d is not finite", d); return WASABI_E_INVALID; }
    const double zl = std::fabs(z) / lambda;
    // (z / lambda)^2, negated for a point behind the plane (conjugate term).
    beta[d] = z < 0 ? -(zl * zl) : zl * zl;
    const double R = support_radius(lambda, pitch, z);
    Rmax = std::max(Rmax, R);
    // n < R^2 for integer n, or the centre pixel alone.
    nlim[d] = aperture ? std::max(1ll, (long long)std::ceil(R * R)) : LLONG_MAX;
  }
  const double pl = pitch / lambda;
  const cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(beta_dev, beta.data(), sizeof(double) * n_depths, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(nlim_dev, nlim.data(), sizeof(long long) * n_depths, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail("cgh_direct: upload", e);
  const int reach = aperture ? (int)std::floor(Rmax) + 1 : (INT_MAX / 4);
  JobDev J;
  std::memset(&J, 0, sizeof J);
  J.pts = points_dev; J.sorted = b.sorted; J.cnt = b.cnt; J.off = b.off; J.cursor = b.cursor;
  J.n = n; J.w = holo_w; J.h = holo_h; J.ncx = b.ncx; J.ncy = b.ncy; J.ncells = b.ncx * b.ncy;
  e = launch_init_single(J, b.jobs, b.batch, 0, s);
  if (e != cudaSuccess) return cuda_fail("cgh_direct: init", e);
  BinArgs ba;
  ba.jobs = b.jobs; ba.batch = b.batch; ba.D = n_depths; ba.cell = cell; ba.reach = reach;
  ba.track_amax = 0; ba.status = status;
  ba.grid = sms * 4;
  e = launch_binning(ba, s);  // also zeroes the tile counter
  if (e != cudaSuccess) return cuda_fail("cgh_direct: binning", e);
  DirectArgs da;
  da.lambda = lambda; da.pitch = pitch; da.jobs = b.jobs;
  da.cell = cell; da.w = holo_w; da.h = holo_h; da.D = n_depths;
  da.beta_dev = beta_dev; da.nlim_dev = nlim_dev; da.alpha = pl * pl; da.reach = reach;
  da.counter = batch_field<int>(b.batch, offsetof(BatchDev, counter));
  da.u = static_cast<float2*>(u_dev); da.status = status;
  const long long ntiles = (long long)((holo_w + 31) / 32) * ((holo_h + 31) / 32);
  da.grid = (int)std::min<long long>(ntiles, (long long)sms * 8);
  e = launch_direct(da, s);
  return e == cudaSuccess ? WASABI_OK : cuda_fail("cgh_direct: launch", e);
}

wasabi_status wasabi_sync_status(void* stream) {
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail("sync_status: stream", e);
  int v = 0;
  e = cudaMemcpyFromSymbol(&v, g_wasabi_status, sizeof(int));
  if (e != cudaSuccess) return cuda_fail("sync_status: read", e);
  const int zero = 0;
  e = cudaMemcpyToSymbol(g_wasabi_status, &zero, sizeof(int));
  if (e != cudaSuccess) return cuda_fail("sync_status: clear", e);
  if (v != 0) set_error("device reported status %d", v);
  return v;
}

wasabi_status wasabi_haar_forward(const void* u_dev, int holo_w, int holo_h, int levels, void* wbuf_dev,
                                  void* stream) {
  if (!u_dev || !wbuf_dev || levels < 1 || levels > kMaxLevels) { set_error("haar_forward: bad arguments"); return WASABI_E_INVALID; }
  const int ts = 1 << levels;
  if (holo_w < ts || holo_h < ts || holo_w % ts || holo_h % ts) { set_error("haar_forward: sizes must be multiples of 2^levels"); return WASABI_E_INVALID; }
  const cudaError_t e = launch_haar_forward(static_cast<const float2*>(u_dev), holo_w, holo_h, levels,
                                            static_cast<float2*>(wbuf_dev), (cudaStream_t)stream);
  return e == cudaSuccess ? WASABI_OK : cuda_fail("haar_forward: launch", e);
}

wasabi_status wasabi_wbuf_to_mallat(const void* wbuf_dev, int holo_w, int holo_h, int levels, void* mallat_dev,
                                    void* stream) {
  if (!wbuf_dev || !mallat_dev || levels < 1 || levels > kMaxLevels) { set_error("wbuf_to_mallat: bad arguments"); return WASABI_E_INVALID; }
  const int ts = 1 << levels;
  if (holo_w < ts || holo_h < ts || holo_w % ts || holo_h % ts) { set_error("wbuf_to_mallat: sizes must be multiples of 2^levels"); return WASABI_E_INVALID; }
  const cudaError_t e = launch_wbuf_to_mallat(static_cast<const float2*>(wbuf_dev), holo_w, holo_h, levels,
                                              static_cast<float2*>(mallat_dev), (cudaStream_t)stream);
  return e == cudaSuccess ? WASABI_OK : cuda_fail("wbuf_to_mallat: launch", e);
}

}  // extern "C"
