// Internal declarations shared by the libwasabi translation units.
//
// Layout notes (the public contract is in include/wasabi.h):
//  * LUT entries, per depth d, live at [meta[d].base, meta[d].base + nr[d]) of
//    the pos/val arrays, ordered by window tile (row-major) and then by in-tile
//    slot.  tile_off[d * (nwt*nwt + 1) + t] is the absolute index of window
//    tile t's first entry; entry t + 1 is its end.
//  * pos packs the coefficient's window sub-band position p:13 | q:13 (in
//    units of its level; p, q < W / 2 <= 8192) | level:3 | band:2 (see
//    pack_pos); its window tile is (p >> (L - level), q >> (L - level)).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/wasabi.h"

namespace wsb {

constexpr int kMaxDepths = 4096;
constexpr int kMaxLevels = 5;
constexpr int kMaxWindowTiles = 2048;  // window / 2^levels
constexpr int kMaxWindow = 16384;      // sub-band positions p, q < window / 2 fit 13 bits
constexpr int kPosBits = 13;
constexpr uint32_t kPosMask = (1u << kPosBits) - 1u;

__host__ __device__ inline uint32_t pack_pos(int p, int q, int lev, int band) {
  return (uint32_t)p | ((uint32_t)q << kPosBits) | ((uint32_t)lev << (2 * kPosBits)) |
         ((uint32_t)band << (2 * kPosBits + 3));
}
__host__ __device__ inline void unpack_pos(uint32_t pos, int* p, int* q, int* lev, int* band) {
  *p = (int)(pos & kPosMask);
  *q = (int)((pos >> kPosBits) & kPosMask);
  *lev = (int)((pos >> (2 * kPosBits)) & 7u);
  *band = (int)((pos >> (2 * kPosBits + 3)) & 3u);
}

// Superposition accumulator of one super-tile of k x k tiles (shared memory):
// per kept level l, square planes of side G_l = (k + 2) 2^(L-l) cells -- the
// super-tile plus a guard band one tile wide on every side -- four at level L
// (approximation and three details), three at finer levels, coarse levels
// first.  Rows are G_l + 1 cells apart and planes are padded to 4 modulo 16
// cells, so that lanes adding into neighbouring rows or other bands of the
// same cells fall into different shared-memory banks.  A coefficient's plane
// code is (l << 29) | 4 (band plane * plane size + q * row + p) with (p, q)
// its window-relative position -- the byte offset of its cell's 32-bit word:
// adding a survivor's per-level base (its shift of Eq. (2), the guard and the
// level's offset, in the same units) gives the accumulator address, with no
// bounds test (every visited coefficient lands inside the guard band by
// construction of the LUT ranges).
__host__ __device__ constexpr int plane_side(int k, int L, int l) { return (k + 2) << (L - l); }
__host__ __device__ constexpr int plane_row(int k, int L, int l) { return plane_side(k, L, l) + 1; }
__host__ __device__ constexpr int plane_size(int k, int L, int l) {
  const int n = plane_row(k, L, l) * plane_side(k, L, l);
  return n + ((4 - n % 16) + 16) % 16;
}
__host__ __device__ constexpr int plane_count(int L, int l) { return l == L ? 4 : 3; }
__host__ __device__ inline uint32_t plane_code(uint32_t pos, int L, int k) {
  int p, q, lev, band;
  unpack_pos(pos, &p, &q, &lev, &band);
  if (lev < 1 || lev > L) return 0;  // unused capacity: never visited
  const int bi = lev == L ? band : band - 1;
  return ((uint32_t)lev << 29) | (uint32_t)(4 * (bi * plane_size(k, L, lev) + q * plane_row(k, L, lev) + p));
}
// Index of level l's first super-tile cell past the guard band (planes of the
// coarse levels first, levels below lmin absent).
__host__ __device__ constexpr int plane_first(int k, int L, int lmin, int l) {
  int base = 0;
  for (int m = L; m > l; --m)
    if (m >= lmin) base += plane_count(L, m) * plane_size(k, L, m);
  const int g = 1 << (L - l);
  return base + g * plane_row(k, L, l) + g;
}
// Accumulator size (cells, a multiple of 4) for levels lmin..L.
__host__ __device__ inline int plane_total(int k, int L, int lmin) {
  int n = 0;
  for (int l = lmin; l <= L; ++l) n += plane_count(L, l) * plane_size(k, L, l);
  return (n + 3) & ~3;
}
// Widest super-tile (pixels) the superposition takes.
constexpr int kMaxSuperTile = 256;
// Records allocated past the last plane-code array: the superposition's
// lanes past a pass's end read up to one pass (64 records) beyond it.
constexpr int kCodePad = 64;
// Most plane codes a LUT keeps: one per super-tile width k the superposition
// can use (super-tiles are multiples of 32 pixels, at most kMaxSuperTile).
constexpr int kMaxCodes = kMaxSuperTile / 32;

// Slot of (level, band, ix, iy) inside a 2^L x 2^L tile (m = L - level).
__host__ __device__ inline int tile_slot(int L, int lev, int band, int ix, int iy) {
  const int m = L - lev;
  return (band << (2 * m)) + (iy << m) + ix;
}

// Inverse of tile_slot.
__host__ __device__ inline void slot_decode(int L, int slot, int* lev, int* band, int* ix, int* iy) {
  if (slot == 0) { *lev = L; *band = 0; *ix = 0; *iy = 0; return; }
  int m = 0;
  while ((4 << (2 * m)) <= slot) ++m;  // slot in [4^m, 4^(m+1))
  *lev = L - m;
  *band = slot >> (2 * m);
  const int rem = slot & ((1 << (2 * m)) - 1);
  *iy = rem >> m;
  *ix = rem & ((1 << m) - 1);
}

// Mallat linear index (row * W + col) of a window coefficient.
__host__ __device__ inline int32_t mallat_index(int W, int L, int tx, int ty, int slot) {
  int lev, band, ix, iy;
  slot_decode(L, slot, &lev, &band, &ix, &iy);
  const int m = L - lev;
  const int p = (tx << m) + ix, q = (ty << m) + iy;
  const int S = W >> lev;
  int row = q, col = p;
  if (band == 1) col += S;
  else if (band == 2) row += S;
  else if (band == 3) { row += S; col += S; }
  return row * W + col;
}

struct DepthMeta {
  int tlo, thi;   // window-tile bounding box of the PSF disk (same on both axes)
  int base, cap;  // first entry and capacity in the LUT arrays
};

struct LutView {
  int D, W, L, nwt, dtype;
  const uint32_t* pos;
  const float2* val;      // FP32 values
  const uint32_t* val16;  // FP16 / BF16 pairs (low half = re)
  const float* scale;     // one per 32 entries (index e >> 5)
  const int32_t* tile_off;
  const DepthMeta* meta;
  const float* cmax;      // largest |re| or |im| of any kept coefficient
  int lmin;               // finest level with a kept coefficient
  const uint2* code;      // records for the launch's super-tile width: plane code (see
                          // plane_code) and value word (FP32 real part or FP16 / BF16 pair)
};

// ------------------------------------------------------------------ launchers
// Each returns the launch error (cudaSuccess when enqueued).

// LUT build: PSF + forward Haar per window tile (coef: D x W*W tile-major), the
// per-depth nonzero count (nnz, zeroed by the caller) and then selection,
// counting, scanning and scattering into the LUT arrays.
struct LutBuildArgs {
  int D, W, L, nwt, dtype;
  int max_nb;               // largest per-depth box side (tiles)
  long long max_cap;        // largest per-depth capacity (entries)
  double lambda, pitch;
  const double* z_dev;      // D depths
  const double* c_dev;      // D values (z / lambda)^2
  const int* psf_blk0;      // D + 1: first PSF block of each depth (prefix over depths)
  int psf_blocks;           // PSF blocks over all depths
  double q;                 // (pitch / lambda)^2
  const double* R2_dev;     // D squared radii (pixels^2)
  const long long* target_dev;  // D budgets (LLONG_MAX = keep all nonzero)
  float2* coef;             // scratch D * W * W
  unsigned long long* keys; // scratch D * W * W: FP64 bit patterns of re^2 + im^2
  unsigned long long* nnz;  // scratch D
  unsigned long long* thr;  // scratch D x 2 selection descriptors
  int* tile_cnt;            // scratch D * nwt * nwt
  long long* nr_dev;        // out D
  uint32_t* pos;
  float2* val;
  uint32_t* val16;
  float* scale;
  int32_t* tile_off;
  const DepthMeta* meta;
  float* cmax;              // out: largest |re| or |im| kept (zeroed by caller)
  unsigned* levels;         // out: bit l set if a level-l coefficient is kept (zeroed by caller)
  uint2* code;              // out: ncode x total records (plane code, value word)
  int ncode;
  int code_k[kMaxCodes];    // super-tile width (tiles) of each code array
  long long total;          // LUT entries (all depths' capacities)
  int* status;
  int wavelet;              // WASABI_HAAR or WASABI_COIF1
  float ctap_lo[6], ctap_hi[6];  // coiflet analysis filters, taps k = -2 .. 3
  float2* img;              // coiflet scratch D * W * W: PSF, then its Mallat transform
  // PSF values on one octant: the PSF depends on n = du^2 + dv^2 alone, so
  // depth d's values for 0 <= dv <= du <= tri_rd[d] are computed once, at
  // tri[tri_off[d] + du (du + 1) / 2 + dv], and every pixel reads them.
  float2* tri;
  const long long* tri_off; // D + 1 prefix
  const int* tri_rd;        // D: floor(R_d)
};
cudaError_t launch_lut_build(const LutBuildArgs& a, cudaStream_t s);

// Order-1 coiflet filters (FP64): scaling filter h_k and wavelet filter
// g_k = (-1)^k h_{1-k}, k = -2 .. 3.
void coif1_filters(double lo[6], double hi[6]);
// Window tiles one PSF block transforms (1,024 threads, one per pixel).
inline int psf_tiles_per_block(int L) {
  const int tsl = 1 << (2 * L);
  return tsl >= 1024 ? 1 : 1024 / tsl;
}

// Points.
cudaError_t launch_quantize(const int32_t* x, const int32_t* y, const double* z, const float* a,
                            int64_t n, double zmin, double zmax, double dz, int D,
                            wasabi_point* out, int* status, cudaStream_t s);

// ------------------------------------------------------------------- batches
// A batch is a table of holograms ("jobs") processed by one fixed-shape
// launch sequence: zero -> count -> scan -> scatter (binning) -> superpose ->
// inverse.  Everything that varies between batches lives in device memory
// (the job table and the BatchDev totals), so the sequence can be captured
// once in a CUDA graph and replayed; a single hologram is a batch of one.
constexpr int kMaxJobs = 1024;

// One inverse Haar step (Sec. 1, step 3; the transpose of the forward step),
// picking output (ax, ay) of the 2x2 block:
//   x00 = ((s + LH) + (HL + HH)) / 2     x01 = ((s - LH) + (HL - HH)) / 2
//   x10 = ((s + LH) - (HL + HH)) / 2     x11 = ((s - LH) - (HL - HH)) / 2
__device__ __forceinline__ float ipick1(float s, float lh, float hl, float hh, int ax, int ay) {
  const float t1 = ax ? s - lh : s + lh;
  const float t2 = ax ? hl - hh : hl + hh;
  return (ay ? t1 - t2 : t1 + t2) * 0.5f;
}
__device__ __forceinline__ float2 ipick(float2 s, float2 lh, float2 hl, float2 hh, int ax, int ay) {
  return make_float2(ipick1(s.x, lh.x, hl.x, hh.x, ax, ay), ipick1(s.y, lh.y, hl.y, hh.y, ax, ay));
}

// Reference wave of the binarisation (Sec. 2): a unit point source at plane
// pixel coordinates (x, y) and signed distance z,
// R = exp(i sgn(z) 2 pi t), t = r / lambda = sqrt(a2 ((i - x)^2 + (j - y)^2) + c)
// with a2 = (pitch / lambda)^2 and c = (z / lambda)^2; bit = Re(u conj R) > 0.
// kind 0 is the unit plane wave R = 1 (nothing below is evaluated).
struct RefDev {
  int kind;
  float sgn;   // sign of z
  float a2f;   // a2 in FP32
  float pad;
  double x, y, a2, c;
};

// Phase of R at an anchor pixel (X, Y) of the plane: frac(t) from an FP64
// reduction, t and the offsets from the source in FP32.
struct RefAnchor {
  float f0, t0, ex, ey;
};
__device__ __forceinline__ RefAnchor ref_anchor(const RefDev& r, long long X, long long Y) {
  const double ex = (double)X - r.x, ey = (double)Y - r.y;
  const double t = sqrt(fma(r.a2, fma(ex, ex, ey * ey), r.c));
  RefAnchor A;
  A.f0 = (float)(t - floor(t));
  A.t0 = (float)t;
  A.ex = (float)ex;
  A.ey = (float)ey;
  return A;
}

// Phase at pixel (dx, dy) from the anchor, reduced to [0, 1), with the
// first and half second derivatives there: t - t0 = a2 m / (t0 + t) with the
// exact difference of squares m = dx (2 ex + dx) + dy (2 ey + dy) (no
// cancellation), and dt/dx = a2 ex / t, d2t/dx2 = (a2 - (dt/dx)^2) / t,
// d2t/dxdy = -(dt/dx)(dt/dy) / t.  Across a 4 x 4 pixel block the dropped
// third-order term is at most about 100 a2 |grad t| / t^2 cycles: 2e-10 for a
// source 0.4 m away (pitch 1 um, lambda 633 nm), growing as 1 / z^2.
struct RefBlock {
  float phi, gx, gy, hxx, hyy, hxy;
};
__device__ __forceinline__ RefBlock ref_block(const RefDev& r, const RefAnchor& A, int dx, int dy) {
  const float fx = (float)dx, fy = (float)dy;
  const float m = fmaf(fx, fmaf(2.f, A.ex, fx), fy * fmaf(2.f, A.ey, fy));
  const float am = r.a2f * m;
  const float dt = am / (A.t0 + sqrtf(fmaf(A.t0, A.t0, am)));
  const float ph = A.f0 + dt;
  const float it = 1.0f / (A.t0 + dt);
  const float ex = A.ex + fx, ey = A.ey + fy;
  RefBlock B;
  B.phi = ph - floorf(ph);
  B.gx = r.a2f * ex * it;
  B.gy = r.a2f * ey * it;
  B.hxx = 0.5f * (r.a2f - B.gx * B.gx) * it;
  B.hyy = 0.5f * (r.a2f - B.gy * B.gy) * it;
  B.hxy = -B.gx * B.gy * it;
  return B;
}
// Re(u conj R) at offset (i, j) from the block's pixel.
__device__ __forceinline__ float ref_value(const RefBlock& B, float sgn, float2 u, int i, int j) {
  const float fi = (float)i, fj = (float)j;
  float ph = B.phi + fi * fmaf(B.hxx, fi, B.gx) + fj * fmaf(B.hyy, fj, B.gy) + B.hxy * (fi * fj);
  ph -= rintf(ph);
  float sn, cs;
  __sincosf(6.28318530717958648f * ph, &sn, &cs);
  return fmaf(u.x, cs, sgn * u.y * sn);
}

struct JobDev {
  const wasabi_point* pts;  // input points (n)
  wasabi_point* sorted;     // binned points (n), scratch
  int* cnt;                 // ncells + 1 cell counts, scratch (zeroed by zero_kernel)
  int* off;                 // ncells + 1 cell offsets, scratch
  int* cursor;              // ncells scatter cursors, scratch
  float2* wbuf;             // tile-major wavelet buffer (w * h)
  float2* u;                // field output of the fused inverse, complex row-major (or null)
  uint8_t* bits;            // binarised output of the fused inverse, packed bits (or null)
  long long n;              // points
  long long pt0;            // first point of this job in the batch's point numbering
  int w, h, ntx, nty;       // pixels and 2^L x 2^L tiles
  int ncx, ncy;             // binning cells of cell x cell pixels
  int rule;                 // shift rule
  int sp0;                  // first superposition item (super-tile) of this job
  int ncells;               // ncx * ncy
  float amax;               // largest |a| over the job's binned points (zeroed by zero_kernel)
  int ox, oy;               // plane pixel of the hologram's pixel (0, 0) (sub-hologram origin)
  int pad;
  RefDev ref;               // reference wave of the bits
};

struct BatchDev {
  int njobs;
  int nsp;                  // superposition items (super-tiles) over all jobs
  int pad[2];
  long long npts;           // points over all jobs
  int counter;              // superposition work counter (zeroed by zero_kernel)
  unsigned long long timers[6];  // phase cycle counters (profiling builds only)
};

// Index of the job holding `item`: binary search over the jobs' first items.
template <typename T>
__device__ __forceinline__ int job_of(const T* starts, int njobs, T item) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (starts[mid] <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

struct BinArgs {
  JobDev* jobs;             // device job table
  BatchDev* batch;          // device totals
  int D;
  int cell;                 // cell side (pixels)
  int reach;                // pixels: a point farther than this outside the hologram is dropped
  int track_amax;           // record each job's largest |a| (superposition uses it)
  int* status;
  int grid;                 // blocks of the grid-stride kernels
};
cudaError_t launch_binning(const BinArgs& b, cudaStream_t s);

struct SuperposeArgs {
  LutView lut;
  const JobDev* jobs;
  BatchDev* batch;
  int cell;             // super-tile side T (pixels) == binning cell
  int reach;            // pixels
  int acc_float;        // 0: exact fixed-point accumulation, 1: FP32 atomics
  int re_only;          // 1: accumulate real parts only (every job wants bits alone)
  int has_ref;          // 1: some job binarises against a spherical reference wave
  int rcap;             // passes per window (superpose_range_cap); survivors per batch rcap / 2, at most 1,024
  int* status;
  int threads;          // block size
  int grid;             // SMs: the launch puts as many CTAs on each as fit
};
cudaError_t launch_superpose(const SuperposeArgs& a, cudaStream_t s);
size_t superpose_smem_bytes(int cell, int L, int lmin, int D, bool re_only, int rcap);
// Range capacity for a launch: larger when only real parts are accumulated
// and the freed shared memory still lets two CTAs share an SM.
int superpose_range_cap(int cell, int L, int lmin, int D, bool re_only, int threads);
// The smallest pass capacity a launch may use (shared-memory feasibility checks).
int superpose_min_range_cap();
// Kinds of superposition launch, for the default configuration.
// kConfigShared: the configuration batches use, and every call on a hologram
// below kConfigLargeSide pixels a side (so such a call and a batch job give
// the same fixed-point results).
constexpr int kConfigComplex = 0, kConfigRe = 1, kConfigRef = 2, kConfigShared = 3;
constexpr int kConfigLargeSide = 8192;
void superpose_default_config(int L, int lmin, int D, int kind, int* cell, int* threads);

struct InverseArgs {
  const float2* wbuf;       // tile-major wavelet buffer
  float2* u;                // complex output (or null)
  uint8_t* bits;            // packed bits output (or null)
  int w, h, ntx;            // pixels; 2^L x 2^L tiles per row
  int nstrips;              // work items: strips of 256 pixels x 2^L rows
  int L;
  int* status;
  int num_sms;
  int ox, oy;               // plane pixel of the output's pixel (0, 0)
  RefDev ref;               // reference wave of the bits
  long long wait_limit;     // clock cycles a stage wait may take before E_TIMEOUT
  long long skip_item;      // test only: strip whose copy is never issued (-1: none)
};
// Default bound on one stage wait of the inverse kernel (about 2 s).
constexpr long long kInverseWaitCycles = 4000000000ll;
cudaError_t launch_inverse(const InverseArgs& a, cudaStream_t s);
// Strips of one hologram as the inverse kernel cuts it (256 pixels x 2^L rows).
int inverse_strips(int w, int h, int L);

// Writes one job and the batch totals of a one-job batch into device memory.
cudaError_t launch_init_single(const JobDev& job, JobDev* jobs_dev, BatchDev* batch_dev, int nsp, cudaStream_t s);
cudaError_t launch_haar_forward(const float2* u, int w, int h, int L, float2* wbuf, cudaStream_t s);
cudaError_t launch_wbuf_to_mallat(const float2* wbuf, int w, int h, int L, float2* out,
                                  cudaStream_t s);

struct DirectArgs {
  double lambda, pitch;
  const JobDev* jobs;   // one job: its binned points and cells
  int cell;
  int w, h;
  int D;
  const double* beta_dev;     // D: (z_d / lambda)^2
  const long long* nlim_dev;  // D: ceil(R_d^2) (aperture) or LLONG_MAX
  double alpha;               // (pitch / lambda)^2
  int reach;
  int* counter;               // zeroed by caller
  float2* u;
  int* status;
  int grid;
};
cudaError_t launch_direct(const DirectArgs& a, cudaStream_t s);

// Status word helpers (abi.cu).
int* device_status_ptr();
void set_error(const char* fmt, ...);

}  // namespace wsb
