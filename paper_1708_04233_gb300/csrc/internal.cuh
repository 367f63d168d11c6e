// Internal declarations shared by the libwasabi translation units.
//
// Layout notes (the public contract is in include/wasabi.h):
//  * LUT entries, per depth d, live at [meta[d].base, meta[d].base + nr[d]) of
//    the pos/val arrays, ordered by window tile (row-major) and then by in-tile
//    slot.  tile_off[d * (nwt*nwt + 1) + t] is the absolute index of window
//    tile t's first entry; entry t + 1 is its end.
//  * pos packs the coefficient's window sub-band position p:12 | q:12 (in
//    units of its level) | level:3 | band:2 (see pack_pos); its window tile is
//    (p >> (L - level), q >> (L - level)).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/wasabi.h"

namespace wsb {

constexpr int kMaxDepths = 4096;
constexpr int kMaxLevels = 5;
constexpr int kMaxWindowTiles = 512;  // window / 2^levels

__host__ __device__ inline uint32_t pack_pos(int p, int q, int lev, int band) {
  return (uint32_t)p | ((uint32_t)q << 12) | ((uint32_t)lev << 24) | ((uint32_t)band << 27);
}

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
  int* status;
};
cudaError_t launch_lut_build(const LutBuildArgs& a, cudaStream_t s);

// Points.
cudaError_t launch_quantize(const int32_t* x, const int32_t* y, const double* z, const float* a,
                            int64_t n, double zmin, double zmax, double dz, int D,
                            wasabi_point* out, int* status, cudaStream_t s);

struct BinArgs {
  const wasabi_point* pts;
  int64_t n;
  int D;
  int w, h;        // hologram pixels
  int cell;        // cell side (pixels)
  int ncx, ncy;
  int reach;       // pixels: a point farther than this outside the hologram is dropped
  int* cnt;        // ncells + 1 (zeroed here)
  float* amax;     // largest |a| of the binned points (zeroed by caller)
  int* off;        // ncells + 1
  int* cursor;     // ncells
  wasabi_point* sorted;
  int* status;
};
cudaError_t launch_binning(const BinArgs& b, cudaStream_t s);

struct SuperposeArgs {
  LutView lut;
  const wasabi_point* sorted;
  const int* cell_off;
  int ncx, ncy, cell;   // cell == super-tile side T (pixels)
  int w, h, ntx, nty;
  int rule;
  int reach;            // pixels
  int* counter;         // zeroed by caller
  const float* amax;    // largest |a| of the binned points
  int acc_float;        // 0: exact fixed-point accumulation, 1: FP32 atomics
  unsigned long long* timers;  // 6 phase cycle counters (profiling builds only)
  float2* wbuf;
  int* status;
  int threads;          // block size
  int grid;             // SMs: the launch puts as many CTAs on each as fit
  long long nst;        // super-tiles
};
cudaError_t launch_superpose(const SuperposeArgs& a, cudaStream_t s);
size_t superpose_smem_bytes(int cell, int L, int lmin, int D);
int superpose_default_cell(int L, int lmin, int D);

cudaError_t launch_inverse(const float2* wbuf, int w, int h, int L, float2* u, uint8_t* bits,
                           int* status, int num_sms, cudaStream_t s);
cudaError_t launch_haar_forward(const float2* u, int w, int h, int L, float2* wbuf, cudaStream_t s);
cudaError_t launch_wbuf_to_mallat(const float2* wbuf, int w, int h, int L, float2* out,
                                  cudaStream_t s);

struct DirectArgs {
  double lambda, pitch;
  const wasabi_point* sorted;
  const int* cell_off;
  int ncx, ncy, cell;
  int w, h;
  int D;
  const double* beta_dev;     // D: (z_d / lambda)^2
  const long long* nlim_dev;  // D: ceil(R_d^2) (aperture) or LLONG_MAX
  double alpha;               // (pitch / lambda)^2
  int reach;
  int* counter;
  float2* u;
  int* status;
  int grid;
};
cudaError_t launch_direct(const DirectArgs& a, cudaStream_t s);

// Status word helpers (abi.cu).
int* device_status_ptr();
void set_error(const char* fmt, ...);

}  // namespace wsb
