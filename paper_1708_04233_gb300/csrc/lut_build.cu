// LUT builder (Sec. 1, step 1 "pre-computation"): per depth, the PSF on a
// W x W window, its L-level orthonormal Haar transform and the N_r strongest
// coefficients, compacted into a per-depth, window-tile-binned table.
//
// Work is confined to the window tiles that meet the PSF disk (the per-depth
// bounding box meta[d].tlo..thi): every coefficient of a tile outside it is 0
// because a tile's Haar coefficients depend only on that tile's pixels.
//
// Kernels (all on one stream):
//   psf_haar_kernel   one block per (bbox tile group, depth): PSF pixels, then
//                     the tile's Haar levels in shared memory (FP32, fixed
//                     operation order, no contraction) -> coef scratch, nnz
//   select_kernel     one cluster of 8 blocks per depth: exact top-N_r of
//                     key = re^2 + im^2 (FP64 bit patterns, MSB radix select,
//                     histograms summed over distributed shared memory),
//                     equal keys resolved by Mallat index (radix select on
//                     the index)
//   tile_count_kernel one warp per window tile: kept count
//   tile_scan_kernel  one block per depth: tile offsets (CSR)
//   scatter_kernel    one warp per window tile: ordered compaction
//   encode_kernel     one warp per 32 entries: FP16/BF16 + FP32 scale
#include <algorithm>

#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.cuh"

namespace wsb {
namespace {

// cos and sin of 2*pi*g, g in [0, 1], FP32.  Quadrant reduction: q = nearest
// integer of 4g, y = g - q/4 (exact), x = 2*pi*y in [-pi/4, pi/4]; Taylor
// series of sin to x^9 and cos to x^10 in Horner form with fused multiply-adds
// (range reduction + polynomial, J.-M. Muller, "Elementary Functions").  Every
// operation is an explicitly rounded intrinsic so the result is a fixed
// function of g.
__device__ __forceinline__ void sincos2pi(float g, float* c_out, float* s_out) {
  constexpr float two_pi = 6.28318530717958647692f;
  constexpr float S3 = -1.0f / 6.0f, S5 = 1.0f / 120.0f, S7 = -1.0f / 5040.0f,
                  S9 = 1.0f / 362880.0f;
  constexpr float C2 = -1.0f / 2.0f, C4 = 1.0f / 24.0f, C6 = -1.0f / 720.0f,
                  C8 = 1.0f / 40320.0f, C10 = -1.0f / 3628800.0f;
  const float q = rintf(__fmul_rn(4.0f, g));
  const float y = __fsub_rn(g, __fmul_rn(0.25f, q));
  const float x = __fmul_rn(y, two_pi);
  const float x2 = __fmul_rn(x, x);
  float ps = __fmaf_rn(x2, S9, S7);
  ps = __fmaf_rn(x2, ps, S5);
  ps = __fmaf_rn(x2, ps, S3);
  const float sn = __fmaf_rn(__fmul_rn(x, x2), ps, x);
  float pc = __fmaf_rn(x2, C10, C8);
  pc = __fmaf_rn(x2, pc, C6);
  pc = __fmaf_rn(x2, pc, C4);
  pc = __fmaf_rn(x2, pc, C2);
  const float cs = __fmaf_rn(x2, pc, 1.0f);
  switch (((int)q) & 3) {
    case 0: *c_out = cs;  *s_out = sn;  break;
    case 1: *c_out = -sn; *s_out = cs;  break;
    case 2: *c_out = -cs; *s_out = -sn; break;
    default: *c_out = sn; *s_out = -cs; break;
  }
}

__device__ __forceinline__ float haar_s(float a, float b, float c, float d) {
  return __fmul_rn(__fadd_rn(__fadd_rn(a, b), __fadd_rn(c, d)), 0.5f);
}
__device__ __forceinline__ float haar_lh(float a, float b, float c, float d) {
  return __fmul_rn(__fadd_rn(__fsub_rn(a, b), __fsub_rn(c, d)), 0.5f);
}
__device__ __forceinline__ float haar_hl(float a, float b, float c, float d) {
  return __fmul_rn(__fsub_rn(__fadd_rn(a, b), __fadd_rn(c, d)), 0.5f);
}
__device__ __forceinline__ float haar_hh(float a, float b, float c, float d) {
  return __fmul_rn(__fsub_rn(__fsub_rn(a, b), __fsub_rn(c, d)), 0.5f);
}

__device__ __forceinline__ unsigned long long key_bits(float2 c) {
  const double k = __dadd_rn(__dmul_rn((double)c.x, (double)c.x), __dmul_rn((double)c.y, (double)c.y));
  return (unsigned long long)__double_as_longlong(k);
}

// Window tile i (row-major) of depth d's bounding box.
struct BoxIter {
  int tlo, nb, L, nwt;
  __device__ __forceinline__ void tile(int i, int* tx, int* ty) const {
    *tx = tlo + i % nb;
    *ty = tlo + i / nb;
  }
  __device__ __forceinline__ long long coef_index(int tx, int ty, int slot) const {
    return (((long long)ty * nwt + tx) << (2 * L)) + slot;
  }
};

// PSF value at offset (du, dv) from the window centre: exp(i 2 pi r / lambda)
// on the open disk n < R^2 and the centre pixel, 0 elsewhere; conjugate for a
// depth behind the plane.
__device__ __forceinline__ float2 psf_pixel(const LutBuildArgs& a, int d, long long du, long long dv) {
  float2 val = make_float2(0.f, 0.f);
  const long long n = du * du + dv * dv;
  if (n == 0 || (double)n < a.R2_dev[d]) {  // the open disk and the centre pixel
    // r / lambda = sqrt(s), s = n (p/lambda)^2 + (z/lambda)^2: FP32 square
    // root plus one FP64 Newton step (residual by a fused multiply-add).
    const double s = __fma_rn((double)n, a.q, a.c_dev[d]);
    const float t0f = __fsqrt_rn(__double2float_rn(s));
    const double t0 = (double)t0f;
    const double res = __fma_rn(-t0, t0, s);
    const float inv = __frcp_rn(2.0f * t0f);
    // s = 0 (a point on the plane, at its own pixel): t = 0.
    const double t = t0f > 0.0f ? __dadd_rn(t0, __dmul_rn(res, (double)inv)) : 0.0;
    const double f = __dsub_rn(t, floor(t));
    sincos2pi(__double2float_rn(f), &val.x, &val.y);
    if (a.z_dev[d] < 0.0) val.y = -val.y;  // behind the plane: the conjugate PSF
  }
  return val;
}

// The octant table: entry i of depth d is (du, dv) with du (du + 1) / 2 + dv = i,
// 0 <= dv <= du, holding psf_pixel(d, du, dv).
__global__ void psf_table_kernel(LutBuildArgs a) {
  const long long n = a.tri_off[a.D];
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += stride) {
    int lo = 0, hi = a.D - 1;  // depth: last d with tri_off[d] <= g
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (__ldg(&a.tri_off[mid]) <= g) lo = mid; else hi = mid - 1;
    }
    const int d = lo;
    const long long i = g - a.tri_off[d];
    long long u = (long long)((sqrt(8.0 * (double)i + 1.0) - 1.0) * 0.5);
    while (u * (u + 1) / 2 > i) --u;
    while ((u + 1) * (u + 2) / 2 <= i) ++u;
    a.tri[g] = psf_pixel(a, d, u, i - u * (u + 1) / 2);
  }
}

// PSF value at (du, dv) from the octant table (0 outside floor(R), where the
// disk holds no pixel).
__device__ __forceinline__ float2 psf_lookup(const LutBuildArgs& a, int d, long long du, long long dv) {
  const long long x = du < 0 ? -du : du, y = dv < 0 ? -dv : dv;
  const long long hi = x > y ? x : y, lo = x > y ? y : x;
  if (hi > __ldg(&a.tri_rd[d])) return make_float2(0.f, 0.f);
  return a.tri[__ldg(&a.tri_off[d]) + hi * (hi + 1) / 2 + lo];
}

template <int L>
__global__ void __launch_bounds__(1024) psf_haar_kernel(LutBuildArgs a) {
  constexpr int TS = 1 << L;
  constexpr int TSL = TS * TS;
  constexpr int NT = TSL >= 1024 ? TSL : 1024;
  constexpr int TPB = NT / TSL;
  __shared__ float2 sa[TPB][TSL];
  __shared__ float2 sb[TPB][TSL];
  __shared__ float2 co[TPB][TSL];
  __shared__ unsigned int nz;
  // Blocks cover the depths' box tiles back to back (no idle blocks): the
  // block's depth by binary search over the per-depth first blocks.
  int dlo = 0, dhi = a.D - 1;
  while (dlo < dhi) {
    const int mid = (dlo + dhi + 1) >> 1;
    if (__ldg(&a.psf_blk0[mid]) <= (int)blockIdx.x) dlo = mid; else dhi = mid - 1;
  }
  const int d = dlo;
  const DepthMeta md = a.meta[d];
  const int nb = md.thi - md.tlo + 1;
  const int tl = threadIdx.x / TSL, pix = threadIdx.x % TSL;
  const int bt = ((int)blockIdx.x - __ldg(&a.psf_blk0[d])) * TPB + tl;  // tile index inside the box
  const bool valid = bt < nb * nb;
  const int tx = md.tlo + (valid ? bt % nb : 0), ty = md.tlo + (valid ? bt / nb : 0);
  if (threadIdx.x == 0) nz = 0;

  // PSF pixel (Eq. (1) PSF with the circular aperture of step 1).
  const int pu = pix % TS, pv = pix / TS;
  const float2 val = valid ? psf_lookup(a, d, (long long)(tx * TS + pu) - a.W / 2, (long long)(ty * TS + pv) - a.W / 2)
                           : make_float2(0.f, 0.f);
  sa[tl][pix] = val;
  __syncthreads();

  float2* cur = sa[tl];
  float2* nxt = sb[tl];
#pragma unroll
  for (int l = 1; l <= L; ++l) {
    const int S = TS >> (l - 1), h = S >> 1, m = L - l;
    if (pix < h * h) {
      const int i = pix / h, j = pix % h;
      const float2 x00 = cur[(2 * i) * TS + 2 * j], x01 = cur[(2 * i) * TS + 2 * j + 1];
      const float2 x10 = cur[(2 * i + 1) * TS + 2 * j], x11 = cur[(2 * i + 1) * TS + 2 * j + 1];
      nxt[i * TS + j] = make_float2(haar_s(x00.x, x01.x, x10.x, x11.x), haar_s(x00.y, x01.y, x10.y, x11.y));
      co[tl][(1 << (2 * m)) + (i << m) + j] =
          make_float2(haar_lh(x00.x, x01.x, x10.x, x11.x), haar_lh(x00.y, x01.y, x10.y, x11.y));
      co[tl][(2 << (2 * m)) + (i << m) + j] =
          make_float2(haar_hl(x00.x, x01.x, x10.x, x11.x), haar_hl(x00.y, x01.y, x10.y, x11.y));
      co[tl][(3 << (2 * m)) + (i << m) + j] =
          make_float2(haar_hh(x00.x, x01.x, x10.x, x11.x), haar_hh(x00.y, x01.y, x10.y, x11.y));
    }
    __syncthreads();
    float2* tmp = cur; cur = nxt; nxt = tmp;
  }
  if (pix == 0) co[tl][0] = cur[0];
  __syncthreads();
  const float2 c = co[tl][pix];
  const bool nzc = c.x != 0.f || c.y != 0.f;
  if (valid) {
    const long long ci = (long long)d * a.W * a.W + (((long long)ty * a.nwt + tx) << (2 * L)) + pix;
    a.coef[ci] = c;
    a.keys[ci] = nzc ? key_bits(c) : 0ull;  // computed once: FP64 is scarce on this part
  }
  const unsigned b = __ballot_sync(0xffffffffu, valid && nzc);
  if ((threadIdx.x & 31) == 0 && b) atomicAdd(&nz, (unsigned)__popc(b));
  __syncthreads();
  if (threadIdx.x == 0 && nz) atomicAdd(&a.nnz[d], (unsigned long long)nz);
}

// Block-wide exclusive scan of one unsigned per thread (blockDim.x = 1024).
__device__ unsigned block_excl_scan(unsigned v, unsigned* total) {
  __shared__ unsigned warp_sum[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sum[wid] = x;
  __syncthreads();
  if (wid == 0) {
    unsigned w = warp_sum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    warp_sum[lane] = w;  // inclusive
  }
  __syncthreads();
  const unsigned before = (wid ? warp_sum[wid - 1] : 0u) + x - v;
  if (total) *total = warp_sum[31];
  __syncthreads();
  return before;
}

// ---- Order-1 coiflet (periodic filter banks on the whole window) --------
// The transform is not tile-local, so the PSF of every depth is written out
// over the whole window (img, row-major), transformed level by level in
// place (analysis along x into coef as scratch, then along y back into img),
// and gathered into the tile-major coefficient order the rest of the build
// uses.  Sum order of every output: the k = -2 product, then fused
// multiply-adds for k = -1 .. 3 (the oracle's order, so that selections match).

__global__ void psf_plain_kernel(LutBuildArgs a) {
  const long long WW = (long long)a.W * a.W, n = WW * a.D;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int d = (int)(i / WW);
    const long long p = i - (long long)d * WW;
    const long long v = p / a.W, u = p - v * a.W;
    a.img[i] = psf_lookup(a, d, u - a.W / 2, v - a.W / 2);
  }
}

__device__ __forceinline__ int pmod(int x, int n) { return ((x % n) + n) % n; }

// One analysis step of 6 taps over x[(2m + k) mod S], k = -2 .. 3, at
// stride `step` (1: along a row, W: down a column).
__device__ __forceinline__ int coif_wrap(int x, int S) {
  if (S < 8) return pmod(x, S);  // taps may wrap more than once
  return x < 0 ? x + S : (x >= S ? x - S : x);
}
__device__ __forceinline__ void coif_analyse(const LutBuildArgs& a, const float2* base, long long step, int S, int m,
                                             float2* lo, float2* hi) {
  float2 x = base[(long long)coif_wrap(2 * m - 2, S) * step];
  float2 sl = make_float2(__fmul_rn(a.ctap_lo[0], x.x), __fmul_rn(a.ctap_lo[0], x.y));
  float2 sh = make_float2(__fmul_rn(a.ctap_hi[0], x.x), __fmul_rn(a.ctap_hi[0], x.y));
#pragma unroll
  for (int i = 1; i < 6; ++i) {
    x = base[(long long)coif_wrap(2 * m + i - 2, S) * step];
    sl.x = __fmaf_rn(a.ctap_lo[i], x.x, sl.x);
    sl.y = __fmaf_rn(a.ctap_lo[i], x.y, sl.y);
    sh.x = __fmaf_rn(a.ctap_hi[i], x.x, sh.x);
    sh.y = __fmaf_rn(a.ctap_hi[i], x.y, sh.y);
  }
  *lo = sl;
  *hi = sh;
}

// Along x on the top-left S x S block of each depth: src rows -> dst rows
// (low half, then high half).
__global__ void coif_rows_kernel(LutBuildArgs a, const float2* src, float2* dst, int S) {
  const int d = blockIdx.y, h = S / 2;
  const long long WW = (long long)a.W * a.W;
  const long long n = (long long)S * h;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i / h), m = (int)(i - (long long)r * h);
    const long long row = (long long)d * WW + (long long)r * a.W;
    float2 lo, hi;
    coif_analyse(a, src + row, 1, S, m, &lo, &hi);
    dst[row + m] = lo;
    dst[row + h + m] = hi;
  }
}

// Along y on the top-left S x S block: src columns -> dst columns (low half
// on top).  Consecutive threads take consecutive columns.
__global__ void coif_cols_kernel(LutBuildArgs a, const float2* src, float2* dst, int S) {
  const int d = blockIdx.y, h = S / 2;
  const long long WW = (long long)a.W * a.W;
  const long long n = (long long)S * h;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int m = (int)(i / S), col = (int)(i - (long long)m * S);
    const long long base = (long long)d * WW + col;
    float2 lo, hi;
    coif_analyse(a, src + base, a.W, S, m, &lo, &hi);
    dst[base + (long long)m * a.W] = lo;
    dst[base + (long long)(h + m) * a.W] = hi;
  }
}

// Mallat image -> tile-major coefficients, selection keys and nonzero counts.
__global__ void __launch_bounds__(256) coif_gather_kernel(LutBuildArgs a) {
  const int d = blockIdx.y;
  const long long WW = (long long)a.W * a.W;
  const int tsl = 1 << (2 * a.L);
  unsigned nz = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < WW; i += (long long)gridDim.x * blockDim.x) {
    const int tile = (int)(i >> (2 * a.L)), slot = (int)(i & (tsl - 1));
    const int tx = tile % a.nwt, ty = tile / a.nwt;
    const float2 c = a.img[(long long)d * WW + mallat_index(a.W, a.L, tx, ty, slot)];
    const bool nzc = c.x != 0.f || c.y != 0.f;
    a.coef[(long long)d * WW + i] = c;
    a.keys[(long long)d * WW + i] = nzc ? key_bits(c) : 0ull;
    nz += nzc ? 1u : 0u;
  }
  for (int o = 16; o > 0; o >>= 1) nz += __shfl_xor_sync(0xffffffffu, nz, o);
  if ((threadIdx.x & 31) == 0 && nz) atomicAdd(&a.nnz[d], (unsigned long long)nz);
}

cudaError_t launch_coif_forward(const LutBuildArgs& a, cudaStream_t s) {
  psf_plain_kernel<<<1024, 256, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  for (int l = 1; l <= a.L && e == cudaSuccess; ++l) {
    const int S = a.W >> (l - 1);
    const long long n = (long long)S * (S / 2);
    const dim3 grid((unsigned)std::min<long long>((n + 255) / 256, 4096), (unsigned)a.D);
    coif_rows_kernel<<<grid, 256, 0, s>>>(a, a.img, a.coef, S);
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    coif_cols_kernel<<<grid, 256, 0, s>>>(a, a.coef, a.img, S);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return e;
  const long long WW = (long long)a.W * a.W;
  const dim3 g((unsigned)std::min<long long>((WW + 255) / 256, 4096), (unsigned)a.D);
  coif_gather_kernel<<<g, 256, 0, s>>>(a);
  return cudaGetLastError();
}

constexpr int kModeGE = 0;   // keep key_bits >= T
constexpr int kModeTie = 1;  // keep key_bits > T, or == T with Mallat index <= I*

constexpr int kCandCap = 2048;   // candidates moved to shared memory
constexpr int kSelCluster = 8;   // CTAs per depth (one thread-block cluster)
constexpr int kDigit = 11;       // bits per radix pass
constexpr int kBins = 1 << kDigit;

// One thread-block cluster of kSelCluster CTAs per depth.  thr[2d] = T,
// thr[2d+1] = (mode << 32) | I*.  MSB-first radix select over the FP64 key
// bit patterns (keys are >= 0, so their bit patterns order like the values),
// 11 bits per pass: each CTA histograms its share of the depth's window tiles
// in its own shared memory, and every CTA sums the cluster's histograms
// through distributed shared memory, so all of them take the same decision.
// Once the bucket holding the threshold has at most kCandCap members, the
// CTAs copy them (with their Mallat indices) into the first CTA's shared
// memory and the others leave; the remaining passes run there.  Equal keys at
// the threshold are resolved by a radix select on the 32-bit Mallat index
// (ascending).
__global__ void __cluster_dims__(kSelCluster, 1, 1) __launch_bounds__(1024) select_kernel(LutBuildArgs a) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  __shared__ unsigned hist[kBins];   // this CTA's counts (read by the whole cluster)
  __shared__ unsigned tot[kBins];    // the cluster's sums
  __shared__ unsigned long long ckey[kCandCap];
  __shared__ unsigned cmi[kCandCap];
  __shared__ int s_found, s_nc;
  __shared__ unsigned s_cum;
  const int crank = (int)cluster.block_rank();
  const bool leader = crank == 0;
  const int d = blockIdx.x / kSelCluster;
  const DepthMeta md = a.meta[d];
  const int nb = md.thi - md.tlo + 1;
  const BoxIter it{md.tlo, nb, a.L, a.nwt};
  const int ntb = nb * nb, tsl = 1 << (2 * a.L);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int t0 = crank * nwarps + warp, tstride = kSelCluster * nwarps;  // this warp's tiles
  const unsigned long long* kd = a.keys + (long long)d * a.W * a.W;
  const long long nnz = (long long)a.nnz[d];
  const long long k = min(nnz, a.target_dev[d]);
  if (leader && threadIdx.x == 0) a.nr_dev[d] = k;
  if (k == nnz || k <= 0) {  // the same for every CTA of the cluster
    if (leader && threadIdx.x == 0) {
      a.thr[2 * d] = k == nnz ? 1ull : ~0ull;  // 1: any nonzero key; ~0: none
      a.thr[2 * d + 1] = (unsigned long long)kModeGE << 32;
    }
    return;
  }
  auto fail = [&]() {  // counts inconsistent with nnz: keep nothing, report
    if (leader && threadIdx.x == 0) {
      a.thr[2 * d] = ~0ull;
      a.thr[2 * d + 1] = (unsigned long long)kModeGE << 32;
      a.nr_dev[d] = 0;
      atomicCAS(a.status, 0, WASABI_E_RANGE);
    }
  };
  // Threads own kBins / 1024 consecutive bins each.
  constexpr int BPT = kBins / 1024;
  // After the counts of a pass are in hist (and, with `shared`, in every CTA
  // of the cluster): the bin holding the rem-th element, counted from the top
  // bin down (desc) or from bin 0 up; -1 if none.  tot receives the totals.
  auto find_bin = [&](bool shared, bool desc, unsigned rem_) -> int {
    if (shared) cluster.sync();  // every CTA's counts complete
    unsigned v[BPT], local = 0;
    const int t = desc ? 1023 - (int)threadIdx.x : (int)threadIdx.x;
#pragma unroll
    for (int j = 0; j < BPT; ++j) {
      const int b = BPT * t + j;
      unsigned c = hist[b];
      if (shared)
        for (int r = 0; r < kSelCluster; ++r)
          if (r != crank) c += cluster.map_shared_rank(hist, r)[b];
      v[j] = c;
      tot[b] = c;
      local += c;
    }
    if (threadIdx.x == 0) s_found = -1;
    unsigned cum = block_excl_scan(local, nullptr);
#pragma unroll
    for (int jj = 0; jj < BPT; ++jj) {
      const int j = desc ? BPT - 1 - jj : jj;
      if (cum < rem_ && rem_ <= cum + v[j]) { s_found = BPT * t + j; s_cum = cum; }
      cum += v[j];
    }
    __syncthreads();
    if (shared) cluster.sync();  // nobody zeroes hist while another CTA reads it
    return s_found;
  };
  auto zero_hist = [&]() {
    for (int i = threadIdx.x; i < kBins; i += blockDim.x) hist[i] = 0;
    __syncthreads();
  };

  unsigned long long prefix = 0, hi_mask = 0;
  unsigned rem = (unsigned)k;
  int shift = 64, nc = 0;
  bool done = false, in_list = false;
  while (shift > 0 && !done) {
    const int width = shift >= kDigit ? kDigit : shift;
    shift -= width;
    const unsigned nbins = 1u << width;
    zero_hist();
    if (in_list) {
      for (int i = threadIdx.x; i < nc; i += blockDim.x) {
        const unsigned long long kb = ckey[i];
        if ((kb & hi_mask) == prefix) atomicAdd(&hist[(kb >> shift) & (nbins - 1)], 1u);
      }
    } else {
      // Eight loads in flight per lane before any is used.
      for (int ti = t0; ti < ntb; ti += tstride) {
        int tx, ty;
        it.tile(ti, &tx, &ty);
        const unsigned long long* kt = kd + it.coef_index(tx, ty, 0);
        for (int slot0 = 0; slot0 < tsl; slot0 += 256) {
          unsigned long long kb[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int slot = slot0 + lane + 32 * j;
            kb[j] = slot < tsl ? __ldg(&kt[slot]) : 0ull;
          }
#pragma unroll
          for (int j = 0; j < 8; ++j)
            if (kb[j] != 0 && (kb[j] & hi_mask) == prefix) atomicAdd(&hist[(kb[j] >> shift) & (nbins - 1)], 1u);
        }
      }
    }
    __syncthreads();
    // Bins above nbins are empty: counting from the top of kBins is the same.
    const int found = find_bin(!in_list, true, rem);
    if (found < 0) { fail(); return; }
    const unsigned bstar = (unsigned)found;
    const unsigned cnt_b = tot[bstar];
    rem -= s_cum;
    prefix |= (unsigned long long)bstar << shift;
    hi_mask |= (unsigned long long)(nbins - 1) << shift;
    if (cnt_b == rem) {
      done = true;
    } else if (!in_list && cnt_b <= (unsigned)kCandCap && shift > 0) {
      // Gather the bucket into the first CTA's shared memory.
      if (leader && threadIdx.x == 0) s_nc = 0;
      cluster.sync();
      int* nc0 = cluster.map_shared_rank(&s_nc, 0);
      unsigned long long* ckey0 = cluster.map_shared_rank(ckey, 0);
      unsigned* cmi0 = cluster.map_shared_rank(cmi, 0);
      for (int ti = t0; ti < ntb; ti += tstride) {
        int tx, ty;
        it.tile(ti, &tx, &ty);
        const unsigned long long* kt = kd + it.coef_index(tx, ty, 0);
        for (int slot = lane; slot < tsl; slot += 32) {
          const unsigned long long kb = __ldg(&kt[slot]);
          if (kb != 0 && (kb & hi_mask) == prefix) {
            const int i = atomicAdd(nc0, 1);
            if (i < kCandCap) {
              ckey0[i] = kb;
              cmi0[i] = (unsigned)mallat_index(a.W, a.L, tx, ty, slot);
            }
          }
        }
      }
      cluster.sync();  // the list is complete; only the first CTA goes on
      if (!leader) return;
      nc = min(s_nc, kCandCap);
      in_list = true;
    }
    __syncthreads();
  }
  if (done) {
    if (leader && threadIdx.x == 0) {
      a.thr[2 * d] = prefix;
      a.thr[2 * d + 1] = (unsigned long long)kModeGE << 32;
    }
    return;
  }
  // Ties at the exact key T = prefix: the rem lowest Mallat indices among
  // them, 11 bits per pass over the 32-bit index.
  unsigned iprefix = 0, ihi = 0;
  for (int ishift = 2 * kDigit; ishift >= 0; ishift -= kDigit) {
    zero_hist();
    if (in_list) {
      for (int i = threadIdx.x; i < nc; i += blockDim.x) {
        if (ckey[i] != prefix) continue;
        const unsigned mi = cmi[i];
        if ((mi & ihi) == iprefix) atomicAdd(&hist[(mi >> ishift) & (kBins - 1)], 1u);
      }
    } else {
      for (int ti = t0; ti < ntb; ti += tstride) {
        int tx, ty;
        it.tile(ti, &tx, &ty);
        const unsigned long long* kt = kd + it.coef_index(tx, ty, 0);
        for (int slot = lane; slot < tsl; slot += 32) {
          if (kt[slot] != prefix) continue;
          const unsigned mi = (unsigned)mallat_index(a.W, a.L, tx, ty, slot);
          if ((mi & ihi) == iprefix) atomicAdd(&hist[(mi >> ishift) & (kBins - 1)], 1u);
        }
      }
    }
    __syncthreads();
    const int found = find_bin(!in_list, false, rem);
    if (found < 0) { fail(); return; }
    rem -= s_cum;
    iprefix |= (unsigned)found << ishift;
    ihi |= (unsigned)(kBins - 1) << ishift;
    __syncthreads();
  }
  if (leader && threadIdx.x == 0) {
    a.thr[2 * d] = prefix;
    a.thr[2 * d + 1] = ((unsigned long long)kModeTie << 32) | iprefix;
  }
}

__device__ __forceinline__ bool kept(unsigned long long kb, unsigned long long T, unsigned long long aux,
                                     int W, int L, int tx, int ty, int slot) {
  if (kb == 0) return false;
  if ((int)(aux >> 32) == kModeGE) return kb >= T;
  if (kb != T) return kb > T;
  return (unsigned)mallat_index(W, L, tx, ty, slot) <= (unsigned)(aux & 0xffffffffu);
}

// Layout of the kept entries of one depth: window tiles row-major, each
// tile's entries in slot order.  tile_off[d * (nwt*nwt + 1) + t] is the
// absolute index of window tile t's first entry; t = nwt*nwt ends the depth.

// One warp per window tile of the whole grid (tiles outside the box: 0).
__global__ void __launch_bounds__(256) tile_count_kernel(LutBuildArgs a) {
  const int d = blockIdx.y;
  const int tile = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  const int ntile = a.nwt * a.nwt;
  if (tile >= ntile) return;
  const DepthMeta md = a.meta[d];
  const int tx = tile % a.nwt, ty = tile / a.nwt;
  int cnt = 0;
  if (tx >= md.tlo && tx <= md.thi && ty >= md.tlo && ty <= md.thi) {
    const unsigned long long T = a.thr[2 * d], aux = a.thr[2 * d + 1];
    const unsigned long long* kt = a.keys + (long long)d * a.W * a.W + ((long long)tile << (2 * a.L));
    const int tsl = 1 << (2 * a.L);
    for (int j0 = 0; j0 < tsl; j0 += 32) {
      const int slot = j0 + lane;
      bool s = false;
      if (slot < tsl) s = kept(kt[slot], T, aux, a.W, a.L, tx, ty, slot);
      cnt += __popc(__ballot_sync(0xffffffffu, s));
    }
  }
  if (lane == 0) a.tile_cnt[(long long)d * ntile + tile] = cnt;
}

__global__ void __launch_bounds__(1024) tile_scan_kernel(LutBuildArgs a) {
  const int d = blockIdx.x;
  const int ntile = a.nwt * a.nwt;
  const int per = (ntile + 1023) / 1024;
  const int t0 = threadIdx.x * per;
  const int* cnt = a.tile_cnt + (long long)d * ntile;
  int32_t* off = a.tile_off + (long long)d * (ntile + 1);
  unsigned local = 0;
  for (int t = t0; t < min(t0 + per, ntile); ++t) local += (unsigned)cnt[t];
  unsigned total;
  unsigned run = block_excl_scan(local, &total);
  const int base = a.meta[d].base, cap = a.meta[d].cap;
  // Offsets never leave the depth's region, even if the counts were wrong.
  for (int t = t0; t < min(t0 + per, ntile); ++t) {
    off[t] = base + min((int)run, cap);
    run += (unsigned)cnt[t];
  }
  if (threadIdx.x == 0) {
    off[ntile] = base + min((int)total, cap);
    if ((long long)total != a.nr_dev[d]) atomicCAS(a.status, 0, WASABI_E_RANGE);
  }
}

__global__ void __launch_bounds__(256) scatter_kernel(LutBuildArgs a) {
  const int d = blockIdx.y;
  const int tile = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  const int ntile = a.nwt * a.nwt;
  if (tile >= ntile) return;
  const DepthMeta md = a.meta[d];
  const int tx = tile % a.nwt, ty = tile / a.nwt;
  if (tx < md.tlo || tx > md.thi || ty < md.tlo || ty > md.thi) return;
  const unsigned long long T = a.thr[2 * d], aux = a.thr[2 * d + 1];
  const long long cbase = (long long)d * a.W * a.W + ((long long)tile << (2 * a.L));
  int off = a.tile_off[(long long)d * (ntile + 1) + tile];
  const int tsl = 1 << (2 * a.L);
  const unsigned lt = (1u << lane) - 1u;
  float cm = 0.f;
  unsigned levmask = 0;  // levels present among this tile's kept entries
  for (int j0 = 0; j0 < tsl; j0 += 32) {
    const int slot = j0 + lane;
    bool s = false;
    float2 v = make_float2(0.f, 0.f);
    if (slot < tsl) {
      v = a.coef[cbase + slot];
      s = kept(a.keys[cbase + slot], T, aux, a.W, a.L, tx, ty, slot);
    }
    const unsigned b = __ballot_sync(0xffffffffu, s);
    const int e = off + __popc(b & lt);
    if (s && e < md.base + md.cap) {
      int lev, band, ix, iy;
      slot_decode(a.L, slot, &lev, &band, &ix, &iy);
      const int m = a.L - lev;
      a.pos[e] = pack_pos((tx << m) + ix, (ty << m) + iy, lev, band);
      a.val[e] = v;
      cm = fmaxf(cm, fmaxf(fabsf(v.x), fabsf(v.y)));
      levmask |= 1u << lev;
    }
    off += __popc(b);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    cm = fmaxf(cm, __shfl_xor_sync(0xffffffffu, cm, o));
    levmask |= __shfl_xor_sync(0xffffffffu, levmask, o);
  }
  if (lane == 0 && cm > 0.f) atomicMax(reinterpret_cast<int*>(a.cmax), __float_as_int(cm));
  if (lane == 0 && levmask) atomicOr(a.levels, levmask);
}

// One warp per block of 32 consecutive entries of one depth.
__global__ void __launch_bounds__(256) encode_kernel(LutBuildArgs a) {
  const int d = blockIdx.y;
  const long long blk = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  const long long nr = a.nr_dev[d];
  if (blk * 32 >= nr) return;
  const long long e = a.meta[d].base + blk * 32 + lane;
  const bool valid = blk * 32 + lane < nr;
  const float2 v = valid ? a.val[e] : make_float2(0.f, 0.f);
  float m = fmaxf(fabsf(v.x), fabsf(v.y));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  const float s = m > 0.f ? m : 1.f;
  const float qr = __fdiv_rn(v.x, s), qi = __fdiv_rn(v.y, s);
  uint32_t packed;
  if (a.dtype == WASABI_F16S) {
    packed = (uint32_t)__half_as_ushort(__float2half_rn(qr)) |
             ((uint32_t)__half_as_ushort(__float2half_rn(qi)) << 16);
  } else {
    packed = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(qr)) |
             ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(qi)) << 16);
  }
  a.val16[e] = valid ? packed : 0u;
  if (lane == 0) a.scale[e >> 5] = s;
}

// Superposition records of every LUT entry for each super-tile width: the
// plane code (plane_code) and the value word the superposition reads with it
// (FP32 real part, or the FP16 / BF16 pair).
__global__ void plane_code_kernel(LutBuildArgs a) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= a.total) return;
  const uint32_t p = a.pos[e];
  const int c = blockIdx.y;
  const uint32_t data = a.dtype == WASABI_F32 ? __float_as_uint(a.val[e].x) : a.val16[e];
  a.code[c * a.total + e] = make_uint2(plane_code(p, a.L, a.code_k[c]), data);
}

template <int L>
cudaError_t launch_psf_haar(const LutBuildArgs& a, int max_nb, cudaStream_t s) {
  (void)max_nb;
  constexpr int TSL = 1 << (2 * L);
  constexpr int NT = TSL >= 1024 ? TSL : 1024;
  if (a.psf_blocks <= 0) return cudaSuccess;
  psf_haar_kernel<L><<<(unsigned)a.psf_blocks, NT, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_lut_build(const LutBuildArgs& a, cudaStream_t s) {
  // The largest per-depth box sizes the psf grid (smaller boxes idle out).
  const int max_nb = a.max_nb;
  cudaError_t e;
  psf_table_kernel<<<2048, 256, 0, s>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (a.wavelet == WASABI_COIF1) {
    e = launch_coif_forward(a, s);
  } else {
    switch (a.L) {
      case 1: e = launch_psf_haar<1>(a, max_nb, s); break;
      case 2: e = launch_psf_haar<2>(a, max_nb, s); break;
      case 3: e = launch_psf_haar<3>(a, max_nb, s); break;
      case 4: e = launch_psf_haar<4>(a, max_nb, s); break;
      case 5: e = launch_psf_haar<5>(a, max_nb, s); break;
      default: return cudaErrorInvalidValue;
    }
  }
  if (e != cudaSuccess) return e;
  select_kernel<<<a.D * kSelCluster, 1024, 0, s>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int ntile = a.nwt * a.nwt;
  const dim3 tgrid((unsigned)((ntile + 7) / 8), (unsigned)a.D);
  tile_count_kernel<<<tgrid, 256, 0, s>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  tile_scan_kernel<<<a.D, 1024, 0, s>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  scatter_kernel<<<tgrid, 256, 0, s>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (a.dtype != WASABI_F32) {
    const long long blocks = (a.max_cap + 31) / 32;
    const dim3 egrid((unsigned)((blocks + 7) / 8), (unsigned)a.D);
    encode_kernel<<<egrid, 256, 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (a.ncode > 0 && a.total > 0) {
    const dim3 cgrid((unsigned)((a.total + 255) / 256), (unsigned)a.ncode);
    plane_code_kernel<<<cgrid, 256, 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace wsb
