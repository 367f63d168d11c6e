// Point preparation and spatial binning.
//
// quantize_kernel: depth index per point (Sec. 1, step 1 depth discretisation).
// Binning (count -> scan -> scatter): points are grouped by the cell x cell
// pixel cell that holds them, cells row-major, so that a consumer working on
// one region reads each row of nearby cells as one contiguous range.  Points
// whose footprint cannot reach the hologram (more than `reach` pixels
// outside it) and points with an invalid depth are left out; the latter
// record WASABI_E_RANGE.
#include "internal.cuh"

namespace wsb {
namespace {

__global__ void quantize_kernel(const int32_t* __restrict__ x, const int32_t* __restrict__ y,
                                const double* __restrict__ z, const float* __restrict__ a, int64_t n,
                                double zmin, double zmax, double dz, int D,
                                wasabi_point* __restrict__ out, int* status) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double zi = z[i];
  uint32_t d;
  if (!(zi >= zmin && zi <= zmax)) {
    d = (uint32_t)D;
    atomicCAS(status, 0, WASABI_E_RANGE);
  } else {
    long long k = (long long)floor(__ddiv_rn(__dsub_rn(zi, zmin), dz));
    if (k > D - 1) k = D - 1;
    d = (uint32_t)k;
  }
  wasabi_point p;
  p.x = x[i];
  p.y = y[i];
  p.a = a[i];
  p.d = d;
  out[i] = p;
}

struct CellOf {
  int w, h, cell, ncx, reach, D;
  // Cell of a point, or -1 if the point is left out.
  __device__ __forceinline__ int operator()(const wasabi_point& p) const {
    if (p.d >= (uint32_t)D) return -1;
    if (p.x < -reach || p.x >= w + reach || p.y < -reach || p.y >= h + reach) return -1;
    const int cx = min(max(p.x, 0), w - 1) / cell;
    const int cy = min(max(p.y, 0), h - 1) / cell;
    return cy * ncx + cx;
  }
};

__global__ void count_kernel(BinArgs b, CellOf cf) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= b.n) return;
  const wasabi_point p = b.pts[i];
  if (p.d >= (uint32_t)b.D) atomicCAS(b.status, 0, WASABI_E_RANGE);
  const int c = cf(p);
  if (c >= 0) {
    atomicAdd(&b.cnt[c], 1);
    // Non-negative floats order like their bit patterns.
    if (b.amax) atomicMax(reinterpret_cast<int*>(b.amax), __float_as_int(fabsf(p.a)));
  }
}

// Single-block exclusive scan of ncells counts into off[0..ncells] and
// cursor[0..ncells): chunks of 4096 counts, each thread a coalesced int4,
// one block scan per chunk, a running carry between chunks.
__global__ void __launch_bounds__(1024) scan_kernel(BinArgs b, int ncells) {
  __shared__ unsigned warp_sum[32];
  __shared__ unsigned s_carry;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (int base = 0; base < ncells; base += 4096) {
    const int i0 = base + 4 * threadIdx.x;
    int c[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) c[j] = i0 + j < ncells ? b.cnt[i0 + j] : 0;
    const unsigned local = (unsigned)(c[0] + c[1] + c[2] + c[3]);
    unsigned x = local;
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
      warp_sum[lane] = w;
    }
    __syncthreads();
    const unsigned carry = s_carry;
    unsigned run = carry + (wid ? warp_sum[wid - 1] : 0u) + x - local;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (i0 + j < ncells) {
        b.off[i0 + j] = (int)run;
        b.cursor[i0 + j] = (int)run;
      }
      run += (unsigned)c[j];
    }
    __syncthreads();
    if (threadIdx.x == 0) s_carry = carry + warp_sum[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) b.off[ncells] = (int)s_carry;
}

__global__ void scatter_points_kernel(BinArgs b, CellOf cf) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= b.n) return;
  const wasabi_point p = b.pts[i];
  const int c = cf(p);
  if (c < 0) return;
  const int slot = atomicAdd(&b.cursor[c], 1);
  b.sorted[slot] = p;
}

}  // namespace

cudaError_t launch_quantize(const int32_t* x, const int32_t* y, const double* z, const float* a,
                            int64_t n, double zmin, double zmax, double dz, int D,
                            wasabi_point* out, int* status, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)((n + 255) / 256);
  quantize_kernel<<<grid, 256, 0, s>>>(x, y, z, a, n, zmin, zmax, dz, D, out, status);
  return cudaGetLastError();
}

cudaError_t launch_binning(const BinArgs& b, cudaStream_t s) {
  const int ncells = b.ncx * b.ncy;
  const CellOf cf{b.w, b.h, b.cell, b.ncx, b.reach, b.D};
  cudaError_t e = cudaMemsetAsync(b.cnt, 0, sizeof(int) * (size_t)(ncells + 1), s);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)((b.n + 255) / 256);
  if (b.n > 0) {
    count_kernel<<<grid, 256, 0, s>>>(b, cf);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  scan_kernel<<<1, 1024, 0, s>>>(b, ncells);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (b.n > 0) {
    scatter_points_kernel<<<grid, 256, 0, s>>>(b, cf);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace wsb
