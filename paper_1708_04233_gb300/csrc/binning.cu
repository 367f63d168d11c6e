// Point preparation and spatial binning.
//
// quantize_kernel: depth index per point (Sec. 1, step 1 depth discretisation).
// Binning of a batch of holograms (zero -> count -> scan -> scatter): each
// job's points are grouped by the cell x cell pixel cell that holds them,
// cells row-major, so that a consumer working on one region reads each row of
// nearby cells as one contiguous range.  Points whose footprint cannot reach
// their hologram (more than `reach` pixels outside it) and points with an
// invalid depth are left out; the latter record WASABI_E_RANGE.  All sizes
// are read from the device-side batch tables, so the launch shapes do not
// depend on the batch.
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

__global__ void init_single_kernel(JobDev job, JobDev* jobs, BatchDev* b, int nsp) {
  jobs[0] = job;
  b->njobs = 1;
  b->nsp = nsp;
  b->npts = job.n;
}

// Cell of a point of job J, or -1 if the point is left out.  The point is
// moved into the job's frame first: x'_j = x_j - origin_x, y'_j = y_j - origin_y
// (the sub-hologram coordinate transform of Sec. 1, large-scale step 3).
__device__ __forceinline__ int cell_of(const JobDev& J, wasabi_point& p, int cell, int reach, int D) {
  if (p.d >= (uint32_t)D) return -1;
  const long long lx = (long long)p.x - J.ox, ly = (long long)p.y - J.oy;
  if (lx < -reach || lx >= (long long)J.w + reach || ly < -reach || ly >= (long long)J.h + reach) return -1;
  p.x = (int)lx;
  p.y = (int)ly;
  const int cx = min(max(p.x, 0), J.w - 1) / cell;
  const int cy = min(max(p.y, 0), J.h - 1) / cell;
  return cy * J.ncx + cx;
}

// Zeroes every job's cell counts (sizes from the job table) and the batch's
// counters.
__global__ void zero_kernel(BinArgs b) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  const int nj = b.batch->njobs;
  for (int j = 0; j < nj; ++j) {
    const JobDev& J = b.jobs[j];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i <= J.ncells; i += stride)
      J.cnt[i] = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) b.jobs[j].amax = 0.f;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    b.batch->counter = 0;
    for (int t = 0; t < 6; ++t) b.batch->timers[t] = 0;
  }
}

// Loads the jobs' first-point indices into shared memory.
__device__ __forceinline__ int load_pt0(const BinArgs& b, long long* spt0) {
  const int nj = min(b.batch->njobs, kMaxJobs);
  for (int j = threadIdx.x; j < nj; j += blockDim.x) spt0[j] = b.jobs[j].pt0;
  __syncthreads();
  return nj;
}

__global__ void __launch_bounds__(256) count_kernel(BinArgs b) {
  __shared__ long long spt0[kMaxJobs];
  const int nj = load_pt0(b, spt0);
  const long long npts = b.batch->npts;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < npts; g += stride) {
    const int jid = job_of(spt0, nj, g);
    const JobDev& J = b.jobs[jid];
    wasabi_point p = J.pts[g - J.pt0];
    if (p.d >= (uint32_t)b.D) atomicCAS(b.status, 0, WASABI_E_RANGE);
    const int c = cell_of(J, p, b.cell, b.reach, b.D);
    if (c >= 0) atomicAdd(&J.cnt[c], 1);
    if (b.track_amax) {
      // Largest |a| of the job: one atomic per warp and job (non-negative
      // floats order like their bit patterns).
      const unsigned v = c >= 0 ? __float_as_uint(fabsf(p.a)) : 0u;
      const unsigned act = __activemask();
      const unsigned grp = __match_any_sync(act, jid);
      const unsigned mx = __reduce_max_sync(grp, v);
      if ((threadIdx.x & 31) == __ffs(grp) - 1 && mx > 0u)
        atomicMax(reinterpret_cast<unsigned*>(&b.jobs[jid].amax), mx);
    }
  }
}

// Exclusive scan of each job's cell counts into off[0..ncells] and
// cursor[0..ncells): one block per job at a time, chunks of 16,384 counts,
// each thread sixteen consecutive counts, a running carry between chunks.
__global__ void __launch_bounds__(1024) scan_kernel(BinArgs b) {
  constexpr int CPT = 16;  // counts per thread
  __shared__ unsigned warp_sum[32];
  __shared__ unsigned s_carry;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nj = b.batch->njobs;
  for (int j = blockIdx.x; j < nj; j += gridDim.x) {
    const JobDev& J = b.jobs[j];
    const int ncells = J.ncells;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base < ncells; base += CPT * 1024) {
      const int i0 = base + CPT * threadIdx.x;
      int c[CPT];
      unsigned local = 0;
      const bool whole = i0 + CPT <= ncells;  // the arrays are 256-byte aligned: 16-byte vectors
      if (whole) {
#pragma unroll
        for (int q = 0; q < CPT / 4; ++q) {
          const int4 v = reinterpret_cast<const int4*>(J.cnt + i0)[q];
          c[4 * q] = v.x; c[4 * q + 1] = v.y; c[4 * q + 2] = v.z; c[4 * q + 3] = v.w;
        }
      } else {
#pragma unroll
        for (int q = 0; q < CPT; ++q) c[q] = i0 + q < ncells ? J.cnt[i0 + q] : 0;
      }
#pragma unroll
      for (int q = 0; q < CPT; ++q) local += (unsigned)c[q];
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
      int o[CPT];
#pragma unroll
      for (int q = 0; q < CPT; ++q) {
        o[q] = (int)run;
        run += (unsigned)c[q];
      }
      if (whole) {
#pragma unroll
        for (int q = 0; q < CPT / 4; ++q) {
          const int4 v = make_int4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
          reinterpret_cast<int4*>(J.off + i0)[q] = v;
          reinterpret_cast<int4*>(J.cursor + i0)[q] = v;
        }
      } else {
#pragma unroll
        for (int q = 0; q < CPT; ++q)
          if (i0 + q < ncells) {
            J.off[i0 + q] = o[q];
            J.cursor[i0 + q] = o[q];
          }
      }
      __syncthreads();
      if (threadIdx.x == 0) s_carry = carry + warp_sum[31];
      __syncthreads();
    }
    if (threadIdx.x == 0) J.off[ncells] = (int)s_carry;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) scatter_points_kernel(BinArgs b) {
  __shared__ long long spt0[kMaxJobs];
  const int nj = load_pt0(b, spt0);
  const long long npts = b.batch->npts;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < npts; g += stride) {
    const JobDev& J = b.jobs[job_of(spt0, nj, g)];
    wasabi_point p = J.pts[g - J.pt0];
    const int c = cell_of(J, p, b.cell, b.reach, b.D);  // p now in the job's frame
    if (c < 0) continue;
    const int slot = atomicAdd(&J.cursor[c], 1);
    J.sorted[slot] = p;
  }
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

cudaError_t launch_init_single(const JobDev& job, JobDev* jobs_dev, BatchDev* batch_dev, int nsp,
                               cudaStream_t s) {
  init_single_kernel<<<1, 1, 0, s>>>(job, jobs_dev, batch_dev, nsp);
  return cudaGetLastError();
}

cudaError_t launch_binning(const BinArgs& b, cudaStream_t s) {
  const unsigned grid = (unsigned)(b.grid > 0 ? b.grid : 1);
  zero_kernel<<<grid, 256, 0, s>>>(b);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  count_kernel<<<grid, 256, 0, s>>>(b);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  scan_kernel<<<(unsigned)(b.grid > 0 ? (b.grid + 7) / 8 : 1), 1024, 0, s>>>(b);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  scatter_points_kernel<<<grid, 256, 0, s>>>(b);
  return cudaGetLastError();
}

}  // namespace wsb
