// Superposition in the wavelet domain (Eq. (2)), owner-computes form.
//
// The hologram's tile-major wavelet buffer is cut into super-tiles of T x T
// pixels (k = T / 2^L tiles a side).  A persistent CTA claims super-tiles from
// a global counter; for each one it
//   1. zeroes a T*T complex accumulator in shared memory;
//   2. scans the binned points of the cell rows within reach and keeps the
//      "survivors" whose footprint (window-tile box of their depth, shifted,
//      plus one tile of carry) meets the super-tile, with their shift data;
//   3. turns every survivor into one LUT range per window-tile row that can
//      land in the super-tile (contiguous by construction of the LUT), and
//      prefix-sums the range lengths into one flat list of coefficient visits;
//   4. splits the visits evenly over the warps: each warp walks a contiguous
//      slice 32 visits at a time (coalesced LUT loads), applies the shift rule
//      and adds a_j * c into shared memory;
//   5. writes the finished super-tile to global memory once, with streaming
//      vector stores.
// Every buffer element is written exactly once: no global atomics and no
// zeroing pass.  Shared-memory atomics resolve collisions between survivors.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.cuh"

namespace wsb {
namespace {

constexpr int kMaxCellRows = 128;
constexpr int kRangeCap = 4096;  // LUT ranges per batch

__device__ __forceinline__ int floor_div(int a, int b) {
  const int q = a / b;
  return (a % b != 0 && ((a < 0) != (b < 0))) ? q - 1 : q;
}

// Tile offset A = floor(X / 2^L) and per-level residual shifts
// delta_l = shift_l(X) - A * 2^(L-l), packed 5 bits per level at bit 5l.
__device__ __forceinline__ void make_shift(int X, int L, int rule, int* A, uint32_t* pk) {
  const int a = X >> L;  // arithmetic shift: floor division by 2^L
  const int r = X - (a << L);
  uint32_t p = 0;
  for (int l = 1; l <= L; ++l) {
    const int dl = rule == WASABI_SHIFT_FLOOR ? (r >> l) : ((r + (1 << (l - 1))) >> l);
    p |= (uint32_t)dl << (5 * l);
  }
  *A = a;
  *pk = p;
}

template <int DT>
__device__ __forceinline__ float2 lut_value(const LutView& lut, int e) {
  if (DT == WASABI_F32) return __ldg(&lut.val[e]);
  const uint32_t q = __ldg(&lut.val16[e]);
  const float s = __ldg(&lut.scale[e >> 5]);
  float re, im;
  if (DT == WASABI_F16S) {
    re = __half2float(__ushort_as_half((unsigned short)(q & 0xffffu)));
    im = __half2float(__ushort_as_half((unsigned short)(q >> 16)));
  } else {
    re = __bfloat162float(__ushort_as_bfloat16((unsigned short)(q & 0xffffu)));
    im = __bfloat162float(__ushort_as_bfloat16((unsigned short)(q >> 16)));
  }
  return make_float2(re * s, im * s);
}

// Exclusive scan over the block of one value per thread; returns the prefix
// and writes the total to *total (all threads).
__device__ __forceinline__ int block_scan(int v, int* total, int* warp_buf) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_buf[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int t = lane < nw ? warp_buf[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    warp_buf[lane] = t;
  }
  __syncthreads();
  const int excl = (wid ? warp_buf[wid - 1] : 0) + x - v;
  *total = warp_buf[31];
  __syncthreads();
  return excl;
}

// Last index r in [lo, hi] with pre[r] <= v (pre non-decreasing, pre[lo] <= v).
__device__ __forceinline__ int last_le(const int* pre, int lo, int hi, int v) {
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= v) lo = mid; else hi = mid - 1;
  }
  return lo;
}

struct Smem {
  float2* acc;    // T * T
  int4* sp;       // survivors: Ax, Ay, dpx, dpy
  float* samp;    // survivors: amplitude
  int* sd;        // survivors: depth
  int* srow;      // survivors: first range index (P + 1)
  int* rdel;      // ranges: LUT index minus visit prefix
  int* rpre;      // ranges: visit prefix (R + 1)
  int* rsv;       // ranges: survivor
  int2* dbox;     // depths: tlo, thi
};

__host__ __device__ inline int survivor_cap(int k) {
  const int p = kRangeCap / (k + 1);
  return p < 1024 ? p : 1024;
}

__host__ __device__ inline size_t smem_layout(int T, int L, int D, Smem* s, unsigned char* base) {
  const int k = T >> L;
  const int P = survivor_cap(k);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = (off + bytes + 15) & ~(size_t)15;
    return base ? base + o : nullptr;
  };
  unsigned char* p0 = take((size_t)T * T * sizeof(float2));
  unsigned char* p1 = take((size_t)P * sizeof(int4));
  unsigned char* p2 = take((size_t)P * sizeof(float));
  unsigned char* p3 = take((size_t)P * sizeof(int));
  unsigned char* p4 = take((size_t)(P + 1) * sizeof(int));
  unsigned char* p5 = take((size_t)kRangeCap * sizeof(int));
  unsigned char* p6 = take((size_t)(kRangeCap + 1) * sizeof(int));
  unsigned char* p7 = take((size_t)kRangeCap * sizeof(int));
  unsigned char* p8 = take((size_t)D * sizeof(int2));
  if (s) {
    s->acc = reinterpret_cast<float2*>(p0);
    s->sp = reinterpret_cast<int4*>(p1);
    s->samp = reinterpret_cast<float*>(p2);
    s->sd = reinterpret_cast<int*>(p3);
    s->srow = reinterpret_cast<int*>(p4);
    s->rdel = reinterpret_cast<int*>(p5);
    s->rpre = reinterpret_cast<int*>(p6);
    s->rsv = reinterpret_cast<int*>(p7);
    s->dbox = reinterpret_cast<int2*>(p8);
  }
  return off;
}

template <int L, int DT>
__global__ void __launch_bounds__(1024, 1) superpose_kernel(SuperposeArgs a) {
  constexpr int TSL = 1 << (2 * L);
  extern __shared__ __align__(16) unsigned char smem[];
  const int T = a.cell;
  const int k = T >> L;
  const int P = survivor_cap(k);
  Smem S;
  smem_layout(T, L, a.lut.D, &S, smem);
  __shared__ int s_st, s_next, s_n, s_nrows, s_total;
  __shared__ int s_rowstart[kMaxCellRows], s_rowpre[kMaxCellRows + 1];
  __shared__ int warp_buf[32];

  const LutView& lut = a.lut;
  const int NT = blockDim.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = NT >> 5;
  const int W2 = lut.W / 2;
  const int ntpd = lut.nwt * lut.nwt + 1;  // tile_off entries per depth
  for (int d = tid; d < lut.D; d += NT) {
    const DepthMeta m = lut.meta[d];
    S.dbox[d] = make_int2(m.tlo, m.thi);
  }
  const int nstx = (a.ntx + k - 1) / k, nsty = (a.nty + k - 1) / k;
  const int nst = nstx * nsty;
  // Largest |a_j| and largest component of any kept coefficient: with the
  // candidate count they bound every accumulated component of a super-tile.
  const float amax_cmax = __ldg(a.amax) * __ldg(lut.cmax);
  float4* acc4 = reinterpret_cast<float4*>(S.acc);
  int* acci = reinterpret_cast<int*>(S.acc);
  const bool fixed = !a.acc_float;
  if (tid == 0) s_next = atomicAdd(a.counter, 1);

  for (;;) {
    __syncthreads();
    if (tid == 0) {
      s_st = s_next;
      s_next = atomicAdd(a.counter, 1);  // claim the next one early
    }
    __syncthreads();
    const int st = s_st;
    if (st >= nst) break;
    const int Sx = (st % nstx) * k, Sy = (st / nstx) * k;
    const int kx = min(k, a.ntx - Sx), ky = min(k, a.nty - Sy);

    for (int i = tid; i < T * T / 2; i += NT) acc4[i] = make_float4(0.f, 0.f, 0.f, 0.f);

    // Cell rows within reach of the super-tile, one thread per row.
    const int X0 = Sx << L, X1 = (Sx + kx) << L, Y0 = Sy << L, Y1 = (Sy + ky) << L;
    const int cx0 = max(0, floor_div(X0 - a.reach, a.cell));
    const int cx1 = min(a.ncx - 1, floor_div(X1 - 1 + a.reach, a.cell));
    const int cy0 = max(0, floor_div(Y0 - a.reach, a.cell));
    const int cy1 = min(a.ncy - 1, floor_div(Y1 - 1 + a.reach, a.cell));
    const int ncrows = (cx0 <= cx1 && cy0 <= cy1) ? cy1 - cy0 + 1 : 0;
    if (tid < ncrows) {
      const int c0 = (cy0 + tid) * a.ncx;
      const int s0 = __ldg(&a.cell_off[c0 + cx0]);
      s_rowstart[tid] = s0;
      s_rowpre[tid] = __ldg(&a.cell_off[c0 + cx1 + 1]) - s0;
    }
    __syncthreads();
    if (warp == 0) {  // exclusive prefix over <= 128 rows, 4 per lane
      int v[4], loc = 0;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int r = 4 * lane + j;
        v[j] = r < ncrows ? s_rowpre[r] : 0;
        loc += v[j];
      }
      int incl = loc;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      int run = incl - loc;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int r = 4 * lane + j;
        if (r < ncrows) s_rowpre[r] = run;
        run += v[j];
      }
      if (lane == 31) { s_rowpre[ncrows] = incl; s_total = incl; }
    }
    __syncthreads();
    const int total = s_total;
    // Fixed-point scale 2^sh: every partial sum stays below 2^31 in magnitude.
    const float bound = (float)total * amax_cmax;
    const int sh = bound > 0.f ? min(30, (int)floorf(log2f(2.0e9f / bound))) : 30;
    const float qs = ldexpf(1.0f, sh);

    const int CH = min(P, NT);  // candidates per batch: at most one per thread
    for (int c0 = 0; c0 < total; c0 += CH) {
      // ---- survivors of this batch of candidates
      if (tid == 0) s_n = 0;
      __syncthreads();
      if (tid < CH && c0 + tid < total) {
        const int i = c0 + tid;
        int r = 0;
        while (r + 1 < ncrows && s_rowpre[r + 1] <= i) ++r;
        const int4 p = __ldg(reinterpret_cast<const int4*>(a.sorted) + s_rowstart[r] + (i - s_rowpre[r]));
        const int2 bx = S.dbox[p.w];
        int Ax, Ay;
        uint32_t dpx, dpy;
        make_shift(p.x - W2, L, a.rule, &Ax, &dpx);
        make_shift(p.y - W2, L, a.rule, &Ay, &dpy);
        const int tya = max(bx.x, Sy - Ay - 1), tyb = min(bx.y, Sy + ky - 1 - Ay);
        const int txa = max(bx.x, Sx - Ax - 1), txb = min(bx.y, Sx + kx - 1 - Ax);
        if (txa <= txb && tya <= tyb) {
          const int s = atomicAdd(&s_n, 1);
          S.sp[s] = make_int4(Ax, Ay, (int)dpx, (int)dpy);
          S.samp[s] = __int_as_float(p.z) * (fixed ? qs : 1.0f);
          S.sd[s] = p.w;
          S.srow[s] = tyb - tya + 1;
        }
      }
      __syncthreads();
      const int n = s_n;
      int nranges;
      {
        const int v = tid < n ? S.srow[tid] : 0;
        const int ex = block_scan(v, &nranges, warp_buf);
        if (tid < n) S.srow[tid] = ex;
        if (tid == 0) S.srow[n] = nranges;
      }
      __syncthreads();
      // ---- one LUT range per (survivor, window-tile row)
      for (int f = tid; f < nranges; f += NT) {
        const int s = last_le(S.srow, 0, n - 1, f);
        const int4 sp = S.sp[s];
        const int d = S.sd[s];
        const int2 bx = S.dbox[d];
        const int tya = max(bx.x, Sy - sp.y - 1);
        const int txa = max(bx.x, Sx - sp.x - 1), txb = min(bx.y, Sx + kx - 1 - sp.x);
        const int ro = d * ntpd + (tya + f - S.srow[s]) * lut.nwt;
        const int st0 = __ldg(&lut.tile_off[ro + txa]);
        const int en0 = __ldg(&lut.tile_off[ro + txb + 1]);
        S.rdel[f] = st0;
        S.rpre[f] = en0 - st0;
        S.rsv[f] = s;
      }
      __syncthreads();
      // ---- prefix of range lengths
      int nvis;
      {
        const int per = (nranges + NT - 1) / NT;
        const int f0 = tid * per;
        int loc = 0;
        for (int f = f0; f < min(f0 + per, nranges); ++f) loc += S.rpre[f];
        int run = block_scan(loc, &nvis, warp_buf);
        for (int f = f0; f < min(f0 + per, nranges); ++f) {
          const int len = S.rpre[f];
          S.rpre[f] = run;
          S.rdel[f] -= run;  // LUT index = visit + rdel
          run += len;
        }
        if (tid == 0) S.rpre[nranges] = nvis;
      }
      __syncthreads();
      // ---- visits: warp w takes [w*per, (w+1)*per), 64 at a time
      if (nvis > 0) {
        const int per = (nvis + nwarps - 1) / nwarps;
        const int v0 = warp * per, v1 = min(nvis, v0 + per);
        int rb = v0 < v1 ? last_le(S.rpre, 0, nranges - 1, v0) : 0;
        for (int b = v0; b < v1; b += 64) {
          int rr[2], ee[2];
          uint32_t pp[2];
          float2 vv[2];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int i = b + 32 * h + lane;
            // Walk forward from the previous range (a chunk spans a few
            // ranges; empty ranges are stepped over; rpre[nranges] = nvis
            // ends the walk).
            const int vi = min(i, v1 - 1);
            int r = h ? rr[0] : rb;
            while (S.rpre[r + 1] <= vi) ++r;
            rr[h] = r;
            ee[h] = vi + S.rdel[r];
            pp[h] = __ldg(&lut.pos[ee[h]]);
            vv[h] = lut_value<DT>(lut, ee[h]);
          }
          rb = __shfl_sync(0xffffffffu, rr[1], 31);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int i = b + 32 * h + lane;
            if (i >= v1) continue;
            const int s = S.rsv[rr[h]];
            const int4 sp = S.sp[s];
            const float amp = S.samp[s];
            const uint32_t q = pp[h];
            const int tx = q & 511, ty = (q >> 9) & 511, lev = (q >> 18) & 7;
            const int band = (q >> 21) & 3, ix = (q >> 23) & 15, iy = q >> 27;
            const int m = L - lev;
            const int sx = ix + (int)(((uint32_t)sp.z >> (5 * lev)) & 31u);
            const int sy = iy + (int)(((uint32_t)sp.w >> (5 * lev)) & 31u);
            const int relx = sp.x + tx + (sx >> m) - Sx;
            const int rely = sp.y + ty + (sy >> m) - Sy;
            if ((unsigned)relx < (unsigned)kx && (unsigned)rely < (unsigned)ky) {
              const int mk = (1 << m) - 1;
              const int slot = (band << (2 * m)) | ((sy & mk) << m) | (sx & mk);
              const int ai = 2 * (((rely * k + relx) << (2 * L)) + slot);
              if (fixed) {
                // a_j c in FP32, then exact scaling by 2^sh (folded into amp)
                // and rounding to the nearest integer; integer sums are exact.
                atomicAdd(&acci[ai], __float2int_rn(amp * vv[h].x));
                atomicAdd(&acci[ai + 1], __float2int_rn(amp * vv[h].y));
              } else {
                atomicAdd(&S.acc[ai >> 1].x, amp * vv[h].x);
                atomicAdd(&S.acc[ai >> 1].y, amp * vv[h].y);
              }
            }
          }
        }
      }
      __syncthreads();
    }

    // Write the super-tile: ky runs of kx tiles, each run contiguous.
    const int run4 = kx * TSL / 2;  // float4 per run
    const float dq = ldexpf(1.0f, -sh);
    for (int i = tid; i < run4 * ky; i += NT) {
      const int j = i / run4, q = i - j * run4;
      float4 v = acc4[(size_t)j * (k * TSL / 2) + q];
      if (fixed) {
        const int4 iv = reinterpret_cast<const int4*>(acc4)[(size_t)j * (k * TSL / 2) + q];
        v = make_float4((float)iv.x * dq, (float)iv.y * dq, (float)iv.z * dq, (float)iv.w * dq);
      }
      float4* dst = reinterpret_cast<float4*>(a.wbuf + ((size_t)(Sy + j) * a.ntx + Sx) * TSL) + q;
      __stcs(dst, v);
    }
  }
}

template <int L, int DT>
cudaError_t launch_t(const SuperposeArgs& a, cudaStream_t s) {
  const size_t smem = superpose_smem_bytes(a.cell, a.lut.L, a.lut.D);
  cudaError_t e = cudaFuncSetAttribute(superpose_kernel<L, DT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  superpose_kernel<L, DT><<<a.grid, a.threads, smem, s>>>(a);
  return cudaGetLastError();
}

template <int L>
cudaError_t launch_l(const SuperposeArgs& a, cudaStream_t s) {
  switch (a.lut.dtype) {
    case WASABI_F32: return launch_t<L, WASABI_F32>(a, s);
    case WASABI_F16S: return launch_t<L, WASABI_F16S>(a, s);
    case WASABI_BF16S: return launch_t<L, WASABI_BF16S>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

size_t superpose_smem_bytes(int cell, int L, int D) {
  return smem_layout(cell, L, D, nullptr, nullptr);
}

int superpose_max_cell_rows() { return kMaxCellRows; }

cudaError_t launch_superpose(const SuperposeArgs& a, cudaStream_t s) {
  if (a.threads > 1024 || a.threads < 64 || a.threads % 32) return cudaErrorInvalidValue;
  switch (a.lut.L) {
    case 1: return launch_l<1>(a, s);
    case 2: return launch_l<2>(a, s);
    case 3: return launch_l<3>(a, s);
    case 4: return launch_l<4>(a, s);
    case 5: return launch_l<5>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace wsb
