// Superposition in the wavelet domain (Eq. (2)), owner-computes form.
//
// The hologram's tile-major wavelet buffer is cut into super-tiles of T x T
// pixels (k = T / 2^L tiles a side).  A persistent CTA claims super-tiles from
// a global counter; for each one it
//   1. zeroes a T*T complex accumulator in shared memory,
//   2. scans the binned points of the cell rows within reach, keeping those
//      whose footprint (window-tile box of their depth, shifted, plus one
//      tile of carry) meets the super-tile,
//   3. lets one warp per kept point walk exactly the LUT ranges whose
//      coefficients can land in the super-tile (one contiguous range per
//      window-tile row), applying the shift rule per coefficient and adding
//      a_j * c into shared memory,
//   4. writes the finished super-tile to global memory once, with streaming
//      vector stores.
// Every buffer element is written exactly once, so there are no global
// atomics and no zeroing pass.  Within a warp all lanes work on one point, and
// a point's shifted coefficient positions are distinct, so lanes never
// collide on an address; shared-memory atomics only resolve collisions
// between warps.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.cuh"

namespace wsb {
namespace {

constexpr int kListCap = 1024;  // >= block size: one candidate per thread per chunk
constexpr int kMaxCellRows = 128;

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

template <int L, int DT>
__global__ void __launch_bounds__(1024, 1) superpose_kernel(SuperposeArgs a) {
  constexpr int TSL = 1 << (2 * L);
  extern __shared__ __align__(16) unsigned char smem[];
  const int T = a.cell;
  const int k = T >> L;
  float2* acc = reinterpret_cast<float2*>(smem);
  int4* list = reinterpret_cast<int4*>(acc + (size_t)T * T);
  int2* dbox = reinterpret_cast<int2*>(list + kListCap);
  __shared__ int s_st, s_nlist, s_nrows, s_total;
  __shared__ int s_rowstart[kMaxCellRows], s_rowpre[kMaxCellRows + 1];

  const LutView& lut = a.lut;
  const int NT = blockDim.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = NT >> 5;
  const int W2 = lut.W / 2;
  const int ntpd = lut.nwt * lut.nwt + 1;  // tile_off entries per depth
  for (int d = tid; d < lut.D; d += NT) {
    const DepthMeta m = lut.meta[d];
    dbox[d] = make_int2(m.tlo, m.thi);
  }
  const int nstx = (a.ntx + k - 1) / k, nsty = (a.nty + k - 1) / k;
  const int nst = nstx * nsty;

  for (;;) {
    if (tid == 0) s_st = atomicAdd(a.counter, 1);
    __syncthreads();
    const int st = s_st;
    if (st >= nst) break;
    const int Sx = (st % nstx) * k, Sy = (st / nstx) * k;
    const int kx = min(k, a.ntx - Sx), ky = min(k, a.nty - Sy);

    float4* acc4 = reinterpret_cast<float4*>(acc);
    for (int i = tid; i < T * T / 2; i += NT) acc4[i] = make_float4(0.f, 0.f, 0.f, 0.f);

    // Cell rows within reach of the super-tile.
    const int X0 = Sx << L, X1 = (Sx + kx) << L, Y0 = Sy << L, Y1 = (Sy + ky) << L;
    const int cx0 = max(0, floor_div(X0 - a.reach, a.cell));
    const int cx1 = min(a.ncx - 1, floor_div(X1 - 1 + a.reach, a.cell));
    const int cy0 = max(0, floor_div(Y0 - a.reach, a.cell));
    const int cy1 = min(a.ncy - 1, floor_div(Y1 - 1 + a.reach, a.cell));
    if (tid == 0) {
      const int nrows = (cx0 <= cx1 && cy0 <= cy1) ? cy1 - cy0 + 1 : 0;
      int run = 0;
      for (int r = 0; r < nrows; ++r) {
        const int c0 = (cy0 + r) * a.ncx;
        const int s0 = a.cell_off[c0 + cx0];
        s_rowstart[r] = s0;
        s_rowpre[r] = run;
        run += a.cell_off[c0 + cx1 + 1] - s0;
      }
      s_rowpre[nrows] = run;
      s_nrows = nrows;
      s_total = run;
    }
    __syncthreads();
    const int total = s_total, nrows = s_nrows;

    for (int c0 = 0; c0 < total; c0 += NT) {
      if (tid == 0) s_nlist = 0;
      __syncthreads();
      const int i = c0 + tid;
      if (i < total) {
        int r = 0;
        while (r + 1 < nrows && s_rowpre[r + 1] <= i) ++r;
        const int4 p = __ldg(reinterpret_cast<const int4*>(a.sorted) + s_rowstart[r] + (i - s_rowpre[r]));
        const int d = p.w;
        const int2 bx = dbox[d];
        const int Ax = (p.x - W2) >> L, Ay = (p.y - W2) >> L;
        if (Ax + bx.x <= Sx + kx - 1 && Ax + bx.y + 1 >= Sx && Ay + bx.x <= Sy + ky - 1 &&
            Ay + bx.y + 1 >= Sy)
          list[atomicAdd(&s_nlist, 1)] = p;
      }
      __syncthreads();
      const int nlist = s_nlist;
      for (int s = warp; s < nlist; s += nwarps) {
        const int4 p = list[s];
        const int d = p.w;
        const float amp = __int_as_float(p.z);
        int Ax, Ay;
        uint32_t dpx, dpy;
        make_shift(p.x - W2, L, a.rule, &Ax, &dpx);
        make_shift(p.y - W2, L, a.rule, &Ay, &dpy);
        const int2 bx = dbox[d];
        const int txa = max(bx.x, Sx - Ax - 1), txb = min(bx.y, Sx + kx - 1 - Ax);
        const int tya = max(bx.x, Sy - Ay - 1), tyb = min(bx.y, Sy + ky - 1 - Ay);
        if (txa > txb || tya > tyb) continue;
        const int nr = tyb - tya + 1;  // <= k + 1 <= 32
        int rs = 0, rl = 0;
        if (lane < nr) {
          const int ro = d * ntpd + (tya + lane) * lut.nwt;
          rs = __ldg(&lut.tile_off[ro + txa]);
          rl = __ldg(&lut.tile_off[ro + txb + 1]) - rs;
        }
        int incl = rl;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += y;
        }
        const int cnt = __shfl_sync(0xffffffffu, incl, nr - 1);
        for (int b0 = 0; b0 < cnt; b0 += 32) {
          const int i2 = b0 + lane;
          int row = 0;
          for (int r = 0; r < nr; ++r) row += (__shfl_sync(0xffffffffu, incl, r) <= i2) ? 1 : 0;
          const int srow = __shfl_sync(0xffffffffu, rs, row & 31);
          const int excl = __shfl_sync(0xffffffffu, incl - rl, row & 31);
          if (i2 < cnt) {
            const int e = srow + (i2 - excl);
            const uint32_t pp = __ldg(&lut.pos[e]);
            const float2 v = lut_value<DT>(lut, e);
            const int tx = pp & 511, ty = (pp >> 9) & 511, lev = (pp >> 18) & 7;
            const int band = (pp >> 21) & 3, ix = (pp >> 23) & 15, iy = pp >> 27;
            const int m = L - lev;
            const int sx = ix + (int)((dpx >> (5 * lev)) & 31u);
            const int sy = iy + (int)((dpy >> (5 * lev)) & 31u);
            const int relx = Ax + tx + (sx >> m) - Sx;
            const int rely = Ay + ty + (sy >> m) - Sy;
            if ((unsigned)relx < (unsigned)kx && (unsigned)rely < (unsigned)ky) {
              const int mk = (1 << m) - 1;
              const int slot = (band << (2 * m)) | ((sy & mk) << m) | (sx & mk);
              float2* dst = acc + (((rely * k + relx) << (2 * L)) + slot);
              atomicAdd(&dst->x, amp * v.x);
              atomicAdd(&dst->y, amp * v.y);
            }
          }
        }
      }
      __syncthreads();
    }

    // Write the super-tile: ky runs of kx tiles, each run contiguous.
    const int run4 = kx * TSL / 2;  // float4 per run
    const int runs = ky;
    for (int i = tid; i < run4 * runs; i += NT) {
      const int j = i / run4, q = i - j * run4;
      const float4 v = acc4[(size_t)j * (k * TSL / 2) + q];
      float4* dst = reinterpret_cast<float4*>(a.wbuf + ((size_t)(Sy + j) * a.ntx + Sx) * TSL) + q;
      __stcs(dst, v);
    }
    __syncthreads();
  }
}

template <int L, int DT>
cudaError_t launch_t(const SuperposeArgs& a, cudaStream_t s) {
  static bool configured = false;
  const size_t smem = superpose_smem_bytes(a.cell, a.lut.D, a.threads);
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(superpose_kernel<L, DT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    configured = true;
  }
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

size_t superpose_smem_bytes(int cell, int D, int threads) {
  (void)threads;
  return (size_t)cell * cell * sizeof(float2) + kListCap * sizeof(int4) + (size_t)D * sizeof(int2);
}

int superpose_max_cell_rows() { return kMaxCellRows; }

cudaError_t launch_superpose(const SuperposeArgs& a, cudaStream_t s) {
  if (a.threads > kListCap || a.threads % 32) return cudaErrorInvalidValue;
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
