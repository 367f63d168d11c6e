// Eq. (1) on the GPU: u(x_h, y_h) = sum_j a_j exp(i 2 pi r_hj / lambda) over
// the points whose PSF disk covers the pixel (or over all points when the
// aperture is off).
//
// A persistent CTA owns 32 x 32 pixel tiles; for each tile it scans the binned
// points of the cell rows within reach, keeps those whose disk meets the tile
// (nearest-point distance test), and every thread accumulates its 4 pixels
// over the kept points in FP32.
//
// Phase: r / lambda = sqrt(q) with q = n (p / lambda)^2 + (z / lambda)^2 and
// n = dx^2 + dy^2.  q is formed in double-float (pairs of FP32 values; the
// error-free transformations are Knuth's two-sum and the exact product
// through one fused multiply-add), an FP32 estimate s0 of sqrt(q) is refined
// by one Newton step whose residual q - s0^2 is exact, so r / lambda mod 1 is
// carried to about 1e-10 cycles in FP32 arithmetic alone (FP64 runs far
// slower), and the fractional cycle feeds an FP32 sincospi.  Whether a pixel
// lies in a disk stays an exact integer test.
#include "dbf.cuh"

namespace wsb {
namespace {

constexpr int kTile = 32;
constexpr int kNT = 256;
constexpr int kCap = kNT;
constexpr int kMaxRows = 128;

__device__ __forceinline__ int floor_div(int a, int b) {
  const int q = a / b;
  return (a % b != 0 && ((a < 0) != (b < 0))) ? q - 1 : q;
}

__global__ void __launch_bounds__(kNT) direct_kernel(DirectArgs a) {
  __shared__ int4 list[kCap];
  __shared__ float4 lbeta[kCap];  // |beta| as hi + lo, the sign of z
  __shared__ long long lnlim[kCap];
  __shared__ int s_tile, s_n, s_nrows, s_total;
  __shared__ int s_rowstart[kMaxRows], s_rowpre[kMaxRows + 1];
  const int tid = threadIdx.x;
  const JobDev& J = a.jobs[0];
  const int ncx = J.ncx, ncy = J.ncy;
  const int* cell_off = J.off;
  const wasabi_point* sorted = J.sorted;
  const int ntx = (a.w + kTile - 1) / kTile, nty = (a.h + kTile - 1) / kTile;
  const int ntiles = ntx * nty;
  const int col = tid & 31, row0 = tid >> 5;  // pixels (col, row0 + 8 q), q < 4
  const float al_h = (float)a.alpha, al_l = (float)(a.alpha - (double)al_h);  // (p / lambda)^2

  for (;;) {
    if (tid == 0) s_tile = atomicAdd(a.counter, 1);
    __syncthreads();
    const int t = s_tile;
    if (t >= ntiles) break;
    const int X0 = (t % ntx) * kTile, Y0 = (t / ntx) * kTile;
    const int X1 = min(X0 + kTile, a.w), Y1 = min(Y0 + kTile, a.h);

    const int cx0 = max(0, floor_div(X0 - a.reach, a.cell));
    const int cx1 = min(ncx - 1, floor_div(X1 - 1 + a.reach, a.cell));
    const int cy0 = max(0, floor_div(Y0 - a.reach, a.cell));
    const int cy1 = min(ncy - 1, floor_div(Y1 - 1 + a.reach, a.cell));
    if (tid == 0) {
      const int nrows = (cx0 <= cx1 && cy0 <= cy1) ? cy1 - cy0 + 1 : 0;
      int run = 0;
      for (int r = 0; r < nrows; ++r) {
        const int c0 = (cy0 + r) * ncx;
        const int s0 = cell_off[c0 + cx0];
        s_rowstart[r] = s0;
        s_rowpre[r] = run;
        run += cell_off[c0 + cx1 + 1] - s0;
      }
      s_rowpre[nrows] = run;
      s_nrows = nrows;
      s_total = run;
    }
    __syncthreads();
    const int total = s_total, nrows = s_nrows;

    float re[4] = {0.f, 0.f, 0.f, 0.f}, im[4] = {0.f, 0.f, 0.f, 0.f};
    for (int c0 = 0; c0 < total; c0 += kNT) {
      if (tid == 0) s_n = 0;
      __syncthreads();
      const int i = c0 + tid;
      if (i < total) {
        int r = 0;
        while (r + 1 < nrows && s_rowpre[r + 1] <= i) ++r;
        const int4 p = __ldg(reinterpret_cast<const int4*>(sorted) + s_rowstart[r] + (i - s_rowpre[r]));
        const long long nlim = __ldg(&a.nlim_dev[p.w]);
        const long long ddx = p.x < X0 ? X0 - p.x : (p.x > X1 - 1 ? p.x - (X1 - 1) : 0);
        const long long ddy = p.y < Y0 ? Y0 - p.y : (p.y > Y1 - 1 ? p.y - (Y1 - 1) : 0);
        if (ddx * ddx + ddy * ddy < nlim) {
          const int slot = atomicAdd(&s_n, 1);
          list[slot] = p;
          const double b = __ldg(&a.beta_dev[p.w]), bm = fabs(b);
          const float bh = (float)bm;
          lbeta[slot] = make_float4(bh, (float)(bm - (double)bh), b < 0.0 ? -1.0f : 1.0f, 0.f);
          lnlim[slot] = nlim;
        }
      }
      __syncthreads();
      const int n = s_n;
      const int px = X0 + col;
      for (int s = 0; s < n; ++s) {
        const int4 p = list[s];
        const float4 lb = lbeta[s];
        const float sgn = lb.z;  // conjugate term for a point behind the plane
        const long long nlim = lnlim[s];
        const float amp = __int_as_float(p.z);
        const long long dx = px - p.x;
        // dx^2 as hi + lo, both exact (|dx| < 2^24).
        const float fdx = (float)dx, xx = __fmul_rn(fdx, fdx), xe = __fmaf_rn(fdx, fdx, -xx);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const long long dy = Y0 + row0 + 8 * q - p.y;
          const long long nn = dx * dx + dy * dy;
          if (nn < nlim) {
            // n = dx^2 + dy^2 as hi + lo (exact), then q = alpha n + beta.
            const float fdy = (float)dy, yy = __fmul_rn(fdy, fdy), ye = __fmaf_rn(fdy, fdy, -yy);
            const Dbf n2 = two_sum(xx, yy);
            const float nl = __fadd_rn(n2.lo, __fadd_rn(xe, ye));
            const float pa = __fmul_rn(al_h, n2.hi);
            const float pe = __fmaf_rn(al_h, n2.hi, -pa) + (al_h * nl + al_l * n2.hi);
            const Dbf q0 = two_sum(pa, lb.x);
            const Dbf qv = two_sum(q0.hi, __fadd_rn(q0.lo, __fadd_rn(pe, lb.y)));
            // sqrt(q) = s0 + corr: s0 in FP32, the residual q - s0^2 exact
            // (s0^2 lies within a factor 2 of q.hi).
            const float qf = qv.hi;
            const float r0 = rsqrtf(qf);
            const float s0 = __fmul_rn(qf, r0);
            const float ss = __fmul_rn(s0, s0), se = __fmaf_rn(s0, s0, -ss);
            const float corr = __fadd_rn(__fsub_rn(__fsub_rn(qf, ss), se), qv.lo) * (0.5f * r0);
            const float f = qf > 0.f ? (s0 - floorf(s0)) + corr : 0.f;  // q = 0: a point on the plane
            float sn, cs;
            sincospif(2.0f * f, &sn, &cs);
            re[q] = fmaf(amp, cs, re[q]);
            im[q] = fmaf(amp, sgn * sn, im[q]);
          }
        }
      }
      __syncthreads();
    }
    const int px = X0 + col;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int py = Y0 + row0 + 8 * q;
      if (px < X1 && py < Y1) a.u[(size_t)py * a.w + px] = make_float2(re[q], im[q]);
    }
    __syncthreads();
  }
}

}  // namespace

int direct_max_cell_rows() { return kMaxRows; }

cudaError_t launch_direct(const DirectArgs& a, cudaStream_t s) {
  direct_kernel<<<a.grid, kNT, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace wsb
