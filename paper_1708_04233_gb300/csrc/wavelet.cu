// The order-1 coiflet (Sec. 1 uses coiflets at level 3; the order is not
// stated): its filters, and the inverse transformation (Sec. 1, step 3) of a
// hologram superposed from a coiflet LUT.
//
// The coiflet transform is periodic over the whole hologram and its filters
// overlap 2^L x 2^L tiles, so the inverse is not tile-local as Haar's is: each
// level is one pass over tiles of its output, which gathers its input bands
// with a one-cell halo (details straight from the tile-major buffer, the
// low-pass band from the coarser level's result) and synthesises along y and
// then x in shared memory; the last level writes the field and/or the binary
// hologram against the frame's reference wave.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "dbf.cuh"
#include "lut_object.h"

namespace wsb {

// h_k, k = -2 .. 3, solves sum h = sqrt 2, sum_k h_k h_{k+2m} = delta_m
// (m = 0, 1, 2), sum (-1)^k k h_k = 0 and sum k h_k = 0; of the two real
// solutions, the one with the largest tap at k = 0:
//   h / sqrt 2 = ((1 - r)/32, (5 + r)/32, (7 + r)/16, (7 - r)/16,
//                (1 - r)/32, (r - 3)/32),  r = sqrt 7.
// g_k = (-1)^k h_{1-k}.
void coif1_filters(double lo[6], double hi[6]) {
  const double r = std::sqrt(7.0), s2 = std::sqrt(2.0);
  lo[0] = s2 * (1.0 - r) / 32.0;
  lo[1] = s2 * (5.0 + r) / 32.0;
  lo[2] = s2 * (7.0 + r) / 16.0;
  lo[3] = s2 * (7.0 - r) / 16.0;
  lo[4] = s2 * (1.0 - r) / 32.0;
  lo[5] = s2 * (r - 3.0) / 32.0;
  for (int k = -2; k <= 3; ++k) hi[k + 2] = ((k & 1) ? -1.0 : 1.0) * lo[(1 - k) + 2];
}

namespace {

struct CoifTaps {
  float lo[6], hi[6];
};

// Re(u conj R) for the frame's reference (R = 1 for the plane wave), phase
// in double-float per pixel.
__device__ __forceinline__ float ref_re(const RefDbf& ref, float2 u, long long X, long long Y) {
  if (ref.kind == 0) return u.x;
  float sn, cs;
  sincospif(2.0f * ref_frac(ref, (float)X, (float)Y), &sn, &cs);
  return fmaf(u.x, cs, ref.sgn * u.y * sn);
}

// One synthesis level (L -> L - 1, ..., 1 -> 0) of the periodic inverse,
// both directions in one pass over a TX x TY tile of the level's output (the
// S x S low-pass band of the next finer level, S = side >> (l - 1)).  Output
// sample j of a line takes h_k s[m] + g_k d[m] for k = j - 2m (mod the half
// length): the taps of j's parity with m = j/2 + 1, j/2, j/2 - 1 (k = -2, 0, 2
// for even j; -1, 1, 3 for odd j), each low tap then each high tap by fused
// multiply-add in that order.  A tile of outputs needs TY/2 + 2 input rows and
// TX/2 + 2 input columns of each of the four input bands (one cell of halo on
// each side, wrapped); they are gathered into shared memory -- the detail
// bands straight from the tile-major buffer, the low-pass band from the
// coarser level's result (or the buffer at the coarsest level) -- then
// synthesised along y for the needed columns and along x for the tile.
constexpr int kCoifTX = 64, kCoifTY = 32;

// Asynchronous global-to-shared copies (cached in L2 only for 16 bytes).
__device__ __forceinline__ void cp_async16(unsigned dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(unsigned dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}
constexpr int kCoifNX = kCoifTX / 2 + 2, kCoifNY = kCoifTY / 2 + 2;

struct CoifLevelArgs {
  const float2* wbuf;  // tile-major wavelet buffer (side x side)
  int side, L, l;      // hologram side, levels, level synthesised
  const float2* prev;  // level-l low-pass band, dense (side >> l)^2; null at l == L (read from the buffer)
  float2* out;         // level-(l - 1) low-pass band, dense S x S; the field (side x side) at l == 1, or null
  uint8_t* bits;       // l == 1: the binary hologram against the reference, or null
  int ox, oy;
  RefDbf ref;
  CoifTaps t;
};

// FULL: the level's side S is at least kCoifTX, so every tile is a whole
// kCoifTX x kCoifTY and one wrap per index suffices (sizes known at compile
// time: no integer division by a run-time value in the index arithmetic).
template <bool FULL>
__global__ void __launch_bounds__(256) coif_level_kernel(const __grid_constant__ CoifLevelArgs a) {
  // LL, LH (high x), HL (high y), HH; input column c at index c + 1 (the
  // row holds columns -1 .. kCoifNX, so that cell pairs land 16-byte aligned).
  __shared__ __align__(16) float2 in[4][kCoifNY][kCoifNX + 2];
  __shared__ float2 lx[kCoifTY][kCoifNX], hx[kCoifTY][kCoifNX];
  const int S = a.side >> (a.l - 1), hh = S / 2;
  const int TX = FULL ? kCoifTX : min(kCoifTX, S), TY = FULL ? kCoifTY : min(kCoifTY, S);
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int NX = TX / 2 + 2, NY = TY / 2 + 2;
  const int m = a.L - a.l, msk = (1 << m) - 1, TSL = 1 << (2 * a.L), ntx = a.side >> a.L;
  const int bx = x0 / 2 - 1, by = y0 / 2 - 1;  // first input column / row (unwrapped)
  auto wrap = [&](int v) {
    if (FULL) return v < 0 ? v + hh : (v >= hh ? v - hh : v);
    return (v % hh + hh) % hh;
  };
  if (FULL) {
    // Pairs of neighbouring cells (P even, P + 1) in one 16-byte copy: both
    // lie in one row of one tile of the buffer (P and P + 1 differ only in
    // the lowest bit) or of the dense low-pass band, and never straddle the
    // periodic wrap (the half side is even).  Input columns c = P - bx run
    // from -1 to kCoifNX, shared indices 0 .. kCoifNX + 1.  The copies are
    // asynchronous (global to shared, no registers), so all of a thread's
    // copies are in flight together.
    constexpr int NP = kCoifNX / 2 + 1;  // pairs per input row
    for (int i = threadIdx.x; i < 4 * kCoifNY * NP; i += blockDim.x) {
      const int part = i / (kCoifNY * NP), r = (i / NP) % kCoifNY, j = i % NP;
      const int P = wrap(bx + 2 * j - 1), Q = wrap(by + r);
      const unsigned dst = (unsigned)__cvta_generic_to_shared(&in[part][r][2 * j]);
      if (part == 0 && a.prev) {
        cp_async16(dst, a.prev + (size_t)Q * hh + P);
      } else {
        const size_t tile = (size_t)(Q >> m) * ntx + (P >> m);
        const int slot = part == 0 ? 0 : (part << (2 * m)) + ((Q & msk) << m) + (P & msk);
        if (m == 0) {  // the coarsest level: neighbouring cells are in neighbouring tiles
          cp_async8(dst, a.wbuf + tile * TSL + slot);
          cp_async8(dst + 8u, a.wbuf + (tile + 1) * TSL + slot);
        } else {
          cp_async16(dst, a.wbuf + tile * TSL + slot);
        }
      }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
  }
  for (int i = threadIdx.x; !FULL && i < 4 * NY * NX; i += blockDim.x) {
    const int part = i / (NY * NX), r = (i / NX) % NY, c = i % NX;
    const int P = wrap(bx + c), Q = wrap(by + r);
    float2 v;
    if (part == 0 && a.prev) {
      v = a.prev[(size_t)Q * hh + P];
    } else {
      // Band `part` of level l at (P, Q): its tile and in-tile slot.
      const size_t tile = (size_t)(Q >> m) * ntx + (P >> m);
      const int slot = part == 0 ? 0 : (part << (2 * m)) + ((Q & msk) << m) + (P & msk);
      v = a.wbuf[tile * TSL + slot];
    }
    in[part][r][c + 1] = v;
  }
  __syncthreads();
  const CoifTaps& t = a.t;
  // Along y: thread -> one input column c and eight output rows; the six
  // input rows those rows need are read once per band.
  auto synth = [&](const float2* sv, const float2* dv, int par, int base) {
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const int k = 2 * q + par, r = base - q;
      acc.x = __fmaf_rn(t.lo[k], sv[r].x, acc.x);
      acc.y = __fmaf_rn(t.lo[k], sv[r].y, acc.y);
      acc.x = __fmaf_rn(t.hi[k], dv[r].x, acc.x);
      acc.y = __fmaf_rn(t.hi[k], dv[r].y, acc.y);
    }
    return acc;
  };
  const int ngy = (TY + 7) / 8;
  for (int i = threadIdx.x; i < ngy * NX; i += blockDim.x) {
    const int gy = i / NX, c = i - gy * NX, yb = 8 * gy;
    // Output rows yb .. yb + 7 need input rows yb/2 .. yb/2 + 5.
    float2 s0[6], d0[6], s1[6], d1[6];
#pragma unroll
    for (int r = 0; r < 6; ++r) {
      const int rr = min(yb / 2 + r, NY - 1);
      s0[r] = in[0][rr][c + 1];
      d0[r] = in[2][rr][c + 1];
      s1[r] = in[1][rr][c + 1];
      d1[r] = in[3][rr][c + 1];
    }
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int yy = yb + e;
      if (yy >= TY) break;
      const int par = (y0 + yy) & 1, base = (e >> 1) + 2;  // (yy >> 1) + 2 - yb / 2
      lx[yy][c] = synth(s0, d0, par, base);
      hx[yy][c] = synth(s1, d1, par, base);
    }
  }
  __syncthreads();
  // Along x: thread -> row yy, E = min(8, TX) consecutive outputs (one byte
  // of bits at the last level, where S is a multiple of 8); the six input
  // columns they need are read once.
  const int E = min(8, TX), per_row = (TX + E - 1) / E;
  for (int i = threadIdx.x; i < TY * per_row; i += blockDim.x) {
    const int yy = i / per_row, xg = (i - yy * per_row) * E;
    const int y = y0 + yy;
    float2 sv[6], dv[6];
#pragma unroll
    for (int cc = 0; cc < 6; ++cc) {
      const int c = min(xg / 2 + cc, NX - 1);
      sv[cc] = lx[yy][c];
      dv[cc] = hx[yy][c];
    }
    float2 o[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      o[e] = make_float2(0.f, 0.f);
      if (e >= E || xg + e >= TX) continue;  // past the tile: no input columns
      o[e] = synth(sv, dv, (x0 + xg + e) & 1, (e >> 1) + 2);
    }
    const int x = x0 + xg;
    if (x >= S || y >= S || xg >= TX) continue;
    if (a.out) {
      if (E == 8 && x + 8 <= S) {
        float4* dst = reinterpret_cast<float4*>(a.out + (size_t)y * S + x);
#pragma unroll
        for (int e = 0; e < 4; ++e) dst[e] = make_float4(o[2 * e].x, o[2 * e].y, o[2 * e + 1].x, o[2 * e + 1].y);
      } else {
        for (int e = 0; e < E && x + e < S && xg + e < TX; ++e) a.out[(size_t)y * S + x + e] = o[e];
      }
    }
    if (a.bits) {  // last level: S is the side, a multiple of 8, and E == 8
      unsigned byte = 0;
#pragma unroll
      for (int e = 0; e < 8; ++e)
        if (ref_re(a.ref, o[e], (long long)a.ox + x + e, (long long)a.oy + y) > 0.f) byte |= 1u << e;
      a.bits[((size_t)y * S + x) >> 3] = (uint8_t)byte;
    }
  }
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

// Inverse of an L-level periodic order-1 coiflet transform of a tile-major
// wavelet buffer: levels L .. 1, each one pass (coif_level_kernel); the
// coarser levels' results alternate between a and b (dense, side >> (l - 1)
// a side); the last level writes the field (out) and/or the bits.
cudaError_t launch_coif_inverse(const float2* wbuf, int side, int L, float2* a, float2* b, float2* out,
                                uint8_t* bits, int ox, int oy, const RefDev& ref, cudaStream_t s) {
  double lo[6], hi[6];
  coif1_filters(lo, hi);
  CoifLevelArgs g;
  for (int i = 0; i < 6; ++i) { g.t.lo[i] = (float)lo[i]; g.t.hi[i] = (float)hi[i]; }
  g.wbuf = wbuf;
  g.side = side;
  g.L = L;
  g.ox = ox;
  g.oy = oy;
  g.ref = ref_dbf(ref);
  const float2* prev = nullptr;
  float2* bufs[2] = {a, b};
  for (int l = L; l >= 1; --l) {
    const int S = side >> (l - 1);
    g.l = l;
    g.prev = prev;
    g.out = l > 1 ? bufs[l & 1] : out;
    g.bits = l > 1 ? nullptr : bits;
    const int TX = std::min(kCoifTX, S), TY = std::min(kCoifTY, S);
    const dim3 grid((unsigned)((S + TX - 1) / TX), (unsigned)((S + TY - 1) / TY));
    if (S >= kCoifTX && S % kCoifTX == 0)
      coif_level_kernel<true><<<grid, 256, 0, s>>>(g);
    else
      coif_level_kernel<false><<<grid, 256, 0, s>>>(g);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    prev = g.out;
  }
  return cudaSuccess;
}

}  // namespace wsb

using namespace wsb;

extern "C" {

wasabi_status wasabi_inverse_wavelet_scratch_bytes(int holo_w, int holo_h, size_t* bytes_out) {
  if (holo_w <= 0 || holo_h <= 0 || !bytes_out) { set_error("inverse_wavelet_scratch_bytes: bad arguments"); return WASABI_E_INVALID; }
  *bytes_out = 2 * align256((size_t)holo_w * holo_h * sizeof(float2));
  return WASABI_OK;
}

wasabi_status wasabi_inverse_wavelet(const void* wbuf_dev, int holo_w, int holo_h, int levels, int wavelet,
                                     const wasabi_frame* frame, void* u_dev, uint8_t* bits_dev, void* scratch_dev,
                                     size_t scratch_bytes, void* stream) {
  if (wavelet == WASABI_HAAR)
    return wasabi_inverse_haar_frame(wbuf_dev, holo_w, holo_h, levels, frame, u_dev, bits_dev, stream);
  if (wavelet != WASABI_COIF1) { set_error("inverse_wavelet: unknown wavelet %d", wavelet); return WASABI_E_INVALID; }
  if (!wbuf_dev || (!u_dev && !bits_dev) || !scratch_dev) {
    set_error("inverse_wavelet: need the buffer, an output and scratch");
    return WASABI_E_INVALID;
  }
  if (levels < 1 || levels > kMaxLevels) { set_error("inverse_wavelet: levels must be in [1, %d]", kMaxLevels); return WASABI_E_INVALID; }
  const int ts = 1 << levels;
  if (holo_w != holo_h || holo_w < ts || holo_w % ts || (bits_dev && holo_w % 8)) {
    set_error("inverse_wavelet: the coiflet inverse needs a square hologram, side a multiple of 2^levels "
              "(and of 8 for bits)");
    return WASABI_E_INVALID;
  }
  if (((uintptr_t)wbuf_dev & 15) || ((uintptr_t)u_dev & 15) || ((uintptr_t)scratch_dev & 255)) {
    set_error("inverse_wavelet: misaligned buffer");
    return WASABI_E_INVALID;
  }
  int ox, oy;
  RefDev ref;
  const char* why = "";
  if (!frame_to_dev(frame, &ox, &oy, &ref, &why)) { set_error("inverse_wavelet: %s", why); return WASABI_E_INVALID; }
  // Plane pixel coordinates are exact in FP32 below 2^24.
  if (std::abs((long long)ox) + holo_w >= (1LL << 24) || std::abs((long long)oy) + holo_h >= (1LL << 24)) {
    set_error("inverse_wavelet: plane pixels must stay below 2^24 in magnitude");
    return WASABI_E_INVALID;
  }
  size_t need = 0;
  wasabi_inverse_wavelet_scratch_bytes(holo_w, holo_h, &need);
  if (scratch_bytes < need) {
    set_error("inverse_wavelet: scratch too small (%zu < %zu bytes)", scratch_bytes, need);
    return WASABI_E_NOMEM;
  }
  const cudaStream_t s = (cudaStream_t)stream;
  float2* a = static_cast<float2*>(scratch_dev);
  float2* b = reinterpret_cast<float2*>(static_cast<char*>(scratch_dev) + need / 2);
  const cudaError_t e = launch_coif_inverse(static_cast<const float2*>(wbuf_dev), holo_w, levels, a, b,
                                            static_cast<float2*>(u_dev), bits_dev, ox, oy, ref, s);
  return e == cudaSuccess ? WASABI_OK : cuda_fail("inverse_wavelet", e);
}

}  // extern "C"
