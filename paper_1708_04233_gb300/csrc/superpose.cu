// Superposition in the wavelet domain (Eq. (2)), owner-computes form, with
// the inverse transform and binarisation fused into its epilogue.
//
// The hologram is cut into super-tiles of T x T pixels (k = T / 2^L tiles a
// side).  Persistent CTAs claim super-tiles from a global counter; for each
// one a CTA
//   1. zeroes its shared-memory accumulator: one plane per kept (level, band)
//      covering the super-tile and a guard band one tile wide (levels finer
//      than the LUT's finest kept level are known to stay zero);
//   2. scans the binned points of the cell rows within reach and keeps the
//      survivors whose footprint (window-tile box of their depth, shifted,
//      plus one tile of carry) meets the super-tile; for each kept level it
//      folds the point's shift of Eq. (2) into one accumulator base;
//   3. cuts every survivor's LUT entries that can land in the super-tile into
//      passes of at most 64 consecutive entries: one LUT range per window-tile
//      row (contiguous by construction of the LUT), split every 64 entries.
//      Each thread loads the ranges of several rows at once, and each warp
//      reserves its passes with one shared-memory add (the list's order
//      varies, the exact fixed-point sums do not); a batch with more passes
//      than the list holds is numbered by a block-wide scan instead and
//      visited in windows;
//   4. deals the passes to the warps in groups of three, lane i visiting
//      entries i and i + 32 of a pass: one 8-byte record load (plane code,
//      value), the survivor's level base from shared memory, a_j * c, one
//      shared-memory add at base + code (no bounds test: coefficients that
//      land outside the super-tile fall into the guard band and are
//      dropped);
//   5. writes the finished super-tile once: to the tile-major wavelet buffer
//      (streaming vector stores, zeros for absent levels) and/or, through the
//      inverse transform in shared memory, as the complex field or the packed
//      binary hologram (each thread rebuilds 8 x 8 pixel blocks).
// Every output element is written exactly once: no global atomics and no
// zeroing pass.  Shared-memory atomics resolve collisions between survivors.
#include <algorithm>
#include <cstdlib>
#include <type_traits>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.cuh"

namespace wsb {
namespace {

constexpr int kMaxCellRows = 256;
constexpr int kPass = 64;         // LUT entries per pass (two per lane)
constexpr int kPassUnroll = 3;    // passes a warp has in flight, at most (see PU in the kernel)
constexpr int kSlotChunk = 4;     // LUT range slots a thread has in flight while building passes
constexpr int kRangeMin = 1024;   // pass capacity per window, at least
constexpr int kRangeMax = 8192;   // pass capacity per window, at most
constexpr int kSurvMax = 1024;    // survivors per candidate batch, at most
constexpr int kComplexTile = 192;  // default super-tile side (pixels) of complex accumulation
// Dynamic shared memory per CTA that still lets two CTAs share an SM (with
// the kernel's static shared memory and the per-CTA reservation).
constexpr size_t kTwoCtaSmem = 104 * 1024;
constexpr size_t kOneCtaSmem = 220 * 1024;

// Survivors per candidate batch for a pass capacity.
__host__ __device__ inline int survivor_cap(int rcap) {
  const int p = rcap / 2;
  return p < kSurvMax ? p : kSurvMax;
}

__device__ __forceinline__ int floor_div(int a, int b) {
  const int q = a / b;
  return (a % b != 0 && ((a < 0) != (b < 0))) ? q - 1 : q;
}

// Value of a reduced-precision LUT entry: the FP16 / BF16 pair (low half =
// real part) of its record word times its block's FP32 scale.
template <int DT>
__device__ __forceinline__ float2 decode16(uint32_t q, float s) {
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

// Exclusive scan over the block of one int per thread; returns the prefix and
// writes the total to *total (all threads).
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
  float2* acc;   // accumulator planes (plane_total cells: complex, or real parts only), see plane_code
  int4* sp;      // survivors: tile_off index of the first range, rows, tiles per row, amplitude bits
                 // (a_j times the fixed-point scale)
  int* sb;       // survivors x 8: at index l, the byte offset of level l's base cell minus (l << 29)
  int4* pass;    // passes: first LUT entry, entries, shared address of the survivor's sb row, amplitude bits
  int2* dbox;    // depths: tlo, thi
};

__host__ __device__ inline size_t smem_layout(int T, int L, int lmin, int D, bool re_only, int rcap, Smem* s,
                                              unsigned char* base) {
  const int k = T >> L;
  const int P = survivor_cap(rcap);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = (off + bytes + 15) & ~(size_t)15;
    return base ? base + o : nullptr;
  };
  unsigned char* p0 = take((size_t)plane_total(k, L, lmin) * (re_only ? sizeof(float) : sizeof(float2)));
  unsigned char* p1 = take((size_t)P * sizeof(int4));
  unsigned char* p2 = take((size_t)P * 8 * sizeof(int));
  unsigned char* p3 = take((size_t)(rcap + kPassUnroll) * sizeof(int4));  // + spare slots read past the end
  unsigned char* p4 = take((size_t)D * sizeof(int2));
  if (s) {
    s->acc = reinterpret_cast<float2*>(p0);
    s->sp = reinterpret_cast<int4*>(p1);
    s->sb = reinterpret_cast<int*>(p2);
    s->pass = reinterpret_cast<int4*>(p3);
    s->dbox = reinterpret_cast<int2*>(p4);
  }
  return off;
}

// Shared-memory accesses by 32-bit shared-window address (the hot loops keep
// their addresses in this form: one register, no generic-address arithmetic).
__device__ __forceinline__ unsigned sh_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ int lds32(unsigned a) {
  int v;
  asm volatile("ld.shared.b32 %0, [%1];" : "=r"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ int2 lds64(unsigned a) {
  int2 v;
  asm volatile("ld.shared.v2.b32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(a));
  return v;
}
__device__ __forceinline__ int4 lds128(unsigned a) {
  int4 v;
  asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a));
  return v;
}
// Shared-memory add without return, only where lane < n.
__device__ __forceinline__ void red_add_lt(unsigned a, int v, int lane, int n) {
  asm volatile("{\n .reg .pred q;\n setp.lt.s32 q, %2, %3;\n @q red.shared.add.s32 [%0], %1;\n}" ::"r"(a), "r"(v),
               "r"(lane), "r"(n));
}
__device__ __forceinline__ void red_add_lt(unsigned a, float v, int lane, int n) {
  asm volatile("{\n .reg .pred q;\n setp.lt.s32 q, %2, %3;\n @q red.shared.add.f32 [%0], %1;\n}" ::"r"(a), "f"(v),
               "r"(lane), "r"(n));
}
// Bit i of an 8-bit value moved to bit 4 i.
__device__ __forceinline__ unsigned spread_nibbles(unsigned x) {
  x = (x | (x << 12)) & 0x000f000fu;
  x = (x | (x << 6)) & 0x03030303u;
  x = (x | (x << 3)) & 0x11111111u;
  return x;
}

// Inverse transform (Sec. 1, step 3) and binarisation (Sec. 2) of a finished
// super-tile, straight from the shared-memory accumulator, in 4 x 4 pixel
// blocks: the form for the spherical-reference epilogue and for L = 2 (the
// 8 x 8 form below serves the others).  The wavelet buffer never goes to
// global memory.  Levels finer than lmin were never
// accumulated and read as zero.  Each thread rebuilds 4 x 4 pixel blocks in
// the add order of the separate inverse kernel, from the same FP32
// coefficient values that kernel would read, so the two paths give the same
// pixels.  Eight consecutive lanes cover 32 pixels of a row, which is one
// 32-bit word of the packed binary hologram (the super-tile side is a
// multiple of 32), and read neighbouring accumulator cells (no bank
// conflicts).  lvC[l], lvG[l], lvPS[l]: index of the level's first
// super-tile cell (past the guard), row stride and plane size.
// RE_ONLY (bits output alone): only real parts are read and transformed; the
// inverse transform acts on real and imaginary parts separately, so Re u is
// unchanged.  re_acc: the accumulator holds real parts only.
// REF: the bits are those of Re(u conj R) for the job's spherical reference
// wave R; ref_a: R's phase anchor at the super-tile's first pixel.
template <int L, bool RE_ONLY, bool REF>
__device__ __forceinline__ void supertile_inverse(const float2* acc, bool fixed, bool re_acc, float dq, int lmin, int k,
                                                  int kx, int ky, int Sx, int Sy, const JobDev& J,
                                                  const int* lvC, const int* lvG, const int* lvPS, int tid,
                                                  int NT, const RefAnchor* ref_a) {
  static_assert(!(RE_ONLY && REF), "a reference wave needs the imaginary parts");
  if constexpr (L >= 2) {
    const int bpr = (k << L) >> 2;           // 4 x 4 blocks per super-tile row
    const int total = bpr * ((ky << L) >> 2);
    const int xvalid = (kx << L) >> 2;       // block columns inside the hologram
    const int w = J.w;
    float2* u = J.u;
    uint8_t* bits = J.bits;
    const int lane = tid & 31;
    const int X0 = Sx << L, Y0 = Sy << L;
    const int xend = (Sx + kx) << L;
    const int* acci = reinterpret_cast<const int*>(acc);
    float rsg = 1.f;
    if constexpr (REF) rsg = J.ref.sgn;
    // Coefficient of level l, band plane bi, at super-tile cell (cx, cy).
    auto coef = [&](int l, int bi, int cx, int cy) -> float2 {
      if (l < lmin) return make_float2(0.f, 0.f);
      const int i = lvC[l] + bi * lvPS[l] + cy * lvG[l] + cx;
      // Bits alone: the fixed-point values are transformed unscaled.  Every
      // step is then exactly 2^sh times the scaled one (power-of-two scaling
      // commutes with the adds and halvings while values stay normal), so
      // the signs -- the bits -- are those of the scaled field.
      if (RE_ONLY) {
        const int wi = re_acc ? i : 2 * i;  // word of the real part
        return make_float2(fixed ? (float)acci[wi] : reinterpret_cast<const float*>(acc)[wi], 0.f);
      }
      if (fixed) {
        const int2 q = reinterpret_cast<const int2*>(acci)[i];
        return make_float2((float)q.x * dq, (float)q.y * dq);
      }
      return acc[i];
    };
    for (int b0 = 0; b0 < total; b0 += NT) {  // uniform trip count: whole warps shuffle
      const int b = b0 + tid;
      const int brow = b / bpr, bcol = b - brow * bpr;
      const bool inrow = b < total;
      const bool valid = inrow && bcol < xvalid;
      const int px0 = 4 * bcol, py0 = 4 * brow;  // block origin in the super-tile
      float2 s1[2][2] = {{make_float2(0.f, 0.f), make_float2(0.f, 0.f)}, {make_float2(0.f, 0.f), make_float2(0.f, 0.f)}};
      if (valid) {  // the block's four level-1 scaling values
        // Levels L .. 3: the block lies inside one level-(l-1) cell.
        float2 s = coef(L, 0, px0 >> L, py0 >> L);
#pragma unroll
        for (int l = L; l >= 3; --l) {
          const int cx = px0 >> l, cy = py0 >> l;
          const int bi = l == L ? 1 : 0;  // plane of band 1 at this level
          const float2 lh = coef(l, bi, cx, cy), hl = coef(l, bi + 1, cx, cy), hh = coef(l, bi + 2, cx, cy);
          s = ipick(s, lh, hl, hh, (px0 >> (l - 1)) & 1, (py0 >> (l - 1)) & 1);
        }
        // Level 2 at the block's own cell -> four level-1 scaling values.
        const int b2 = L == 2 ? 1 : 0;
        const float2 lh = coef(2, b2, px0 >> 2, py0 >> 2), hl = coef(2, b2 + 1, px0 >> 2, py0 >> 2),
                     hh = coef(2, b2 + 2, px0 >> 2, py0 >> 2);
#pragma unroll
        for (int ay = 0; ay < 2; ++ay)
#pragma unroll
          for (int ax = 0; ax < 2; ++ax) s1[ay][ax] = ipick(s, lh, hl, hh, ax, ay);
      }
      const int x0 = X0 + px0;
      const int xw = X0 + 32 * (bcol >> 3);  // first pixel of this lane group's bit word
      RefBlock RB;
      if constexpr (REF) RB = ref_block(J.ref, *ref_a, px0, py0);  // anchor re-read from shared memory
      // One pixel row of the block: complex values, and its bit word (eight
      // lanes OR their nibbles into the word at xw).
      auto put_u = [&](int y, float2 p0, float2 p1, float2 p2, float2 p3) {
        if (!RE_ONLY && u != nullptr && valid) {
          float4* dst = reinterpret_cast<float4*>(u + (size_t)y * w + x0);
          __stcs(dst, make_float4(p0.x, p0.y, p1.x, p1.y));
          __stcs(dst + 1, make_float4(p2.x, p2.y, p3.x, p3.y));
        }
      };
      auto word = [&](float r0, float r1, float r2, float r3) -> unsigned {
        unsigned nib = 0;
        if (valid) nib = (r0 > 0.f ? 1u : 0u) | (r1 > 0.f ? 2u : 0u) | (r2 > 0.f ? 4u : 0u) | (r3 > 0.f ? 8u : 0u);
        unsigned v = nib << (4 * (lane & 7));
        v |= __shfl_xor_sync(0xffffffffu, v, 1);
        v |= __shfl_xor_sync(0xffffffffu, v, 2);
        v |= __shfl_xor_sync(0xffffffffu, v, 4);
        return v;
      };
      auto put_bits = [&](int y, unsigned v) {
        if ((lane & 7) == 0 && inrow && xw < xend) {
          const size_t byte0 = ((size_t)y * w + xw) >> 3;
          if (xw + 32 <= xend && (w & 31) == 0) {
            *reinterpret_cast<unsigned*>(bits + byte0) = v;
          } else {
            const int nb = min(4, (xend - xw) >> 3);
            for (int q = 0; q < nb; ++q) bits[byte0 + q] = (uint8_t)(v >> (8 * q));
          }
        }
      };
      const int y0 = Y0 + py0;
      if (lmin >= 2) {
        // No level-1 details: the level-1 step gives s1 / 2 for all four
        // pixels of each 2 x 2 group (the same values, up to the sign of a
        // zero, as the step with zero details).
#pragma unroll
        for (int ay = 0; ay < 2; ++ay) {
          float2 pa = make_float2(0.f, 0.f), pb = pa;
          if (valid) {
            pa = make_float2(s1[ay][0].x * 0.5f, s1[ay][0].y * 0.5f);
            pb = make_float2(s1[ay][1].x * 0.5f, s1[ay][1].y * 0.5f);
          }
          put_u(y0 + 2 * ay, pa, pa, pb, pb);
          put_u(y0 + 2 * ay + 1, pa, pa, pb, pb);
          if (REF && bits != nullptr) {
#pragma unroll
            for (int qy = 0; qy < 2; ++qy) {
              const int j = 2 * ay + qy;
              put_bits(y0 + j, word(ref_value(RB, rsg, pa, 0, j), ref_value(RB, rsg, pa, 1, j),
                                    ref_value(RB, rsg, pb, 2, j), ref_value(RB, rsg, pb, 3, j)));
            }
          } else if (bits != nullptr) {
            // Both rows of the pair are equal, and each level-1 value covers
            // two neighbouring pixels: two warp votes give the signs of the
            // warp's 64 values; lane group q (8 lanes, 32 pixels) owns byte q
            // of each vote, spread to one bit per nibble and doubled.
            const unsigned va = __ballot_sync(0xffffffffu, valid && pa.x > 0.f);
            const unsigned vb = __ballot_sync(0xffffffffu, valid && pb.x > 0.f);
            const int q = (lane >> 3) * 8;
            const unsigned v = spread_nibbles((va >> q) & 0xffu) * 3u | (spread_nibbles((vb >> q) & 0xffu) * 3u) << 2;
            put_bits(y0 + 2 * ay, v);
            put_bits(y0 + 2 * ay + 1, v);
          }
        }
      } else {
        // Level 1, one pair of pixel rows at a time -> 2 x 4 pixels.
#pragma unroll
        for (int ay = 0; ay < 2; ++ay) {
          float2 px[2][4];
#pragma unroll
          for (int ax = 0; ax < 2; ++ax) {
            float2 l1 = make_float2(0.f, 0.f), h1 = l1, d1 = l1;
            if (valid) {
              const int cx = (px0 >> 1) + ax, cy = (py0 >> 1) + ay;
              l1 = coef(1, 0, cx, cy);
              h1 = coef(1, 1, cx, cy);
              d1 = coef(1, 2, cx, cy);
            }
#pragma unroll
            for (int qy = 0; qy < 2; ++qy)
#pragma unroll
              for (int qx = 0; qx < 2; ++qx) px[qy][2 * ax + qx] = ipick(s1[ay][ax], l1, h1, d1, qx, qy);
          }
#pragma unroll
          for (int qy = 0; qy < 2; ++qy) {
            put_u(y0 + 2 * ay + qy, px[qy][0], px[qy][1], px[qy][2], px[qy][3]);
            if (REF && bits != nullptr) {
              const int j = 2 * ay + qy;
              put_bits(y0 + j, word(ref_value(RB, rsg, px[qy][0], 0, j), ref_value(RB, rsg, px[qy][1], 1, j),
                                    ref_value(RB, rsg, px[qy][2], 2, j), ref_value(RB, rsg, px[qy][3], 3, j)));
            } else if (bits != nullptr) {
              put_bits(y0 + 2 * ay + qy, word(px[qy][0].x, px[qy][1].x, px[qy][2].x, px[qy][3].x));
            }
          }
        }
      }
    }
  }
}



__device__ __forceinline__ float ipv(float s, float lh, float hl, float hh, int ax, int ay) {
  return ipick1(s, lh, hl, hh, ax, ay);
}
__device__ __forceinline__ float2 ipv(float2 s, float2 lh, float2 hl, float2 hh, int ax, int ay) {
  return ipick(s, lh, hl, hh, ax, ay);
}
__device__ __forceinline__ float re_of(float v) { return v; }
__device__ __forceinline__ float re_of(float2 v) { return v.x; }
__device__ __forceinline__ float half_of(float v) { return v * 0.5f; }
__device__ __forceinline__ float2 half_of(float2 v) { return make_float2(v.x * 0.5f, v.y * 0.5f); }
template <bool R>
struct EpiVal { using T = float2; };
template <>
struct EpiVal<true> { using T = float; };

// Inverse transform (Sec. 1, step 3) and binarisation (Sec. 2) of a finished
// super-tile in 8 x 8 pixel blocks (L >= 3, plane reference), one block per
// thread: the block's level-3 scaling value from the coarser levels along its
// path, the level-3 details give four level-2 scaling values, the level-2
// details sixteen level-1 values, and the level-1 details (when kept) the 64
// pixels.  Every step is the separate inverse kernel's (ipick, same add
// order, same FP32 inputs), so the pixels equal that kernel's; levels finer
// than lmin were never accumulated and read as zero (with no level-1 details
// each level-1 value s gives s / 2 to its four pixels).  Four consecutive
// lanes hold four neighbouring blocks: their rows of eight bits form one
// 32-bit word of the packed hologram.
// RE_ONLY (bits alone): real parts only, transformed unscaled from the
// fixed-point integers (power-of-two scaling commutes with the adds and
// halvings, so the signs are those of the scaled field); re_acc: the
// accumulator holds real parts only.  Otherwise complex values go to u and/or
// are binarised.
// KC > 0: the form for super-tiles of k = KC tiles with fixed-point sums and
// lmin = LMC (the caller checks), the layout then known at compile time.
template <int L, bool RE_ONLY, int KC = 0, int LMC = 0>
__device__ __forceinline__ void supertile_inverse8(const float2* acc, bool fixed, bool re_acc, float dq, int lmin,
                                                   int k, int kx, int ky, int Sx, int Sy, const JobDev& J,
                                                   const int* lvC, const int* lvG, const int* lvPS, int tid,
                                                   int NT) {
  static_assert(L >= 3, "8 x 8 blocks need at least three levels");
  using V = typename EpiVal<RE_ONLY>::T;
  int C[L + 1], G[L + 1], PS[L + 1];
  if constexpr (KC > 0) {
    fixed = true;
    lmin = LMC;
    k = KC;
  }
#pragma unroll
  for (int l = 1; l <= L; ++l) {
    if constexpr (KC > 0) {
      C[l] = plane_first(KC, L, LMC, l);
      G[l] = plane_row(KC, L, l);
      PS[l] = plane_size(KC, L, l);
    } else {
      C[l] = lvC[l];
      G[l] = lvG[l];
      PS[l] = lvPS[l];
    }
  }
  const unsigned acc_s = sh_addr(acc);
  auto zero = []() -> V {
    if constexpr (RE_ONLY) return 0.f;
    else return make_float2(0.f, 0.f);
  };
  // Coefficient of level l, band plane pl, at super-tile cell (cx, cy).
  auto coef = [&](int l, int pl, int cx, int cy) -> V {
    if (l < lmin) return zero();
    const unsigned i = (unsigned)(C[l] + pl * PS[l] + cy * G[l] + cx);
    if constexpr (RE_ONLY) {
      const int q = lds32(acc_s + (re_acc ? 4u : 8u) * i);  // word of the real part
      return fixed ? (float)q : __int_as_float(q);
    } else {
      const int2 q = lds64(acc_s + 8u * i);
      if (fixed) return make_float2((float)q.x * dq, (float)q.y * dq);
      return make_float2(__int_as_float(q.x), __int_as_float(q.y));
    }
  };
  const int bpr = (k << L) >> 3;  // 8 x 8 blocks per super-tile row
  const int total = bpr * ((ky << L) >> 3);
  const int xvalid = (kx << L) >> 3;
  const int X0 = Sx << L, Y0 = Sy << L, xend = (Sx + kx) << L;
  const int w = J.w;
  float2* u = J.u;
  uint8_t* bits = J.bits;
  const int lane = tid & 31;
  for (int b0 = 0; b0 < total; b0 += NT) {  // uniform trip count: whole warps shuffle
    const int b = b0 + tid;
    const int brow = b / bpr, bcol = b - brow * bpr;
    const bool inrow = b < total;
    const bool valid = inrow && bcol < xvalid;
    const int px0 = 8 * bcol, py0 = 8 * brow;
    V s3 = zero(), lh3 = zero(), hl3 = zero(), hh3 = zero();
    if (valid) {
      s3 = coef(L, 0, px0 >> L, py0 >> L);
#pragma unroll
      for (int l = L; l >= 4; --l) {
        const int cx = px0 >> l, cy = py0 >> l, pl = l == L ? 1 : 0;
        s3 = ipv(s3, coef(l, pl, cx, cy), coef(l, pl + 1, cx, cy), coef(l, pl + 2, cx, cy), (px0 >> (l - 1)) & 1,
                 (py0 >> (l - 1)) & 1);
      }
      const int pl3 = L == 3 ? 1 : 0;
      lh3 = coef(3, pl3, bcol, brow);
      hl3 = coef(3, pl3 + 1, bcol, brow);
      hh3 = coef(3, pl3 + 2, bcol, brow);
    }
    const int xw = X0 + 32 * (bcol >> 2);  // first pixel of this lane group's bit word
    const int x0 = X0 + px0;
    // One bit word per pixel row: the four lanes' bytes, row y written by one lane.
    auto put_bits = [&](int y, unsigned byte, int r) {
      unsigned v = byte << (8 * (lane & 3));
      v |= __shfl_xor_sync(0xffffffffu, v, 1);
      v |= __shfl_xor_sync(0xffffffffu, v, 2);
      if ((lane & 3) == (r & 3) && inrow && xw < xend) {
        const size_t byte0 = ((size_t)y * w + xw) >> 3;
        if (xw + 32 <= xend && (w & 31) == 0) {
          *reinterpret_cast<unsigned*>(bits + byte0) = v;
        } else {
          const int nb = min(4, (xend - xw) >> 3);
          for (int q = 0; q < nb; ++q) bits[byte0 + q] = (uint8_t)(v >> (8 * q));
        }
      }
    };
#pragma unroll
    for (int ay = 0; ay < 2; ++ay) {
      V s1[2][4];
#pragma unroll
      for (int ax = 0; ax < 2; ++ax) {
        const V s2 = ipv(s3, lh3, hl3, hh3, ax, ay);
        V l2 = zero(), h2 = zero(), d2 = zero();
        if (valid) {
          const int cx = 2 * bcol + ax, cy = 2 * brow + ay;
          l2 = coef(2, 0, cx, cy);
          h2 = coef(2, 1, cx, cy);
          d2 = coef(2, 2, cx, cy);
        }
#pragma unroll
        for (int qy = 0; qy < 2; ++qy)
#pragma unroll
          for (int qx = 0; qx < 2; ++qx) s1[qy][2 * ax + qx] = ipv(s2, l2, h2, d2, qx, qy);
      }
      if constexpr (RE_ONLY) {
        if (lmin >= 2) {
          // No level-1 details: both pixel rows of level-1 row j are the signs
          // of s1[.][0..3] / 2, each covering two pixels (the halving does not
          // change a sign: the values are integers, or FP32 sums far from the
          // subnormal range).  One word per pair of rows.
#pragma unroll
          for (int qy = 0; qy < 2; ++qy) {
            const int j = 2 * ay + qy;
            unsigned b4 = 0;
            if (valid) {
#pragma unroll
              for (int i = 0; i < 4; ++i) b4 |= (s1[qy][i] > 0.f ? 1u : 0u) << i;
            }
            const unsigned byte = (b4 & 1u) * 3u | (b4 & 2u) * 6u | (b4 & 4u) * 12u | (b4 & 8u) * 24u;
            unsigned v = byte << (8 * (lane & 3));
            v |= __shfl_xor_sync(0xffffffffu, v, 1);
            v |= __shfl_xor_sync(0xffffffffu, v, 2);
            if ((lane & 3) == j && inrow && xw < xend) {
              const int y = Y0 + py0 + 2 * j;
#pragma unroll
              for (int ry = 0; ry < 2; ++ry) {
                const size_t byte0 = ((size_t)(y + ry) * w + xw) >> 3;
                if (xw + 32 <= xend && (w & 31) == 0) {
                  *reinterpret_cast<unsigned*>(bits + byte0) = v;
                } else {
                  const int nb = min(4, (xend - xw) >> 3);
                  for (int q = 0; q < nb; ++q) bits[byte0 + q] = (uint8_t)(v >> (8 * q));
                }
              }
            }
          }
          continue;
        }
      }
#pragma unroll
      for (int qy = 0; qy < 2; ++qy) {
        const int j = 2 * ay + qy;         // level-1 row of the block: pixel rows 2j, 2j + 1
        const int y = Y0 + py0 + 2 * j;
        unsigned byte[2] = {0u, 0u};
#pragma unroll
        for (int i = 0; i < 4; ++i) {      // level-1 column: pixels 2i, 2i + 1
          V p[2][2];
          if (lmin >= 2) {
            const V h = half_of(s1[qy][i]);
            p[0][0] = p[0][1] = p[1][0] = p[1][1] = h;
          } else {
            V l1 = zero(), h1 = zero(), d1 = zero();
            if (valid) {
              const int cx = 4 * bcol + i, cy = 4 * brow + j;
              l1 = coef(1, 0, cx, cy);
              h1 = coef(1, 1, cx, cy);
              d1 = coef(1, 2, cx, cy);
            }
#pragma unroll
            for (int ry = 0; ry < 2; ++ry)
#pragma unroll
              for (int rx = 0; rx < 2; ++rx) p[ry][rx] = ipv(s1[qy][i], l1, h1, d1, rx, ry);
          }
#pragma unroll
          for (int ry = 0; ry < 2; ++ry) {
            if constexpr (!RE_ONLY) {
              if (u != nullptr && valid)
                __stcs(reinterpret_cast<float4*>(u + (size_t)(y + ry) * w + x0 + 2 * i),
                       make_float4(p[ry][0].x, p[ry][0].y, p[ry][1].x, p[ry][1].y));
            }
            if (valid)
              byte[ry] |= (re_of(p[ry][0]) > 0.f ? 1u : 0u) << (2 * i) | (re_of(p[ry][1]) > 0.f ? 1u : 0u)
                                                                         << (2 * i + 1);
          }
        }
        if (bits != nullptr) {
          put_bits(y, byte[0], 2 * j);
          put_bits(y + 1, byte[1], 2 * j + 1);
        }
      }
    }
  }
}

// Kernel modes: complex accumulation; real parts only (every job of the
// launch wants bits alone with R = 1); complex accumulation with the
// reference-wave epilogue compiled in (a launch where some job binarises
// against a spherical R -- a kernel of its own, so that the other two keep
// their register allocation).
constexpr int kModeComplex = 0, kModeRe = 1, kModeRef = 2;

template <int L, int DT, int MODE>
__global__ void __launch_bounds__(1024, 1) superpose_kernel(SuperposeArgs a) {
  constexpr int TSL = 1 << (2 * L);
  extern __shared__ __align__(16) unsigned char smem[];
  const int T = a.cell;
  const int k = T >> L;
  constexpr bool RE = MODE == kModeRe;
  constexpr bool re_acc = RE;
  // Passes a warp has in flight: three where the registers allow it (FP32
  // LUT, plane reference, three or more levels), else two.
  constexpr int PU = (MODE == kModeRef || DT != WASABI_F32 || L <= 2) ? 2 : kPassUnroll;
  const int rcap = a.rcap;
  const int P = survivor_cap(rcap);
  const int lmin = a.lut.lmin;
  const int NA = plane_total(k, L, lmin);  // accumulator size (cells)
  Smem S;
  smem_layout(T, L, lmin, a.lut.D, re_acc, rcap, &S, smem);
  const int NW = NA * (re_acc ? 1 : 2);  // accumulator words (a multiple of 4)
  __shared__ int s_st, s_n, s_np, s_rmax, s_total;
  __shared__ int warp_buf[32];
  __shared__ int s_rowstart[kMaxCellRows], s_rowpre[kMaxCellRows + 1];
  // Per level l: index of the first super-tile cell past the guard, row
  // stride, plane size (see plane_code).
  __shared__ int lvC[8], lvG[8], lvPS[8];
  __shared__ RefAnchor s_ref;  // reference-wave phase anchor of the current super-tile

  const LutView& lut = a.lut;
  const int NT = blockDim.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = NT >> 5;
  const int W2 = lut.W / 2;
  const int ntpd = lut.nwt * lut.nwt + 1;  // tile_off entries per depth
  __shared__ int s_sp0[kMaxJobs];
  const int nj = min(a.batch->njobs, kMaxJobs), nsp = a.batch->nsp;
  for (int j = tid; j < nj; j += NT) s_sp0[j] = a.jobs[j].sp0;
  for (int d = tid; d < lut.D; d += NT) {
    const DepthMeta m = lut.meta[d];
    S.dbox[d] = make_int2(m.tlo, m.thi);
  }
  if (tid == 0) {
    for (int l = L; l >= 1; --l) {
      lvG[l] = plane_row(k, L, l);
      lvPS[l] = plane_size(k, L, l);
      lvC[l] = plane_first(k, L, lmin, l);
    }
  }
  int* counter = &a.batch->counter;
  const float cmax = __ldg(lut.cmax);
  float4* acc4 = reinterpret_cast<float4*>(S.acc);
  const bool fixed = !a.acc_float;
  int next = 0;  // thread 0: the item claimed for the next iteration
  if (tid == 0) next = atomicAdd(counter, 1);

  for (;;) {
    __syncthreads();
    if (tid == 0) {
      s_st = next;
      next = atomicAdd(counter, 1);  // claim the next item early
    }
    __syncthreads();
    const int item = s_st;
    if (item >= nsp) break;
    // Item -> (job, super-tile).
    const JobDev& J = a.jobs[job_of(s_sp0, nj, item)];
    const int ntx = J.ntx, nty = J.nty, ncx = J.ncx, ncy = J.ncy;
    const int half = J.rule == WASABI_SHIFT_FLOOR ? 0 : 1;
    const int* cell_off = J.off;
    const wasabi_point* sorted = J.sorted;
    float2* wbuf = J.wbuf;
    const int nstx = (ntx + k - 1) / k;
    const int st = item - J.sp0;
    const int Sx = (st % nstx) * k, Sy = (st / nstx) * k;
    const int kx = min(k, ntx - Sx), ky = min(k, nty - Sy);

    // Cell rows within reach of the super-tile, one thread per row; their
    // offsets are loaded before the accumulator is zeroed, so the zeroing
    // covers the load latency.
    const int X0 = Sx << L, X1 = (Sx + kx) << L, Y0 = Sy << L, Y1 = (Sy + ky) << L;
    if (MODE == kModeRef && tid == 0 && J.ref.kind != 0 && J.bits != nullptr)  // read after the syncs below
      s_ref = ref_anchor(J.ref, (long long)J.ox + X0, (long long)J.oy + Y0);
    const int cx0 = max(0, floor_div(X0 - a.reach, a.cell));
    const int cx1 = min(ncx - 1, floor_div(X1 - 1 + a.reach, a.cell));
    const int cy0 = max(0, floor_div(Y0 - a.reach, a.cell));
    const int cy1 = min(ncy - 1, floor_div(Y1 - 1 + a.reach, a.cell));
    const int ncrows = (cx0 <= cx1 && cy0 <= cy1) ? cy1 - cy0 + 1 : 0;
    int row_s0 = 0, row_s1 = 0;
    if (tid < ncrows) {
      const int c0 = (cy0 + tid) * ncx;
      row_s0 = __ldg(&cell_off[c0 + cx0]);
      row_s1 = __ldg(&cell_off[c0 + cx1 + 1]);
    }
    for (int i = tid; i < NW / 4; i += NT) acc4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (tid < ncrows) {
      s_rowstart[tid] = row_s0;
      s_rowpre[tid] = row_s1 - row_s0;
    }
    __syncthreads();
    if (warp == 0) {  // exclusive prefix over <= kMaxCellRows rows, RPL per lane
      constexpr int RPL = kMaxCellRows / 32;
      int v[RPL], loc = 0;
#pragma unroll
      for (int j = 0; j < RPL; ++j) {
        const int r = RPL * lane + j;
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
      for (int j = 0; j < RPL; ++j) {
        const int r = RPL * lane + j;
        if (r < ncrows) s_rowpre[r] = run;
        run += v[j];
      }
      if (lane == 31) s_total = incl;
    }
    __syncthreads();
    const int total = s_total;
    // Fixed-point scale 2^sh: every partial sum stays below 2^31 in magnitude.
    const float bound = (float)total * (J.amax * cmax);
    const int sh = bound > 0.f ? max(-100, min(30, (int)floorf(log2f(2.0e9f / bound)))) : 30;
    const float qs = __int_as_float((sh + 127) << 23);  // 2^sh (-100 <= sh <= 30)

    const int CH = min(P, NT);  // candidates per batch: at most one per thread
    for (int c0 = 0; c0 < total; c0 += CH) {
      // ---- survivors of this batch of candidates
      if (tid == 0) {
        s_n = 0;
        s_np = 0;
        s_rmax = 1;
      }
      __syncthreads();
      if (tid < CH && c0 + tid < total) {
        const int i = c0 + tid;
        const int r = last_le(s_rowpre, 0, ncrows - 1, i);
        const int4 p = __ldg(reinterpret_cast<const int4*>(sorted) + s_rowstart[r] + (i - s_rowpre[r]));
        const int2 bx = S.dbox[p.w];
        const int X = p.x - W2, Y = p.y - W2;
        const int Ax = X >> L, Ay = Y >> L;  // arithmetic shifts: floor division
        if (Ax + bx.x <= Sx + kx - 1 && Ax + bx.y + 1 >= Sx && Ay + bx.x <= Sy + ky - 1 &&
            Ay + bx.y + 1 >= Sy) {
          const int s = atomicAdd(&s_n, 1);
          const float amp = __int_as_float(p.z) * (fixed ? qs : 1.0f);
          // The survivor's window tiles that can land in the super-tile (its
          // depth's tile box shifted by (Ax, Ay), one tile of carry): rows
          // tya .. tyb, columns txa .. txb; one LUT range per row.
          const int tya = max(bx.x, Sy - Ay - 1), tyb = min(bx.y, Sy + ky - 1 - Ay);
          const int txa = max(bx.x, Sx - Ax - 1), txb = min(bx.y, Sx + kx - 1 - Ax);
          const int rows = txa <= txb ? max(0, tyb - tya + 1) : 0;
          S.sp[s] = make_int4(p.w * ntpd + tya * lut.nwt + txa, rows, txb - txa + 1, __float_as_int(amp));
          atomicMax(&s_rmax, rows);
          // shift_l(X) of Eq. (2): floor((X + half * 2^(l-1)) / 2^l), made
          // relative to the super-tile origin in level-l units, folded with
          // the level's accumulator offset into one base per level (minus
          // the level bits of the plane codes it is added to), plus the
          // accumulator's shared address (halved for complex cells, whose
          // word offsets are doubled).
          const unsigned acc0 = sh_addr(S.acc) >> (re_acc ? 0 : 1);
          for (int l = lmin; l <= L; ++l) {
            const int hb = half << (l - 1);
            const int ox = ((X + hb) >> l) - (Sx << (L - l)), oy = ((Y + hb) >> l) - (Sy << (L - l));
            S.sb[s * 8 + l] = (int)(acc0 + 4u * (unsigned)(lvC[l] + oy * lvG[l] + ox) - ((unsigned)l << 29));
          }
        }
      }
      __syncthreads();
      const int n = s_n;
      // ---- slot f = s * K1 + j is window-tile row j of the survivor's
      // clipped tile box (K1: the batch's most rows, at most k + 1).
      const int K1 = s_rmax;
      const int nslot = n * K1;
      const unsigned sp_s = sh_addr(S.sp), sb_s = sh_addr(S.sb), pass_s = sh_addr(S.pass);
      // Walks this thread's slots t, t + NT, t + 2 NT, ... kSlotChunk at a
      // time, the LUT range loads of a chunk in flight together, and calls
      // fn(st, ln, sv, am, np) per chunk with each slot's first entry, entry
      // count, survivor and amplitude bits (empty slots: no entries), np the
      // chunk's passes; fn returns false to stop.  While fn returns true the
      // trip count is the same for every thread.
      auto walk_slots = [&](auto&& fn) {
        // tid / K1 and NT / K1 in FP32: n + 1/2 is exact and the product's
        // relative error is below 2^-23, so for n <= 1024 and K1 <= 257 it
        // stays under the 1 / (2 K1) that separates n / K1 + 1 / (2 K1) from
        // the next integer.
        const float rk = __frcp_rn((float)K1);
        int s = __float2int_rz(((float)tid + 0.5f) * rk), j = tid - s * K1;
        const int ds = __float2int_rz(((float)NT + 0.5f) * rk), dj = NT - ds * K1;
        for (int f0 = 0; f0 < nslot; f0 += kSlotChunk * NT) {
          int st[kSlotChunk], ln[kSlotChunk], sv[kSlotChunk], am[kSlotChunk];
#pragma unroll
          for (int c = 0; c < kSlotChunk; ++c) {
            st[c] = 0;
            ln[c] = 0;
            sv[c] = s;
            am[c] = 0;
            if (f0 + c * NT + tid < nslot) {
              const int4 sp = lds128(sp_s + 16u * s);
              if (j < sp.y) {
                const int* to = lut.tile_off + sp.x + j * lut.nwt;
                st[c] = __ldg(to);
                ln[c] = __ldg(to + sp.z);
              }
              am[c] = sp.w;
            }
            s += ds;
            j += dj;
            if (j >= K1) {
              j -= K1;
              ++s;
            }
          }
          int np = 0;
#pragma unroll
          for (int c = 0; c < kSlotChunk; ++c) {
            ln[c] -= st[c];
            np += (int)((unsigned)(ln[c] + kPass - 1) / kPass);  // ln >= 0
          }
          if (!fn(st, ln, sv, am, np)) break;
        }
      };
      // ---- visits: warp w takes groups w, w + warps, ... of the ng groups
      // of PU passes; a group's records and LUT loads are all
      // issued before any is consumed.  Lane i visits entries i, i + 32, ...
      // of each pass; lanes past a pass's end load the records that follow
      // (a code array is followed by the next one or by kCodePad records of
      // padding) and add nothing.
      auto visit = [&](auto fixed_tag, int ng) {
          constexpr bool FX = decltype(fixed_tag)::value;
          constexpr int EPL = kPass / 32;  // entries per lane and pass
          for (int g = warp; g < ng; g += nwarps) {
            uint2 rec[PU][EPL];
            float vy[PU][EPL];  // FP32 imaginary part (complex accumulation), or the block scale
            unsigned sbo[PU];
            float amp[PU];
            int cnt[PU];
#pragma unroll
            for (int u = 0; u < PU; ++u) {
              const int4 r = lds128(pass_s + 16u * (PU * g + u));
              cnt[u] = r.y;
              sbo[u] = (unsigned)r.z;
              amp[u] = __int_as_float(r.w);
#pragma unroll
              for (int h = 0; h < EPL; ++h) {
                const int e = r.x + lane + 32 * h;
                rec[u][h] = __ldg(&lut.code[e]);
                if (DT != WASABI_F32) vy[u][h] = __ldg(&lut.scale[e >> 5]);
                else if (!re_acc) vy[u][h] = __ldg(&lut.val[e].y);
              }
            }
#pragma unroll
            for (int u = 0; u < PU; ++u) {
#pragma unroll
              for (int h = 0; h < EPL; ++h) {
                const int li = lane + 32 * h;
                const uint2 pe = rec[u][h];
                const float2 v = DT == WASABI_F32 ? make_float2(__uint_as_float(pe.y), vy[u][h])
                                                  : decode16<DT>(pe.y, vy[u][h]);
                // Shared address of the accumulator word (halved for complex
                // cells): plane code plus the survivor's base of the code's
                // level (which carries minus the level bits).
                const unsigned ab = pe.x + (unsigned)lds32(sbo[u] + 4u * (pe.x >> 29));
                // a_j c in FP32; in fixed point exactly scaled by 2^sh (folded
                // into amp) and rounded to the nearest integer: the integer
                // sums are exact.
                if constexpr (re_acc) {
                  if constexpr (FX) red_add_lt(ab, __float2int_rn(amp[u] * v.x), li, cnt[u]);
                  else red_add_lt(ab, amp[u] * v.x, li, cnt[u]);
                } else {
                  const unsigned a2 = 2u * ab;
                  if constexpr (FX) {
                    red_add_lt(a2, __float2int_rn(amp[u] * v.x), li, cnt[u]);
                    red_add_lt(a2 + 4u, __float2int_rn(amp[u] * v.y), li, cnt[u]);
                  } else {
                    red_add_lt(a2, amp[u] * v.x, li, cnt[u]);
                    red_add_lt(a2 + 4u, amp[u] * v.y, li, cnt[u]);
                  }
                }
              }
            }
          }
        };
      auto pad_visit = [&](int np) {
        // The last group is filled with empty passes (no entries; their
        // loaded entries are entry 0 and their level bases those of survivor 0).
        const int ng = (np + PU - 1) / PU;
        if (tid < ng * PU - np) S.pass[np + tid] = make_int4(1, 0, (int)sb_s, 0);
        __syncthreads();
        if (fixed) visit(std::true_type{}, ng);
        else visit(std::false_type{}, ng);
        __syncthreads();
      };
      // ---- passes, one walk: a warp reserves its passes with one
      // shared-memory add and stores those that fit in the list.  The list's
      // order varies from run to run; the fixed-point sums do not depend on
      // it.  A thread's reservations grow along its slot order, so the passes
      // it has stored are the first `done` of its sequence of `total`.
      int done = 0, total = 0;
      walk_slots([&](const int* st, const int* ln, const int* sv, const int* am, int np) {
        int incl = np;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += y;
        }
        const int wtot = __shfl_sync(0xffffffffu, incl, 31);
        int wb = 0;
        if (lane == 0 && wtot > 0) wb = atomicAdd(&s_np, wtot);
        int pi = __shfl_sync(0xffffffffu, wb, 0) + incl - np;
        done += max(0, min(np, rcap - pi));
        total += np;
#pragma unroll
        for (int c = 0; c < kSlotChunk; ++c)
          for (int o = 0; o < ln[c]; o += kPass, ++pi)
            if (pi < rcap) S.pass[pi] = make_int4(st[c] + o, min(kPass, ln[c] - o), (int)(sb_s + 32u * sv[c]), am[c]);
        return true;
      });
      __syncthreads();
      const int nres = s_np;
      pad_visit(min(nres, rcap));
      if (nres > rcap) {
        // The passes that did not fit: a block-wide scan numbers each
        // thread's rest, and every list of rcap of them is written by the
        // threads whose numbers meet it (walking up to the list's end), then
        // visited.
        const int rest = total - done;
        int nrest;
        const int pbase = block_scan(rest, &nrest, warp_buf);
        for (int w0 = 0; w0 < nrest; w0 += rcap) {
          if (rest > 0 && pbase < w0 + rcap && pbase + rest > w0) {
            int pi = pbase - done;  // number of the sequence's first pass (the stored ones fall below pbase)
            walk_slots([&](const int* st, const int* ln, const int* sv, const int* am, int np) {
              if (pi + np > max(pbase, w0)) {
                int q = pi;
#pragma unroll
                for (int c = 0; c < kSlotChunk; ++c)
                  for (int o = 0; o < ln[c]; o += kPass, ++q)
                    if (q >= pbase && q >= w0 && q < w0 + rcap)
                      S.pass[q - w0] = make_int4(st[c] + o, min(kPass, ln[c] - o), (int)(sb_s + 32u * sv[c]), am[c]);
              }
              pi += np;
              return pi < w0 + rcap;
            });
          }
          pad_visit(min(rcap, nrest - w0));
        }
      }
    }


    const float dq = __int_as_float((127 - sh) << 23);  // 2^-sh
    // Write the super-tile's tiles to the tile-major buffer: each tile's TSL
    // slots are contiguous there; slots of levels finer than lmin are zero.
    // Slot -> accumulator offset table (in the free pass records): offset of
    // the slot's cell for tile (0, 0), row stride and m = L - level.
    if (wbuf != nullptr) {
      int2* tab = reinterpret_cast<int2*>(S.pass);
      for (int q = tid; q < TSL; q += NT) {
        int lev, band, ix, iy;
        slot_decode(L, q, &lev, &band, &ix, &iy);
        const int bi = lev == L ? band : band - 1;
        tab[q] = lev >= lmin ? make_int2(lvC[lev] + bi * lvPS[lev] + iy * lvG[lev] + ix, (lvG[lev] << 8) | (L - lev))
                             : make_int2(-1, 0);
      }
      __syncthreads();
      const unsigned acc_s = sh_addr(S.acc);
      // Thread -> one pair of slots (2 q, 2 q + 1) and every (NT / (TSL / 2))-th
      // tile: the slot table is read once, and the 16-byte stores of
      // consecutive threads are consecutive in the tile.
      constexpr int QP = TSL / 2;
      const int ntiles = kx * ky;
      const int q = tid % QP, step = NT / QP;
      int co[2], rs[2], shf[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int2 e = tab[2 * q + h];
        co[h] = e.x;
        rs[h] = e.y >> 8;
        shf[h] = e.y & 255;
      }
      int tj = 0, tt = tid / QP;
      while (tt >= kx && step > 0) {
        tt -= kx;
        ++tj;
      }
      for (int tile = tid / QP; step > 0 && tile < ntiles; tile += step) {
        float v[4];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          float2 c = make_float2(0.f, 0.f);
          if (co[h] >= 0) {
            const unsigned ci = (unsigned)(co[h] + ((tj * rs[h] + tt) << shf[h]));
            const int2 iv = lds64(acc_s + 8u * ci);
            c = fixed ? make_float2((float)iv.x * dq, (float)iv.y * dq)
                      : make_float2(__int_as_float(iv.x), __int_as_float(iv.y));
          }
          v[2 * h] = c.x;
          v[2 * h + 1] = c.y;
        }
        float4* dst = reinterpret_cast<float4*>(wbuf + ((size_t)(Sy + tj) * ntx + Sx + tt) * TSL) + q;
        __stcs(dst, make_float4(v[0], v[1], v[2], v[3]));
        tt += step;
        while (tt >= kx) {
          tt -= kx;
          ++tj;
        }
      }
      // Blocks narrower than a tile's slot pairs: one pair per thread-step.
      if (step == 0) {
        const int nq = ntiles * QP;
        for (int i = tid; i < nq; i += NT) {
          const int tile = i / QP, qq = i - tile * QP;
          const int tj2 = tile / kx, tt2 = tile - tj2 * kx;
          float v[4];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int2 e = tab[2 * qq + h];
            float2 c = make_float2(0.f, 0.f);
            if (e.x >= 0) {
              const unsigned ci = (unsigned)(e.x + ((tj2 * (e.y >> 8) + tt2) << (e.y & 255)));
              const int2 iv = lds64(acc_s + 8u * ci);
              c = fixed ? make_float2((float)iv.x * dq, (float)iv.y * dq)
                        : make_float2(__int_as_float(iv.x), __int_as_float(iv.y));
            }
            v[2 * h] = c.x;
            v[2 * h + 1] = c.y;
          }
          float4* dst = reinterpret_cast<float4*>(wbuf + ((size_t)(Sy + tj2) * ntx + Sx + tt2) * TSL) + qq;
          __stcs(dst, make_float4(v[0], v[1], v[2], v[3]));
        }
      }
    }
    if constexpr (RE) {  // bits alone, plane reference (the host sends nothing else here)
      if (J.bits != nullptr) {
        constexpr int KD = kMaxSuperTile >> L;  // the widest super-tile, the default for bits
        if constexpr (L >= 3) {
          if (k == KD && lmin == 2 && fixed)
            supertile_inverse8<L, true, KD, 2>(S.acc, fixed, re_acc, dq, lmin, k, kx, ky, Sx, Sy, J, lvC, lvG, lvPS,
                                               tid, NT);
          else
            supertile_inverse8<L, true>(S.acc, fixed, re_acc, dq, lmin, k, kx, ky, Sx, Sy, J, lvC, lvG, lvPS, tid,
                                        NT);
        } else if constexpr (L == 2) {
          supertile_inverse<L, true, false>(S.acc, fixed, re_acc, dq, lmin, k, kx, ky, Sx, Sy, J, lvC, lvG, lvPS,
                                            tid, NT, nullptr);
        }
      }
    } else if (MODE == kModeRef && L >= 2 && J.bits != nullptr && J.ref.kind != 0) {
      supertile_inverse<L, false, MODE == kModeRef>(S.acc, fixed, re_acc, dq, lmin, k, kx, ky, Sx, Sy, J, lvC, lvG,
                                                    lvPS, tid, NT, &s_ref);
    } else if (J.u != nullptr) {
      if constexpr (L >= 3) {
        constexpr int KX = kComplexTile >> L;  // the default super-tile of complex accumulation
        if (k == KX && lmin == 2 && fixed)
          supertile_inverse8<L, false, KX, 2>(S.acc, fixed, re_acc, dq, lmin, k, kx, ky, Sx, Sy, J, lvC, lvG, lvPS,
                                              tid, NT);
        else
          supertile_inverse8<L, false>(S.acc, fixed, re_acc, dq, lmin, k, kx, ky, Sx, Sy, J, lvC, lvG, lvPS, tid,
                                       NT);
      } else if constexpr (L == 2)
        supertile_inverse<L, false, false>(S.acc, fixed, re_acc, dq, lmin, k, kx, ky, Sx, Sy, J, lvC, lvG, lvPS,
                                           tid, NT, nullptr);
    } else if (J.bits != nullptr) {
      if constexpr (L >= 3)
        supertile_inverse8<L, true>(S.acc, fixed, re_acc, dq, lmin, k, kx, ky, Sx, Sy, J, lvC, lvG, lvPS, tid, NT);
      else if constexpr (L == 2)
        supertile_inverse<L, true, false>(S.acc, fixed, re_acc, dq, lmin, k, kx, ky, Sx, Sy, J, lvC, lvG, lvPS,
                                          tid, NT, nullptr);
    }
  }
}

template <int L, int DT, int MODE>
cudaError_t launch_t(const SuperposeArgs& a, cudaStream_t s) {
  const size_t smem = superpose_smem_bytes(a.cell, a.lut.L, a.lut.lmin, a.lut.D, MODE == kModeRe, a.rcap);
  cudaError_t e = cudaFuncSetAttribute(superpose_kernel<L, DT, MODE>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, superpose_kernel<L, DT, MODE>, a.threads, smem);
  if (e != cudaSuccess) return e;
  // A fixed grid (independent of the batch, so the launch can be replayed
  // from a graph): CTAs without work exit at their first claim.
  const long long grid = (long long)a.grid * std::max(per_sm, 1);
  superpose_kernel<L, DT, MODE><<<(unsigned)grid, a.threads, smem, s>>>(a);
  return cudaGetLastError();
}

template <int L, int DT>
cudaError_t launch_re(const SuperposeArgs& a, cudaStream_t s) {
  // Real-only accumulation serves the bits-only fused path (levels >= 2).
  // The spherical-reference epilogue likewise (levels >= 2).
  if (a.re_only) return L >= 2 ? launch_t<L, DT, (L >= 2 ? kModeRe : kModeComplex)>(a, s) : cudaErrorInvalidValue;
  if (a.has_ref) return L >= 2 ? launch_t<L, DT, (L >= 2 ? kModeRef : kModeComplex)>(a, s) : cudaErrorInvalidValue;
  return launch_t<L, DT, kModeComplex>(a, s);
}

template <int L>
cudaError_t launch_l(const SuperposeArgs& a, cudaStream_t s) {
  switch (a.lut.dtype) {
    case WASABI_F32: return launch_re<L, WASABI_F32>(a, s);
    case WASABI_F16S: return launch_re<L, WASABI_F16S>(a, s);
    case WASABI_BF16S: return launch_re<L, WASABI_BF16S>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

size_t superpose_smem_bytes(int cell, int L, int lmin, int D, bool re_only, int rcap) {
  return smem_layout(cell, L, lmin, D, re_only, rcap, nullptr, nullptr);
}

int superpose_min_range_cap() { return kRangeMin; }

// Pass capacity per window for a launch: the largest power of two up to
// kRangeMax whose shared memory fits the CTA's share of the SM (one
// 1,024-thread CTA per SM, or two smaller ones), at least kRangeMin.
int superpose_range_cap(int cell, int L, int lmin, int D, bool re_only, int threads) {
  const size_t budget = threads > 512 ? kOneCtaSmem : kTwoCtaSmem;
  if (const char* v = std::getenv("WASABI_RANGE_CAP")) {  // tuning override
    int r = std::max(kRangeMin, std::min(kRangeMax, std::atoi(v)));
    r = r / 4 * 4;
    if (superpose_smem_bytes(cell, L, lmin, D, re_only, r) <= kOneCtaSmem) return r;
  }
  for (int r = kRangeMax; r > kRangeMin; r >>= 1)
    if (superpose_smem_bytes(cell, L, lmin, D, re_only, r) <= budget) return r;
  return kRangeMin;
}

// Default configuration per kind of launch (measured on C2, C3 and the
// paper's geometry):
//  - real parts only (bits, plane reference): one 1,024-thread CTA per SM on
//    the widest super-tile (128 to 256 pixels) whose shared memory fits the
//    SM -- wider tiles mean fewer candidates and LUT ranges per pixel;
//  - complex accumulation: one 1,024-thread CTA per SM on 192, else 128;
//  - the reference-wave epilogue and the shared configuration (batches and
//    holograms below 8,192 pixels a side, where more, smaller CTAs keep the
//    SMs busy and latency low): two
//    512-thread CTAs per SM on the largest power-of-two side whose shared
//    memory fits half the SM, or one 1,024-thread CTA on 128 pixels when that
//    side would be below 128.
void superpose_default_config(int L, int lmin, int D, int kind, int* cell, int* threads) {
  const int unit = (1 << L) > 32 ? (1 << L) : 32;
  const bool re = kind == kConfigRe;
  auto fits_one = [&](int T) { return superpose_smem_bytes(T, L, lmin, D, re, kRangeMin) <= kOneCtaSmem; };
  if (kind == kConfigRe) {
    for (int T = kMaxSuperTile / unit * unit; T >= 128 && T >= unit; T -= unit)
      if (fits_one(T)) { *cell = T; *threads = 1024; return; }
  } else if (kind == kConfigComplex) {
    for (int T : {kComplexTile, 128})
      if (T % unit == 0 && fits_one(T)) { *cell = T; *threads = 1024; return; }
  }
  int T = 256;
  while (T > unit && superpose_smem_bytes(T, L, lmin, D, false, kRangeMin) > kTwoCtaSmem) T >>= 1;
  if (T < unit) T = unit;
  if (T < 128 && 128 % unit == 0 && fits_one(128)) { *cell = 128; *threads = 1024; return; }
  *cell = T;
  *threads = 512;
}

int superpose_max_cell_rows() { return kMaxCellRows; }
int superpose_min_threads() { return 128; }

cudaError_t launch_superpose(const SuperposeArgs& a, cudaStream_t s) {
  if (a.threads > 1024 || a.threads < superpose_min_threads() || a.threads % 32 || !a.lut.code ||
      a.rcap < kRangeMin || a.rcap > kRangeMax || a.rcap % 4)
    return cudaErrorInvalidValue;
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
