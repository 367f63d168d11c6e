// Inverse transformation (Sec. 1, step 3) and binary hologram (Sec. 2).
//
// inverse_kernel: a persistent CTA streams horizontal strips of G tiles
// (256 pixels x 2^L rows; the strip's G*4^L coefficients are contiguous in the
// tile-major buffer) through a STAGES-deep shared-memory ring filled by bulk
// asynchronous copies (cp.async.bulk, one per tile into a padded slot,
// completion tracked by an mbarrier transaction count).  Each thread rebuilds
// a 4 x 4 pixel block: the scaling value is carried down the levels it shares
// with its neighbours, then the level-2 and level-1 steps fan out to 16 pixels
// held in registers.  Output is either complex64 row-major (two 16-byte
// streaming stores per row of the block) or packed bits (Re(u conj R) > 0
// for the reference wave R, R = 1 by default), gathered across the warp with
// shuffles into 32-bit words.  A spherical R is anchored once per strip (FP64
// phase reduction by one thread, double-buffered in shared memory) and carried
// to the pixels in FP32.
//
// The wavelet buffer is read exactly once and each output byte is written
// once: the kernel is bound by HBM bandwidth.
#include <algorithm>

#include "internal.cuh"

namespace wsb {
namespace {

constexpr int kStages = 3;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false after `limit` clock cycles without completion.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, long long limit) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > limit) return false;
  }
  return true;
}

template <int L>
struct InvCfg {
  static constexpr int TS = 1 << L;
  static constexpr int TSL = TS * TS;
  static constexpr int G = 256 / TS;        // tiles per strip
  static constexpr int STRIDE = TSL + 8;    // padded tile slot (complex)
  static constexpr int NT = 16 * TS;        // threads: 64 blocks across x 2^L/4 down
  static constexpr size_t STAGE_BYTES = (size_t)G * STRIDE * sizeof(float2);
  static constexpr size_t SMEM = kStages * STAGE_BYTES + 64;
};

// REF: bits against a spherical reference wave (a kernel of its own, so that
// the plane-reference kernel carries none of its code).
template <int L, bool REF>
__global__ void __launch_bounds__(InvCfg<L>::NT) inverse_kernel(const __grid_constant__ InverseArgs a) {
  using C = InvCfg<L>;
  extern __shared__ __align__(128) unsigned char smem[];
  float2* ring = reinterpret_cast<float2*>(smem);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * C::STAGE_BYTES);

  // Items are the strips of the hologram, dealt to the CTAs round-robin.
  const long long nitems = a.nstrips;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const long long count = nitems > blockIdx.x ? (nitems - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  int* status = a.status;
  const int spr = (a.ntx + C::G - 1) / C::G;  // strips per tile row
  __shared__ RefAnchor s_anc[2];  // reference phase anchors of items i and i + 1
  constexpr bool ref = REF;

  // Tile row and strip column of the CTA's i-th item.
  auto locate = [&](long long i, int* ty, int* sx) {
    const int item = (int)(blockIdx.x + i * gridDim.x);
    *ty = item / spr;
    *sx = item - *ty * spr;
  };
  // Reference phase at the first pixel of the CTA's i-th strip.
  auto anchor = [&](long long i) {
    int ty, sx;
    locate(i, &ty, &sx);
    return ref_anchor(a.ref, (long long)a.ox + sx * 256, (long long)a.oy + (long long)ty * C::TS);
  };

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(&full[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (ref && count > 0) s_anc[0] = anchor(0);
  }
  __syncthreads();

  auto issue = [&](long long i, int stage) {  // warp 0 only
    // A test names one strip whose copy is never issued: its stage wait then
    // runs out and the kernel reports E_TIMEOUT instead of waiting forever.
    if (blockIdx.x + i * gridDim.x == a.skip_item) return;
    int ty, sx;
    locate(i, &ty, &sx);
    const int ntx = a.ntx;
    const int tx0 = sx * C::G;
    const int gv = min(C::G, ntx - tx0);
    const float2* src = a.wbuf + ((size_t)ty * ntx + tx0) * C::TSL;
    float2* dst = ring + (size_t)stage * C::G * C::STRIDE;
    if (lane == 0) mbar_expect_tx(&full[stage], (unsigned)(gv * C::TSL * sizeof(float2)));
    __syncwarp();
    for (int g = lane; g < gv; g += 32)
      bulk_g2s(dst + (size_t)g * C::STRIDE, src + (size_t)g * C::TSL, C::TSL * sizeof(float2), &full[stage]);
  };

  if (wid == 0)
    for (int s = 0; s < kStages && s < count; ++s) issue(s, s);

  // Thread -> 4x4 pixel block: bxs in [0, 64) along the strip, by down the tile.
  const int bxs = (wid & 1) * 32 + lane;
  const int by = wid >> 1;
  const int g = bxs >> (L - 2);
  const int bx = bxs & ((C::TS >> 2) - 1);

  bool timed_out = false;
  long long i = 0;
  for (; i < count; ++i) {
    const int stage = (int)(i % kStages);
    const unsigned parity = (unsigned)((i / kStages) & 1);
    const bool arrived = mbar_wait(&full[stage], parity, a.wait_limit);
    if (__syncthreads_or(!arrived)) {  // leave together, never split the CTA
      timed_out = true;
      break;
    }
    int ty, sx;
    locate(i, &ty, &sx);
    const int w = a.w;
    float2* u = a.u;
    uint8_t* bits = a.bits;
    const int gv = min(C::G, a.ntx - sx * C::G);
    const bool valid = g < gv;
    const float2* c = ring + (size_t)stage * C::G * C::STRIDE + (size_t)(valid ? g : 0) * C::STRIDE;

    // Levels L .. 3: the block lies inside one level-(l-1) cell.
    float2 s = c[0];
#pragma unroll
    for (int l = L; l >= 3; --l) {
      const int m = L - l;
      const int o = (((4 * by) >> l) << m) + ((4 * bx) >> l);
      const float2 lh = c[(1 << (2 * m)) + o], hl = c[(2 << (2 * m)) + o], hh = c[(3 << (2 * m)) + o];
      s = ipick(s, lh, hl, hh, ((4 * bx) >> (l - 1)) & 1, ((4 * by) >> (l - 1)) & 1);
    }
    // Level 2 at (bx, by) -> four level-1 scaling values.
    float2 s1[2][2];
    {
      const int m = L - 2;
      const int o = (by << m) + bx;
      const float2 lh = c[(1 << (2 * m)) + o], hl = c[(2 << (2 * m)) + o], hh = c[(3 << (2 * m)) + o];
#pragma unroll
      for (int ay = 0; ay < 2; ++ay)
#pragma unroll
        for (int ax = 0; ax < 2; ++ax) s1[ay][ax] = ipick(s, lh, hl, hh, ax, ay);
    }
    // Level 1 -> 4 x 4 pixels.
    float2 px[4][4];
    {
      const int m = L - 1;
#pragma unroll
      for (int ay = 0; ay < 2; ++ay) {
        const int o = ((2 * by + ay) << m) + 2 * bx;
        const float4 lh = *reinterpret_cast<const float4*>(&c[(1 << (2 * m)) + o]);
        const float4 hl = *reinterpret_cast<const float4*>(&c[(2 << (2 * m)) + o]);
        const float4 hh = *reinterpret_cast<const float4*>(&c[(3 << (2 * m)) + o]);
#pragma unroll
        for (int ax = 0; ax < 2; ++ax) {
          const float2 l1 = ax ? make_float2(lh.z, lh.w) : make_float2(lh.x, lh.y);
          const float2 h1 = ax ? make_float2(hl.z, hl.w) : make_float2(hl.x, hl.y);
          const float2 d1 = ax ? make_float2(hh.z, hh.w) : make_float2(hh.x, hh.y);
#pragma unroll
          for (int qy = 0; qy < 2; ++qy)
#pragma unroll
            for (int qx = 0; qx < 2; ++qx) px[2 * ay + qy][2 * ax + qx] = ipick(s1[ay][ax], l1, h1, d1, qx, qy);
        }
      }
    }

    const int x0 = sx * 256 + g * C::TS + 4 * bx;  // first pixel column of the block
    const int y0 = ty * C::TS + 4 * by;
    if (u != nullptr && valid) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float4* dst = reinterpret_cast<float4*>(u + (size_t)(y0 + j) * w + x0);
        __stcs(dst, make_float4(px[j][0].x, px[j][0].y, px[j][1].x, px[j][1].y));
        __stcs(dst + 1, make_float4(px[j][2].x, px[j][2].y, px[j][3].x, px[j][3].y));
      }
    }
    if (bits != nullptr) {
      const int xend = min(w, sx * 256 + gv * C::TS);
      const int xw = sx * 256 + (wid & 1) * 128 + 32 * (lane >> 3);  // word's first pixel
      RefBlock RB;
      if (ref) RB = ref_block(a.ref, s_anc[i & 1], g * C::TS + 4 * bx, 4 * by);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        unsigned nib = 0;
        if (valid) {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float v = ref ? ref_value(RB, a.ref.sgn, px[j][q], q, j) : px[j][q].x;
            nib |= (v > 0.f ? 1u : 0u) << q;
          }
        }
        unsigned v = nib << (4 * (lane & 7));
        v |= __shfl_xor_sync(0xffffffffu, v, 1);
        v |= __shfl_xor_sync(0xffffffffu, v, 2);
        v |= __shfl_xor_sync(0xffffffffu, v, 4);
        if ((lane & 7) == 0 && xw < xend) {
          const size_t byte0 = ((size_t)(y0 + j) * w + xw) >> 3;
          if (xw + 32 <= xend && (w & 31) == 0) {
            *reinterpret_cast<unsigned*>(bits + byte0) = v;
          } else {
            const int nb = min(4, (xend - xw) >> 3);
            for (int q = 0; q < nb; ++q) bits[byte0 + q] = (uint8_t)(v >> (8 * q));
          }
        }
      }
    }
    // Item i + 1's anchor goes to the buffer item i - 1 used (every read of
    // it ended before the previous barrier).
    if (ref && tid == 0 && i + 1 < count) s_anc[(i + 1) & 1] = anchor(i + 1);
    __syncthreads();
    if (wid == 0 && i + kStages < count) issue(i + kStages, stage);
  }
  if (timed_out) {
    if (tid == 0) {
      atomicCAS(status, 0, WASABI_E_TIMEOUT);
      // Bounded wait for this CTA's copies still in flight before exiting.
      for (long long j = i; j < count && j < i + kStages; ++j)
        (void)mbar_wait(&full[j % kStages], (unsigned)((j / kStages) & 1), a.wait_limit);
    }
    __syncthreads();
  }
}

// Forward transform of one tile per block (test export).
template <int L>
__global__ void haar_forward_kernel(const float2* __restrict__ u, int w, float2* __restrict__ wbuf) {
  constexpr int TS = 1 << L, TSL = TS * TS;
  __shared__ float2 cur[TSL], nxt[TSL], co[TSL];
  const int ntx = w >> L;
  const int tile = blockIdx.x;
  const int tx = tile % ntx, ty = tile / ntx;
  const int pix = threadIdx.x;
  cur[pix] = u[(size_t)(ty * TS + pix / TS) * w + tx * TS + pix % TS];
  __syncthreads();
  float2* a = cur;
  float2* b = nxt;
  for (int l = 1; l <= L; ++l) {
    const int S = TS >> (l - 1), hh = S >> 1, m = L - l;
    if (pix < hh * hh) {
      const int i = pix / hh, j = pix % hh;
      const float2 x00 = a[2 * i * TS + 2 * j], x01 = a[2 * i * TS + 2 * j + 1];
      const float2 x10 = a[(2 * i + 1) * TS + 2 * j], x11 = a[(2 * i + 1) * TS + 2 * j + 1];
      b[i * TS + j] = make_float2(((x00.x + x01.x) + (x10.x + x11.x)) * 0.5f,
                                  ((x00.y + x01.y) + (x10.y + x11.y)) * 0.5f);
      co[(1 << (2 * m)) + (i << m) + j] = make_float2(((x00.x - x01.x) + (x10.x - x11.x)) * 0.5f,
                                                      ((x00.y - x01.y) + (x10.y - x11.y)) * 0.5f);
      co[(2 << (2 * m)) + (i << m) + j] = make_float2(((x00.x + x01.x) - (x10.x + x11.x)) * 0.5f,
                                                      ((x00.y + x01.y) - (x10.y + x11.y)) * 0.5f);
      co[(3 << (2 * m)) + (i << m) + j] = make_float2(((x00.x - x01.x) - (x10.x - x11.x)) * 0.5f,
                                                      ((x00.y - x01.y) - (x10.y - x11.y)) * 0.5f);
    }
    __syncthreads();
    float2* t = a; a = b; b = t;
  }
  if (pix == 0) co[0] = a[0];
  __syncthreads();
  wbuf[(size_t)tile * TSL + pix] = co[pix];
}

__global__ void wbuf_to_mallat_kernel(const float2* __restrict__ wbuf, int w, int h, int L,
                                      float2* __restrict__ out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long n = (long long)w * h;
  if (i >= n) return;
  const int TSL = 1 << (2 * L);
  const long long tile = i / TSL;
  const int slot = (int)(i % TSL);
  const int ntx = w >> L;
  const int tx = (int)(tile % ntx), ty = (int)(tile / ntx);
  int lev, band, ix, iy;
  slot_decode(L, slot, &lev, &band, &ix, &iy);
  const int m = L - lev;
  const long long P = ((long long)tx << m) + ix, Q = ((long long)ty << m) + iy;
  const long long Sx = w >> lev, Sy = h >> lev;
  long long row = Q, col = P;
  if (band == 1) col += Sx;
  else if (band == 2) row += Sy;
  else if (band == 3) { row += Sy; col += Sx; }
  out[row * w + col] = wbuf[i];
}

template <int L, bool REF>
cudaError_t launch_inv_lr(const InverseArgs& a, cudaStream_t s) {
  using C = InvCfg<L>;
  cudaError_t e = cudaFuncSetAttribute(inverse_kernel<L, REF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)C::SMEM);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, inverse_kernel<L, REF>, C::NT, C::SMEM);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  // No more CTAs than strips.
  const long long grid = std::min<long long>((long long)a.num_sms * per_sm, a.nstrips);
  if (grid <= 0) return cudaSuccess;
  inverse_kernel<L, REF><<<(unsigned)grid, C::NT, C::SMEM, s>>>(a);
  return cudaGetLastError();
}

template <int L>
cudaError_t launch_inv_l(const InverseArgs& a, cudaStream_t s) {
  if (a.ref.kind != 0 && a.bits != nullptr) return launch_inv_lr<L, true>(a, s);
  return launch_inv_lr<L, false>(a, s);
}

template <int L>
int strips_l(int w, int h) {
  using C = InvCfg<L>;
  return (((w >> L) + C::G - 1) / C::G) * (h >> L);
}

template <int L>
cudaError_t launch_fwd_l(const float2* u, int w, int h, float2* wbuf, cudaStream_t s) {
  const int ntiles = (w >> L) * (h >> L);
  haar_forward_kernel<L><<<ntiles, 1 << (2 * L), 0, s>>>(u, w, wbuf);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_inverse(const InverseArgs& a, cudaStream_t s) {
  switch (a.L) {
    case 2: return launch_inv_l<2>(a, s);
    case 3: return launch_inv_l<3>(a, s);
    case 4: return launch_inv_l<4>(a, s);
    case 5: return launch_inv_l<5>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

int inverse_strips(int w, int h, int L) {
  switch (L) {
    case 2: return strips_l<2>(w, h);
    case 3: return strips_l<3>(w, h);
    case 4: return strips_l<4>(w, h);
    case 5: return strips_l<5>(w, h);
    default: return 0;
  }
}

cudaError_t launch_haar_forward(const float2* u, int w, int h, int L, float2* wbuf, cudaStream_t s) {
  switch (L) {
    case 1: return launch_fwd_l<1>(u, w, h, wbuf, s);
    case 2: return launch_fwd_l<2>(u, w, h, wbuf, s);
    case 3: return launch_fwd_l<3>(u, w, h, wbuf, s);
    case 4: return launch_fwd_l<4>(u, w, h, wbuf, s);
    case 5: return launch_fwd_l<5>(u, w, h, wbuf, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_wbuf_to_mallat(const float2* wbuf, int w, int h, int L, float2* out, cudaStream_t s) {
  const long long n = (long long)w * h;
  if (n == 0) return cudaSuccess;
  wbuf_to_mallat_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(wbuf, w, h, L, out);
  return cudaGetLastError();
}

}  // namespace wsb
