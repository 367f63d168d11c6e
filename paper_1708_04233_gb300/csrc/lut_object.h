// Host-side objects shared by the C-ABI translation units (abi.cu, batch.cu).
#pragma once

#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "internal.cuh"

// A device-resident look-up table (library-owned; see wasabi_build_lut).
struct wasabi_lut {
  int device = 0;
  cudaStream_t stream = nullptr;
  double lambda = 0, pitch = 0, gamma = 0;
  int D = 0, W = 0, L = 0, nwt = 0, dtype = 0;
  int reach = 0;  // pixels: footprint half-extent bound (max floor(R) + 2^(L+1))
  std::vector<double> z, R;
  std::vector<wsb::DepthMeta> meta;
  long long total_cap = 0;
  void* block = nullptr;  // one device allocation for all arrays below
  uint32_t* pos = nullptr;
  float2* val = nullptr;
  uint32_t* val16 = nullptr;
  float* scale = nullptr;
  int32_t* tile_off = nullptr;
  wsb::DepthMeta* meta_dev = nullptr;
  long long* nr_dev = nullptr;
  float* cmax = nullptr;
  unsigned* levels = nullptr;  // bit l: a level-l coefficient is kept
  uint2* code = nullptr;       // ncode x total_cap (plane code, value word), one array per super-tile width
  int ncode = 0;
  int code_k[wsb::kMaxCodes] = {};
  int lmin = 1;                // finest kept level (host copy)
  int wavelet = 0;             // WASABI_HAAR or WASABI_COIF1
  // Autotuned superposition configurations: hologram size class -> (super-tile, threads).
  mutable std::mutex tune_mu;
  std::map<int, std::pair<int, int>> tuned;

  wsb::LutView view() const {
    wsb::LutView v;
    v.D = D; v.W = W; v.L = L; v.nwt = nwt; v.dtype = dtype;
    v.pos = pos; v.val = val; v.val16 = val16; v.scale = scale;
    v.tile_off = tile_off; v.meta = meta_dev; v.cmax = cmax; v.lmin = lmin;
    v.code = nullptr;
    return v;
  }
  // The view for super-tiles of k x k tiles (null codes if k is not built).
  wsb::LutView view(int k) const {
    wsb::LutView v = view();
    for (int i = 0; i < ncode; ++i)
      if (code_k[i] == k) v.code = code + (size_t)i * total_cap;
    return v;
  }
};

namespace wsb {

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Carves consecutive 256-byte-aligned regions out of one block.
struct Carver {
  size_t off = 0;
  char* base = nullptr;
  template <typename T>
  T* take(size_t count) {
    off = align_up(off, 256);
    T* p = reinterpret_cast<T*>(base ? base + off : nullptr);
    off += count * sizeof(T);
    return p;
  }
};

// Size class of a hologram for tuning: its longer side rounded up to a power of two.
inline int size_class(int w, int h) {
  int s = 1;
  const int m = w > h ? w : h;
  while (s < m) s <<= 1;
  return s;
}

// Super-tile side and block size for a hologram: an environment override,
// else the autotuned choice for its size class, else the default.
// kind: kConfigComplex / kConfigRe / kConfigRef / kConfigShared (the default
// of a hologram of at least kConfigLargeSide pixels a side depends on it);
// see superpose_config_kind for a call's kind.
void superpose_config(const wasabi_lut* lut, int w, int h, int kind, int* cell, int* threads);
// The kind of launch a superposition call makes from its outputs and frame.
inline int superpose_config_kind(bool wbuf, bool u, bool bits, const wasabi_frame* frame) {
  if (bits && frame && frame->ref.kind != WASABI_REF_PLANE) return kConfigRef;
  return (!wbuf && !u && bits) ? kConfigRe : kConfigComplex;
}

// wasabi_superpose / wasabi_hologram with an explicit configuration: any of
// the wavelet buffer, the complex field and the packed bits may be written.
// frame may be NULL (whole plane from pixel (0, 0), unit plane reference).
wasabi_status superpose_impl(const wasabi_lut* lut, const wasabi_point* points_dev, int64_t n, int holo_w,
                             int holo_h, int rule, void* wbuf_dev, void* u_dev, uint8_t* bits_dev,
                             void* scratch_dev, size_t scratch_bytes, cudaStream_t s, int cell, int threads,
                             const wasabi_frame* frame = nullptr);

// Checks a frame (NULL = all zero) and converts it for the kernels: origin
// and reference wave.  false (message in *why) for an invalid frame.
bool frame_to_dev(const wasabi_frame* f, int* ox, int* oy, RefDev* ref, const char** why);
// True when the frame's bits need the field's imaginary part (spherical R).
inline bool frame_needs_complex(const wasabi_frame* f) { return f && f->ref.kind != WASABI_REF_PLANE; }

bool device_info(int** status, int* sms);
wasabi_status cuda_fail(const char* what, cudaError_t e);
int superpose_min_threads();
int superpose_max_cell_rows();

}  // namespace wsb
