// WASABI oracle — TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, single-threaded CPU restatement of the WASABI method of
// Shimobaba et al., "Fast, large-scale hologram calculation in wavelet domain"
// (arXiv 1708.04233), written from the paper's text.  Only the tests, the
// package's smoke check and the benchmark's CPU-baseline leg may load it; the
// product path (the CUDA library) never does, and the two share no code.
//
// Every function cites the passage it follows.  Where the paper is silent or
// ambiguous the reading taken is stated beside the code (readings R1-R12;
// R10 is the sub-hologram driver, R11 the image-type sign convention):
//   R1 PSF support radius (Sec. 1, step 1: "W_j is the PSF radius"):
//      one radius R(z) = z * tan(asin(lambda / (2 p))) / p  [pixels], the
//      alias-free diffraction limit of pitch p; support is the open disk
//      n = du^2 + dv^2 < R^2; W_j is read as the diameter 2R.
//   R2 depth quantisation (Sec. 1, step 1; Sec. 2 "Delta z = 30mm/29"):
//      D bins of width dz = (zmax - zmin)/D, centre z_d = zmin + (d + 1/2) dz,
//      d_j = min(D - 1, floor((z_j - zmin)/dz)).
//   R3 coefficients kept (Sec. 1, step 1: N_r = pi (W_j/2)^2 gamma):
//      gamma < 1: N_r = min(nnz, ceil(gamma * pi * R^2 - 1e-9));
//      gamma >= 1: every nonzero coefficient.
//   R4 wavelet: orthonormal 2-D Haar (the paper used coiflets, Sec. 1), Mallat
//      layout of Fig. 2(a); LH is high-pass along x (columns) and sits at rows
//      [0,S) x columns [S,2S), HL at rows [S,2S) x columns [0,S), HH at [S,2S)^2.
//   R5 "strong" coefficients: key = re^2 + im^2 in FP64, descending; equal
//      keys go to the lower Mallat linear index (row * W + col).
//   R6 shift weight alpha (Eq. (2)): alpha = 2^-l at level l (l = L for the
//      scaling band); a window sub-band position (p,q) lands at
//      P = p + floor((x_j - W/2) / 2^l) (rule 0, "floor") or
//      P = p + floor((x_j - W/2 + 2^(l-1)) / 2^l) (rule 1, "nearest");
//      m <-> column <-> x, n <-> row <-> y; positions outside [0, Nh/2^l)
//      are dropped.
//   R7 binary hologram (Sec. 2): bit = 1 iff Re(u) > 0 (unit plane reference).
//   R8 phase arithmetic of the FP32 PSF used for selection (so that the CPU
//      and the GPU select the same coefficients): t = r / lambda =
//      sqrt(s), s = fma(n, (p/lambda)^2, (z/lambda)^2) in FP64, evaluated as
//      the FP32 square root t0 of s plus one FP64 Newton step
//      t = t0 + fma(-t0, t0, s) * (float)(1 / (2 t0)); f = t - floor(t);
//      g = (float) f; cos and sin of 2 pi g from quadrant reduction and
//      Taylor series in Horner form with fused multiply-adds in FP32
//      (J.-M. Muller, "Elementary Functions", range reduction + polynomial
//      evaluation).  The FP64 PSF and Eq. (1) use the plain definition
//      r = sqrt(n p^2 + z^2), t = r / lambda.
//   R9 Eq. (1) has no 1/r factor and a +i sign, as printed; a_j is used as an
//      amplitude.
//   R14 coiflet wavelet (Sec. 1 uses coiflets at level 3; the order is not
//      stated): order 1, the 6-tap orthonormal filter below (coif1_taps),
//      periodic filter banks on the W x W window and on the N_h x N_h buffer,
//      the same Mallat layout and sub-band letters as R4 (analysis along x
//      first), the same shift rule R6.  FP32 analysis in a fixed order: the
//      k = -2 product, then fused multiply-adds for k = -1 .. 3.
//   R12 reference wave (Sec. 2, a spherical wave from (x_r, y_r, z_r)): the
//      wave of a unit point source in the object points' convention (R9,
//      R11), R = exp(i sgn(z_r) 2 pi r / lambda),
//      r = sqrt(((x_h - x_r) p)^2 + ((y_h - y_r) p)^2 + z_r^2), with x_r, y_r
//      in plane pixels (real) and pixel (i, j) at (i, j); the binary
//      hologram is bit = Re(u conj R) > 0, the sign of the interference term
//      of |u + R|^2.  R7 is the case R = 1.
//
// Build: g++ -O2 -ffp-contract=off -fPIC -shared (contraction must stay off:
// the FP32 selection path depends on every rounding being the written one).

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

constexpr double kPi = 3.14159265358979323846264338327950288;

// ---------------------------------------------------------------- geometry --

// R1: support radius in pixels for depth z (Sec. 1, step 1).
double support_radius_px(double lambda, double pitch, double z) {
  const double s = lambda / (2.0 * pitch);
  const double t = s / std::sqrt(1.0 - s * s);  // tan(asin(s))
  return (std::fabs(z) * t) / pitch;
}

// R11 (image-type holograms, points on both sides of the hologram plane): the
// support is the open disk n < R(|z|)^2 plus the centre pixel (a point on
// the plane is a single pixel), and a point behind the plane (z < 0) has the
// conjugate PSF -- the wave converging on it.
bool in_support(int64_t n, double R2) { return n == 0 || (double)n < R2; }

// R3: coefficient budget for gamma < 1 (Sec. 1, step 1).
int64_t keep_target(double gamma, double R) {
  // R11: a support of the centre pixel alone (R <= 1) is a delta; all of its
  // (at most 3L + 1) nonzero coefficients are kept.
  if (R <= 1.0) return INT64_MAX;
  const double area = kPi * (R * R);
  return (int64_t)std::ceil(gamma * area - 1e-9);
}

// Floor division by a power of two, written out (no reliance on >> of a
// negative number).
int64_t floor_div(int64_t a, int64_t b) {
  int64_t q = a / b;
  if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
  return q;
}

// R6: the level-l shift of Eq. (2) for a displacement X = x_j - W/2.
int64_t level_shift(int64_t X, int l, int rule) {
  const int64_t step = (int64_t)1 << l;
  if (rule == 0) return floor_div(X, step);
  return floor_div(X + step / 2, step);
}

// ------------------------------------------------------------------- phase --

// R8: cos and sin of 2*pi*g for g in [0, 1], FP32, every step rounded as
// written.  Quadrant reduction: g = q/4 + y with q = nearest integer of 4g and
// |y| <= 1/8 (the subtraction is exact), x = 2*pi*y in [-pi/4, pi/4]; then the
// Taylor series of sin to x^9 and of cos to x^10 in Horner form.
void sincos2pi_f32(float g, float* c_out, float* s_out) {
  const float two_pi = 6.28318530717958647692f;
  const float S3 = -1.0f / 6.0f, S5 = 1.0f / 120.0f, S7 = -1.0f / 5040.0f,
              S9 = 1.0f / 362880.0f;
  const float C2 = -1.0f / 2.0f, C4 = 1.0f / 24.0f, C6 = -1.0f / 720.0f,
              C8 = 1.0f / 40320.0f, C10 = -1.0f / 3628800.0f;
  const float q = std::nearbyint(4.0f * g);
  const float y = g - 0.25f * q;
  const float x = y * two_pi;
  const float x2 = x * x;
  float ps = std::fma(x2, S9, S7);
  ps = std::fma(x2, ps, S5);
  ps = std::fma(x2, ps, S3);
  const float sn = std::fma(x * x2, ps, x);
  float pc = std::fma(x2, C10, C8);
  pc = std::fma(x2, pc, C6);
  pc = std::fma(x2, pc, C4);
  pc = std::fma(x2, pc, C2);
  const float cs = std::fma(x2, pc, 1.0f);
  switch (((int)q) & 3) {
    case 0: *c_out = cs;  *s_out = sn;  break;
    case 1: *c_out = -sn; *s_out = cs;  break;
    case 2: *c_out = -cs; *s_out = -sn; break;
    default: *c_out = sn; *s_out = -cs; break;
  }
}

// Fractional part of r / lambda for r = sqrt(n p^2 + z^2) (Eq. (1): the
// phase 2*pi*r/lambda reduced modulo 2*pi).
double phase_frac(int64_t n, double p2, double z2, double lambda) {
  const double r = std::sqrt(std::fma((double)n, p2, z2));
  const double t = r / lambda;
  return t - std::floor(t);
}

// The same fractional part, evaluated the way the FP32 PSF (R8) and the GPU
// LUT builder evaluate it: t = r / lambda = sqrt(s) with s = n (p/lambda)^2 +
// (z/lambda)^2, taken as the FP32 square root of s plus one Newton step in
// FP64 (residual s - t0^2 by a fused multiply-add, divided by 2 t0 through
// the FP32 reciprocal).  The error against phase_frac is ~1e-11 (the Newton
// step squares the FP32 error); q = (p/lambda)^2, c = (z/lambda)^2.
double phase_frac_newton(int64_t n, double q, double c) {
  const double s = std::fma((double)n, q, c);
  const float t0f = std::sqrt((float)s);
  const double t0 = (double)t0f;
  const double res = std::fma(-t0, t0, s);
  if (t0f == 0.0f) return 0.0;  // s = 0: a point on the plane, at its own pixel
  const float inv = 1.0f / (2.0f * t0f);
  const double t = t0 + res * (double)inv;
  return t - std::floor(t);
}

// ---------------------------------------------------------------- the PSF --

// Sec. 1, step 1: u_z = exp(i k r) circ(...), sampled on a W x W window whose
// centre pixel (W/2, W/2) holds the point; du = u - W/2, dv = v - W/2.
// FP32 form (R8).  Output: interleaved complex, row-major (row = v).
void psf_f32(double lambda, double pitch, double z, int W, float* out) {
  const double R = support_radius_px(lambda, pitch, z);
  const double R2 = R * R;
  const double pl = pitch / lambda, zl = std::fabs(z) / lambda;
  const double q = pl * pl, cz = zl * zl;
  for (int v = 0; v < W; ++v) {
    for (int u = 0; u < W; ++u) {
      const int64_t du = u - W / 2, dv = v - W / 2;
      const int64_t n = du * du + dv * dv;
      float c = 0.0f, s = 0.0f;
      if (in_support(n, R2)) {
        const float g = (float)phase_frac_newton(n, q, cz);
        sincos2pi_f32(g, &c, &s);
        if (z < 0) s = -s;  // R11
      }
      out[2 * ((int64_t)v * W + u) + 0] = c;
      out[2 * ((int64_t)v * W + u) + 1] = s;
    }
  }
}

// FP64 form: the definition exp(i 2 pi r / lambda) evaluated with the C
// library's cos and sin.
void psf_f64(double lambda, double pitch, double z, int W, double* out) {
  const double R = support_radius_px(lambda, pitch, z);
  const double R2 = R * R;
  const double p2 = pitch * pitch, z2 = z * z;
  for (int v = 0; v < W; ++v) {
    for (int u = 0; u < W; ++u) {
      const int64_t du = u - W / 2, dv = v - W / 2;
      const int64_t n = du * du + dv * dv;
      double c = 0.0, s = 0.0;
      if (in_support(n, R2)) {
        const double f = phase_frac(n, p2, z2, lambda);
        c = std::cos(2.0 * kPi * f);
        s = (z < 0 ? -1.0 : 1.0) * std::sin(2.0 * kPi * f);  // R11
      }
      out[2 * ((int64_t)v * W + u) + 0] = c;
      out[2 * ((int64_t)v * W + u) + 1] = s;
    }
  }
}

// -------------------------------------------------------------- Haar (R4) --

// One forward level on the top-left S x S block of an n x n interleaved
// complex array (row stride n): each 2x2 block (x00 x01 / x10 x11) gives
//   s  = ((x00 + x01) + (x10 + x11)) / 2
//   LH = ((x00 - x01) + (x10 - x11)) / 2   (high along x)
//   HL = ((x00 + x01) - (x10 + x11)) / 2   (high along y)
//   HH = ((x00 - x01) - (x10 - x11)) / 2
template <typename T>
void haar_fwd_level(T* a, int64_t n, int64_t S, std::vector<T>& tmp) {
  const int64_t h = S / 2;
  tmp.assign((size_t)(2 * S * S), T(0));
  for (int64_t i = 0; i < h; ++i) {
    for (int64_t j = 0; j < h; ++j) {
      for (int c = 0; c < 2; ++c) {
        const T x00 = a[2 * ((2 * i) * n + 2 * j) + c];
        const T x01 = a[2 * ((2 * i) * n + 2 * j + 1) + c];
        const T x10 = a[2 * ((2 * i + 1) * n + 2 * j) + c];
        const T x11 = a[2 * ((2 * i + 1) * n + 2 * j + 1) + c];
        const T half = T(0.5);
        tmp[2 * (i * S + j) + c] = ((x00 + x01) + (x10 + x11)) * half;
        tmp[2 * (i * S + h + j) + c] = ((x00 - x01) + (x10 - x11)) * half;
        tmp[2 * ((h + i) * S + j) + c] = ((x00 + x01) - (x10 + x11)) * half;
        tmp[2 * ((h + i) * S + h + j) + c] = ((x00 - x01) - (x10 - x11)) * half;
      }
    }
  }
  for (int64_t r = 0; r < S; ++r)
    std::memcpy(&a[2 * r * n], &tmp[2 * r * S], sizeof(T) * 2 * S);
}

// Inverse of one level: the transpose of the orthonormal map above,
//   x00 = ((s + LH) + (HL + HH)) / 2      x01 = ((s - LH) + (HL - HH)) / 2
//   x10 = ((s + LH) - (HL + HH)) / 2      x11 = ((s - LH) - (HL - HH)) / 2
template <typename T>
void haar_inv_level(T* a, int64_t n, int64_t S, std::vector<T>& tmp) {
  const int64_t h = S / 2;
  tmp.assign((size_t)(2 * S * S), T(0));
  for (int64_t i = 0; i < h; ++i) {
    for (int64_t j = 0; j < h; ++j) {
      for (int c = 0; c < 2; ++c) {
        const T s = a[2 * (i * n + j) + c];
        const T lh = a[2 * (i * n + h + j) + c];
        const T hl = a[2 * ((h + i) * n + j) + c];
        const T hh = a[2 * ((h + i) * n + h + j) + c];
        const T half = T(0.5);
        tmp[2 * ((2 * i) * S + 2 * j) + c] = ((s + lh) + (hl + hh)) * half;
        tmp[2 * ((2 * i) * S + 2 * j + 1) + c] = ((s - lh) + (hl - hh)) * half;
        tmp[2 * ((2 * i + 1) * S + 2 * j) + c] = ((s + lh) - (hl + hh)) * half;
        tmp[2 * ((2 * i + 1) * S + 2 * j + 1) + c] = ((s - lh) - (hl - hh)) * half;
      }
    }
  }
  for (int64_t r = 0; r < S; ++r)
    std::memcpy(&a[2 * r * n], &tmp[2 * r * S], sizeof(T) * 2 * S);
}

// Sec. 1, step 1 ("FWT") and step 3 ("inverse FWT"), L levels, in place.
template <typename T>
void haar_fwd(T* a, int64_t n, int L) {
  std::vector<T> tmp;
  for (int l = 1; l <= L; ++l) haar_fwd_level(a, n, n >> (l - 1), tmp);
}
template <typename T>
void haar_inv(T* a, int64_t n, int L) {
  std::vector<T> tmp;
  for (int l = L; l >= 1; --l) haar_inv_level(a, n, n >> (l - 1), tmp);
}

// ------------------------------------------------------------ coiflet (R14) --

// Order-1 coiflet: the scaling filter h_k (k = -2 .. 3) solves
//   sum_k h_k = sqrt 2,  sum_k h_k h_{k+2m} = delta_m (m = 0, 1, 2),
//   sum_k (-1)^k k h_k = 0  (with the zeroth moment: two vanishing wavelet
//   moments),  sum_k k h_k = 0  (a vanishing first scaling moment).
// Of its two real roots this is the one whose largest tap is h_0:
//   h / sqrt 2 = ((1 - r)/32, (5 + r)/32, (7 + r)/16, (7 - r)/16, (1 - r)/32,
//                (r - 3)/32),  r = sqrt 7.
// The wavelet filter is g_k = (-1)^k h_{1-k}, on the same support.
void coif1_taps(double lo[6], double hi[6]) {
  const double r = std::sqrt(7.0), s2 = std::sqrt(2.0);
  lo[0] = s2 * (1.0 - r) / 32.0;
  lo[1] = s2 * (5.0 + r) / 32.0;
  lo[2] = s2 * (7.0 + r) / 16.0;
  lo[3] = s2 * (7.0 - r) / 16.0;
  lo[4] = s2 * (1.0 - r) / 32.0;
  lo[5] = s2 * (r - 3.0) / 32.0;
  for (int i = 0; i < 6; ++i) {
    const int k = i - 2;         // tap index
    const int j = (1 - k) + 2;   // array slot of h_{1-k}
    hi[i] = (k % 2 != 0 ? -1.0 : 1.0) * lo[j];
  }
}

int64_t pmod(int64_t a, int64_t n) { return ((a % n) + n) % n; }

// One periodic analysis level on the top-left S x S block of an n x n
// interleaved complex array: along x (each row: low half, then high half),
// then along y (each column: low half on top).  Sum order per output: the
// k = -2 product, then fused multiply-adds for k = -1 .. 3.
template <typename T>
void coif_fwd_level(T* a, int64_t n, int64_t S, const T* lo, const T* hi, std::vector<T>& tmp) {
  const int64_t h = S / 2;
  tmp.assign((size_t)(2 * S * S), T(0));
  for (int64_t r = 0; r < S; ++r)
    for (int64_t m = 0; m < h; ++m)
      for (int c = 0; c < 2; ++c) {
        T x = a[2 * (r * n + pmod(2 * m - 2, S)) + c];
        T sl = lo[0] * x, sh = hi[0] * x;
        for (int i = 1; i < 6; ++i) {
          x = a[2 * (r * n + pmod(2 * m + i - 2, S)) + c];
          sl = std::fma(lo[i], x, sl);
          sh = std::fma(hi[i], x, sh);
        }
        tmp[(size_t)(2 * (r * S + m) + c)] = sl;
        tmp[(size_t)(2 * (r * S + h + m) + c)] = sh;
      }
  for (int64_t col = 0; col < S; ++col)
    for (int64_t m = 0; m < h; ++m)
      for (int c = 0; c < 2; ++c) {
        T x = tmp[(size_t)(2 * (pmod(2 * m - 2, S) * S + col) + c)];
        T sl = lo[0] * x, sh = hi[0] * x;
        for (int i = 1; i < 6; ++i) {
          x = tmp[(size_t)(2 * (pmod(2 * m + i - 2, S) * S + col) + c)];
          sl = std::fma(lo[i], x, sl);
          sh = std::fma(hi[i], x, sh);
        }
        a[2 * (m * n + col) + c] = sl;
        a[2 * ((h + m) * n + col) + c] = sh;
      }
}

// The transpose of coif_fwd_level (its inverse, the filters being
// orthonormal): along y, then along x; sample j receives
// h_k s[m] + g_k d[m] for every k = j - 2m (mod S), k = -2 .. 3.
template <typename T>
void coif_inv_level(T* a, int64_t n, int64_t S, const T* lo, const T* hi, std::vector<T>& tmp) {
  const int64_t h = S / 2;
  tmp.assign((size_t)(2 * S * S), T(0));
  for (int64_t col = 0; col < S; ++col)
    for (int64_t j = 0; j < S; ++j)
      for (int c = 0; c < 2; ++c) {
        T acc = T(0);
        for (int i = 0; i < 6; ++i) {
          const int k = i - 2;
          if (((j - k) % 2 + 2) % 2 != 0) continue;
          const int64_t m = pmod((j - k) / 2, h);
          acc = std::fma(lo[i], a[2 * (m * n + col) + c], acc);
          acc = std::fma(hi[i], a[2 * ((h + m) * n + col) + c], acc);
        }
        tmp[(size_t)(2 * (j * S + col) + c)] = acc;
      }
  for (int64_t r = 0; r < S; ++r)
    for (int64_t j = 0; j < S; ++j)
      for (int c = 0; c < 2; ++c) {
        T acc = T(0);
        for (int i = 0; i < 6; ++i) {
          const int k = i - 2;
          if (((j - k) % 2 + 2) % 2 != 0) continue;
          const int64_t m = pmod((j - k) / 2, h);
          acc = std::fma(lo[i], tmp[(size_t)(2 * (r * S + m) + c)], acc);
          acc = std::fma(hi[i], tmp[(size_t)(2 * (r * S + h + m) + c)], acc);
        }
        a[2 * (r * n + j) + c] = acc;
      }
}

// Forward / inverse L-level transform, in place: wavelet 0 = Haar (R4),
// 1 = order-1 coiflet (R14).
template <typename T>
void wavelet_fwd(T* a, int64_t n, int L, int wavelet) {
  if (wavelet == 0) { haar_fwd(a, n, L); return; }
  double lo[6], hi[6];
  coif1_taps(lo, hi);
  T lt[6], ht[6];
  for (int i = 0; i < 6; ++i) { lt[i] = (T)lo[i]; ht[i] = (T)hi[i]; }
  std::vector<T> tmp;
  for (int l = 1; l <= L; ++l) coif_fwd_level(a, n, n >> (l - 1), lt, ht, tmp);
}
template <typename T>
void wavelet_inv(T* a, int64_t n, int L, int wavelet) {
  if (wavelet == 0) { haar_inv(a, n, L); return; }
  double lo[6], hi[6];
  coif1_taps(lo, hi);
  T lt[6], ht[6];
  for (int i = 0; i < 6; ++i) { lt[i] = (T)lo[i]; ht[i] = (T)hi[i]; }
  std::vector<T> tmp;
  for (int l = L; l >= 1; --l) coif_inv_level(a, n, n >> (l - 1), lt, ht, tmp);
}

// Position of Mallat entry (row, col) of an n x n, L-level transform:
// level l (1..L), band 0 = scaling (l = L only), 1 = LH, 2 = HL, 3 = HH,
// sub-band coordinates p (x, column) and q (y, row).  Fig. 2(a).
void mallat_decode(int64_t row, int64_t col, int64_t n, int L, int* lev,
                   int* band, int64_t* p, int64_t* q) {
  for (int l = 1; l <= L; ++l) {
    const int64_t S = n >> l;
    if (row >= S || col >= S) {
      *lev = l;
      if (row < S) { *band = 1; *p = col - S; *q = row; }
      else if (col < S) { *band = 2; *p = col; *q = row - S; }
      else { *band = 3; *p = col - S; *q = row - S; }
      return;
    }
  }
  *lev = L; *band = 0; *p = col; *q = row;
}

// Inverse of mallat_decode for a hologram-sized buffer of side n.
void mallat_encode(int lev, int band, int64_t P, int64_t Q, int64_t n,
                   int64_t* row, int64_t* col) {
  const int64_t S = n >> lev;
  switch (band) {
    case 0: *row = Q; *col = P; break;
    case 1: *row = Q; *col = S + P; break;
    case 2: *row = S + Q; *col = P; break;
    default: *row = S + Q; *col = S + P; break;
  }
}

// ---------------------------------------------------------- selection (R5) --

// Sec. 1, step 1: keep N_r strong coefficients.  Returns N_r; idx_out gets
// the kept Mallat linear indices in ascending order.
template <typename T>
int64_t select_strong(const T* coef, int W, double gamma, double R,
                      int32_t* idx_out) {
  const int64_t n = (int64_t)W * W;
  std::vector<std::pair<double, int32_t>> nz;
  for (int64_t i = 0; i < n; ++i) {
    const double re = (double)coef[2 * i], im = (double)coef[2 * i + 1];
    const double key = re * re + im * im;
    if (key > 0.0) nz.emplace_back(key, (int32_t)i);
  }
  int64_t nr = (int64_t)nz.size();
  if (gamma < 1.0) nr = std::min<int64_t>(nr, keep_target(gamma, R));
  if (nr < 0) nr = 0;
  std::sort(nz.begin(), nz.end(), [](const std::pair<double, int32_t>& a,
                                     const std::pair<double, int32_t>& b) {
    if (a.first != b.first) return a.first > b.first;
    return a.second < b.second;
  });
  std::vector<int32_t> kept((size_t)nr);
  for (int64_t k = 0; k < nr; ++k) kept[(size_t)k] = nz[(size_t)k].second;
  std::sort(kept.begin(), kept.end());
  std::copy(kept.begin(), kept.end(), idx_out);
  return nr;
}

// ------------------------------------------------------------------- LUT --

// Sec. 1, step 1 for every depth: PSF, L-level FWT, keep N_r strong.
// Per depth d, entries [off_d, off_d + nr[d]) of idx/val, off_d = sum of the
// earlier nr.  Returns 0, or -1 when cap is too small or a window is too
// small for its PSF (2R + 1 > W).
template <typename T>
int build_lut(double lambda, double pitch, const double* zd, int D, int W,
              int L, double gamma, int64_t* nr, int64_t cap, int32_t* idx,
              T* val, int threads, bool fp32_psf, bool select_fp32, int wavelet) {
  const int64_t n = (int64_t)W * W;
  std::vector<std::vector<int32_t>> sel((size_t)D);
  std::vector<std::vector<T>> vals((size_t)D);
  int bad = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads > 0 ? threads : 1) reduction(+ : bad)
#endif
  for (int d = 0; d < D; ++d) {
    const double R = support_radius_px(lambda, pitch, zd[d]);
    if (2.0 * R + 1.0 > (double)W) { bad += 1; continue; }
    std::vector<T> coef((size_t)(2 * n));
    if (fp32_psf) {
      std::vector<float> tmp((size_t)(2 * n));
      psf_f32(lambda, pitch, zd[d], W, tmp.data());
      for (int64_t i = 0; i < 2 * n; ++i) coef[(size_t)i] = (T)tmp[(size_t)i];
    } else {
      std::vector<double> tmp((size_t)(2 * n));
      psf_f64(lambda, pitch, zd[d], W, tmp.data());
      for (int64_t i = 0; i < 2 * n; ++i) coef[(size_t)i] = (T)tmp[(size_t)i];
    }
    wavelet_fwd(coef.data(), W, L, wavelet);
    std::vector<int32_t> kept((size_t)n);
    int64_t k;
    if (!fp32_psf && select_fp32) {
      // Keep the coefficients that the FP32 path keeps (the selection is an
      // integer decision taken in the GPU kernel's precision), with FP64
      // values.
      std::vector<float> c32((size_t)(2 * n));
      psf_f32(lambda, pitch, zd[d], W, c32.data());
      wavelet_fwd(c32.data(), W, L, wavelet);
      k = select_strong(c32.data(), W, gamma, R, kept.data());
    } else {
      k = select_strong(coef.data(), W, gamma, R, kept.data());
    }
    kept.resize((size_t)k);
    std::vector<T> v((size_t)(2 * k));
    for (int64_t i = 0; i < k; ++i) {
      v[(size_t)(2 * i)] = coef[(size_t)(2 * kept[(size_t)i])];
      v[(size_t)(2 * i + 1)] = coef[(size_t)(2 * kept[(size_t)i] + 1)];
    }
    sel[(size_t)d] = std::move(kept);
    vals[(size_t)d] = std::move(v);
  }
  if (bad) return -1;
  int64_t off = 0;
  for (int d = 0; d < D; ++d) {
    const int64_t k = (int64_t)sel[(size_t)d].size();
    if (off + k > cap) return -1;
    nr[d] = k;
    std::copy(sel[(size_t)d].begin(), sel[(size_t)d].end(), idx + off);
    std::copy(vals[(size_t)d].begin(), vals[(size_t)d].end(), val + 2 * off);
    off += k;
  }
  return 0;
}

// ----------------------------------------------------- superposition (Eq. 2) --

// Eq. (2) with the sub-hologram coordinate transform of Sec. 1, large-scale
// step 2 (x'_j = x_j - ox): psi (an Nh x Nh Mallat buffer, interleaved
// complex, accumulated into) += a_j c_k at the shifted position of every kept
// coefficient k of point j's depth (R6).  Accumulation order: points in input
// order, coefficients in LUT order.
template <typename T>
int superpose(int W, int L, int D, const int64_t* nr, const int32_t* idx,
              const T* val, const int32_t* x, const int32_t* y, const float* a,
              const uint32_t* d, int64_t N, int64_t Nh, int64_t ox, int64_t oy,
              int rule, T* psi) {
  std::vector<int64_t> off((size_t)D + 1, 0);
  for (int k = 0; k < D; ++k) off[(size_t)k + 1] = off[(size_t)k] + nr[k];
  // The (level, band, p, q) of every LUT entry (a pure function of its index).
  const int64_t total = off[(size_t)D];
  std::vector<int> lev((size_t)total), band((size_t)total);
  std::vector<int64_t> pp((size_t)total), qq((size_t)total);
  for (int64_t e = 0; e < total; ++e)
    mallat_decode(idx[e] / W, idx[e] % W, W, L, &lev[(size_t)e],
                  &band[(size_t)e], &pp[(size_t)e], &qq[(size_t)e]);
  const int64_t margin = (int64_t)1 << L;
  for (int64_t j = 0; j < N; ++j) {
    if (d[j] >= (uint32_t)D) return -1;
    const int64_t X = (int64_t)x[j] - ox - W / 2;
    const int64_t Y = (int64_t)y[j] - oy - W / 2;
    // A point whose whole window (plus one tile) lies off this buffer has
    // every coefficient dropped by the range test below; skip it early.
    if (X + W + margin < 0 || X - margin >= Nh || Y + W + margin < 0 ||
        Y - margin >= Nh)
      continue;
    const T aj = (T)a[j];
    for (int64_t e = off[d[j]]; e < off[d[j] + 1]; ++e) {
      const int l = lev[(size_t)e];
      const int64_t P = pp[(size_t)e] + level_shift(X, l, rule);
      const int64_t Q = qq[(size_t)e] + level_shift(Y, l, rule);
      const int64_t Sh = Nh >> l;
      if (P < 0 || P >= Sh || Q < 0 || Q >= Sh) continue;
      int64_t row, col;
      mallat_encode(l, band[(size_t)e], P, Q, Nh, &row, &col);
      T* dst = psi + 2 * (row * Nh + col);
      dst[0] += aj * val[2 * e];
      dst[1] += aj * val[2 * e + 1];
    }
  }
  return 0;
}

// --------------------------------------------------------- Eq. (1) directly --

// u(x_h, y_h) = sum_j a_j exp(i 2 pi r_hj / lambda) [aperture], FP64, for the
// region [ox, ox + w) x [oy, oy + h) (row-major, interleaved).  z is per point.
void cgh_direct(double lambda, double pitch, const int32_t* x, const int32_t* y,
                const float* a, const double* z, int64_t N, int64_t ox,
                int64_t oy, int64_t w, int64_t h, int aperture, double* u,
                int threads) {
  const double p2 = pitch * pitch;
  std::vector<double> R2((size_t)N);
  for (int64_t j = 0; j < N; ++j) {
    const double R = support_radius_px(lambda, pitch, z[j]);
    R2[(size_t)j] = R * R;
  }
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads > 0 ? threads : 1)
#endif
  for (int64_t yy = 0; yy < h; ++yy) {
    for (int64_t xx = 0; xx < w; ++xx) {
      double re = 0.0, im = 0.0;
      for (int64_t j = 0; j < N; ++j) {
        const int64_t dx = ox + xx - x[j], dy = oy + yy - y[j];
        const int64_t n = dx * dx + dy * dy;
        if (aperture && !in_support(n, R2[(size_t)j])) continue;
        const double f = phase_frac(n, p2, z[j] * z[j], lambda);
        re += (double)a[j] * std::cos(2.0 * kPi * f);
        im += (double)a[j] * (z[j] < 0 ? -1.0 : 1.0) * std::sin(2.0 * kPi * f);  // R11
      }
      u[2 * (yy * w + xx) + 0] = re;
      u[2 * (yy * w + xx) + 1] = im;
    }
  }
}

// R12: reference wave over the region [ox, ox + w) x [oy, oy + h) of the
// plane, FP64, interleaved complex, row-major.
void reference_wave(double lambda, double pitch, double xr, double yr,
                    double zr, int64_t ox, int64_t oy, int64_t w, int64_t h,
                    double* R) {
  const double sg = zr < 0 ? -1.0 : 1.0;
  for (int64_t yy = 0; yy < h; ++yy)
    for (int64_t xx = 0; xx < w; ++xx) {
      const double dx = ((double)(ox + xx) - xr) * pitch;
      const double dy = ((double)(oy + yy) - yr) * pitch;
      const double t = std::sqrt(dx * dx + dy * dy + zr * zr) / lambda;
      const double f = t - std::floor(t);
      R[2 * (yy * w + xx) + 0] = std::cos(2.0 * kPi * f);
      R[2 * (yy * w + xx) + 1] = sg * std::sin(2.0 * kPi * f);
    }
}

}  // namespace

// =================================================================== C ABI ==

extern "C" {

double orc_support_radius(double lambda, double pitch, double z) {
  return support_radius_px(lambda, pitch, z);
}

int64_t orc_keep_target(double gamma, double R) { return keep_target(gamma, R); }

// R2: bin centres of D depth bins over [zmin, zmax].
void orc_depth_grid(double zmin, double zmax, int D, double* zd) {
  const double dz = (zmax - zmin) / (double)D;
  for (int d = 0; d < D; ++d) zd[d] = zmin + ((double)d + 0.5) * dz;
}

// R2: depth index of each point; returns the number of points outside
// [zmin, zmax] (their index is set to D).
int64_t orc_quantize(const double* z, int64_t N, double zmin, double zmax,
                     int D, uint32_t* d) {
  const double dz = (zmax - zmin) / (double)D;
  int64_t bad = 0;
  for (int64_t j = 0; j < N; ++j) {
    if (!(z[j] >= zmin && z[j] <= zmax)) { d[j] = (uint32_t)D; ++bad; continue; }
    int64_t k = (int64_t)std::floor((z[j] - zmin) / dz);
    if (k > D - 1) k = D - 1;
    d[j] = (uint32_t)k;
  }
  return bad;
}

void orc_sincos2pi_f32(const float* g, int64_t n, float* c, float* s) {
  for (int64_t i = 0; i < n; ++i) sincos2pi_f32(g[i], &c[i], &s[i]);
}

void orc_psf_f32(double lambda, double pitch, double z, int W, float* out) {
  psf_f32(lambda, pitch, z, W, out);
}
void orc_psf_f64(double lambda, double pitch, double z, int W, double* out) {
  psf_f64(lambda, pitch, z, W, out);
}

void orc_haar_fwd_f32(float* a, int64_t n, int L) { haar_fwd(a, n, L); }
void orc_wavelet_fwd_f32(float* a, int64_t n, int L, int w) { wavelet_fwd(a, n, L, w); }
void orc_wavelet_inv_f32(float* a, int64_t n, int L, int w) { wavelet_inv(a, n, L, w); }
void orc_wavelet_fwd_f64(double* a, int64_t n, int L, int w) { wavelet_fwd(a, n, L, w); }
void orc_wavelet_inv_f64(double* a, int64_t n, int L, int w) { wavelet_inv(a, n, L, w); }
void orc_coif1_taps(double* lo, double* hi) { coif1_taps(lo, hi); }
void orc_haar_inv_f32(float* a, int64_t n, int L) { haar_inv(a, n, L); }
void orc_haar_fwd_f64(double* a, int64_t n, int L) { haar_fwd(a, n, L); }
void orc_haar_inv_f64(double* a, int64_t n, int L) { haar_inv(a, n, L); }

void orc_mallat_decode(int64_t row, int64_t col, int64_t n, int L, int* lev,
                       int* band, int64_t* p, int64_t* q) {
  mallat_decode(row, col, n, L, lev, band, p, q);
}

int64_t orc_select_f32(const float* coef, int W, double gamma, double R,
                       int32_t* idx_out) {
  return select_strong(coef, W, gamma, R, idx_out);
}
int64_t orc_select_f64(const double* coef, int W, double gamma, double R,
                       int32_t* idx_out) {
  return select_strong(coef, W, gamma, R, idx_out);
}

int orc_build_lut_f32(double lambda, double pitch, const double* zd, int D,
                      int W, int L, double gamma, int64_t* nr, int64_t cap,
                      int32_t* idx, float* val, int threads, int wavelet) {
  return build_lut<float>(lambda, pitch, zd, D, W, L, gamma, nr, cap, idx, val,
                          threads, true, false, wavelet);
}
// select_fp32 != 0: FP64 values at the indices the FP32 path selects.
int orc_build_lut_f64(double lambda, double pitch, const double* zd, int D,
                      int W, int L, double gamma, int64_t* nr, int64_t cap,
                      int32_t* idx, double* val, int threads, int select_fp32,
                      int wavelet) {
  return build_lut<double>(lambda, pitch, zd, D, W, L, gamma, nr, cap, idx,
                           val, threads, false, select_fp32 != 0, wavelet);
}

int orc_superpose_f32(int W, int L, int D, const int64_t* nr, const int32_t* idx,
                      const float* val, const int32_t* x, const int32_t* y,
                      const float* a, const uint32_t* d, int64_t N, int64_t Nh,
                      int64_t ox, int64_t oy, int rule, float* psi) {
  return superpose<float>(W, L, D, nr, idx, val, x, y, a, d, N, Nh, ox, oy,
                          rule, psi);
}
int orc_superpose_f64(int W, int L, int D, const int64_t* nr, const int32_t* idx,
                      const double* val, const int32_t* x, const int32_t* y,
                      const float* a, const uint32_t* d, int64_t N, int64_t Nh,
                      int64_t ox, int64_t oy, int rule, double* psi) {
  return superpose<double>(W, L, D, nr, idx, val, x, y, a, d, N, Nh, ox, oy,
                           rule, psi);
}

// Sec. 1, large-scale steps 2-4 for one sub-hologram (s, t) of side Ns:
// shift the points, superpose into a fresh Ns x Ns Mallat buffer, inverse
// FWT.  u_sub: Ns x Ns interleaved complex, row-major.
int orc_subhologram_f32(int W, int L, int D, const int64_t* nr,
                        const int32_t* idx, const float* val, const int32_t* x,
                        const int32_t* y, const float* a, const uint32_t* d,
                        int64_t N, int64_t Ns, int64_t s, int64_t t, int rule,
                        float* u_sub, int wavelet) {
  std::memset(u_sub, 0, sizeof(float) * 2 * Ns * Ns);
  const int rc = superpose<float>(W, L, D, nr, idx, val, x, y, a, d, N, Ns,
                                  s * Ns, t * Ns, rule, u_sub);
  if (rc) return rc;
  wavelet_inv(u_sub, Ns, L, wavelet);
  return 0;
}
int orc_subhologram_f64(int W, int L, int D, const int64_t* nr,
                        const int32_t* idx, const double* val, const int32_t* x,
                        const int32_t* y, const float* a, const uint32_t* d,
                        int64_t N, int64_t Ns, int64_t s, int64_t t, int rule,
                        double* u_sub, int wavelet) {
  std::memset(u_sub, 0, sizeof(double) * 2 * Ns * Ns);
  const int rc = superpose<double>(W, L, D, nr, idx, val, x, y, a, d, N, Ns,
                                   s * Ns, t * Ns, rule, u_sub);
  if (rc) return rc;
  wavelet_inv(u_sub, Ns, L, wavelet);
  return 0;
}

// R7: bits row-major, 8 pixels per byte, least significant bit = lowest x.
void orc_binarize_f32(const float* u, int64_t w, int64_t h, uint8_t* bits) {
  std::memset(bits, 0, (size_t)((w * h + 7) / 8));
  for (int64_t yy = 0; yy < h; ++yy)
    for (int64_t xx = 0; xx < w; ++xx) {
      const int64_t i = yy * w + xx;
      if (u[2 * i] > 0.0f) bits[i >> 3] |= (uint8_t)(1u << (i & 7));
    }
}

void orc_reference_wave(double lambda, double pitch, double xr, double yr,
                        double zr, int64_t ox, int64_t oy, int64_t w, int64_t h,
                        double* R) {
  reference_wave(lambda, pitch, xr, yr, zr, ox, oy, w, h, R);
}

// R12: bits of Re(u conj R) > 0 for the field u (interleaved complex FP64)
// of the region at (ox, oy); val receives Re(u conj R) per pixel.
void orc_binarize_ref_f64(const double* u, int64_t w, int64_t h, double lambda,
                          double pitch, double xr, double yr, double zr,
                          int64_t ox, int64_t oy, uint8_t* bits, double* val) {
  std::vector<double> R((size_t)(2 * w * h));
  reference_wave(lambda, pitch, xr, yr, zr, ox, oy, w, h, R.data());
  std::memset(bits, 0, (size_t)((w * h + 7) / 8));
  for (int64_t i = 0; i < w * h; ++i) {
    // Re(u conj R) = Re u Re R + Im u Im R
    const double v = u[2 * i] * R[(size_t)(2 * i)] + u[2 * i + 1] * R[(size_t)(2 * i + 1)];
    val[i] = v;
    if (v > 0.0) bits[i >> 3] |= (uint8_t)(1u << (i & 7));
  }
}

void orc_cgh_direct_f64(double lambda, double pitch, const int32_t* x,
                        const int32_t* y, const float* a, const double* z,
                        int64_t N, int64_t ox, int64_t oy, int64_t w, int64_t h,
                        int aperture, double* u, int threads) {
  cgh_direct(lambda, pitch, x, y, a, z, N, ox, oy, w, h, aperture, u, threads);
}

int orc_have_openmp(void) {
#ifdef _OPENMP
  return 1;
#else
  return 0;
#endif
}

}  // extern "C"
