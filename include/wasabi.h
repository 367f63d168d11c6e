/*
 * wasabi.h — C ABI of libwasabi, a GB300 (sm_103a) implementation of WASABI
 * (wavelet shrinkage-based superposition) hologram synthesis, after
 * T. Shimobaba et al., "Fast, large-scale hologram calculation in wavelet
 * domain", arXiv 1708.04233.
 *
 * Conventions (all entry points):
 *  - Every function returns a wasabi_status; no exception and no abort ever
 *    crosses this boundary.  On failure wasabi_last_error() returns a
 *    thread-local message.
 *  - "dev" pointers are CUDA device pointers on the CURRENT device; "host"
 *    pointers are ordinary host memory.  Streams are cudaStream_t passed as
 *    void* (NULL = the legacy default stream).
 *  - Argument checks are synchronous.  Device work is asynchronous on the
 *    given stream unless stated otherwise; errors that only the device can see
 *    (a point's depth index out of range, a timed-out wait) are recorded in a
 *    per-device status word that wasabi_sync_status() reads and clears.
 *  - The caller owns points, wavelet buffers, outputs and scratch memory; the
 *    library owns only wasabi_lut objects.
 *  - Lengths (wavelength, pitch, depths) share one unit, e.g. metres.
 *
 * Geometry shared by all calls (the readings of the paper taken here):
 *  - Pixel (x, y): x is the column, y the row; row-major images.
 *  - PSF support radius at depth z (Sec. 1, step 1 "PSF radius"):
 *      R(z) = z * s / sqrt(1 - s^2) / pitch  [pixels],  s = lambda / (2 pitch),
 *    i.e. z tan(asin(lambda / 2p)) / p, the alias-free limit; the support is
 *    the open disk du^2 + dv^2 < R^2 around the point.
 *  - Haar: orthonormal, L levels.  On each 2x2 block (x00 x01 / x10 x11)
 *      s  = ((x00 + x01) + (x10 + x11)) / 2     LH = ((x00 - x01) + (x10 - x11)) / 2
 *      HL = ((x00 + x01) - (x10 + x11)) / 2     HH = ((x00 - x01) - (x10 - x11)) / 2
 *    (LH is high-pass along x).  Mallat layout (Fig. 2(a)): at level l with
 *    sub-band side S, LH sits at rows [0,S) x cols [S,2S), HL at rows [S,2S) x
 *    cols [0,S), HH at [S,2S)^2; the scaling band of level L at [0,S)^2.
 *  - Tile-major wavelet buffer ("wbuf"): a hologram of holo_w x holo_h pixels
 *    is cut into 2^L x 2^L tiles (holo_w, holo_h multiples of 2^L); tile
 *    (TX, TY) holds the 4^L Haar coefficients whose support lies inside it,
 *    contiguously, at complex offset (TY * holo_w/2^L + TX) * 4^L.  Within a
 *    tile, the coefficient of level l, band b (0 = scaling, only at l = L;
 *    1 = LH, 2 = HL, 3 = HH) and in-tile position (ix, iy), with m = L - l and
 *    0 <= ix, iy < 2^m, is at slot  (b << 2m) + (iy << m) + ix.
 *    Complex values are float2 (re, im), i.e. complex64.
 *  - Shift rule of Eq. (2) (alpha = 2^-l): a window coefficient at sub-band
 *    position (p, q) of level l lands at P = p + shift_l(x - W/2),
 *    Q = q + shift_l(y - W/2) with shift_l(X) = floor(X / 2^l) (FLOOR) or
 *    floor((X + 2^(l-1)) / 2^l) (NEAREST); the scaling band uses l = L.
 *    Positions outside [0, holo/2^l) are dropped.
 */
#ifndef WASABI_H
#define WASABI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int wasabi_status;
#define WASABI_OK 0
#define WASABI_E_INVALID (-1) /* bad argument (sizes, window, levels, keep ratio ...) */
#define WASABI_E_NOMEM (-2)   /* a library allocation failed or scratch too small  */
#define WASABI_E_CUDA (-3)    /* a CUDA runtime call or a launch failed            */
#define WASABI_E_RANGE (-4)   /* device-detected: depth index >= D, z outside range */
#define WASABI_E_TIMEOUT (-5) /* device-detected: a bounded wait gave up           */

/* Object point, 16 bytes (one float4 load), caller-owned.  x, y: integer pixel
 * indices (may lie outside the hologram, |x|, |y| < 2^30); a: amplitude a_j of
 * Eq. (1); d: index of the point's quantised depth in the LUT. */
typedef struct {
  int32_t x, y;
  float a;
  uint32_t d;
} wasabi_point;

typedef struct wasabi_lut wasabi_lut; /* opaque, library-owned, device-resident */

typedef enum { WASABI_F32 = 0, WASABI_F16S = 1, WASABI_BF16S = 2 } wasabi_lut_dtype;
typedef enum { WASABI_HAAR = 0, WASABI_COIF1 = 1 } wasabi_wavelet;
typedef enum { WASABI_SHIFT_FLOOR = 0, WASABI_SHIFT_NEAREST = 1 } wasabi_shift_rule;

/* Thread-local description of the last failure on this thread ("" if none). */
const char* wasabi_last_error(void);

/* Depth quantisation grid (Sec. 1, step 1 "discretized by Delta z"; Sec. 2):
 * D bins of width dz = (zmax - zmin) / D over [zmin, zmax]; writes the D bin
 * centres zmin + (d + 1/2) dz to depths_host.  E_INVALID if D < 1 or
 * zmax <= zmin. */
wasabi_status wasabi_depth_grid(double zmin, double zmax, int n_depths, double* depths_host);

/* Point preparation (Sec. 1, step 1 depth discretisation): for i < n,
 * out_dev[i] = {x[i], y[i], a[i], d} with d = min(D - 1, floor((z[i] - zmin) / dz)),
 * dz = (zmax - zmin) / D, in FP64.  All arrays are device arrays of n
 * elements.  A z outside [zmin, zmax] (or NaN) gets d = D and records
 * WASABI_E_RANGE in the status word. */
wasabi_status wasabi_quantize_points(const int32_t* x_dev, const int32_t* y_dev,
                                     const double* z_dev, const float* a_dev, int64_t n,
                                     double zmin, double zmax, int n_depths,
                                     wasabi_point* out_dev, void* stream);

/* The look-up table (Sec. 1, step 1): for each depth z_d
 * (depths_host[0..n_depths)), the PSF u_z = exp(i 2 pi r / lambda) on the
 * W x W window centred at pixel (W/2, W/2) with r = sqrt(n pitch^2 + z^2),
 * n = du^2 + dv^2, restricted to the disk n < R(|z|)^2 and the centre pixel;
 * its L-level Haar transform; and the N_r strongest coefficients by
 * re^2 + im^2 (FP64), equal strengths going to the lower Mallat index
 * row * W + col.  Depths may lie on both sides of the hologram plane (an
 * image-type hologram): a depth z < 0 has the conjugate PSF (the wave
 * converging on a point behind the plane), and z = 0 is a single-pixel delta.
 * N_r = min(nnz, ceil(keep_ratio * pi * R^2 - 1e-9)) for keep_ratio < 1 and
 * R > 1, and every nonzero coefficient for keep_ratio >= 1 or R <= 1 (Sec. 1,
 * step 1: N_r = pi (W_j/2)^2 gamma with W_j the PSF diameter 2R).
 * Phase arithmetic (so CPU and GPU select identical sets): t = r / lambda =
 * sqrt(s), s = n (pitch/lambda)^2 + (z/lambda)^2 in FP64, as the FP32 square
 * root t0 of s plus one FP64 Newton step t0 + (s - t0^2) / (2 t0);
 * f = t - floor(t); cos/sin of 2 pi (float) f by quadrant reduction and
 * Taylor polynomials in FP32 with fused multiply-adds.
 * Requires 1 <= levels <= 5 (2 <= levels for the inverse), window a multiple
 * of 2^(levels+1) with window <= 16384, window / 2^levels <= 2048 and
 * n_depths (window / 2^levels)^2 < 2^31, 2 R(z_d) + 1 <= window for every
 * depth, s = lambda / (2 pitch) < 1, keep_ratio > 0, 1 <= n_depths <= 4096.
 * The build's temporary device memory is about 16 n_depths window^2 bytes.
 * dtype selects how superposition reads the values: FP32, or FP16 / BF16 with
 * one FP32 scale per 32 consecutive entries (scale = max |re|, |im| of the
 * block; stored value = value / scale, rounded to nearest).
 * Allocates device memory (stream-ordered), enqueues the build on stream and
 * waits for it to finish (the library reads back which levels hold kept
 * coefficients, which sizes the superposition's accumulator).
 * E_INVALID on bad arguments, E_NOMEM, E_CUDA. */
wasabi_status wasabi_build_lut(double lambda, double pitch, const double* depths_host,
                               int n_depths, int window, int levels, double keep_ratio,
                               int dtype, void* stream, wasabi_lut** out);

/* wasabi_build_lut with a choice of wavelet (Sec. 1 uses coiflets at level 3,
 * order unstated).  WASABI_HAAR: as above.  WASABI_COIF1: the order-1 coiflet,
 * 6-tap orthonormal filters h_k (k = -2 .. 3) with
 * h / sqrt 2 = ((1 - r)/32, (5 + r)/32, (7 + r)/16, (7 - r)/16, (1 - r)/32, (r - 3)/32),
 * r = sqrt 7 (the solution of the coiflet equations whose largest tap is h_0),
 * wavelet filter g_k = (-1)^k h_{1-k}; periodic filter banks on the W x W
 * window, analysis along x then y per level, the Haar layout and letters
 * (Mallat, LH = high along x).  Its filters overlap window tiles, so the
 * whole window is transformed (PSF written out over W^2, analysis passes in
 * FP32 in a fixed order: the k = -2 product, then fused multiply-adds for
 * k = -1 .. 3), every window tile may hold kept coefficients and the
 * superposition reach is W/2 + 2^(L+1).  A coiflet LUT superposes into the
 * tile-major buffer with wasabi_superpose; its inverse is
 * wasabi_inverse_wavelet (the fused wasabi_hologram is Haar's alone).
 * Temporary device memory: about 24 n_depths W^2 bytes. */
wasabi_status wasabi_build_lut_wavelet(double lambda, double pitch, const double* depths_host,
                                       int n_depths, int window, int levels, double keep_ratio,
                                       int dtype, int wavelet, void* stream, wasabi_lut** out);

/* Releases a LUT (stream-ordered on the stream it was built on). */
wasabi_status wasabi_lut_destroy(wasabi_lut* lut);

/* Kept-coefficient counts N_r per depth into nr_host[0..n_depths).
 * Synchronises with the LUT's build stream. */
wasabi_status wasabi_lut_counts(const wasabi_lut* lut, int64_t* nr_host);

/* Depth `depth`'s kept coefficients as Mallat linear indices (row * W + col of
 * the W x W window transform), sorted ascending, into idx_host; *n_inout is
 * the capacity on entry and the count on return (E_NOMEM, with the count, if
 * too small).  Synchronising. */
wasabi_status wasabi_lut_selection(const wasabi_lut* lut, int depth, int32_t* idx_host,
                                   int64_t* n_inout);

/* Depth `depth`'s LUT entries in storage order (window tiles row-major, then
 * slot order): Mallat index and the value superposition uses (decoded to
 * FP32 for F16S / BF16S) as interleaved (re, im).  Synchronising. */
wasabi_status wasabi_lut_entries(const wasabi_lut* lut, int depth, int32_t* idx_host,
                                 float* val_host, int64_t* n_inout);

/* Scratch bytes wasabi_superpose needs for n points on a holo_w x holo_h
 * hologram with this LUT. */
wasabi_status wasabi_scratch_bytes(const wasabi_lut* lut, int64_t n, int holo_w, int holo_h,
                                   size_t* bytes_out);

/* Size of the fixed scratch array behind wasabi_superpose_static: 32 MiB. */
#define WASABI_STATIC_SCRATCH_BYTES (32 * 1024 * 1024)

/* Binning and superposition in the wavelet domain (Eq. (2)):
 *   psi = sum_j a_j sum_k c_{d_j,k} placed by the shift rule,
 * written to wbuf_dev (tile-major, holo_w * holo_h complex64, fully
 * overwritten: no prior zeroing needed).  points_dev: n wasabi_point;
 * scratch_dev: at least wasabi_scratch_bytes() bytes, 256-byte aligned.
 * holo_w, holo_h: multiples of 2^L (the LUT's levels), >= 2^L.
 * A point with d >= D records WASABI_E_RANGE and contributes nothing.
 * Configuration (super-tile side T, threads per CTA): the autotuned one for
 * the hologram's size class if wasabi_autotune ran, else a default: below
 * 8,192 pixels a side, and in batches, two 512-thread CTAs per SM on the
 * largest power-of-two T whose shared memory fits half an SM; from 8,192 up,
 * one 1,024-thread CTA per SM on T = 256 for bits with the plane reference
 * (real parts only), T = 192 for complex accumulation, and the two-CTA
 * choice for the spherical-reference epilogue.  Results depend on T only
 * through the rounding of each super-tile's fixed-point scale.
 * Environment overrides (tuning and tests; read at each call):
 * WASABI_SUPERPOSE_T and WASABI_SUPERPOSE_THREADS force the super-tile side
 * and threads per CTA (clamped to valid values), WASABI_RANGE_CAP the LUT
 * ranges per candidate batch, and WASABI_ACC_FLOAT=1 replaces the exact
 * fixed-point accumulation with FP32 shared-memory atomics. */
wasabi_status wasabi_superpose(const wasabi_lut* lut, const wasabi_point* points_dev, int64_t n,
                               int holo_w, int holo_h, int rule, void* wbuf_dev,
                               void* scratch_dev, size_t scratch_bytes, void* stream);

/* wasabi_superpose without a scratch argument, for callers that cannot
 * allocate device memory while they run: plug-ins whose host application
 * owns all device memory, real-time loops that forbid allocation after
 * start-up, and bindings that reach the C ABI but no CUDA allocator.  (The
 * paper has no counterpart; this is an interface convenience.)
 * Same arguments and result as wasabi_superpose, minus scratch.  The scratch
 * is one file-scope device array of WASABI_STATIC_SCRATCH_BYTES that every
 * device loading the library holds until the process exits; this call
 * allocates nothing.  Problems whose wasabi_scratch_bytes() exceeds that size
 * are rejected with WASABI_E_NOMEM (use wasabi_superpose then).
 * The first call on a device looks the array's device address up (a
 * synchronous runtime query): make that first call before any stream capture.
 * All calls share the array and it keeps the previous call's contents (each
 * call re-initialises what it reads); calls that overlap on the GPU race on
 * it, so serialise them (one stream, or events between streams).
 * The looked-up address is kept for the life of the device's primary
 * context: resetting the device (cudaDeviceReset) while the library is
 * loaded is not supported (the library's other per-device state, such as the
 * status word's address, is kept the same way). */
wasabi_status wasabi_superpose_static(const wasabi_lut* lut, const wasabi_point* points_dev, int64_t n,
                                      int holo_w, int holo_h, int rule, void* wbuf_dev, void* stream);

/* ---- Frame of a hologram: sub-hologram origin and reference wave --------
 * Sub-hologram (Sec. 1, large-scale calculation, steps 2-4): the output's
 * pixel (i, j) is pixel (origin_x + i, origin_y + j) of the hologram plane,
 * the frame in which the points' (x_j, y_j) are given; the points are
 * shifted by (-origin_x, -origin_y) before the superposition, the paper's
 * coordinate transform x'_j = x_j - s N_h, y'_j = y_j - t N_h.  Points whose
 * footprint misses the output contribute nothing; points partly outside it
 * contribute the part inside.
 * Reference wave (Sec. 2): the binary hologram is bit = Re(u conj(R)) > 0.
 * WASABI_REF_PLANE: R = 1 (a unit plane wave at normal incidence).
 * WASABI_REF_SPHERICAL: the wave of a unit point source at plane pixel
 * coordinates (x, y) (real numbers; the plane's pixel (i, j) sits at (i, j))
 * and signed distance z (metres, nonzero) from the plane, in the convention of
 * the object points: R = exp(i sgn(z) 2 pi r / lambda),
 * r = sqrt(pitch^2 ((i - x)^2 + (j - y)^2) + z^2) -- z < 0 (a source behind
 * the plane) is the converging, conjugate wave.  lambda and pitch in metres
 * (normally the LUT's).  The phase is reduced in FP64 once per 128- to
 * 256-pixel-wide anchor and carried to each pixel in FP32 by an exact
 * difference of squares and a quadratic expansion (phase error below
 * about 3e-5 cycles); bits can differ from an exact evaluation only where
 * |Re(u conj R)| is within that of zero.
 * An all-zero frame is the whole plane from pixel (0, 0) with R = 1. */
typedef enum { WASABI_REF_PLANE = 0, WASABI_REF_SPHERICAL = 1 } wasabi_reference_kind;

typedef struct {
  int32_t kind;          /* wasabi_reference_kind */
  int32_t reserved;      /* 0 */
  double lambda, pitch;  /* metres (spherical) */
  double x, y;           /* source position, plane pixels (spherical) */
  double z;              /* signed source distance from the plane, metres, nonzero (spherical) */
} wasabi_reference;

typedef struct {
  int32_t origin_x, origin_y; /* plane pixel of the output's pixel (0, 0) */
  wasabi_reference ref;       /* reference wave of the binarisation */
} wasabi_frame;

/* Inverse transformation (Sec. 1, step 3; Sec. 2 binary hologram):
 * the L-level inverse Haar of the tile-major wbuf_dev gives the field u.
 * u_dev (may be NULL): holo_w x holo_h complex64, row-major.
 * bits_dev (may be NULL): the binary hologram bit = (Re u > 0) for a unit
 * plane reference wave, row-major, 8 pixels per byte, least significant bit =
 * lowest x; holo_w must be a multiple of 8.  At least one output non-NULL.
 * 2 <= levels <= 5. */
wasabi_status wasabi_inverse_haar(const void* wbuf_dev, int holo_w, int holo_h, int levels,
                                  void* u_dev, uint8_t* bits_dev, void* stream);
/* wasabi_inverse_haar with a frame (may be NULL = all zero): the bits use the
 * frame's reference wave, evaluated at the output's plane pixels.
 * E_INVALID for an unknown kind, a nonzero reserved word, or a spherical
 * reference with non-finite or non-positive lambda / pitch, non-finite x / y,
 * or z zero or non-finite. */
wasabi_status wasabi_inverse_haar_frame(const void* wbuf_dev, int holo_w, int holo_h, int levels,
                                        const wasabi_frame* frame, void* u_dev, uint8_t* bits_dev,
                                        void* stream);

/* Inverse transformation for either wavelet of wasabi_build_lut_wavelet:
 * WASABI_HAAR runs wasabi_inverse_haar_frame (scratch unused); WASABI_COIF1
 * permutes the tile-major buffer into the Mallat layout and runs L periodic
 * synthesis levels over the holo_w x holo_h buffer (along y, then x, the
 * transpose of the analysis), then writes u and/or the bits against the
 * frame's reference (phase of a spherical R carried in double-float, pairs of
 * FP32 values, per pixel; plane pixels below 2^24 in magnitude).
 * 1 <= levels <= 5; COIF1 needs a square hologram (holo_w == holo_h, the
 * periodic transform's domain), side a multiple of 2^levels (and of 8 for bits).
 * scratch_dev: wasabi_inverse_wavelet_scratch_bytes() bytes (two buffers
 * of holo_w holo_h complex64), 256-byte aligned. */
wasabi_status wasabi_inverse_wavelet_scratch_bytes(int holo_w, int holo_h, size_t* bytes_out);
wasabi_status wasabi_inverse_wavelet(const void* wbuf_dev, int holo_w, int holo_h, int levels, int wavelet,
                                     const wasabi_frame* frame, void* u_dev, uint8_t* bits_dev,
                                     void* scratch_dev, size_t scratch_bytes, void* stream);

/* Binning, superposition, inverse and binarisation in one call: the
 * superposition (Eq. (2)) fused with the inverse transformation (Sec. 1,
 * step 3) and binarisation (Sec. 2).  Each
 * super-tile's wavelet coefficients are accumulated in shared memory and
 * inverse-transformed there, so the wavelet buffer is never written to (or
 * read back from) device memory unless asked for.  Outputs as in
 * wasabi_inverse_haar: u_dev (complex64 row-major, 16-byte aligned) and/or
 * bits_dev (packed, 4-byte aligned, holo_w % 8 == 0); at least one of them.
 * wbuf_dev may be NULL; when given, it also receives the tile-major wavelet
 * buffer as wasabi_superpose writes it.  The pixels equal those of
 * wasabi_superpose followed by wasabi_inverse_haar.  Needs levels >= 2;
 * scratch as for wasabi_superpose. */
wasabi_status wasabi_hologram(const wasabi_lut* lut, const wasabi_point* points_dev, int64_t n,
                              int holo_w, int holo_h, int rule, void* wbuf_dev, void* u_dev,
                              uint8_t* bits_dev, void* scratch_dev, size_t scratch_bytes, void* stream);
/* wasabi_hologram of a frame (may be NULL = all zero): the sub-hologram at
 * the frame's origin, binarised against its reference wave.  Here wbuf_dev
 * alone is also allowed (the superposition of a sub-hologram).  A spherical
 * reference needs complex accumulation (the bits-only fast path accumulates
 * real parts only).  Frame errors as for wasabi_inverse_haar_frame. */
wasabi_status wasabi_hologram_frame(const wasabi_lut* lut, const wasabi_point* points_dev, int64_t n,
                                    int holo_w, int holo_h, int rule, const wasabi_frame* frame,
                                    void* wbuf_dev, void* u_dev, uint8_t* bits_dev, void* scratch_dev,
                                    size_t scratch_bytes, void* stream);

/* Sub-hologram streaming (Sec. 1, large-scale calculation, steps 2-4): the
 * holo_w x holo_h hologram of the frame (may be NULL), computed as bands of
 * band_h rows -- band k is the sub-hologram at (origin_x, origin_y + k band_h),
 * fused as in wasabi_hologram_frame -- with each band's outputs copied into
 * host memory while the next band is computed.  The device holds two bands
 * (outputs and binning scratch), so the hologram is bounded by host memory.
 * bits_host: packed bits of the whole hologram (holo_w % 8 == 0); u_host:
 * complex64 row-major; at least one; pinned host memory makes the copies
 * asynchronous.  band_h: a multiple of 2^L (the last band may be shorter).
 * Work starts after what is queued on `stream`; the call returns when every
 * band has been copied.  Allocates and frees its band buffers (device memory)
 * and two streams per call.  Pixels equal the sub-holograms' (up to the
 * rounding of a per-band fixed-point scale: each band is its own job). */
wasabi_status wasabi_hologram_stream(const wasabi_lut* lut, const wasabi_point* points_dev, int64_t n,
                                     int holo_w, int holo_h, int band_h, int rule, const wasabi_frame* frame,
                                     uint8_t* bits_host, void* u_host, void* stream);

/* ---- Batches: many holograms through one launch sequence ---------------
 * One job = one hologram with its own points, wavelet buffer and outputs, all
 * sharing the LUT.  A batch runs every job through five launches (binning:
 * zero, count, scan, scatter; superposition with the fused inverse of
 * wasabi_hologram) whose grids do not depend on the batch; work items
 * (super-tiles) are claimed from a device-side job table.  With use_graph,
 * the job-table upload and the five launches are captured into a CUDA graph
 * on the first run on a stream and replayed by later runs (not on the legacy
 * default stream).  The graph holds the LUT's device pointers: destroy the
 * batch before the LUT.
 * The batch object owns pinned host staging and the device job table; the
 * caller owns the jobs' buffers and the scratch.  A run returns as soon as the
 * work is enqueued; a later run on the same batch object first waits for the
 * previous job-table upload. */
typedef struct {
  const wasabi_point* points_dev; /* n points (device) */
  int64_t n;
  int holo_w, holo_h;             /* multiples of 2^L; holo_w % 8 == 0 for bits */
  int rule;                       /* wasabi_shift_rule */
  void* wbuf_dev;                 /* tile-major wavelet buffer, holo_w * holo_h complex64, 256-B aligned,
                                     or NULL when only u / bits are wanted */
  void* u_dev;                    /* complex64 row-major output (16-B aligned), or NULL */
  uint8_t* bits_dev;              /* packed bits output (4-B aligned), or NULL; not all three NULL */
  wasabi_frame frame;             /* sub-hologram origin and reference wave; all zero = whole plane, R = 1 */
} wasabi_job;

typedef struct wasabi_batch wasabi_batch;

/* max_jobs <= 1024.  holo_side_hint picks the autotuned (or default)
 * superposition configuration of that size class for the whole batch. */
wasabi_status wasabi_batch_create(const wasabi_lut* lut, int max_jobs, int holo_side_hint, int use_graph,
                                  wasabi_batch** out);
/* Waits for the batch's last job-table upload, then frees it. */
wasabi_status wasabi_batch_destroy(wasabi_batch* batch);
/* The batch's super-tile side (pixels) and block size. */
wasabi_status wasabi_batch_config(const wasabi_batch* batch, int* cell_out, int* threads_out);
wasabi_status wasabi_batch_scratch_bytes(const wasabi_batch* batch, const wasabi_job* jobs_host, int njobs,
                                         size_t* bytes_out);
/* Superposition (Eq. (2)) and, for jobs that ask for it, inverse transform
 * and binarisation (Sec. 1 step 3, Sec. 2) of every job; results equal the
 * one-job calls.  jobs_host: njobs descriptors (host memory, read during the
 * call).  E_INVALID / E_NOMEM on bad jobs or short scratch; device-side errors
 * go to the status word. */
wasabi_status wasabi_batch_run(wasabi_batch* batch, const wasabi_job* jobs_host, int njobs, void* scratch_dev,
                               size_t scratch_bytes, void* stream);

/* Autotuner: times the superposition of n synthetic points on a
 * holo_side^2 hologram for super-tiles {64, 128, 192, 256} x blocks {256,
 * 384, 512, 1024} (those that fit), keeps the fastest in the LUT for that size class
 * (holo_side rounded up to a power of two) and returns it.  Later
 * superposition calls and batches of that class use it.  Synchronising;
 * allocates temporary device memory. */
wasabi_status wasabi_autotune(wasabi_lut* lut, int holo_side, int64_t n_points, void* stream, int* cell_out,
                              int* threads_out);

/* ---- Serving loop ---------------------------------------------------------
 * Hologram requests of mixed size and point count, admitted by a device-memory
 * budget and continuously batched.  The server reserves hbm_budget_bytes of
 * device memory once (an arena for every request's points, outputs and
 * binning scratch) and runs one scheduler thread with `streams` CUDA streams.
 * Whenever a stream is free, the scheduler takes requests from the head of the
 * FIFO queue while their buffers fit in the free arena (at most max_batch per
 * launch), uploads their points, runs them as one batch (wasabi_batch_run:
 * superposition with the fused inverse transform and binarisation, replayed
 * from a CUDA graph) and copies the outputs back into the request's host
 * buffers.  Requests arriving while others run join the next launch on a free
 * stream, so their work overlaps on the device.  The LUT stays resident; no
 * wavelet buffer is needed (the fused path keeps it in shared memory).
 * A request's result depends only on its own points and the server's
 * super-tile configuration (picked from holo_side_hint), so it is the same
 * alone and in any mix of requests. */
typedef struct wasabi_server wasabi_server;

typedef struct {
  const wasabi_point* points_host; /* n points in host memory (pinned: asynchronous upload) */
  int64_t n;
  int holo_w, holo_h;               /* multiples of 2^L; holo_w % 8 == 0 for bits */
  int rule;                         /* wasabi_shift_rule */
  uint8_t* bits_host;               /* packed binary hologram (host), or NULL */
  void* u_host;                     /* complex64 row-major field (host), or NULL; not both NULL */
  wasabi_frame frame;               /* sub-hologram origin and reference wave; all zero = whole plane, R = 1 */
} wasabi_request;

typedef struct {
  double submit_s, launch_s, done_s; /* seconds since the server was created: queued, launched,
                                        outputs copied back */
  int batch_jobs;                    /* requests in the launch that carried this one */
  int status;                        /* wasabi_status of the request */
} wasabi_request_info;

/* streams in [1, 16]; max_batch in [1, 1024]; budget >= 1 MiB; levels >= 2.
 * E_NOMEM if the budget cannot be reserved. */
wasabi_status wasabi_server_create(const wasabi_lut* lut, size_t hbm_budget_bytes, int streams,
                                   int max_batch, int holo_side_hint, wasabi_server** out);
/* Queues a request (thread-safe, returns at once with its id).  The host
 * buffers must stay valid until wasabi_server_wait returns for it.
 * E_INVALID on bad sizes, E_RANGE if a point's depth index is >= D (checked
 * on the host), E_NOMEM if the request alone exceeds the budget. */
wasabi_status wasabi_server_submit(wasabi_server* server, const wasabi_request* request, int64_t* id_out);
/* Blocks until the request has finished (its outputs are in host memory),
 * fills *info and forgets the request.  timeout_s <= 0 waits without limit;
 * E_TIMEOUT if it runs out (the request stays queryable).  Returns the
 * request's status. */
wasabi_status wasabi_server_wait(wasabi_server* server, int64_t id, double timeout_s,
                                 wasabi_request_info* info);
/* Peak arena use (bytes), requests completed and launches so far. */
wasabi_status wasabi_server_stats(wasabi_server* server, size_t* peak_bytes, int64_t* completed,
                                  int64_t* launches);
/* Finishes the launches in flight, cancels queued requests (status
 * E_INVALID) and frees the server.  Destroy the server before its LUT. */
wasabi_status wasabi_server_destroy(wasabi_server* server);

/* Eq. (1), the direct sum, on the GPU:
 *   u(x_h, y_h) = sum_j a_j exp(i 2 pi r_hj / lambda) [aperture],
 * r_hj = sqrt(((x_h - x_j)^2 + (y_h - y_j)^2) pitch^2 + z_{d_j}^2), with the
 * point's quantised depth z_{d_j} = depths_host[d_j] (a point behind the plane,
 * z < 0, contributes the conjugate term); aperture = 1 restricts each term to
 * the PSF disk n < R(|z|)^2 and the point's own pixel (the second form of
 * Eq. (1)), 0 sums every pixel.  u_dev: holo_w x holo_h complex64, row-major, overwritten.
 * The phase r / lambda mod 1 is carried in double-float (pairs of FP32 values,
 * about 44 bits) and the disk test is exact in integers; FP32 elsewhere.
 * scratch_dev: at least cgh_direct_scratch_bytes() bytes. */
wasabi_status cgh_direct_scratch_bytes(int64_t n, int holo_w, int holo_h, size_t* bytes_out);
wasabi_status cgh_direct(double lambda, double pitch, const double* depths_host, int n_depths,
                         const wasabi_point* points_dev, int64_t n, int holo_w, int holo_h,
                         int aperture, void* u_dev, void* scratch_dev, size_t scratch_bytes,
                         void* stream);

/* ---- Numerical reconstruction (Sec. 2, Fig. 3(b)) -----------------------
 * The field of the plane at signed distance d from the hologram, by the
 * angular spectrum method: U_d = IFFT2( FFT2(U_0) H ), with
 * H(fx, fy) = exp(i 2 pi d sqrt(1/lambda^2 - fx^2 - fy^2)) for
 * fx^2 + fy^2 < 1/lambda^2 and 0 for evanescent frequencies,
 * fx = k / (w pitch), k in FFT order.  In the sign convention of the object
 * points (Eq. (1) as printed, with a +i sign), a point at depth z comes to
 * focus at d = -z.  The phases of the transfer function and of the reference
 * wave are carried in double-float (pairs of FP32 values, about 44 bits) and
 * reduced to [0, 1); the FFTs are cuFFT C2C transforms in FP32.  Plane
 * pixels (origin plus index) must stay below 2^24 in magnitude.
 * input_kind WASABI_RECON_FIELD: input_dev is a complex64 field (w x h,
 * row-major).  WASABI_RECON_BITS: input_dev is a packed binary hologram
 * (w % 8 == 0), an amplitude transmittance t in {0, 1}, illuminated by the
 * frame's reference wave: U_0 = t R (the frame may be NULL: R = 1, origin 0).
 * Outputs (either may be NULL, not both): field_out_dev complex64 U_d,
 * intensity_out_dev float |U_d|^2, both w x h row-major.
 * scratch_dev: wasabi_reconstruct_scratch_bytes() bytes, 256-byte aligned
 * (the cuFFT work area; calls in flight at once need separate scratch).
 * The cuFFT plans of the first 8 (device, w, h) shapes either function meets
 * are kept for the life of the process, and a call on such a shape is
 * asynchronous on `stream`; for any other shape the plan lives for the call
 * only and the call returns after the result is in place.  Calls are
 * serialised on the host by one mutex. */
typedef enum { WASABI_RECON_FIELD = 0, WASABI_RECON_BITS = 1 } wasabi_recon_input;
wasabi_status wasabi_reconstruct_scratch_bytes(int w, int h, size_t* bytes_out);
wasabi_status wasabi_reconstruct(const void* input_dev, int input_kind, int w, int h, double lambda, double pitch,
                                 double d, const wasabi_frame* frame, void* field_out_dev,
                                 float* intensity_out_dev, void* scratch_dev, size_t scratch_bytes,
                                 void* stream);

/* Synchronises `stream`, then returns and clears the current device's status
 * word: WASABI_OK, WASABI_E_RANGE or WASABI_E_TIMEOUT (E_CUDA if the stream
 * itself failed). */
wasabi_status wasabi_sync_status(void* stream);

/* Test exports.  Forward L-level Haar of a row-major complex64 image into the
 * tile-major layout (the inverse of wasabi_inverse_haar's complex output),
 * and the permutation of a tile-major buffer into the whole-image Mallat
 * layout (row-major complex64, holo_w x holo_h). */
wasabi_status wasabi_haar_forward(const void* u_dev, int holo_w, int holo_h, int levels,
                                  void* wbuf_dev, void* stream);
wasabi_status wasabi_wbuf_to_mallat(const void* wbuf_dev, int holo_w, int holo_h, int levels,
                                    void* mallat_dev, void* stream);

/* Test export: the separate inverse transform to bits (as
 * wasabi_inverse_haar with u_dev = NULL and the plane reference), except that
 * the bulk copy of strip `skip_strip` (strips are 256 pixels x 2^levels rows,
 * numbered row-major) is never issued and every stage wait gives up after
 * `wait_cycles` SM clock cycles (1 .. 4e9; the normal calls use 4e9, about
 * 2 s).  The CTA that owns the strip stops waiting, lets its copies in flight
 * land and exits; the call then reports WASABI_E_TIMEOUT through
 * wasabi_sync_status, and the context stays usable.  It exercises the failure
 * path of the bounded waits (failure detection without a GPU fault); the bits
 * of the skipped strip and of the strips after it in that CTA are left
 * unwritten. */
wasabi_status wasabi_test_inverse_stall(const void* wbuf_dev, int holo_w, int holo_h, int levels,
                                        uint8_t* bits_dev, int64_t skip_strip, int64_t wait_cycles,
                                        void* stream);

#ifdef __cplusplus
}
#endif
#endif /* WASABI_H */
