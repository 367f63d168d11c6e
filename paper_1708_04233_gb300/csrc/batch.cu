// Batched hologram synthesis (many jobs, one launch sequence) and the
// autotuner of the superposition's super-tile and block sizes.
//
// A batch runs every job through the same five launches -- zero, count, scan,
// scatter (binning) and superpose, whose epilogue also runs the inverse
// transform and binarisation of each finished super-tile -- with grids that
// do not depend on the batch: the work items (super-tiles of all jobs) are
// claimed from the device-side job table.  The launch sequence, together with the upload
// of the job table from pinned host memory, is captured once into a CUDA
// graph and replayed for every later batch (when the caller's stream allows
// capture).
#include <algorithm>
#include <cstring>
#include <vector>

#include "internal.cuh"
#include "lut_object.h"

using namespace wsb;

struct wasabi_batch {
  const wasabi_lut* lut = nullptr;
  int device = 0;
  int max_jobs = 0;
  int cell = 128, threads = 512;
  bool use_graph = false;
  JobDev* staging_jobs = nullptr;   // pinned host
  BatchDev* staging_batch = nullptr;
  JobDev* jobs_dev = nullptr;       // device
  BatchDev* batch_dev = nullptr;
  cudaEvent_t staged = nullptr;     // the last upload of the staging buffers has completed
  bool staged_pending = false;
  // One graph per accumulation mode (complex, or real parts only when every
  // job wants bits alone), each bound to the stream it was captured on.
  // One graph per kernel mode: complex accumulation, real parts only,
  // complex with the spherical-reference epilogue.
  cudaGraphExec_t exec[3] = {nullptr, nullptr, nullptr};
  cudaStream_t graph_stream[3] = {nullptr, nullptr, nullptr};
};

namespace {

// Scratch bytes of one job: cell arrays and binned points.
size_t job_scratch(const wasabi_job& j, int cell) {
  const size_t ncx = (size_t)(j.holo_w + cell - 1) / cell, ncy = (size_t)(j.holo_h + cell - 1) / cell;
  const size_t nc = ncx * ncy;
  return align_up((nc + 1) * 4, 256) + align_up((nc + 1) * 4, 256) + align_up(nc * 4, 256) +
         align_up((size_t)std::max<int64_t>(j.n, 1) * sizeof(wasabi_point), 256);
}

wasabi_status check_job(const wasabi_lut* lut, const wasabi_job& j, int idx) {
  const int ts = 1 << lut->L;
  if (j.n < 0 || (j.n > 0 && !j.points_dev) || (!j.wbuf_dev && !j.u_dev && !j.bits_dev) || j.holo_w < ts ||
      j.holo_h < ts ||
      j.holo_w % ts || j.holo_h % ts || j.holo_w > (1 << 29) || j.holo_h > (1 << 29) ||
      (j.rule != WASABI_SHIFT_FLOOR && j.rule != WASABI_SHIFT_NEAREST)) {
    set_error("batch: job %d has bad arguments", idx);
    return WASABI_E_INVALID;
  }
  if ((j.u_dev || j.bits_dev) && lut->wavelet != WASABI_HAAR) {
    set_error("batch: job %d asks for the fused inverse, which is Haar's", idx);
    return WASABI_E_INVALID;
  }
  if ((j.u_dev || j.bits_dev) && lut->L < 2) {
    set_error("batch: job %d asks for an inverse, which needs levels >= 2", idx);
    return WASABI_E_INVALID;
  }
  if (j.bits_dev && j.holo_w % 8) {
    set_error("batch: job %d: bits output needs holo_w %% 8 == 0", idx);
    return WASABI_E_INVALID;
  }
  if (((uintptr_t)j.wbuf_dev & 255) || ((uintptr_t)j.u_dev & 15) || ((uintptr_t)j.bits_dev & 3)) {
    set_error("batch: job %d: misaligned buffer", idx);
    return WASABI_E_INVALID;
  }
  int ox, oy;
  RefDev ref;
  const char* why = "";
  if (!frame_to_dev(&j.frame, &ox, &oy, &ref, &why)) {
    set_error("batch: job %d: %s", idx, why);
    return WASABI_E_INVALID;
  }
  return WASABI_OK;
}

// Enqueues the upload and the five launches of a batch on s.  Under stream
// capture the record of `staged` becomes an external event node, so the host
// can wait on it after each replay.
cudaError_t enqueue_batch(wasabi_batch* b, cudaStream_t s, int* status, int sms, bool capturing, int mode) {
  const bool re_only = mode == 1;
  cudaError_t e = cudaMemcpyAsync(b->jobs_dev, b->staging_jobs, sizeof(JobDev) * b->max_jobs,
                                  cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->batch_dev, b->staging_batch, sizeof(BatchDev), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = capturing ? cudaEventRecordWithFlags(b->staged, s, cudaEventRecordExternal) : cudaEventRecord(b->staged, s);
  if (e != cudaSuccess) return e;
  const wasabi_lut* lut = b->lut;
  BinArgs ba;
  ba.jobs = b->jobs_dev; ba.batch = b->batch_dev; ba.D = lut->D; ba.cell = b->cell; ba.reach = lut->reach;
  ba.track_amax = 1; ba.status = status; ba.grid = sms * 4;
  if ((e = launch_binning(ba, s)) != cudaSuccess) return e;
  SuperposeArgs sa;
  sa.lut = lut->view(b->cell >> lut->L);
  sa.jobs = b->jobs_dev; sa.batch = b->batch_dev; sa.cell = b->cell; sa.reach = lut->reach;
  sa.acc_float = 0; sa.status = status; sa.threads = b->threads; sa.grid = sms;
  sa.re_only = re_only ? 1 : 0;
  sa.has_ref = mode == 2 ? 1 : 0;
  sa.rcap = superpose_range_cap(b->cell, lut->L, lut->lmin, lut->D, re_only, b->threads);
  if ((e = launch_superpose(sa, s)) != cudaSuccess) return e;
  return cudaSuccess;
}

// Synthetic points for tuning: positions uniform over the hologram (an
// integer hash of the index), depths uniform over the LUT, amplitudes in (0, 1].
__global__ void synth_points_kernel(wasabi_point* p, int64_t n, int w, int h, int D) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  auto mix = [](uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  const uint64_t r0 = mix((uint64_t)i * 4 + 1), r1 = mix((uint64_t)i * 4 + 2), r2 = mix((uint64_t)i * 4 + 3);
  wasabi_point q;
  q.x = (int32_t)(r0 % (uint64_t)w);
  q.y = (int32_t)(r1 % (uint64_t)h);
  q.d = (uint32_t)(r2 % (uint64_t)D);
  q.a = 1.0f - (float)((r2 >> 40) & 0xffffff) / 16777216.0f;
  p[i] = q;
}

}  // namespace

extern "C" {

wasabi_status wasabi_batch_create(const wasabi_lut* lut, int max_jobs, int holo_side_hint, int use_graph,
                                  wasabi_batch** out) {
  if (!out || !lut || max_jobs < 1 || max_jobs > kMaxJobs) {
    set_error("batch_create: need a LUT, an output and 1 <= max_jobs <= %d", kMaxJobs);
    return WASABI_E_INVALID;
  }
  *out = nullptr;
  int* status;
  int sms;
  if (!device_info(&status, &sms)) return WASABI_E_CUDA;
  wasabi_batch* b = new wasabi_batch;
  b->lut = lut;
  cudaGetDevice(&b->device);
  b->max_jobs = max_jobs;
  b->use_graph = use_graph != 0;
  const int side = holo_side_hint > 0 ? holo_side_hint : 4096;
  superpose_config(lut, side, side, kConfigShared, &b->cell, &b->threads);
  cudaError_t e = cudaMallocHost(&b->staging_jobs, sizeof(JobDev) * max_jobs);
  if (e == cudaSuccess) e = cudaMallocHost(&b->staging_batch, sizeof(BatchDev));
  if (e == cudaSuccess) e = cudaMalloc(&b->jobs_dev, sizeof(JobDev) * max_jobs);
  if (e == cudaSuccess) e = cudaMalloc(&b->batch_dev, sizeof(BatchDev));
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->staged, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    wasabi_batch_destroy(b);
    set_error("batch_create: %s", cudaGetErrorString(e));
    return WASABI_E_NOMEM;
  }
  std::memset(b->staging_jobs, 0, sizeof(JobDev) * max_jobs);
  std::memset(b->staging_batch, 0, sizeof(BatchDev));
  *out = b;
  return WASABI_OK;
}

wasabi_status wasabi_batch_destroy(wasabi_batch* b) {
  if (!b) return WASABI_OK;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(b->device);
  if (b->staged) cudaEventSynchronize(b->staged);
  for (int m = 0; m < 3; ++m)
    if (b->exec[m]) cudaGraphExecDestroy(b->exec[m]);
  if (b->staged) cudaEventDestroy(b->staged);
  if (b->jobs_dev) cudaFree(b->jobs_dev);
  if (b->batch_dev) cudaFree(b->batch_dev);
  if (b->staging_jobs) cudaFreeHost(b->staging_jobs);
  if (b->staging_batch) cudaFreeHost(b->staging_batch);
  cudaSetDevice(prev);
  cudaGetLastError();  // nothing above is reported; leave no stale error behind
  delete b;
  return WASABI_OK;
}

wasabi_status wasabi_batch_config(const wasabi_batch* b, int* cell_out, int* threads_out) {
  if (!b) { set_error("batch_config: NULL batch"); return WASABI_E_INVALID; }
  if (cell_out) *cell_out = b->cell;
  if (threads_out) *threads_out = b->threads;
  return WASABI_OK;
}

wasabi_status wasabi_batch_scratch_bytes(const wasabi_batch* b, const wasabi_job* jobs, int njobs, size_t* bytes) {
  if (!b || !bytes || njobs < 0 || (njobs > 0 && !jobs)) { set_error("batch_scratch_bytes: bad arguments"); return WASABI_E_INVALID; }
  size_t total = 0;
  for (int i = 0; i < njobs; ++i) total += job_scratch(jobs[i], b->cell);
  *bytes = total;
  return WASABI_OK;
}

wasabi_status wasabi_batch_run(wasabi_batch* b, const wasabi_job* jobs, int njobs, void* scratch_dev,
                               size_t scratch_bytes, void* stream) {
  if (!b || njobs < 0 || njobs > b->max_jobs || (njobs > 0 && (!jobs || !scratch_dev))) {
    set_error("batch_run: bad arguments (njobs %d, capacity %d)", njobs, b ? b->max_jobs : 0);
    return WASABI_E_INVALID;
  }
  if ((uintptr_t)scratch_dev & 255) { set_error("batch_run: scratch must be 256-byte aligned"); return WASABI_E_INVALID; }
  const wasabi_lut* lut = b->lut;
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != b->device || cur != lut->device) { set_error("batch_run: batch or LUT lives on another device"); return WASABI_E_INVALID; }
  size_t need = 0;
  for (int i = 0; i < njobs; ++i) {
    const wasabi_status st = check_job(lut, jobs[i], i);
    if (st != WASABI_OK) return st;
    need += job_scratch(jobs[i], b->cell);
  }
  if (scratch_bytes < need) {
    set_error("batch_run: scratch too small (%zu < %zu bytes)", scratch_bytes, need);
    return WASABI_E_NOMEM;
  }
  if ((b->cell + 2 * lut->reach) / b->cell + 2 > superpose_max_cell_rows()) {
    set_error("batch_run: window too large for the super-tile");
    return WASABI_E_INVALID;
  }
  int* status;
  int sms;
  if (!device_info(&status, &sms)) return WASABI_E_CUDA;
  // The staging buffers may still be read by the previous batch's upload.
  if (b->staged_pending) {
    const cudaError_t e = cudaEventSynchronize(b->staged);
    if (e != cudaSuccess) return cuda_fail("batch_run: wait for staging", e);
  }
  const int k = b->cell >> lut->L;
  Carver c;
  c.base = static_cast<char*>(scratch_dev);
  long long pt0 = 0;
  int sp0 = 0;
  for (int i = 0; i < njobs; ++i) {
    const wasabi_job& j = jobs[i];
    JobDev& J = b->staging_jobs[i];
    std::memset(&J, 0, sizeof J);
    J.pts = j.points_dev;
    J.wbuf = static_cast<float2*>(j.wbuf_dev);
    J.u = static_cast<float2*>(j.u_dev);
    J.bits = j.bits_dev;
    J.n = j.n;
    J.w = j.holo_w;
    J.h = j.holo_h;
    J.ntx = j.holo_w >> lut->L;
    J.nty = j.holo_h >> lut->L;
    J.ncx = (j.holo_w + b->cell - 1) / b->cell;
    J.ncy = (j.holo_h + b->cell - 1) / b->cell;
    J.ncells = J.ncx * J.ncy;
    J.rule = j.rule;
    const char* why = "";
    frame_to_dev(&j.frame, &J.ox, &J.oy, &J.ref, &why);  // checked above
    J.cnt = c.take<int>((size_t)J.ncells + 1);
    J.off = c.take<int>((size_t)J.ncells + 1);
    J.cursor = c.take<int>((size_t)J.ncells);
    J.sorted = c.take<wasabi_point>((size_t)std::max<int64_t>(j.n, 1));
    J.pt0 = pt0;
    J.sp0 = sp0;
    pt0 += j.n;
    sp0 += ((J.ntx + k - 1) / k) * ((J.nty + k - 1) / k);
  }
  BatchDev& B = *b->staging_batch;
  std::memset(&B, 0, sizeof B);
  B.njobs = njobs;
  B.nsp = sp0;
  B.npts = pt0;
  bool re_only = njobs > 0;
  for (int i = 0; i < njobs; ++i)
    re_only = re_only && !jobs[i].wbuf_dev && !jobs[i].u_dev && jobs[i].bits_dev && !frame_needs_complex(&jobs[i].frame);
  bool has_ref = false;
  for (int i = 0; i < njobs; ++i) has_ref = has_ref || (jobs[i].bits_dev && frame_needs_complex(&jobs[i].frame));
  const int m = re_only ? 1 : has_ref ? 2 : 0;
  const cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (b->use_graph && s != nullptr) {
    if (!b->exec[m] || b->graph_stream[m] != s) {
      if (b->exec[m]) { cudaGraphExecDestroy(b->exec[m]); b->exec[m] = nullptr; }
      cudaGraph_t g = nullptr;
      e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        const cudaError_t e2 = enqueue_batch(b, s, status, sms, true, m);
        e = cudaStreamEndCapture(s, &g);
        if (e2 != cudaSuccess) e = e2;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec[m], g, 0);
      if (g) cudaGraphDestroy(g);
      if (e != cudaSuccess) { b->exec[m] = nullptr; return cuda_fail("batch_run: graph capture", e); }
      b->graph_stream[m] = s;
    }
    e = cudaGraphLaunch(b->exec[m], s);
  } else {
    e = enqueue_batch(b, s, status, sms, false, m);
  }
  if (e != cudaSuccess) return cuda_fail("batch_run: launch", e);
  b->staged_pending = true;
  return WASABI_OK;
}

wasabi_status wasabi_autotune(wasabi_lut* lut, int holo_side, int64_t n_points, void* stream, int* cell_out,
                              int* threads_out) {
  if (!lut || holo_side < (1 << lut->L) || holo_side % (1 << lut->L) || n_points < 1) {
    set_error("autotune: bad arguments");
    return WASABI_E_INVALID;
  }
  const cudaStream_t s = (cudaStream_t)stream;
  const int side = holo_side;
  wasabi_point* pts = nullptr;
  void* wbuf = nullptr;
  void* scratch = nullptr;
  size_t sbytes = 0;
  wasabi_scratch_bytes(lut, n_points, side, side, &sbytes);
  cudaError_t e = cudaMallocAsync((void**)&pts, sizeof(wasabi_point) * (size_t)n_points, s);
  if (e == cudaSuccess) e = cudaMallocAsync(&wbuf, sizeof(float2) * (size_t)side * side, s);
  if (e == cudaSuccess) e = cudaMallocAsync(&scratch, sbytes, s);
  if (e != cudaSuccess) {
    if (pts) cudaFreeAsync(pts, s);
    if (wbuf) cudaFreeAsync(wbuf, s);
    set_error("autotune: allocation: %s", cudaGetErrorString(e));
    return WASABI_E_NOMEM;
  }
  synth_points_kernel<<<(unsigned)((n_points + 255) / 256), 256, 0, s>>>(pts, n_points, side, side, lut->D);
  cudaEvent_t t0, t1;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  int best_cell = 0, best_threads = 0;
  float best = 1e30f;
  const int cells[] = {64, 128, 192, 256};
  const int tcounts[] = {256, 384, 512, 1024};
  for (int cell : cells) {
    if (cell < std::max(1 << lut->L, 32) || superpose_smem_bytes(cell, lut->L, lut->lmin, lut->D, false, superpose_min_range_cap()) > 220 * 1024)
      continue;
    for (int nt : tcounts) {
      if (nt < superpose_min_threads()) continue;
      float ms = 0.f;
      bool ok = superpose_impl(lut, pts, n_points, side, side, 0, wbuf, nullptr, nullptr, scratch, sbytes, s, cell, nt) == WASABI_OK;
      ok = ok && cudaEventRecord(t0, s) == cudaSuccess;
      for (int r = 0; r < 3 && ok; ++r)
        ok = superpose_impl(lut, pts, n_points, side, side, 0, wbuf, nullptr, nullptr, scratch, sbytes, s, cell, nt) == WASABI_OK;
      ok = ok && cudaEventRecord(t1, s) == cudaSuccess && cudaEventSynchronize(t1) == cudaSuccess &&
           cudaEventElapsedTime(&ms, t0, t1) == cudaSuccess;
      if (ok && ms < best) { best = ms; best_cell = cell; best_threads = nt; }
    }
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  cudaFreeAsync(pts, s);
  cudaFreeAsync(wbuf, s);
  cudaFreeAsync(scratch, s);
  if (!best_cell) { set_error("autotune: no configuration ran"); return WASABI_E_CUDA; }
  {
    std::lock_guard<std::mutex> lk(lut->tune_mu);
    lut->tuned[size_class(side, side)] = std::make_pair(best_cell, best_threads);
  }
  if (cell_out) *cell_out = best_cell;
  if (threads_out) *threads_out = best_threads;
  return WASABI_OK;
}

}  // extern "C"
