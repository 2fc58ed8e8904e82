// C-ABI of libdic (declared in include/dic.h): handle life cycle, argument
// checks, device buffers, the wave loop and result export. Every computation of
// the method runs in the kernels of prefilter.cu, seed.cu and correlate.cu.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <string>
#include <unordered_map>
#include <vector>

#include "dic_internal.cuh"

using namespace dic;

namespace {

thread_local std::string g_last_error;
// dic_test_expire_tile_waits: 1 makes every later wave launch give up its tile waits
std::atomic<int> g_expire_waits{0};

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? DIC_ENOMEM : DIC_ECUDA, "%s: %s", what,
              cudaGetErrorString(e));
}

#define DIC_CUDA(call, what)                      \
  do {                                            \
    cudaError_t e_ = (call);                      \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

size_t dtype_size(int dt) {
  switch (dt) {
    case DIC_U8: return 1;
    case DIC_U16: return 2;
    case DIC_BF16: return 2;
    case DIC_F32: return 4;
    case DIC_F64: return 8;
    default: return 0;
  }
}

int nparams_of(int shape) { return shape == DIC_RIGID ? 2 : shape == DIC_AFFINE ? 6 : 12; }

int64_t floor_div(int64_t a, int64_t b) {
  int64_t q = a / b;
  if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
  return q;
}

template <typename P>
int dev_alloc(P** ptr, size_t count, const char* what) {
  void* raw = nullptr;
  cudaError_t e = cudaMalloc(&raw, count * sizeof(P) > 0 ? count * sizeof(P) : 1);
  if (e != cudaSuccess) {
    *ptr = nullptr;
    return cuda_fail(e, what);
  }
  *ptr = static_cast<P*>(raw);
  return DIC_OK;
}

void dev_free(void* p) {
  if (p) cudaFree(p);
}

}  // namespace

struct dic_handle {
  int W = 0, H = 0, S = 0, step = 0, r = 0, shape = 0, nparams = 0, nx = 0, ny = 0;
  int interp = DIC_BSPLINE3;  // dic_interp of both coefficient planes
  int64_t npts = 0;
  dic_params prm{};
  int device = 0;
  // images: borrowed device pointers or owned copies
  GrayPlane ref{}, def{};
  void* ref_owned = nullptr;
  void* def_owned = nullptr;
  int ref_dtype = 0, def_dtype = 0;
  bool ref_dirty = true, def_dirty = true;
  // ROI flags per point (NULL: all in)
  uint8_t* roi_ok = nullptr;
  // TMA descriptors of the reference coefficients, deformed coefficients and
  // reference gray plane (valid when the matching flag is set)
  CUtensorMap maps[3];
  int maps_ok[3] = {0, 0, 0};
  int maps_prec = -1;
  // spline coefficient planes in the working precision
  void* c_ref = nullptr;
  void* c_def = nullptr;
  int64_t ldc = 0;
  int plane_prec = -1;
  // per-point state
  int32_t* x = nullptr;
  int32_t* y = nullptr;
  double* u = nullptr;
  double* v = nullptr;
  double* p = nullptr;
  float* zncc = nullptr;
  int64_t* accept = nullptr;
  int32_t* iters = nullptr;
  int32_t* wave = nullptr;
  uint8_t* conv = nullptr;
  uint8_t* status = nullptr;
  // frontier
  int32_t* front[2] = {nullptr, nullptr};
  int32_t* counters = nullptr;
  int32_t* wave_sizes = nullptr;
  int32_t* h_counters = nullptr;  // pinned, [kBatchSlots][kNumCounters]
  // seeds
  int32_t* seed_xy = nullptr;
  int32_t* seed_q = nullptr;
  int32_t* seed_best = nullptr;
  double* seed_scores = nullptr;
  size_t seed_cap = 0, score_cap = 0;
  // host copies of the results
  void* h_res = nullptr;
  size_t h_res_bytes = 0;
  // device allocations owned by the handle and their requested sizes
  std::unordered_map<void*, size_t> allocs;
  int64_t device_bytes = 0;
  // capacity of the per-point arrays (points; elements of p)
  int64_t pts_cap = 0;
  int64_t p_cap = 0;
  bool grid_ok = false;
  // stream of the last correlation (result read-back is ordered on it)
  cudaStream_t last_stream = nullptr;
  // last run
  bool has_results = false;
  int n_waves = 0;
  int64_t n_accepted = 0;
  dic_timing timing{};
  std::vector<cudaEvent_t> events;       // stage boundaries
  std::vector<cudaEvent_t> wave_events;  // two per wave kernel when profiling
  cudaEvent_t batch_ev[2] = {nullptr, nullptr};
  // multi-window FFT initialiser: twiddles (and the odd length they hold), window
  // origins, per-level raw and filtered fields, large-window scratch, results
  float2* fft_tw = nullptr;
  int fft_tw_odd = -1;
  int4* fft_org = nullptr;
  float* fft_raw[3] = {nullptr, nullptr, nullptr};       // u, v, peak
  float* fft_filt[4] = {nullptr, nullptr, nullptr, nullptr};  // ping-pong (u, v) x 2
  float2* fft_work = nullptr;
  double* fft_norms = nullptr;
  unsigned long long* fft_keys = nullptr;
  int32_t* fft_nonflat = nullptr;
  float* fft_res[3] = {nullptr, nullptr, nullptr};       // u, v, peak per grid point
  uint8_t* fft_status = nullptr;
  uint8_t* fft_rep = nullptr;
  int64_t fft_win_cap = 0, fft_mid_cap = 0, fft_large_cap = 0, fft_work_cap = 0, fft_res_cap = 0;
  bool has_fft = false;
  int fft_levels = 0;
  int fft_window[kFftMaxLevels] = {};
  // incremental reference updating: accumulated warps from the first reference, and
  // the total warps of the last frame
  double* acc_u = nullptr;
  double* acc_v = nullptr;
  double* acc_A = nullptr;
  uint8_t* acc_ok = nullptr;
  double* tot_u = nullptr;
  double* tot_v = nullptr;
  double* tot_p = nullptr;
  uint8_t* tot_status = nullptr;
  int64_t inc_cap = 0, tot_p_cap = 0;
  bool acc_identity = true;
  int n_updates = 0;
};

namespace {

constexpr int kBatchSlots = 2;

// Device allocation owned by a handle: counted in device_bytes until hfree.
template <typename P>
int halloc(dic_handle* h, P** ptr, size_t count, const char* what) {
  int rc = dev_alloc(ptr, count, what);
  if (rc) return rc;
  const size_t bytes = count * sizeof(P) > 0 ? count * sizeof(P) : 1;
  h->allocs[static_cast<void*>(*ptr)] = bytes;
  h->device_bytes += static_cast<int64_t>(bytes);
  return DIC_OK;
}

template <typename P>
void hfree(dic_handle* h, P*& ptr) {
  if (!ptr) return;
  auto it = h->allocs.find(static_cast<void*>(ptr));
  if (it != h->allocs.end()) {
    h->device_bytes -= static_cast<int64_t>(it->second);
    h->allocs.erase(it);
  }
  dev_free(ptr);
  ptr = nullptr;
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  // initialised once, thread-safely, on first use
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    return nullptr;
  }();
  return fn;
}

// 2-D tiled tensor map of a row-major plane; false when the driver call is
// unavailable or the plane breaks a TMA rule (16-byte aligned base and pitch).
bool encode_plane(CUtensorMap* map, CUtensorMapDataType type, const void* base, int W, int H,
                  int64_t pitch_bytes, int box_w, int box_h) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc || !base) return false;
  if ((reinterpret_cast<uintptr_t>(base) & 15) != 0 || (pitch_bytes & 15) != 0) return false;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(W), static_cast<cuuint64_t>(H)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(pitch_bytes)};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(box_w), static_cast<cuuint32_t>(box_h)};
  cuuint32_t estr[2] = {1, 1};
  return enc(map, type, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

CUtensorMapDataType gray_map_type(int dtype) {
  switch (dtype) {
    case DIC_U8: return CU_TENSOR_MAP_DATA_TYPE_UINT8;
    case DIC_U16: return CU_TENSOR_MAP_DATA_TYPE_UINT16;
    case DIC_BF16: return CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    case DIC_F32: return CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    default: return CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
  }
}

int check_image(const dic_image* im, const char* name) {
  if (!im) return fail(DIC_EINVAL, "%s image is NULL", name);
  if (!im->data) return fail(DIC_EINVAL, "%s image has no data", name);
  if (dtype_size(im->dtype) == 0) return fail(DIC_EINVAL, "%s image has an unknown dtype %d", name, im->dtype);
  if (im->width < 8 || im->height < 8)
    return fail(DIC_EINVAL, "%s image is %dx%d; at least 8x8 is needed", name, im->width, im->height);
  const int64_t min_stride = static_cast<int64_t>(im->width) * dtype_size(im->dtype);
  if (im->row_stride_bytes != 0 && im->row_stride_bytes < min_stride)
    return fail(DIC_EINVAL, "%s image row stride %lld is below width * element size", name,
                static_cast<long long>(im->row_stride_bytes));
  return DIC_OK;
}

// owned image copies get a 128-byte row pitch so that tiles can be loaded by TMA
size_t owned_pitch(const dic_image* im) {
  const size_t row_bytes = static_cast<size_t>(im->width) * dtype_size(im->dtype);
  return (row_bytes + 127) & ~static_cast<size_t>(127);
}

// Adopts a device image or copies a host image into a device buffer; the buffer
// is tracked by the handle when h is given, else the caller frees it.
int bind_image(dic_handle* h, const dic_image* im, GrayPlane* plane, void** owned, int* dtype_out) {
  const size_t es = dtype_size(im->dtype);
  const int64_t stride = im->row_stride_bytes ? im->row_stride_bytes : im->width * static_cast<int64_t>(es);
  const size_t row_bytes = static_cast<size_t>(im->width) * es;
  if (im->on_device) {
    plane->data = im->data;
    plane->stride = stride;
  } else {
    const size_t pitch = owned_pitch(im);
    if (!*owned) {
      uint8_t* buf = nullptr;
      int rc = h ? halloc(h, &buf, pitch * im->height, "image buffer")
                 : dev_alloc(&buf, pitch * im->height, "image buffer");
      if (rc) return rc;
      *owned = buf;
    }
    // one linear copy when the rows are contiguous on both sides (a 2-D copy moves
    // the image row by row)
    if (stride == static_cast<int64_t>(pitch)) {
      DIC_CUDA(cudaMemcpy(*owned, im->data, pitch * im->height, cudaMemcpyHostToDevice), "image upload");
    } else {
      DIC_CUDA(cudaMemcpy2D(*owned, pitch, im->data, stride, row_bytes, im->height, cudaMemcpyHostToDevice),
               "image upload");
    }
    plane->data = *owned;
    plane->stride = static_cast<int64_t>(pitch);
  }
  plane->dtype = im->dtype;
  *dtype_out = im->dtype;
  return DIC_OK;
}

void free_planes(dic_handle* h) {
  hfree(h, h->c_ref);
  hfree(h, h->c_def);
  h->plane_prec = -1;
}

// Element type of the coefficient planes of a precision: DIC_FP64 (double) or
// DIC_MIXED (float; also for DIC_MIXED_FP64_SOLVE).
int plane_kind(int precision) { return precision == DIC_FP64 ? DIC_FP64 : DIC_MIXED; }

int ensure_planes(dic_handle* h) {
  const int prec = plane_kind(h->prm.precision);
  if (h->plane_prec == prec) return DIC_OK;
  free_planes(h);
  const size_t es = prec == DIC_FP64 ? sizeof(double) : sizeof(float);
  h->ldc = (h->W + 31) & ~31;
  const size_t bytes = es * static_cast<size_t>(h->ldc) * h->H;
  uint8_t* cr = nullptr;
  uint8_t* cd = nullptr;
  int rc = halloc(h, &cr, bytes, "reference coefficients");
  if (rc) return rc;
  h->c_ref = cr;
  rc = halloc(h, &cd, bytes, "deformed coefficients");
  if (rc) return rc;
  h->c_def = cd;
  h->plane_prec = prec;
  h->ref_dirty = h->def_dirty = true;
  return DIC_OK;
}

cudaEvent_t pool_event(std::vector<cudaEvent_t>& pool, size_t i) {
  while (pool.size() <= i) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    pool.push_back(e);
  }
  return pool[i];
}

cudaEvent_t event_at(dic_handle* h, size_t i) { return pool_event(h->events, i); }

float elapsed(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) return 0.f;
  return ms;
}

template <typename T>
int prefilter(dic_handle* h, const GrayPlane& src, void* dst, cudaStream_t s) {
  PrefilterArgs<T> a{src, h->W, h->H, static_cast<T*>(dst), h->ldc};
  if (h->interp == DIC_BICUBIC) {
    DIC_CUDA(launch_gray_plane<T>(a, s), "gray plane launch");
  } else {
    DIC_CUDA(launch_prefilter<T>(a, s), "prefilter launch");
  }
  return DIC_OK;
}

PointArrays point_arrays(dic_handle* h) {
  PointArrays pa{};
  pa.n = h->npts;
  pa.nx = h->nx;
  pa.ny = h->ny;
  pa.u = h->u;
  pa.v = h->v;
  pa.p = h->p;
  pa.zncc = h->zncc;
  pa.accept = h->accept;
  pa.iters = h->iters;
  pa.converged = h->conv;
  pa.status = h->status;
  pa.wave = h->wave;
  return pa;
}

template <typename T>
int run_waves(dic_handle* h, cudaStream_t s) {
  WaveArgs<T> a{};
  a.W = h->W;
  a.H = h->H;
  a.ref_gray = h->ref;
  a.c_ref = static_cast<const T*>(h->c_ref);
  a.c_def = static_cast<const T*>(h->c_def);
  a.ldc = h->ldc;
  a.S = h->S;
  a.r = h->r;
  a.step = h->step;
  a.nx = h->nx;
  a.ny = h->ny;
  a.threads = wave_threads(h->S);
  wave_bands(h->S, a.threads, &a.bands, &a.band_h);
  a.tiles = wave_tiles<T>(h->S, h->ref.dtype);
  {
    const CUtensorMapDataType ct = sizeof(T) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const int64_t cp = h->ldc * static_cast<int64_t>(sizeof(T));
    h->maps_ok[0] = encode_plane(&h->maps[0], ct, h->c_ref, h->W, h->H, cp, a.tiles.bxc, a.tiles.byc);
    h->maps_ok[1] = encode_plane(&h->maps[1], ct, h->c_def, h->W, h->H, cp, a.tiles.bxc, a.tiles.byc);
    h->maps_ok[2] = encode_plane(&h->maps[2], gray_map_type(h->ref.dtype), h->ref.data, h->W, h->H,
                                 h->ref.stride, a.tiles.bxg, h->S);
    a.tiles.coef_tma = h->maps_ok[0] && h->maps_ok[1];
    a.tiles.gray_tma = h->maps_ok[2];
  }
  a.pts = point_arrays(h);
  a.roi_ok = h->roi_ok;
  a.counters = h->counters;
  a.wave_sizes = h->wave_sizes;
  a.max_iter = h->prm.max_iter;
  a.cost = h->prm.cost;
  a.lm = h->prm.optimizer == DIC_OPT_LEVENBERG_MARQUARDT;
  a.interp = h->interp;
  a.conv_threshold = h->prm.conv_threshold;
  a.zncc_min = h->prm.zncc_min;
  a.expire_waits = g_expire_waits.load();
  a.solve64 = h->prm.precision == DIC_MIXED_FP64_SOLVE ? 1 : 0;
  if (a.solve64 && h->interp != DIC_BSPLINE3)
    return fail(DIC_EINVAL, "DIC_MIXED_FP64_SOLVE runs on the B-spline interpolant only");

  int sms = 0;
  DIC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device), "device query");
  const size_t smem = static_cast<size_t>(a.tiles.smem_bytes);
  const int per_sm = wave_blocks_per_sm<T>(h->nparams, a.threads, wave_mode(a.lm, a.cost, a.interp, a.solve64), smem);
  const int grid = sms * per_sm;

  const bool prof = h->prm.profile != 0;
  const int64_t max_waves = h->npts + 2;
  int64_t launched = 0;
  int batch = 4;
  int pending_slot = -1;
  int64_t pending_end = 0;
  int slot = 0;
  cudaEvent_t* batch_ev = h->batch_ev;
  for (int i = 0; i < kBatchSlots; ++i)
    if (!batch_ev[i] && cudaEventCreateWithFlags(&batch_ev[i], cudaEventDisableTiming) != cudaSuccess)
      return fail(DIC_ECUDA, "event creation failed");
  // A non-empty wave holds at least one point never attempted before, so at most
  // npts waves are non-empty and the front of wave npts is empty: launching up to
  // max_waves waves always reaches an empty front. Batches are clipped to that
  // bound; the loop fails only when every allowed wave has been launched and the
  // last batch still left a front.
  bool done = false;
  while (!done) {
    if (launched >= max_waves) {
      if (pending_slot >= 0) {
        DIC_CUDA(cudaEventSynchronize(batch_ev[pending_slot]), "wave batch wait");
        const int32_t* pc = h->h_counters + pending_slot * kNumCounters;
        if (pc[kCount + pending_end % 3] == 0) break;
      }
      return fail(DIC_ETIMEOUT, "wave loop exceeded %lld waves", (long long)max_waves);
    }
    const int nb = static_cast<int>(batch < max_waves - launched ? batch : max_waves - launched);
    for (int b = 0; b < nb; ++b) {
      const int64_t k = launched + b;
      a.k = static_cast<int>(k);
      a.cur = h->front[k & 1];
      a.next = h->front[(k + 1) & 1];
      if (prof) {
        cudaEvent_t e0 = pool_event(h->wave_events, 2 * k), e1 = pool_event(h->wave_events, 2 * k + 1);
        if (!e0 || !e1) return fail(DIC_ECUDA, "event creation failed");
        cudaEventRecord(e0, s);
        DIC_CUDA(launch_wave<T>(a, a.tiles, h->maps, h->nparams, grid, s), "wave launch");
        cudaEventRecord(e1, s);
      } else {
        DIC_CUDA(launch_wave<T>(a, a.tiles, h->maps, h->nparams, grid, s), "wave launch");
      }
    }
    launched += nb;
    int32_t* hc = h->h_counters + slot * kNumCounters;
    DIC_CUDA(cudaMemcpyAsync(hc, h->counters, sizeof(int32_t) * kNumCounters, cudaMemcpyDeviceToHost, s),
             "counter read-back");
    DIC_CUDA(cudaEventRecord(batch_ev[slot], s), "event record");
    if (pending_slot >= 0) {
      DIC_CUDA(cudaEventSynchronize(batch_ev[pending_slot]), "wave batch wait");
      const int32_t* pc = h->h_counters + pending_slot * kNumCounters;
      if (pc[kCount + pending_end % 3] == 0) done = true;
    }
    pending_slot = slot;
    pending_end = launched;
    slot = (slot + 1) % kBatchSlots;
    if (batch < 32) batch *= 2;
  }
  // last non-empty wave
  std::vector<int32_t> sizes(static_cast<size_t>(launched));
  DIC_CUDA(cudaMemcpyAsync(sizes.data(), h->wave_sizes, sizeof(int32_t) * launched, cudaMemcpyDeviceToHost, s),
           "wave sizes");
  DIC_CUDA(cudaStreamSynchronize(s), "wave loop");
  int nw = 0;
  int64_t attempted = 0;
  for (int64_t k = 0; k < launched; ++k)
    if (sizes[k] > 0) {
      nw = static_cast<int>(k) + 1;
      attempted += sizes[k];
    }
  h->n_waves = nw;
  h->timing.n_wave_launches = static_cast<int>(launched);
  h->timing.n_waves = nw;
  h->timing.n_points_attempted = attempted;
  if (prof) {
    double sum = 0.0;
    for (int64_t k = 0; k < launched; ++k)
      sum += elapsed(h->wave_events[2 * k], h->wave_events[2 * k + 1]);
    h->timing.icgn_kernel_ms = sum;
  }
  return DIC_OK;
}

void free_points(dic_handle* h) {
  hfree(h, h->x);
  hfree(h, h->y);
  hfree(h, h->u);
  hfree(h, h->v);
  hfree(h, h->zncc);
  hfree(h, h->accept);
  hfree(h, h->iters);
  hfree(h, h->wave);
  hfree(h, h->conv);
  hfree(h, h->status);
  hfree(h, h->front[0]);
  hfree(h, h->front[1]);
  hfree(h, h->wave_sizes);
  h->pts_cap = 0;
}

// Per-point arrays for the current grid (kept when large enough) and the subset
// centres written on the device.
int size_points(dic_handle* h) {
  const size_t n = static_cast<size_t>(h->npts);
  int rc;
  if (h->npts > h->pts_cap) {
    free_points(h);
    if ((rc = halloc(h, &h->x, n, "points"))) return rc;
    if ((rc = halloc(h, &h->y, n, "points"))) return rc;
    if ((rc = halloc(h, &h->u, n, "points"))) return rc;
    if ((rc = halloc(h, &h->v, n, "points"))) return rc;
    if ((rc = halloc(h, &h->zncc, n, "points"))) return rc;
    if ((rc = halloc(h, &h->accept, n, "points"))) return rc;
    if ((rc = halloc(h, &h->iters, n, "points"))) return rc;
    if ((rc = halloc(h, &h->wave, n, "points"))) return rc;
    if ((rc = halloc(h, &h->conv, n, "points"))) return rc;
    if ((rc = halloc(h, &h->status, n, "points"))) return rc;
    if ((rc = halloc(h, &h->front[0], n + 1, "frontier"))) return rc;
    if ((rc = halloc(h, &h->front[1], n + 1, "frontier"))) return rc;
    if ((rc = halloc(h, &h->wave_sizes, n + 2, "wave sizes"))) return rc;
    h->pts_cap = h->npts;
  }
  const int64_t np = h->npts * h->nparams;
  if (np > h->p_cap) {
    hfree(h, h->p);
    h->p_cap = 0;
    if ((rc = halloc(h, &h->p, static_cast<size_t>(np), "points"))) return rc;
    h->p_cap = np;
  }
  if (!h->counters && (rc = halloc(h, &h->counters, kNumCounters, "counters"))) return rc;
  if (!h->h_counters) {
    void* pinned = nullptr;
    DIC_CUDA(cudaMallocHost(&pinned, sizeof(int32_t) * kNumCounters * kBatchSlots), "pinned counters");
    h->h_counters = static_cast<int32_t*>(pinned);
  }
  DIC_CUDA(launch_grid_points(h->x, h->y, h->r, h->step, h->nx, h->npts, 0), "grid");
  DIC_CUDA(cudaStreamSynchronize(0), "grid");
  return DIC_OK;
}

// Subset geometry checks shared by dic_create and dic_set_subsets.
int check_subsets(int W, int H, const dic_image* roi, int32_t subset_size, int32_t subset_step,
                  int32_t shape_fn) {
  if (subset_size < 3 || subset_size > kMaxSubset || subset_size % 2 == 0)
    return fail(DIC_EINVAL, "subset_size %d must be odd and in [3, %d]", subset_size, kMaxSubset);
  if (subset_size > W || subset_size > H) return fail(DIC_EINVAL, "subset_size %d exceeds the image", subset_size);
  if (subset_step < 1) return fail(DIC_EINVAL, "subset_step %d must be >= 1", subset_step);
  if (shape_fn != DIC_RIGID && shape_fn != DIC_AFFINE && shape_fn != DIC_QUADRATIC)
    return fail(DIC_EINVAL, "unknown shape function %d", shape_fn);
  if (roi) {
    int rc = check_image(roi, "roi");
    if (rc) return rc;
    if (roi->dtype != DIC_U8) return fail(DIC_EINVAL, "roi mask must be DIC_U8");
    if (roi->width != W || roi->height != H) return fail(DIC_EINVAL, "roi mask size differs from the images");
  }
  return DIC_OK;
}

// Grid, per-point arrays and ROI flags for (subset_size, subset_step, shape_fn);
// the images and coefficient planes are kept.
int configure_subsets(dic_handle* h, const dic_image* roi, int32_t subset_size, int32_t subset_step,
                      int32_t shape_fn) {
  h->grid_ok = false;
  h->has_results = false;
  h->n_waves = 0;
  h->n_accepted = 0;
  h->acc_identity = true;
  h->n_updates = 0;
  h->S = subset_size;
  h->r = (subset_size - 1) / 2;
  h->step = subset_step;
  h->shape = shape_fn;
  h->nparams = nparams_of(shape_fn);
  h->nx = (h->W - 1 - 2 * h->r) / h->step + 1;
  h->ny = (h->H - 1 - 2 * h->r) / h->step + 1;
  h->npts = static_cast<int64_t>(h->nx) * h->ny;
  int rc = size_points(h);
  if (rc) return rc;
  hfree(h, h->roi_ok);
  if (roi) {
    GrayPlane mask{};
    void* owned = nullptr;
    int dt = 0;
    if ((rc = halloc(h, &h->roi_ok, static_cast<size_t>(h->npts), "roi flags")) ||
        (rc = bind_image(nullptr, roi, &mask, &owned, &dt))) {
      dev_free(owned);
      return rc;
    }
    RoiArgs ra{mask, h->S, h->r, h->step, h->nx, h->ny, h->roi_ok};
    cudaError_t e = launch_roi_flags(ra, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(0);
    dev_free(owned);
    if (e != cudaSuccess) return cuda_fail(e, "roi flags");
  }
  h->grid_ok = true;
  return DIC_OK;
}

// Device bytes a handle holds after one correlation with these settings: the sum
// of halloc sizes. With cur given, the handle is re-gridded rather than created:
// the reference copy is kept, and every array keeps its capacity unless it is too
// small, the same rules as configure_subsets, replace_image and dic_correlate.
int64_t fft_bytes_for(const dic_handle* cur, int W, int H, int S, int64_t npts, int D);

int64_t footprint(const dic_handle* cur, const dic_image* ref, const dic_image* def, bool roi, int S, int step,
                  int shape, int precision, int n_seeds, int R, int fft_D) {
  const int64_t W = ref->width, H = ref->height;
  const int r = (S - 1) / 2;
  const int64_t n = ((W - 1 - 2 * r) / step + 1) * ((H - 1 - 2 * r) / step + 1);
  const int64_t np = nparams_of(shape);
  const int64_t ldc = (W + 31) & ~static_cast<int64_t>(31);
  const int64_t side = 2 * static_cast<int64_t>(R) + 1;
  const int64_t plane_bytes = 2 * (precision == DIC_FP64 ? 8 : 4) * ldc * H;
  const int64_t per_point = 4 + 4 + 8 + 8 + 4 + 8 + 4 + 4 + 1 + 1;  // x y u v zncc accept iters wave conv status
  auto points_bytes = [&](int64_t m) { return m * per_point + 2 * 4 * (m + 1) + 4 * (m + 2); };
  auto owned_bytes = [&](const dic_handle* h, const void* owned) -> int64_t {
    auto it = h->allocs.find(const_cast<void*>(owned));
    return it == h->allocs.end() ? 0 : static_cast<int64_t>(it->second);
  };
  int64_t b = 4 * kNumCounters + (roi ? n : 0);
  if (!cur) {
    if (!ref->on_device) b += static_cast<int64_t>(owned_pitch(ref)) * H;
    if (!def->on_device) b += static_cast<int64_t>(owned_pitch(def)) * H;
    b += plane_bytes + points_bytes(n) + 8 * n * np;
    b += static_cast<int64_t>(n_seeds) * (8 + 4 + 4) + (fft_D < 0 ? 8 * n_seeds * side * side : 0);
    if (fft_D >= 0) b += fft_bytes_for(nullptr, static_cast<int>(W), static_cast<int>(H), S, n, fft_D);
    return b;
  }
  b += cur->ref_owned ? owned_bytes(cur, cur->ref_owned) : 0;
  if (!def->on_device)
    b += (cur->def_owned && dtype_size(def->dtype) == dtype_size(cur->def_dtype))
             ? owned_bytes(cur, cur->def_owned)
             : static_cast<int64_t>(owned_pitch(def)) * H;
  b += cur->plane_prec == plane_kind(precision) ? owned_bytes(cur, cur->c_ref) + owned_bytes(cur, cur->c_def) : plane_bytes;
  b += points_bytes(n > cur->pts_cap ? n : cur->pts_cap);
  b += 8 * (n * np > cur->p_cap ? n * np : cur->p_cap);
  const int64_t sc = static_cast<int64_t>(n_seeds) > static_cast<int64_t>(cur->seed_cap)
                         ? n_seeds : static_cast<int64_t>(cur->seed_cap);
  const int64_t want_scores = fft_D < 0 ? n_seeds * side * side : 0;
  const int64_t scores = want_scores > static_cast<int64_t>(cur->score_cap) ? want_scores
                                                                           : static_cast<int64_t>(cur->score_cap);
  b += sc * (8 + 4 + 4) + 8 * scores;
  if (fft_D >= 0)
    b += fft_bytes_for(cur, static_cast<int>(W), static_cast<int>(H), S, n, fft_D);
  else if (cur->fft_tw)
    b += fft_bytes_for(cur, static_cast<int>(W), static_cast<int>(H), S, 0, -1);
  if (cur->inc_cap > 0) b += cur->inc_cap * (8 + 8 + 32 + 1 + 8 + 8 + 1) + 8 * cur->tot_p_cap;  // kept until used
  return b;
}

int validate_params(const dic_params* p) {
  if (!p) return fail(DIC_EINVAL, "params is NULL");
  if (p->max_iter < 1 || p->max_iter > 100000) return fail(DIC_EINVAL, "max_iter %d out of range", p->max_iter);
  if (!(p->conv_threshold > 0.0)) return fail(DIC_EINVAL, "conv_threshold must be > 0");
  if (!(p->zncc_min >= -1.0 && p->zncc_min <= 1.0)) return fail(DIC_EINVAL, "zncc_min must be in [-1, 1]");
  if (p->search_radius < 0 || p->search_radius > 256)
    return fail(DIC_EINVAL, "search_radius %d out of range", p->search_radius);
  if (p->precision != DIC_FP64 && p->precision != DIC_MIXED && p->precision != DIC_MIXED_FP64_SOLVE)
    return fail(DIC_EINVAL, "unknown precision %d", p->precision);
  if (p->precision == DIC_MIXED_FP64_SOLVE && (p->cost != DIC_COST_ZNSSD || p->optimizer != DIC_OPT_GAUSS_NEWTON))
    return fail(DIC_EINVAL, "DIC_MIXED_FP64_SOLVE runs Gauss-Newton with ZNSSD only");
  if (p->cost != DIC_COST_ZNSSD && p->cost != DIC_COST_NSSD && p->cost != DIC_COST_SSD)
    return fail(DIC_EINVAL, "unknown cost %d", p->cost);
  if (p->optimizer != DIC_OPT_GAUSS_NEWTON && p->optimizer != DIC_OPT_LEVENBERG_MARQUARDT)
    return fail(DIC_EINVAL, "unknown optimizer %d", p->optimizer);
  if (p->init != DIC_INIT_SEARCH && p->init != DIC_INIT_FFT) return fail(DIC_EINVAL, "unknown init %d", p->init);
  if (p->max_displacement < 0 || p->max_displacement >= kFftLargeMax)
    return fail(DIC_EINVAL, "max_displacement %d outside [0, %d]", p->max_displacement, kFftLargeMax - 1);
  if (!(p->mad_eps >= 0.0) || p->mad_tau != p->mad_tau) return fail(DIC_EINVAL, "mad_tau/mad_eps invalid");
  return DIC_OK;
}

int check_estimate_args(const dic_image* ref, const dic_image* def, int32_t subset_size, int32_t subset_step,
                        int32_t shape_fn, const dic_params* params, int32_t n_seeds) {
  if (!ref || !def || !params) return fail(DIC_EINVAL, "NULL argument");
  if (dtype_size(ref->dtype) == 0 || dtype_size(def->dtype) == 0) return fail(DIC_EINVAL, "unknown image dtype");
  if (ref->width != def->width || ref->height != def->height)
    return fail(DIC_EINVAL, "reference %dx%d and deformed %dx%d differ in size", ref->width, ref->height,
                def->width, def->height);
  if (ref->width < 8 || ref->height < 8) return fail(DIC_EINVAL, "images must be at least 8x8");
  int rc = check_subsets(ref->width, ref->height, nullptr, subset_size, subset_step, shape_fn);
  if (rc) return rc;
  if ((rc = validate_params(params))) return rc;
  if (n_seeds < 1) return fail(DIC_EINVAL, "at least one seed is needed");
  return DIC_OK;
}

void release(dic_handle* h) {
  if (!h) return;
  for (auto& kv : h->allocs) dev_free(kv.first);
  h->allocs.clear();
  if (h->h_counters) cudaFreeHost(h->h_counters);
  if (h->h_res) cudaFreeHost(h->h_res);
  for (cudaEvent_t e : h->events) cudaEventDestroy(e);
  for (cudaEvent_t e : h->wave_events) cudaEventDestroy(e);
  for (cudaEvent_t e : h->batch_ev)
    if (e) cudaEventDestroy(e);
  delete h;
}


// The wave loop and everything after it, shared by dic_correlate and
// dic_correlate_sequence (wave 0 is already in front[0] and the counters).
int finish_run(dic_handle* h, cudaStream_t s) {
  const bool prof = h->prm.profile != 0;
  const bool fp64 = h->prm.precision == DIC_FP64;
  cudaEvent_t w0 = event_at(h, 5), w1 = event_at(h, 6);
  if (!w0 || !w1) return fail(DIC_ECUDA, "event creation failed");
  if (prof) cudaEventRecord(w0, s);
  int rc = fp64 ? run_waves<double>(h, s) : run_waves<float>(h, s);
  if (rc) return rc;
  if (prof) cudaEventRecord(w1, s);
  PointArrays pa = point_arrays(h);
  DIC_CUDA(cudaMemsetAsync(h->counters + kAccepted, 0, sizeof(int32_t), s), "counter reset");
  DIC_CUDA(launch_finalize_points(pa, h->nparams, h->prm.nan_unconverged, h->counters + kAccepted, s),
           "finalize");
  if (prof) cudaEventRecord(h->events[4], s);
  DIC_CUDA(cudaMemcpyAsync(h->h_counters, h->counters, sizeof(int32_t) * kNumCounters,
                           cudaMemcpyDeviceToHost, s), "counter read-back");
  DIC_CUDA(cudaStreamSynchronize(s), "correlate");
  const int64_t accepted = h->h_counters[kAccepted];
  h->n_accepted = accepted;
  h->has_results = true;
  if (h->h_counters[kError]) return fail(DIC_ETIMEOUT, "a tile load did not complete in time");
  if (prof) {
    h->timing.prefilter_ms = elapsed(h->events[0], h->events[1]);
    h->timing.setup_ms = elapsed(h->events[1], h->events[3]);
    h->timing.seed_kernel_ms = elapsed(h->events[2], h->events[3]);
    h->timing.waves_ms = elapsed(w0, w1);
  }
  if (accepted == 0) return fail(DIC_ENOSEED, "no point was accepted");
  return DIC_OK;
}

}  // namespace

namespace {

// Window sizes of the initialiser: the powers of two above D, largest first, that
// exceed the subset size and fit in the image, then the subset size.
std::vector<int> fft_sizes(int D, int S, int W, int H) {
  int L = 1;
  while (L <= D) L *= 2;
  std::vector<int> out;
  for (; L > S; L /= 2)
    if (L <= W && L <= H) out.push_back(L);
  out.push_back(S);
  return out;
}

struct FftCaps {
  int64_t win = 0, mid = 0, large = 0, work = 0, res = 0;
};

FftCaps fft_caps(int W, int H, int S, int64_t npts, int D) {
  FftCaps c;
  const std::vector<int> sizes = fft_sizes(D, S, W, H);
  for (size_t i = 0; i + 1 < sizes.size(); ++i) {
    const int64_t L = sizes[i];
    const int64_t n = (W / L) * (H / L);
    c.mid = n > c.mid ? n : c.mid;
    if (L > kFftSmallMax) {
      c.large = n > c.large ? n : c.large;
      c.work = n * L * L > c.work ? n * L * L : c.work;
    }
  }
  c.res = npts;
  c.win = c.mid > npts ? c.mid : npts;
  return c;
}

constexpr int64_t kFftTwiddleEntries = kFftTwiddlesPow2 + kFftSmallMax;

// Device bytes of the initialiser's arrays once a run with caps has grown them
// from cur's capacities (cur NULL: a fresh handle).
int64_t fft_bytes(const FftCaps& c, const dic_handle* cur) {
  auto mx = [](int64_t a, int64_t b) { return a > b ? a : b; };
  const int64_t win = mx(c.win, cur ? cur->fft_win_cap : 0), mid = mx(c.mid, cur ? cur->fft_mid_cap : 0);
  const int64_t large = mx(c.large, cur ? cur->fft_large_cap : 0), work = mx(c.work, cur ? cur->fft_work_cap : 0);
  const int64_t res = mx(c.res, cur ? cur->fft_res_cap : 0);
  int64_t b = 8 * kFftTwiddleEntries + 16 * win + 12 * win + 16 * mid + 14 * res;
  if (large > 0) b += 8 * work + 16 * large + 8 * large + 8 * large;
  return b;
}

int64_t fft_bytes_for(const dic_handle* cur, int W, int H, int S, int64_t npts, int D) {
  return fft_bytes(D >= 0 ? fft_caps(W, H, S, npts, D) : FftCaps{}, cur);
}

template <typename P>
int regrow(dic_handle* h, P** ptr, int64_t need, const char* what) {
  hfree(h, *ptr);
  return halloc(h, ptr, static_cast<size_t>(need), what);
}

int fft_prepare(dic_handle* h, const FftCaps& c) {
  int rc;
  if (!h->fft_tw && (rc = halloc(h, &h->fft_tw, static_cast<size_t>(kFftTwiddleEntries), "fft twiddles"))) return rc;
  if (c.win > h->fft_win_cap) {
    h->fft_win_cap = 0;
    if ((rc = regrow(h, &h->fft_org, c.win, "fft origins"))) return rc;
    for (int i = 0; i < 3; ++i)
      if ((rc = regrow(h, &h->fft_raw[i], c.win, "fft level"))) return rc;
    h->fft_win_cap = c.win;
  }
  if (c.mid > h->fft_mid_cap) {
    h->fft_mid_cap = 0;
    for (int i = 0; i < 4; ++i)
      if ((rc = regrow(h, &h->fft_filt[i], c.mid, "fft level"))) return rc;
    h->fft_mid_cap = c.mid;
  }
  if (c.large > h->fft_large_cap) {
    h->fft_large_cap = 0;
    if ((rc = regrow(h, &h->fft_norms, 2 * c.large, "fft norms")) ||
        (rc = regrow(h, &h->fft_keys, c.large, "fft peaks")) ||
        (rc = regrow(h, &h->fft_nonflat, 2 * c.large, "fft flags")))
      return rc;
    h->fft_large_cap = c.large;
  }
  if (c.work > h->fft_work_cap) {
    h->fft_work_cap = 0;
    if ((rc = regrow(h, &h->fft_work, c.work, "fft work"))) return rc;
    h->fft_work_cap = c.work;
  }
  if (c.res > h->fft_res_cap) {
    h->fft_res_cap = 0;
    for (int i = 0; i < 3; ++i)
      if ((rc = regrow(h, &h->fft_res[i], c.res, "fft results"))) return rc;
    if ((rc = regrow(h, &h->fft_status, c.res, "fft results")) ||
        (rc = regrow(h, &h->fft_rep, c.res, "fft results")))
      return rc;
    h->fft_res_cap = c.res;
  }
  return DIC_OK;
}

FftccArgs fftcc_args(dic_handle* h, int L, int64_t n, int subpixel, float* u, float* v, float* peak) {
  FftccArgs a{};
  a.ref = h->ref;
  a.def = h->def;
  a.W = h->W;
  a.H = h->H;
  a.L = L;
  a.n = n;
  a.org = h->fft_org;
  a.tw_pow2 = h->fft_tw;
  a.tw_odd = h->fft_tw + kFftTwiddlesPow2;
  a.subpixel = subpixel;
  a.u = u;
  a.v = v;
  a.peak = peak;
  a.work = h->fft_work;
  a.norms = h->fft_norms;
  a.keys = h->fft_keys;
  a.nonflat = h->fft_nonflat;
  return a;
}

int fft_twiddles(dic_handle* h, int L_odd, cudaStream_t s) {
  if (h->fft_tw_odd == L_odd) return DIC_OK;
  DIC_CUDA(launch_twiddles(h->fft_tw, L_odd, s), "fft twiddles");
  h->fft_tw_odd = L_odd;
  return DIC_OK;
}

// The whole initialiser over the handle's grid: every level's origins, Eq. 1 and
// the MAD rule; the last level's values land in fft_res, fft_rep and fft_status.
int run_fft(dic_handle* h, int D, int subpixel, double tau, double eps, cudaStream_t s) {
  const std::vector<int> sizes = fft_sizes(D, h->S, h->W, h->H);
  if (static_cast<int>(sizes.size()) > kFftMaxLevels) return fail(DIC_EINVAL, "too many window levels");
  int rc = fft_prepare(h, fft_caps(h->W, h->H, h->S, h->npts, D));
  if (rc) return rc;
  if ((rc = fft_twiddles(h, h->S, s))) return rc;
  const float* pu = nullptr;
  const float* pv = nullptr;
  int pnx = 0, pny = 0, ping = 0;
  double pc0 = 0.0, pstep = 1.0;
  h->has_fft = false;
  for (size_t li = 0; li < sizes.size(); ++li) {
    const int L = sizes[li];
    const bool last = li + 1 == sizes.size();
    const int nx = last ? h->nx : h->W / L, ny = last ? h->ny : h->H / L;
    const int64_t n = static_cast<int64_t>(nx) * ny;
    FftLevelArgs la{};
    la.W = h->W;
    la.H = h->H;
    la.L = L;
    la.nx = nx;
    la.ny = ny;
    la.grid = last ? 1 : 0;
    la.r = h->r;
    la.step = h->step;
    la.roi_ok = last ? h->roi_ok : nullptr;
    la.pu = pu;
    la.pv = pv;
    la.pnx = pnx;
    la.pny = pny;
    la.pc0 = pc0;
    la.pstep = pstep;
    la.org = h->fft_org;
    DIC_CUDA(launch_fftcc_origins(la, s), "fft origins");
    float* peak_out = last ? h->fft_res[2] : h->fft_raw[2];
    DIC_CUDA(launch_fftcc(fftcc_args(h, L, n, last ? subpixel : 0, h->fft_raw[0], h->fft_raw[1], peak_out), s),
             "fft cross-correlation");
    MadArgs ma{};
    ma.u = h->fft_raw[0];
    ma.v = h->fft_raw[1];
    ma.valid = last ? h->roi_ok : nullptr;
    ma.nx = nx;
    ma.ny = ny;
    ma.tau = tau;
    ma.eps = eps;
    ma.u_out = last ? h->fft_res[0] : h->fft_filt[2 * ping];
    ma.v_out = last ? h->fft_res[1] : h->fft_filt[2 * ping + 1];
    ma.replaced = last ? h->fft_rep : nullptr;
    DIC_CUDA(launch_mad(ma, s), "fft outlier removal");
    pu = ma.u_out;
    pv = ma.v_out;
    pnx = nx;
    pny = ny;
    pc0 = L / 2;
    pstep = L;
    ping ^= 1;
  }
  DIC_CUDA(launch_fft_status(h->roi_ok, h->fft_status, h->npts, s), "fft status");
  h->fft_levels = static_cast<int>(sizes.size());
  for (size_t i = 0; i < sizes.size(); ++i) h->fft_window[i] = sizes[i];
  h->has_fft = true;
  return DIC_OK;
}

int ensure_increments(dic_handle* h) {
  const int64_t n = h->npts, np = h->npts * h->nparams;
  if (h->inc_cap >= n && h->tot_p_cap >= np) return DIC_OK;
  int rc;
  h->inc_cap = 0;
  h->tot_p_cap = 0;
  if ((rc = regrow(h, &h->acc_u, n, "accumulated warps")) || (rc = regrow(h, &h->acc_v, n, "accumulated warps")) ||
      (rc = regrow(h, &h->acc_A, 4 * n, "accumulated warps")) ||
      (rc = regrow(h, &h->acc_ok, n, "accumulated warps")) || (rc = regrow(h, &h->tot_u, n, "total warps")) ||
      (rc = regrow(h, &h->tot_v, n, "total warps")) || (rc = regrow(h, &h->tot_p, np, "total warps")) ||
      (rc = regrow(h, &h->tot_status, n, "total warps")))
    return rc;
  h->inc_cap = n;
  h->tot_p_cap = np;
  return DIC_OK;
}

int run_totals(dic_handle* h, int update, cudaStream_t s) {
  TotalArgs a{};
  a.nx = h->nx;
  a.ny = h->ny;
  a.r = h->r;
  a.step = h->step;
  a.nparams = h->nparams;
  a.roi_ok = h->roi_ok;
  a.status = h->status;
  a.p = h->p;
  a.identity = h->acc_identity ? 1 : 0;
  a.acc_u = h->acc_u;
  a.acc_v = h->acc_v;
  a.acc_A = h->acc_A;
  a.acc_ok = h->acc_ok;
  a.tot_u = h->tot_u;
  a.tot_v = h->tot_v;
  a.tot_p = h->tot_p;
  a.tot_status = h->tot_status;
  a.update = update;
  DIC_CUDA(launch_totals(a, s), "total warps");
  return DIC_OK;
}

}  // namespace

extern "C" {

dic_params dic_default_params(void) {
  dic_params p{};
  p.max_iter = 40;
  p.search_radius = 8;
  p.conv_threshold = 0.01;
  p.zncc_min = 0.70;
  p.precision = DIC_MIXED;
  p.nan_unconverged = 0;
  p.profile = 0;
  p.cost = DIC_COST_ZNSSD;
  p.optimizer = DIC_OPT_GAUSS_NEWTON;
  p.init = DIC_INIT_SEARCH;
  p.max_displacement = 32;
  p.reserved = 0;
  p.mad_tau = 3.0;
  p.mad_eps = 0.5;
  return p;
}

dic_fft_params dic_fft_default_params(void) {
  dic_fft_params f{};
  f.max_displacement = 32;
  f.subpixel = 1;
  f.mad_tau = 3.0;
  f.mad_eps = 0.5;
  return f;
}

const char* dic_last_error(void) { return g_last_error.c_str(); }

int dic_test_expire_tile_waits(int32_t on) {
  g_expire_waits.store(on != 0 ? 1 : 0);
  return DIC_OK;
}

int dic_create(const dic_image* ref, const dic_image* def, const dic_image* roi, int32_t subset_size,
               int32_t subset_step, int32_t shape_fn, int32_t interp, dic_handle** out) {
  g_last_error.clear();
  if (!out) return fail(DIC_EINVAL, "out is NULL");
  *out = nullptr;
  int rc;
  if ((rc = check_image(ref, "reference"))) return rc;
  if ((rc = check_image(def, "deformed"))) return rc;
  if (ref->width != def->width || ref->height != def->height)
    return fail(DIC_EINVAL, "reference %dx%d and deformed %dx%d differ in size", ref->width, ref->height,
                def->width, def->height);
  if ((rc = check_subsets(ref->width, ref->height, roi, subset_size, subset_step, shape_fn))) return rc;
  if (interp != DIC_BSPLINE3 && interp != DIC_BICUBIC) return fail(DIC_EINVAL, "unknown interpolation %d", interp);
  dic_handle* h = new (std::nothrow) dic_handle();
  if (!h) return fail(DIC_ENOMEM, "handle allocation");
  cudaGetDevice(&h->device);
  h->W = ref->width;
  h->H = ref->height;
  h->prm = dic_default_params();
  h->interp = interp;
  if ((rc = bind_image(h, ref, &h->ref, &h->ref_owned, &h->ref_dtype)) ||
      (rc = bind_image(h, def, &h->def, &h->def_owned, &h->def_dtype)) ||
      (rc = configure_subsets(h, roi, subset_size, subset_step, shape_fn))) {
    release(h);
    return rc;
  }
  *out = h;
  return DIC_OK;
}

int dic_set_subsets(dic_handle* h, const dic_image* roi, int32_t subset_size, int32_t subset_step,
                    int32_t shape_fn) {
  if (!h) return fail(DIC_EINVAL, "handle is NULL");
  g_last_error.clear();
  int rc = check_subsets(h->W, h->H, roi, subset_size, subset_step, shape_fn);
  if (rc) return rc;
  return configure_subsets(h, roi, subset_size, subset_step, shape_fn);
}

int dic_estimate_device_bytes(const dic_image* ref, const dic_image* def, int32_t has_roi, int32_t subset_size,
                              int32_t subset_step, int32_t shape_fn, const dic_params* params, int32_t n_seeds,
                              int64_t* bytes) {
  g_last_error.clear();
  if (!bytes) return fail(DIC_EINVAL, "NULL argument");
  int rc = check_estimate_args(ref, def, subset_size, subset_step, shape_fn, params, n_seeds);
  if (rc) return rc;
  *bytes = footprint(nullptr, ref, def, has_roi != 0, subset_size, subset_step, shape_fn, params->precision,
                     n_seeds, params->search_radius, params->init == DIC_INIT_FFT ? params->max_displacement : -1);
  return DIC_OK;
}

int dic_estimate_regrid_bytes(const dic_handle* h, const dic_image* def, int32_t has_roi, int32_t subset_size,
                              int32_t subset_step, int32_t shape_fn, const dic_params* params, int32_t n_seeds,
                              int64_t* bytes) {
  g_last_error.clear();
  if (!h || !bytes) return fail(DIC_EINVAL, "NULL argument");
  dic_image ref{};
  ref.width = h->W;
  ref.height = h->H;
  ref.dtype = h->ref_dtype;
  ref.on_device = h->ref_owned ? 0 : 1;
  int rc = check_estimate_args(&ref, def, subset_size, subset_step, shape_fn, params, n_seeds);
  if (rc) return rc;
  *bytes = footprint(h, &ref, def, has_roi != 0, subset_size, subset_step, shape_fn, params->precision, n_seeds,
                     params->search_radius, params->init == DIC_INIT_FFT ? params->max_displacement : -1);
  return DIC_OK;
}

int dic_get_device_bytes(const dic_handle* h, int64_t* bytes) {
  if (!h || !bytes) return fail(DIC_EINVAL, "NULL argument");
  *bytes = h->device_bytes;
  return DIC_OK;
}

int dic_set_params(dic_handle* h, const dic_params* params) {
  if (!h) return fail(DIC_EINVAL, "handle is NULL");
  int rc = validate_params(params);
  if (rc) return rc;
  h->prm = *params;
  return DIC_OK;
}

int dic_get_params(const dic_handle* h, dic_params* out) {
  if (!h || !out) return fail(DIC_EINVAL, "NULL argument");
  *out = h->prm;
  return DIC_OK;
}

static int replace_image(dic_handle* h, const dic_image* im, bool is_ref) {
  if (!h) return fail(DIC_EINVAL, "handle is NULL");
  int rc = check_image(im, is_ref ? "reference" : "deformed");
  if (rc) return rc;
  if (im->width != h->W || im->height != h->H)
    return fail(DIC_EINVAL, "image is %dx%d, the handle holds %dx%d", im->width, im->height, h->W, h->H);
  const int old_dtype = is_ref ? h->ref_dtype : h->def_dtype;
  void** owned = is_ref ? &h->ref_owned : &h->def_owned;
  // an owned copy that no longer fits (or is no longer used) is released
  if (*owned && (im->on_device || dtype_size(im->dtype) != dtype_size(old_dtype))) hfree(h, *owned);
  if (is_ref) {
    rc = bind_image(h, im, &h->ref, owned, &h->ref_dtype);
    h->ref_dirty = true;
  } else {
    rc = bind_image(h, im, &h->def, owned, &h->def_dtype);
    h->def_dirty = true;
  }
  return rc;
}

int dic_set_reference(dic_handle* h, const dic_image* ref) {
  const int rc = replace_image(h, ref, true);
  if (rc == DIC_OK) {                // a new first reference: no accumulated warps
    h->acc_identity = true;
    h->n_updates = 0;
  }
  return rc;
}
int dic_set_deformed(dic_handle* h, const dic_image* def) { return replace_image(h, def, false); }

int dic_correlate(dic_handle* h, const int32_t* seeds_xy, int32_t n_seeds, void* cuda_stream) {
  if (!h) return fail(DIC_EINVAL, "handle is NULL");
  g_last_error.clear();
  if (!seeds_xy || n_seeds < 1) return fail(DIC_EINVAL, "at least one seed is needed");
  if (!h->grid_ok) return fail(DIC_ESTATE, "the handle has no subset grid; call dic_set_subsets");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  h->last_stream = s;
  int rc = ensure_planes(h);
  if (rc) return rc;
  h->timing = dic_timing{};
  const bool prof = h->prm.profile != 0;
  const bool fp64 = h->prm.precision == DIC_FP64;
  // events: 0 start, 1 after prefilter, 2 after setup, 3 after seed scores, 4 end
  for (int i = 0; i < 5; ++i)
    if (!event_at(h, i)) return fail(DIC_ECUDA, "event creation failed");
  if (prof) cudaEventRecord(h->events[0], s);

  if (h->ref_dirty) {
    rc = fp64 ? prefilter<double>(h, h->ref, h->c_ref, s) : prefilter<float>(h, h->ref, h->c_ref, s);
    if (rc) return rc;
    h->ref_dirty = false;
  }
  if (h->def_dirty) {
    rc = fp64 ? prefilter<double>(h, h->def, h->c_def, s) : prefilter<float>(h, h->def, h->c_def, s);
    if (rc) return rc;
    h->def_dirty = false;
  }
  if (prof) cudaEventRecord(h->events[1], s);

  // seeds: snap to the nearest grid point (ties to the lower index)
  std::vector<int32_t> centres(2 * static_cast<size_t>(n_seeds)), qs(static_cast<size_t>(n_seeds));
  for (int i = 0; i < n_seeds; ++i) {
    int64_t gi = floor_div(2 * (static_cast<int64_t>(seeds_xy[2 * i]) - h->r) + h->step - 1, 2 * h->step);
    int64_t gj = floor_div(2 * (static_cast<int64_t>(seeds_xy[2 * i + 1]) - h->r) + h->step - 1, 2 * h->step);
    gi = gi < 0 ? 0 : (gi > h->nx - 1 ? h->nx - 1 : gi);
    gj = gj < 0 ? 0 : (gj > h->ny - 1 ? h->ny - 1 : gj);
    qs[i] = static_cast<int32_t>(gj * h->nx + gi);
    centres[2 * i] = h->r + static_cast<int32_t>(gi) * h->step;
    centres[2 * i + 1] = h->r + static_cast<int32_t>(gj) * h->step;
  }
  const int R = h->prm.search_radius;
  const size_t side = 2 * static_cast<size_t>(R) + 1;
  if (static_cast<size_t>(n_seeds) > h->seed_cap) {
    hfree(h, h->seed_xy);
    hfree(h, h->seed_q);
    hfree(h, h->seed_best);
    h->seed_cap = 0;
    if ((rc = halloc(h, &h->seed_xy, 2 * static_cast<size_t>(n_seeds), "seeds")) ||
        (rc = halloc(h, &h->seed_q, static_cast<size_t>(n_seeds), "seeds")) ||
        (rc = halloc(h, &h->seed_best, static_cast<size_t>(n_seeds), "seeds")))
      return rc;
    h->seed_cap = n_seeds;
  }
  const bool fft_init = h->prm.init == DIC_INIT_FFT;
  h->acc_identity = true;            // correlating from seeds: the reference is the first one
  h->n_updates = 0;
  if (!fft_init && n_seeds * side * side > h->score_cap) {
    hfree(h, h->seed_scores);
    h->score_cap = 0;
    if ((rc = halloc(h, &h->seed_scores, n_seeds * side * side, "seed scores"))) return rc;
    h->score_cap = n_seeds * side * side;
  }
  DIC_CUDA(cudaMemcpyAsync(h->seed_xy, centres.data(), centres.size() * sizeof(int32_t),
                           cudaMemcpyHostToDevice, s), "seed upload");
  DIC_CUDA(cudaMemcpyAsync(h->seed_q, qs.data(), qs.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s),
           "seed upload");
  PointArrays pa = point_arrays(h);
  DIC_CUDA(launch_reset_points(pa, h->nparams, h->roi_ok, s), "point reset");
  DIC_CUDA(cudaMemsetAsync(h->counters, 0, sizeof(int32_t) * kNumCounters, s), "counter reset");
  if (prof) cudaEventRecord(h->events[2], s);
  SeedCommitArgs ca{n_seeds, R, h->nparams, h->seed_q, h->seed_scores, h->seed_best, h->p, h->status,
                    h->wave, h->front[0], h->counters, h->roi_ok, nullptr, nullptr};
  if (fft_init) {
    // the seeds start from the multi-window FFT estimate (no sub-pixel fit)
    if ((rc = run_fft(h, h->prm.max_displacement, 0, h->prm.mad_tau, h->prm.mad_eps, s))) return rc;
    ca.fft_u = h->fft_res[0];
    ca.fft_v = h->fft_res[1];
  } else {
    SeedArgs sa{h->ref, h->def, h->W, h->H, h->S, R, n_seeds, h->seed_xy, h->seed_scores};
    DIC_CUDA(launch_seed_scores(sa, s), "seed search");
  }
  if (prof) cudaEventRecord(h->events[3], s);
  DIC_CUDA(launch_seed_commit(ca, s), "seed commit");

  return finish_run(h, s);
}

int dic_correlate_sequence(dic_handle* h, void* cuda_stream) {
  if (!h) return fail(DIC_EINVAL, "handle is NULL");
  g_last_error.clear();
  if (!h->has_results) return fail(DIC_ESTATE, "dic_correlate_sequence needs an earlier correlation");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  h->last_stream = s;
  if (h->plane_prec != plane_kind(h->prm.precision))
    return fail(DIC_ESTATE, "the precision changed since the last correlation; correlate with seeds");
  h->timing = dic_timing{};
  const bool prof = h->prm.profile != 0;
  const bool fp64 = h->prm.precision == DIC_FP64;
  for (int i = 0; i < 5; ++i)
    if (!event_at(h, i)) return fail(DIC_ECUDA, "event creation failed");
  if (prof) cudaEventRecord(h->events[0], s);
  int rc = DIC_OK;
  if (h->ref_dirty) {
    rc = fp64 ? prefilter<double>(h, h->ref, h->c_ref, s) : prefilter<float>(h, h->ref, h->c_ref, s);
    if (rc) return rc;
    h->ref_dirty = false;
  }
  if (h->def_dirty) {
    rc = fp64 ? prefilter<double>(h, h->def, h->c_def, s) : prefilter<float>(h, h->def, h->c_def, s);
    if (rc) return rc;
    h->def_dirty = false;
  }
  if (prof) cudaEventRecord(h->events[1], s);
  PointArrays pa = point_arrays(h);
  DIC_CUDA(cudaMemsetAsync(h->counters, 0, sizeof(int32_t) * kNumCounters, s), "counter reset");
  if (prof) cudaEventRecord(h->events[2], s);
  DIC_CUDA(launch_sequence_reset(pa, h->nparams, h->roi_ok, h->front[0], h->counters, s), "sequence reset");
  if (prof) cudaEventRecord(h->events[3], s);
  return finish_run(h, s);
}

int dic_get_results(dic_handle* h, dic_results* out, int32_t on_device) {
  if (!h || !out) return fail(DIC_EINVAL, "NULL argument");
  if (!h->has_results) return fail(DIC_ESTATE, "no correlation since the handle was created or re-gridded");
  const size_t n = static_cast<size_t>(h->npts);
  out->n_points = h->npts;
  out->nx = h->nx;
  out->ny = h->ny;
  out->n_params = h->nparams;
  out->n_waves = h->n_waves;
  out->n_accepted = h->n_accepted;
  if (on_device) {
    out->x = h->x;
    out->y = h->y;
    out->u = h->u;
    out->v = h->v;
    out->p = h->p;
    out->zncc = h->zncc;
    out->iters = h->iters;
    out->converged = h->conv;
    out->status = h->status;
    out->wave = h->wave;
    return DIC_OK;
  }
  const size_t bytes = n * (4 + 4 + 8 + 8 + 8 * h->nparams + 4 + 4 + 1 + 1 + 4) + 256;
  if (h->h_res_bytes < bytes) {
    if (h->h_res) cudaFreeHost(h->h_res);
    h->h_res = nullptr;
    h->h_res_bytes = 0;
    DIC_CUDA(cudaMallocHost(&h->h_res, bytes), "pinned result buffer");
    h->h_res_bytes = bytes;
  }
  char* base = static_cast<char*>(h->h_res);
  size_t off = 0;
  auto take = [&](const void* src, size_t len) -> void* {
    void* dst = base + off;
    off += (len + 15) & ~static_cast<size_t>(15);
    cudaMemcpyAsync(dst, src, len, cudaMemcpyDeviceToHost, h->last_stream);
    return dst;
  };
  out->p = static_cast<const double*>(take(h->p, n * 8 * h->nparams));
  out->u = static_cast<const double*>(take(h->u, n * 8));
  out->v = static_cast<const double*>(take(h->v, n * 8));
  out->x = static_cast<const int32_t*>(take(h->x, n * 4));
  out->y = static_cast<const int32_t*>(take(h->y, n * 4));
  out->zncc = static_cast<const float*>(take(h->zncc, n * 4));
  out->iters = static_cast<const int32_t*>(take(h->iters, n * 4));
  out->wave = static_cast<const int32_t*>(take(h->wave, n * 4));
  out->converged = static_cast<const uint8_t*>(take(h->conv, n));
  out->status = static_cast<const uint8_t*>(take(h->status, n));
  DIC_CUDA(cudaStreamSynchronize(h->last_stream), "result read-back");
  return DIC_OK;
}

int dic_get_coefficients(const dic_handle* h, int32_t which, const void** plane, int64_t* ld,
                         int32_t* elem_bytes) {
  if (!h || !plane || !ld || !elem_bytes) return fail(DIC_EINVAL, "NULL argument");
  if (which != 0 && which != 1) return fail(DIC_EINVAL, "which must be 0 or 1");
  if (h->plane_prec < 0 || (which == 0 ? h->ref_dirty : h->def_dirty))
    return fail(DIC_ESTATE, "coefficients are computed by dic_correlate");
  *plane = which == 0 ? h->c_ref : h->c_def;
  *ld = h->ldc;
  *elem_bytes = h->plane_prec == DIC_FP64 ? 8 : 4;
  return DIC_OK;
}

int dic_get_timing(const dic_handle* h, dic_timing* out) {
  if (!h || !out) return fail(DIC_EINVAL, "NULL argument");
  *out = h->timing;
  return DIC_OK;
}

int dic_strain_field(const double* u, const double* v, const uint8_t* status, int32_t nx, int32_t ny,
                     int32_t subset_step, int32_t window, int32_t basis, int32_t measure,
                     const dic_strain_outputs* out, void* cuda_stream) {
  g_last_error.clear();
  if (!u || !v || !status || !out) return fail(DIC_EINVAL, "NULL argument");
  if (!out->dudx || !out->dudy || !out->dvdx || !out->dvdy || !out->exx || !out->eyy || !out->exy || !out->valid)
    return fail(DIC_EINVAL, "an output array is NULL");
  if (nx < 1 || ny < 1) return fail(DIC_EINVAL, "grid %dx%d is empty", nx, ny);
  if (subset_step < 1) return fail(DIC_EINVAL, "subset_step %d must be >= 1", subset_step);
  if (window < 3 || window > 31 || window % 2 == 0)
    return fail(DIC_EINVAL, "window %d must be odd and in [3, 31]", window);
  if (basis != DIC_STRAIN_BILINEAR && basis != DIC_STRAIN_BIQUADRATIC)
    return fail(DIC_EINVAL, "unknown strain basis %d", basis);
  if (measure < DIC_GREEN_LAGRANGE || measure > DIC_BIOT_LEFT)
    return fail(DIC_EINVAL, "unknown strain measure %d", measure);
  StrainArgs a{};
  a.u = u;
  a.v = v;
  a.status = status;
  a.nx = nx;
  a.ny = ny;
  a.step = subset_step;
  a.window = window;
  a.basis = basis;
  a.measure = measure;
  // full-window slope weights: the odd-in-x terms {x} (bilinear) or {x, x y^2}
  // (biquadratic) are orthogonal to the rest on the symmetric window
  const int h = (window - 1) / 2;
  double s2 = 0.0, s4 = 0.0;
  for (int i = -h; i <= h; ++i) {
    s2 += static_cast<double>(i) * i;
    s4 += static_cast<double>(i) * i * i * i;
  }
  const double n = window;
  if (basis == DIC_STRAIN_BILINEAR) {
    a.wa = static_cast<float>(1.0 / (n * s2));
    a.wb = 0.0f;
  } else {
    const double den = n * s4 - s2 * s2;
    a.wa = static_cast<float>(s4 / (s2 * den));
    a.wb = static_cast<float>(-1.0 / den);
  }
  a.dudx = out->dudx;
  a.dudy = out->dudy;
  a.dvdx = out->dvdx;
  a.dvdy = out->dvdy;
  a.exx = out->exx;
  a.eyy = out->eyy;
  a.exy = out->exy;
  a.valid = out->valid;
  DIC_CUDA(launch_strain(a, static_cast<cudaStream_t>(cuda_stream)), "strain launch");
  return DIC_OK;
}

int dic_fft_field(dic_handle* h, const dic_fft_params* fp, void* cuda_stream) {
  if (!h || !fp) return fail(DIC_EINVAL, "NULL argument");
  g_last_error.clear();
  if (fp->max_displacement < 0 || fp->max_displacement >= kFftLargeMax)
    return fail(DIC_EINVAL, "max_displacement %d outside [0, %d]", fp->max_displacement, kFftLargeMax - 1);
  if (!(fp->mad_eps >= 0.0) || fp->mad_tau != fp->mad_tau) return fail(DIC_EINVAL, "mad_tau/mad_eps invalid");
  if (!h->grid_ok) return fail(DIC_ESTATE, "the handle has no subset grid; call dic_set_subsets");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  h->last_stream = s;
  return run_fft(h, fp->max_displacement, fp->subpixel ? 1 : 0, fp->mad_tau, fp->mad_eps, s);
}

int dic_get_fft_results(const dic_handle* h, dic_fft_results* out) {
  if (!h || !out) return fail(DIC_EINVAL, "NULL argument");
  if (!h->has_fft) return fail(DIC_ESTATE, "no FFT initialiser run on this handle");
  dic_fft_results r{};
  r.n_points = h->npts;
  r.nx = h->nx;
  r.ny = h->ny;
  r.n_levels = h->fft_levels;
  for (int i = 0; i < h->fft_levels; ++i) r.window[i] = h->fft_window[i];
  r.u = h->fft_res[0];
  r.v = h->fft_res[1];
  r.peak = h->fft_res[2];
  r.status = h->fft_status;
  r.replaced = h->fft_rep;
  *out = r;
  return DIC_OK;
}

int dic_fftcc_windows(dic_handle* h, int32_t window, int64_t n_windows, const int32_t* origins, int32_t subpixel,
                      float* u, float* v, float* peak, void* cuda_stream) {
  if (!h) return fail(DIC_EINVAL, "handle is NULL");
  g_last_error.clear();
  const bool pow2 = window >= 4 && (window & (window - 1)) == 0;
  const bool odd = (window & 1) == 1 && window >= 3 && window < kFftSmallMax;
  if (!(pow2 && window <= kFftLargeMax) && !odd)
    return fail(DIC_EINVAL, "window %d: odd 3..%d or a power of two 4..%d", window, kFftSmallMax - 1, kFftLargeMax);
  if (window > h->W || window > h->H) return fail(DIC_EINVAL, "window %d larger than the images", window);
  if (subpixel && window > kFftSmallMax) return fail(DIC_EINVAL, "the sub-pixel fit needs window <= %d", kFftSmallMax);
  if (n_windows < 0) return fail(DIC_EINVAL, "n_windows < 0");
  if (n_windows == 0) return DIC_OK;
  if (n_windows > (int64_t{1} << 31) - 1) return fail(DIC_EINVAL, "too many windows");
  if (!origins || !u || !v || !peak) return fail(DIC_EINVAL, "NULL array");
  if ((reinterpret_cast<uintptr_t>(origins) & 15) != 0) return fail(DIC_EINVAL, "origins must be 16-byte aligned");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  FftCaps c;
  if (window > kFftSmallMax) {
    c.large = n_windows;
    c.work = n_windows * window * window;
  }
  int rc = fft_prepare(h, c);
  if (rc) return rc;
  if ((rc = fft_twiddles(h, odd ? window : (h->fft_tw_odd > 0 ? h->fft_tw_odd : 1), s))) return rc;
  FftccArgs a = fftcc_args(h, window, n_windows, subpixel ? 1 : 0, u, v, peak);
  a.org = reinterpret_cast<const int4*>(origins);
  DIC_CUDA(launch_fftcc(a, s), "fft cross-correlation");
  return DIC_OK;
}

int dic_mad_filter(const float* u, const float* v, const uint8_t* valid, int32_t nx, int32_t ny, double tau,
                   double eps, float* u_out, float* v_out, uint8_t* replaced, void* cuda_stream) {
  g_last_error.clear();
  if (nx < 0 || ny < 0) return fail(DIC_EINVAL, "negative field size");
  if (static_cast<int64_t>(nx) * ny == 0) return DIC_OK;
  if (!u || !v || !u_out || !v_out) return fail(DIC_EINVAL, "NULL array");
  if (u_out == u || v_out == v || u_out == v || v_out == u) return fail(DIC_EINVAL, "in-place filtering");
  if (!(eps >= 0.0) || tau != tau) return fail(DIC_EINVAL, "tau/eps invalid");
  MadArgs a{u, v, valid, nx, ny, tau, eps, u_out, v_out, replaced};
  DIC_CUDA(launch_mad(a, static_cast<cudaStream_t>(cuda_stream)), "outlier removal");
  return DIC_OK;
}

int dic_update_reference(dic_handle* h, void* cuda_stream) {
  if (!h) return fail(DIC_EINVAL, "handle is NULL");
  g_last_error.clear();
  if (!h->has_results) return fail(DIC_ESTATE, "no correlation to update the reference from");
  if (h->shape == DIC_QUADRATIC)
    return fail(DIC_EINVAL, "reference updating needs a rigid or affine shape function");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  h->last_stream = s;
  int rc = ensure_increments(h);
  if (rc) return rc;
  if ((rc = run_totals(h, 1, s))) return rc;
  h->acc_identity = false;
  ++h->n_updates;
  // the deformed image and its coefficients become the reference's
  if (h->ref_owned) hfree(h, h->ref_owned);
  h->ref = h->def;
  h->ref_owned = h->def_owned;
  h->ref_dtype = h->def_dtype;
  h->def_owned = nullptr;
  void* t = h->c_ref;
  h->c_ref = h->c_def;
  h->c_def = t;
  h->ref_dirty = h->def_dirty;
  h->def_dirty = true;
  DIC_CUDA(launch_identity_start(point_arrays(h), h->nparams, h->roi_ok, s), "identity start");
  return DIC_OK;
}

int dic_get_total_results(dic_handle* h, dic_total_results* out, void* cuda_stream) {
  if (!h || !out) return fail(DIC_EINVAL, "NULL argument");
  g_last_error.clear();
  if (!h->has_results) return fail(DIC_ESTATE, "no correlation since the handle was created or re-gridded");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  int rc = ensure_increments(h);
  if (rc) return rc;
  if ((rc = run_totals(h, 0, s))) return rc;
  dic_total_results r{};
  r.n_points = h->npts;
  r.nx = h->nx;
  r.ny = h->ny;
  r.n_params = h->nparams;
  r.n_updates = h->n_updates;
  r.u = h->tot_u;
  r.v = h->tot_v;
  r.p = h->tot_p;
  r.status = h->tot_status;
  *out = r;
  return DIC_OK;
}

void dic_destroy(dic_handle* h) { release(h); }

}  // extern "C"
