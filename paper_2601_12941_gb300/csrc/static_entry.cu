// dic_correlate_static: the correlation of dic_correlate for small problems,
// without any memory allocation. For callers that cannot allocate device memory
// at the point of the call (for instance code running inside an allocator's
// callback, a real-time loop that must not take the driver's allocation locks, or
// a host that hands every byte of device memory to its own pool): the caller
// passes device images and device output arrays, and every intermediate buffer
// (spline coefficients, frontier lists, counters, seed scores, neighbour records)
// lives in one statically sized device array of this library, g_static_scratch.
//
// The array is shared by all calls in the process and keeps the last call's
// contents; the calls clear what has to start from zero. Two calls whose work
// overlaps on the GPU (different streams, or different host threads) race on it,
// so callers serialise them. The first call on a device looks up the array's
// device address (cudaGetSymbolAddress) and caches it; make that first call
// before any stream capture. Limits: see DIC_STATIC_* in include/dic.h.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>

#include <string.h>

#include <mutex>

#include "dic_internal.cuh"

using namespace dic;

namespace {

constexpr size_t kAlign = 256;
constexpr size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// worst-case layout of the scratch under the DIC_STATIC_* limits
constexpr size_t kPlaneBytes = align_up(sizeof(float) * static_cast<size_t>(DIC_STATIC_MAX_PIXELS));
constexpr size_t kPointsPlus = static_cast<size_t>(DIC_STATIC_MAX_POINTS) + 2;
constexpr size_t kSide = 2 * static_cast<size_t>(DIC_STATIC_MAX_RADIUS) + 1;
constexpr size_t kScratchBytes = 2 * kPlaneBytes                               // coefficient planes
                                 + align_up(sizeof(int64_t) * kPointsPlus)      // accept records
                                 + 2 * align_up(sizeof(int32_t) * kPointsPlus)  // frontier lists
                                 + align_up(sizeof(int32_t) * kPointsPlus)      // wave sizes
                                 + align_up(sizeof(int32_t) * kNumCounters)     // counters
                                 + align_up(sizeof(int32_t) * 4 * DIC_STATIC_MAX_SEEDS)   // seed centres, indices, best
                                 + align_up(sizeof(double) * DIC_STATIC_MAX_SEEDS * kSide * kSide);

static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

// the caller's message buffer of the current call (no allocation: formatted in place)
thread_local char* g_errbuf = nullptr;
thread_local int g_errlen = 0;

int sfail(int code, const char* fmt, ...) {
  if (g_errbuf && g_errlen > 0) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_errbuf, static_cast<size_t>(g_errlen), fmt, ap);
    va_end(ap);
  }
  return code;
}

int scuda(cudaError_t e, const char* what) {
  return sfail(DIC_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define SCUDA(call, what)                             \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return scuda(e_, what);    \
  } while (0)

// device address of g_static_scratch, looked up once per device
constexpr int kMaxDevices = 64;
unsigned char* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mutex;

int scratch_for_current_device(unsigned char** out) {
  int dev = 0;
  SCUDA(cudaGetDevice(&dev), "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return sfail(DIC_EINVAL, "device %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    SCUDA(cudaGetSymbolAddress(&p, g_static_scratch), "cudaGetSymbolAddress");
    g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_ptr[dev];
  return DIC_OK;
}

bool encode_plane_static(CUtensorMap* map, CUtensorMapDataType type, const void* base, int W, int H,
                         int64_t pitch_bytes, int box_w, int box_h) {
  static const PFN_cuTensorMapEncodeTiled_v12000 enc = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    return nullptr;
  }();
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

CUtensorMapDataType gray_type(int dtype) {
  switch (dtype) {
    case DIC_U8: return CU_TENSOR_MAP_DATA_TYPE_UINT8;
    case DIC_U16: return CU_TENSOR_MAP_DATA_TYPE_UINT16;
    case DIC_BF16: return CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    case DIC_F32: return CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    default: return CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
  }
}

size_t elem_size(int dt) {
  static const size_t es[5] = {1, 2, 2, 4, 8};
  return dt >= 0 && dt < 5 ? es[dt] : 0;
}

int64_t fdiv(int64_t a, int64_t b) {
  int64_t q = a / b;
  if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
  return q;
}

}  // namespace

extern "C" int dic_correlate_static(const dic_image* ref, const dic_image* def, int32_t subset_size,
                                    int32_t subset_step, int32_t shape_fn, const dic_params* params,
                                    const int32_t* seeds_xy, int32_t n_seeds, const dic_static_outputs* out,
                                    void* cuda_stream, char* errbuf, int32_t errlen) {
  g_errbuf = errbuf;
  g_errlen = errlen;
  if (errbuf && errlen > 0) errbuf[0] = '\0';
  // ---- arguments
  if (!ref || !def || !params || !seeds_xy || !out) return sfail(DIC_EINVAL, "NULL argument");
  if (!ref->data || !def->data || !ref->on_device || !def->on_device)
    return sfail(DIC_EINVAL, "images must be device buffers (on_device = 1)");
  if (ref->width != def->width || ref->height != def->height || ref->dtype != def->dtype)
    return sfail(DIC_EINVAL, "reference and deformed images differ in size or dtype");
  const size_t es = elem_size(ref->dtype);
  if (es == 0) return sfail(DIC_EINVAL, "unknown dtype %d", ref->dtype);
  const int W = ref->width, H = ref->height;
  if (W < 8 || H < 8) return sfail(DIC_EINVAL, "images must be at least 8 x 8");
  const int64_t ldc = (static_cast<int64_t>(W) + 31) / 32 * 32;
  if (ldc * H > DIC_STATIC_MAX_PIXELS)
    return sfail(DIC_EINVAL, "image %dx%d exceeds the static limit of %d padded pixels", W, H,
                 DIC_STATIC_MAX_PIXELS);
  if (subset_size < 3 || subset_size > kMaxSubset || subset_size % 2 == 0 || subset_size > W ||
      subset_size > H)
    return sfail(DIC_EINVAL, "subset_size %d invalid", subset_size);
  if (subset_step < 1) return sfail(DIC_EINVAL, "subset_step must be >= 1");
  if (shape_fn != DIC_RIGID && shape_fn != DIC_AFFINE && shape_fn != DIC_QUADRATIC)
    return sfail(DIC_EINVAL, "unknown shape function %d", shape_fn);
  if (params->precision != DIC_MIXED) return sfail(DIC_EINVAL, "only DIC_MIXED is available here");
  if (params->init != DIC_INIT_SEARCH) return sfail(DIC_EINVAL, "only DIC_INIT_SEARCH is available here");
  if (params->max_iter < 1 || !(params->conv_threshold > 0.0) || !(params->zncc_min >= -1.0) ||
      !(params->zncc_min <= 1.0))
    return sfail(DIC_EINVAL, "invalid parameters");
  if (params->search_radius < 0 || params->search_radius > DIC_STATIC_MAX_RADIUS)
    return sfail(DIC_EINVAL, "search_radius %d exceeds the static limit of %d", params->search_radius,
                 DIC_STATIC_MAX_RADIUS);
  if (n_seeds < 1 || n_seeds > DIC_STATIC_MAX_SEEDS)
    return sfail(DIC_EINVAL, "n_seeds must be in [1, %d]", DIC_STATIC_MAX_SEEDS);
  const int r = (subset_size - 1) / 2;
  const int nx = (W - 1 - 2 * r) / subset_step + 1, ny = (H - 1 - 2 * r) / subset_step + 1;
  const int64_t npts = static_cast<int64_t>(nx) * ny;
  if (npts > DIC_STATIC_MAX_POINTS)
    return sfail(DIC_EINVAL, "%lld grid points exceed the static limit of %d", static_cast<long long>(npts),
                 DIC_STATIC_MAX_POINTS);
  if (!out->u || !out->v || !out->p || !out->zncc || !out->iters || !out->converged || !out->status ||
      !out->wave)
    return sfail(DIC_EINVAL, "every output array is required");
  const int nparams = shape_fn == DIC_RIGID ? 2 : shape_fn == DIC_AFFINE ? 6 : 12;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);

  // ---- carve the scratch
  unsigned char* base = nullptr;
  int rc = scratch_for_current_device(&base);
  if (rc) return rc;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    unsigned char* p = base + off;
    off += align_up(bytes);
    return p;
  };
  float* c_ref = reinterpret_cast<float*>(take(kPlaneBytes));
  float* c_def = reinterpret_cast<float*>(take(kPlaneBytes));
  int64_t* accept = reinterpret_cast<int64_t*>(take(sizeof(int64_t) * kPointsPlus));
  int32_t* front0 = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * kPointsPlus));
  int32_t* front1 = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * kPointsPlus));
  int32_t* wave_sizes = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * kPointsPlus));
  int32_t* counters = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * kNumCounters));
  int32_t* seed_buf = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * 4 * DIC_STATIC_MAX_SEEDS));
  double* scores = reinterpret_cast<double*>(take(sizeof(double) * DIC_STATIC_MAX_SEEDS * kSide * kSide));
  if (off > kScratchBytes) return sfail(DIC_EINVAL, "scratch layout exceeds the static array");
  int32_t* seed_xy = seed_buf;
  int32_t* seed_q = seed_buf + 2 * DIC_STATIC_MAX_SEEDS;
  int32_t* seed_best = seed_buf + 3 * DIC_STATIC_MAX_SEEDS;

  // ---- spline coefficients of both images
  GrayPlane gref{ref->data, ref->row_stride_bytes ? ref->row_stride_bytes : static_cast<int64_t>(W * es),
                 ref->dtype};
  GrayPlane gdef{def->data, def->row_stride_bytes ? def->row_stride_bytes : static_cast<int64_t>(W * es),
                 def->dtype};
  SCUDA(launch_prefilter<float>(PrefilterArgs<float>{gref, W, H, c_ref, ldc}, s), "prefilter");
  SCUDA(launch_prefilter<float>(PrefilterArgs<float>{gdef, W, H, c_def, ldc}, s), "prefilter");

  // ---- per-point state: the caller's outputs plus the accept records
  PointArrays pa{};
  pa.n = npts;
  pa.nx = nx;
  pa.ny = ny;
  pa.u = out->u;
  pa.v = out->v;
  pa.p = out->p;
  pa.zncc = out->zncc;
  pa.accept = accept;
  pa.iters = out->iters;
  pa.converged = out->converged;
  pa.status = out->status;
  pa.wave = out->wave;
  SCUDA(launch_reset_points(pa, nparams, nullptr, s), "point reset");
  SCUDA(cudaMemsetAsync(counters, 0, sizeof(int32_t) * kNumCounters, s), "counter reset");

  // ---- seeds (snapped to the nearest grid point, ties to the lower index)
  int32_t hseed[3 * DIC_STATIC_MAX_SEEDS];
  for (int i = 0; i < n_seeds; ++i) {
    int64_t gi = fdiv(2 * (static_cast<int64_t>(seeds_xy[2 * i]) - r) + subset_step - 1, 2 * subset_step);
    int64_t gj = fdiv(2 * (static_cast<int64_t>(seeds_xy[2 * i + 1]) - r) + subset_step - 1, 2 * subset_step);
    gi = gi < 0 ? 0 : (gi > nx - 1 ? nx - 1 : gi);
    gj = gj < 0 ? 0 : (gj > ny - 1 ? ny - 1 : gj);
    hseed[2 * i] = r + static_cast<int32_t>(gi) * subset_step;
    hseed[2 * i + 1] = r + static_cast<int32_t>(gj) * subset_step;
    hseed[2 * DIC_STATIC_MAX_SEEDS + i] = static_cast<int32_t>(gj * nx + gi);
  }
  SCUDA(cudaMemcpyAsync(seed_buf, hseed, sizeof hseed, cudaMemcpyHostToDevice, s), "seed upload");
  const int R = params->search_radius;
  SCUDA(launch_seed_scores(SeedArgs{gref, gdef, W, H, subset_size, R, n_seeds, seed_xy, scores}, s),
        "seed search");
  SCUDA(launch_seed_commit(SeedCommitArgs{n_seeds, R, nparams, seed_q, scores, seed_best, out->p, out->status,
                                          out->wave, front0, counters, nullptr, nullptr, nullptr},
                           s),
        "seed commit");

  // ---- propagation waves
  WaveArgs<float> a{};
  a.W = W;
  a.H = H;
  a.ref_gray = gref;
  a.c_ref = c_ref;
  a.c_def = c_def;
  a.ldc = ldc;
  a.S = subset_size;
  a.r = r;
  a.step = subset_step;
  a.nx = nx;
  a.ny = ny;
  a.threads = wave_threads(subset_size);
  wave_bands(subset_size, a.threads, &a.bands, &a.band_h);
  a.tiles = wave_tiles<float>(subset_size, ref->dtype);
  CUtensorMap maps[3];
  const bool m0 = encode_plane_static(&maps[0], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, c_ref, W, H, ldc * 4,
                                      a.tiles.bxc, a.tiles.byc);
  const bool m1 = encode_plane_static(&maps[1], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, c_def, W, H, ldc * 4,
                                      a.tiles.bxc, a.tiles.byc);
  const bool m2 = encode_plane_static(&maps[2], gray_type(ref->dtype), gref.data, W, H, gref.stride,
                                      a.tiles.bxg, subset_size);
  a.tiles.coef_tma = m0 && m1;
  a.tiles.gray_tma = m2;
  a.pts = pa;
  a.roi_ok = nullptr;
  a.counters = counters;
  a.wave_sizes = wave_sizes;
  a.max_iter = params->max_iter;
  a.cost = params->cost;
  a.lm = params->optimizer == DIC_OPT_LEVENBERG_MARQUARDT;
  a.interp = DIC_BSPLINE3;
  a.conv_threshold = params->conv_threshold;
  a.zncc_min = params->zncc_min;
  int dev = 0, sms = 0;
  SCUDA(cudaGetDevice(&dev), "cudaGetDevice");
  SCUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "device query");
  const int grid = sms * wave_blocks_per_sm<float>(nparams, a.threads, wave_mode(a.lm, a.cost, a.interp),
                                                    static_cast<size_t>(a.tiles.smem_bytes));
  // A non-empty wave holds at least one point never attempted before, so the front
  // of wave npts is empty: batches are clipped to max_waves launches in all, and the
  // loop fails only if the front is still non-empty after the last allowed wave.
  int32_t hc[kNumCounters];
  int64_t k = 0;
  const int64_t max_waves = npts + 2;
  for (;;) {
    if (k >= max_waves) return sfail(DIC_ETIMEOUT, "wave loop exceeded its bound");
    const int64_t batch = max_waves - k < 8 ? max_waves - k : 8;
    for (int64_t b = 0; b < batch; ++b, ++k) {
      a.k = static_cast<int>(k);
      a.cur = (k & 1) ? front1 : front0;
      a.next = (k & 1) ? front0 : front1;
      SCUDA(launch_wave<float>(a, a.tiles, maps, nparams, grid, s), "wave launch");
    }
    // pageable destination: the copy returns once the counters have arrived
    SCUDA(cudaMemcpyAsync(hc, counters, sizeof hc, cudaMemcpyDeviceToHost, s), "counter read-back");
    SCUDA(cudaStreamSynchronize(s), "wave batch");
    if (hc[kCount + k % 3] == 0) break;
  }
  SCUDA(launch_finalize_points(pa, nparams, params->nan_unconverged, counters + kAccepted, s), "finalize");
  SCUDA(cudaMemcpyAsync(hc, counters, sizeof hc, cudaMemcpyDeviceToHost, s), "counter read-back");
  SCUDA(cudaStreamSynchronize(s), "correlate");
  if (out->n_accepted) *out->n_accepted = hc[kAccepted];
  if (hc[kError]) return sfail(DIC_ETIMEOUT, "a tile load did not complete in time");
  if (hc[kAccepted] == 0) return sfail(DIC_ENOSEED, "no seed was accepted");
  return DIC_OK;
}
