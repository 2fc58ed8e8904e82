// Internal declarations of libdic: kernel argument blocks, launchers and the
// small device helpers the kernels share. Nothing here is part of the C-ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dic.h"

namespace dic {

constexpr int kThreads = 256;        // threads per block of the subset kernels
constexpr int kWarps = kThreads / 32;
constexpr int kMaxSubset = 61;       // largest odd subset side supported
constexpr int kMaxParams = 12;

// device counters: frontier sizes and work cursors, each triple-buffered by wave
enum { kCount = 0, kWork = 3, kNumCounters = 8 };

// Gray-level plane as given by the caller (borrowed or owned).
struct GrayPlane {
  const void* data;
  int64_t stride;  // bytes per row
  int dtype;       // dic_dtype
};

template <typename T>
__device__ __forceinline__ T load_gray(const GrayPlane& g, int64_t x, int64_t y) {
  const char* row = static_cast<const char*>(g.data) + y * g.stride;
  switch (g.dtype) {
    case DIC_U8:
      return static_cast<T>(reinterpret_cast<const uint8_t*>(row)[x]);
    case DIC_U16:
      return static_cast<T>(reinterpret_cast<const uint16_t*>(row)[x]);
    case DIC_BF16: {
      uint32_t bits = static_cast<uint32_t>(reinterpret_cast<const uint16_t*>(row)[x]) << 16;
      return static_cast<T>(__uint_as_float(bits));
    }
    case DIC_F32:
      return static_cast<T>(reinterpret_cast<const float*>(row)[x]);
    default:
      return static_cast<T>(reinterpret_cast<const double*>(row)[x]);
  }
}

// Whole-sample mirror of index k into [0, n), n >= 2 (period 2n - 2).
__host__ __device__ __forceinline__ int64_t mirror_index(int64_t k, int64_t n) {
  const int64_t period = 2 * (n - 1);
  int64_t m = k % period;
  if (m < 0) m += period;
  return m < n ? m : period - m;
}

// Cubic B-spline weights for the four knots around x = i + t, t in [0, 1):
// knots i-1, i, i+1, i+2 get beta(t+1), beta(t), beta(1-t), beta(2-t).
template <typename T>
__device__ __forceinline__ void bspline_weights(T t, T& w0, T& w1, T& w2, T& w3) {
  const T one_sixth = T(1) / T(6);
  const T t2 = t * t;
  const T t3 = t2 * t;
  const T s = T(1) - t;
  w0 = s * s * s * one_sixth;
  w3 = t3 * one_sixth;
  w1 = T(0.5) * t3 - t2 + T(2) / T(3);
  w2 = T(1) - w0 - w1 - w3;
}

// ---------------------------------------------------------------- prefilter
template <typename T>
struct PrefilterArgs {
  GrayPlane src;
  int W, H;
  T* coef;      // [H][ldc]
  int64_t ldc;  // elements per coefficient row
};

// Interpolating cubic B-spline coefficients of a whole image (mirror boundary).
template <typename T>
cudaError_t launch_prefilter(const PrefilterArgs<T>& a, cudaStream_t s);

// ---------------------------------------------------------------- seeds
struct SeedArgs {
  GrayPlane ref, def;
  int W, H, S, R;
  int n_seeds;
  const int32_t* seed_xy;    // [n_seeds][2] subset centres (already snapped)
  double* scores;            // [n_seeds][(2R+1)^2], scratch
};
cudaError_t launch_seed_scores(const SeedArgs& a, cudaStream_t s);

// picks the best offset of every seed and puts the seeds on wave 0
struct SeedCommitArgs {
  int n_seeds, R, nparams;
  const int32_t* seed_q;     // [n_seeds] point index of each snapped seed
  const double* scores;
  double* p;                 // [n_points][nparams]
  uint8_t* status;
  int32_t* wave;
  int32_t* frontier0;        // wave-0 list
  int32_t* counters;
  const uint8_t* roi_ok;     // NULL: all points in the ROI
};
cudaError_t launch_seed_commit(const SeedCommitArgs& a, cudaStream_t s);

// ---------------------------------------------------------------- points
struct PointArrays {
  int64_t n;
  int nx, ny;
  double* u;
  double* v;
  double* p;         // [n][nparams]
  float* zncc;
  double* zncc64;    // ranks neighbours for the initial guess
  int32_t* iters;
  uint8_t* converged;
  uint8_t* status;
  int32_t* wave;
};

struct RoiArgs {
  GrayPlane mask;    // DIC_U8
  int S, r, step, nx, ny;
  uint8_t* roi_ok;   // [n_points]
};
cudaError_t launch_roi_flags(const RoiArgs& a, cudaStream_t s);
cudaError_t launch_reset_points(const PointArrays& pa, int nparams, const uint8_t* roi_ok,
                                cudaStream_t s);
cudaError_t launch_finalize_points(const PointArrays& pa, int nparams, int nan_rejected,
                                   int32_t* accepted, cudaStream_t s);

// ---------------------------------------------------------------- waves
template <typename T>
struct WaveArgs {
  // image geometry and planes
  int W, H;
  GrayPlane ref_gray;
  const T* c_ref;
  const T* c_def;
  int64_t ldc;
  // subset grid
  int S, r, step, nx, ny;
  int bands, band_h;         // thread t < S*bands: column t % S, rows band_h*(t/S) ...
  int win_cap;               // coefficient-window capacity in elements
  // per-point state
  PointArrays pts;
  const uint8_t* roi_ok;     // NULL: all in ROI
  // frontier
  const int32_t* cur;
  int32_t* next;
  int32_t* counters;
  int32_t* wave_sizes;       // [max waves] size of each wave's front
  int k;                     // wave index
  // controls
  int max_iter;
  double conv_threshold;
  double zncc_min;
};

template <typename T>
size_t wave_smem_bytes(int S, int win_cap);

template <typename T>
cudaError_t launch_wave(const WaveArgs<T>& a, int nparams, int grid, cudaStream_t s);

template <typename T>
int wave_blocks_per_sm(int nparams, size_t smem);

}  // namespace dic
