// Internal declarations of libdic: kernel argument blocks, launchers and the
// small device helpers the kernels share. Nothing here is part of the C-ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "dic.h"

namespace dic {

constexpr int kThreads = 256;        // threads per block of the image kernels
constexpr int kWaveThreads = 128;    // threads per block of the subset (wave) kernel, S > 31
constexpr int kWaveThreadsSmall = 64;  // the same for S <= 31
constexpr int kMaxSubset = 61;       // largest odd subset side supported
constexpr int kMaxParams = 12;

// device counters: frontier sizes and work cursors, each triple-buffered by wave;
// the accepted-point total; an error flag (a bounded wait ran out)
enum { kCount = 0, kWork = 3, kAccepted = 6, kError = 7, kNumCounters = 8 };

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

// Mirror of an index that lies at most n - 1 outside [0, n) (n >= 2).
__host__ __device__ __forceinline__ int mirror_near(int k, int n) {
  k = k < 0 ? -k : k;
  return k > n - 1 ? 2 * (n - 1) - k : k;
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

// Six times those weights: 6 beta(t+1) = s^3, 6 beta(t) = t^2 (3t - 6) + 4,
// 6 beta(1-t) = s^2 (3s - 6) + 4, 6 beta(2-t) = t^3, s = 1 - t; a sample is
// sum w_y w_x c / 36.
template <typename T>
__device__ __forceinline__ void bspline_weights6(T t, T& w0, T& w1, T& w2, T& w3) {
  const T s = T(1) - t;
  const T t2 = t * t, s2 = s * s;
  w3 = t2 * t;
  w0 = s2 * s;
  w1 = t2 * (T(3) * t - T(6)) + T(4);
  w2 = s2 * (T(3) * s - T(6)) + T(4);
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
// The gray levels themselves as the coefficient plane (the bicubic convolution
// interpolant needs no prefilter).
template <typename T>
cudaError_t launch_gray_plane(const PrefilterArgs<T>& a, cudaStream_t s);

// ---------------------------------------------------------------- FFT initialiser
constexpr int kFftSmallMax = 64;           // windows up to this side: one block each
constexpr int kFftLargeMax = 4096;
constexpr int kFftTwiddlesPow2 = 4095;     // nested table: exp(-2 pi i k / (2 ns)) at ns - 1 + k
constexpr int kFftMaxLevels = 16;

struct FftccArgs {
  GrayPlane ref, def;
  int W, H, L;
  int64_t n;                   // windows
  const int4* org;             // [n] (x0, y0, gx0, gy0); x0 < 0: skipped
  const float2* tw_pow2;       // kFftTwiddlesPow2 entries
  const float2* tw_odd;        // exp(-2 pi i t / L), t < L (odd L)
  int subpixel;                // Gaussian peak fit (L <= kFftSmallMax)
  float* u;                    // [n] outputs
  float* v;
  float* peak;
  float2* work;                // L > kFftSmallMax: [n][L][L] scratch
  double* norms;               // [n][2]
  unsigned long long* keys;    // [n]
  int32_t* nonflat;            // [n][2]
};

struct FftLevelArgs {
  int W, H, L;                 // image and window side
  int nx, ny;                  // windows of the level
  int grid;                    // 1: the subsets of the correlation grid; 0: tiles of side L
  int r, step;                 // grid geometry (grid = 1)
  const uint8_t* roi_ok;       // grid = 1: NULL or per grid point
  const float* pu;             // previous level's filtered field, NULL on the first level
  const float* pv;
  int pnx, pny;
  double pc0, pstep;           // its window centres: pc0 + i pstep
  int4* org;                   // [nx * ny] out
};

struct MadArgs {
  const float* u;
  const float* v;
  const uint8_t* valid;        // NULL: every value
  int nx, ny;
  double tau, eps;
  float* u_out;
  float* v_out;
  uint8_t* replaced;           // NULL or [nx * ny]
};

cudaError_t launch_twiddles(float2* tw, int L_odd, cudaStream_t s);
cudaError_t launch_fftcc_origins(const FftLevelArgs& a, cudaStream_t s);
cudaError_t launch_fftcc(const FftccArgs& a, cudaStream_t s);
cudaError_t launch_mad(const MadArgs& a, cudaStream_t s);

// ---------------------------------------------------------------- reference updating
struct TotalArgs {
  int nx, ny, r, step, nparams;
  const uint8_t* roi_ok;       // NULL: every point in the ROI
  const uint8_t* status;       // last correlation, against the current reference
  const double* p;             // [n][nparams]
  int identity;                // 1: no update yet (the accumulated warps are the identity)
  double* acc_u;               // [n] accumulated warps from the first reference
  double* acc_v;
  double* acc_A;               // [n][4] A00 A01 A10 A11
  uint8_t* acc_ok;             // [n]
  double* tot_u;               // [n] outputs: total warps to the last frame
  double* tot_v;
  double* tot_p;               // [n][nparams]
  uint8_t* tot_status;         // [n]
  int update;                  // 1: the totals also become the accumulated warps
};
cudaError_t launch_totals(const TotalArgs& a, cudaStream_t s);

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
  int32_t* best;             // [n_seeds] scratch: best offset index per seed
  double* p;                 // [n_points][nparams]
  uint8_t* status;
  int32_t* wave;
  int32_t* frontier0;        // wave-0 list
  int32_t* counters;
  const uint8_t* roi_ok;     // NULL: all points in the ROI
  const float* fft_u;        // non-NULL: seeds start from these estimates (rounded,
  const float* fft_v;        //   halves up) instead of the search scores
};
cudaError_t launch_seed_commit(const SeedCommitArgs& a, cudaStream_t s);
cudaError_t launch_fft_status(const uint8_t* roi_ok, uint8_t* status, int64_t n, cudaStream_t s);

// ---------------------------------------------------------------- points
struct PointArrays {
  int64_t n;
  int nx, ny;
  double* u;
  double* v;
  double* p;         // [n][nparams]
  float* zncc;
  int64_t* accept;   // (wave << 32) | ZNCC float bits of accepted points, else -1:
                     // one load tells a neighbour's wave, acceptance and rank
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
// subset centres of the grid in point order: x = r + (q % nx) step, y = r + (q / nx) step
cudaError_t launch_grid_points(int32_t* x, int32_t* y, int r, int step, int nx, int64_t n, cudaStream_t s);
cudaError_t launch_reset_points(const PointArrays& pa, int nparams, const uint8_t* roi_ok,
                                cudaStream_t s);
cudaError_t launch_finalize_points(const PointArrays& pa, int nparams, int nan_rejected,
                                   int32_t* accepted, cudaStream_t s);
// wave 0 of a sequence frame: the points the previous run accepted, keeping their warps
// (counters must be zero; counters[kCount] receives the size of front0)
cudaError_t launch_sequence_reset(const PointArrays& pa, int nparams, const uint8_t* roi_ok,
                                  int32_t* front0, int32_t* counters, cudaStream_t s);
// every in-ROI point starts the next sequence frame from the identity warp
cudaError_t launch_identity_start(const PointArrays& pa, int nparams, const uint8_t* roi_ok, cudaStream_t s);

// ---------------------------------------------------------------- waves
// Shared-memory tiles of the wave kernel: the reference gradients (fx, fy) and
// gray levels f - f0 of the subset pixels, the coefficient window (bxc x byc
// elements, also the TMA box of the coefficient planes), the reference gray tile
// (bxg x S elements of gray_es bytes, the TMA box of the gray plane) and where
// each region starts in dynamic shared memory (128-byte aligned).
struct WaveTiles {
  int bxc, byc;
  int bxg, gray_es;
  int coef_tma, gray_tma;    // 1: tiles arrive by TMA; 0: cooperative copies
  int off_fg, off_f, off_win, off_gray;
  int gray_alias;            // 1: the gray tile lies in the gradient region
  int smem_bytes;
};

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
  int threads;               // block size (wave_threads(S))
  int bands, band_h;         // thread t < S*bands: column t % S, rows band_h*(t/S) ...
                             // (S * bands <= threads)
  WaveTiles tiles;
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
  int cost;                  // dic_cost
  int lm;                    // 1: Levenberg-Marquardt (dic_optimizer)
  int interp;                // dic_interp of the coefficient planes
  double conv_threshold;
  double zncc_min;
  int solve64;               // 1: FP64 Hessian inverse, solve and ZNCC normalisation on the
                             // FP32 path (DIC_MIXED_FP64_SOLVE; kernel variant 3)
  int expire_waits;          // 1 (tests of the timeout path only): every tile-load wait
                             // gives up at once, as a wait that ran out of polls would
};

// Block size of the wave kernel for subset side S: two warps up to S = 31, four
// above. A point's serial steps run on warp 0 while the block's other warps wait,
// so smaller blocks for small subsets (whose shared memory allows twice as many
// resident points) keep more warps busy.
inline int wave_threads(int S) { return S <= 31 ? kWaveThreadsSmall : kWaveThreads; }

// Thread t < S * bands owns column t % S and rows [band_h (t / S), band_h (t / S + 1))
// of the subset: the fewest rows per band with S * bands <= threads.
inline void wave_bands(int S, int threads, int* bands, int* band_h) {
  for (int hgt = 1; hgt <= S; ++hgt) {
    const int b = (S + hgt - 1) / hgt;
    if (S * b <= threads) {
      *bands = b;
      *band_h = hgt;
      return;
    }
  }
  *bands = 1;
  *band_h = S;
}

template <typename T>
WaveTiles wave_tiles(int S, int gray_dtype);

// ---------------------------------------------------------------- strain
struct StrainArgs {
  const double* u;
  const double* v;
  const uint8_t* status;
  int nx, ny, step, window, basis, measure;
  float wa, wb;   // full-window slope weights in grid units: x slope = sum i (wa + wb j^2) u_ij
  float *dudx, *dudy, *dvdx, *dvdy, *exx, *eyy, *exy;
  uint8_t* valid;
};

cudaError_t launch_strain(const StrainArgs& a, cudaStream_t s);

template <typename T>
cudaError_t launch_wave(const WaveArgs<T>& a, const WaveTiles& t, const CUtensorMap* maps, int nparams,
                        int grid, cudaStream_t s);

template <typename T>
int wave_blocks_per_sm(int nparams, int threads, int mode, size_t smem);

// Kernel variant: 0 Gauss-Newton with ZNSSD on the B-spline (the default, leanest
// instantiation); 1 Gauss-Newton with any cost or interpolant; 2 Levenberg-Marquardt;
// 3 variant 0 with the Hessian inverse, the solve and the ZNCC normalisation in FP64
// (FP32 coefficients only).
inline int wave_mode(int lm, int cost, int interp, int solve64 = 0) {
  if (lm) return 2;
  if (cost == DIC_COST_ZNSSD && interp == DIC_BSPLINE3) return solve64 ? 3 : 0;
  return 1;
}

}  // namespace dic
