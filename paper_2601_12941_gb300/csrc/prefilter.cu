// Cubic B-spline prefilter (Sec. 2.2: bicubic B-spline interpolation set-up), and
// the plain gray-level plane of the bicubic convolution interpolant.
//
// The interpolating coefficients c of a line I satisfy (c[k-1] + 4 c[k] + c[k+1]) / 6
// = I[k] with the whole-sample mirror boundary. On the mirror-extended line this is
// the convolution c = h * I with the two-sided exponential
//     h[k] = -6 z / (1 - z^2) * z^|k|,   z = sqrt(3) - 2,
// the inverse of the symmetric filter (1, 4, 1) / 6. The kernel applies h truncated
// to |k| <= K (|z|^(K+1) below the working precision: K = 14 in FP32, 28 in FP64)
// along x then along y, one 32x32 output tile per block, the input tile plus a
// K-pixel mirrored halo staged in shared memory. This replaces the usual pair of
// sequential recursive passes, whose per-line dependency chain does not map onto
// thousands of threads, by independent tiles that read the gray image once.
#include <math.h>

#include "dic_internal.cuh"

namespace dic {
namespace {

constexpr int kTile = 32;

template <typename T>
struct Taps {
  T h[29];
};

template <typename T>
constexpr int taps_radius();
template <>
constexpr int taps_radius<float>() { return 14; }
template <>
constexpr int taps_radius<double>() { return 28; }

template <typename T>
Taps<T> make_taps() {
  Taps<T> t{};
  const double z = sqrt(3.0) - 2.0;
  const double c0 = -6.0 * z / (1.0 - z * z);
  double zk = 1.0;
  for (int k = 0; k <= taps_radius<T>(); ++k) {
    t.h[k] = static_cast<T>(c0 * zk);
    zk *= z;
  }
  return t;
}

// outputs per thread along the filtered axis: each thread loads one run of
// G + 2K inputs and produces G outputs from it
template <typename T>
struct OutputsPerThread;
template <>
struct OutputsPerThread<float> { static constexpr int kValue = 4; };
template <>
struct OutputsPerThread<double> { static constexpr int kValue = 2; };

template <typename T, int K>
__global__ void __launch_bounds__(kThreads) prefilter_kernel(PrefilterArgs<T> a, Taps<T> taps) {
  constexpr int G = OutputsPerThread<T>::kValue;
  constexpr int IX = kTile + 2 * K;  // staged input tile width (and height)
  constexpr int RUN = G + 2 * K;     // inputs behind G outputs
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* in = reinterpret_cast<T*>(smem_raw);  // [IX][IX]
  T* mid = in + IX * IX;                   // [IX][kTile] after the x pass
  const int64_t x0 = static_cast<int64_t>(blockIdx.x) * kTile;
  const int64_t y0 = static_cast<int64_t>(blockIdx.y) * kTile;
  const int tid = threadIdx.x;

  const bool inside = x0 - K >= 0 && y0 - K >= 0 && x0 + kTile + K <= a.W && y0 + kTile + K <= a.H;
  if (inside) {
    for (int e = tid; e < IX * IX; e += kThreads) {
      const int iy = e / IX, ix = e % IX;
      in[e] = load_gray<T>(a.src, x0 - K + ix, y0 - K + iy);
    }
  } else {
    for (int e = tid; e < IX * IX; e += kThreads) {
      const int iy = e / IX, ix = e % IX;
      in[e] = load_gray<T>(a.src, mirror_index(x0 - K + ix, a.W), mirror_index(y0 - K + iy, a.H));
    }
  }
  __syncthreads();

  // x pass: every staged row, G consecutive outputs per item
  for (int e = tid; e < IX * (kTile / G); e += kThreads) {
    const int iy = e / (kTile / G), c0 = (e % (kTile / G)) * G;
    const T* row = in + iy * IX + c0;
    T v[RUN];
#pragma unroll
    for (int j = 0; j < RUN; ++j) v[j] = row[j];
#pragma unroll
    for (int m = 0; m < G; ++m) {
      T acc = taps.h[0] * v[m + K];
#pragma unroll
      for (int k = 1; k <= K; ++k) acc += taps.h[k] * (v[m + K - k] + v[m + K + k]);
      mid[iy * kTile + c0 + m] = acc;
    }
  }
  __syncthreads();

  // y pass: G consecutive output rows of one column per item
  for (int e = tid; e < kTile * (kTile / G); e += kThreads) {
    const int c = e % kTile, r0 = (e / kTile) * G;
    const T* colp = mid + r0 * kTile + c;
    T v[RUN];
#pragma unroll
    for (int j = 0; j < RUN; ++j) v[j] = colp[j * kTile];
    const int64_t gx = x0 + c;
#pragma unroll
    for (int m = 0; m < G; ++m) {
      T acc = taps.h[0] * v[m + K];
#pragma unroll
      for (int k = 1; k <= K; ++k) acc += taps.h[k] * (v[m + K - k] + v[m + K + k]);
      const int64_t gy = y0 + r0 + m;
      if (gx < a.W && gy < a.H) a.coef[gy * a.ldc + gx] = acc;
    }
  }
}

// Bicubic convolution (Keys, a = -1/2) interpolates the gray levels directly: the
// coefficient plane is the image converted to T, row by row, coalesced.
template <typename T>
__global__ void __launch_bounds__(kThreads) gray_plane_kernel(PrefilterArgs<T> a) {
  const int64_t n = static_cast<int64_t>(a.W) * a.H;
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * kThreads + threadIdx.x; e < n;
       e += static_cast<int64_t>(gridDim.x) * kThreads) {
    const int y = static_cast<int>(e / a.W), x = static_cast<int>(e % a.W);
    a.coef[static_cast<int64_t>(y) * a.ldc + x] = load_gray<T>(a.src, x, y);
  }
}

}  // namespace

template <typename T>
cudaError_t launch_gray_plane(const PrefilterArgs<T>& a, cudaStream_t s) {
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t need = (static_cast<int64_t>(a.W) * a.H + kThreads - 1) / kThreads;
  const int64_t cap = static_cast<int64_t>(sms > 0 ? sms : 1) * 8;
  const unsigned blocks = static_cast<unsigned>(need < cap ? (need > 0 ? need : 1) : cap);
  gray_plane_kernel<T><<<blocks, kThreads, 0, s>>>(a);
  return cudaGetLastError();
}

template cudaError_t launch_gray_plane<float>(const PrefilterArgs<float>&, cudaStream_t);
template cudaError_t launch_gray_plane<double>(const PrefilterArgs<double>&, cudaStream_t);

template <typename T>
cudaError_t launch_prefilter(const PrefilterArgs<T>& a, cudaStream_t s) {
  constexpr int K = taps_radius<T>();
  constexpr int IX = kTile + 2 * K;
  const size_t smem = sizeof(T) * static_cast<size_t>(IX * IX + IX * kTile);
  static const cudaError_t configured = cudaFuncSetAttribute(
      prefilter_kernel<T, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (configured != cudaSuccess) return configured;
  static const Taps<T> taps = make_taps<T>();
  dim3 grid((a.W + kTile - 1) / kTile, (a.H + kTile - 1) / kTile);
  prefilter_kernel<T, K><<<grid, kThreads, smem, s>>>(a, taps);
  return cudaGetLastError();
}

template cudaError_t launch_prefilter<float>(const PrefilterArgs<float>&, cudaStream_t);
template cudaError_t launch_prefilter<double>(const PrefilterArgs<double>&, cudaStream_t);

}  // namespace dic
