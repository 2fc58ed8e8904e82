// Cubic B-spline prefilter (Sec. 2.2: "bicubic b-spline" interpolation set-up).
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

template <typename T, int K>
__global__ void __launch_bounds__(kThreads) prefilter_kernel(PrefilterArgs<T> a, Taps<T> taps) {
  constexpr int IX = kTile + 2 * K;  // staged input tile width (and height)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* in = reinterpret_cast<T*>(smem_raw);  // [IX][IX]
  T* mid = in + IX * IX;                   // [IX][kTile] after the x pass
  const int64_t x0 = static_cast<int64_t>(blockIdx.x) * kTile;
  const int64_t y0 = static_cast<int64_t>(blockIdx.y) * kTile;
  const int tid = threadIdx.x;

  for (int e = tid; e < IX * IX; e += kThreads) {
    const int iy = e / IX, ix = e % IX;
    const int64_t gx = mirror_index(x0 - K + ix, a.W);
    const int64_t gy = mirror_index(y0 - K + iy, a.H);
    in[e] = load_gray<T>(a.src, gx, gy);
  }
  __syncthreads();

  for (int e = tid; e < IX * kTile; e += kThreads) {
    const int iy = e / kTile, c = e % kTile;
    const T* row = in + iy * IX + c + K;
    T acc = taps.h[0] * row[0];
#pragma unroll
    for (int m = 1; m <= K; ++m) acc += taps.h[m] * (row[-m] + row[m]);
    mid[e] = acc;
  }
  __syncthreads();

  for (int e = tid; e < kTile * kTile; e += kThreads) {
    const int r = e / kTile, c = e % kTile;
    const int64_t gx = x0 + c, gy = y0 + r;
    if (gx >= a.W || gy >= a.H) continue;
    const T* col = mid + (r + K) * kTile + c;
    T acc = taps.h[0] * col[0];
#pragma unroll
    for (int m = 1; m <= K; ++m) acc += taps.h[m] * (col[-m * kTile] + col[m * kTile]);
    a.coef[gy * a.ldc + gx] = acc;
  }
}

}  // namespace

template <typename T>
cudaError_t launch_prefilter(const PrefilterArgs<T>& a, cudaStream_t s) {
  constexpr int K = taps_radius<T>();
  constexpr int IX = kTile + 2 * K;
  const size_t smem = sizeof(T) * static_cast<size_t>(IX * IX + IX * kTile);
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(prefilter_kernel<T, K>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    configured = true;
  }
  static const Taps<T> taps = make_taps<T>();
  dim3 grid((a.W + kTile - 1) / kTile, (a.H + kTile - 1) / kTile);
  prefilter_kernel<T, K><<<grid, kThreads, smem, s>>>(a, taps);
  return cudaGetLastError();
}

template cudaError_t launch_prefilter<float>(const PrefilterArgs<float>&, cudaStream_t);
template cudaError_t launch_prefilter<double>(const PrefilterArgs<double>&, cudaStream_t);

}  // namespace dic
