// Cubic B-spline prefilter (Sec. 2.2: bicubic B-spline interpolation set-up), and
// the plain gray-level plane of the bicubic convolution interpolant.
//
// The interpolating coefficients c of a line I satisfy (c[k-1] + 4 c[k] + c[k+1]) / 6
// = I[k] with the whole-sample mirror boundary. On the mirror-extended line this is
// the convolution c = h * I with the two-sided exponential
//     h[k] = -6 z / (1 - z^2) * z^|k|,   z = sqrt(3) - 2,
// the inverse of the symmetric filter (1, 4, 1) / 6; h factors into a causal and an
// anticausal first-order recursion, c = -6 z A(C(I)) with C: q[k] = I[k] + z q[k-1]
// and A: d[k] = q[k] + z d[k+1] (Unser, Aldroubi and Eden 1993).
//
// FP32 coefficients (prefilter_iir_kernel): one block per 128-column strip and 256
// rows. The x pass runs both recursions along 60-pixel runs of a row (32 outputs and
// 14 warm-up samples on each side: |z|^15 < 3e-9, below FP32 rounding), reading the
// gray levels straight from global memory with 16-byte loads; the y pass runs them
// down each column of the strip over a ring of 64 x-filtered rows in shared memory,
// so the y halo is filtered once per 256 rows and every gray byte is read once from
// DRAM. A thread's recursions are serial chains; the 30k blocks of a gigapixel image
// supply the parallelism.
//
// FP64 coefficients (prefilter_kernel): h truncated to |k| <= 28 (|z|^29 below FP64
// rounding), one 32 x 32 output tile per block with its mirrored halo in shared
// memory, x pass then y pass.
#include <math.h>

#include "dic_internal.cuh"

namespace dic {
namespace {

constexpr int kTile = 32;

template <typename T>
struct Taps {
  T h[29];
};

// truncation radius of the FIR form (FP64; the FP32 path runs the recursions)
template <typename T>
constexpr int taps_radius();
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

// ---------------------------------------------------------------- FP32: recursive passes
constexpr int kPfThreads = 128;
constexpr int kPfStrip = 128;                  // output columns per block
constexpr int kPfRows = 256;                   // output rows per block
constexpr int kPfBatch = 32;                   // rows per x-pass batch (4 segments of 32 columns each)
constexpr int kPfLead = 14;                    // warm-up samples of each recursion
constexpr int kPfRun = 32 + 2 * kPfLead;       // samples behind 32 outputs
constexpr int kPfSegPitch = 36;                // ring floats per 32-column segment (bank spread)
constexpr int kPfRowPitch = 4 * kPfSegPitch;   // ring floats per row
constexpr int kPfSlots = 64;                   // ring rows (>= 32 + kPfRun - 1... two batches)
constexpr size_t kPfSmem = sizeof(float) * kPfSlots * kPfRowPitch;

template <int DT>
struct GrayBytes;
template <>
struct GrayBytes<DIC_U8> { static constexpr int kValue = 1; };
template <>
struct GrayBytes<DIC_U16> { static constexpr int kValue = 2; };
template <>
struct GrayBytes<DIC_BF16> { static constexpr int kValue = 2; };
template <>
struct GrayBytes<DIC_F32> { static constexpr int kValue = 4; };
template <>
struct GrayBytes<DIC_F64> { static constexpr int kValue = 8; };

// element i of 16 gray-level bytes as FP32, exactly (integers through the
// 2^23 exponent: 0x4B000000 | n is the float 2^23 + n); FP64 gray levels arrive
// already rounded to FP32 (see RowRun)
template <int DT>
__device__ __forceinline__ float unpack(const uint4& w, int i) {
  constexpr int B = DT == DIC_F64 ? 4 : GrayBytes<DT>::kValue;   // bytes per element as held
  const uint32_t word = i * B < 4 ? w.x : i * B < 8 ? w.y : i * B < 12 ? w.z : w.w;
  if constexpr (DT == DIC_U8) {
    return __uint_as_float(__byte_perm(word, 0x4B000000u, 0x7440u + (i & 3))) - 8388608.0f;
  } else if constexpr (DT == DIC_U16) {
    return __uint_as_float(__byte_perm(word, 0x4B000000u, (i & 1) ? 0x7432u : 0x7410u)) - 8388608.0f;
  } else if constexpr (DT == DIC_BF16) {
    return __uint_as_float(__byte_perm(word, 0u, (i & 1) ? 0x3244u : 0x1044u));
  } else {   // F32, and F64 (held as FP32 values, see RowRun)
    return __uint_as_float(word);
  }
}

// x-pass item: 64 gray levels of one row, columns xa .. xa + 63 (mirrored into the
// image where they leave it); held as raw 16-byte words when the row allows
// aligned vector loads. FP64 gray levels are rounded to FP32 as they arrive (the
// recursions run in FP32), which keeps the run at 16 words.
template <int DT>
struct RowBytes {
  static constexpr int kValue = DT == DIC_F64 ? 4 : GrayBytes<DT>::kValue;
};
template <int DT>
struct RowRun {
  static constexpr int kVec = 64 * RowBytes<DT>::kValue / 16;
  uint4 w[kVec];
};

template <int DT>
__device__ __forceinline__ void load_run(RowRun<DT>& run, const PrefilterArgs<float>& a, bool fast, int xa,
                                         int y) {
  const int gy = static_cast<int>(mirror_index(y, a.H));
  const char* row = static_cast<const char*>(a.src.data) + static_cast<int64_t>(gy) * a.src.stride;
  if (fast && DT == DIC_F64) {
    const double2* src = reinterpret_cast<const double2*>(row + static_cast<int64_t>(xa) * 8);
#pragma unroll 4
    for (int v = 0; v < RowRun<DT>::kVec; ++v) {
      const double2 p = src[2 * v], q = src[2 * v + 1];
      run.w[v] = make_uint4(__float_as_uint(static_cast<float>(p.x)), __float_as_uint(static_cast<float>(p.y)),
                            __float_as_uint(static_cast<float>(q.x)), __float_as_uint(static_cast<float>(q.y)));
    }
  } else if (fast) {
    const uint4* src = reinterpret_cast<const uint4*>(row + static_cast<int64_t>(xa) * GrayBytes<DT>::kValue);
#pragma unroll
    for (int v = 0; v < RowRun<DT>::kVec; ++v) run.w[v] = src[v];
  } else if (DT == DIC_F64) {
#pragma unroll
    for (int v = 0; v < RowRun<DT>::kVec; ++v) {
      uint32_t q[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int64_t gx = mirror_index(xa + 4 * v + e, a.W);
        q[e] = __float_as_uint(static_cast<float>(reinterpret_cast<const double*>(row)[gx]));
      }
      run.w[v] = make_uint4(q[0], q[1], q[2], q[3]);
    }
  } else {
    // edge strips: element by element through the mirror, repacked into words
    constexpr int EPV = 16 / GrayBytes<DT>::kValue;
#pragma unroll
    for (int v = 0; v < RowRun<DT>::kVec; ++v) {
      uint32_t q[4] = {0u, 0u, 0u, 0u};
#pragma unroll
      for (int e = 0; e < EPV; ++e) {
        const int64_t gx = mirror_index(xa + v * EPV + e, a.W);
        const unsigned char* px = reinterpret_cast<const unsigned char*>(row) + gx * GrayBytes<DT>::kValue;
#pragma unroll
        for (int b = 0; b < GrayBytes<DT>::kValue; ++b) {
          const int byte = e * GrayBytes<DT>::kValue + b;
          q[byte >> 2] |= static_cast<uint32_t>(px[b]) << (8 * (byte & 3));
        }
      }
      run.w[v] = make_uint4(q[0], q[1], q[2], q[3]);
    }
  }
}

// Both recursions over the 60 samples run[2 .. 61] of a row (columns xa + 2 ...);
// the 32 outputs (columns xa + 16 .. xa + 47) go to dst[0 .. 31] (16-byte aligned).
template <int DT>
__device__ __forceinline__ void x_recursions(const RowRun<DT>& run, float z, float gain, float* dst) {
  float q[kPfRun - kPfLead];   // causal values of samples kPfLead .. kPfRun - 1
  float acc = 0.0f;
#pragma unroll
  for (int j = 0; j < kPfRun; ++j) {
    const int e = j + 2;
    const float x = unpack<DT>(run.w[e * RowBytes<DT>::kValue / 16], e % (16 / RowBytes<DT>::kValue));
    acc = j == 0 ? x : fmaf(z, acc, x);
    if (j >= kPfLead) q[j - kPfLead] = acc;
  }
  float d = q[kPfRun - kPfLead - 1];
  float o[4];
#pragma unroll
  for (int j = kPfRun - 2; j >= kPfLead; --j) {
    d = fmaf(z, d, q[j - kPfLead]);
    if (j < kPfLead + 32) {
      const int k = j - kPfLead;   // output 0 .. 31
      o[k & 3] = gain * d;
      if ((k & 3) == 0) *reinterpret_cast<float4*>(dst + k) = make_float4(o[0], o[1], o[2], o[3]);
    }
  }
}

// Both recursions down one column of the ring, rows BASE .. BASE + 59 (mod 64); the
// 32 outputs go to out[i * ld], i < valid.
template <int BASE>
__device__ __forceinline__ void y_recursions(const float* col, float z, float gain, float* out, int64_t ld,
                                             int valid) {
  float q[kPfRun - kPfLead];
  float acc = 0.0f;
#pragma unroll
  for (int j = 0; j < kPfRun; ++j) {
    const float x = col[((BASE + j) & (kPfSlots - 1)) * kPfRowPitch];
    acc = j == 0 ? x : fmaf(z, acc, x);
    if (j >= kPfLead) q[j - kPfLead] = acc;
  }
  float d = q[kPfRun - kPfLead - 1];
#pragma unroll
  for (int j = kPfRun - 2; j >= kPfLead; --j) {
    d = fmaf(z, d, q[j - kPfLead]);
    if (j < kPfLead + 32) {
      const int i = j - kPfLead;
      if (i < valid) out[static_cast<int64_t>(i) * ld] = gain * d;
    }
  }
}

// Block: columns x0 .. x0 + 127, rows y0 .. y0 + 255. Ring row of image row y:
// (y - y0 + kPfLead) mod 64; batch b holds rows y0 - 14 + 32 b .. + 31, and the y pass
// of chunk k (output rows y0 + 32 k ..) reads batches k and k + 1.
template <int DT>
__global__ void __launch_bounds__(kPfThreads, 4) prefilter_iir_kernel(PrefilterArgs<float> a, int vec_ok, float z,
                                                                    float gain) {
  extern __shared__ __align__(16) float ring[];
  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * kPfStrip;
  const int y0 = blockIdx.y * kPfRows;
  const int rows = min(kPfRows, a.H - y0);
  const int nchunks = (rows + kPfBatch - 1) / kPfBatch;
  // x-pass item of this thread: row r of each batch, 32-column segment s
  const int s = tid & 3, r = tid >> 2;
  const int xa = x0 + 32 * s - 16;
  const bool fast = vec_ok && x0 - 16 >= 0 && x0 + kPfStrip + 16 <= a.W;
  // y-pass column of this thread and its place in a ring row
  const int c = tid;
  const int ph = (c >> 5) * kPfSegPitch + (c & 31);
  const bool col_ok = x0 + c < a.W;

  RowRun<DT> run;
  load_run<DT>(run, a, fast, xa, y0 - kPfLead + r);
  x_recursions<DT>(run, z, gain, ring + r * kPfRowPitch + s * kPfSegPitch);
  load_run<DT>(run, a, fast, xa, y0 - kPfLead + kPfBatch + r);
  for (int k = 0; k < nchunks; ++k) {
    x_recursions<DT>(run, z, gain, ring + ((kPfBatch * (k + 1) + r) & (kPfSlots - 1)) * kPfRowPitch + s * kPfSegPitch);
    if (k + 2 <= nchunks) load_run<DT>(run, a, fast, xa, y0 - kPfLead + kPfBatch * (k + 2) + r);
    __syncthreads();
    // y pass of output rows y0 + 32 k .. + 31 from ring rows 32 k .. 32 k + 59 (mod 64)
    float* out = a.coef + static_cast<int64_t>(y0 + kPfBatch * k) * a.ldc + x0 + c;
    const int valid_rows = col_ok ? min(32, a.H - (y0 + kPfBatch * k)) : 0;
    if (k & 1)
      y_recursions<kPfBatch>(ring + ph, z, gain, out, a.ldc, valid_rows);
    else
      y_recursions<0>(ring + ph, z, gain, out, a.ldc, valid_rows);
    __syncthreads();
  }
}

template <int DT>
cudaError_t launch_iir(const PrefilterArgs<float>& a, cudaStream_t s) {
  static const cudaError_t configured = cudaFuncSetAttribute(
      prefilter_iir_kernel<DT>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(kPfSmem));
  if (configured != cudaSuccess) return configured;
  const int vec_ok = (reinterpret_cast<uintptr_t>(a.src.data) % 16 == 0) && (a.src.stride % 16 == 0);
  const double zd = sqrt(3.0) - 2.0;
  dim3 grid((a.W + kPfStrip - 1) / kPfStrip, (a.H + kPfRows - 1) / kPfRows);
  prefilter_iir_kernel<DT><<<grid, kPfThreads, kPfSmem, s>>>(a, vec_ok, static_cast<float>(zd),
                                                              static_cast<float>(-6.0 * zd));
  return cudaGetLastError();
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

template <>
cudaError_t launch_prefilter<float>(const PrefilterArgs<float>& a, cudaStream_t s) {
  switch (a.src.dtype) {
    case DIC_U8: return launch_iir<DIC_U8>(a, s);
    case DIC_U16: return launch_iir<DIC_U16>(a, s);
    case DIC_BF16: return launch_iir<DIC_BF16>(a, s);
    case DIC_F32: return launch_iir<DIC_F32>(a, s);
    default: return launch_iir<DIC_F64>(a, s);
  }
}

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

template cudaError_t launch_prefilter<double>(const PrefilterArgs<double>&, cudaStream_t);

}  // namespace dic
