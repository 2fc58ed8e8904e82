// Dispatch of the wave kernel over its instantiations (compiled in wave_inst_*.cu),
// and the per-point bookkeeping kernels: ROI flags, grid centres, resets, finalize.
#include <math.h>

#include "wave_kernel.cuh"

namespace dic {
namespace {

__global__ void roi_flags_kernel(RoiArgs a) {
  const int64_t n = static_cast<int64_t>(a.nx) * a.ny;
  const int lane = threadIdx.x & 31;
  for (int64_t q = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; q < n;
       q += (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5) {
    const int xc = a.r + static_cast<int>(q % a.nx) * a.step;
    const int yc = a.r + static_cast<int>(q / a.nx) * a.step;
    bool all_in = true;
    for (int row = 0; row < a.S && all_in; ++row) {
      const uint8_t* m = static_cast<const uint8_t*>(a.mask.data) + (yc - a.r + row) * a.mask.stride;
      bool ok = true;
      for (int c = lane; c < a.S; c += 32) ok &= m[xc - a.r + c] != 0;
      all_in = __all_sync(0xffffffffu, ok);
    }
    if (lane == 0) a.roi_ok[q] = all_in ? 1 : 0;
  }
}

__global__ void grid_points_kernel(int32_t* x, int32_t* y, int r, int step, int nx, int64_t n) {
  for (int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; q < n;
       q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    x[q] = r + static_cast<int32_t>(q % nx) * step;
    y[q] = r + static_cast<int32_t>(q / nx) * step;
  }
}

__global__ void reset_points_kernel(PointArrays pa, int nparams, const uint8_t* roi_ok) {
  for (int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; q < pa.n;
       q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    pa.u[q] = 0.0;
    pa.v[q] = 0.0;
    for (int c = 0; c < nparams; ++c) pa.p[q * nparams + c] = 0.0;
    pa.zncc[q] = nanf("");
    pa.accept[q] = -1;
    pa.iters[q] = 0;
    pa.converged[q] = 0;
    pa.status[q] = (roi_ok && !roi_ok[q]) ? DIC_PT_NOT_IN_ROI : DIC_PT_NOT_REACHED;
    pa.wave[q] = -1;
  }
}

// Next frame of a sequence: every point accepted in the previous run joins wave 0
// and keeps its warp as the start; every other point is reset as for a new pair.
__global__ void sequence_reset_kernel(PointArrays pa, int nparams, const uint8_t* roi_ok,
                                      int32_t* front0, int32_t* counters) {
  for (int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; q < pa.n;
       q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const bool in_roi = !(roi_ok && !roi_ok[q]);
    const bool keep = in_roi && pa.status[q] == DIC_PT_OK;
    if (!keep) {
      pa.u[q] = 0.0;
      pa.v[q] = 0.0;
      for (int c = 0; c < nparams; ++c) pa.p[q * nparams + c] = 0.0;
    }
    pa.zncc[q] = nanf("");
    pa.accept[q] = -1;
    pa.iters[q] = 0;
    pa.converged[q] = 0;
    pa.status[q] = in_roi ? DIC_PT_NOT_REACHED : DIC_PT_NOT_IN_ROI;
    pa.wave[q] = keep ? 0 : -1;
    if (keep) front0[atomicAdd(&counters[kCount + 0], 1)] = static_cast<int32_t>(q);
  }
}

__global__ void finalize_points_kernel(PointArrays pa, int nparams, int nan_rejected,
                                       int32_t* accepted) {
  int count = 0;
  for (int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; q < pa.n;
       q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const bool ok = pa.status[q] == DIC_PT_OK;
    count += ok ? 1 : 0;
    if (nan_rejected && !ok) {
      const double nanv = nan("");
      pa.u[q] = nanv;
      pa.v[q] = nanv;
      for (int c = 0; c < nparams; ++c) pa.p[q * nparams + c] = nanv;
    }
  }
  count = warp_sum(count);
  if ((threadIdx.x & 31) == 0 && count) atomicAdd(accepted, count);
}

template <typename T, int NP>
cudaError_t launch_wave_np(const WaveArgs<T>& a, const CUtensorMap* maps, int grid, cudaStream_t s) {
  switch (dic::wave_mode(a.lm, a.cost, a.interp, a.solve64)) {
    case 0:
      return launch_wave_inst<T, NP, 0>(a, maps, grid, s);
    case 1:
      return launch_wave_inst<T, NP, 1>(a, maps, grid, s);
    case 3:
      if constexpr (std::is_same<T, float>::value) return launch_wave_inst<T, NP, 3>(a, maps, grid, s);
      return cudaErrorInvalidValue;
    default:
      return launch_wave_inst<T, NP, 2>(a, maps, grid, s);
  }
}

template <typename T, int NP>
int blocks_per_sm_np(int threads, int mode, size_t smem) {
  switch (mode) {
    case 0:
      return blocks_per_sm_inst<T, NP, 0>(threads, smem);
    case 1:
      return blocks_per_sm_inst<T, NP, 1>(threads, smem);
    case 3:
      if constexpr (std::is_same<T, float>::value) return blocks_per_sm_inst<T, NP, 3>(threads, smem);
      return 1;
    default:
      return blocks_per_sm_inst<T, NP, 2>(threads, smem);
  }
}

}  // namespace

template <typename T>
WaveTiles wave_tiles(int S, int gray_dtype) {
  WaveTiles t{};
  const int xalign = 16 / static_cast<int>(sizeof(T));
  t.bxc = ((S + 8 + xalign - 1) / xalign) * xalign;
  t.byc = S + 7;
  static const int es_of[5] = {1, 2, 2, 4, 8};
  t.gray_es = es_of[gray_dtype];
  const int galign = 16 / t.gray_es;
  t.bxg = ((S + galign - 1 + galign - 1) / galign) * galign;
  const int SS = ((S * S + 31) / 32) * 32;
  auto al = [](int x) { return (x + 127) & ~127; };
  // reference gradients: (fx, fy) pairs of T per subset pixel; then f - f0 in T
  t.off_fg = 0;
  t.off_f = al(2 * SS * static_cast<int>(sizeof(T)));
  t.off_win = al(t.off_f + SS * static_cast<int>(sizeof(T)));
  const int win_end = al(t.off_win + t.bxc * t.byc * static_cast<int>(sizeof(T)));
  // the gray tile is read only before the gradients are written: it shares their
  // region when it fits
  t.gray_alias = t.bxg * S * t.gray_es <= 2 * SS * static_cast<int>(sizeof(T));
  t.off_gray = t.gray_alias ? t.off_fg : win_end;
  t.smem_bytes = t.gray_alias ? win_end : al(win_end + t.bxg * S * t.gray_es);
  return t;
}

template <typename T>
cudaError_t launch_wave(const WaveArgs<T>& a, const WaveTiles& t, const CUtensorMap* maps, int nparams,
                        int grid, cudaStream_t s) {
  (void)t;
  switch (nparams) {
    case 2:
      return launch_wave_np<T, 2>(a, maps, grid, s);
    case 6:
      return launch_wave_np<T, 6>(a, maps, grid, s);
    default:
      return launch_wave_np<T, 12>(a, maps, grid, s);
  }
}

template <typename T>
int wave_blocks_per_sm(int nparams, int threads, int mode, size_t smem) {
  switch (nparams) {
    case 2:
      return blocks_per_sm_np<T, 2>(threads, mode, smem);
    case 6:
      return blocks_per_sm_np<T, 6>(threads, mode, smem);
    default:
      return blocks_per_sm_np<T, 12>(threads, mode, smem);
  }
}

cudaError_t launch_roi_flags(const RoiArgs& a, cudaStream_t s) {
  const int64_t n = static_cast<int64_t>(a.nx) * a.ny;
  const int64_t blocks = (n * 32 + 255) / 256;
  roi_flags_kernel<<<static_cast<unsigned>(blocks < 65535 ? blocks : 65535), 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_grid_points(int32_t* x, int32_t* y, int r, int step, int nx, int64_t n, cudaStream_t s) {
  const int64_t blocks = (n + 255) / 256;
  grid_points_kernel<<<static_cast<unsigned>(blocks < 8192 ? blocks : 8192), 256, 0, s>>>(x, y, r, step, nx, n);
  return cudaGetLastError();
}

cudaError_t launch_reset_points(const PointArrays& pa, int nparams, const uint8_t* roi_ok,
                                cudaStream_t s) {
  const int64_t blocks = (pa.n + 255) / 256;
  reset_points_kernel<<<static_cast<unsigned>(blocks < 8192 ? blocks : 8192), 256, 0, s>>>(
      pa, nparams, roi_ok);
  return cudaGetLastError();
}

cudaError_t launch_sequence_reset(const PointArrays& pa, int nparams, const uint8_t* roi_ok,
                                  int32_t* front0, int32_t* counters, cudaStream_t s) {
  const int64_t blocks = (pa.n + 255) / 256;
  sequence_reset_kernel<<<static_cast<unsigned>(blocks < 8192 ? blocks : 8192), 256, 0, s>>>(
      pa, nparams, roi_ok, front0, counters);
  return cudaGetLastError();
}

cudaError_t launch_finalize_points(const PointArrays& pa, int nparams, int nan_rejected,
                                   int32_t* accepted, cudaStream_t s) {
  const int64_t blocks = (pa.n + 255) / 256;
  finalize_points_kernel<<<static_cast<unsigned>(blocks < 8192 ? blocks : 8192), 256, 0, s>>>(
      pa, nparams, nan_rejected, accepted);
  return cudaGetLastError();
}

template WaveTiles wave_tiles<float>(int, int);
template WaveTiles wave_tiles<double>(int, int);
template cudaError_t launch_wave<float>(const WaveArgs<float>&, const WaveTiles&, const CUtensorMap*, int, int,
                                        cudaStream_t);
template cudaError_t launch_wave<double>(const WaveArgs<double>&, const WaveTiles&, const CUtensorMap*, int, int,
                                         cudaStream_t);
template int wave_blocks_per_sm<float>(int, int, int, size_t);
template int wave_blocks_per_sm<double>(int, int, int, size_t);

}  // namespace dic
