// Instantiations of the wave kernel: FP32, kernel variant 2 (0 Gauss-Newton with
// ZNSSD on the B-spline, 1 Gauss-Newton with any cost or interpolant, 2
// Levenberg-Marquardt), every shape function and block size.
#include "wave_kernel.cuh"

namespace dic {

template <typename T, int NP, int MODE>
cudaError_t launch_wave_inst(const WaveArgs<T>& a, const CUtensorMap* maps, int grid, cudaStream_t s) {
  return launch_wave_mode<T, NP, MODE>(a, maps, grid, s);
}

template <typename T, int NP, int MODE>
int blocks_per_sm_inst(int threads, size_t smem) {
  return threads == kWaveThreadsSmall ? blocks_per_sm_nt<T, NP, kWaveThreadsSmall, MODE>(smem)
                                      : blocks_per_sm_nt<T, NP, kWaveThreads, MODE>(smem);
}

template cudaError_t launch_wave_inst<float, 2, 2>(const WaveArgs<float>&, const CUtensorMap*, int, cudaStream_t);
template int blocks_per_sm_inst<float, 2, 2>(int, size_t);
template cudaError_t launch_wave_inst<float, 6, 2>(const WaveArgs<float>&, const CUtensorMap*, int, cudaStream_t);
template int blocks_per_sm_inst<float, 6, 2>(int, size_t);
template cudaError_t launch_wave_inst<float, 12, 2>(const WaveArgs<float>&, const CUtensorMap*, int, cudaStream_t);
template int blocks_per_sm_inst<float, 12, 2>(int, size_t);

}  // namespace dic
