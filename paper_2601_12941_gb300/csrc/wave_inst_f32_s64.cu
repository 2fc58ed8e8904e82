// Instantiations of the wave kernel: FP32 coefficients and sums, kernel variant 3
// (Gauss-Newton with ZNSSD on the B-spline, with the Hessian inverse, the solve and
// the ZNCC normalisation in FP64: DIC_MIXED_FP64_SOLVE), every shape function and
// block size.
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

template cudaError_t launch_wave_inst<float, 2, 3>(const WaveArgs<float>&, const CUtensorMap*, int, cudaStream_t);
template int blocks_per_sm_inst<float, 2, 3>(int, size_t);
template cudaError_t launch_wave_inst<float, 6, 3>(const WaveArgs<float>&, const CUtensorMap*, int, cudaStream_t);
template int blocks_per_sm_inst<float, 6, 3>(int, size_t);
template cudaError_t launch_wave_inst<float, 12, 3>(const WaveArgs<float>&, const CUtensorMap*, int, cudaStream_t);
template int blocks_per_sm_inst<float, 12, 3>(int, size_t);

}  // namespace dic
