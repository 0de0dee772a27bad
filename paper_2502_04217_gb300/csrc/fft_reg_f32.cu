// Register-engine FFT pass kernels in FP32 (the mixed-precision products).
#include "fft_passes.cuh"

namespace sdft {
cudaError_t launch_reg_f32(int kind, bool inv, const PassArgs& a, int threads, size_t smem, dim3 grid,
                           cudaStream_t st) {
  return launch_reg<float>(kind, inv, a, threads, smem, grid, st);
}
}  // namespace sdft
