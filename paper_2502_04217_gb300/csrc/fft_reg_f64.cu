// Register-engine FFT pass kernels in FP64.
#include "fft_passes.cuh"

namespace sdft {
cudaError_t launch_reg_f64(int kind, bool inv, const PassArgs& a, int threads, size_t smem, dim3 grid,
                           cudaStream_t st) {
  return launch_reg<double>(kind, inv, a, threads, smem, grid, st);
}
}  // namespace sdft
