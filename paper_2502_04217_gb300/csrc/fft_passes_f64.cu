// FFT pass kernels in FP64.
#include "fft_passes.cuh"

namespace sdft {
cudaError_t launch_pass_f64(int kind, bool inv, int E, const PassArgs& a, int threads, size_t smem, dim3 grid,
                            cudaStream_t st) {
  return launch_e<double>(kind, inv, E, a, threads, smem, grid, st);
}
}  // namespace sdft
