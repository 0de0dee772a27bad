// FFT pass kernels in FP32 (the mixed-precision products).
#include "fft_passes.cuh"

namespace sdft {
cudaError_t launch_pass_f32(int kind, bool inv, int E, const PassArgs& a, int threads, size_t smem, dim3 grid,
                            cudaStream_t st) {
  return launch_e<float>(kind, inv, E, a, threads, smem, grid, st);
}
}  // namespace sdft
