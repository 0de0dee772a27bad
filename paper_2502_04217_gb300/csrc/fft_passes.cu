// Launch of one FFT pass of G = M_perp^T M_perp (kernels: fft_passes.cuh and
// fft_reg.cuh; each engine's FP32 and FP64 instantiations are compiled as
// separate translation units).
#include "internal.h"

namespace sdft {

cudaError_t launch_pass_f32(int kind, bool inv, int E, const PassArgs& a, int threads, size_t smem, dim3 grid,
                            cudaStream_t st);
cudaError_t launch_pass_f64(int kind, bool inv, int E, const PassArgs& a, int threads, size_t smem, dim3 grid,
                            cudaStream_t st);
cudaError_t launch_reg_f32(int kind, bool inv, const PassArgs& a, int threads, size_t smem, dim3 grid,
                           cudaStream_t st);
cudaError_t launch_reg_f64(int kind, bool inv, const PassArgs& a, int threads, size_t smem, dim3 grid,
                           cudaStream_t st);

cudaError_t launch_pass(int kind, bool inv, bool fp32, int E, const PassArgs& a, int threads, size_t smem,
                        dim3 grid, cudaStream_t st) {
  if (a.reg)
    return fp32 ? launch_reg_f32(kind, inv, a, threads, smem, grid, st)
                : launch_reg_f64(kind, inv, a, threads, smem, grid, st);
  return fp32 ? launch_pass_f32(kind, inv, E, a, threads, smem, grid, st)
              : launch_pass_f64(kind, inv, E, a, threads, smem, grid, st);
}

}  // namespace sdft
