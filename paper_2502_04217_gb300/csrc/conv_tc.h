// tcgen05 (5th-generation tensor core) 3x3x3 convolution of the warm-start
// network, channels last, zero padding (conv_tc.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace sdft {

struct ConvTcArgs {
  const __nv_bfloat16* x;     // [D0][D1][D2][cin]
  const __nv_bfloat16* w;     // [27][cout][cin], tap (a+1)*9 + (b+1)*3 + (c+1) for offset (a, b, c)
  const float* bias;          // [cout] or nullptr
  int D0, D1, D2;
  int relu;                   // max(0, .) on the output
  const __nv_bfloat16* aux;   // [V][cout] or nullptr: output *= (aux > 0)
  __nv_bfloat16* ybf;         // [V][cout] BF16 output (or nullptr)
  float* yf;                  // [V][cout] FP32 output (or nullptr)
  // failure-detection test only (zero otherwise): the producer of every CTA skips
  // the copy (and the barrier arrival) of its triple number drop_triple - 1, and
  // every pipeline wait gives up after 2^wait_log2 polls instead of 2^24
  int drop_triple;
  int wait_log2;
};

// Shapes the tensor-core kernel takes: (cin, cout) in {16, 32} x {8, 32} and
// at least 64 voxels along D2 (the tile is 128 voxels along D2).
bool conv_tc_supported(int cin, int cout, int D0, int D1, int D2);

// Launch on stream st; cudaErrorNotSupported for other shapes or when the
// driver offers no tensor-map encoder.
cudaError_t conv_tc(int cin, int cout, const ConvTcArgs& a, cudaStream_t st);

// After synchronising st: code of the first expired wait since the last call
// (0: none), then reset.
cudaError_t conv_tc_take_error(unsigned* code, cudaStream_t st);

// Failure-detection test: make the NEXT launch drop one copy (see ConvTcArgs).
void conv_tc_inject_stall(int drop_triple, int wait_log2);

}  // namespace sdft
