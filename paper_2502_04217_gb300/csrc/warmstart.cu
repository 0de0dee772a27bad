// Learned warm start: a 4-layer 3D convolution network over the grid of
// half-spectrum slots predicts the solution beta and its support; the
// prediction is turned into a strictly interior, centred start point for the
// IPM.  The paper has no such component (it cold-starts MadNLP).
//
// Network (channels last, BF16 activations and weights, FP32 accumulation):
//   x (8 features, stored as 16 channels) -conv-> 32 -relu-> 32 -relu-> 32
//   -relu-> 4 outputs (stored as 8): y[0:2] corrects the soft-threshold guess
//   soft(c/lambda, 1) of the two beta coordinates of a slot, y[2:4] are the
//   logits of "coordinate is non-zero".
// Every convolution is 3x3x3 with zero padding over the slot grid
// (D0, D1, D2) = (Hl, N0, N1) in 3D, (Hl, 1, N0) in 2D, (Hl, 1, 1) in 1D, so the
// voxel index equals the slot index of the beta layout.
//
// Tensor cores: on grids with at least 64 voxels along D2 the convolutions run
// on tcgen05 (conv_tc.cu: TMA-staged lines, MMA into TMEM).  The kernels below
// use mma.sync m16n8k16 (BF16 in, FP32 accumulate) and serve the small grids
// and the weight gradient.  Forward: M = 64 voxels along D2 per block (16 per warp),
// N = output channels, K = 27 taps x input channels, input halo tile and all
// weights staged in shared memory.  The data gradient is the same kernel on the
// mirrored, channel-transposed weights with the ReLU mask of the layer input
// fused in its epilogue.  The weight gradient is a GEMM with K = voxels, taps
// split across 9 warps, per-block partials reduced in block order.
#include <cuda_bf16.h>

#include <cmath>
#include <string>
#include <vector>

#include "../../include/sdft_ipm.h"
#include "conv_tc.h"
#include "internal.h"
#include "kernels.h"

namespace sdft {
void record_error(const char* msg);
bool handle_view(sdft_ipm* h, HandleView* v);
void handle_point_set(sdft_ipm* h);
}

using namespace sdft;
using bf16 = __nv_bfloat16;

namespace {

constexpr int TZ = 64;       // output voxels per block along D2
constexpr int PADC = 8;      // shared-memory row padding (bf16 elements)
constexpr int kWgradWarps = 9;

__device__ __forceinline__ uint32_t ld32(const bf16* p) { return *reinterpret_cast<const uint32_t*>(p); }
__device__ __forceinline__ uint32_t pack2(bf16 lo, bf16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// D = A (16x16, row) * B (16x8, col) + D, BF16 inputs, FP32 accumulators
__device__ __forceinline__ void mma16816(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

struct ConvArgs {
  const bf16* x;        // [V][CIN]
  const bf16* w;        // [27][COUT][CIN], tap t = (a+1)*9 + (b+1)*3 + (c+1) for offset (a, b, c)
  const float* bias;    // [COUT] or nullptr
  int D0, D1, D2;
  int relu;             // max(0, .) on the output
  const bf16* aux;      // [V][COUT] or nullptr: output *= (aux > 0)
  bf16* ybf;            // [V][COUT] BF16 output, or
  float* yf;            // [V][COUT] FP32 output
};

// y[v, o] = bias[o] + sum_t sum_i x[v + off(t), i] w[t, o, i]
template <int CIN, int COUT>
__global__ void __launch_bounds__(128) conv_fwd_kernel(ConvArgs a) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  constexpr int RS = CIN + PADC;
  bf16* ws = reinterpret_cast<bf16*>(sm_raw);       // [27][COUT][RS]
  bf16* xs = ws + 27 * COUT * RS;                     // [9][TZ + 2][RS]
  const int z0 = blockIdx.x * TZ, i1 = blockIdx.y, i0 = blockIdx.z;
  constexpr int CH = CIN / 8;                         // 16-byte chunks per row
  for (int idx = threadIdx.x; idx < 27 * COUT * CH; idx += blockDim.x) {
    const int row = idx / CH, ch = idx - row * CH;
    *reinterpret_cast<uint4*>(ws + row * RS + ch * 8) = *reinterpret_cast<const uint4*>(a.w + (size_t)row * CIN + ch * 8);
  }
  for (int idx = threadIdx.x; idx < 9 * (TZ + 2) * CH; idx += blockDim.x) {
    const int ch = idx % CH, r = idx / CH;
    const int zz = r % (TZ + 2), ab = r / (TZ + 2);
    const int j0 = i0 + ab / 3 - 1, j1 = i1 + ab % 3 - 1, j2 = z0 + zz - 1;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (j0 >= 0 && j0 < a.D0 && j1 >= 0 && j1 < a.D1 && j2 >= 0 && j2 < a.D2)
      v = *reinterpret_cast<const uint4*>(a.x + ((size_t)(j0 * a.D1 + j1) * a.D2 + j2) * CIN + ch * 8);
    *reinterpret_cast<uint4*>(xs + r * RS + ch * 8) = v;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, tg = lane & 3;
  float acc[COUT / 8][4];
#pragma unroll
  for (int nt = 0; nt < COUT / 8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
  for (int t = 0; t < 27; ++t) {
    const int ta = t / 9, tb = (t / 3) % 3, tc = t % 3;
    const bf16* xr = xs + ((ta * 3 + tb) * (TZ + 2) + warp * 16 + tc) * RS;
#pragma unroll
    for (int kc = 0; kc < CIN / 16; ++kc) {
      const bf16* p = xr + kc * 16 + 2 * tg;
      const uint32_t a0 = ld32(p + g * RS), a1 = ld32(p + (g + 8) * RS);
      const uint32_t a2 = ld32(p + g * RS + 8), a3 = ld32(p + (g + 8) * RS + 8);
#pragma unroll
      for (int nt = 0; nt < COUT / 8; ++nt) {
        const bf16* wr = ws + (t * COUT + nt * 8 + g) * RS + kc * 16 + 2 * tg;
        mma16816(acc[nt], a0, a1, a2, a3, ld32(wr), ld32(wr + 8));
      }
    }
  }
#pragma unroll
  for (int nt = 0; nt < COUT / 8; ++nt) {
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      const int z = z0 + warp * 16 + g + 8 * hh;
      if (z >= a.D2) continue;
      const size_t v = (size_t)(i0 * a.D1 + i1) * a.D2 + z;
      const int co = nt * 8 + 2 * tg;
      float y0 = acc[nt][2 * hh], y1 = acc[nt][2 * hh + 1];
      if (a.bias) { y0 += a.bias[co]; y1 += a.bias[co + 1]; }
      if (a.relu) { y0 = fmaxf(y0, 0.f); y1 = fmaxf(y1, 0.f); }
      if (a.aux) {
        const bf16* ax = a.aux + v * COUT + co;
        if (!(__bfloat162float(ax[0]) > 0.f)) y0 = 0.f;
        if (!(__bfloat162float(ax[1]) > 0.f)) y1 = 0.f;
      }
      if (a.ybf) *reinterpret_cast<uint32_t*>(a.ybf + v * COUT + co) = pack2(__float2bfloat16_rn(y0), __float2bfloat16_rn(y1));
      if (a.yf) { a.yf[v * COUT + co] = y0; a.yf[v * COUT + co + 1] = y1; }
    }
  }
}

// Per-block partial weight gradient: part[b][t][m][i] = sum over the block's
// voxels v of dy[v][m] x[v + off(t)][i], for m < M (dy has M channels, M in {16, 32}).
template <int CIN, int M>
__global__ void __launch_bounds__(32 * kWgradWarps) conv_wgrad_kernel(const bf16* __restrict__ x, const bf16* __restrict__ dy,
                                                                     int D0, int D1, int D2, float* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  constexpr int RS = CIN + PADC, RD = M + PADC;
  bf16* xs = reinterpret_cast<bf16*>(sm_raw);         // [9][TZ + 2][RS]
  bf16* ds = xs + 9 * (TZ + 2) * RS;                  // [TZ][RD]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, tg = lane & 3;
  constexpr int MT = M / 16, NT = CIN / 8;
  float acc[3][MT][NT][4];
#pragma unroll
  for (int q = 0; q < 3; ++q)
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) acc[q][mt][nt][0] = acc[q][mt][nt][1] = acc[q][mt][nt][2] = acc[q][mt][nt][3] = 0.f;
  const int ztiles = (D2 + TZ - 1) / TZ;
  const long long ntiles = (long long)D0 * D1 * ztiles;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int zt = (int)(tile % ztiles);
    const long long row = tile / ztiles;
    const int i1 = (int)(row % D1), i0 = (int)(row / D1);
    const int z0 = zt * TZ;
    __syncthreads();
    constexpr int CH = CIN / 8, CHD = M / 8;
    for (int idx = threadIdx.x; idx < 9 * (TZ + 2) * CH; idx += blockDim.x) {
      const int ch = idx % CH, r = idx / CH;
      const int zz = r % (TZ + 2), ab = r / (TZ + 2);
      const int j0 = i0 + ab / 3 - 1, j1 = i1 + ab % 3 - 1, j2 = z0 + zz - 1;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (j0 >= 0 && j0 < D0 && j1 >= 0 && j1 < D1 && j2 >= 0 && j2 < D2)
        v = *reinterpret_cast<const uint4*>(x + ((size_t)(j0 * D1 + j1) * D2 + j2) * CIN + ch * 8);
      *reinterpret_cast<uint4*>(xs + r * RS + ch * 8) = v;
    }
    for (int idx = threadIdx.x; idx < TZ * CHD; idx += blockDim.x) {
      const int ch = idx % CHD, zz = idx / CHD;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (z0 + zz < D2) v = *reinterpret_cast<const uint4*>(dy + ((size_t)(i0 * D1 + i1) * D2 + z0 + zz) * M + ch * 8);
      *reinterpret_cast<uint4*>(ds + zz * RD + ch * 8) = v;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const int t = warp + kWgradWarps * q;
      const int ta = t / 9, tb = (t / 3) % 3, tc = t % 3;
      const bf16* xr = xs + ((ta * 3 + tb) * (TZ + 2) + tc) * RS;
#pragma unroll
      for (int kc = 0; kc < TZ / 16; ++kc) {
        const int k0 = kc * 16 + 2 * tg;              // voxel (K) index of this thread's first pair
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) {
          const int m0 = mt * 16 + g;
          const uint32_t a0 = pack2(ds[k0 * RD + m0], ds[(k0 + 1) * RD + m0]);
          const uint32_t a1 = pack2(ds[k0 * RD + m0 + 8], ds[(k0 + 1) * RD + m0 + 8]);
          const uint32_t a2 = pack2(ds[(k0 + 8) * RD + m0], ds[(k0 + 9) * RD + m0]);
          const uint32_t a3 = pack2(ds[(k0 + 8) * RD + m0 + 8], ds[(k0 + 9) * RD + m0 + 8]);
#pragma unroll
          for (int nt = 0; nt < NT; ++nt) {
            const int n0 = nt * 8 + g;
            const uint32_t b0 = pack2(xr[k0 * RS + n0], xr[(k0 + 1) * RS + n0]);
            const uint32_t b1 = pack2(xr[(k0 + 8) * RS + n0], xr[(k0 + 9) * RS + n0]);
            mma16816(acc[q][mt][nt], a0, a1, a2, a3, b0, b1);
          }
        }
      }
    }
  }
  float* out = part + (size_t)blockIdx.x * 27 * M * CIN;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const int t = warp + kWgradWarps * q;
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        const int m = mt * 16 + g, i = nt * 8 + 2 * tg;
        out[((size_t)t * M + m) * CIN + i] = acc[q][mt][nt][0];
        out[((size_t)t * M + m) * CIN + i + 1] = acc[q][mt][nt][1];
        out[((size_t)t * M + m + 8) * CIN + i] = acc[q][mt][nt][2];
        out[((size_t)t * M + m + 8) * CIN + i + 1] = acc[q][mt][nt][3];
      }
  }
}

// dW[t][m][i] (m < mout) = sum of the block partials in block order; writes into grad (FP32, [27][mout][CIN])
__global__ void wgrad_reduce_kernel(const float* __restrict__ part, int nblocks, int M, int CIN, int mout,
                                    float* __restrict__ grad) {
  const int total = 27 * mout * CIN;
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < total; o += gridDim.x * blockDim.x) {
    const int i = o % CIN, m = (o / CIN) % mout, t = o / (CIN * mout);
    const size_t src = ((size_t)t * M + m) * CIN + i;
    float s = 0.f;
    for (int b = 0; b < nblocks; ++b) s += part[(size_t)b * 27 * M * CIN + src];
    grad[o] = s;
  }
}

// db[m] = sum_v dy[v][m], m < mout: per-block partials, then block-ordered sum
__global__ void bgrad_kernel(const bf16* __restrict__ dy, long long V, int M, int mout, float* __restrict__ part) {
  __shared__ float sh[32][33];
  const int m = threadIdx.x & 31, lane_v = threadIdx.x >> 5;       // 32 channels x 8 voxel lanes
  float s = 0.f;
  if (m < mout)
    for (long long v = (long long)blockIdx.x * 8 + lane_v; v < V; v += (long long)gridDim.x * 8)
      s += __bfloat162float(dy[v * M + m]);
  sh[lane_v][m] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    float t = 0.f;
    for (int k = 0; k < 8; ++k) t += sh[k][threadIdx.x];
    part[(size_t)blockIdx.x * 32 + threadIdx.x] = t;
  }
}

__global__ void bgrad_reduce_kernel(const float* __restrict__ part, int nblocks, int mout, float* __restrict__ db) {
  const int m = threadIdx.x;
  if (m >= mout) return;
  float s = 0.f;
  for (int b = 0; b < nblocks; ++b) s += part[(size_t)b * 32 + m];
  db[m] = s;
}

__device__ __forceinline__ double soft1(double u) { return u > 1.0 ? u - 1.0 : (u < -1.0 ? u + 1.0 : 0.0); }

__device__ __forceinline__ float soft1f(float u) { return u > 1.f ? u - 1.f : (u < -1.f ? u + 1.f : 0.f); }

// Input features of every slot (16 channels, 8 used), from c = M_perp^T b and lambda.
// They feed BF16 convolutions, so they are formed in FP32 (the FP64 operands converted
// on the integer pipe, the slot's grid indices by the layout's multiply-high divisions):
// nothing of this kernel runs on the FP64 pipe.
__global__ void features_kernel(Layout lay, const double* __restrict__ c, const DevScalars* sc, bf16* __restrict__ x) {
  const float il = d2f_int(1.0 / sc->lambda);
  const int D1 = lay.d == 3 ? lay.N0 : 1, D2 = lay.d == 3 ? lay.N1 : (lay.d == 2 ? lay.N0 : 1);
  const float sl = lay.Hl > 1 ? 1.f / (float)(lay.Hl - 1) : 0.f, s1 = 2.f / (float)D1, s2 = 2.f / (float)D2;
  const double2* c2 = reinterpret_cast<const double2*>(c);
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < lay.H; s += (long long)gridDim.x * blockDim.x) {
    const double2 cv = c2[s];
    const float c0 = d2f_int(cv.x) * il, c1 = d2f_int(cv.y) * il;
    // slot = kl * M + k' with k' = k1 * D2 + k2 (k1 = 0 for d < 3; H < 2^31)
    const unsigned su = (unsigned)s;
    const int kl = (int)fast_div(su, lay.divM);
    const int kp = (int)(su - (unsigned)kl * (unsigned)lay.M);
    const int k1 = lay.d == 3 ? (int)fast_div((unsigned)kp, lay.divN1) : 0;
    const int k2 = lay.d == 3 ? kp - k1 * lay.N1 : (lay.d == 2 ? kp : 0);
    const float f0 = lay.d == 3 ? (float)min(k1, lay.N0 - k1) * s1 : 0.f;
    const float f1 = lay.d >= 2 ? (float)min(k2, D2 - k2) * s2 : 0.f;
    float f[8] = {c0, c1, soft1f(c0), soft1f(c1), sqrtf(c0 * c0 + c1 * c1), (float)kl * sl, f0, f1};
    uint32_t w[8];
#pragma unroll
    for (int k = 0; k < 4; ++k) w[k] = pack2(__float2bfloat16_rn(f[2 * k]), __float2bfloat16_rn(f[2 * k + 1]));
#pragma unroll
    for (int k = 4; k < 8; ++k) w[k] = 0u;
    uint4* dst = reinterpret_cast<uint4*>(x + s * 16);
    dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
    dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
  }
}

// Loss of the outputs y (FP32 [V][8], 4 used) against beta* and its gradient dy
// (BF16 [V][16], 4 used):  mean over LASSO coordinates of (y_c - t_c)^2 with
// t_c = beta*_c / lambda - soft(c_c / lambda, 1), plus 0.1 x mean cross-entropy of
// the logits y_{2+c} against 1[|beta*_c| > 1e-6 lambda].
__global__ void loss_kernel(Layout lay, const float* __restrict__ y, const double* __restrict__ c,
                            const double* __restrict__ bstar, const DevScalars* sc, bf16* __restrict__ dy,
                            double* partials, unsigned* counter, double* loss_out) {
  __shared__ double scratch[64];
  const double lam = sc->lambda, il = 1.0 / lam, inv_n = 1.0 / (double)lay.n;
  double v[2] = {0.0, 0.0};
  const int ops[2] = {RED_SUM, RED_SUM};
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < lay.H; s += (long long)gridDim.x * blockDim.x) {
    float g[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int cc = 0; cc < 2; ++cc) {
      const long long i = 2 * s + cc;
      if (is_ghost(lay, i)) continue;
      const double t = bstar[i] * il - soft1(c[i] * il);
      const double d = (double)y[s * 8 + cc] - t;
      const double sup = fabs(bstar[i]) > 1e-6 * lam ? 1.0 : 0.0;
      const double lg = (double)y[s * 8 + 2 + cc];
      const double sp = lg > 0 ? lg + log1p(exp(-lg)) : log1p(exp(lg));     // softplus
      v[0] += d * d;
      v[1] += sp - sup * lg;
      g[cc] = (float)(2.0 * d * inv_n);
      g[2 + cc] = (float)(0.1 * (1.0 / (1.0 + exp(-lg)) - sup) * inv_n);
    }
    uint4* dst = reinterpret_cast<uint4*>(dy + s * 16);
    dst[0] = make_uint4(pack2(__float2bfloat16_rn(g[0]), __float2bfloat16_rn(g[1])),
                        pack2(__float2bfloat16_rn(g[2]), __float2bfloat16_rn(g[3])), 0u, 0u);
    dst[1] = make_uint4(0u, 0u, 0u, 0u);
  }
  if (grid_reduce<2>(v, ops, partials, counter, scratch) && threadIdx.x == 0)
    *loss_out = (v[0] + 0.1 * v[1]) * inv_n;
}

// Start point from the prediction: beta0 = lambda (soft(c/lambda) + y[0:2]),
// p = sigmoid(y[2:4]); z = |beta0| + delta with delta = (mu0 / lambda)(2 - p);
// s1 = z + beta0, s2 = z - beta0, nu_i = mu0 / s_i.  A coordinate predicted
// inactive gets s1 = s2 = 2 mu0/lambda and nu1 = nu2 = lambda/2 (feasible and
// centred); an active one gets its small slack mu0/lambda with multiplier
// lambda.  Every s_i nu_i equals mu0 (to the Newton reciprocal's 1.4e-14).  The
// sigmoid only shapes the margin delta in [mu0/lambda, 2 mu0/lambda] and is
// evaluated in FP32 (z, s within 1.2e-7 mu0/lambda of an FP64 evaluation).
__global__ void point_kernel(Layout lay, const float* __restrict__ y, const double* __restrict__ c, const DevScalars* sc,
                             double mu_scale, IpmVectors w) {
  const double lam = sc->lambda, il = 1.0 / lam;
  const double mu0 = mu_scale * lam * lam;
  const long long n2 = 2 * lay.H;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n2; i += (long long)gridDim.x * blockDim.x) {
    if (is_ghost(lay, i)) {
      w.beta[i] = 0.0; w.z[i] = 0.0; w.s1[i] = 0.0; w.s2[i] = 0.0; w.nu1[i] = 0.0; w.nu2[i] = 0.0;
      continue;
    }
    const long long s = i >> 1;
    const int cc = (int)(i & 1);
    const double b0 = lam * (soft1(c[i] * il) + (double)y[s * 8 + cc]);
    const float p = 1.0f / (1.0f + expf(-y[s * 8 + 2 + cc]));
    const double z = fabs(b0) + (mu0 * il) * (2.0 - f2d_int(p));
    const double s1 = z + b0, s2 = z - b0;
    w.beta[i] = b0;
    w.z[i] = z;
    w.s1[i] = s1;
    w.s2[i] = s2;
    w.nu1[i] = mu0 * rcp1(s1);
    w.nu2[i] = mu0 * rcp1(s2);
  }
}

// Adam on the FP32 master parameters, then the BF16 copies used by the kernels:
// forward weights [27][COUT][CIN] and, for the data gradient, the mirrored taps
// with channels swapped [27][CIN][COUT_b] (COUT_b >= COUT, extra columns 0).
struct LayerDesc {
  int cin, cout;          // stored (padded) channel counts of the forward conv
  int cin_real, cout_real;
  long long w_off, b_off; // offsets in the parameter vector
  long long wf_off;       // offset of the forward BF16 weights
  long long wb_off;       // offset of the backward BF16 weights (-1: none)
  int cout_b;             // padded input channels of the backward conv (= channels of dy)
};

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                            long long n, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
  }
}

__global__ void pack_weights_kernel(const float* __restrict__ p, LayerDesc L, bf16* __restrict__ wf, bf16* __restrict__ wb) {
  const long long total = 27LL * L.cout * L.cin;
  for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < total; o += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(o % L.cin), co = (int)((o / L.cin) % L.cout), t = (int)(o / ((long long)L.cin * L.cout));
    const float val = p[L.w_off + o];
    wf[L.wf_off + o] = __float2bfloat16_rn(val);
    if (L.wb_off >= 0) {
      // backward weights: tap 26 - t, out channel i (forward input), in channel co (forward output)
      wb[L.wb_off + ((long long)(26 - t) * L.cin + i) * L.cout_b + co] = __float2bfloat16_rn(val);
    }
  }
}

// counter-based initialisation: He-uniform from a 64-bit mix of (seed, index)
__device__ __forceinline__ float hash_uniform(unsigned long long seed, unsigned long long i) {
  unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (i + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (float)((z >> 11) * (1.0 / 9007199254740992.0));
}

__global__ void init_params_kernel(float* p, LayerDesc L, unsigned long long seed, float scale) {
  const long long total = 27LL * L.cout * L.cin;
  const float bound = scale * sqrtf(6.f / (27.f * L.cin_real));
  for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < total; o += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(o % L.cin), co = (int)((o / L.cin) % L.cout);
    const bool real = i < L.cin_real && co < L.cout_real;
    p[L.w_off + o] = real ? bound * (2.f * hash_uniform(seed, (unsigned long long)(L.w_off + o)) - 1.f) : 0.f;
  }
  for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < L.cout; o += (long long)gridDim.x * blockDim.x)
    p[L.b_off + o] = 0.f;
}

int blocks_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  if (b > 152 * 16) b = 152 * 16;
  return (int)(b < 1 ? 1 : b);
}

template <int CIN, int COUT>
cudaError_t conv_fwd(const ConvArgs& a, cudaStream_t st) {
  const size_t smem = (size_t)(27 * COUT + 9 * (TZ + 2)) * (CIN + PADC) * sizeof(bf16);
  cudaError_t e = cudaFuncSetAttribute(conv_fwd_kernel<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((a.D2 + TZ - 1) / TZ, a.D1, a.D0);
  conv_fwd_kernel<CIN, COUT><<<grid, 128, smem, st>>>(a);
  return cudaGetLastError();
}

// The tcgen05 kernel (conv_tc.cu) takes every layer shape once D2 >= 64; the
// mma.sync kernel above covers the small grids.
cudaError_t conv_fwd_any(int cin, int cout, const ConvArgs& a, cudaStream_t st) {
  if (conv_tc_supported(cin, cout, a.D0, a.D1, a.D2)) {
    const ConvTcArgs t{a.x, a.w, a.bias, a.D0, a.D1, a.D2, a.relu, a.aux, a.ybf, a.yf};
    const cudaError_t e = conv_tc(cin, cout, t, st);
    if (e != cudaErrorNotSupported) return e;
  }
  if (cin == 16 && cout == 32) return conv_fwd<16, 32>(a, st);
  if (cin == 32 && cout == 32) return conv_fwd<32, 32>(a, st);
  if (cin == 32 && cout == 8) return conv_fwd<32, 8>(a, st);
  if (cin == 16 && cout == 8) return conv_fwd<16, 8>(a, st);
  return cudaErrorInvalidValue;
}

constexpr int kWgradBlocks = 2 * 152;

template <int CIN, int M>
cudaError_t conv_wgrad(const bf16* x, const bf16* dy, int D0, int D1, int D2, float* part, cudaStream_t st) {
  const size_t smem = ((size_t)9 * (TZ + 2) * (CIN + PADC) + (size_t)TZ * (M + PADC)) * sizeof(bf16);
  cudaError_t e = cudaFuncSetAttribute(conv_wgrad_kernel<CIN, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  conv_wgrad_kernel<CIN, M><<<kWgradBlocks, 32 * kWgradWarps, smem, st>>>(x, dy, D0, D1, D2, part);
  return cudaGetLastError();
}

cudaError_t conv_wgrad_any(int cin, int m, const bf16* x, const bf16* dy, int D0, int D1, int D2, float* part,
                           cudaStream_t st) {
  if (cin == 16 && m == 32) return conv_wgrad<16, 32>(x, dy, D0, D1, D2, part, st);
  if (cin == 32 && m == 32) return conv_wgrad<32, 32>(x, dy, D0, D1, D2, part, st);
  if (cin == 32 && m == 16) return conv_wgrad<32, 16>(x, dy, D0, D1, D2, part, st);
  if (cin == 16 && m == 16) return conv_wgrad<16, 16>(x, dy, D0, D1, D2, part, st);
  return cudaErrorInvalidValue;
}

}  // namespace

// ---------------------------------------------------------------------------
// The network object
// ---------------------------------------------------------------------------
struct sdft_ws {
  cudaStream_t st = nullptr;
  LayerDesc L[4];
  long long nparams = 0, nwf = 0, nwb = 0;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  bf16 *wf = nullptr, *wb = nullptr;
  int steps = 0;
  // activations, sized for the largest grid seen
  long long cap = 0;
  bf16 *x0 = nullptr, *h1 = nullptr, *h2 = nullptr, *h3 = nullptr, *dy4 = nullptr, *da = nullptr, *db = nullptr;
  float* y = nullptr;
  float* wpart = nullptr;
  float* bpart = nullptr;
  double* dsc = nullptr;        // [0] loss; partials follow
  double* partials = nullptr;
  unsigned* counter = nullptr;
  std::vector<void*> allocs;
};

namespace {

template <typename T>
cudaError_t walloc(sdft_ws* n, T** p, size_t bytes) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, bytes ? bytes : 16);
  if (e == cudaSuccess) { n->allocs.push_back(q); *p = (T*)q; }
  return e;
}

ipm_status ws_err(const std::string& m, ipm_status s) {
  record_error(m.c_str());
  return s;
}

#define CKW(call)                                                                                    \
  do {                                                                                               \
    cudaError_t e_ = (call);                                                                         \
    if (e_ != cudaSuccess) return ws_err(std::string(#call) + ": " + cudaGetErrorString(e_),         \
                                         e_ == cudaErrorMemoryAllocation ? IPM_ERR_OOM : IPM_ERR_CUDA); \
  } while (0)

ipm_status ensure_capacity(sdft_ws* n, long long V) {
  if (V <= n->cap) return IPM_OK;
  for (void** p : {(void**)&n->x0, (void**)&n->h1, (void**)&n->h2, (void**)&n->h3, (void**)&n->dy4, (void**)&n->da,
                   (void**)&n->db, (void**)&n->y})
    if (*p) {
      cudaFree(*p);
      for (auto& a : n->allocs)
        if (a == *p) a = nullptr;
      *p = nullptr;
    }
  CKW(walloc(n, &n->x0, (size_t)V * 16 * sizeof(bf16)));
  CKW(walloc(n, &n->h1, (size_t)V * 32 * sizeof(bf16)));
  CKW(walloc(n, &n->h2, (size_t)V * 32 * sizeof(bf16)));
  CKW(walloc(n, &n->h3, (size_t)V * 32 * sizeof(bf16)));
  CKW(walloc(n, &n->dy4, (size_t)V * 16 * sizeof(bf16)));
  CKW(walloc(n, &n->da, (size_t)V * 32 * sizeof(bf16)));
  CKW(walloc(n, &n->db, (size_t)V * 32 * sizeof(bf16)));
  CKW(walloc(n, &n->y, (size_t)V * 8 * sizeof(float)));
  n->cap = V;
  return IPM_OK;
}

void grid_dims(const Layout& lay, int& D0, int& D1, int& D2) {
  D0 = lay.Hl;
  D1 = lay.d == 3 ? lay.N0 : 1;
  D2 = lay.d == 3 ? lay.N1 : (lay.d == 2 ? lay.N0 : 1);
}

ipm_status repack(sdft_ws* n) {
  CKW(cudaMemsetAsync(n->wb, 0, (size_t)n->nwb * sizeof(bf16), n->st));
  for (int l = 0; l < 4; ++l) {
    const long long tot = 27LL * n->L[l].cout * n->L[l].cin;
    pack_weights_kernel<<<blocks_for(tot, 256), 256, 0, n->st>>>(n->p, n->L[l], n->wf, n->wb);
    CKW(cudaGetLastError());
  }
  return IPM_OK;
}

// Synchronise st, then report an expired pipeline wait of the tensor-core convolution.
ipm_status sync_check(cudaStream_t st) {
  unsigned code = 0;
  CKW(conv_tc_take_error(&code, st));
  if (code)
    return ws_err("tensor-core convolution: a pipeline wait expired (code " + std::to_string(code) + ")",
                  IPM_TIMEOUT);
  return IPM_OK;
}

// Forward pass on the handle's c: features -> 4 convolutions -> y (FP32 [V][8]).
ipm_status forward(sdft_ws* n, const HandleView& hv) {
  int D0, D1, D2;
  grid_dims(hv.lay, D0, D1, D2);
  ipm_status s = ensure_capacity(n, hv.lay.H);
  if (s != IPM_OK) return s;
  features_kernel<<<blocks_for(hv.lay.H, 256), 256, 0, n->st>>>(hv.lay, hv.w.c, hv.sc, n->x0);
  CKW(cudaGetLastError());
  const bf16* in[4] = {n->x0, n->h1, n->h2, n->h3};
  bf16* out[3] = {n->h1, n->h2, n->h3};
  for (int l = 0; l < 4; ++l) {
    const LayerDesc& L = n->L[l];
    ConvArgs a{};
    a.x = in[l];
    a.w = n->wf + L.wf_off;
    a.bias = n->p + L.b_off;
    a.D0 = D0; a.D1 = D1; a.D2 = D2;
    a.relu = l < 3;
    if (l < 3) a.ybf = out[l]; else a.yf = n->y;
    CKW(conv_fwd_any(L.cin, L.cout, a, n->st));
  }
  return IPM_OK;
}

ipm_status layer_grads(sdft_ws* n, int l, const bf16* x, const bf16* dy, int dyC, int D0, int D1, int D2, long long V) {
  const LayerDesc& L = n->L[l];
  CKW(conv_wgrad_any(L.cin, dyC, x, dy, D0, D1, D2, n->wpart, n->st));
  wgrad_reduce_kernel<<<blocks_for(27LL * L.cout * L.cin, 256), 256, 0, n->st>>>(n->wpart, kWgradBlocks, dyC, L.cin,
                                                                                 L.cout, n->g + L.w_off);
  CKW(cudaGetLastError());
  bgrad_kernel<<<kWgradBlocks, 256, 0, n->st>>>(dy, V, dyC, L.cout, n->bpart);
  CKW(cudaGetLastError());
  bgrad_reduce_kernel<<<1, 32, 0, n->st>>>(n->bpart, kWgradBlocks, L.cout, n->g + L.b_off);
  CKW(cudaGetLastError());
  return IPM_OK;
}

}  // namespace

extern "C" {

ipm_status ws_create(sdft_ws** out, uint64_t seed, void* stream) {
  if (!out) return ws_err("ws_create: out must not be NULL", IPM_ERR_ARG);
  *out = nullptr;
  sdft_ws* n = new sdft_ws();
  n->st = (cudaStream_t)stream;
  const int cin[4] = {16, 32, 32, 32}, cout[4] = {32, 32, 32, 8};
  const int cin_r[4] = {8, 32, 32, 32}, cout_r[4] = {32, 32, 32, 4};
  const int cout_b[4] = {0, 32, 32, 16};
  long long po = 0, fo = 0, bo = 0;
  for (int l = 0; l < 4; ++l) {
    LayerDesc& L = n->L[l];
    L.cin = cin[l]; L.cout = cout[l]; L.cin_real = cin_r[l]; L.cout_real = cout_r[l];
    L.w_off = po; po += 27LL * L.cout * L.cin;
    L.b_off = po; po += L.cout;
    L.wf_off = fo; fo += 27LL * L.cout * L.cin;
    L.cout_b = cout_b[l];
    if (l > 0) { L.wb_off = bo; bo += 27LL * L.cin * L.cout_b; } else { L.wb_off = -1; }
  }
  n->nparams = po; n->nwf = fo; n->nwb = bo;
  auto fail = [&](ipm_status s) { ws_destroy(n); return s; };
#define CKC(call) do { cudaError_t e_ = (call); if (e_ != cudaSuccess) { \
    ws_err(std::string(#call) + ": " + cudaGetErrorString(e_), IPM_ERR_CUDA); return fail(IPM_ERR_CUDA); } } while (0)
  CKC(walloc(n, &n->p, po * sizeof(float)));
  CKC(walloc(n, &n->g, po * sizeof(float)));
  CKC(walloc(n, &n->m, po * sizeof(float)));
  CKC(walloc(n, &n->v, po * sizeof(float)));
  CKC(walloc(n, &n->wf, fo * sizeof(bf16)));
  CKC(walloc(n, &n->wb, bo * sizeof(bf16)));
  CKC(walloc(n, &n->wpart, (size_t)kWgradBlocks * 27 * 32 * 32 * sizeof(float)));
  CKC(walloc(n, &n->bpart, (size_t)kWgradBlocks * 32 * sizeof(float)));
  CKC(walloc(n, &n->dsc, 8 * sizeof(double)));
  CKC(walloc(n, &n->partials, 2 * 152 * 16 * sizeof(double)));
  CKC(walloc(n, &n->counter, 16 * sizeof(unsigned)));
  CKC(cudaMemsetAsync(n->counter, 0, 16 * sizeof(unsigned), n->st));
  CKC(cudaMemsetAsync(n->g, 0, po * sizeof(float), n->st));
  CKC(cudaMemsetAsync(n->m, 0, po * sizeof(float), n->st));
  CKC(cudaMemsetAsync(n->v, 0, po * sizeof(float), n->st));
  for (int l = 0; l < 4; ++l) {
    init_params_kernel<<<blocks_for(27LL * n->L[l].cout * n->L[l].cin, 256), 256, 0, n->st>>>(
        n->p, n->L[l], (unsigned long long)seed, l == 3 ? 0.1f : 1.0f);
    CKC(cudaGetLastError());
  }
#undef CKC
  ipm_status s = repack(n);
  if (s != IPM_OK) return fail(s);
  *out = n;
  return IPM_OK;
}

void ws_destroy(sdft_ws* n) {
  if (!n) return;
  if (n->st) cudaStreamSynchronize(n->st); else cudaDeviceSynchronize();
  for (void* p : n->allocs)
    if (p) cudaFree(p);
  delete n;
}

int64_t ws_num_params(const sdft_ws* n) { return n ? n->nparams : 0; }

ipm_status ws_get_params(sdft_ws* n, float* dst) {
  if (!n || !dst) return ws_err("ws_get_params: NULL argument", IPM_ERR_ARG);
  CKW(cudaMemcpyAsync(dst, n->p, n->nparams * sizeof(float), cudaMemcpyDefault, n->st));
  CKW(cudaStreamSynchronize(n->st));
  return IPM_OK;
}

ipm_status ws_get_grads(sdft_ws* n, float* dst) {
  if (!n || !dst) return ws_err("ws_get_grads: NULL argument", IPM_ERR_ARG);
  CKW(cudaMemcpyAsync(dst, n->g, n->nparams * sizeof(float), cudaMemcpyDefault, n->st));
  CKW(cudaStreamSynchronize(n->st));
  return IPM_OK;
}

ipm_status ws_set_params(sdft_ws* n, const float* src) {
  if (!n || !src) return ws_err("ws_set_params: NULL argument", IPM_ERR_ARG);
  CKW(cudaMemcpyAsync(n->p, src, n->nparams * sizeof(float), cudaMemcpyDefault, n->st));
  ipm_status s = repack(n);
  if (s != IPM_OK) return s;
  CKW(cudaStreamSynchronize(n->st));
  return IPM_OK;
}

ipm_status ws_forward(sdft_ws* n, sdft_ipm* h, float* y) {
  HandleView hv;
  if (!n || !handle_view(h, &hv)) return ws_err("ws_forward: NULL argument", IPM_ERR_ARG);
  ipm_status s = forward(n, hv);
  if (s != IPM_OK) return s;
  if (y) CKW(cudaMemcpyAsync(y, n->y, (size_t)hv.lay.H * 8 * sizeof(float), cudaMemcpyDefault, n->st));
  return sync_check(n->st);
}

ipm_status ws_predict(sdft_ws* n, sdft_ipm* h, double mu_scale) {
  HandleView hv;
  if (!n || !handle_view(h, &hv)) return ws_err("ws_predict: NULL argument", IPM_ERR_ARG);
  if (!(mu_scale > 0)) return ws_err("ws_predict: mu_scale must be positive", IPM_ERR_ARG);
  ipm_status s = forward(n, hv);
  if (s != IPM_OK) return s;
  point_kernel<<<blocks_for(2 * hv.lay.H, 256), 256, 0, n->st>>>(hv.lay, n->y, hv.w.c, hv.sc, mu_scale, hv.w);
  CKW(cudaGetLastError());
  if ((s = sync_check(n->st)) != IPM_OK) return s;
  handle_point_set(h);
  return IPM_OK;
}

ipm_status ws_train_step(sdft_ws* n, sdft_ipm* h, const double* beta_star, float lr, double* loss) {
  HandleView hv;
  if (!n || !beta_star || !handle_view(h, &hv)) return ws_err("ws_train_step: NULL argument", IPM_ERR_ARG);
  int D0, D1, D2;
  grid_dims(hv.lay, D0, D1, D2);
  const long long V = hv.lay.H;
  ipm_status s = forward(n, hv);
  if (s != IPM_OK) return s;
  loss_kernel<<<blocks_for(V, 256), 256, 0, n->st>>>(hv.lay, n->y, hv.w.c, beta_star, hv.sc, n->dy4, n->partials,
                                                    n->counter, n->dsc);
  CKW(cudaGetLastError());
  // layer 4: input h3, output gradient dy4 (16 channels, 4 used)
  if ((s = layer_grads(n, 3, n->h3, n->dy4, 16, D0, D1, D2, V)) != IPM_OK) return s;
  ConvArgs a{};
  a.D0 = D0; a.D1 = D1; a.D2 = D2;
  a.x = n->dy4; a.w = n->wb + n->L[3].wb_off; a.aux = n->h3; a.ybf = n->da;
  CKW(conv_fwd_any(16, 32, a, n->st));                                   // dh3 = (dy4 * W4^T) relu'(h3)
  if ((s = layer_grads(n, 2, n->h2, n->da, 32, D0, D1, D2, V)) != IPM_OK) return s;
  a.x = n->da; a.w = n->wb + n->L[2].wb_off; a.aux = n->h2; a.ybf = n->db;
  CKW(conv_fwd_any(32, 32, a, n->st));                                   // dh2
  if ((s = layer_grads(n, 1, n->h1, n->db, 32, D0, D1, D2, V)) != IPM_OK) return s;
  a.x = n->db; a.w = n->wb + n->L[1].wb_off; a.aux = n->h1; a.ybf = n->da;
  CKW(conv_fwd_any(32, 32, a, n->st));                                   // dh1
  if ((s = layer_grads(n, 0, n->x0, n->da, 32, D0, D1, D2, V)) != IPM_OK) return s;
  if (lr > 0.f) {
    n->steps += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f / (1.f - powf(b1, (float)n->steps)), c2 = 1.f / (1.f - powf(b2, (float)n->steps));
    adam_kernel<<<blocks_for(n->nparams, 256), 256, 0, n->st>>>(n->p, n->g, n->m, n->v, n->nparams, lr, b1, b2, 1e-8f,
                                                                c1, c2);
    CKW(cudaGetLastError());
    if ((s = repack(n)) != IPM_OK) return s;
  }
  if (loss) CKW(cudaMemcpyAsync(loss, n->dsc, sizeof(double), cudaMemcpyDeviceToHost, n->st));
  return sync_check(n->st);
}

// Low-level kernels on caller buffers (checked against the CPU reference by the tests).
ipm_status ws_conv_forward(int cin, int cout, int d0, int d1, int d2, const uint16_t* x, const uint16_t* w,
                           const float* bias, int relu, const uint16_t* aux, float* y, void* stream) {
  if (!x || !w || !y || d0 < 1 || d1 < 1 || d2 < 1) return ws_err("ws_conv_forward: bad argument", IPM_ERR_ARG);
  ConvArgs a{};
  a.x = (const bf16*)x; a.w = (const bf16*)w; a.bias = bias; a.relu = relu; a.aux = (const bf16*)aux; a.yf = y;
  a.D0 = d0; a.D1 = d1; a.D2 = d2;
  cudaError_t e = conv_fwd_any(cin, cout, a, (cudaStream_t)stream);
  if (e == cudaErrorInvalidValue) return ws_err("ws_conv_forward: channels must be (16|32, 8|32)", IPM_ERR_ARG);
  if (e != cudaSuccess) return ws_err(cudaGetErrorString(e), IPM_ERR_CUDA);
  return sync_check((cudaStream_t)stream);
}

ipm_status ws_test_conv_stall(int drop_triple, int wait_log2) {
  if (drop_triple < 1 || wait_log2 < 8 || wait_log2 > 24) return ws_err("ws_test_conv_stall: bad argument", IPM_ERR_ARG);
  conv_tc_inject_stall(drop_triple, wait_log2);
  return IPM_OK;
}

ipm_status ws_conv_wgrad(int cin, int m, int mout, int d0, int d1, int d2, const uint16_t* x, const uint16_t* dy,
                         float* dw, float* db, void* stream) {
  if (!x || !dy || !dw || !db || mout < 1 || mout > m || d0 < 1 || d1 < 1 || d2 < 1)
    return ws_err("ws_conv_wgrad: bad argument", IPM_ERR_ARG);
  if (!((cin == 16 || cin == 32) && (m == 16 || m == 32))) return ws_err("ws_conv_wgrad: channels", IPM_ERR_ARG);
  cudaStream_t st = (cudaStream_t)stream;
  float *part = nullptr, *bpart = nullptr;
  cudaError_t e = cudaMalloc(&part, (size_t)kWgradBlocks * 27 * m * cin * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&bpart, (size_t)kWgradBlocks * 32 * sizeof(float));
  if (e == cudaSuccess) e = conv_wgrad_any(cin, m, (const bf16*)x, (const bf16*)dy, d0, d1, d2, part, st);
  if (e == cudaSuccess) {
    wgrad_reduce_kernel<<<blocks_for(27LL * mout * cin, 256), 256, 0, st>>>(part, kWgradBlocks, m, cin, mout, dw);
    bgrad_kernel<<<kWgradBlocks, 256, 0, st>>>((const bf16*)dy, (long long)d0 * d1 * d2, m, mout, bpart);
    bgrad_reduce_kernel<<<1, 32, 0, st>>>(bpart, kWgradBlocks, mout, db);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (part) cudaFree(part);
  if (bpart) cudaFree(bpart);
  if (e != cudaSuccess) return ws_err(cudaGetErrorString(e), IPM_ERR_CUDA);
  return IPM_OK;
}

}  // extern "C"
