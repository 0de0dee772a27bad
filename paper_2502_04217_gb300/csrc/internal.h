// Internal declarations shared by the kernels and the C-ABI layer.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "fft_core.cuh"

namespace sdft {

// Device-resident scalars of one solve.  Written by the last block of the
// reduction kernels, read by later kernels, copied to the host only at the
// points where the host decides (IPM convergence, PCG chunk boundaries).
struct DevScalars {
  // PCG
  double rho;        // r^T z of the current iterate
  double cg_stop;    // stop when sqrt(rho) <= cg_stop
  double pq;         // p^T K p of the last product
  double alpha_cg;   // rho / p^T K p
  double beta_cg;    // rho_new / rho (0 before the first product)
  double zw_old;     // conjugate residuals: z^T K z of the previous iteration (0 at a PCG start);
                     // conjugate A-residuals: y^T K y of the previous iteration (0 at a (re)start)
  double rho_car0;   // conjugate A-residuals: y^T K y at the start of the current cycle
  int cg_done;       // 1 once PCG has stopped (kernels then return at once)
  int cg_iter;       // PCG iterations of the current solve
  int cg_status;     // 0 ok, 1 hit max_cg, 2 non-finite value
  int pad0;
  // IPM
  double lambda;     // penalty
  double mu;         // duality measure (nu1^T s1 + nu2^T s2) / 2n
  double sigma;      // centring parameter for the next direction
  double alpha;      // last IPM step
  double alpha_aff;  // predictor-corrector: step to the boundary along the affine predictor (<= 1)
  double mu_aff;     // predictor-corrector: duality measure after that step
  double primal, dual, gap;
  double yy;         // ||b||^2 over observed samples
  double cmax;       // ||M_perp^T b||_inf
  double theta2;     // ||b - M_perp beta||^2
  double corr;       // ||M_perp^T (b - M_perp beta)||_inf
  double l1;         // ||beta||_1
  double nobs;       // number of observed samples
  // IPM control, kept on the device so a whole solve can run inside one graph
  int ipm_done;      // 1 once the stop test has fired
  int ipm_it;        // Newton directions taken
  int ipm_status;    // 0 converged, 4 iteration cap, 6 non-finite
  int cg_total;      // PCG iterations over the solve
  int cg_max;        // largest PCG count of one IPM iteration
  int cg_cap_hit;    // some PCG solve stopped at max_cg
  int refine_now;    // mixed precision: recompute the PCG residual in FP64 after this update;
                     // conjugate A-residuals: (re)start product w = K z requested
  int refine_exit;   // ... because PCG had stopped (1) or periodically (0)
  int refinements;   // FP64 residual replacements over the solve
  int incr;          // 1: G beta is updated from the PCG products and recomputed only to confirm the stop
  int exact_now;     // (incr) G beta is recomputed by an FP64 product in this IPM iteration
  int gb_products;   // FP64 products that recomputed G beta over the solve
  int pc_skip;       // predictor-corrector: the last PCG solve stopped at max_cg, so this direction
                     // takes the fixed centring rule and no second-order term
  int confirming;    // (incr) this iteration's exact product confirms a stop test passed on the
                     // carried G beta; if it fails, G beta is recomputed every iteration from then on
  int wait_expired;  // a bounded device-side wait gave up (staged K operands): the solve reports IPM_TIMEOUT
  int cert_ready;    // cert_sum holds the certificate's sums at the current point (left by step_update;
                     // not after an exact G beta product, which changes G beta)
  int pad2;
  double cert_sum[4];  // c^T beta, beta^T G beta, ||beta||_1, ||c - G beta||_inf
  unsigned long long launches;   // kernels launched by the library (every kernel adds 1)
};

// Count one launch (thread 0 of block 0 of every kernel).
__device__ __forceinline__ void count_launch(DevScalars* sc) {
  if (threadIdx.x == 0 && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0) atomicAdd(&sc->launches, 1ull);
}

enum MapIn { MAPIN_NONE = 0, MAPIN_BETA = 1, MAPIN_PCG = 2 };
enum MapOut { MAPOUT_NONE = 0, MAPOUT_BETA = 1, MAPOUT_K = 2 };

// Arguments of one FFT pass kernel.  Vectors in the beta layout are doubles
// (2H per block); the work buffer holds H complex values of the pass type.
struct PassArgs {
  Layout lay;
  FftPlan plan;          // length L (row/column passes); middle pass: h = Nl/2 (even Nl) or Nl (odd Nl)
  int lgP, PP;           // pencils per tile = 1 << lgP, smem pencil stride
  int nwork;             // threads carrying FFT work = P * L / E
  long long npencils;    // pencils of the pass (row: number of rows; middle: M)
  const void* tw;        // roots of unity for plan.L (pass type)
  const void* twN;       // middle pass: roots of unity for Nl
  void* buf;             // in-place complex work buffer (H values)
  int mapin, mapout;
  const double* src;     // MAPIN_BETA: beta-layout vector (2H)
  double* p;             // MAPIN_PCG / MAPOUT_K: p (4H: beta block, z block)
  const double* zv;      // MAPIN_PCG: preconditioned residual (4H)
  double* dst;           // MAPOUT_BETA: output beta-layout vector (2H)
  double out_scale;      // MAPOUT_BETA scale
  const double* lam1;    // MAPOUT_K: Lambda1, Lambda2 (2H each)
  const double* lam2;
  double* q;             // MAPOUT_K: K p (4H)
  int pcg_mode;          // MAPOUT_K inside PCG: form alpha = rho / p^T q
  int cr_mode;           // with pcg_mode: conjugate residuals, only store the product's p^T q (= z^T K z)
  int check_done;        // return at once when sc->cg_done
  int check_refine;      // return at once unless sc->refine_now
  int check_exact;       // return at once unless sc->exact_now
  double* gp_out;        // MAPOUT_K in PCG (incremental G beta): also store (G p)_beta here (2H)
  const uint32_t* maskw; // middle pass: bit-packed mask, word (xl/32)*M + x'
  double inv_n;          // 1/n, applied with the mask
  const double* yreal;   // middle pass "from real": the signal on the grid (row-major)
  int from_real;         // middle pass: R2C only, of yreal * mask
  double* partials;
  unsigned* counter;
  DevScalars* sc;
  int reg;               // 1: register-engine kernels (fft_reg.cuh), E = 16
  int kstage;            // forward row pass with MAPOUT_K: how its FP64 operands (p, Lambda1, Lambda2)
                         // reach the epilogue: 0 per-slot loads after the transform, 1 an L2 bulk
                         // prefetch of the tile's operands when the block starts, 2 bulk copies
                         // into shared memory (at byte offset kst_off) completing on an mbarrier
  unsigned kst_off;
  int kst_wait_log2;     // failure-detection test: 0 normally; else leave out the fourth operand copy
                         // and give up each wait after 2^kst_wait_log2 polls
};

// Launch with programmatic stream serialization while g_pdl is set (by the
// solve and operator entry points of the calling thread); every kernel launched
// through here starts with pdl_wait().
extern thread_local bool g_pdl;

template <typename... KArgs, typename... Args>
cudaError_t launch_k(void (*fn)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = g_pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, fn, static_cast<KArgs>(args)...);
}

// The tile a pass gets without the autotuner (FFT length L, `rows` shared-memory
// rows, npen pencils): the same choice as a handle with autotune = 0 (capi.cu).
struct TileChoice {
  FftPlan plan;
  int E, lgP, PP, nwork, threads;
  size_t smem;
};
bool default_tile(int L, int rows, long long npen, bool fp32, TileChoice* out);

// Launchers (fft_passes.cu).  `pass_kind`: 0 row, 1 column, 2 middle.
cudaError_t launch_pass(int pass_kind, bool inv, bool fp32, int E, const PassArgs& a, int threads,
                        size_t smem, dim3 grid, cudaStream_t st);

}  // namespace sdft
