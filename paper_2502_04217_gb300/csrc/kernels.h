// Launchers of the IPM kernels (ipm_kernels.cu), used by the C-ABI layer.
#pragma once

#include "internal.h"

namespace sdft {

// Device vectors of one problem, all in the beta layout (2H doubles per block).
struct IpmVectors {
  double *beta, *z, *s1, *s2, *nu1, *nu2;     // IPM iterate
  double *c;                                  // M_perp^T b
  double *Gb;                                 // G beta at the current iterate
  double *lam1, *lam2;                        // Lambda1, Lambda2 of K
  double *pa, *pb, *pc;                       // P^{-1} = [pa, -pb; -pb, pc] per element
  double *is1, *is2;                          // 1/s1, 1/s2 at the current iterate (step kernels)
  double *x, *r, *zv, *p, *q;                 // PCG vectors, 2 blocks each (4H)
  double *rhs;                                // right-hand side of the current Newton system (4H)
  double *wcr, *ucr;                          // conjugate residuals: w = K z and u = P^{-1} q (4H each);
                                              // conjugate A-residuals: w = K z and y = P^{-1} w
  double *vcar, *Ucar;                        // conjugate A-residuals: v = K y and U = v + beta U (4H each)
  double *Gp, *Gx;                            // incremental G beta: (G p)_beta of the last PCG product and
                                              // (G x)_beta = sum alpha (G p)_beta over the PCG solve (2H each)
  double *ds1a, *ds2a;                        // predictor-corrector: the second-order terms ds1 o dnu1,
                                              // ds2 o dnu2 of the affine predictor (2H each); after
                                              // step_length the direction's ds1, ds2
  double *rba, *rca;                          // predictor-corrector: the condensed right-hand side of the
                                              // affine system (sigma = 0, no second-order term; 2H each);
                                              // after step_length the direction's dnu1, dnu2
};

// grid size used by every elementwise kernel (also sizes the partials buffer)
constexpr int kMaxElementwiseBlocks = 152 * 8;

struct Reduce {
  double* partials;
  unsigned* counter;
};

// Loop condition of a conditional WHILE graph node, written by the kernel that
// decides the loop (use = 0 outside graphs).
struct LoopCtl {
  cudaGraphConditionalHandle handle;
  int use;
};

// What other parts of the library (the warm start) may use of a handle.
struct HandleView {
  Layout lay;
  IpmVectors w;
  DevScalars* sc;
  cudaStream_t st;
  double* partials;
  unsigned* counter;
};

cudaError_t k_pack_mask(const uint8_t* mask, uint32_t* words, int Nl, int M, DevScalars* sc, cudaStream_t st);
cudaError_t k_observed_norm(const double* y, const uint8_t* mask, long long n, Reduce red, DevScalars* sc, cudaStream_t st);
cudaError_t k_cmax(const double* c, long long n2, double lam, int relative, Reduce red, DevScalars* sc, cudaStream_t st);
cudaError_t k_init_point(const Layout& lay, IpmVectors w, Reduce red, DevScalars* sc, double sigma0, int incr,
                         cudaStream_t st);
cudaError_t k_mu(const Layout& lay, IpmVectors w, Reduce red, DevScalars* sc, double sigma0, int incr, cudaStream_t st);
cudaError_t k_certificate(const Layout& lay, const double* beta, const double* Gb, const double* c, Reduce red,
                          DevScalars* sc, double gap_tol, int max_ipm, LoopCtl loop, cudaStream_t st);
cudaError_t k_prepare(const Layout& lay, IpmVectors w, Reduce red, DevScalars* sc, double cg_tol, int cg_relative,
                      LoopCtl loop, double rho, int car, int pc, int keep_rhs, cudaStream_t st);
cudaError_t k_predictor(const Layout& lay, IpmVectors w, Reduce red, DevScalars* sc, double rho, double sigma_min,
                        double sigma_max, cudaStream_t st);
cudaError_t k_sigma_coef(const Layout& lay, const double* s1, const double* nu1, const double* s2, const double* nu2,
                         IpmVectors w, DevScalars* sc, double rho, cudaStream_t st);
cudaError_t k_precond(const Layout& lay, IpmVectors w, const double* r, double* z, DevScalars* sc, cudaStream_t st);
cudaError_t k_pcg_update(const Layout& lay, IpmVectors w, Reduce red, DevScalars* sc, int max_cg, int refine_every,
                         LoopCtl loop, cudaStream_t st);
cudaError_t k_refine(const Layout& lay, IpmVectors w, Reduce red, DevScalars* sc, LoopCtl loop, cudaStream_t st);
cudaError_t k_cr_update_a(const Layout& lay, IpmVectors w, Reduce red, DevScalars* sc, LoopCtl loop, cudaStream_t st);
cudaError_t k_cr_update_b(const Layout& lay, IpmVectors w, Reduce red, DevScalars* sc, int max_cg, LoopCtl loop,
                          cudaStream_t st);
cudaError_t k_car_start(const Layout& lay, IpmVectors w, DevScalars* sc, cudaStream_t st);
cudaError_t k_car_update_a(const Layout& lay, IpmVectors w, Reduce red, DevScalars* sc, double restart_eps, LoopCtl loop,
                           cudaStream_t st);
cudaError_t k_car_update_b(const Layout& lay, IpmVectors w, Reduce red, DevScalars* sc, int max_cg, LoopCtl loop,
                           cudaStream_t st);
cudaError_t k_step_length(const Layout& lay, IpmVectors w, Reduce red, DevScalars* sc, double tau, int pc,
                          cudaStream_t st);
cudaError_t k_step_update(const Layout& lay, IpmVectors w, Reduce red, DevScalars* sc, double sigma0, double sigma_slow,
                          int sigma_rule, double sigma_min, cudaStream_t st);
cudaError_t k_unpack(const Layout& lay, const double* beta, double* vh, DevScalars* sc, cudaStream_t st);
cudaError_t k_pack(const Layout& lay, const double* vh, double* beta, DevScalars* sc, cudaStream_t st);
cudaError_t k_clear_ghosts(const Layout& lay, double* v, int blocks, DevScalars* sc, cudaStream_t st);

}  // namespace sdft
