// Elementwise and reduction kernels of the interior-point method (FP64).
//
// Vectors use the beta layout of common.cuh (2H doubles, ghost coordinates
// held at 0 and skipped by every reduction).  Two-block vectors (x, r, z, p, q
// of the condensed system) are [beta block | z block], 4H doubles.
//
// The stop decisions live on the device (DevScalars), so that a whole solve
// can run as one CUDA graph with two nested conditional WHILE nodes: the IPM
// loop (condition written by certificate_kernel) and, inside it, the PCG loop
// (condition written by prepare_kernel and pcg_update_kernel).  Every kernel
// that writes a condition writes it from exactly one thread, on every path,
// and both loops are bounded by their iteration caps.
#include <map>
#include <mutex>

#include "internal.h"
#include "kernels.h"

namespace sdft {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ bool first_thread() { return threadIdx.x == 0 && blockIdx.x == 0; }

// |x| as the bit pattern of a non-negative double (orders like the numbers)
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}

__device__ __forceinline__ void set_cond(const LoopCtl& c, unsigned v) {
  if (c.use) cudaGraphSetConditional(c.handle, v);
}

__global__ void __launch_bounds__(kThreads) pack_mask_kernel(const uint8_t* __restrict__ mask, uint32_t* __restrict__ words,
                                                             int Nl, int M, DevScalars* sc) {
  pdl_wait();
  count_launch(sc);
  // one thread per output word: 32 consecutive samples of one row x'
  const long long nw = (long long)((Nl + 31) / 32) * M;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nw; i += (long long)gridDim.x * blockDim.x) {
    const int blk = (int)(i / M), xp = (int)(i - (long long)blk * M);
    uint32_t w = 0;
    for (int b = 0; b < 32; ++b) {
      const int xl = blk * 32 + b;
      if (xl < Nl && mask[(size_t)xp * Nl + xl]) w |= (1u << b);
    }
    words[i] = w;
  }
}

// ||b||^2 over observed samples, and the count of observed samples
__global__ void __launch_bounds__(kThreads) observed_norm_kernel(const double* __restrict__ y, const uint8_t* __restrict__ mask,
                                                                 long long n, double* partials, unsigned* counter,
                                                                 DevScalars* sc) {
  pdl_wait();
  __shared__ double scratch[64];
  count_launch(sc);
  double v[2] = {0.0, 0.0};
  const int ops[2] = {RED_SUM, RED_SUM};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    if (mask[i]) { v[0] += y[i] * y[i]; v[1] += 1.0; }
  }
  if (grid_reduce<2>(v, ops, partials, counter, scratch) && threadIdx.x == 0) { sc->yy = v[0]; sc->nobs = v[1]; }
}

// ||c||_inf for lambda_max; sets lambda (relative or absolute)
__global__ void __launch_bounds__(kThreads) cmax_kernel(const double* __restrict__ c, long long n2, double lam_in, int relative,
                                                        double* partials, unsigned* counter, DevScalars* sc) {
  pdl_wait();
  __shared__ double scratch[32];
  count_launch(sc);
  double v[1] = {0.0};
  const int ops[1] = {RED_MAX};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n2; i += (long long)gridDim.x * blockDim.x)
    v[0] = fmax(v[0], fabs(c[i]));
  if (grid_reduce<1>(v, ops, partials, counter, scratch) && threadIdx.x == 0) {
    sc->cmax = v[0];
    sc->lambda = relative ? lam_in * v[0] : lam_in;
  }
}

// incr: G beta carried; exact0: the first residual product is needed (0 when G beta is
// known exactly at the start, as for the cold start beta = 0).
__device__ __forceinline__ void reset_control(DevScalars* sc, double mu, double sigma0, int incr, int exact0) {
  sc->incr = incr;
  sc->pc_skip = 0;
  sc->confirming = 0;
  sc->exact_now = exact0;
  sc->gb_products = 0;
  sc->mu = mu;
  sc->sigma = sigma0;
  sc->alpha = 0.0;
  sc->ipm_done = 0;
  sc->ipm_it = 0;
  sc->ipm_status = 0;
  sc->cg_total = 0;
  sc->cg_max = 0;
  sc->cg_cap_hit = 0;
  sc->cg_done = 1;
  sc->refine_now = 0;
  sc->refine_exit = 0;
  sc->refinements = 0;
  sc->wait_expired = 0;
  sc->cert_ready = 0;
}

// Start point: beta = 0, z = s1 = s2 = zeta, nu1 = nu2 = lambda/2 (ghosts 0); mu; control reset
__global__ void __launch_bounds__(kThreads) init_point_kernel(Layout lay, double* beta, double* z, double* s1, double* s2,
                                                              double* nu1, double* nu2, double* Gb, double* partials,
                                                              unsigned* counter, DevScalars* sc, double sigma0, int incr) {
  pdl_wait();
  __shared__ double scratch[32];
  count_launch(sc);
  const double zeta = fmax(1.0, sc->cmax), hl = 0.5 * sc->lambda;
  double v[1] = {0.0};
  const int ops[1] = {RED_SUM};
  const long long n2 = 2 * lay.H;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n2; i += (long long)gridDim.x * blockDim.x) {
    const bool gh = is_ghost(lay, i);
    beta[i] = 0.0;
    Gb[i] = 0.0;                     // G beta of beta = 0, exactly: no first product
    z[i] = gh ? 0.0 : zeta;
    s1[i] = gh ? 0.0 : zeta;
    s2[i] = gh ? 0.0 : zeta;
    nu1[i] = gh ? 0.0 : hl;
    nu2[i] = gh ? 0.0 : hl;
    if (!gh) v[0] += hl * zeta + hl * zeta;
  }
  if (grid_reduce<1>(v, ops, partials, counter, scratch) && threadIdx.x == 0)
    reset_control(sc, v[0] / (2.0 * (double)lay.n), sigma0, incr, incr ? 0 : 1);
}

// mu = (nu1^T s1 + nu2^T s2) / 2n at a given point (after ipm_set_point); control reset
__global__ void __launch_bounds__(kThreads) mu_kernel(Layout lay, IpmVectors w, double* partials, unsigned* counter,
                                                      DevScalars* sc, double sigma0, int incr) {
  pdl_wait();
  __shared__ double scratch[32];
  count_launch(sc);
  double v[1] = {0.0};
  const int ops[1] = {RED_SUM};
  const long long n2 = 2 * lay.H;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n2; i += (long long)gridDim.x * blockDim.x)
    if (!is_ghost(lay, i)) v[0] += w.nu1[i] * w.s1[i] + w.nu2[i] * w.s2[i];
  if (grid_reduce<1>(v, ops, partials, counter, scratch) && threadIdx.x == 0)
    reset_control(sc, v[0] / (2.0 * (double)lay.n), sigma0, incr, 1);
}

// Duality-gap certificate at beta from G beta and c = M_perp^T b, and the IPM stop test:
//   ||theta||^2 = ||b||^2 - 2 c^T beta + beta^T G beta,  b^T theta = ||b||^2 - c^T beta,
//   ||M_perp^T theta||_inf = ||c - G beta||_inf,  P = ||theta||^2/2 + lambda ||beta||_1,
//   D = s b^T theta - s^2 ||theta||^2 / 2 with s = min(1, lambda / ||M_perp^T theta||_inf).
// Stop when the relative gap (P - D) / max(1, |P|) <= gap_tol, at the iteration cap,
// or on a non-finite value; the IPM loop condition is !ipm_done.
// The objective, the scaled dual point and the stop decision from the four sums
// v = (c^T beta, beta^T G beta, ||beta||_1, ||c - G beta||_inf); one thread.
__device__ void certify(DevScalars* sc, const double (&v)[4], double gap_tol, int max_ipm, LoopCtl ipm_loop) {
  const double lam = sc->lambda;
  const double th2 = fmax(sc->yy - 2.0 * v[0] + v[1], 0.0);
  const double bth = sc->yy - v[0];
  const double P = 0.5 * th2 + lam * v[2];
  const double s = (v[3] <= lam) ? 1.0 : lam / v[3];
  const double D = s * bth - 0.5 * s * s * th2;
  const double gap = (P - D) / fmax(1.0, fabs(P));
  sc->theta2 = th2;
  sc->corr = v[3];
  sc->l1 = v[2];
  sc->primal = P;
  sc->dual = D;
  sc->gap = gap;
  // incremental G beta: a stop test passed on the updated G beta is confirmed
  // by an exact FP64 product first (this iteration takes no step).  A confirmation
  // that fails shows the carried value is not accurate enough at this gap any more:
  // from then on G beta is recomputed by an FP64 product every iteration (incr = 0,
  // exact_now = 1: the residual product runs and the iteration steps as usual).
  const bool exact = !sc->incr || sc->exact_now;           // an FP64 product formed G beta
  const bool confirm = sc->confirming != 0;
  sc->confirming = 0;
  if (exact) sc->gb_products += 1;
  if (!isfinite(gap) || !isfinite(sc->mu)) { sc->ipm_done = 1; sc->ipm_status = 6; }
  else if (gap <= gap_tol && exact) { sc->ipm_done = 1; sc->ipm_status = 0; }
  else if (gap <= gap_tol) { sc->exact_now = 1; sc->confirming = 1; }
  else if (sc->ipm_it >= max_ipm) { sc->ipm_done = 1; sc->ipm_status = 4; }
  else if (confirm) { sc->incr = 0; sc->exact_now = 1; }
  else sc->exact_now = sc->incr ? 0 : 1;
  set_cond(ipm_loop, sc->ipm_done ? 0u : 1u);
}

// Certificate and stop test (once per IPM iteration).  When step_update left the four
// sums at this point and G beta is the carried one (no exact product since), one
// thread takes the decision from them; otherwise (the first point, after an exact FP64
// product of G beta) the kernel forms the sums in a pass over beta, G beta and c.
__global__ void __launch_bounds__(kThreads) certificate_kernel(long long n2, const double* __restrict__ beta,
                                                               const double* __restrict__ Gb, const double* __restrict__ c,
                                                               double* partials, unsigned* counter, DevScalars* sc,
                                                               double gap_tol, int max_ipm, LoopCtl ipm_loop) {
  pdl_wait();
  __shared__ double scratch[4 * 32];
  count_launch(sc);
  const bool exact = !sc->incr || sc->exact_now;
  if (sc->cert_ready && !exact) {
    // the decision rewrites the flags just read, so it waits until every block has
    // read them: each block arrives on the grid counter and the last one decides
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == gridDim.x * gridDim.y - 1;
    __syncthreads();
    if (last && threadIdx.x == 0) {
      __threadfence();
      const double v[4] = {sc->cert_sum[0], sc->cert_sum[1], sc->cert_sum[2], sc->cert_sum[3]};
      sc->cert_ready = 0;
      certify(sc, v, gap_tol, max_ipm, ipm_loop);
      *counter = 0u;
    }
    return;
  }
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  const int ops[4] = {RED_SUM, RED_SUM, RED_SUM, RED_MAX};
  // one half-spectrum slot (two coordinates, 16-byte loads) per step
  const double2* b2 = reinterpret_cast<const double2*>(beta);
  const double2* g2 = reinterpret_cast<const double2*>(Gb);
  const double2* c2 = reinterpret_cast<const double2*>(c);
  // ||c - G beta||_inf on the integer pipe: the bit patterns of non-negative doubles
  // order like the numbers (a non-finite G beta also makes the sum v[1] non-finite)
  unsigned long long m3 = 0ull;
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < (n2 >> 1); j += (long long)gridDim.x * blockDim.x) {
    const double2 b = b2[j], g = g2[j], ci = c2[j];
    v[0] = fma(ci.y, b.y, fma(ci.x, b.x, v[0]));     // FMAs into the running sums: the FP64
    v[1] = fma(b.y, g.y, fma(b.x, g.x, v[1]));       // pipe bounds this kernel
    v[2] += fabs(b.x) + fabs(b.y);
    m3 = max(m3, max(abs_bits(ci.x - g.x), abs_bits(ci.y - g.y)));
  }
  v[3] = __longlong_as_double((long long)m3);
  if (grid_reduce<4>(v, ops, partials, counter, scratch) && threadIdx.x == 0) {
    sc->cert_ready = 0;
    certify(sc, v, gap_tol, max_ipm, ipm_loop);
  }
}

// Barrier diagonals, preconditioner coefficients, condensed right-hand side and
// PCG start (x = 0, r = rhs, z = P^{-1} r, p = z, rho = r^T z).
// rho > 0: the identity block of P is scaled by rho; rho <= 0: rho = n / (observed samples)
__device__ __forceinline__ double precond_scale(double rho, const Layout& lay, const DevScalars* sc) {
  return rho > 0.0 ? rho : (double)lay.n / fmax(sc->nobs, 1.0);
}

// pc = 1 (predictor-corrector): 1/s, P^{-1} and the affine right-hand side (rb_aff, rc_aff for
// sigma = 0) were formed by predictor_kernel for this iterate and are read back; the
// complementarity rows carry the second-order terms c_i = ds_i,aff o dnu_i,aff left in ds1a,
// ds2a: r_ci = s_i nu_i - sigma mu + c_i adds e_i = (c_i - sigma mu) / s_i to r_ci / s_i, so
// rb = rb_aff - e1 + e2, rc = rc_aff - e1 - e2.  keep_rhs: also store the right-hand side
// (read by refine_kernel only).
__global__ void __launch_bounds__(kThreads) prepare_kernel(Layout lay, IpmVectors w, double* partials, unsigned* counter,
                                                           DevScalars* sc, double cg_tol, int cg_relative, LoopCtl cg_loop,
                                                           double rho_opt, int car, int pc, int keep_rhs) {
  pdl_wait();
  __shared__ double scratch[32];
  count_launch(sc);
  if (sc->ipm_done || (sc->incr && sc->exact_now)) {   // after the stop test, or before an exact re-test: no PCG
    if (first_thread()) { sc->cg_done = 1; set_cond(cg_loop, 0u); }
    return;
  }
  const bool incr = sc->incr;
  const long long n2 = 2 * lay.H;
  const double lam = sc->lambda, smu = sc->sigma * sc->mu;
  const double prho = precond_scale(rho_opt, lay, sc);  // identity scale of P (1: the paper's P)
  double v[1] = {0.0};
  const int ops[1] = {RED_SUM};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n2; i += (long long)gridDim.x * blockDim.x) {
    double l1 = 0, l2 = 0, pa = 0, pb = 0, pc_ = 0, rb = 0, rc = 0, zb = 0, zz = 0, is1 = 0, is2 = 0;
    if (pc && !is_ghost(lay, i)) {
      is1 = w.is1[i];
      is2 = w.is2[i];
      const double e1 = (w.ds1a[i] - smu) * is1, e2 = (w.ds2a[i] - smu) * is2;
      rb = w.rba[i] - e1 + e2;
      rc = w.rca[i] - e1 - e2;
      pa = w.pa[i];
      pb = w.pb[i];
      pc_ = w.pc[i];
      zb = pa * rb - pb * rc;
      zz = -pb * rb + pc_ * rc;
    } else if (!is_ghost(lay, i)) {
      const double b = w.beta[i], z = w.z[i], s1 = w.s1[i], s2 = w.s2[i], n1 = w.nu1[i], n2_ = w.nu2[i];
      is1 = rcp1(s1);
      is2 = rcp1(s2);
      const double r_p1 = z + b - s1, r_p2 = z - b - s2;
      const double S1 = n1 * is1, S2 = n2_ * is2;                // Sigma_i = S_i^{-1} V_i
      // r_c_i / s_i + Sigma_i r_p_i = nu_i + Sigma_i r_p_i - sigma mu / s_i; the nu terms
      // cancel against those of r_d = G beta - c - nu1 + nu2 and r_z = lambda - nu1 - nu2:
      // with e_i = Sigma_i r_p_i - sigma mu / s_i, rb = (c - G beta) - e1 + e2, rc = -lambda - e1 - e2
      const double e1 = fma(S1, r_p1, -smu * is1), e2 = fma(S2, r_p2, -smu * is2);
      rb = (w.c[i] - w.Gb[i]) - e1 + e2;
      rc = -lam - e1 - e2;
      {
        l1 = S1 + S2;
        l2 = S1 - S2;
        const double iD = rcp1(fma(4.0 * S1, S2, prho * l1));   // D = rho (Sigma1 + Sigma2) + 4 Sigma1 Sigma2
        pa = l1 * iD;
        pb = l2 * iD;
        pc_ = fma(prho, iD, pa);                                   // (rho + Lambda1) / D
      }
      zb = pa * rb - pb * rc;
      zz = -pb * rb + pc_ * rc;
    }
    if (!pc) {
      w.is1[i] = is1; w.is2[i] = is2;
      w.lam1[i] = l1; w.lam2[i] = l2;
      w.pa[i] = pa; w.pb[i] = pb; w.pc[i] = pc_;
    }
    w.x[i] = 0.0; w.x[n2 + i] = 0.0;
    w.r[i] = rb; w.r[n2 + i] = rc;
    if (keep_rhs) { w.rhs[i] = rb; w.rhs[n2 + i] = rc; }
    w.zv[i] = zb; w.zv[n2 + i] = zz;
    w.p[i] = zb; w.p[n2 + i] = zz;
    if (incr) w.Gx[i] = 0.0;
    v[0] += rb * zb + rc * zz;
  }
  if (grid_reduce<1>(v, ops, partials, counter, scratch) && threadIdx.x == 0) {
    const double rho = v[0];
    sc->rho = rho;
    sc->beta_cg = 0.0;
    sc->zw_old = 0.0;
    sc->cg_iter = 0;
    sc->cg_status = 0;
    sc->cg_stop = cg_relative ? cg_tol * sqrt(fmax(rho, 0.0)) : cg_tol;
    sc->cg_done = (sqrt(fmax(rho, 0.0)) <= sc->cg_stop) ? 1 : 0;
    sc->refine_now = car ? 1 : 0;       // conjugate A-residuals start with w = K z
    sc->rho_car0 = 0.0;
    if (!isfinite(rho)) { sc->cg_status = 2; sc->cg_done = 1; }
    set_cond(cg_loop, sc->cg_done ? 0u : 1u);
  }
}

// Single-step predictor-corrector (Mehrotra's method with one Krylov solve per
// iteration).  The affine-scaling predictor (the Newton direction for sigma = 0) is
// taken as P^{-1} rhs_aff with the closed-form inverse of Eq. (invprecond1): P differs
// from K only by [G - I, 0; 0, 0], minus the projector onto the missing samples, so
// the estimate costs no product with G.  This kernel forms, at the current iterate,
// everything of the Newton system that does not depend on sigma (1/s, Lambda1,
// Lambda2, P^{-1}'s coefficients, exactly as prepare_kernel would) and the affine
// right-hand side (rba, rca), then the predictor ds_i = dz +- dbeta + r_p_i,
// dnu_i = -nu_i - Sigma_i ds_i and the corrector's second-order terms ds1 o dnu1,
// ds2 o dnu2 (written to ds1a, ds2a; 0 when pc_skip),
// all in FP64: near convergence Sigma_i reaches 1e10 and more, and dnu_i = -nu_i -
// Sigma_i ds_i amplifies any rounding of ds_i by that much (an FP32 predictor drove
// solves into the iteration cap).  One grid reduction gives the largest step
// alpha_aff <= 1 keeping (s, nu) >= 0 (ratio test in FP32 on FP32 roundings, as
// step_length_kernel) and ds^T dnu; the predictor satisfies s o dnu + nu o ds = -s o nu
// by construction of dnu, so (s + a ds)^T (nu + a dnu) = (1 - a) s^T nu + a^2 ds^T dnu and
//     mu_aff = (1 - alpha_aff) mu + alpha_aff^2 ds^T dnu / 2n;
// sigma = (mu_aff / mu)^3 clamped to [sigma_min, sigma_max] follows in the last block.
// After a PCG solve stopped at max_cg (pc_skip) sigma stays the fixed rule's.
__global__ void __launch_bounds__(kThreads) predictor_kernel(Layout lay, IpmVectors w, double* partials, unsigned* counter,
                                                             DevScalars* sc, double rho_opt, double sigma_min,
                                                             double sigma_max) {
  pdl_wait();
  __shared__ double scratch[2 * 32];
  count_launch(sc);
  if (sc->ipm_done || (sc->incr && sc->exact_now)) return;
  const long long n2 = 2 * lay.H;
  const double lam = sc->lambda;
  const double prho = precond_scale(rho_opt, lay, sc);
  const bool rho_one = prho == 1.0;        // the paper's P: no multiply by rho
  const bool skip = sc->pc_skip != 0;
  float best = __int_as_float(0x7f800000);   // +inf
  auto consider = [&](double wv, double dw) {
    if (__double_as_longlong(dw) < 0) best = fminf(best, d2f_int(wv) / d2f_int(-dw));
  };
  double a2 = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n2; i += (long long)gridDim.x * blockDim.x) {
    double l1 = 0, l2 = 0, pa = 0, pb = 0, pc = 0, is1 = 0, is2 = 0, c1 = 0, c2 = 0, rb = 0, rc = 0;
    if (!is_ghost(lay, i)) {
      const double b = w.beta[i], z = w.z[i], s1 = w.s1[i], s2 = w.s2[i], n1 = w.nu1[i], n2_ = w.nu2[i];
      is1 = rcp1(s1);
      is2 = rcp1(s2);
      const double S1 = n1 * is1, S2 = n2_ * is2;
      l1 = S1 + S2;
      l2 = S1 - S2;
      const double iD = rcp1(fma(4.0 * S1, S2, rho_one ? l1 : prho * l1));
      pa = l1 * iD;
      pb = l2 * iD;
      pc = fma(prho, iD, pa);             // (rho + Lambda1) / D
      const double r_p1 = z + b - s1, r_p2 = z - b - s2;
      // sigma = 0: r_c_i / s_i + Sigma_i r_p_i = nu_i + Sigma_i r_p_i, and the nu terms
      // cancel against those of r_d = G beta - c - nu1 + nu2 and r_z = lambda - nu1 - nu2:
      // rb = (c - G beta) - Sigma1 r_p1 + Sigma2 r_p2, rc = -lambda - Sigma1 r_p1 - Sigma2 r_p2
      rb = fma(S2, r_p2, fma(-S1, r_p1, w.c[i] - w.Gb[i]));
      rc = fma(-S2, r_p2, fma(-S1, r_p1, -lam));
      const double db = fma(pa, rb, -pb * rc), dz = fma(pc, rc, -pb * rb);
      const double ds1 = dz + db + r_p1, ds2 = dz - db + r_p2;
      const double dn1 = -fma(S1, ds1, n1), dn2 = -fma(S2, ds2, n2_);
      consider(s1, ds1);
      consider(s2, ds2);
      consider(n1, dn1);
      consider(n2_, dn2);
      c1 = ds1 * dn1;
      c2 = ds2 * dn2;
      a2 += c1 + c2;
    }
    w.is1[i] = is1; w.is2[i] = is2;
    w.lam1[i] = l1; w.lam2[i] = l2;
    w.pa[i] = pa; w.pb[i] = pb; w.pc[i] = pc;
    w.ds1a[i] = skip ? 0.0 : c1;
    w.ds2a[i] = skip ? 0.0 : c2;
    w.rba[i] = rb;
    w.rca[i] = rc;
  }
  double v[2] = {(double)best, a2};
  const int ops[2] = {RED_MIN, RED_SUM};
  if (grid_reduce<2>(v, ops, partials, counter, scratch) && threadIdx.x == 0) {
    const double al = fmin(1.0, v[0]);
    const double mu = sc->mu;
    const double mu_aff = fma(1.0 - al, mu, al * al * v[1] / (2.0 * (double)lay.n));
    sc->alpha_aff = al;
    sc->mu_aff = mu_aff;
    if (!skip) {
      const double t = mu_aff / mu;
      sc->sigma = fmin(sigma_max, fmax(sigma_min, t * t * t));
    }
  }
}

// Preconditioner coefficients only (for precond_apply / kkt_apply on a given Sigma)
__global__ void __launch_bounds__(kThreads) sigma_coef_kernel(Layout lay, const double* s1, const double* nu1, const double* s2,
                                                              const double* nu2, double* lam1, double* lam2, double* pa,
                                                              double* pb, double* pc, DevScalars* sc, double rho_opt) {
  pdl_wait();
  count_launch(sc);
  const long long n2 = 2 * lay.H;
  const double prho = precond_scale(rho_opt, lay, sc);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n2; i += (long long)gridDim.x * blockDim.x) {
    double l1 = 0, l2 = 0, a = 0, b = 0, c = 0;
    if (!is_ghost(lay, i)) {
      const double S1 = nu1[i] / s1[i], S2 = nu2[i] / s2[i];
      l1 = S1 + S2;
      l2 = S1 - S2;
      const double iD = 1.0 / (prho * (S1 + S2) + 4.0 * S1 * S2);
      a = l1 * iD;
      b = l2 * iD;
      c = (prho + l1) * iD;
    }
    lam1[i] = l1; lam2[i] = l2; pa[i] = a; pb[i] = b; pc[i] = c;
  }
}

// z = P^{-1} r  (Eq. (invprecond1): [L1/D, -L2/D; -L2/D, (1+L1)/D])
__global__ void __launch_bounds__(kThreads) precond_kernel(long long n2, const double* __restrict__ pa, const double* __restrict__ pb,
                                                           const double* __restrict__ pc, const double* __restrict__ r,
                                                           double* __restrict__ z, DevScalars* sc) {
  pdl_wait();
  count_launch(sc);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n2; i += (long long)gridDim.x * blockDim.x) {
    const double rb = r[i], rz = r[n2 + i], a = pa[i], b = pb[i], c = pc[i];
    z[i] = a * rb - b * rz;
    z[n2 + i] = -b * rb + c * rz;
  }
}

// One PCG update after q = K p: x += alpha p, r -= alpha q, z = P^{-1} r, rho' = r^T z,
// beta_cg = rho'/rho, stop test; the PCG loop condition is !cg_done.  One thread step
// handles one half-spectrum slot (both coordinates, 16-byte loads and stores) of both
// blocks: the kernel streams about 320 bytes per slot and is bound by HBM, so the
// loads of a slot are all issued before any is used.
__global__ void __launch_bounds__(kThreads) pcg_update_kernel(long long n2, IpmVectors w, double* partials, unsigned* counter,
                                                              DevScalars* sc, int max_cg, int refine_every, LoopCtl cg_loop) {
  pdl_wait();
  __shared__ double scratch[32];
  count_launch(sc);
  if (sc->cg_done) {
    if (first_thread()) set_cond(cg_loop, 0u);
    return;
  }
  const double alpha = sc->alpha_cg;
  const bool incr = sc->incr;
  const long long H = n2 >> 1;                     // slots; the z block starts at slot H
  double2* x2 = reinterpret_cast<double2*>(w.x);
  double2* r2 = reinterpret_cast<double2*>(w.r);
  double2* z2 = reinterpret_cast<double2*>(w.zv);
  const double2* p2 = reinterpret_cast<const double2*>(w.p);
  const double2* q2 = reinterpret_cast<const double2*>(w.q);
  const double2* a2 = reinterpret_cast<const double2*>(w.pa);
  const double2* b2 = reinterpret_cast<const double2*>(w.pb);
  const double2* c2 = reinterpret_cast<const double2*>(w.pc);
  double v[1] = {0.0};
  const int ops[1] = {RED_SUM};
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < H; j += (long long)gridDim.x * blockDim.x) {
    const double2 pb = p2[j], pz = p2[H + j], qb = q2[j], qz = q2[H + j];
    double2 xb = x2[j], xz = x2[H + j], rb = r2[j], rz = r2[H + j];
    const double2 a = a2[j], b = b2[j], c = c2[j];
    if (incr) {                                    // (G x)_beta alongside x_beta
      double2* gx2 = reinterpret_cast<double2*>(w.Gx);
      const double2 gp = reinterpret_cast<const double2*>(w.Gp)[j];
      double2 gx = gx2[j];
      gx.x = fma(alpha, gp.x, gx.x);
      gx.y = fma(alpha, gp.y, gx.y);
      gx2[j] = gx;
    }
    xb.x = fma(alpha, pb.x, xb.x); xb.y = fma(alpha, pb.y, xb.y);
    xz.x = fma(alpha, pz.x, xz.x); xz.y = fma(alpha, pz.y, xz.y);
    rb.x = fma(-alpha, qb.x, rb.x); rb.y = fma(-alpha, qb.y, rb.y);
    rz.x = fma(-alpha, qz.x, rz.x); rz.y = fma(-alpha, qz.y, rz.y);
    double2 zb, zz;
    zb.x = a.x * rb.x - b.x * rz.x; zb.y = a.y * rb.y - b.y * rz.y;
    zz.x = -b.x * rb.x + c.x * rz.x; zz.y = -b.y * rb.y + c.y * rz.y;
    x2[j] = xb; x2[H + j] = xz;
    r2[j] = rb; r2[H + j] = rz;
    z2[j] = zb; z2[H + j] = zz;
    v[0] += (rb.x * zb.x + rz.x * zz.x) + (rb.y * zb.y + rz.y * zz.y);
  }
  if (grid_reduce<1>(v, ops, partials, counter, scratch) && threadIdx.x == 0) {
    const double rho_new = v[0];
    sc->beta_cg = rho_new / sc->rho;
    sc->rho = rho_new;
    sc->cg_iter += 1;
    const bool conv = sqrt(fmax(rho_new, 0.0)) <= sc->cg_stop;
    if (!isfinite(rho_new)) { sc->cg_status = 2; sc->cg_done = 1; }
    else if (conv) sc->cg_done = 1;
    else if (sc->cg_iter >= max_cg) { sc->cg_status = 1; sc->cg_done = 1; }
    // mixed precision: replace the recurrence residual by the FP64 one every
    // refine_every iterations and whenever PCG has converged on FP32 products
    sc->refine_now = 0;
    if (refine_every > 0 && sc->cg_status == 0 && sc->cg_iter < max_cg &&
        (conv || sc->cg_iter % refine_every == 0)) {
      sc->refine_now = 1;
      sc->refine_exit = conv ? 1 : 0;
    }
    set_cond(cg_loop, sc->cg_done ? 0u : 1u);
  }
}

// Conjugate residuals (Sec. 3.5 lists CR beside CG), after w = K z and
// sc->pq = z^T w: beta = z^T w / (z^T w)_previous (0 at a PCG start),
// p = z + beta p, q = w + beta q (= K p), u = P^{-1} q, alpha = z^T w / q^T u.
__global__ void __launch_bounds__(kThreads) cr_update_a_kernel(long long n2, IpmVectors w, double* partials, unsigned* counter,
                                                               DevScalars* sc, LoopCtl cg_loop) {
  pdl_wait();
  __shared__ double scratch[32];
  count_launch(sc);
  if (sc->cg_done) {
    if (first_thread()) set_cond(cg_loop, 0u);
    return;
  }
  const double zw = sc->pq, zw0 = sc->zw_old;
  const bool first = !(zw0 > 0.0);              // a PCG start: p = z, q = w (old p, q not read)
  const double beta = first ? 0.0 : zw / zw0;
  double v[1] = {0.0};
  const int ops[1] = {RED_SUM};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n2; i += (long long)gridDim.x * blockDim.x) {
    double pb = w.zv[i], pz = w.zv[n2 + i], qb = w.wcr[i], qz = w.wcr[n2 + i];
    if (!first) {
      pb += beta * w.p[i];
      pz += beta * w.p[n2 + i];
      qb += beta * w.q[i];
      qz += beta * w.q[n2 + i];
    }
    w.p[i] = pb; w.p[n2 + i] = pz;
    w.q[i] = qb; w.q[n2 + i] = qz;
    const double a = w.pa[i], b = w.pb[i], c = w.pc[i];
    const double ub = a * qb - b * qz, uz = -b * qb + c * qz;
    w.ucr[i] = ub; w.ucr[n2 + i] = uz;
    v[0] += qb * ub + qz * uz;
  }
  if (grid_reduce<1>(v, ops, partials, counter, scratch) && threadIdx.x == 0) {
    const double qu = v[0];
    sc->zw_old = zw;
    if (!(qu > 0.0) || !isfinite(qu)) { sc->cg_status = 2; sc->cg_done = 1; sc->alpha_cg = 0.0; }
    else sc->alpha_cg = zw / qu;
    set_cond(cg_loop, sc->cg_done ? 0u : 1u);
  }
}

// Conjugate residuals, second half: x += alpha p, r -= alpha q, z -= alpha u,
// rho = r^T z and the stop test of PCG.
__global__ void __launch_bounds__(kThreads) cr_update_b_kernel(long long n2, IpmVectors w, double* partials, unsigned* counter,
                                                               DevScalars* sc, int max_cg, LoopCtl cg_loop) {
  pdl_wait();
  __shared__ double scratch[32];
  count_launch(sc);
  if (sc->cg_done) {
    if (first_thread()) set_cond(cg_loop, 0u);
    return;
  }
  const double alpha = sc->alpha_cg;
  double v[1] = {0.0};
  const int ops[1] = {RED_SUM};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n2; i += (long long)gridDim.x * blockDim.x) {
    w.x[i] += alpha * w.p[i];
    w.x[n2 + i] += alpha * w.p[n2 + i];
    const double rb = w.r[i] - alpha * w.q[i], rz = w.r[n2 + i] - alpha * w.q[n2 + i];
    const double zb = w.zv[i] - alpha * w.ucr[i], zz = w.zv[n2 + i] - alpha * w.ucr[n2 + i];
    w.r[i] = rb; w.r[n2 + i] = rz;
    w.zv[i] = zb; w.zv[n2 + i] = zz;
    v[0] += rb * zb + rz * zz;
  }
  if (grid_reduce<1>(v, ops, partials, counter, scratch) && threadIdx.x == 0) {
    const double rho_new = v[0];
    sc->rho = rho_new;
    sc->cg_iter += 1;
    const bool conv = sqrt(fmax(rho_new, 0.0)) <= sc->cg_stop;
    if (!isfinite(rho_new)) { sc->cg_status = 2; sc->cg_done = 1; }
    else if (conv) sc->cg_done = 1;
    else if (sc->cg_iter >= max_cg) { sc->cg_status = 1; sc->cg_done = 1; }
    sc->refine_now = 0;
    set_cond(cg_loop, sc->cg_done ? 0u : 1u);
  }
}

// Conjugate A-residuals (CAr; Sec. 3.5 names it beside CG and CR): CG in the
// inner product of the cube of the split operator L^T K L (M = P^{-1} = L L^T),
// i.e. the Krylov iterate minimising (K M r)^T M (K M r).  Vectors: z = M r,
// w = K z, y = M w (both kept by recurrence), v = K y (the product of every
// iteration), p, q = K p, U = K M K p.  A (re)start computes w = K z by one more
// product (its passes run only while refine_now is set) and y here.
__global__ void __launch_bounds__(kThreads) car_start_kernel(long long n2, IpmVectors w, DevScalars* sc) {
  pdl_wait();
  count_launch(sc);
  if (sc->cg_done || !sc->refine_now) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) sc->refinements += 1;     // the extra product
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n2; i += (long long)gridDim.x * blockDim.x) {
    const double wb = w.wcr[i], wz = w.wcr[n2 + i];
    const double a = w.pa[i], b = w.pb[i], c = w.pc[i];
    w.ucr[i] = a * wb - b * wz;
    w.ucr[n2 + i] = -b * wb + c * wz;
  }
}

// After v = K y and sc->pq = y^T v = rho.  At a cycle start (zw_old = 0): beta = 0
// and rho_car0 = rho.  Otherwise, when rho has fallen to restart_eps * rho_car0 or
// below (the recurred w and y have drifted from K M r), no update is made and the
// next iteration restarts from the current residual; else beta = rho / zw_old.
// p = z + beta p, q = w + beta q, U = v + beta U, alpha = rho / U^T M U.
__global__ void __launch_bounds__(kThreads) car_update_a_kernel(long long n2, IpmVectors w, double* partials,
                                                                unsigned* counter, DevScalars* sc, double restart_eps,
                                                                LoopCtl cg_loop) {
  pdl_wait();
  __shared__ double scratch[32];
  count_launch(sc);
  if (sc->cg_done) {
    if (first_thread()) set_cond(cg_loop, 0u);
    return;
  }
  const double rho = sc->pq, rho0 = sc->zw_old;
  const bool first = !(rho0 > 0.0);
  const bool restart = !first && !(rho > restart_eps * sc->rho_car0);
  const double beta = (first || restart) ? 0.0 : rho / rho0;
  double v[1] = {0.0};
  const int ops[1] = {RED_SUM};
  if (!restart) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n2; i += (long long)gridDim.x * blockDim.x) {
      double pb = w.zv[i], pz = w.zv[n2 + i], qb = w.wcr[i], qz = w.wcr[n2 + i];
      double ub = w.vcar[i], uz = w.vcar[n2 + i];
      if (!first) {
        pb += beta * w.p[i];
        pz += beta * w.p[n2 + i];
        qb += beta * w.q[i];
        qz += beta * w.q[n2 + i];
        ub += beta * w.Ucar[i];
        uz += beta * w.Ucar[n2 + i];
      }
      w.p[i] = pb; w.p[n2 + i] = pz;
      w.q[i] = qb; w.q[n2 + i] = qz;
      w.Ucar[i] = ub; w.Ucar[n2 + i] = uz;
      const double a = w.pa[i], b = w.pb[i], c = w.pc[i];
      v[0] += ub * (a * ub - b * uz) + uz * (-b * ub + c * uz);
    }
  }
  if (grid_reduce<1>(v, ops, partials, counter, scratch) && threadIdx.x == 0) {
    if (restart) {
      sc->refine_now = 1;
      sc->zw_old = 0.0;
      sc->alpha_cg = 0.0;
      sc->refinements += 1;            // this iteration's product is not used
    } else {
      const double um = v[0];
      sc->refine_now = 0;
      sc->zw_old = rho;
      if (first) sc->rho_car0 = rho;
      if (!(rho > 0.0) || !(um > 0.0) || !isfinite(um)) { sc->cg_status = 2; sc->cg_done = 1; sc->alpha_cg = 0.0; }
      else sc->alpha_cg = rho / um;
    }
    set_cond(cg_loop, sc->cg_done ? 0u : 1u);
  }
}

// x += alpha p, r -= alpha q, w -= alpha U, y -= alpha M U, z = M r, rho = r^T z
// and the stop test (nothing when the first half asked for a restart).
__global__ void __launch_bounds__(kThreads) car_update_b_kernel(long long n2, IpmVectors w, double* partials,
                                                                unsigned* counter, DevScalars* sc, int max_cg,
                                                                LoopCtl cg_loop) {
  pdl_wait();
  __shared__ double scratch[32];
  count_launch(sc);
  if (sc->cg_done || sc->refine_now) return;
  const double alpha = sc->alpha_cg;
  double v[1] = {0.0};
  const int ops[1] = {RED_SUM};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n2; i += (long long)gridDim.x * blockDim.x) {
    const double a = w.pa[i], b = w.pb[i], c = w.pc[i];
    w.x[i] += alpha * w.p[i];
    w.x[n2 + i] += alpha * w.p[n2 + i];
    const double rb = w.r[i] - alpha * w.q[i], rz = w.r[n2 + i] - alpha * w.q[n2 + i];
    const double Ub = w.Ucar[i], Uz = w.Ucar[n2 + i];
    w.wcr[i] -= alpha * Ub;
    w.wcr[n2 + i] -= alpha * Uz;
    w.ucr[i] -= alpha * (a * Ub - b * Uz);
    w.ucr[n2 + i] -= alpha * (-b * Ub + c * Uz);
    const double zb = a * rb - b * rz, zz = -b * rb + c * rz;
    w.r[i] = rb; w.r[n2 + i] = rz;
    w.zv[i] = zb; w.zv[n2 + i] = zz;
    v[0] += rb * zb + rz * zz;
  }
  if (grid_reduce<1>(v, ops, partials, counter, scratch) && threadIdx.x == 0) {
    const double rho_new = v[0];
    sc->rho = rho_new;
    sc->cg_iter += 1;
    const bool conv = sqrt(fmax(rho_new, 0.0)) <= sc->cg_stop;
    if (!isfinite(rho_new)) { sc->cg_status = 2; sc->cg_done = 1; }
    else if (conv) sc->cg_done = 1;
    else if (sc->cg_iter >= max_cg) { sc->cg_status = 1; sc->cg_done = 1; }
    set_cond(cg_loop, sc->cg_done ? 0u : 1u);
  }
}

// FP64 residual replacement (mixed precision, after q = K x in FP64):
// r = rhs - q, z = P^{-1} r, rho = r^T z, and PCG restarts (beta_cg = 0).  After
// a converged FP32 phase, PCG stops only if the FP64 residual passes the test.
__global__ void __launch_bounds__(kThreads) refine_kernel(long long n2, IpmVectors w, double* partials, unsigned* counter,
                                                          DevScalars* sc, LoopCtl cg_loop) {
  pdl_wait();
  __shared__ double scratch[32];
  count_launch(sc);
  if (!sc->refine_now) return;
  double v[1] = {0.0};
  const int ops[1] = {RED_SUM};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n2; i += (long long)gridDim.x * blockDim.x) {
    const double rb = w.rhs[i] - w.q[i], rz = w.rhs[n2 + i] - w.q[n2 + i];
    const double a = w.pa[i], b = w.pb[i], c = w.pc[i];
    const double zb = a * rb - b * rz, zz = -b * rb + c * rz;
    w.r[i] = rb; w.r[n2 + i] = rz;
    w.zv[i] = zb; w.zv[n2 + i] = zz;
    v[0] += rb * zb + rz * zz;
  }
  if (grid_reduce<1>(v, ops, partials, counter, scratch) && threadIdx.x == 0) {
    const double rho = v[0];
    sc->rho = rho;
    sc->beta_cg = 0.0;
    sc->refine_now = 0;
    sc->refinements += 1;
    if (!isfinite(rho)) { sc->cg_status = 2; sc->cg_done = 1; }
    else sc->cg_done = (sqrt(fmax(rho, 0.0)) <= sc->cg_stop) ? 1 : 0;
    set_cond(cg_loop, sc->cg_done ? 0u : 1u);
  }
}

// Newton direction of the eliminated variables (same arithmetic in both step kernels):
// ds1 = dz + dbeta + r_p1, ds2 = dz - dbeta + r_p2, dnu_i = -r_ci / s_i - Sigma_i ds_i with
// r_ci = s_i nu_i - sigma mu (+ the predictor-corrector's second-order term c_i when pc).
struct Dir { double ds1, ds2, dn1, dn2; };
__device__ __forceinline__ Dir direction(const IpmVectors& w, long long i, long long n2, double smu, int pc) {
  const double b = w.beta[i], z = w.z[i], s1 = w.s1[i], s2 = w.s2[i], n1 = w.nu1[i], n2_ = w.nu2[i];
  const double db = w.x[i], dz = w.x[n2 + i];
  const double is1 = w.is1[i], is2 = w.is2[i];       // 1/s of this iterate, from prepare_kernel
  const double c1 = pc ? w.ds1a[i] : 0.0, c2 = pc ? w.ds2a[i] : 0.0;
  Dir d;
  d.ds1 = dz + db + (z + b - s1);
  d.ds2 = dz - db + (z - b - s2);
  d.dn1 = -fma(is1, fma(n1, d.ds1, c1 - smu), n1);     // -nu1 - (c1 - sigma mu + nu1 ds1) / s1
  d.dn2 = -fma(is2, fma(n2_, d.ds2, c2 - smu), n2_);
  return d;
}

// Largest step keeping (s, nu) >= 0; alpha = min(1, tau * alpha_max).  With the
// predictor-corrector (pc) the direction is also left for step_update_kernel in the
// predictor's scratch vectors, which prepare_kernel has consumed: ds1, ds2 over the
// second-order terms (ds1a, ds2a; each thread reads its own term before writing),
// dnu1, dnu2 over the affine right-hand side (rba, rca).
__global__ void __launch_bounds__(kThreads) step_length_kernel(Layout lay, IpmVectors w, double* partials, unsigned* counter,
                                                               DevScalars* sc, double tau, int pc) {
  pdl_wait();
  __shared__ double scratch[32];
  count_launch(sc);
  if (sc->ipm_done || (sc->incr && sc->exact_now)) return;
  const double smu = sc->sigma * sc->mu;
  // ratio test min over {w / (-dw) : dw < 0} in FP32 (operands converted on the
  // integer pipe): alpha_max is then known to ~1e-7 relative, far inside the
  // fraction-to-boundary margin tau < 1, so the step keeps s, nu > 0
  float best = __int_as_float(0x7f800000);   // +inf
  auto consider = [&](double wv, double dw) {
    if (__double_as_longlong(dw) < 0) best = fminf(best, d2f_int(wv) / d2f_int(-dw));
  };
  // one half-spectrum slot (two coordinates, 16-byte loads) per step
  const long long H = lay.H;
  auto ld = [&](const double* v, long long j) { return reinterpret_cast<const double2*>(v)[j]; };
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < H; j += (long long)gridDim.x * blockDim.x) {
    const double2 b = ld(w.beta, j), z = ld(w.z, j), s1 = ld(w.s1, j), s2 = ld(w.s2, j), n1 = ld(w.nu1, j),
                  n2_ = ld(w.nu2, j), db = ld(w.x, j), dz = ld(w.x, H + j), is1 = ld(w.is1, j), is2 = ld(w.is2, j);
    double2 c1 = make_double2(0.0, 0.0), c2 = c1;
    if (pc) { c1 = ld(w.ds1a, j); c2 = ld(w.ds2a, j); }
    double2 o1, o2, o3, o4;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      auto g = [&](const double2& v) { return k ? v.y : v.x; };
      const double ds1 = g(dz) + g(db) + (g(z) + g(b) - g(s1));
      const double ds2 = g(dz) - g(db) + (g(z) - g(b) - g(s2));
      const double dn1 = -fma(g(is1), fma(g(n1), ds1, g(c1) - smu), g(n1));
      const double dn2 = -fma(g(is2), fma(g(n2_), ds2, g(c2) - smu), g(n2_));
      if (!is_ghost(lay, 2 * j + k)) {
        consider(g(s1), ds1);
        consider(g(s2), ds2);
        consider(g(n1), dn1);
        consider(g(n2_), dn2);
      }
      (k ? o1.y : o1.x) = ds1;
      (k ? o2.y : o2.x) = ds2;
      (k ? o3.y : o3.x) = dn1;
      (k ? o4.y : o4.x) = dn2;
    }
    if (pc) {       // ghost coordinates hold 0 in every operand, so their direction is 0 too
      reinterpret_cast<double2*>(w.ds1a)[j] = o1;
      reinterpret_cast<double2*>(w.ds2a)[j] = o2;
      reinterpret_cast<double2*>(w.rba)[j] = o3;
      reinterpret_cast<double2*>(w.rca)[j] = o4;
    }
  }
  double v[1] = {(double)best};
  const int ops[1] = {RED_MIN};
  if (grid_reduce<1>(v, ops, partials, counter, scratch) && threadIdx.x == 0) sc->alpha = fmin(1.0, tau * v[0]);
}

// Take the step, form the new duality measure mu, count the iteration
__global__ void __launch_bounds__(kThreads, 4) step_update_kernel(Layout lay, IpmVectors w, double* partials, unsigned* counter,
                                                               DevScalars* sc, double sigma0, double sigma_slow,
                                                               int sigma_rule, double sigma_min) {
  pdl_wait();
  __shared__ double scratch[5 * 32];
  count_launch(sc);
  if (sc->ipm_done || (sc->incr && sc->exact_now)) return;
  const long long n2 = 2 * lay.H;
  const double smu = sc->sigma * sc->mu, alpha = sc->alpha;
  const bool incr = sc->incr;
  // mu's sum, and with G beta carried the certificate's sums at the new point (c^T beta,
  // beta^T G beta, ||beta||_1, ||c - G beta||_inf; ghost coordinates are 0 in beta,
  // G beta and c), so that the next stop test needs no pass of its own
  double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  const int ops[5] = {RED_SUM, RED_SUM, RED_SUM, RED_SUM, RED_MAX};
  unsigned long long m3 = 0ull;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n2; i += (long long)gridDim.x * blockDim.x) {
    if (is_ghost(lay, i)) continue;
    Dir d;
    if (sigma_rule == 2) {               // the direction step_length_kernel left
      d.ds1 = w.ds1a[i];
      d.ds2 = w.ds2a[i];
      d.dn1 = w.rba[i];
      d.dn2 = w.rca[i];
    } else {
      d = direction(w, i, n2, smu, 0);
    }
    const double b = w.beta[i] + alpha * w.x[i];
    w.beta[i] = b;
    if (incr) {                          // G beta follows beta (G is linear)
      const double g = w.Gb[i] + alpha * w.Gx[i], ci = w.c[i];
      w.Gb[i] = g;
      v[1] = fma(ci, b, v[1]);
      v[2] = fma(b, g, v[2]);
      v[3] += fabs(b);
      m3 = max(m3, abs_bits(ci - g));
    }
    w.z[i] += alpha * w.x[n2 + i];
    const double s1 = w.s1[i] + alpha * d.ds1, s2 = w.s2[i] + alpha * d.ds2;
    const double n1 = w.nu1[i] + alpha * d.dn1, n2_ = w.nu2[i] + alpha * d.dn2;
    w.s1[i] = s1; w.s2[i] = s2; w.nu1[i] = n1; w.nu2[i] = n2_;
    v[0] += n1 * s1 + n2_ * s2;
  }
  v[4] = __longlong_as_double((long long)m3);
  if (grid_reduce<5>(v, ops, partials, counter, scratch) && threadIdx.x == 0) {
    for (int k = 0; k < 4; ++k) sc->cert_sum[k] = v[k + 1];
    sc->cert_ready = incr ? 1 : 0;
    sc->mu = v[0] / (2.0 * (double)lay.n);
    if (sigma_rule == 1 && sc->cg_status != 1) {
      // adaptive centring: (1 - alpha)^3 stands in for Mehrotra's (mu_aff / mu)^3;
      // after a PCG solve stopped at max_cg (an inexact direction) the fixed rule
      // below keeps the iterate centred (aggressive centring then drove mu to 0
      // while the gap stalled)
      const double t = 1.0 - alpha;
      sc->sigma = fmin(sigma_slow, fmax(sigma_min, t * t * t));
    } else {
      // the fixed rule; with the predictor-corrector (sigma_rule 2) the next corrector
      // replaces it unless this PCG solve stopped at max_cg
      sc->sigma = (alpha < 0.1) ? sigma_slow : sigma0;
    }
    sc->pc_skip = sc->cg_status == 1 ? 1 : 0;
    sc->ipm_it += 1;
    sc->cg_total += sc->cg_iter;
    if (sc->cg_iter > sc->cg_max) sc->cg_max = sc->cg_iter;
    if (sc->cg_status == 1) sc->cg_cap_hit = 1;
    if (sc->cg_status == 2) { sc->ipm_done = 1; sc->ipm_status = 6; }
  }
}

// Canonical half spectrum (row-major, last axis halved, interleaved re/im) <-> beta layout.
// unpack: v = B^H beta restricted to the half spectrum, twins filled with conj(rep).
__global__ void __launch_bounds__(kThreads) unpack_kernel(Layout lay, const double* __restrict__ beta, double* __restrict__ vh,
                                                          DevScalars* sc) {
  pdl_wait();
  count_launch(sc);
  const long long H = lay.H;
  const double rh = 0.70710678118654752440;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < H; t += (long long)gridDim.x * blockDim.x) {
    // t = canonical index: k' * Hl + kl
    const long long kp = t / lay.Hl;
    const int kl = (int)(t - kp * lay.Hl);
    const long long s = (long long)kl * lay.M + kp;
    const int cls = slot_class(lay, s);
    double re = 0, im = 0;
    if (cls == INTERIOR || cls == EDGE_REP) { re = beta[2 * s] * rh; im = beta[2 * s + 1] * rh; }
    else if (cls == EDGE_SC) { re = beta[2 * s]; }
    else {
      // twin: conj of the representative at -k' on the same edge plane
      int k0 = 0, k1 = 0;
      if (lay.d == 2) k0 = (int)kp;
      else { k0 = (int)(kp / lay.N1); k1 = (int)(kp - (long long)k0 * lay.N1); }
      const int m0 = (lay.N0 - k0) % lay.N0;
      const int m1 = (lay.d == 3) ? (lay.N1 - k1) % lay.N1 : 0;
      const long long kpr = (lay.d == 3) ? (long long)m0 * lay.N1 + m1 : m0;
      const long long sr = (long long)kl * lay.M + kpr;
      re = beta[2 * sr] * rh;
      im = -beta[2 * sr + 1] * rh;
    }
    vh[2 * t] = re;
    vh[2 * t + 1] = im;
  }
}

// pack: beta = B v from the canonical half spectrum (twin slots of vh ignored)
__global__ void __launch_bounds__(kThreads) pack_kernel(Layout lay, const double* __restrict__ vh, double* __restrict__ beta,
                                                        DevScalars* sc) {
  pdl_wait();
  count_launch(sc);
  const long long H = lay.H;
  const double r2 = 1.41421356237309504880;
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < H; s += (long long)gridDim.x * blockDim.x) {
    const int kl = (int)(s / lay.M);
    const long long kp = s - (long long)kl * lay.M;
    const long long t = kp * lay.Hl + kl;
    const int cls = slot_class(lay, s);
    double b0 = 0, b1 = 0;
    if (cls == INTERIOR || cls == EDGE_REP) { b0 = r2 * vh[2 * t]; b1 = r2 * vh[2 * t + 1]; }
    else if (cls == EDGE_SC) { b0 = vh[2 * t]; }
    beta[2 * s] = b0;
    beta[2 * s + 1] = b1;
  }
}

// ghost coordinates of a beta-layout vector forced to 0
__global__ void __launch_bounds__(kThreads) clear_ghosts_kernel(Layout lay, double* v, int blocks, DevScalars* sc) {
  pdl_wait();
  count_launch(sc);
  const long long n2 = 2 * lay.H;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n2; i += (long long)gridDim.x * blockDim.x) {
    if (is_ghost(lay, i))
      for (int b = 0; b < blocks; ++b) v[b * n2 + i] = 0.0;
  }
}

// Blocks of an elementwise kernel over n elements: at least 4 elements per thread
// (fewer blocks to schedule and to reduce over on small grids: the 512 x 512 solve
// ran 7 % faster than with one element per thread), but at least 2 blocks per SM
// while there is work, at most kMaxElementwiseBlocks.
int grid_for(long long n) {
  const long long one = (n + kThreads - 1) / kThreads;    // blocks at one element per thread
  long long g = (n + 4 * kThreads - 1) / (4 * kThreads);
  if (g < 2 * 152) g = one < 2 * 152 ? one : 2 * 152;
  if (g > kMaxElementwiseBlocks) g = kMaxElementwiseBlocks;
  if (g < 1) g = 1;
  return (int)g;
}

// grid_for's count rounded to whole waves of fn's resident blocks (the SMs times the
// blocks of kThreads threads one SM holds at fn's register use), at most
// kMaxElementwiseBlocks.  Every block of these grid-stride kernels has the same work,
// so a last wave that is partly empty idles SMs: at 1216 blocks a kernel with room for
// 3 (or 6) blocks per SM ran 2.67 (1.33) waves.  The occupancy is looked up once per
// kernel (a query, allowed during stream capture) and the grid stays fixed for a given
// kernel and device, which keeps the reductions' block order and results reproducible.
template <typename... KArgs>
int waves_for(void (*fn)(KArgs...), long long n) {
  const int g = grid_for(n);
  static std::mutex mu;
  static std::map<const void*, int> per_sm;
  static int sms = 0;
  int bps = 0;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (sms == 0) {
      int dev = 0;
      if (cudaGetDevice(&dev) != cudaSuccess ||
          cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        sms = -1;
    }
    auto it = per_sm.find((const void*)fn);
    if (it != per_sm.end()) {
      bps = it->second;
    } else {
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, kThreads, 0) != cudaSuccess) bps = 0;
      per_sm[(const void*)fn] = bps;
    }
  }
  if (bps <= 0 || sms <= 0) return g;
  const int wave = bps * sms;
  if (g <= wave) return g;
  int k = (g + wave / 2) / wave;          // the nearest whole number of waves
  while (k > 1 && k * wave > kMaxElementwiseBlocks) --k;
  return k * wave <= kMaxElementwiseBlocks ? k * wave : g;
}

}  // namespace

cudaError_t k_pack_mask(const uint8_t* mask, uint32_t* words, int Nl, int M, DevScalars* sc, cudaStream_t st) {
  const long long nw = (long long)((Nl + 31) / 32) * M;
  return launch_k(pack_mask_kernel, dim3(grid_for(nw)), dim3(kThreads), 0, st, mask, words, Nl, M, sc);
}
cudaError_t k_observed_norm(const double* y, const uint8_t* mask, long long n, Reduce red, DevScalars* sc, cudaStream_t st) {
  return launch_k(observed_norm_kernel, dim3(grid_for(n)), dim3(kThreads), 0, st, y, mask, n, red.partials, red.counter, sc);
}
cudaError_t k_cmax(const double* c, long long n2, double lam, int relative, Reduce red, DevScalars* sc, cudaStream_t st) {
  return launch_k(cmax_kernel, dim3(grid_for(n2)), dim3(kThreads), 0, st, c, n2, lam, relative, red.partials, red.counter, sc);
}
cudaError_t k_init_point(const Layout& lay, IpmVectors w, Reduce red, DevScalars* sc, double sigma0, int incr,
                         cudaStream_t st) {
  return launch_k(init_point_kernel, dim3(waves_for(init_point_kernel, 2 * lay.H)), dim3(kThreads), 0, st, lay, w.beta, w.z, w.s1, w.s2, w.nu1, w.nu2, w.Gb, red.partials, red.counter, sc, sigma0, incr);
}
cudaError_t k_mu(const Layout& lay, IpmVectors w, Reduce red, DevScalars* sc, double sigma0, int incr, cudaStream_t st) {
  return launch_k(mu_kernel, dim3(waves_for(mu_kernel, 2 * lay.H)), dim3(kThreads), 0, st, lay, w, red.partials, red.counter, sc, sigma0, incr);
}
cudaError_t k_certificate(const Layout& lay, const double* beta, const double* Gb, const double* c, Reduce red,
                          DevScalars* sc, double gap_tol, int max_ipm, LoopCtl loop, cudaStream_t st) {
  return launch_k(certificate_kernel, dim3(waves_for(certificate_kernel, 2 * lay.H)), dim3(kThreads), 0, st, 2 * lay.H, beta, Gb, c, red.partials, red.counter, sc, gap_tol, max_ipm, loop);
}
cudaError_t k_prepare(const Layout& lay, IpmVectors w, Reduce red, DevScalars* sc, double cg_tol, int cg_relative,
                      LoopCtl loop, double rho, int car, int pc, int keep_rhs, cudaStream_t st) {
  return launch_k(prepare_kernel, dim3(waves_for(prepare_kernel, 2 * lay.H)), dim3(kThreads), 0, st, lay, w, red.partials, red.counter, sc, cg_tol, cg_relative, loop, rho, car, pc, keep_rhs);
}
cudaError_t k_predictor(const Layout& lay, IpmVectors w, Reduce red, DevScalars* sc, double rho, double sigma_min,
                        double sigma_max, cudaStream_t st) {
  return launch_k(predictor_kernel, dim3(waves_for(predictor_kernel, 2 * lay.H)), dim3(kThreads), 0, st, lay, w, red.partials, red.counter,
                  sc, rho, sigma_min, sigma_max);
}
cudaError_t k_sigma_coef(const Layout& lay, const double* s1, const double* nu1, const double* s2, const double* nu2,
                         IpmVectors w, DevScalars* sc, double rho, cudaStream_t st) {
  return launch_k(sigma_coef_kernel, dim3(waves_for(sigma_coef_kernel, 2 * lay.H)), dim3(kThreads), 0, st, lay, s1, nu1, s2, nu2, w.lam1, w.lam2, w.pa, w.pb, w.pc, sc, rho);
}
cudaError_t k_precond(const Layout& lay, IpmVectors w, const double* r, double* z, DevScalars* sc, cudaStream_t st) {
  return launch_k(precond_kernel, dim3(waves_for(precond_kernel, 2 * lay.H)), dim3(kThreads), 0, st, 2 * lay.H, w.pa, w.pb, w.pc, r, z, sc);
}
cudaError_t k_pcg_update(const Layout& lay, IpmVectors w, Reduce red, DevScalars* sc, int max_cg, int refine_every,
                         LoopCtl loop, cudaStream_t st) {
  return launch_k(pcg_update_kernel, dim3(waves_for(pcg_update_kernel, 2 * lay.H)), dim3(kThreads), 0, st, 2 * lay.H, w, red.partials, red.counter, sc, max_cg, refine_every, loop);
}
cudaError_t k_refine(const Layout& lay, IpmVectors w, Reduce red, DevScalars* sc, LoopCtl loop, cudaStream_t st) {
  return launch_k(refine_kernel, dim3(waves_for(refine_kernel, 2 * lay.H)), dim3(kThreads), 0, st, 2 * lay.H, w, red.partials, red.counter, sc, loop);
}
cudaError_t k_cr_update_a(const Layout& lay, IpmVectors w, Reduce red, DevScalars* sc, LoopCtl loop, cudaStream_t st) {
  return launch_k(cr_update_a_kernel, dim3(waves_for(cr_update_a_kernel, 2 * lay.H)), dim3(kThreads), 0, st, 2 * lay.H, w, red.partials,
                  red.counter, sc, loop);
}
cudaError_t k_cr_update_b(const Layout& lay, IpmVectors w, Reduce red, DevScalars* sc, int max_cg, LoopCtl loop,
                          cudaStream_t st) {
  return launch_k(cr_update_b_kernel, dim3(waves_for(cr_update_b_kernel, 2 * lay.H)), dim3(kThreads), 0, st, 2 * lay.H, w, red.partials,
                  red.counter, sc, max_cg, loop);
}
cudaError_t k_car_start(const Layout& lay, IpmVectors w, DevScalars* sc, cudaStream_t st) {
  return launch_k(car_start_kernel, dim3(grid_for(2 * lay.H)), dim3(kThreads), 0, st, 2 * lay.H, w, sc);
}
cudaError_t k_car_update_a(const Layout& lay, IpmVectors w, Reduce red, DevScalars* sc, double restart_eps, LoopCtl loop,
                           cudaStream_t st) {
  return launch_k(car_update_a_kernel, dim3(waves_for(car_update_a_kernel, 2 * lay.H)), dim3(kThreads), 0, st, 2 * lay.H, w, red.partials,
                  red.counter, sc, restart_eps, loop);
}
cudaError_t k_car_update_b(const Layout& lay, IpmVectors w, Reduce red, DevScalars* sc, int max_cg, LoopCtl loop,
                           cudaStream_t st) {
  return launch_k(car_update_b_kernel, dim3(waves_for(car_update_b_kernel, 2 * lay.H)), dim3(kThreads), 0, st, 2 * lay.H, w, red.partials,
                  red.counter, sc, max_cg, loop);
}
cudaError_t k_step_length(const Layout& lay, IpmVectors w, Reduce red, DevScalars* sc, double tau, int pc,
                          cudaStream_t st) {
  return launch_k(step_length_kernel, dim3(waves_for(step_length_kernel, 2 * lay.H)), dim3(kThreads), 0, st, lay, w, red.partials, red.counter, sc, tau, pc);
}
cudaError_t k_step_update(const Layout& lay, IpmVectors w, Reduce red, DevScalars* sc, double sigma0, double sigma_slow,
                          int sigma_rule, double sigma_min, cudaStream_t st) {
  return launch_k(step_update_kernel, dim3(waves_for(step_update_kernel, 2 * lay.H)), dim3(kThreads), 0, st, lay, w, red.partials, red.counter, sc, sigma0, sigma_slow, sigma_rule, sigma_min);
}
cudaError_t k_unpack(const Layout& lay, const double* beta, double* vh, DevScalars* sc, cudaStream_t st) {
  return launch_k(unpack_kernel, dim3(grid_for(lay.H)), dim3(kThreads), 0, st, lay, beta, vh, sc);
}
cudaError_t k_pack(const Layout& lay, const double* vh, double* beta, DevScalars* sc, cudaStream_t st) {
  return launch_k(pack_kernel, dim3(grid_for(lay.H)), dim3(kThreads), 0, st, lay, vh, beta, sc);
}
cudaError_t k_clear_ghosts(const Layout& lay, double* v, int blocks, DevScalars* sc, cudaStream_t st) {
  return launch_k(clear_ghosts_kernel, dim3(grid_for(2 * lay.H)), dim3(kThreads), 0, st, lay, v, blocks, sc);
}

}  // namespace sdft
