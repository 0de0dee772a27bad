// FFT passes of the masked projector G = M_perp^T M_perp = A^T diag(m) A
// (Sec. 3.1: M_perp beta = (IDFT(B^H beta))_observed, M_perp^T b = B DFT(b_hat)).
//
// The half spectrum is held with the halved axis outermost (slot = kl*M + k').
// One application of G runs, for a grid of dimension d:
//   d = 1: one middle pass          (map beta->v, C2R, mask/n, R2C, map v->beta)
//   d = 2: row(inv) -> middle -> row(fwd)
//   d = 3: row(inv) -> column(inv) -> middle -> column(fwd) -> row(fwd)
// Row passes transform the contiguous in-plane axis, column passes the other
// in-plane axis (stride N1), the middle pass the halved axis (stride M) through
// a real transform of length Nl computed as a complex one of length Nl/2.
//
// The beta -> v map is folded into the first pass.  On the two edge planes
// kl in {0, Nl/2} only representatives carry data; instead of filling their
// conjugate twins we feed 2 v at the representative and 0 at the twin, and the
// middle pass keeps only the real part of those two planes.  After the
// in-plane inverse transforms the edge planes of the true (Hermitian) input are
// real, and Re(sum_k 2 v_k e_k) over representatives plus the self-conjugate
// terms equals that real value, so the result is exact.
// Included by fft_passes_f32.cu and fft_passes_f64.cu (one precision each).
#pragma once

#include <type_traits>

#include "internal.h"

namespace sdft {

namespace {

constexpr double kSqrt2 = 1.41421356237309504880;

// The scalings run in the pass type T: FP64 passes scale in FP64, FP32 passes
// round to FP32 first and scale there (their products are FP32 anyway).
template <typename V>
__device__ __forceinline__ V map_in(int cls, double b0, double b1) {
  using T = decltype(V::x);
  if (cls == EDGE_TWIN) return cmake<V>((T)0, (T)0);
  if (cls == EDGE_SC) return cmake<V>(from_double<T>(b0), (T)0);
  const T s = (cls == INTERIOR) ? (T)kSqrtHalf : (T)kSqrt2;
  return cmake<V>(from_double<T>(b0) * s, from_double<T>(b1) * s);
}

template <typename V>
__device__ __forceinline__ void map_out(int cls, V w, double scale, double& o0, double& o1) {
  using T = decltype(V::x);
  if (cls == EDGE_TWIN) { o0 = 0.0; o1 = 0.0; return; }
  if (cls == EDGE_SC) { o0 = to_double(w.x * (T)scale); o1 = 0.0; return; }
  const T s = (T)(kSqrt2 * scale);
  o0 = to_double(w.x * s);
  o1 = to_double(w.y * s);
}

// Load the complex value of slot g for the first pass.  The FP64 vectors stream
// through with the evict-first hint (ld/st .cs) so that the pass-to-pass work
// buffer (67.6 MB in FP32 at 256^3) keeps its place in L2.
template <typename V>
__device__ __forceinline__ V load_slot(const PassArgs& a, long long g) {
  if (a.mapin == MAPIN_NONE) return reinterpret_cast<const V*>(a.buf)[g];
  const int cls = slot_class(a.lay, g);
  if (a.mapin == MAPIN_BETA) {
    const double2 b = __ldcs(reinterpret_cast<const double2*>(a.src) + g);
    return map_in<V>(cls, b.x, b.y);
  }
  if (a.mapin == MAPIN_PCG) {
    // fused PCG direction update p = z + beta_cg * p on both blocks of the slot
    const long long H2 = a.lay.H;    // offset of the z block, in double2 units
    const double bc = a.sc->beta_cg;
    double2* p2 = reinterpret_cast<double2*>(a.p);
    const double2* z2 = reinterpret_cast<const double2*>(a.zv);
    double2 pb = __ldcs(p2 + g), pz = __ldcs(p2 + H2 + g);
    const double2 zb = __ldcs(z2 + g), zz = __ldcs(z2 + H2 + g);
    pb.x = zb.x + bc * pb.x; pb.y = zb.y + bc * pb.y;
    pz.x = zz.x + bc * pz.x; pz.y = zz.y + bc * pz.y;
    __stcs(p2 + g, pb);
    __stcs(p2 + H2 + g, pz);
    return map_in<V>(cls, pb.x, pb.y);
  }
  return reinterpret_cast<const V*>(a.buf)[g];
}

// Store the complex value of slot g for the last pass; inside PCG also adds this
// slot's share of p^T q to acc (FP64 work only where it is needed).
template <typename V, bool PQ>
__device__ __forceinline__ void store_slot(const PassArgs& a, long long g, V w, double& acc) {
  if (a.mapout == MAPOUT_NONE) {
    reinterpret_cast<V*>(a.buf)[g] = w;
    return;
  }
  const int cls = slot_class(a.lay, g);
  double o0, o1;
  if (a.mapout == MAPOUT_BETA) {
    map_out(cls, w, a.out_scale, o0, o1);
    __stcs(reinterpret_cast<double2*>(a.dst) + g, make_double2(o0, o1));
    return;
  }
  // MAPOUT_K: q = [G p_b + L1 p_b + L2 p_z ; L2 p_b + L1 p_z]
  map_out(cls, w, 1.0, o0, o1);
  const long long H2 = a.lay.H;
  const double2* p2 = reinterpret_cast<const double2*>(a.p);
  const double2 pb = __ldcs(p2 + g), pz = __ldcs(p2 + H2 + g);
  const double2 l1 = __ldcs(reinterpret_cast<const double2*>(a.lam1) + g);
  const double2 l2 = __ldcs(reinterpret_cast<const double2*>(a.lam2) + g);
  double2 qb, qz;
  qb.x = o0 + l1.x * pb.x + l2.x * pz.x;
  qb.y = o1 + l1.y * pb.y + l2.y * pz.y;
  qz.x = l2.x * pb.x + l1.x * pz.x;
  qz.y = l2.y * pb.y + l1.y * pz.y;
  double2* q2 = reinterpret_cast<double2*>(a.q);
  __stcs(q2 + g, qb);
  __stcs(q2 + H2 + g, qz);
  if constexpr (PQ) acc += pb.x * qb.x + pb.y * qb.y + pz.x * qz.x + pz.y * qz.y;
}

__device__ __forceinline__ void finish_pq(const PassArgs& a, double acc, double* scratch) {
  double v[1] = {acc};
  const int ops[1] = {RED_SUM};
  if (grid_reduce<1>(v, ops, a.partials, a.counter, scratch) && threadIdx.x == 0) {
    DevScalars* sc = a.sc;
    const double pq = v[0];
    sc->pq = pq;
    if (!(pq > 0.0) || !isfinite(pq)) {       // K is positive definite: anything else is breakdown
      sc->cg_status = 2;
      sc->cg_done = 1;
      sc->alpha_cg = 0.0;
    } else {
      sc->alpha_cg = sc->rho / pq;
    }
  }
}

// ---------------------------------------------------------------------------
// Row pass: P consecutive rows of length L (contiguous), slot = row * L + e.
// ---------------------------------------------------------------------------
template <typename T, int E, bool INV, int LC>
__global__ void __launch_bounds__(E == 16 ? 256 : 512, 1) row_pass_kernel(PassArgs a) {
  using V = typename cvec<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double scratch[32];
  count_launch(a.sc);
  if ((a.check_done && a.sc->cg_done) || (a.check_refine && !a.sc->refine_now)) return;
  V* buf = reinterpret_cast<V*>(smem_raw);
  const int P = 1 << a.lgP, PP = a.PP, L = LC > 0 ? LC : a.plan.L;
  const long long row0 = (long long)blockIdx.x * P;
  for (int idx = threadIdx.x; idx < P * L; idx += blockDim.x) {
    const int p = idx / L, e = idx - p * L;
    const long long row = row0 + p;
    V v = cmake<V>((T)0, (T)0);
    if (row < a.npencils) v = load_slot<V>(a, row * L + e);
    buf[e * PP + p] = v;
  }
  __syncthreads();
  fft_tile_l<E, INV, LC>(buf, a.plan, a.lgP, PP, reinterpret_cast<const V*>(a.tw), threadIdx.x, a.nwork);
  double acc = 0.0;
  auto store_all = [&](auto pq) {
    for (int idx = threadIdx.x; idx < P * L; idx += blockDim.x) {
      const int p = idx / L, e = idx - p * L;
      const long long row = row0 + p;
      if (row < a.npencils) store_slot<V, decltype(pq)::value>(a, row * L + e, buf[e * PP + p], acc);
    }
  };
  if (a.pcg_mode) store_all(std::true_type{});
  else store_all(std::false_type{});
  if (a.mapout == MAPOUT_K && a.pcg_mode) finish_pq(a, acc, scratch);
}

// ---------------------------------------------------------------------------
// Column pass (d = 3): pencils along k0 (length N0, stride N1) at fixed kl,
// P consecutive k1 per tile.  grid = (ceil(N1 / P), Hl).
// ---------------------------------------------------------------------------
template <typename T, int E, bool INV, int LC>
__global__ void __launch_bounds__(E == 16 ? 256 : 512, 1) col_pass_kernel(PassArgs a) {
  using V = typename cvec<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  count_launch(a.sc);
  if ((a.check_done && a.sc->cg_done) || (a.check_refine && !a.sc->refine_now)) return;
  V* buf = reinterpret_cast<V*>(smem_raw);
  const int P = 1 << a.lgP, PP = a.PP, L = LC > 0 ? LC : a.plan.L;
  const int N1 = a.lay.N1;
  const int k1_0 = blockIdx.x * P;
  const long long plane = (long long)blockIdx.y * a.lay.N0;     // kl * N0
  V* g = reinterpret_cast<V*>(a.buf);
  for (int idx = threadIdx.x; idx < P * L; idx += blockDim.x) {
    const int e = idx >> a.lgP, p = idx & (P - 1);
    const int k1 = k1_0 + p;
    V v = cmake<V>((T)0, (T)0);
    if (k1 < N1) v = g[(plane + e) * N1 + k1];
    buf[e * PP + p] = v;
  }
  __syncthreads();
  fft_tile_l<E, INV, LC>(buf, a.plan, a.lgP, PP, reinterpret_cast<const V*>(a.tw), threadIdx.x, a.nwork);
  for (int idx = threadIdx.x; idx < P * L; idx += blockDim.x) {
    const int e = idx >> a.lgP, p = idx & (P - 1);
    const int k1 = k1_0 + p;
    if (k1 < N1) g[(plane + e) * N1 + k1] = buf[e * PP + p];
  }
}

// ---------------------------------------------------------------------------
// Middle pass: pencils along the halved axis (Hl complex, stride M), P
// consecutive in-plane positions x' per tile.  Computes, per pencil,
//   x = C2R(X) (length Nl, unnormalised; Re taken on the two edge planes),
//   y = x * m / n,   Y = R2C(y),
// with the real transforms done as complex transforms of length h = Nl/2 on
// z_j = x_{2j} + i x_{2j+1}.  With from_real the input is the real signal
// y * m itself (used once for M_perp^T b) and only R2C runs.
// ---------------------------------------------------------------------------
template <typename T, int E, int LC>
__global__ void __launch_bounds__(E == 16 ? 256 : 512, 1) middle_pass_kernel(PassArgs a) {
  using V = typename cvec<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double scratch[32];
  count_launch(a.sc);
  if ((a.check_done && a.sc->cg_done) || (a.check_refine && !a.sc->refine_now)) return;
  V* buf = reinterpret_cast<V*>(smem_raw);
  const int P = 1 << a.lgP, PP = a.PP;
  const int h = LC > 0 ? LC : a.plan.L, Nl = a.lay.Nl, M = a.lay.M;
  const int x0 = blockIdx.x * P;
  const int tid = threadIdx.x, nwork = a.nwork;
  const V* twh = reinterpret_cast<const V*>(a.tw);
  const V* twN = reinterpret_cast<const V*>(a.twN);

  if (a.from_real) {
    // z_j = (y m)[2j] + i (y m)[2j+1] for each of the P pencils (rows of the grid)
    for (int idx = tid; idx < P * h; idx += blockDim.x) {
      const int p = idx / h, j = idx - p * h;
      const int xp = x0 + p;
      V v = cmake<V>((T)0, (T)0);
      if (xp < M) {
        const uint32_t w = a.maskw[(size_t)((2 * j) >> 5) * M + xp];
        const double y0 = a.yreal[(size_t)xp * Nl + 2 * j];
        const double y1 = a.yreal[(size_t)xp * Nl + 2 * j + 1];
        v = cmake<V>((T)(((w >> ((2 * j) & 31)) & 1u) ? y0 : 0.0), (T)(((w >> ((2 * j + 1) & 31)) & 1u) ? y1 : 0.0));
      }
      buf[j * PP + p] = v;
    }
    __syncthreads();
  } else {
    // load X (Hl rows)
    const int Hl = h + 1;
    for (int idx = tid; idx < P * Hl; idx += blockDim.x) {
      const int e = idx >> a.lgP, p = idx & (P - 1);
      const int xp = x0 + p;
      V v = cmake<V>((T)0, (T)0);
      if (xp < M) v = load_slot<V>(a, (long long)e * M + xp);
      buf[e * PP + p] = v;
    }
    __syncthreads();
    // C2R pre-processing: Z_k = (X_k + conj X_{h-k}) + i (X_k - conj X_{h-k}) conj(W^k), W = exp(-2 pi i / Nl)
    V zr[E];
    if (tid < nwork) {
#pragma unroll
      for (int b = 0; b < E; ++b) {
        const int w = tid + b * nwork;
        const int p = w & (P - 1), k = w >> a.lgP;
        V A = buf[k * PP + p];
        V Bc = cconj(buf[(h - k) * PP + p]);
        if (k == 0) { A.y = (T)0; Bc.y = (T)0; }     // edge planes: real part only
        const V s = cadd(A, Bc);
        const V d = cmul_i(cmulconj(csub(A, Bc), __ldg(&twN[k])));
        zr[b] = cadd(s, d);
      }
    }
    __syncthreads();
    if (tid < nwork) {
#pragma unroll
      for (int b = 0; b < E; ++b) {
        const int w = tid + b * nwork;
        buf[(w >> a.lgP) * PP + (w & (P - 1))] = zr[b];
      }
    }
    __syncthreads();
    fft_tile_l<E, true, LC>(buf, a.plan, a.lgP, PP, twh, tid, nwork);
    const T invn = (T)a.inv_n;
    // mask and 1/n: Re z_j <-> sample 2j, Im z_j <-> sample 2j+1 of pencil x'
    if (tid < nwork) {
#pragma unroll
      for (int b = 0; b < E; ++b) {
        const int w = tid + b * nwork;
        const int p = w & (P - 1), j = w >> a.lgP;
        const int xp = x0 + p;
        const uint32_t mw = (xp < M) ? __ldg(&a.maskw[(size_t)((2 * j) >> 5) * M + xp]) : 0u;
        const T m0 = ((mw >> ((2 * j) & 31)) & 1u) ? invn : (T)0;
        const T m1 = ((mw >> ((2 * j + 1) & 31)) & 1u) ? invn : (T)0;
        V z = buf[j * PP + p];
        z.x *= m0;
        z.y *= m1;
        buf[j * PP + p] = z;
      }
    }
    __syncthreads();
  }
  fft_tile_l<E, false, LC>(buf, a.plan, a.lgP, PP, twh, tid, nwork);
  // R2C post-processing: X'_k = (Z_k + conj Z_{h-k})/2 - i W^k (Z_k - conj Z_{h-k})/2, X'_h = Re Z_0 - Im Z_0
  double acc = 0.0;
  auto store_all = [&](auto pq) {
    if (tid < nwork) {
#pragma unroll
      for (int b = 0; b < E; ++b) {
        const int w = tid + b * nwork;
        const int p = w & (P - 1), k = w >> a.lgP;
        const int xp = x0 + p;
        const V zk = buf[k * PP + p];
        const V zc = cconj(buf[((h - k) % h) * PP + p]);
        const V s = cscale(cadd(zk, zc), (T)0.5);
        const V d = cscale(csub(zk, zc), (T)0.5);
        const V X = csub(s, cmul_i(cmul(__ldg(&twN[k]), d)));
        if (xp < M) {
          store_slot<V, decltype(pq)::value>(a, (long long)k * M + xp, X, acc);
          if (k == 0) store_slot<V, decltype(pq)::value>(a, (long long)h * M + xp, cmake<V>(zk.x - zk.y, (T)0), acc);
        }
      }
    }
  };
  if (a.pcg_mode) store_all(std::true_type{});
  else store_all(std::false_type{});
  if (a.mapout == MAPOUT_K && a.pcg_mode) finish_pq(a, acc, scratch);
}

template <typename T, int E, int LC>
cudaError_t launch_typed(int kind, bool inv, const PassArgs& a, int threads, size_t smem, dim3 grid, cudaStream_t st) {
  void (*fn)(PassArgs) = nullptr;
  if (kind == 0) fn = inv ? row_pass_kernel<T, E, true, LC> : row_pass_kernel<T, E, false, LC>;
  else if (kind == 1) fn = inv ? col_pass_kernel<T, E, true, LC> : col_pass_kernel<T, E, false, LC>;
  else fn = middle_pass_kernel<T, E, LC>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  fn<<<grid, threads, smem, st>>>(a);
  return cudaGetLastError();
}

// Power-of-two lengths 128, 256 and 512 run kernels with the length (and so
// the whole stage schedule) fixed at compile time.
template <typename T, int E>
cudaError_t launch_l(int kind, bool inv, const PassArgs& a, int threads, size_t smem, dim3 grid, cudaStream_t st) {
  if constexpr (E == 4 || E == 8 || E == 16) {
    switch (a.plan.L) {
      case 128: return launch_typed<T, E, 128>(kind, inv, a, threads, smem, grid, st);
      case 256: return launch_typed<T, E, 256>(kind, inv, a, threads, smem, grid, st);
      case 512: return launch_typed<T, E, 512>(kind, inv, a, threads, smem, grid, st);
      default: break;
    }
  }
  return launch_typed<T, E, 0>(kind, inv, a, threads, smem, grid, st);
}

template <typename T>
cudaError_t launch_e(int kind, bool inv, int E, const PassArgs& a, int threads, size_t smem, dim3 grid, cudaStream_t st) {
  switch (E) {
    case 4: return launch_l<T, 4>(kind, inv, a, threads, smem, grid, st);
    case 6: return launch_l<T, 6>(kind, inv, a, threads, smem, grid, st);
    case 8: return launch_l<T, 8>(kind, inv, a, threads, smem, grid, st);
    case 12: return launch_l<T, 12>(kind, inv, a, threads, smem, grid, st);
    case 16: return launch_l<T, 16>(kind, inv, a, threads, smem, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace
}  // namespace sdft
