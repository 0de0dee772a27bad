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
// a real transform of length Nl: for even Nl a complex one of length Nl/2 per
// pencil, for odd Nl one complex transform of length Nl per two pencils.
//
// The beta -> v map is folded into the first pass.  On the edge planes (kl = 0,
// and kl = Nl/2 for even Nl) only representatives carry data; instead of filling
// their conjugate twins we feed 2 v at the representative and 0 at the twin, and
// the middle pass keeps only the real part of those planes.  After the
// in-plane inverse transforms the edge planes of the true (Hermitian) input are
// real, and Re(sum_k 2 v_k e_k) over representatives plus the self-conjugate
// terms equals that real value, so the result is exact.
// Included by fft_passes_f32.cu and fft_passes_f64.cu (one precision each).
#pragma once

#include <type_traits>

#include "fft_reg.cuh"
#include "internal.h"
#include "mbarrier.cuh"

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

// Load the complex value of slot g for the first pass (one slot at a time).
// The FP64 vectors stream through with the evict-first hint (ld/st .cs) so
// that the pass-to-pass work buffer (67.6 MB in FP32 at 256^3) keeps its place
// in L2.
template <typename V>
__device__ __forceinline__ V load_slot(const PassArgs& a, long long g) {
  if (a.mapin == MAPIN_NONE) return reinterpret_cast<const V*>(a.buf)[g];
  const int cls = slot_class(a.lay, g);
  if (a.mapin == MAPIN_BETA) {
    const double2 b = __ldcs(reinterpret_cast<const double2*>(a.src) + g);
    return map_in<V>(cls, b.x, b.y);
  }
  // MAPIN_PCG: fused PCG direction update p = z + beta_cg * p on both blocks of the slot
  const long long H2 = a.lay.H;
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

// A pass inside a loop returns at once when its product is not wanted: PCG
// products once PCG has stopped, the FP64 replacement products unless asked
// for, and the incremental-G-beta residual product unless an exact one is due.
__device__ __forceinline__ bool pass_skipped(const PassArgs& a) {
  return (a.check_done && a.sc->cg_done) || (a.check_refine && !a.sc->refine_now) ||
         (a.check_exact && !a.sc->exact_now);
}

// FP64 operands of the K epilogue for one slot: p on both blocks and the two
// diagonal coefficients of K.
struct KIn {
  double2 pb, pz, l1, l2;
};

__device__ __forceinline__ KIn k_load(const PassArgs& a, long long g) {
  const long long H2 = a.lay.H;    // offset of the z block, in double2 units
  const double2* p2 = reinterpret_cast<const double2*>(a.p);
  KIn k;
  k.pb = __ldcs(p2 + g);
  k.pz = __ldcs(p2 + H2 + g);
  k.l1 = __ldcs(reinterpret_cast<const double2*>(a.lam1) + g);
  k.l2 = __ldcs(reinterpret_cast<const double2*>(a.lam2) + g);
  return k;
}

// The same operands for a whole tile of n consecutive slots g0 .. g0 + n - 1, staged in
// shared memory as four arrays of n double2 (p_beta, p_z, Lambda1, Lambda2).
struct KStage {
  const double2* s = nullptr;
  long long g0 = 0;
  int n = 0;
};

__device__ __forceinline__ KIn k_load_staged(const KStage& ks, long long g) {
  const int i = (int)(g - ks.g0);
  KIn k;
  k.pb = ks.s[i];
  k.pz = ks.s[ks.n + i];
  k.l1 = ks.s[2 * ks.n + i];
  k.l2 = ks.s[3 * ks.n + i];
  return k;
}

// Thread 0 of a forward row pass with the K epilogue, before the tile is loaded:
// start moving the tile's operands (kstage 1: into L2; kstage 2: into shared memory at
// dst, completing on the mbarrier bar).  The operand rows are contiguous (a row pass
// tile is P consecutive rows), so each of the four arrays is one bulk copy of 16 n bytes;
// the launcher guarantees 16-byte aligned operand pointers.
__device__ __forceinline__ void k_stage_issue(const PassArgs& a, const KStage& ks, unsigned char* dst,
                                              unsigned long long* bar) {
  const uint32_t bytes = (uint32_t)ks.n * 16u;
  const double2* p2 = reinterpret_cast<const double2*>(a.p);
  const void* src[4] = {p2 + ks.g0, p2 + a.lay.H + ks.g0, reinterpret_cast<const double2*>(a.lam1) + ks.g0,
                        reinterpret_cast<const double2*>(a.lam2) + ks.g0};
  if (a.kstage == 1) {
#pragma unroll
    for (int j = 0; j < 4; ++j) bulk_prefetch_l2(src[j], bytes);
    return;
  }
  const uint32_t b = smem_u32(bar);
  mbar_init(b, 1);
  mbar_fence_init();
  mbar_expect_tx(b, 4u * bytes);
  const int ncopy = a.kst_wait_log2 ? 3 : 4;     // the failure-detection test leaves one out
  for (int j = 0; j < ncopy; ++j) bulk_load(smem_u32(dst) + (uint32_t)j * bytes, src[j], bytes, b);
}

// q = [G p_b + L1 p_b + L2 p_z ; L2 p_b + L1 p_z] for slot g from (G p_b)_g = w;
// inside PCG also adds this slot's share of p^T q to acc.
template <typename V, bool PQ>
__device__ __forceinline__ void k_store(const PassArgs& a, long long g, V w, const KIn& k, double& acc) {
  const int cls = slot_class(a.lay, g);
  double o0, o1;
  map_out(cls, w, 1.0, o0, o1);
  double2 qb, qz;
  qb.x = o0 + k.l1.x * k.pb.x + k.l2.x * k.pz.x;
  qb.y = o1 + k.l1.y * k.pb.y + k.l2.y * k.pz.y;
  qz.x = k.l2.x * k.pb.x + k.l1.x * k.pz.x;
  qz.y = k.l2.y * k.pb.y + k.l1.y * k.pz.y;
  double2* q2 = reinterpret_cast<double2*>(a.q);
  __stcs(q2 + g, qb);
  __stcs(q2 + a.lay.H + g, qz);
  if (a.gp_out) __stcs(reinterpret_cast<double2*>(a.gp_out) + g, make_double2(o0, o1));
  if constexpr (PQ) {       // four FMAs into the running sum (the FP64 pipe bounds this pass)
    acc = fma(k.pb.x, qb.x, acc);
    acc = fma(k.pb.y, qb.y, acc);
    acc = fma(k.pz.x, qz.x, acc);
    acc = fma(k.pz.y, qz.y, acc);
  }
}

// Store the complex value of slot g for the last pass (one slot at a time:
// used where the operands need no batching).
template <typename V, bool PQ>
__device__ __forceinline__ void store_slot(const PassArgs& a, long long g, V w, double& acc,
                                           const KStage* ks = nullptr) {
  if (a.mapout == MAPOUT_NONE) {
    reinterpret_cast<V*>(a.buf)[g] = w;
    return;
  }
  if (a.mapout == MAPOUT_BETA) {
    double o0, o1;
    map_out(slot_class(a.lay, g), w, a.out_scale, o0, o1);
    __stcs(reinterpret_cast<double2*>(a.dst) + g, make_double2(o0, o1));
    return;
  }
  k_store<V, PQ>(a, g, w, ks ? k_load_staged(*ks, g) : k_load(a, g), acc);
}

// Loads of the E elements b = 0..E-1 of a thread: `elem(b, g)` gives the global
// slot g (false outside the grid: value 0) and `sink(b, v)` takes the value.
// Plain work-buffer loads are all issued before the first value is used (a
// tile waits for one memory latency, not E).  Mapped inputs (beta layout, the
// PCG update p = z + beta p) go one slot at a time: these passes are bound by
// HBM and the FP64 pipe, and holding several slots' FP64 operands costs more
// registers, and so resident warps, than the latency it hides.  MAPPED kernels
// (the first pass of a product) carry the mapping code; in the others a mapped
// input takes the generic one-slot path.
template <typename V, int E, bool MAPPED, typename F, typename S>
__device__ __forceinline__ void load_vals(const PassArgs& a, F&& elem, S&& sink) {
  using T = decltype(V::x);
  const V zero = cmake<V>((T)0, (T)0);
  if (a.mapin == MAPIN_NONE) {
    const V* src = reinterpret_cast<const V*>(a.buf);
    V v[E];
#pragma unroll
    for (int b = 0; b < E; ++b) {
      long long g;
      v[b] = elem(b, g) ? src[g] : zero;
    }
#pragma unroll
    for (int b = 0; b < E; ++b) sink(b, v[b]);
    return;
  }
  if constexpr (!MAPPED) {
#pragma unroll
    for (int b = 0; b < E; ++b) {
      long long g;
      sink(b, elem(b, g) ? load_slot<V>(a, g) : zero);
    }
  } else if (a.mapin == MAPIN_BETA) {
    const double2* src = reinterpret_cast<const double2*>(a.src);
#pragma unroll
    for (int b = 0; b < E; ++b) {
      long long g;
      V v = zero;
      if (elem(b, g)) {
        const double2 r = __ldcs(src + g);
        v = map_in<V>(slot_class(a.lay, g), r.x, r.y);
      }
      sink(b, v);
    }
  } else {
    // MAPIN_PCG: p = z + beta_cg p on both blocks of the slot
    const long long H2 = a.lay.H;
    const double bc = a.sc->beta_cg;
    double2* p2 = reinterpret_cast<double2*>(a.p);
    const double2* z2 = reinterpret_cast<const double2*>(a.zv);
#pragma unroll
    for (int b = 0; b < E; ++b) {
      long long g;
      V v = zero;
      if (elem(b, g)) {
        double2 pb = __ldcs(p2 + g), pz = __ldcs(p2 + H2 + g);
        const double2 zb = __ldcs(z2 + g), zz = __ldcs(z2 + H2 + g);
        pb.x = zb.x + bc * pb.x;
        pb.y = zb.y + bc * pb.y;
        pz.x = zz.x + bc * pz.x;
        pz.y = zz.y + bc * pz.y;
        __stcs(p2 + g, pb);
        __stcs(p2 + H2 + g, pz);
        v = map_in<V>(slot_class(a.lay, g), pb.x, pb.y);
      }
      sink(b, v);
    }
  }
}

// Stores of the E values src(b) to the slots named by `elem` (one slot at a
// time; the K epilogue loads its FP64 operands per slot, as above).  Issuing the
// loads of four slots before their stores was measured: it raised the forward row
// kernel from 48 to 112 registers and made the 256^3 product slower (0.324 -> 0.379 ms).
template <typename V, int E, bool PQ, typename F, typename S>
__device__ __forceinline__ void store_vals(const PassArgs& a, double& acc, F&& elem, S&& src,
                                           const KStage* ks = nullptr) {
#pragma unroll
  for (int b = 0; b < E; ++b) {
    long long g;
    if (elem(b, g)) store_slot<V, PQ>(a, g, src(b), acc, ks);
  }
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
    } else if (!a.cr_mode) {
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
  __shared__ __align__(8) unsigned long long kbar;   // staged K operands (kstage 2)
  pdl_wait();
  count_launch(a.sc);
  if (pass_skipped(a)) return;
  V* buf = reinterpret_cast<V*>(smem_raw);
  const int PP = a.PP, L = LC > 0 ? LC : a.plan.L, nwork = a.nwork, tid = threadIdx.x;
  const long long row0 = (long long)blockIdx.x << a.lgP;
  // forward pass with the K epilogue: the tile's FP64 operands start moving now and
  // arrive while the tile is loaded and transformed
  int kst = 0;
  KStage ks;
  if constexpr (!INV) {
    if (a.mapout == MAPOUT_K && a.kstage != 0) {
      kst = a.kstage;
      const long long rows = min((long long)1 << a.lgP, a.npencils - row0);
      ks.g0 = row0 * L;
      ks.n = (int)(rows * L);
      ks.s = reinterpret_cast<const double2*>(smem_raw + a.kst_off);
      if (tid == 0) k_stage_issue(a, ks, smem_raw + a.kst_off, &kbar);
    }
  }
  // element b of a working thread: idx = tid + b nwork, pencil idx / L, position idx % L
  // (consecutive threads walk one row: coalesced global access)
  auto sidx = [&](int b) {
    const int idx = tid + b * nwork;
    const int p = idx / L;
    return (idx - p * L) * PP + p;
  };
  auto elem = [&](int b, long long& g) -> bool {
    const int idx = tid + b * nwork;
    const int p = idx / L;
    const long long row = row0 + p;
    g = row * L + (idx - p * L);
    return row < a.npencils;
  };
  // inverse row passes start a product (beta-layout input), forward ones end it
  if (tid < nwork) load_vals<V, E, INV>(a, elem, [&](int b, V v) { buf[sidx(b)] = v; });
  __syncthreads();
  fft_tile_l<E, INV, LC>(buf, a.plan, a.lgP, PP, reinterpret_cast<const V*>(a.tw), tid, nwork);
  double acc = 0.0;
  // staged operands: wait (bounded) for the copies; if the wait gives up, the tile
  // writes nothing, records the expiry for the host (IPM_TIMEOUT) and waits once more,
  // again bounded, so that no copy is still landing in shared memory when it exits
  bool ready = true;
  if (kst == 2 && tid < nwork) {
    const unsigned limit = a.kst_wait_log2 ? (1u << a.kst_wait_log2) : kWaitLimit;
    ready = mbar_wait(smem_u32(&kbar), 0, limit);
    if (!ready) {
      a.sc->wait_expired = 1;
      mbar_wait(smem_u32(&kbar), 0, limit);
    }
  }
  if (tid < nwork && ready) {
    auto src = [&](int b) { return buf[sidx(b)]; };
    const KStage* kp = kst == 2 ? &ks : nullptr;
    if (a.pcg_mode) store_vals<V, E, true>(a, acc, elem, src, kp);
    else store_vals<V, E, false>(a, acc, elem, src, kp);
  }
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
  pdl_wait();
  count_launch(a.sc);
  if (pass_skipped(a)) return;
  V* buf = reinterpret_cast<V*>(smem_raw);
  const int P = 1 << a.lgP, PP = a.PP, nwork = a.nwork, tid = threadIdx.x;
  const int N1 = a.lay.N1;
  const int k1_0 = blockIdx.x * P;
  const long long plane = (long long)blockIdx.y * a.lay.N0;     // kl * N0
  // element b of a working thread: idx = tid + b nwork, row idx >> lgP, pencil idx & (P - 1)
  auto sidx = [&](int b) {
    const int idx = tid + b * nwork;
    return (idx >> a.lgP) * PP + (idx & (P - 1));
  };
  auto elem = [&](int b, long long& g) -> bool {
    const int idx = tid + b * nwork;
    const int k1 = k1_0 + (idx & (P - 1));
    g = (plane + (idx >> a.lgP)) * N1 + k1;
    return k1 < N1;
  };
  if (tid < nwork) load_vals<V, E, false>(a, elem, [&](int b, V v) { buf[sidx(b)] = v; });
  __syncthreads();
  fft_tile_l<E, INV, LC>(buf, a.plan, a.lgP, PP, reinterpret_cast<const V*>(a.tw), tid, nwork);
  if (tid < nwork) {
    V* g = reinterpret_cast<V*>(a.buf);
#pragma unroll
    for (int b = 0; b < E; ++b) {
      long long gi;
      if (elem(b, gi)) g[gi] = buf[sidx(b)];
    }
  }
}

// ---------------------------------------------------------------------------
// Middle pass for even Nl: pencils along the halved axis (Hl complex, stride
// M), P consecutive in-plane positions x' per tile.  Computes, per pencil,
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
  pdl_wait();
  count_launch(a.sc);
  if (pass_skipped(a)) return;
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
    // load X (Hl = h + 1 rows): rows 0..h-1 E per working thread, batched, then row h
    if (tid < nwork) {
      auto elem = [&](int b, long long& g) -> bool {
        const int idx = tid + b * nwork;
        const int xp = x0 + (idx & (P - 1));
        g = (long long)(idx >> a.lgP) * M + xp;
        return xp < M;
      };
      load_vals<V, E, false>(a, elem, [&](int b, V v) {
        const int idx = tid + b * nwork;
        buf[(idx >> a.lgP) * PP + (idx & (P - 1))] = v;
      });
      for (int p = tid; p < P; p += nwork) {
        const int xp = x0 + p;
        buf[h * PP + p] = (xp < M) ? load_slot<V>(a, (long long)h * M + xp) : cmake<V>((T)0, (T)0);
      }
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

// ---------------------------------------------------------------------------
// Middle pass for an odd halved-axis length Nl = 2 h + 1 (Sec. 3, the subspace
// F for odd n: v_0 real and the pairs k = 1 .. h; no Nyquist plane, so the
// edge plane is kl = 0 alone).  The real transforms of two pencils a and b run
// as ONE complex transform of length Nl: with the full Hermitian columns
// Y[Nl - k] = conj Y[k] of both, the inverse transform of Y_a + i Y_b is
// y_a + i y_b with y_a, y_b real; after the mask the forward transform W of
// m_a y_a / n + i m_b y_b / n separates as
//   Y'_a[k] = (W_k + conj W_{-k}) / 2,   Y'_b[k] = (W_k - conj W_{-k}) / (2 i).
// A tile holds P pencil pairs: pencils x0 + q (a) and x0 + P + q (b).  The
// half spectra (h + 1 slots each) are staged first, one load per slot (the
// PCG-form load also writes p back), then expanded to the Nl rows of the tile.
// With from_real the input is the real signal y * m itself and only the
// forward transform runs.
// ---------------------------------------------------------------------------
template <typename T, int E>
__global__ void __launch_bounds__(E == 16 ? 256 : 512, 1) middle_odd_kernel(PassArgs a) {
  using V = typename cvec<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double scratch[32];
  pdl_wait();
  count_launch(a.sc);
  if (pass_skipped(a)) return;
  V* buf = reinterpret_cast<V*>(smem_raw);       // FFT rows 0..Nl-1, P pairs each (stride PP)
  const int lgP = a.lgP, P = 1 << lgP, PP = a.PP;
  const int Nl = a.lay.Nl, h = Nl >> 1, M = a.lay.M;
  const int x0 = blockIdx.x * 2 * P;
  const int tid = threadIdx.x, nwork = a.nwork, nthr = blockDim.x;
  const V* tw = reinterpret_cast<const V*>(a.tw);
  const V zero = cmake<V>((T)0, (T)0);
  auto mask_bit = [&](int x, int n) -> bool {
    return x < M && ((__ldg(&a.maskw[(size_t)(n >> 5) * M + x]) >> (n & 31)) & 1u);
  };

  if (a.from_real) {
    for (int idx = tid; idx < P * Nl; idx += nthr) {
      const int q = idx & (P - 1), n = idx >> lgP;
      const int xa = x0 + q, xb = xa + P;
      const T va = mask_bit(xa, n) ? (T)a.yreal[(size_t)xa * Nl + n] : (T)0;
      const T vb = mask_bit(xb, n) ? (T)a.yreal[(size_t)xb * Nl + n] : (T)0;
      buf[n * PP + q] = cmake<V>(va, vb);
    }
    __syncthreads();
  } else {
    // stage the half spectra: X[kl * 2P + pp] = slot kl * M + x0 + pp
    V* X = buf;
    for (int idx = tid; idx < (h + 1) * 2 * P; idx += nthr) {
      const int pp = idx & (2 * P - 1), kl = idx >> (lgP + 1);
      const int x = x0 + pp;
      X[idx] = (x < M) ? load_slot<V>(a, (long long)kl * M + x) : zero;
    }
    __syncthreads();
    // Z[k] = Y_a[k] + i Y_b[k]; on the edge plane kl = 0 only the real part is kept
    V zr[E];
    if (tid < nwork) {
#pragma unroll
      for (int b = 0; b < E; ++b) {
        const int w = tid + b * nwork;
        const int q = w & (P - 1), k = w >> lgP;
        const bool cj = k > h;
        const int kk = cj ? Nl - k : k;
        V ya = X[kk * 2 * P + q], yb = X[kk * 2 * P + P + q];
        if (kk == 0) { ya.y = (T)0; yb.y = (T)0; }
        if (cj) { ya = cconj(ya); yb = cconj(yb); }
        zr[b] = cmake<V>(ya.x - yb.y, ya.y + yb.x);
      }
    }
    __syncthreads();
    if (tid < nwork) {
#pragma unroll
      for (int b = 0; b < E; ++b) {
        const int w = tid + b * nwork;
        buf[(w >> lgP) * PP + (w & (P - 1))] = zr[b];
      }
    }
    __syncthreads();
    fft_tile<E, true, true>(buf, a.plan, lgP, PP, tw, tid, nwork);
    // mask and 1/n: Re <-> sample n of pencil a, Im <-> sample n of pencil b
    const T invn = (T)a.inv_n;
    if (tid < nwork) {
#pragma unroll
      for (int b = 0; b < E; ++b) {
        const int w = tid + b * nwork;
        const int q = w & (P - 1), n = w >> lgP;
        V z = buf[n * PP + q];
        z.x *= mask_bit(x0 + q, n) ? invn : (T)0;
        z.y *= mask_bit(x0 + P + q, n) ? invn : (T)0;
        buf[n * PP + q] = z;
      }
    }
    __syncthreads();
  }
  fft_tile<E, false, true>(buf, a.plan, lgP, PP, tw, tid, nwork);
  double acc = 0.0;
  auto store_all = [&](auto pq) {
    for (int idx = tid; idx < (h + 1) * P; idx += nthr) {
      const int q = idx & (P - 1), k = idx >> lgP;
      const V wk = buf[k * PP + q];
      const V wc = cconj(buf[(k == 0 ? 0 : Nl - k) * PP + q]);
      const V ya = cscale(cadd(wk, wc), (T)0.5);
      const V d = csub(wk, wc);
      const V yb = cmake<V>(d.y * (T)0.5, -d.x * (T)0.5);
      const int xa = x0 + q, xb = xa + P;
      if (xa < M) store_slot<V, decltype(pq)::value>(a, (long long)k * M + xa, ya, acc);
      if (xb < M) store_slot<V, decltype(pq)::value>(a, (long long)k * M + xb, yb, acc);
    }
  };
  if (a.pcg_mode) store_all(std::true_type{});
  else store_all(std::false_type{});
  if (a.mapout == MAPOUT_K && a.pcg_mode) finish_pq(a, acc, scratch);
}

// ---------------------------------------------------------------------------
// Register-engine passes (fft_reg.cuh): lengths fixed at compile time, E = 16
// values per thread, the first stage loading from and the last stage storing to
// global memory; shared memory only for the exchanges between stages.
// ---------------------------------------------------------------------------
// Row pass: P rows of length L per block, TT = L / E consecutive threads per
// row (coalesced along the row); shared memory pencil-major with one pad slot
// per 16 elements (conflict-free for the stride-R exchange writes).
template <typename T, int L, int E, bool INV>
__global__ void __launch_bounds__(256) row_reg_kernel(PassArgs a) {
  using V = typename cvec<T>::type;
  constexpr int TT = L / E, LP = L + L / 16;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double scratch[32];
  pdl_wait();
  count_launch(a.sc);
  if (pass_skipped(a)) return;
  const int tid = threadIdx.x, t = tid % TT, p = tid / TT;
  const long long row = ((long long)blockIdx.x << a.lgP) + p;
  const bool ok = row < a.npencils;
  V* sm = reinterpret_cast<V*>(smem_raw) + p * LP;
  auto elem = [&](int m, long long& g) -> bool {
    g = row * L + t + TT * m;
    return ok;
  };
  V x[E];
  load_vals<V, E, INV>(a, elem, [&](int m, V v) { x[m] = v; });
  reg_fft<E, INV, L>(x, t, reinterpret_cast<const V*>(a.tw), sm, [](int e) { return e + (e >> 4); });
  double acc = 0.0;
  auto src = [&](int m) { return x[m]; };
  if (a.pcg_mode) store_vals<V, E, true>(a, acc, elem, src);
  else store_vals<V, E, false>(a, acc, elem, src);
  if (a.mapout == MAPOUT_K && a.pcg_mode) finish_pq(a, acc, scratch);
}

// Column pass (d = 3): P consecutive k1 per block (pencil index fastest across
// threads: coalesced), TT = L / E threads per pencil; grid = (ceil(N1 / P), Hl).
template <typename T, int L, int E, bool INV>
__global__ void __launch_bounds__(256) col_reg_kernel(PassArgs a) {
  using V = typename cvec<T>::type;
  constexpr int TT = L / E;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pdl_wait();
  count_launch(a.sc);
  if (pass_skipped(a)) return;
  const int lgP = a.lgP, tid = threadIdx.x, p = tid & ((1 << lgP) - 1), t = tid >> lgP;
  const int N1 = a.lay.N1, k1 = (blockIdx.x << lgP) + p;
  const long long plane = (long long)blockIdx.y * a.lay.N0;     // kl * N0
  auto elem = [&](int m, long long& g) -> bool {
    g = (plane + t + TT * m) * N1 + k1;
    return k1 < N1;
  };
  V x[E];
  load_vals<V, E, false>(a, elem, [&](int m, V v) { x[m] = v; });
  reg_fft<E, INV, L>(x, t, reinterpret_cast<const V*>(a.tw), reinterpret_cast<V*>(smem_raw),
                     [&](int e) { return (e << lgP) + p; });
  V* gb = reinterpret_cast<V*>(a.buf);
#pragma unroll
  for (int m = 0; m < E; ++m) {
    long long g;
    if (elem(m, g)) gb[g] = x[m];
  }
}

// Middle pass: the real transform of length Nl = 2 H along the halved axis, P
// consecutive in-plane positions per block (pencil index fastest), TT = H / E
// threads per pencil.  Shared memory: one (H + 1) x P tile, holding the loaded
// half spectrum, then every exchange of both transforms, then the spectrum for
// the post-processing.  Same arithmetic as middle_pass_kernel: C2R
// pre-processing, inverse transform, mask and 1/n, forward transform, R2C
// post-processing; the inverse transform leaves element t + TT m in the
// registers from which the forward one starts, so no exchange joins them.  The
// FP32 kernel is held to 64 registers (no spills), so that 8 blocks of 128
// threads share an SM.
template <typename T, int H, int E>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 1) mid_reg_kernel(PassArgs a) {
  using V = typename cvec<T>::type;
  constexpr int TT = H / E;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double scratch[32];
  pdl_wait();
  count_launch(a.sc);
  if (pass_skipped(a)) return;
  const int lgP = a.lgP, tid = threadIdx.x, p = tid & ((1 << lgP) - 1), t = tid >> lgP;
  const int M = a.lay.M, Nl = a.lay.Nl, xp = (blockIdx.x << lgP) + p;
  const bool ok = xp < M;
  V* tile = reinterpret_cast<V*>(smem_raw);          // rows 0..H
  auto at = [&](int e) { return (e << lgP) + p; };
  const V* twh = reinterpret_cast<const V*>(a.tw);
  const V* twN = reinterpret_cast<const V*>(a.twN);
  V x[E];
  if (a.from_real) {
    // z_j = (y m)[2j] + i (y m)[2j+1] of the signal row of pencil xp
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const int j = t + TT * m;
      T v0 = (T)0, v1 = (T)0;
      if (ok) {
        const uint32_t w = a.maskw[(size_t)((2 * j) >> 5) * M + xp];
        const double y0 = a.yreal[(size_t)xp * Nl + 2 * j];
        const double y1 = a.yreal[(size_t)xp * Nl + 2 * j + 1];
        v0 = (T)(((w >> ((2 * j) & 31)) & 1u) ? y0 : 0.0);
        v1 = (T)(((w >> ((2 * j + 1) & 31)) & 1u) ? y1 : 0.0);
      }
      x[m] = cmake<V>(v0, v1);
    }
  } else {
    {
      auto elem = [&](int m, long long& g) -> bool {
        g = (long long)(t + TT * m) * M + xp;
        return ok;
      };
      load_vals<V, E, false>(a, elem, [&](int m, V v) { tile[at(t + TT * m)] = v; });
      if (t == 0) tile[at(H)] = ok ? load_slot<V>(a, (long long)H * M + xp) : cmake<V>((T)0, (T)0);
    }
    __syncthreads();
    // C2R pre-processing: Z_k = (X_k + conj X_{H-k}) + i (X_k - conj X_{H-k}) conj(W^k), W = exp(-2 pi i / Nl)
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const int k = t + TT * m;
      V A = tile[at(k)];
      V Bc = cconj(tile[at(H - k)]);
      if (k == 0) { A.y = (T)0; Bc.y = (T)0; }     // edge planes: real part only
      const V sum = cadd(A, Bc);
      const V d = cmul_i(cmulconj(csub(A, Bc), __ldg(&twN[k])));
      x[m] = cadd(sum, d);
    }
    __syncthreads();                                 // pre-processing reads done: the tile is free
    reg_fft<E, true, H>(x, t, twh, tile, at);
    // mask and 1/n: Re z_j <-> sample 2j, Im z_j <-> sample 2j+1 of pencil xp
    const T invn = (T)a.inv_n;
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const int j = t + TT * m;
      const uint32_t mw = ok ? __ldg(&a.maskw[(size_t)(j >> 4) * M + xp]) : 0u;
      x[m].x *= ((mw >> ((2 * j) & 31)) & 1u) ? invn : (T)0;
      x[m].y *= ((mw >> ((2 * j + 1) & 31)) & 1u) ? invn : (T)0;
    }
  }
  // forward transform; its exchanges reuse the tile once every thread has read
  // its last exchange of the inverse transform
  if (!a.from_real) __syncthreads();
  reg_fft<E, false, H>(x, t, twh, tile, at);
  __syncthreads();                                   // last exchange reads done
#pragma unroll
  for (int m = 0; m < E; ++m) tile[at(t + TT * m)] = x[m];
  __syncthreads();
  // R2C post-processing: X'_k = (Z_k + conj Z_{H-k})/2 - i W^k (Z_k - conj Z_{H-k})/2, X'_H = Re Z_0 - Im Z_0
  double acc = 0.0;
  auto store_all = [&](auto pq) {
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const int k = t + TT * m;
      const V zk = tile[at(k)];
      const V zc = cconj(tile[at((H - k) & (H - 1))]);
      const V sum = cscale(cadd(zk, zc), (T)0.5);
      const V d = cscale(csub(zk, zc), (T)0.5);
      const V X = csub(sum, cmul_i(cmul(__ldg(&twN[k]), d)));
      if (ok) {
        store_slot<V, decltype(pq)::value>(a, (long long)k * M + xp, X, acc);
        if (k == 0) store_slot<V, decltype(pq)::value>(a, (long long)H * M + xp, cmake<V>(zk.x - zk.y, (T)0), acc);
      }
    }
  };
  if (a.pcg_mode) store_all(std::true_type{});
  else store_all(std::false_type{});
  if (a.mapout == MAPOUT_K && a.pcg_mode) finish_pq(a, acc, scratch);
}

template <typename T, int L>
cudaError_t launch_reg_l(int kind, bool inv, const PassArgs& a, int threads, size_t smem, dim3 grid, cudaStream_t st) {
  constexpr int E = 16;
  void (*fn)(PassArgs) = nullptr;
  if (kind == 0) fn = inv ? row_reg_kernel<T, L, E, true> : row_reg_kernel<T, L, E, false>;
  else if (kind == 1) fn = inv ? col_reg_kernel<T, L, E, true> : col_reg_kernel<T, L, E, false>;
  else fn = mid_reg_kernel<T, L, E>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  return launch_k(fn, grid, dim3(threads), smem, st, a);
}

// Register engine: E = 16 and L (for the middle pass h = Nl / 2) in {32, ..., 512}.
template <typename T>
cudaError_t launch_reg(int kind, bool inv, const PassArgs& a, int threads, size_t smem, dim3 grid, cudaStream_t st) {
  switch (a.plan.L) {
    case 32: return launch_reg_l<T, 32>(kind, inv, a, threads, smem, grid, st);
    case 64: return launch_reg_l<T, 64>(kind, inv, a, threads, smem, grid, st);
    case 128: return launch_reg_l<T, 128>(kind, inv, a, threads, smem, grid, st);
    case 256: return launch_reg_l<T, 256>(kind, inv, a, threads, smem, grid, st);
    case 512: return launch_reg_l<T, 512>(kind, inv, a, threads, smem, grid, st);
    default: return cudaErrorInvalidValue;
  }
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
  return launch_k(fn, grid, dim3(threads), smem, st, a);
}

// Power-of-two lengths 128, 256 and 512 run kernels with the length (and so
// the whole stage schedule) fixed at compile time.
template <typename T, int E>
cudaError_t launch_l(int kind, bool inv, const PassArgs& a, int threads, size_t smem, dim3 grid, cudaStream_t st) {
  if (kind == 2 && (a.lay.Nl & 1)) {
    void (*fn)(PassArgs) = middle_odd_kernel<T, E>;
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    return launch_k(fn, grid, dim3(threads), smem, st, a);
  }
  // 5s, 7s or more than one 3: the general-Ns odd stages
  int threes = 0;
  for (int s = 0; s < a.plan.nst; ++s) {
    if (a.plan.radix[s] == 5 || a.plan.radix[s] == 7) return launch_typed<T, E, -1>(kind, inv, a, threads, smem, grid, st);
    if (a.plan.radix[s] == 3) ++threes;
  }
  if (threes > 1) return launch_typed<T, E, -1>(kind, inv, a, threads, smem, grid, st);
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
