// Shared-memory Stockham FFT on a tile of P pencils (Sec. 3.1: the masked
// operators are applied with forward / inverse DFTs; this is our own
// mixed-radix, self-sorting formulation).
//
// Tile layout in shared memory: element e of pencil p lives at buf[e * PP + p]
// (pencil index fastest, PP = P or P + 1 to spread banks), so the threads of a
// warp, which walk p fastest, touch consecutive words.
//
// Each thread owns E complex values per stage (E/R butterflies of radix R;
// R in {2, 3, 4, 8, 16}, the radix-16 butterfly done as 4 x 4 in registers;
// radices 5 and 7, which need not divide E, take ceil(E/R) guarded butterflies).
// A stage reads all its inputs into registers, synchronises, then writes its
// outputs into the same buffer (Stockham autosort, decimation in time):
//     for butterfly j of a stage of radix R after Ns = R_1 ... R_{s-1}:
//       a_r = x[j + r L/R] * w_L^{(j mod Ns) r L/(Ns R)},   r = 0..R-1
//       a   = DFT_R(a)
//       y[(j div Ns) Ns R + (j mod Ns) + r Ns] = a_r
// Forward transforms use w_L = exp(-2 pi i / L), inverse ones its conjugate;
// neither is normalised.  Radix 3 (if present) is always the last stage, so Ns
// is a power of two in every stage.
#pragma once

#include "common.cuh"

namespace sdft {

constexpr double kSqrtHalf = 0.70710678118654752440;
constexpr double kSin60 = 0.86602540378443864676;

struct FftPlan {
  int L;           // transform length
  int nst;         // number of stages
  int radix[12];   // stage radices in application order
};

template <bool INV, typename V> __device__ __forceinline__ void dft2(V* a) {
  V t = a[0];
  a[0] = cadd(t, a[1]);
  a[1] = csub(t, a[1]);
}

template <bool INV, typename V> __device__ __forceinline__ void dft4(V* a) {
  V t0 = cadd(a[0], a[2]), t1 = csub(a[0], a[2]);
  V t2 = cadd(a[1], a[3]), t3 = csub(a[1], a[3]);
  V r3 = INV ? cmul_i(t3) : cmul_mi(t3);
  a[0] = cadd(t0, t2);
  a[2] = csub(t0, t2);
  a[1] = cadd(t1, r3);
  a[3] = csub(t1, r3);
}

template <bool INV, typename V> __device__ __forceinline__ void dft8(V* a) {
  using T = decltype(V::x);
  V e[4] = {a[0], a[2], a[4], a[6]};
  V o[4] = {a[1], a[3], a[5], a[7]};
  dft4<INV>(e);
  dft4<INV>(o);
  const T h = (T)kSqrtHalf;
  // o[q] *= w8^q with w8 = exp(-+ 2 pi i / 8)
  V o1 = INV ? cmake<V>((o[1].x - o[1].y) * h, (o[1].x + o[1].y) * h)
             : cmake<V>((o[1].x + o[1].y) * h, (o[1].y - o[1].x) * h);
  V o2 = INV ? cmul_i(o[2]) : cmul_mi(o[2]);
  V o3 = INV ? cmake<V>((-o[3].x - o[3].y) * h, (o[3].x - o[3].y) * h)
             : cmake<V>((o[3].y - o[3].x) * h, (-o[3].x - o[3].y) * h);
  a[0] = cadd(e[0], o[0]);
  a[4] = csub(e[0], o[0]);
  a[1] = cadd(e[1], o1);
  a[5] = csub(e[1], o1);
  a[2] = cadd(e[2], o2);
  a[6] = csub(e[2], o2);
  a[3] = cadd(e[3], o3);
  a[7] = csub(e[3], o3);
}

template <bool INV, typename V> __device__ __forceinline__ void dft3(V* a) {
  using T = decltype(V::x);
  const T s = INV ? (T)kSin60 : -(T)kSin60;
  V t1 = cadd(a[1], a[2]);
  V d = csub(a[1], a[2]);
  V m = cmake<V>(a[0].x - (T)0.5 * t1.x, a[0].y - (T)0.5 * t1.y);
  V isd = cmake<V>(-s * d.y, s * d.x);      // i * s * d
  a[0] = cadd(a[0], t1);
  a[1] = cadd(m, isd);
  a[2] = csub(m, isd);
}

// a * W16^e (forward: W16 = exp(-2 pi i / 16); inverse: its conjugate), e = 0..9
template <int e, bool INV, typename V> __device__ __forceinline__ V mul_w16(V a) {
  using T = decltype(V::x);
  constexpr double c1 = 0.92387953251128675613, s1 = 0.38268343236508977173, h = 0.70710678118654752440;
  constexpr double cs[10] = {1.0, c1, h, s1, 0.0, -s1, -h, -c1, -1.0, -c1};
  constexpr double sn[10] = {0.0, s1, h, c1, 1.0, c1, h, s1, 0.0, -s1};
  if constexpr (e == 0) return a;
  else {
    const T c = (T)cs[e], sg = INV ? (T)sn[e] : -(T)sn[e];   // W = c + i sg
    return cmake<V>(a.x * c - a.y * sg, a.x * sg + a.y * c);
  }
}

// 16-point DFT in registers as 4 x 4: with n = n1 + 4 n2 and k = k1 + 4 k2,
// X[k] = sum_n1 W4^{n1 k2} W16^{n1 k1} sum_n2 a[n1 + 4 n2] W4^{n2 k1}.
template <bool INV, typename V> __device__ __forceinline__ void dft16(V* a) {
  V t[4][4];
#pragma unroll
  for (int n1 = 0; n1 < 4; ++n1) {
    V u[4] = {a[n1], a[n1 + 4], a[n1 + 8], a[n1 + 12]};
    dft4<INV>(u);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) t[n1][k1] = u[k1];
  }
  t[1][1] = mul_w16<1, INV>(t[1][1]); t[1][2] = mul_w16<2, INV>(t[1][2]); t[1][3] = mul_w16<3, INV>(t[1][3]);
  t[2][1] = mul_w16<2, INV>(t[2][1]); t[2][2] = mul_w16<4, INV>(t[2][2]); t[2][3] = mul_w16<6, INV>(t[2][3]);
  t[3][1] = mul_w16<3, INV>(t[3][1]); t[3][2] = mul_w16<6, INV>(t[3][2]); t[3][3] = mul_w16<9, INV>(t[3][3]);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    V u[4] = {t[0][k1], t[1][k1], t[2][k1], t[3][k1]};
    dft4<INV>(u);
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) a[k1 + 4 * k2] = u[k2];
  }
}

// Odd prime R (5, 7): pairing x_n with x_{R-n}, a_n = x_n + x_{R-n}, b_n = x_n - x_{R-n},
// every output pair k, R-k shares A_k = x_0 + sum_n a_n cos(2 pi n k / R) and
// B_k = sum_n b_n sin(2 pi n k / R): forward X_k = A_k - i B_k, X_{R-k} = A_k + i B_k
// (inverse: the signs of i B_k swap), X_0 = x_0 + sum_n a_n.
// cos(2 pi m / R) and sin(2 pi m / R) for 0 <= m <= (R - 1) / 2, R in {5, 7}
__host__ __device__ constexpr double odd_cos(int R, int m) {
  return R == 5 ? (m == 0 ? 1.0 : m == 1 ? 0.30901699437494742410 : -0.80901699437494742410)
                : (m == 0 ? 1.0 : m == 1 ? 0.62348980185873353053 : m == 2 ? -0.22252093395631440429
                                                                           : -0.90096886790241912624);
}
__host__ __device__ constexpr double odd_sin(int R, int m) {
  return R == 5 ? (m == 0 ? 0.0 : m == 1 ? 0.95105651629515357212 : 0.58778525229247312917)
                : (m == 0 ? 0.0 : m == 1 ? 0.78183148246802980871 : m == 2 ? 0.97492791218182360702
                                                                           : 0.43388373911755812048);
}

template <int R, bool INV, typename V> __device__ __forceinline__ void dft_odd(V* a) {
  using T = decltype(V::x);
  constexpr int Q = (R - 1) / 2;
  V sum[Q + 1], dif[Q + 1];
  V x0 = a[0];
  V X0 = x0;
#pragma unroll
  for (int n = 1; n <= Q; ++n) {
    sum[n] = cadd(a[n], a[R - n]);
    dif[n] = csub(a[n], a[R - n]);
    X0 = cadd(X0, sum[n]);
  }
#pragma unroll
  for (int k = 1; k <= Q; ++k) {
    V A = x0, B = cmake<V>((T)0, (T)0);
#pragma unroll
    for (int n = 1; n <= Q; ++n) {
      // cos / sin of 2 pi n k / R from the table of the first Q + 1 multiples
      const int m = (n * k) % R;
      const int mm = m <= Q ? m : R - m;
      const T c = (T)odd_cos(R, mm);
      const T sn = m <= Q ? (T)odd_sin(R, mm) : -(T)odd_sin(R, mm);
      A = cmake<V>(A.x + c * sum[n].x, A.y + c * sum[n].y);
      B = cmake<V>(B.x + sn * dif[n].x, B.y + sn * dif[n].y);
    }
    const V iB = cmul_i(B);
    a[k] = INV ? cadd(A, iB) : csub(A, iB);
    a[R - k] = INV ? csub(A, iB) : cadd(A, iB);
  }
  a[0] = X0;
}

template <int R, bool INV, typename V> __device__ __forceinline__ void dft_r(V* a) {
  if constexpr (R == 2) dft2<INV>(a);
  else if constexpr (R == 3) dft3<INV>(a);
  else if constexpr (R == 4) dft4<INV>(a);
  else if constexpr (R == 8) dft8<INV>(a);
  else if constexpr (R == 5 || R == 7) dft_odd<R, INV>(a);
  else dft16<INV>(a);
}

// One Stockham stage of radix R over the tile.  nwork = P * L / E threads
// carry the work (threads beyond that only join the barriers).
template <int E, int R, bool INV, typename V>
__device__ __forceinline__ void fft_stage(V* buf, int L, int lgNs, int lgP, int PP, const V* __restrict__ tw,
                                          int tid, int nwork) {
  constexpr int B = E / R;
  const int Ns = 1 << lgNs;
  const int LR = L / R;
  const int twstride = L / (Ns * R);
  V a[B][R];
  const bool active = tid < nwork;
  if (active) {
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int w = tid + b * nwork;
      const int p = w & ((1 << lgP) - 1), j = w >> lgP, k = j & (Ns - 1);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        V v = buf[(j + r * LR) * PP + p];
        if (r > 0 && Ns > 1) {
          V t = __ldg(&tw[k * r * twstride]);
          v = INV ? cmulconj(v, t) : cmul(v, t);
        }
        a[b][r] = v;
      }
    }
  }
  __syncthreads();
  if (active) {
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int w = tid + b * nwork;
      const int p = w & ((1 << lgP) - 1), j = w >> lgP, k = j & (Ns - 1);
      dft_r<R, INV>(a[b]);
      const int base = ((j >> lgNs) << lgNs) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) buf[(base + r * Ns) * PP + p] = a[b][r];
    }
  }
  __syncthreads();
}

// One stage of an odd radix R in {3, 5, 7} that need not divide E: the P L / R
// butterflies w = tid + b nwork (b < ceil(E / R)) are spread over the working
// threads with a guard, and Ns (the product of the earlier radices) may be any
// integer.  Same formulas as fft_stage.
template <int E, int R, bool INV, typename V>
__device__ __forceinline__ void fft_stage_odd(V* buf, int L, int Ns, int lgP, int PP, const V* __restrict__ tw,
                                              int tid, int nwork) {
  constexpr int B = (E + R - 1) / R;
  const int LR = L / R;
  const int twstride = L / (Ns * R);
  const int nbfly = (LR << lgP);
  V a[B][R];
  const bool active = tid < nwork;
  if (active) {
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int w = tid + b * nwork;
      if (w < nbfly) {
        const int p = w & ((1 << lgP) - 1), j = w >> lgP, k = j % Ns;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          V v = buf[(j + r * LR) * PP + p];
          if (r > 0 && Ns > 1) {
            V t = __ldg(&tw[k * r * twstride]);
            v = INV ? cmulconj(v, t) : cmul(v, t);
          }
          a[b][r] = v;
        }
      }
    }
  }
  __syncthreads();
  if (active) {
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int w = tid + b * nwork;
      if (w < nbfly) {
        const int p = w & ((1 << lgP) - 1), j = w >> lgP, k = j % Ns;
        dft_r<R, INV>(a[b]);
        const int base = (j / Ns) * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) buf[(base + r * Ns) * PP + p] = a[b][r];
      }
    }
  }
  __syncthreads();
}

// Full transform of the P pencils held in buf (length plan.L each), in place.
// ODD: the plan may hold radix-5 / radix-7 stages or several radix-3 stages,
// all run by the guarded general-Ns stage (a separate instantiation, so that
// the registers of those stages do not weigh on the other kernels).
template <int E, bool INV, bool ODD, typename V>
__device__ __forceinline__ void fft_tile(V* buf, const FftPlan& plan, int lgP, int PP, const V* __restrict__ tw,
                                         int tid, int nwork) {
  int lgNs = 0, Ns = 1;
  for (int s = 0; s < plan.nst; ++s) {
    const int R = plan.radix[s];
    if constexpr (ODD) {
      // the odd radices come last (after the powers of two)
      if (R == 3 || R == 5 || R == 7) {
        if (R == 3) fft_stage_odd<E, 3, INV>(buf, plan.L, Ns, lgP, PP, tw, tid, nwork);
        if (R == 5) fft_stage_odd<E, 5, INV>(buf, plan.L, Ns, lgP, PP, tw, tid, nwork);
        if (R == 7) fft_stage_odd<E, 7, INV>(buf, plan.L, Ns, lgP, PP, tw, tid, nwork);
        Ns *= R;
        continue;
      }
    }
    Ns *= R;
    if constexpr (E % 16 == 0) {
      if (R == 16) fft_stage<E, 16, INV>(buf, plan.L, lgNs, lgP, PP, tw, tid, nwork);
    }
    if constexpr (E % 8 == 0) {
      if (R == 8) fft_stage<E, 8, INV>(buf, plan.L, lgNs, lgP, PP, tw, tid, nwork);
    }
    if constexpr (E % 4 == 0) {
      if (R == 4) fft_stage<E, 4, INV>(buf, plan.L, lgNs, lgP, PP, tw, tid, nwork);
    }
    if (R == 2) fft_stage<E, 2, INV>(buf, plan.L, lgNs, lgP, PP, tw, tid, nwork);
    if constexpr (!ODD && E % 3 == 0) {
      if (R == 3) fft_stage<E, 3, INV>(buf, plan.L, lgNs, lgP, PP, tw, tid, nwork);
    }
    lgNs += (R == 16) ? 4 : (R == 8) ? 3 : (R == 4 ? 2 : (R == 2 ? 1 : 0));   // odd radices come last
  }
}

// ---- compile-time lengths ------------------------------------------------
// For the common power-of-two lengths the stage schedule (the same as the
// host plan: 16s, then 8s, 4s, 2s as E allows) is fixed at compile time, so
// every stride, mask and twiddle step below is a constant.
__host__ __device__ constexpr int stage_radix_c(int L, int E, int s) {
  int m = L, r = 2;
  for (int i = 0; i <= s; ++i) {
    r = (E % 16 == 0 && m % 16 == 0) ? 16 : (E % 8 == 0 && m % 8 == 0) ? 8 : (E % 4 == 0 && m % 4 == 0) ? 4 : 2;
    if (i < s) m /= r;
  }
  return r;
}
__host__ __device__ constexpr int stage_count_c(int L, int E) {
  int m = L, n = 0;
  while (m > 1) { m /= stage_radix_c(m, E, 0); ++n; }
  return n;
}
__host__ __device__ constexpr int log2_c(int v) { return v <= 1 ? 0 : 1 + log2_c(v / 2); }

template <int E, int R, bool INV, int L, int LGNS, typename V>
__device__ __forceinline__ void fft_stage_c(V* buf, int lgP, int PP, const V* __restrict__ tw, int tid, int nwork) {
  constexpr int B = E / R, Ns = 1 << LGNS, LR = L / R, TWS = L / (Ns * R);
  V a[B][R];
  const bool active = tid < nwork;
  const int pmask = (1 << lgP) - 1, sLR = LR * PP, sNs = Ns * PP;
  if (active) {
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int w = tid + b * nwork;
      const int p = w & pmask, j = w >> lgP, k = j & (Ns - 1);
      const V* src = buf + j * PP + p;
      const int kt = k * TWS;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        V v = src[r * sLR];
        if (r > 0 && Ns > 1) {
          const V t = __ldg(tw + kt * r);
          v = INV ? cmulconj(v, t) : cmul(v, t);
        }
        a[b][r] = v;
      }
    }
  }
  __syncthreads();
  if (active) {
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int w = tid + b * nwork;
      const int p = w & pmask, j = w >> lgP, k = j & (Ns - 1);
      dft_r<R, INV>(a[b]);
      V* dst = buf + (((j >> LGNS) << LGNS) * R + k) * PP + p;
#pragma unroll
      for (int r = 0; r < R; ++r) dst[r * sNs] = a[b][r];
    }
  }
  __syncthreads();
}

template <int E, bool INV, int L, int S, int LGNS, typename V>
__device__ __forceinline__ void fft_stages_c(V* buf, int lgP, int PP, const V* __restrict__ tw, int tid, int nwork) {
  if constexpr (S < stage_count_c(L, E)) {
    constexpr int R = stage_radix_c(L, E, S);
    fft_stage_c<E, R, INV, L, LGNS>(buf, lgP, PP, tw, tid, nwork);
    fft_stages_c<E, INV, L, S + 1, LGNS + log2_c(R)>(buf, lgP, PP, tw, tid, nwork);
  }
}

// Full transform with the length fixed at compile time (LC > 0) or taken from
// the plan (LC = 0; LC = -1 for plans with a radix-5 or radix-7 stage).
template <int E, bool INV, int LC, typename V>
__device__ __forceinline__ void fft_tile_l(V* buf, const FftPlan& plan, int lgP, int PP, const V* __restrict__ tw,
                                           int tid, int nwork) {
  if constexpr (LC > 0) fft_stages_c<E, INV, LC, 0, 0>(buf, lgP, PP, tw, tid, nwork);
  else fft_tile<E, INV, (LC < 0)>(buf, plan, lgP, PP, tw, tid, nwork);
}

}  // namespace sdft
