// Register-resident Stockham FFT for a tile of P pencils (Sec. 3.1: the masked
// operators are applied with forward / inverse DFTs; this formulation is ours).
//
// A pencil of length L is carried by T = L / E threads, each holding E complex
// values.  With the butterflies of a radix-R stage assigned as j = t + b T
// (b = 0 .. E/R - 1), the inputs of thread t in EVERY stage are the elements
// t + T m (m = 0 .. E-1), and the outputs of the LAST stage are again the
// elements t + T m.  So the first stage reads its operands straight from
// global memory and the last stage writes straight to global memory (both
// coalesced across t); shared memory is only used for the S - 1 exchanges
// between the S stages (one for L = 128 and 256 with E = 16).
//
// Stage formulas (decimation in time, self-sorting), as in fft_core.cuh: for
// butterfly j of a radix-R stage after Ns = R_1 ... R_{s-1},
//     a_r = x[j + r L/R] * w_L^{(j mod Ns) r L/(Ns R)},  a = DFT_R(a),
//     y[(j div Ns) Ns R + (j mod Ns) + r Ns] = a_r.
#pragma once

#include "fft_core.cuh"

namespace sdft {

// One stage on the registers of thread t: x[m] is element t + T m on entry;
// on exit x[b + r B] holds output r of butterfly b (B = E / R).
template <int E, int R, bool INV, int L, int LGNS, typename V>
__device__ __forceinline__ void reg_stage(V (&x)[E], int t, const V* __restrict__ tw) {
  constexpr int T = L / E, B = E / R, Ns = 1 << LGNS, TWS = L / (Ns * R);
#pragma unroll
  for (int b = 0; b < B; ++b) {
    V a[R];
#pragma unroll
    for (int r = 0; r < R; ++r) a[r] = x[b + r * B];
    if constexpr (Ns > 1) {
      const int kt = ((t + b * T) & (Ns - 1)) * TWS;
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const V w = __ldg(tw + kt * r);
        a[r] = INV ? cmulconj(a[r], w) : cmul(a[r], w);
      }
    }
    dft_r<R, INV>(a);
#pragma unroll
    for (int r = 0; r < R; ++r) x[b + r * B] = a[r];
  }
}

// Exchange after a (non-last) stage through shared memory: every output goes to
// its element index, then x[m] = element t + T m for the next stage.  `addr`
// maps an element index of this thread's pencil to its shared-memory slot.
template <int E, int R, int L, int LGNS, typename V, typename A>
__device__ __forceinline__ void reg_exchange(V (&x)[E], int t, V* sm, A&& addr) {
  constexpr int T = L / E, B = E / R, Ns = 1 << LGNS;
#pragma unroll
  for (int b = 0; b < B; ++b) {
    const int j = t + b * T;
    const int base = (j >> LGNS) * (Ns * R) + (j & (Ns - 1));
#pragma unroll
    for (int r = 0; r < R; ++r) sm[addr(base + r * Ns)] = x[b + r * B];
  }
  __syncthreads();
#pragma unroll
  for (int m = 0; m < E; ++m) x[m] = sm[addr(t + T * m)];
}

template <int E, bool INV, int L, int S, int LGNS, typename V, typename A>
__device__ __forceinline__ void reg_stages(V (&x)[E], int t, const V* __restrict__ tw, V* sm, A&& addr) {
  constexpr int NS = stage_count_c(L, E);
  if constexpr (S < NS) {
    constexpr int R = stage_radix_c(L, E, S);
    reg_stage<E, R, INV, L, LGNS>(x, t, tw);
    if constexpr (S + 1 < NS) {
      reg_exchange<E, R, L, LGNS>(x, t, sm, addr);
      if constexpr (S + 2 < NS) __syncthreads();   // reads done before the next exchange writes
      reg_stages<E, INV, L, S + 1, LGNS + log2_c(R)>(x, t, tw, sm, addr);
    }
  }
}

// Whole transform of length L on the registers of thread t of a pencil.  The
// caller synchronises before `sm` is written again after this returns.
template <int E, bool INV, int L, typename V, typename A>
__device__ __forceinline__ void reg_fft(V (&x)[E], int t, const V* __restrict__ tw, V* sm, A&& addr) {
  reg_stages<E, INV, L, 0, 0>(x, t, tw, sm, addr);
}

}  // namespace sdft
