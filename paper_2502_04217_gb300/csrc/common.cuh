// Shared device/host helpers of the sdft_ipm CUDA library: complex arithmetic,
// the padded half-spectrum layout of the beta vector, and deterministic
// block/grid reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sdft {

// Programmatic dependent launch (sm_90+).  Kernels of the solve loop start with
// pdl_wait(): when launched with programmatic stream serialization it blocks
// until the preceding grid has completed and its memory is visible (without
// that attribute it returns at once), so a kernel may be launched while its
// predecessor drains.  pdl_launch() after a block's main work lets the next
// kernel of the stream begin launching.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch() { asm volatile("griddepcontrol.launch_dependents;" :::); }

// ---------------------------------------------------------------------------
// Complex helpers (double2 / float2 as interleaved re, im)
// ---------------------------------------------------------------------------
// double <-> float conversions in integer arithmetic, without branches.  On this
// GPU a conversion with a 64-bit operand runs on the FP64 pipe (1/64 of FP32),
// where it costs as much as an FP64 FMA; the FP32 pass kernels convert every
// element of their FP64 vectors, so these take the integer pipe instead.
// Normal numbers convert exactly as the hardware does (round to nearest even for
// d2f, the carry into the exponent and the overflow to infinity done by the
// addition); zeros and infinities keep their sign, NaN stays NaN, and values in
// the subnormal range of the narrower side are flushed to a signed zero (below
// 1.2e-38, far under the FP32 rounding of every product they enter).
__device__ __forceinline__ float d2f_int(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32);
  const unsigned ex = (hi >> 20) & 0x7ffu;
  const int e = (int)ex - 1023 + 127;
  const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  const unsigned r = (unsigned)(m >> 29);               // leading 23 mantissa bits
  const unsigned rem = (unsigned)(m & 0x1FFFFFFFull);   // the 29 bits dropped
  unsigned f = ((unsigned)e << 23) | r;
  f += (rem > 0x10000000u || (rem == 0x10000000u && (r & 1u))) ? 1u : 0u;
  const unsigned special = (ex == 0x7ffu && m != 0ull) ? 0x7fc00000u : 0x7f800000u;   // NaN : overflow / inf
  f = (e < 1) ? 0u : (e > 254 ? special : f);
  return __uint_as_float(f | (hi & 0x80000000u));
}
__device__ __forceinline__ double f2d_int(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned e = (u >> 23) & 0xffu;
  const unsigned long long s = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned long long mant = (unsigned long long)(u & 0x7FFFFFu) << 29;
  const unsigned long long nrm = s | ((unsigned long long)(e + (1023u - 127u)) << 52) | mant;
  const unsigned long long b = (e == 0u) ? s : (e == 255u ? (s | 0x7FF0000000000000ull | mant) : nrm);
  return __longlong_as_double((long long)b);
}

// 1/x by ONE Newton step y <- y + y (1 - x y) from the single-precision seed
// (conversions on the integer pipe): relative error about (1.2e-7)^2 = 1.4e-14,
// used for the barrier scalings of the Newton system, whose perturbation at that
// level is invisible next to the PCG tolerance.  GB300 executes FP64 divides at
// ~58 G/s; outside 2^+-120 (and for 0, inf, NaN) this falls back to a divide.
__device__ __forceinline__ double rcp1(double x) {
  const unsigned hi = (unsigned)((unsigned long long)__double_as_longlong(x) >> 32);
  const int ex = (int)((hi >> 20) & 0x7ffu) - 1023;
  if (ex < -120 || ex > 120) return 1.0 / x;
  const double y = f2d_int(__frcp_rn(d2f_int(x)));
  return fma(y, fma(-x, y, 1.0), y);
}
template <typename T> __device__ __forceinline__ T from_double(double x);
template <> __device__ __forceinline__ double from_double<double>(double x) { return x; }
template <> __device__ __forceinline__ float from_double<float>(double x) { return d2f_int(x); }
__device__ __forceinline__ double to_double(double x) { return x; }
__device__ __forceinline__ double to_double(float x) { return f2d_int(x); }

template <typename T> struct cvec;
template <> struct cvec<double> { using type = double2; };
template <> struct cvec<float> { using type = float2; };

template <typename V> __device__ __forceinline__ V cmake(decltype(V::x) x, decltype(V::x) y) { V v; v.x = x; v.y = y; return v; }
template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return cmake<V>(a.x + b.x, a.y + b.y); }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return cmake<V>(a.x - b.x, a.y - b.y); }
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
  return cmake<V>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename V> __device__ __forceinline__ V cmulconj(V a, V b) {   // a * conj(b)
  return cmake<V>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename V> __device__ __forceinline__ V cconj(V a) { return cmake<V>(a.x, -a.y); }
template <typename V> __device__ __forceinline__ V cmul_i(V a) { return cmake<V>(-a.y, a.x); }      // i * a
template <typename V> __device__ __forceinline__ V cmul_mi(V a) { return cmake<V>(a.y, -a.x); }     // -i * a
template <typename V, typename S> __device__ __forceinline__ V cscale(V a, S s) { return cmake<V>(a.x * s, a.y * s); }

// ---------------------------------------------------------------------------
// Layout of the half spectrum.  A grid N_0 x ... x N_{d-1} (row-major, last
// axis contiguous; every extent even or odd) has H = Hl * M complex
// half-spectrum slots, Hl = floor(N_l/2) + 1 along the halved last axis l and
// M = N_0 ... N_{d-2} in-plane frequencies.  Slot s = kl * M + k' (the halved
// axis is OUTERMOST), k' = k0 for d = 2 and k' = k0 * N1 + k1 for d = 3.  The
// beta vector has 2H doubles: beta[2s] and beta[2s+1] are the two real
// coordinates carried by slot s.
//
// Slot classes (the representative rule of the real parametrisation; the edge
// planes are those with 2 kl = 0 mod N_l: kl = 0, and kl = N_l/2 for even N_l):
//   INTERIOR  1 <= kl, 2 kl < N_l: the slot is its pair's representative,
//             beta = (sqrt2 Re v, sqrt2 Im v);
//   EDGE_REP  edge plane, k' lexicographically before -k': as INTERIOR;
//   EDGE_SC   edge plane, k' = -k' (self-conjugate): beta = (v, ghost);
//   EDGE_TWIN edge plane, the other member of a pair: (ghost, ghost).
// On an odd in-plane axis only index 0 is its own negative.
// Ghost coordinates are kept at exactly 0 in every vector.
// ---------------------------------------------------------------------------
enum SlotClass { INTERIOR = 0, EDGE_REP = 1, EDGE_SC = 2, EDGE_TWIN = 3 };

// Unsigned 32-bit division by a divisor fixed at set-up, as a multiply-high, an
// add and two shifts (integer pipe only; a run-time division needs conversions
// that this GPU runs on its narrow FP64 pipe).  With l = ceil(log2 d) and
// m = floor(2^32 (2^l - d) / d) + 1, floor(n / d) = (t + ((n - t) >> 1)) >> (l - 1)
// for every 32-bit n, where t = floor(m n / 2^32) (the shifts become 0 and 0 for
// d = 1 and 1 and 0 for d = 2).
struct FastDiv {
  unsigned m;
  int s1, s2;
};

__host__ __device__ inline FastDiv make_fastdiv(unsigned d) {
  int l = 0;
  while ((1ull << l) < (unsigned long long)d) ++l;
  FastDiv f;
  f.m = (unsigned)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
  f.s1 = l < 1 ? l : 1;
  f.s2 = l > 1 ? l - 1 : 0;
  return f;
}

__host__ __device__ __forceinline__ unsigned fast_div(unsigned n, FastDiv f) {
#ifdef __CUDA_ARCH__
  const unsigned t = __umulhi(f.m, n);
#else
  const unsigned t = (unsigned)(((unsigned long long)f.m * n) >> 32);
#endif
  return (t + ((n - t) >> f.s1)) >> f.s2;
}

struct Layout {
  int d;          // 1, 2 or 3
  int N0, N1;     // in-plane lengths (d=3: N0 x N1; d=2: N0, N1 = 1; d=1: 1, 1)
  int Nl;         // last (halved) axis length
  int Hl;         // floor(Nl / 2) + 1
  int M;          // in-plane count
  long long H;    // number of complex slots = Hl * M
  long long n;    // number of grid points = Nl * M
  FastDiv divM, divN1;   // division by M and by N1 (set by layout_init)
};

// Fill a layout from the grid extents (d = 1: {Nl}; d = 2: {N0, Nl}; d = 3: {N0, N1, Nl}).
inline Layout layout_init(int d, int N0, int N1, int Nl) {
  Layout L{};
  L.d = d;
  L.N0 = N0;
  L.N1 = N1;
  L.Nl = Nl;
  L.M = N0 * N1;
  L.Hl = Nl / 2 + 1;
  L.H = (long long)L.Hl * L.M;
  L.n = (long long)Nl * L.M;
  L.divM = make_fastdiv((unsigned)L.M);
  L.divN1 = make_fastdiv((unsigned)N1);
  return L;
}

__host__ __device__ __forceinline__ int slot_class(const Layout& L, long long s) {
  // H < 2^31 for every supported grid, so 32-bit division suffices
  const unsigned su = (unsigned)s;
  const int kl = (int)fast_div(su, L.divM);
  if (kl >= 1 && 2 * kl < L.Nl) return INTERIOR;
  const int kp = (int)(su - (unsigned)kl * (unsigned)L.M);
  if (L.d == 1) return EDGE_SC;
  int k0, k1;
  if (L.d == 2) { k0 = kp; k1 = 0; }
  else { k0 = (int)fast_div((unsigned)kp, L.divN1); k1 = kp - k0 * L.N1; }
  if (k0 == 0 || 2 * k0 == L.N0) {
    if (L.d == 2) return EDGE_SC;
    if (k1 == 0 || 2 * k1 == L.N1) return EDGE_SC;
    return (2 * k1 < L.N1) ? EDGE_REP : EDGE_TWIN;
  }
  return (2 * k0 < L.N0) ? EDGE_REP : EDGE_TWIN;
}

// true when beta element i (0 <= i < 2H) is a ghost coordinate
__host__ __device__ __forceinline__ bool is_ghost(const Layout& L, long long i) {
  int c = slot_class(L, i >> 1);
  return c == EDGE_TWIN || (c == EDGE_SC && (i & 1));
}

// ---------------------------------------------------------------------------
// Deterministic reductions: a fixed tree inside each block, then the last
// block to finish (ticket counter) combines the per-block partials in block
// order.  The result is bit-identical from run to run for a fixed grid.
// ---------------------------------------------------------------------------
enum RedOp { RED_SUM = 0, RED_MAX = 1, RED_MIN = 2 };

__device__ __forceinline__ double red_combine(double a, double b, int op) {
  return op == RED_SUM ? a + b : (op == RED_MAX ? fmax(a, b) : fmin(a, b));
}
__device__ __forceinline__ double red_identity(int op) {
  return op == RED_SUM ? 0.0 : (op == RED_MAX ? -1.0 / 0.0 : 1.0 / 0.0);
}

// Reduce NV values over the block; result valid in thread 0.  scratch must hold
// NV * 32 doubles.  blockDim.x must be a multiple of 32.
template <int NV>
__device__ __forceinline__ void block_reduce(double (&v)[NV], const int (&ops)[NV], double* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] = red_combine(v[k], __shfl_down_sync(0xffffffffu, v[k], o), ops[k]);
  }
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) scratch[k * 32 + warp] = v[k];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      v[k] = lane < nw ? scratch[k * 32 + lane] : red_identity(ops[k]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v[k] = red_combine(v[k], __shfl_down_sync(0xffffffffu, v[k], o), ops[k]);
    }
  }
}

// Store this block's partials; returns true in exactly one block (the last to
// arrive), in which thread 0 holds the grid-wide result in v on return.
// partials must hold NV * gridDim.x doubles; counter is reset for the next use.
template <int NV>
__device__ __forceinline__ bool grid_reduce(double (&v)[NV], const int (&ops)[NV], double* partials,
                                            unsigned* counter, double* scratch) {
  __shared__ bool am_last;
  block_reduce<NV>(v, ops, scratch);
  const unsigned nb = gridDim.x * gridDim.y;
  const unsigned bid = blockIdx.y * gridDim.x + blockIdx.x;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) partials[(size_t)k * nb + bid] = v[k];
    __threadfence();
    unsigned t = atomicAdd(counter, 1u);
    am_last = (t == nb - 1);
  }
  __syncthreads();
  if (!am_last) return false;
  __threadfence();
  // combine partials in block order, each thread a strided slice, then a block tree
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double acc = red_identity(ops[k]);
    for (unsigned b = threadIdx.x; b < nb; b += blockDim.x)
      acc = red_combine(acc, ((volatile double*)partials)[(size_t)k * nb + b], ops[k]);
    v[k] = acc;
  }
  block_reduce<NV>(v, ops, scratch);
  if (threadIdx.x == 0) *counter = 0u;
  return true;
}

}  // namespace sdft
