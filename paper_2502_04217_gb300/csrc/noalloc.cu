// gapply_noalloc: one product with M_perp^T M_perp that allocates no device
// memory.  For callers that cannot call cudaMalloc: hosts that hand all device
// memory out through their own allocator or a fixed budget, code that must not
// trigger the implicit device synchronisation of cudaMalloc / cudaFree (for
// example between the launches of a latency-critical pipeline), and plugins
// running inside another program's CUDA context.
//
// Scratch lives in one file-scope __device__ array of fixed size
// (kNoAllocScratchBytes, about 4.7 MB) that every GPU which loads the library
// keeps until the process exits.  Host code cannot use the array's name as a
// device address, so the first call on each device (with that device current)
// asks the runtime for the address once with cudaGetSymbolAddress and caches
// it; make that first call before any stream capture.  Every call shares the
// array and finds the previous call's contents: the parts that must start from
// a known state (the launch counter, the packed mask, the twiddle tables) are
// rewritten by each call.  Two calls whose work overlaps on the GPU (different
// streams, or different host threads on one device) race on the array: order
// them on one stream.
#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/sdft_ipm.h"
#include "internal.h"
#include "kernels.h"

namespace sdft {
void record_error(const char* msg);   // capi.cu: message returned by ipm_last_error(NULL)
}

using namespace sdft;

namespace {

constexpr long long kNoAllocMaxSlots = 262144;          // largest H = N_0..N_{d-2} (N_{d-1}/2 + 1)
constexpr size_t kScalarBytes = 1024;                     // DevScalars (launch counter)
constexpr size_t kMaskBytes = 640 * 1024;                 // packed mask words, bound for H <= kNoAllocMaxSlots
constexpr size_t kTableBytes = 4 * 512 * 16;              // four FP64 twiddle tables of length <= 512
constexpr size_t kWorkBytes = (size_t)kNoAllocMaxSlots * 16;   // FP64 complex work buffer
constexpr size_t kNoAllocScratchBytes = kScalarBytes + kMaskBytes + kTableBytes + kWorkBytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];
static_assert(sizeof(DevScalars) <= kScalarBytes, "scalar region too small");

constexpr int kMaxDevices = 256;
std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {};

bool length_ok(int64_t L) {
  if (L < 2 || L % 2 || L > 512) return false;
  int64_t m = L;
  while (m % 2 == 0) m /= 2;
  if (m % 3 == 0) m /= 3;
  return m == 1;
}

ipm_status arg_error(const char* msg) {
  record_error(msg);
  return IPM_ERR_ARG;
}

// Tile plan of one FP64 pass: FFT length L, `rows` shared-memory rows, npen pencils.
struct Plan {
  FftPlan fft{};
  int E = 8, lgP = 0, PP = 1, nwork = 0, threads = 64;
  size_t smem = 0;
};

Plan plan_fp64(int L, int rows, long long npen) {
  Plan c;
  c.E = (L % 3 == 0) ? 12 : 8;
  c.fft.L = L;
  int m = L;
  const bool three = (m % 3 == 0);
  if (three) m /= 3;
  while (c.E % 8 == 0 && m % 8 == 0) { c.fft.radix[c.fft.nst++] = 8; m /= 8; }
  while (m % 4 == 0) { c.fft.radix[c.fft.nst++] = 4; m /= 4; }
  while (m % 2 == 0) { c.fft.radix[c.fft.nst++] = 2; m /= 2; }
  if (three) c.fft.radix[c.fft.nst++] = 3;
  int P = 8;
  while (P > 2 && (npen + P - 1) / P < 2 * 152) P /= 2;
  while ((P * L) % c.E != 0) P *= 2;
  while (P > 1 && ((P * L) / c.E > 512 || (size_t)rows * (P + 1) * 16 > 200 * 1024)) P /= 2;
  while ((1 << c.lgP) < P) ++c.lgP;
  c.PP = (P >= 8) ? P + 1 : P;
  c.nwork = (P * L) / c.E;
  c.threads = ((c.nwork + 31) / 32) * 32;
  if (c.threads < 64) c.threads = 64;
  c.smem = (size_t)rows * c.PP * 16;
  return c;
}

void push_table(std::vector<double>& t, int L) {
  for (int k = 0; k < L; ++k) {
    const long double ang = 2.0L * 3.14159265358979323846264338327950288L * (long double)k / (long double)L;
    t.push_back((double)cosl(ang));
    t.push_back((double)(-sinl(ang)));
  }
}

}  // namespace

extern "C" ipm_status gapply_noalloc(int ndim, const int64_t* dims, const uint8_t* mask, const double* p, double* q,
                                     void* stream) {
  if (ndim < 1 || ndim > 3 || !dims) return arg_error("gapply_noalloc: ndim must be 1, 2 or 3");
  for (int i = 0; i < ndim; ++i)
    if (!length_ok(dims[i]))
      return arg_error("gapply_noalloc: every extent must be even, of the form 2^a 3^b (b <= 1), and at most 512");
  if (!mask || !p || !q) return arg_error("gapply_noalloc: mask, p and q must be device pointers");
  const Layout L = layout_init(ndim, ndim >= 2 ? (int)dims[0] : 1, ndim == 3 ? (int)dims[1] : 1, (int)dims[ndim - 1]);
  if (L.H > kNoAllocMaxSlots)
    return arg_error("gapply_noalloc: grid too large for the fixed scratch (at most 262144 half-spectrum "
                     "slots; 512 x 512 and 64 x 64 x 64 fit); use ipm_create / gapply");
  const size_t mask_words = (size_t)((L.Nl + 31) / 32) * L.M;
  if (mask_words * 4 > kMaskBytes) return arg_error("gapply_noalloc: mask does not fit the fixed scratch");

  // once per device, with that device current: the device address of the scratch array
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    record_error("gapply_noalloc: no usable current CUDA device");
    return IPM_ERR_CUDA;
  }
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_addr[dev]) {
      void* a = nullptr;
      e = cudaGetSymbolAddress(&a, g_noalloc_scratch);
      if (e != cudaSuccess || !a) {
        record_error((std::string("gapply_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e)).c_str());
        return IPM_ERR_CUDA;
      }
      g_scratch_addr[dev] = a;
    }
    base = (unsigned char*)g_scratch_addr[dev];
  }
  DevScalars* sc = (DevScalars*)base;
  uint32_t* maskw = (uint32_t*)(base + kScalarBytes);
  double* tables = (double*)(base + kScalarBytes + kMaskBytes);
  void* work = base + kScalarBytes + kMaskBytes + kTableBytes;
  cudaStream_t st = (cudaStream_t)stream;

  // twiddle tables: row axis, column axis, h = Nl/2 and Nl
  const int Lrow = L.d == 3 ? L.N1 : L.N0, Lcol = L.N0, h = L.Nl / 2;
  std::vector<double> t;
  t.reserve(2 * (size_t)(Lrow + Lcol + h + L.Nl));
  const size_t off_row = 0;
  if (L.d >= 2) push_table(t, Lrow);
  const size_t off_col = t.size();
  if (L.d == 3) push_table(t, Lcol);
  const size_t off_h = t.size();
  push_table(t, h);
  const size_t off_N = t.size();
  push_table(t, L.Nl);

  auto fail = [](cudaError_t err) {
    record_error((std::string("gapply_noalloc: ") + cudaGetErrorString(err)).c_str());
    return IPM_ERR_CUDA;
  };
  if ((e = cudaMemsetAsync(sc, 0, sizeof(DevScalars), st)) != cudaSuccess) return fail(e);
  if ((e = cudaMemcpyAsync(tables, t.data(), t.size() * sizeof(double), cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return fail(e);
  if ((e = k_pack_mask(mask, maskw, L.Nl, L.M, sc, st)) != cudaSuccess) return fail(e);

  auto args = [&](const Plan& c, long long npen, size_t tw_off) {
    PassArgs a{};
    a.lay = L;
    a.plan = c.fft;
    a.lgP = c.lgP;
    a.PP = c.PP;
    a.nwork = c.nwork;
    a.npencils = npen;
    a.tw = tables + tw_off;
    a.twN = tables + off_N;
    a.buf = work;
    a.maskw = maskw;
    a.inv_n = 1.0 / (double)L.n;
    a.out_scale = 1.0;
    a.sc = sc;
    return a;
  };
  auto grid1 = [](long long npen, int lgP) { return dim3((unsigned)((npen + (1 << lgP) - 1) >> lgP)); };
  const Plan mid = plan_fp64(h, L.Hl, L.M);
  if (L.d == 1) {
    PassArgs a = args(mid, L.M, off_h);
    a.mapin = MAPIN_BETA;
    a.src = p;
    a.mapout = MAPOUT_BETA;
    a.dst = q;
    if ((e = launch_pass(2, false, false, mid.E, a, mid.threads, mid.smem, grid1(L.M, mid.lgP), st)) != cudaSuccess)
      return fail(e);
    return IPM_OK;
  }
  const long long nrows = L.H / Lrow;
  const Plan row = plan_fp64(Lrow, Lrow, nrows);
  const Plan col = L.d == 3 ? plan_fp64(Lcol, Lcol, (long long)L.N1 * L.Hl) : Plan{};
  const dim3 gcol((unsigned)((L.N1 + (1 << col.lgP) - 1) >> col.lgP), (unsigned)L.Hl);
  {
    PassArgs a = args(row, nrows, off_row);
    a.mapin = MAPIN_BETA;
    a.src = p;
    if ((e = launch_pass(0, true, false, row.E, a, row.threads, row.smem, grid1(nrows, row.lgP), st)) != cudaSuccess)
      return fail(e);
  }
  if (L.d == 3) {
    PassArgs a = args(col, (long long)L.N1 * L.Hl, off_col);
    if ((e = launch_pass(1, true, false, col.E, a, col.threads, col.smem, gcol, st)) != cudaSuccess) return fail(e);
  }
  {
    PassArgs a = args(mid, L.M, off_h);
    if ((e = launch_pass(2, false, false, mid.E, a, mid.threads, mid.smem, grid1(L.M, mid.lgP), st)) != cudaSuccess)
      return fail(e);
  }
  if (L.d == 3) {
    PassArgs a = args(col, (long long)L.N1 * L.Hl, off_col);
    if ((e = launch_pass(1, false, false, col.E, a, col.threads, col.smem, gcol, st)) != cudaSuccess) return fail(e);
  }
  {
    PassArgs a = args(row, nrows, off_row);
    a.mapout = MAPOUT_BETA;
    a.dst = q;
    if ((e = launch_pass(0, false, false, row.E, a, row.threads, row.smem, grid1(nrows, row.lgP), st)) != cudaSuccess)
      return fail(e);
  }
  return IPM_OK;
}
