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
// device address, so the first call in each CUDA context asks the runtime for
// the address once with cudaGetSymbolAddress (the device current, the context
// current) and caches it per context; make that first call before any stream
// capture.  A context destroyed after its first call (cudaDeviceReset) must not
// be followed by further calls in a new context whose handle reuses the old one.
// Every call shares the array and finds the previous call's contents: the parts
// that must start from a known state (the launch counter, the packed mask, the
// twiddle tables) are rewritten on the device by each call, so a call queues
// only kernels and one memset and returns without waiting for the stream.  Two
// calls whose work overlaps on the GPU (different streams, or different host
// threads on one device) race on the array: order them on one stream.
#include <cuda.h>

#include <cmath>
#include <mutex>
#include <string>

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

// Device address of the scratch array per CUDA context (looked up once per context).
constexpr int kMaxContexts = 64;
std::mutex g_setup_mu;
struct CtxAddr {
  CUcontext ctx;
  void* addr;
};
CtxAddr g_addr[kMaxContexts] = {};
int g_naddr = 0;

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);

CtxGetCurrentFn ctx_get_current() {
  static CtxGetCurrentFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<CtxGetCurrentFn>(f);
  }
  return fn;
}

// The scratch array's device address in the current context.  Called with
// g_setup_mu held.  Without a context handle (no driver entry point) the address
// is looked up on every call instead of cached.
cudaError_t scratch_address(void** out) {
  CUcontext ctx = nullptr;
  CtxGetCurrentFn get = ctx_get_current();
  const bool keyed = get && get(&ctx) == CUDA_SUCCESS && ctx;
  if (keyed)
    for (int i = 0; i < g_naddr; ++i)
      if (g_addr[i].ctx == ctx) {
        *out = g_addr[i].addr;
        return cudaSuccess;
      }
  void* a = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&a, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  if (!a) return cudaErrorInvalidSymbol;
  if (keyed && g_naddr < kMaxContexts) g_addr[g_naddr++] = {ctx, a};
  *out = a;
  return cudaSuccess;
}

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

// The twiddle tables of the passes, back to back: tables of lengths L0..L3 (0: absent),
// entry k of a length-L table exp(-2 pi i k / L) as (cos, -sin) of pi (2k / L).
__global__ void noalloc_twiddles_kernel(double* __restrict__ t, int L0, int L1, int L2, int L3, DevScalars* sc) {
  count_launch(sc);
  const long long total = (long long)L0 + L1 + L2 + L3;
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < total; j += (long long)gridDim.x * blockDim.x) {
    long long k = j;
    int L = L0;
    if (k >= L0) {
      k -= L0;
      L = L1;
      if (k >= L1) {
        k -= L1;
        L = L2;
        if (k >= L2) {
          k -= L2;
          L = L3;
        }
      }
    }
    double sn, cs;
    sincospi(2.0 * (double)k / (double)L, &sn, &cs);
    t[2 * j] = cs;
    t[2 * j + 1] = -sn;
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

  // once per CUDA context (the device current): the device address of the scratch array
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    void* a = nullptr;
    cudaError_t e = scratch_address(&a);
    if (e != cudaSuccess) {
      record_error((std::string("gapply_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e)).c_str());
      return IPM_ERR_CUDA;
    }
    base = (unsigned char*)a;
  }
  cudaError_t e = cudaSuccess;
  DevScalars* sc = (DevScalars*)base;
  uint32_t* maskw = (uint32_t*)(base + kScalarBytes);
  double* tables = (double*)(base + kScalarBytes + kMaskBytes);
  void* work = base + kScalarBytes + kMaskBytes + kTableBytes;
  cudaStream_t st = (cudaStream_t)stream;

  // twiddle tables, built on the device: row axis, column axis, h = Nl/2 and Nl
  const int Lrow = L.d == 3 ? L.N1 : L.N0, Lcol = L.N0, h = L.Nl / 2;
  const int t_row = L.d >= 2 ? Lrow : 0, t_col = L.d == 3 ? Lcol : 0;
  const size_t off_row = 0;
  const size_t off_col = off_row + 2 * (size_t)t_row;
  const size_t off_h = off_col + 2 * (size_t)t_col;
  const size_t off_N = off_h + 2 * (size_t)h;

  auto fail = [](cudaError_t err) {
    record_error((std::string("gapply_noalloc: ") + cudaGetErrorString(err)).c_str());
    return IPM_ERR_CUDA;
  };
  if ((e = cudaMemsetAsync(sc, 0, sizeof(DevScalars), st)) != cudaSuccess) return fail(e);
  noalloc_twiddles_kernel<<<8, 256, 0, st>>>(tables, t_row, t_col, h, L.Nl, sc);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(e);
  if ((e = k_pack_mask(mask, maskw, L.Nl, L.M, sc, st)) != cudaSuccess) return fail(e);

  auto args = [&](const TileChoice& c, long long npen, size_t tw_off) {
    PassArgs a{};
    a.lay = L;
    a.plan = c.plan;
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
  TileChoice mid{}, row{}, col{};
  if (!default_tile(h, L.Hl, L.M, false, &mid)) return arg_error("gapply_noalloc: no launchable tile");
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
  if (!default_tile(Lrow, Lrow, nrows, false, &row) ||
      (L.d == 3 && !default_tile(Lcol, Lcol, (long long)L.N1 * L.Hl, false, &col)))
    return arg_error("gapply_noalloc: no launchable tile");
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
