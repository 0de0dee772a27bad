// C ABI of the solver (declared in include/sdft_ipm.h): handle lifetime,
// FFT pass planning, and the host side of the interior-point loop
// (Sec. 3.3-3.5): every arithmetic step runs in the kernels of
// fft_passes.cu and ipm_kernels.cu; the host only queues launches and reads
// the device scalars where it has to decide (IPM stop, PCG chunk boundaries).
#include <algorithm>
#include <chrono>
#include <map>
#include <mutex>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/sdft_ipm.h"
#include "internal.h"
#include "kernels.h"

using namespace sdft;

namespace sdft {
thread_local bool g_pdl = false;
}

namespace {

// Sets programmatic dependent launch for the kernels this thread queues while
// the guard lives (solve loops and operator calls of a handle with opt.pdl).
struct PdlScope {
  bool saved;
  explicit PdlScope(bool on) : saved(g_pdl) { g_pdl = on; }
  ~PdlScope() { g_pdl = saved; }
};

thread_local std::string g_create_error;

// One planned launch of an FFT pass.
struct PassCfg {
  int kind = 0;             // 0 row, 1 column, 2 middle
  int E = 8;
  int lgP = 0, PP = 1, nwork = 0, threads = 32;
  size_t smem = 0;
  dim3 grid;
  FftPlan plan{};
  long long npencils = 0;
  const void* tw = nullptr;
  const void* twN = nullptr;
  int reg = 0;              // 1: register engine (fft_reg.cuh)
  int kstage = 0;           // forward row pass: staging of the K epilogue's operands (PassArgs::kstage)
  unsigned kst_off = 0;     // kstage 2: byte offset of the staged operands in shared memory
  size_t smem_staged = 0;   // shared memory of a launch with kstage 2
};

struct PassSet {
  PassCfg row_inv, row_fwd, col_inv, col_fwd, mid;
  PassCfg row_inv_beta;     // first row pass reading a plain beta-layout vector (G and K products, residuals)
  PassCfg row_fwd_k;        // last row pass of a product with K outside PCG (kkt_apply, residual replacement):
                            // tuned without PCG's p^T q reduction and (G p)_beta store
};

// Kernel classes of the per-launch timing (ipm_profile_get): 0 row, 1 column and
// 2 middle FFT passes, 3 PCG updates, 4 other IPM kernels, 5 the launch counter (no
// timing), 6 the Newton-system kernel (prepare), 7 the step kernels, 8 the certificate.
constexpr int kProfClasses = 9, kProfPrepare = 6, kProfStep = 7, kProfCertificate = 8;

struct ProfEntry {
  int cls;
  cudaEvent_t a, b;
};

// Supported transform lengths: 2^a 3^b 5^c 7^d (even or odd).
bool factor_ok(int L) {
  int m = L;
  for (int q : {2, 3, 5, 7})
    while (m % q == 0) m /= q;
  return m == 1;
}

// Radices for length L: with element budget E per thread, 16s (E = 16), then 8s
// (E divisible by 8), then 4s (E divisible by 4), then 2s, and last the odd
// factors of L: every 3, then every 5, then every 7.  Every power-of-two stage
// then has a power-of-two Ns; the odd stages take any Ns.
FftPlan make_plan(int L, int E) {
  FftPlan p{};
  p.L = L;
  int m = L;
  int cnt[3] = {0, 0, 0};
  const int q[3] = {3, 5, 7};
  for (int i = 0; i < 3; ++i)
    while (m % q[i] == 0) { ++cnt[i]; m /= q[i]; }
  while (E % 16 == 0 && m % 16 == 0) { p.radix[p.nst++] = 16; m /= 16; }
  while (E % 8 == 0 && m % 8 == 0) { p.radix[p.nst++] = 8; m /= 8; }
  while (E % 4 == 0 && m % 4 == 0) { p.radix[p.nst++] = 4; m /= 4; }
  while (m % 2 == 0) { p.radix[p.nst++] = 2; m /= 2; }
  for (int i = 0; i < 3; ++i)
    for (int c = 0; c < cnt[i]; ++c) p.radix[p.nst++] = q[i];
  return p;
}

int ilog2(int v) { int l = 0; while ((1 << l) < v) ++l; return l; }

}  // namespace

struct sdft_ipm {
  int device = 0;
  cudaStream_t st = nullptr;
  ipm_options opt{};
  Layout lay{};
  int dims[3] = {0, 0, 0};
  std::string err;
  int stall_log2 = 0;               // ipm_test_stage_stall: the next kkt_apply drops a staged copy
  double lambda_in = 0.0;
  // device memory
  std::vector<void*> allocs;
  uint8_t* d_mask = nullptr;
  double* d_y = nullptr;
  uint32_t* d_maskw = nullptr;
  IpmVectors w{};
  void* d_U = nullptr;          // complex work buffer (H values, sized for double)
  double* d_tmp = nullptr;      // 2H scratch for pack/unpack and spectrum readback
  double* d_partials = nullptr;
  unsigned* d_counter = nullptr;
  DevScalars* d_sc = nullptr;
  DevScalars* h_sc = nullptr;   // pinned mirror
  size_t partial_cap = 0;
  PassSet pass64, pass32;
  std::vector<void*> tables;
  bool point_set = false;
  bool sigma_ready = false;
  // profiling
  bool prof = false;
  std::vector<ProfEntry> prof_live;
  std::vector<cudaEvent_t> ev_pool;
  long long prof_count[kProfClasses] = {};
  double prof_ms[kProfClasses] = {};
  unsigned long long launch_base = 0;   // device launch counter at the last profile reset
  // whole-solve CUDA graph (two nested conditional WHILE loops)
  cudaStream_t cap[3] = {nullptr, nullptr, nullptr};
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  bool graph_valid = false;
  cudaGraphConditionalHandle c_ipm = 0, c_cg = 0;
};

namespace {

#define CK(call)                                                                       \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      h->err = std::string(#call) + ": " + cudaGetErrorString(e_);                     \
      return e_ == cudaErrorMemoryAllocation ? IPM_ERR_OOM : IPM_ERR_CUDA;             \
    }                                                                                  \
  } while (0)

// FP64 mode updates G beta from the PCG products (G x accumulated alongside x)
// and recomputes it with an FP64 product only to confirm a passed stop test;
// mixed precision recomputes it every iteration (its PCG products are FP32).
int incremental_gb(const sdft_ipm* h) {
  return (!h->opt.exact_residual && h->opt.krylov == 0 && h->opt.refine_every == 0) ? 1 : 0;
}

ipm_status fail_arg(sdft_ipm* h, const char* msg) {
  if (h) h->err = msg; else g_create_error = msg;
  return IPM_ERR_ARG;
}

template <typename Ptr>
cudaError_t dalloc(sdft_ipm* h, Ptr** p, size_t bytes) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, bytes > 0 ? bytes : 16);
  if (e == cudaSuccess) { h->allocs.push_back(q); *p = (Ptr*)q; }
  return e;
}

cudaEvent_t pool_event(sdft_ipm* h) {
  if (!h->ev_pool.empty()) { cudaEvent_t e = h->ev_pool.back(); h->ev_pool.pop_back(); return e; }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

struct ProfScope {
  sdft_ipm* h;
  int cls;
  cudaEvent_t a = nullptr;
  ProfScope(sdft_ipm* h_, int c) : h(h_), cls(c) {
    if (h->prof) { a = pool_event(h); cudaEventRecord(a, h->st); }
  }
  ~ProfScope() {
    if (h->prof) {
      cudaEvent_t b = pool_event(h);
      cudaEventRecord(b, h->st);
      h->prof_live.push_back({cls, a, b});
    }
  }
};

void prof_collect(sdft_ipm* h) {
  if (h->prof_live.empty()) return;
  cudaStreamSynchronize(h->st);
  for (auto& e : h->prof_live) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e.a, e.b);
    h->prof_count[e.cls] += 1;
    h->prof_ms[e.cls] += ms;
    h->ev_pool.push_back(e.a);
    h->ev_pool.push_back(e.b);
  }
  h->prof_live.clear();
}

// Twiddle table exp(-2 pi i t / L), t = 0..L-1, in double and float.
ipm_status make_tables(sdft_ipm* h, int L, const void** t64, const void** t32) {
  std::vector<double> d(2 * (size_t)L);
  std::vector<float> f(2 * (size_t)L);
  for (int t = 0; t < L; ++t) {
    const long double ang = 2.0L * 3.14159265358979323846264338327950288L * (long double)t / (long double)L;
    d[2 * t] = (double)cosl(ang);
    d[2 * t + 1] = (double)(-sinl(ang));
    f[2 * t] = (float)d[2 * t];
    f[2 * t + 1] = (float)d[2 * t + 1];
  }
  void *a = nullptr, *b = nullptr;
  CK(dalloc(h, &a, d.size() * sizeof(double)));
  CK(dalloc(h, &b, f.size() * sizeof(float)));
  CK(cudaMemcpy(a, d.data(), d.size() * sizeof(double), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(b, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice));
  *t64 = a;
  *t32 = b;
  return IPM_OK;
}

// Tile configuration of a pass: FFT length L, `rows` shared-memory rows, npen
// pencils, element budget E per thread, P pencils per tile.  Returns false when
// the combination is not launchable (P * L must be a multiple of E, at most 512
// threads (256 for E = 16, whose kernels keep 16 values per thread and are
// compiled for that block size), at most 200 KB of shared memory).
bool make_cfg(PassCfg& c, int L, int rows, long long npen, bool fp32, int E, int P) {
  const int esz = fp32 ? 8 : 16;
  const int max_threads = E == 16 ? 256 : 512;
  if ((P * L) % E != 0 || (P * L) / E > max_threads || (P * L) / E < 1) return false;
  const int PP = (P >= (fp32 ? 16 : 8)) ? P + 1 : P;
  if ((size_t)rows * PP * esz > 200 * 1024) return false;
  c.E = E;
  c.plan = make_plan(L, E);
  c.lgP = ilog2(P);
  c.PP = PP;
  c.nwork = (P * L) / E;
  c.threads = ((c.nwork + 31) / 32) * 32;
  if (c.threads < 64) c.threads = 64;
  c.smem = (size_t)rows * PP * esz;
  c.npencils = npen;
  c.reg = 0;
  return true;
}

// Tile of the register engine: E = 16 values per thread, L / 16 threads per
// pencil, P pencils per block (a power of two; the block a multiple of 32 threads,
// at most 256, the kernels' launch bound).  Shared memory: row passes P padded rows (L + L/16 values), column
// passes L x P, middle passes (h + 1) x P (the half spectrum, reused for the exchanges).
bool make_cfg_reg(PassCfg& c, int kind, int L, long long npen, bool fp32, int P) {
  if (L != 32 && L != 64 && L != 128 && L != 256 && L != 512) return false;
  const int esz = fp32 ? 8 : 16, threads = P * (L / 16);
  if (threads % 32 != 0 || threads > 256) return false;
  const size_t rows = kind == 0 ? (size_t)(L + L / 16) : kind == 1 ? (size_t)L : (size_t)(L + 1);
  const size_t smem = rows * P * esz;
  if (smem > 200 * 1024) return false;
  c.E = 16;
  c.plan = make_plan(L, 16);
  c.lgP = ilog2(P);
  c.PP = P;
  c.nwork = threads;
  c.threads = threads;
  c.smem = smem;
  c.npencils = npen;
  c.reg = 1;
  return true;
}

// Staging of the K epilogue's FP64 operands in a forward row pass of the shared-memory
// engine (kstage 1: L2 prefetch; 2: shared memory, 64 bytes per slot of the tile after the
// transform's rows, 128-byte aligned).  False when the stage does not fit in the 227 KB
// a block can have.
bool stage_cfg(PassCfg& c, int kstage) {
  c.kstage = 0;
  c.kst_off = 0;
  c.smem_staged = c.smem;
  if (kstage == 0) return true;
  if (c.reg) return false;
  c.kstage = kstage;
  if (kstage == 2) {
    c.kst_off = (unsigned)((c.smem + 127) & ~(size_t)127);
    c.smem_staged = c.kst_off + (size_t)64 * ((size_t)1 << c.lgP) * (size_t)c.plan.L;
    if (c.smem_staged > 227 * 1024) return false;
  }
  return true;
}

// Default choice without timing: E = 8 (12 with a factor 3), P as large as keeps
// two tiles per SM, at least 2 (FP64) or 4 (FP32); failing that, the first
// launchable (E, P).  Returns false when no shape fits the pass.
bool plan_tile(PassCfg& c, int L, int rows, long long npen, bool fp32) {
  const int E = (L % 3 == 0) ? 12 : 8;
  int P = fp32 ? 16 : 8;
  const int Pmin = fp32 ? 4 : 2;
  while (P > Pmin && (npen + P - 1) / P < 2 * 152) P /= 2;
  while ((P * L) % E != 0 && P <= 32) P *= 2;
  while (P > 1 && !make_cfg(c, L, rows, npen, fp32, E, P)) P /= 2;
  if (make_cfg(c, L, rows, npen, fp32, E, P)) return true;
  const int Es[3] = {(L % 3 == 0) ? 12 : 16, (L % 3 == 0) ? 6 : 8, (L % 3 == 0) ? 6 : 4};
  for (int e : Es)
    for (int q = 1; q <= 32; q *= 2)
      if (make_cfg(c, L, rows, npen, fp32, e, q)) return true;
  return false;
}

}  // namespace

namespace sdft {
bool default_tile(int L, int rows, long long npen, bool fp32, TileChoice* out) {
  PassCfg c;
  if (!plan_tile(c, L, rows, npen, fp32)) return false;
  out->plan = c.plan;
  out->E = c.E;
  out->lgP = c.lgP;
  out->PP = c.PP;
  out->nwork = c.nwork;
  out->threads = c.threads;
  out->smem = c.smem;
  return true;
}
}  // namespace sdft

namespace {

// The FFT passes of a layout (length, shared-memory rows) all have a
// launchable tile in FP64 (whose tiles are the larger).  Odd lengths without a
// factor 3 need P = E pencils, so their P L / E threads exceed the block limit
// above 512 (625 and 875).
bool passes_launchable(const Layout& L) {
  PassCfg c;
  const bool odd = (L.Nl & 1) != 0;
  if (!plan_tile(c, odd ? L.Nl : L.Nl / 2, odd ? L.Nl + 1 : L.Hl, 1, false)) return false;
  if (L.d >= 2) {
    const int Lr = (L.d == 3) ? L.N1 : L.N0;
    if (!plan_tile(c, Lr, Lr, 1, false)) return false;
  }
  if (L.d == 3 && !plan_tile(c, L.N0, L.N0, 1, false)) return false;
  return true;
}

dim3 pass_grid(const Layout& L, int kind, long long npen, int lgP) {
  if (kind == 1) return dim3((unsigned)((L.N1 + (1 << lgP) - 1) >> lgP), (unsigned)L.Hl);
  return dim3((unsigned)((npen + (1 << lgP) - 1) >> lgP));
}

// Autotuner: time every launchable (E, P) of a pass on the handle's own work
// buffer (the FFT core only, no prologue or epilogue) and keep the fastest.
// Results are cached per (pass, length, rows, pencils, precision) for the process.
struct TuneKey {
  int kind, L, rows, fp32;
  long long npen;
  int engine;
  bool operator<(const TuneKey& o) const {
    if (engine != o.engine) return engine < o.engine;
    if (kind != o.kind) return kind < o.kind;
    if (L != o.L) return L < o.L;
    if (rows != o.rows) return rows < o.rows;
    if (fp32 != o.fp32) return fp32 < o.fp32;
    return npen < o.npen;
  }
};
std::mutex g_tune_mu;
struct TuneVal {
  int E, P, reg;
  int kstage;
};
std::map<TuneKey, TuneVal> g_tuned;

// Optional tile cache shared between processes: when the environment variable
// SDFT_TUNE_CACHE names a file, tuned shapes are read from it (first use) and
// every new choice is appended, so that a later process (for instance one run
// under a profiler, whose launch timings are perturbed) launches the same tiles.
// One line per shape: engine kind L rows fp32 npen E P reg kstage.  Lines that do
// not parse are ignored.  Called with g_tune_mu held.
const char* tune_cache_path() {
  const char* p = std::getenv("SDFT_TUNE_CACHE");
  return (p && *p) ? p : nullptr;
}
void tune_cache_load() {
  static bool loaded = false;
  if (loaded) return;
  loaded = true;
  const char* path = tune_cache_path();
  if (!path) return;
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  char line[256];
  while (std::fgets(line, sizeof(line), f)) {
    TuneKey k{};
    TuneVal v{};
    if (std::sscanf(line, "%d %d %d %d %d %lld %d %d %d %d", &k.engine, &k.kind, &k.L, &k.rows, &k.fp32, &k.npen, &v.E,
                    &v.P, &v.reg, &v.kstage) == 10)
      g_tuned[k] = v;
  }
  std::fclose(f);
}
void tune_cache_append(const TuneKey& k, const TuneVal& v) {
  const char* path = tune_cache_path();
  if (!path) return;
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "%d %d %d %d %d %lld %d %d %d %d\n", k.engine, k.kind, k.L, k.rows, k.fp32, k.npen, v.E, v.P, v.reg,
               v.kstage);
  std::fclose(f);
}

// `last`: for a row pass, tune the forward (last) pass of a product instead of the
// inverse (first) one.  Row passes are timed in the form the PCG loop runs them
// (first: p = z + beta p and the beta map; last: the K epilogue with the p^T q
// reduction and the (G p)_beta store), on operands filled with a non-zero pattern by
// the caller; column and middle passes on the work buffer alone.  `beta_form`: the
// first pass reading a plain beta-layout vector, or the last pass with the K epilogue
// alone (the products with K outside PCG).
ipm_status tune_tile(sdft_ipm* h, PassCfg& c, int kind, int L, int rows, long long npen, bool fp32,
                     bool last = false, bool beta_form = false) {
  c.kind = kind;
  if (!plan_tile(c, L, rows, npen, fp32)) return fail_arg(h, "no launchable FFT tile for a pass of this grid");
  c.grid = pass_grid(h->lay, kind, npen, c.lgP);
  if (h->opt.tile_engine == 2) {
    // forced register engine: the given P (else the smallest launchable one
    // with at least 2 blocks per SM), where the length allows
    for (int P = (h->opt.tile_p > 0 ? h->opt.tile_p : 1); P <= 32; P *= 2) {
      PassCfg t = c;
      if (make_cfg_reg(t, kind, L, npen, fp32, P)) {
        c = t;
        c.grid = pass_grid(h->lay, kind, npen, c.lgP);
        break;
      }
      if (h->opt.tile_p > 0) break;
    }
    return IPM_OK;
  }
  if (h->opt.tile_e > 0 || h->opt.tile_p > 0) {
    // forced shape (tests and experiments): keep the default for what is not forced
    const int E = h->opt.tile_e > 0 ? h->opt.tile_e : c.E;
    const int P = h->opt.tile_p > 0 ? h->opt.tile_p : (1 << c.lgP);
    const bool e_ok = (L % 3 == 0) ? (E == 6 || E == 12) : (E == 4 || E == 8 || E == 16);
    PassCfg t = c;
    if (e_ok && make_cfg(t, L, rows, npen, fp32, E, P)) {
      c = t;
      c.grid = pass_grid(h->lay, kind, npen, c.lgP);
    }
    return IPM_OK;
  }
  if (!h->opt.autotune) return IPM_OK;
  const TuneKey key{kind + (last ? 3 : 0) + (beta_form ? 6 : 0), L, rows, fp32 ? 1 : 0, npen, h->opt.tile_engine};
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    tune_cache_load();
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) {
      if (it->second.reg) make_cfg_reg(c, kind, L, npen, fp32, it->second.P);
      else make_cfg(c, L, rows, npen, fp32, it->second.E, it->second.P);
      if (!stage_cfg(c, it->second.kstage)) stage_cfg(c, 0);
      c.grid = pass_grid(h->lay, kind, npen, c.lgP);
      return IPM_OK;
    }
  }
  const bool three = (L % 3 == 0);
  const int Es[3] = {three ? 12 : 16, three ? 6 : 8, three ? 0 : 4};
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  // candidates: the shared-memory engine at every (E, P), the register engine at every P;
  // the forward row pass (K epilogue) also with the L2 prefetch of its operands (the
  // shared-memory stage, 64 bytes per slot, lowers the blocks per SM and measured 11-30 %
  // slower on this pass: it runs only when tile_kstage forces it)
  struct Cand {
    int E, P, kstage;     // E = 0 marks the register engine
  };
  std::vector<Cand> cands;
  const int nstage = (kind == 0 && last) ? 2 : 1;
  if (h->opt.tile_engine != 2)
    for (int E : Es)
      if (E != 0)
        for (int P = 1; P <= 32; P *= 2)
          for (int ks = 0; ks < nstage; ++ks) cands.push_back({E, P, ks});
  if (h->opt.tile_engine != 1)
    for (int P = 1; P <= 32; P *= 2) cands.push_back({0, P, 0});
  struct Trial {
    PassCfg t;
    PassArgs a;
    size_t smem;
    bool inv;
    float ms;
  };
  std::vector<Trial> trials;
  for (const Cand& cand : cands) {
    const int E = cand.E, P = cand.P;
    PassCfg t = c;
    if (E == 0 ? !make_cfg_reg(t, kind, L, npen, fp32, P) : !make_cfg(t, L, rows, npen, fp32, E, P)) continue;
    if (!stage_cfg(t, cand.kstage)) continue;
    t.grid = pass_grid(h->lay, kind, npen, t.lgP);
    PassArgs a{};
    a.lay = h->lay;
    a.plan = t.plan;
    a.lgP = t.lgP;
    a.PP = t.PP;
    a.nwork = t.nwork;
    a.npencils = npen;
    a.tw = t.tw;
    a.twN = t.twN;
    a.buf = h->d_U;
    a.maskw = h->d_maskw;
    a.inv_n = 1.0 / (double)h->lay.n;
    a.out_scale = 1.0;
    a.sc = h->d_sc;
    a.reg = t.reg;
    const bool inv = (kind == 0 && last) ? false : (kind != 2);
    if (kind == 0 && !last && beta_form) {
      a.mapin = MAPIN_BETA;
      a.src = h->w.p;
    } else if (kind == 0 && !last) {
      a.mapin = MAPIN_PCG;
      a.p = h->w.p;
      a.zv = h->w.zv;
    } else if (kind == 0) {
      a.mapout = MAPOUT_K;
      a.p = h->w.p;
      a.q = h->w.q;
      a.lam1 = h->w.lam1;
      a.lam2 = h->w.lam2;
      a.kstage = t.kstage;
      a.kst_off = t.kst_off;
      if (!beta_form) {
        // the form PCG runs: with the p^T q grid reduction and, when G beta is carried, (G p)_beta
        a.pcg_mode = 1;
        a.partials = h->d_partials;
        a.counter = h->d_counter;
        a.gp_out = incremental_gb(h) ? h->w.Gp : nullptr;
      }
    }
    trials.push_back({t, a, a.kstage == 2 ? t.smem_staged : t.smem, inv, 1e30f});
  }
  auto once = [&](const Trial& tr) -> cudaError_t {
    return launch_pass(kind, tr.inv, fp32, tr.t.E, tr.a, tr.t.threads, tr.smem, tr.t.grid, h->st);
  };
  for (const Trial& tr : trials) CK(once(tr));     // warm-up
  // three rounds over all candidates, five launches each, best round per candidate:
  // candidates interleaved in time, so that a drift of the clocks or of the memory
  // state during tuning does not favour the ones timed first
  for (int round = 0; round < 3; ++round) {
    for (Trial& tr : trials) {
      CK(cudaEventRecord(e0, h->st));
      for (int r = 0; r < 5; ++r) CK(once(tr));
      CK(cudaEventRecord(e1, h->st));
      CK(cudaEventSynchronize(e1));
      float m = 0.f;
      CK(cudaEventElapsedTime(&m, e0, e1));
      if (m < tr.ms) tr.ms = m;
    }
  }
  float best = 1e30f;
  PassCfg best_c = c;
  for (const Trial& tr : trials)
    if (tr.ms < best) { best = tr.ms; best_c = tr.t; }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c = best_c;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tuned[key] = {c.E, 1 << c.lgP, c.reg, c.kstage};
  tune_cache_append(key, g_tuned[key]);
  return IPM_OK;
}

ipm_status plan_passes(sdft_ipm* h, PassSet& ps, bool fp32) {
  const Layout& L = h->lay;
  const void *t64, *t32;
  ipm_status s;
  // middle pass.  Even Nl: complex FFT of length Nl/2, Hl rows, M pencils.
  // Odd Nl: complex FFT of length Nl carrying two pencils, Nl + 1 rows (the
  // half spectra of both staged first), ceil(M/2) pencil pairs.
  {
    PassCfg& c = ps.mid;
    const bool odd = (L.Nl & 1) != 0;
    if ((s = make_tables(h, odd ? L.Nl : L.Nl / 2, &t64, &t32)) != IPM_OK) return s;
    c.tw = fp32 ? t32 : t64;
    if ((s = make_tables(h, L.Nl, &t64, &t32)) != IPM_OK) return s;
    c.twN = fp32 ? t32 : t64;
    if (odd) {
      if ((s = tune_tile(h, c, 2, L.Nl, L.Nl + 1, (L.M + 1) / 2, fp32)) != IPM_OK) return s;
    } else {
      if ((s = tune_tile(h, c, 2, L.Nl / 2, L.Hl, L.M, fp32)) != IPM_OK) return s;
    }
  }
  if (L.d >= 2) {
    // row pass along the contiguous in-plane axis: rows of length Lr
    const int Lr = (L.d == 3) ? L.N1 : L.N0;
    const long long nrows = L.H / Lr;
    PassCfg c;
    if ((s = make_tables(h, Lr, &t64, &t32)) != IPM_OK) return s;
    c.tw = fp32 ? t32 : t64;
    PassCfg f = c, b = c, k = c;
    if ((s = tune_tile(h, c, 0, Lr, Lr, nrows, fp32)) != IPM_OK) return s;
    if ((s = tune_tile(h, f, 0, Lr, Lr, nrows, fp32, true)) != IPM_OK) return s;
    if ((s = tune_tile(h, k, 0, Lr, Lr, nrows, fp32, true, true)) != IPM_OK) return s;
    for (PassCfg* q : {&f, &k}) {
      if (h->opt.tile_kstage > 0) {
        PassCfg t = *q;
        if (stage_cfg(t, h->opt.tile_kstage - 1)) *q = t;
        else stage_cfg(*q, 0);
      } else if (!h->opt.autotune) {
        stage_cfg(*q, 0);
      }
    }
    if ((s = tune_tile(h, b, 0, Lr, Lr, nrows, fp32, false, true)) != IPM_OK) return s;
    ps.row_inv = c;
    ps.row_fwd = f;
    ps.row_fwd_k = k;
    ps.row_inv_beta = b;
  }
  if (L.d == 3) {
    // column tiles cover P consecutive k1 of one plane
    PassCfg c;
    if ((s = make_tables(h, L.N0, &t64, &t32)) != IPM_OK) return s;
    c.tw = fp32 ? t32 : t64;
    if ((s = tune_tile(h, c, 1, L.N0, L.N0, (long long)L.N1 * L.Hl, fp32)) != IPM_OK) return s;
    ps.col_inv = c;
    ps.col_fwd = c;
  }
  return IPM_OK;
}

PassArgs base_args(sdft_ipm* h, const PassCfg& c) {
  PassArgs a{};
  a.lay = h->lay;
  a.plan = c.plan;
  a.lgP = c.lgP;
  a.PP = c.PP;
  a.nwork = c.nwork;
  a.npencils = c.npencils;
  a.tw = c.tw;
  a.twN = c.twN;
  a.buf = h->d_U;
  a.maskw = h->d_maskw;
  a.inv_n = 1.0 / (double)h->lay.n;
  a.partials = h->d_partials;
  a.counter = h->d_counter;
  a.sc = h->d_sc;
  a.out_scale = 1.0;
  a.reg = c.reg;
  return a;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// A forward row pass with the K epilogue runs with its tuned operand staging (the
// operand pointers are 16-byte aligned on every path; checked all the same, since the
// bulk copies require it); every other launch of the same tile without.
ipm_status launch(sdft_ipm* h, const PassCfg& c, bool inv, bool fp32, PassArgs a) {
  ProfScope ps(h, c.kind);
  size_t smem = c.smem;
  a.kstage = 0;
  a.kst_off = 0;
  if (c.kstage && c.kind == 0 && !inv && a.mapout == MAPOUT_K && aligned16(a.p) && aligned16(a.lam1) &&
      aligned16(a.lam2)) {
    a.kstage = c.kstage;
    a.kst_off = c.kst_off;
    if (c.kstage == 2) smem = c.smem_staged;
  }
  CK(launch_pass(c.kind, inv, fp32, c.E, a, c.threads, smem, c.grid, h->st));
  return IPM_OK;
}

// What one application of G starts from and ends in.
struct GSpec {
  int mapin = MAPIN_BETA;
  const double* src = nullptr;   // MAPIN_BETA
  int mapout = MAPOUT_BETA;
  double* dst = nullptr;         // MAPOUT_BETA
  double out_scale = 1.0;
  bool pcg = false;              // MAPIN_PCG / MAPOUT_K inside PCG (p, zv, q of the handle)
  bool refine = false;           // only when the device asks for an FP64 residual replacement
  bool exact = false;            // only when the device asks for an exact G beta (incremental mode)
  bool cr = false;               // conjugate residuals: w = K z (z of the handle) with z^T w
  double* cr_in = nullptr;       // (cr) input and output of that product: z and w unless set
  double* cr_out = nullptr;
  const double* p_in = nullptr;  // kkt_apply: p and q given by the caller
  double* q_out = nullptr;
  int stall_log2 = 0;            // failure-detection test of the staged K epilogue (ipm_test_stage_stall)
};

// One application of G = A^T diag(m) A (with the chosen prologue/epilogue).
ipm_status run_g(sdft_ipm* h, bool fp32, const GSpec& g) {
  const Layout& L = h->lay;
  const PassSet& ps = fp32 ? h->pass32 : h->pass64;
  auto fill = [&](PassArgs& a, bool first, bool last) {
    if (first) {
      a.mapin = g.mapin;
      a.src = g.src;
      a.p = g.pcg ? h->w.p : const_cast<double*>(g.p_in);
      a.zv = h->w.zv;
    }
    if (last) {
      a.mapout = g.mapout;
      a.dst = g.dst;
      a.out_scale = g.out_scale;
      a.p = g.pcg ? h->w.p : const_cast<double*>(g.p_in);
      a.q = g.pcg ? h->w.q : g.q_out;
      a.lam1 = h->w.lam1;
      a.lam2 = h->w.lam2;
      a.pcg_mode = g.pcg ? 1 : 0;
    }
    if (g.cr) {
      double* in = g.cr_in ? g.cr_in : h->w.zv;
      if (first) { a.mapin = MAPIN_BETA; a.src = in; }
      if (last) {
        a.mapout = MAPOUT_K;
        a.p = in;
        a.q = g.cr_out ? g.cr_out : h->w.wcr;
        a.pcg_mode = 1;
        a.cr_mode = 1;
      }
    }
    a.check_done = (g.pcg || g.cr) ? 1 : 0;
    a.check_refine = g.refine ? 1 : 0;
    a.check_exact = g.exact ? 1 : 0;
    if (last) a.gp_out = (g.pcg && incremental_gb(h)) ? h->w.Gp : nullptr;
    if (last) a.kst_wait_log2 = g.stall_log2;
  };
  ipm_status s;
  if (L.d == 1) {
    PassArgs a = base_args(h, ps.mid);
    fill(a, true, true);
    return launch(h, ps.mid, false, fp32, a);
  }
  {
    const PassCfg& first = (g.mapin == MAPIN_BETA) ? ps.row_inv_beta : ps.row_inv;
    PassArgs a = base_args(h, first);
    fill(a, true, false);
    if ((s = launch(h, first, true, fp32, a)) != IPM_OK) return s;
  }
  if (L.d == 3) {
    PassArgs a = base_args(h, ps.col_inv);
    fill(a, false, false);
    if ((s = launch(h, ps.col_inv, true, fp32, a)) != IPM_OK) return s;
  }
  {
    PassArgs a = base_args(h, ps.mid);
    fill(a, false, false);
    if ((s = launch(h, ps.mid, false, fp32, a)) != IPM_OK) return s;
  }
  if (L.d == 3) {
    PassArgs a = base_args(h, ps.col_fwd);
    fill(a, false, false);
    if ((s = launch(h, ps.col_fwd, false, fp32, a)) != IPM_OK) return s;
  }
  const PassCfg& lastc = (g.mapout == MAPOUT_K && !g.pcg && !g.cr) ? ps.row_fwd_k : ps.row_fwd;
  PassArgs a = base_args(h, lastc);
  fill(a, false, true);
  return launch(h, lastc, false, fp32, a);
}

// c = M_perp^T b = B DFT(b_hat) / sqrt(n) scaling, in FP64 (Eq. (xi)).
ipm_status compute_c(sdft_ipm* h) {
  const Layout& L = h->lay;
  const PassSet& ps = h->pass64;
  const double scale = 1.0 / std::sqrt((double)L.n);
  PassArgs a = base_args(h, ps.mid);
  a.from_real = 1;
  a.yreal = h->d_y;
  ipm_status s;
  if (L.d == 1) {
    a.mapout = MAPOUT_BETA;
    a.dst = h->w.c;
    a.out_scale = scale;
    return launch(h, ps.mid, false, false, a);
  }
  if ((s = launch(h, ps.mid, false, false, a)) != IPM_OK) return s;
  if (L.d == 3) {
    PassArgs b = base_args(h, ps.col_fwd);
    if ((s = launch(h, ps.col_fwd, false, false, b)) != IPM_OK) return s;
  }
  PassArgs b = base_args(h, ps.row_fwd);
  b.mapout = MAPOUT_BETA;
  b.dst = h->w.c;
  b.out_scale = scale;
  return launch(h, ps.row_fwd, false, false, b);
}

ipm_status read_scalars(sdft_ipm* h) {
  CK(cudaMemcpyAsync(h->h_sc, h->d_sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  return IPM_OK;
}

ipm_status upload_problem(sdft_ipm* h, const uint8_t* mask, const double* y, double lambda) {
  const Layout& L = h->lay;
  if (!mask || !y) return fail_arg(h, "mask and y must not be NULL");
  if (!(lambda > 0.0) || !std::isfinite(lambda)) return fail_arg(h, "lambda must be positive and finite");
  CK(cudaMemcpyAsync(h->d_mask, mask, (size_t)L.n, cudaMemcpyDefault, h->st));
  CK(cudaMemcpyAsync(h->d_y, y, (size_t)L.n * sizeof(double), cudaMemcpyDefault, h->st));
  Reduce red{h->d_partials, h->d_counter};
  {
    ProfScope ps(h, 4);
    CK(k_pack_mask(h->d_mask, h->d_maskw, L.Nl, L.M, h->d_sc, h->st));
  }
  {
    ProfScope ps(h, 4);
    CK(k_observed_norm(h->d_y, h->d_mask, L.n, red, h->d_sc, h->st));
  }
  ipm_status s = compute_c(h);
  if (s != IPM_OK) return s;
  {
    ProfScope ps(h, 4);
    CK(k_cmax(h->w.c, 2 * L.H, lambda, h->opt.lambda_relative, red, h->d_sc, h->st));
  }
  h->lambda_in = lambda;
  h->point_set = false;
  return IPM_OK;
}

// After an upload: at least one observed sample and a positive lambda.
ipm_status check_resolved(sdft_ipm* h) {
  if (!(h->h_sc->nobs > 0)) return fail_arg(h, "the mask observes no sample");
  if (!(h->h_sc->lambda > 0) || !std::isfinite(h->h_sc->lambda))
    return fail_arg(h, "lambda resolved to a non-positive value (lambda_max = 0?)");
  return IPM_OK;
}

ipm_status check_options(sdft_ipm* h, const ipm_options& o) {
  if (o.precision != IPM_FP64 && o.precision != IPM_MIXED) return fail_arg(h, "precision must be IPM_FP64 or IPM_MIXED");
  if (!(o.gap_tol > 0) || !(o.cg_tol > 0)) return fail_arg(h, "gap_tol and cg_tol must be positive");
  if (o.max_ipm < 0 || o.max_cg < 1 || o.cg_chunk < 1) return fail_arg(h, "iteration caps must be positive");
  if (o.refine_every < 0) return fail_arg(h, "refine_every must be >= 0");
  if (o.tile_engine < 0 || o.tile_engine > 2) return fail_arg(h, "tile_engine must be 0, 1 or 2");
  if (o.sigma_rule < 0 || o.sigma_rule > 2) return fail_arg(h, "sigma_rule must be 0, 1 or 2");
  if (o.exact_residual < 0 || o.exact_residual > 1) return fail_arg(h, "exact_residual must be 0 or 1");
  if (!(o.precond_rho >= 0.0) || !std::isfinite(o.precond_rho)) return fail_arg(h, "precond_rho must be >= 0 and finite");
  if (o.pdl < 0 || o.pdl > 1) return fail_arg(h, "pdl must be 0 or 1");
  if (o.krylov < 0 || o.krylov > 2) return fail_arg(h, "krylov must be 0 (CG), 1 (CR) or 2 (CAr)");
  if (o.tile_kstage < 0 || o.tile_kstage > 3) return fail_arg(h, "tile_kstage must be 0 (tuned), 1, 2 or 3");
  if (o.krylov >= 1 && o.refine_every > 0) return fail_arg(h, "krylov = 1 (CR) or 2 (CAr) does not combine with refine_every");
  if (o.sigma_rule == 1 && !(o.sigma_min > 0 && o.sigma_min <= o.sigma_slow))
    return fail_arg(h, "sigma_min must lie in (0, sigma_slow]");
  if (o.sigma_rule == 2 && !(o.sigma_min >= 0 && o.sigma_min < 1))
    return fail_arg(h, "sigma_min must lie in [0, 1) for the predictor-corrector");
  if (!(o.sigma > 0 && o.sigma < 1) || !(o.sigma_slow > 0 && o.sigma_slow < 1)) return fail_arg(h, "sigma must lie in (0,1)");
  if (!(o.tau > 0 && o.tau < 1)) return fail_arg(h, "tau must lie in (0,1)");
  return IPM_OK;
}

}  // namespace

extern "C" {

void ipm_default_options(ipm_options* o) {
  if (!o) return;
  o->precision = IPM_FP64;
  o->gap_tol = 1e-6;
  o->cg_tol = 1e-6;
  o->cg_relative = 1;
  o->max_ipm = 200;
  o->max_cg = 500;
  o->sigma = 0.1;
  o->sigma_slow = 0.5;
  o->tau = 0.995;
  o->lambda_relative = 0;
  o->cg_chunk = 4;
  o->use_graph = 1;
  o->autotune = 1;
  o->tile_e = 0;
  o->tile_p = 0;
  o->refine_every = 0;
  o->tile_engine = 0;
  o->sigma_rule = 2;
  o->sigma_min = 0.01;
  o->exact_residual = 0;
  o->precond_rho = 1.0;
  o->pdl = 1;
  o->krylov = 0;
  o->tile_kstage = 0;
}

ipm_status ipm_create(sdft_ipm** out, int ndim, const int64_t* dims, const uint8_t* mask, const double* y, double lambda,
                      const ipm_options* opt, void* stream) {
  g_create_error.clear();
  if (!out) return fail_arg(nullptr, "out must not be NULL");
  *out = nullptr;
  if (ndim < 1 || ndim > 3 || !dims) return fail_arg(nullptr, "ndim must be 1, 2 or 3");
  for (int i = 0; i < ndim; ++i) {
    if (dims[i] < 2 || dims[i] > 1024 || !factor_ok((int)dims[i]))
      return fail_arg(nullptr, "every extent must be of the form 2^a 3^b 5^c 7^d, at least 2 and at most 1024");
  }
  ipm_options o;
  ipm_default_options(&o);
  if (opt) o = *opt;
  sdft_ipm* h = new sdft_ipm();
  h->opt = o;
  if (check_options(h, o) != IPM_OK) { g_create_error = h->err; delete h; return IPM_ERR_ARG; }
  cudaGetDevice(&h->device);
  h->st = (cudaStream_t)stream;
  for (int i = 0; i < ndim; ++i) h->dims[i] = (int)dims[i];
  h->lay = layout_init(ndim, ndim >= 2 ? (int)dims[0] : 1, ndim == 3 ? (int)dims[1] : 1, (int)dims[ndim - 1]);
  Layout& L = h->lay;
  if (!passes_launchable(L)) {
    g_create_error = "an extent has no launchable FFT tile (odd extents without a factor 3 must be at most 512)";
    delete h;
    return IPM_ERR_ARG;
  }
  auto cleanup_fail = [&](ipm_status s) {
    g_create_error = h->err;
    ipm_destroy(h);
    return s;
  };
#define CKC(call)                                                                   \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      h->err = std::string(#call) + ": " + cudaGetErrorString(e_);                  \
      return cleanup_fail(e_ == cudaErrorMemoryAllocation ? IPM_ERR_OOM : IPM_ERR_CUDA); \
    }                                                                               \
  } while (0)
  const size_t v2 = 2 * (size_t)L.H * sizeof(double), v4 = 2 * v2;
  CKC(dalloc(h, &h->d_mask, (size_t)L.n));
  CKC(dalloc(h, &h->d_y, (size_t)L.n * sizeof(double)));
  CKC(dalloc(h, &h->d_maskw, (size_t)((L.Nl + 31) / 32) * L.M * sizeof(uint32_t)));
  double** vec2[] = {&h->w.beta, &h->w.z, &h->w.s1, &h->w.s2, &h->w.nu1, &h->w.nu2, &h->w.c, &h->w.Gb,
                     &h->w.lam1, &h->w.lam2, &h->w.pa, &h->w.pb, &h->w.pc, &h->w.is1, &h->w.is2, &h->d_tmp,
                     &h->w.Gp, &h->w.Gx};
  for (double** p : vec2) CKC(dalloc(h, p, v2));
  double** vec4[] = {&h->w.x, &h->w.r, &h->w.zv, &h->w.p, &h->w.q, &h->w.rhs};
  for (double** p : vec4) CKC(dalloc(h, p, v4));
  // vectors of the other Krylov methods only when they are chosen
  if (o.krylov >= 1) for (double** p : {&h->w.wcr, &h->w.ucr}) CKC(dalloc(h, p, v4));
  if (o.krylov == 2) for (double** p : {&h->w.vcar, &h->w.Ucar}) CKC(dalloc(h, p, v4));
  // the predictor-corrector's affine direction only when it is chosen
  if (o.sigma_rule == 2)
    for (double** p : {&h->w.ds1a, &h->w.ds2a, &h->w.rba, &h->w.rca}) {
      CKC(dalloc(h, p, v2));
      CKC(cudaMemsetAsync(*p, 0, v2, h->st));
    }
  CKC(dalloc(h, &h->d_U, (size_t)L.H * 2 * sizeof(double)));
  CKC(cudaMemsetAsync(h->d_U, 0, (size_t)L.H * 2 * sizeof(double), h->st));
  CKC(dalloc(h, &h->d_sc, sizeof(DevScalars)));
  CKC(cudaMemsetAsync(h->d_sc, 0, sizeof(DevScalars), h->st));
  {
    void* p = nullptr;
    CKC(cudaMallocHost(&p, sizeof(DevScalars)));
    h->h_sc = (DevScalars*)p;
  }
  for (cudaStream_t& c : h->cap) CKC(cudaStreamCreateWithFlags(&c, cudaStreamNonBlocking));
  ipm_status s;
  // the tuner times row passes on p, z, Lambda1, Lambda2: give them normal,
  // non-zero values (every byte 0x3F) until the vectors are cleared below
  for (double* p : {h->w.p, h->w.zv, h->w.lam1, h->w.lam2})
    CKC(cudaMemsetAsync(p, 0x3F, (p == h->w.lam1 || p == h->w.lam2) ? v2 : v4, h->st));
  // partials of the grid reductions: up to 5 values per elementwise block (step_update:
  // mu and the certificate's four sums), 1 per block of an FFT pass that reduces (the
  // last pass of a PCG product, p^T q), whose tiles hold at least one pencil: allocated
  // before the tuner, which times that pass with its reduction
  size_t cap = 5 * (size_t)kMaxElementwiseBlocks;
  if (L.d >= 2) cap = std::max(cap, (size_t)(L.H / ((L.d == 3) ? L.N1 : L.N0)));
  cap = std::max(cap, (size_t)L.M);
  h->partial_cap = cap;
  CKC(dalloc(h, &h->d_partials, cap * sizeof(double)));
  CKC(dalloc(h, &h->d_counter, 64 * sizeof(unsigned)));
  CKC(cudaMemsetAsync(h->d_counter, 0, 64 * sizeof(unsigned), h->st));
  if ((s = plan_passes(h, h->pass64, false)) != IPM_OK) return cleanup_fail(s);
  if ((s = plan_passes(h, h->pass32, true)) != IPM_OK) return cleanup_fail(s);
  for (const PassSet* ps : {&h->pass64, &h->pass32})
    for (const PassCfg* c : {&ps->row_fwd, &ps->row_fwd_k, &ps->mid})
      if ((size_t)c->grid.x * c->grid.y * c->grid.z > cap) return cleanup_fail(fail_arg(h, "reduction partials too small"));
  // vectors start at 0 (ghosts stay 0 from here on)
  for (double** p : vec2) CKC(cudaMemsetAsync(*p, 0, v2, h->st));
  for (double** p : vec4) CKC(cudaMemsetAsync(*p, 0, v4, h->st));
  if ((s = upload_problem(h, mask, y, lambda)) != IPM_OK) return cleanup_fail(s);
  if ((s = read_scalars(h)) != IPM_OK) return cleanup_fail(s);
  if ((s = check_resolved(h)) != IPM_OK) return cleanup_fail(s);
#undef CKC
  *out = h;
  return IPM_OK;
}

ipm_status ipm_set_problem(sdft_ipm* h, const uint8_t* mask, const double* y, double lambda) {
  if (!h) return fail_arg(nullptr, "handle is NULL");
  ipm_status s = upload_problem(h, mask, y, lambda);
  if (s != IPM_OK) return s;
  if ((s = read_scalars(h)) != IPM_OK) return s;
  return check_resolved(h);
}

ipm_status ipm_set_options(sdft_ipm* h, const ipm_options* opt) {
  if (!h || !opt) return fail_arg(h, "handle and options must not be NULL");
  ipm_status s = check_options(h, *opt);
  if (s != IPM_OK) return s;
  const bool rel_changed = opt->lambda_relative != h->opt.lambda_relative;
  // vectors of a Krylov method chosen only now
  const size_t v4 = 4 * (size_t)h->lay.H * sizeof(double);
  if (opt->krylov >= 1 && !h->w.wcr)
    for (double** p : {&h->w.wcr, &h->w.ucr}) CK(dalloc(h, p, v4));
  if (opt->krylov == 2 && !h->w.vcar)
    for (double** p : {&h->w.vcar, &h->w.Ucar}) CK(dalloc(h, p, v4));
  if (opt->sigma_rule == 2 && !h->w.ds1a)
    for (double** p : {&h->w.ds1a, &h->w.ds2a, &h->w.rba, &h->w.rca}) {
      CK(dalloc(h, p, v4 / 2));
      CK(cudaMemsetAsync(*p, 0, v4 / 2, h->st));
    }
  h->opt = *opt;
  h->graph_valid = false;            // kernel arguments of the graph depend on the options
  if (rel_changed) {
    Reduce red{h->d_partials, h->d_counter};
    {
      ProfScope ps(h, 4);
      CK(k_cmax(h->w.c, 2 * h->lay.H, h->lambda_in, h->opt.lambda_relative, red, h->d_sc, h->st));
    }
    ipm_status r = read_scalars(h);
    return r != IPM_OK ? r : check_resolved(h);
  }
  return IPM_OK;
}

ipm_status ipm_sizes(const sdft_ipm* h, int64_t* nslots, int64_t* n) {
  if (!h) return IPM_ERR_ARG;
  if (nslots) *nslots = h->lay.H;
  if (n) *n = h->lay.n;
  return IPM_OK;
}

}  // extern "C"

namespace {

// Swap the handle onto a capturing stream with per-launch profiling off.
struct StreamSwap {
  sdft_ipm* h;
  cudaStream_t saved;
  bool prof;
  StreamSwap(sdft_ipm* h_, cudaStream_t s) : h(h_), saved(h_->st), prof(h_->prof) { h->st = s; h->prof = false; }
  ~StreamSwap() { h->st = saved; h->prof = prof; }
};

// Conditional handle for a WHILE node to be added to the graph being captured on h->st.
ipm_status make_cond(sdft_ipm* h, cudaGraphConditionalHandle* hc, unsigned dflt) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  CK(cudaStreamGetCaptureInfo(h->st, &cs, nullptr, &g, nullptr, nullptr, nullptr));
  if (cs != cudaStreamCaptureStatusActive) { h->err = "stream is not capturing"; return IPM_ERR_CUDA; }
  CK(cudaGraphConditionalHandleCreate(hc, g, dflt, cudaGraphCondAssignDefault));
  return IPM_OK;
}

// Append a WHILE node (condition hc) to the graph captured on h->st; its body is
// captured from `body` on stream bs.
template <typename F>
ipm_status add_while(sdft_ipm* h, cudaGraphConditionalHandle hc, cudaStream_t bs, F&& body) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* ed = nullptr;
  size_t nd = 0;
  CK(cudaStreamGetCaptureInfo(h->st, &cs, nullptr, &g, &deps, &ed, &nd));
  cudaGraphNodeParams p{};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = hc;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  CK(cudaGraphAddNode(&node, g, deps, ed, nd, &p));
  CK(cudaStreamUpdateCaptureDependencies(h->st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  cudaGraph_t bodyg = p.conditional.phGraph_out[0];
  CK(cudaStreamBeginCaptureToGraph(bs, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  ipm_status s;
  {
    StreamSwap sw(h, bs);
    s = body();
  }
  cudaGraph_t out = nullptr;
  cudaError_t e = cudaStreamEndCapture(bs, &out);
  if (s != IPM_OK) return s;
  CK(e);
  return IPM_OK;
}

// One IPM iteration as launched work: residual product, certificate + stop test,
// Newton system, PCG loop, step.  In graph mode `pcg_loop` wraps the PCG body
// in a WHILE node; in host mode the caller drives PCG.
ipm_status queue_residual_and_test(sdft_ipm* h, LoopCtl ipm_loop) {
  const Layout& L = h->lay;
  const ipm_options& o = h->opt;
  Reduce red{h->d_partials, h->d_counter};
  GSpec g;
  g.src = h->w.beta;
  g.dst = h->w.Gb;
  g.exact = incremental_gb(h) != 0;                    // incremental mode: only when a stop test is to be confirmed
  ipm_status s = run_g(h, false, g);                   // residual always in FP64
  if (s != IPM_OK) return s;
  ProfScope ps(h, kProfCertificate);
  CK(k_certificate(L, h->w.beta, h->w.Gb, h->w.c, red, h->d_sc, o.gap_tol, o.max_ipm, ipm_loop, h->st));
  return IPM_OK;
}

ipm_status queue_prepare(sdft_ipm* h, LoopCtl cg_loop) {
  Reduce red{h->d_partials, h->d_counter};
  const int pc = h->opt.sigma_rule == 2 ? 1 : 0;
  if (pc) {
    // single-step predictor-corrector: affine predictor from P^{-1}, Mehrotra's sigma and the
    // second-order terms in one pass, then the Newton system of the corrector
    ProfScope ps(h, kProfPrepare);
    CK(k_predictor(h->lay, h->w, red, h->d_sc, h->opt.precond_rho, h->opt.sigma_min, 1.0, h->st));
  }
  ProfScope ps(h, kProfPrepare);
  const int keep_rhs = (h->opt.precision == IPM_MIXED && h->opt.refine_every > 0) ? 1 : 0;
  CK(k_prepare(h->lay, h->w, red, h->d_sc, h->opt.cg_tol, h->opt.cg_relative, cg_loop, h->opt.precond_rho,
               h->opt.krylov == 2 ? 1 : 0, pc, keep_rhs, h->st));
  return IPM_OK;
}

ipm_status queue_pcg_iteration(sdft_ipm* h, LoopCtl cg_loop) {
  const bool mixed = h->opt.precision == IPM_MIXED;
  if (h->opt.krylov == 2) {
    // conjugate A-residuals: at a (re)start w = K z and y = P^{-1} w (the passes
    // and the kernel return at once otherwise), then v = K y and the two updates
    GSpec st;
    st.cr = true;
    st.refine = true;
    ipm_status s = run_g(h, mixed, st);
    if (s != IPM_OK) return s;
    {
      ProfScope ps(h, 3);
      CK(k_car_start(h->lay, h->w, h->d_sc, h->st));
    }
    GSpec k;
    k.cr = true;
    k.cr_in = h->w.ucr;
    k.cr_out = h->w.vcar;
    if ((s = run_g(h, mixed, k)) != IPM_OK) return s;
    Reduce red{h->d_partials, h->d_counter};
    ProfScope ps(h, 3);
    // the restart threshold: the unit round-off of the products' precision
    const double eps = mixed ? 1.1920928955078125e-07 : 2.220446049250313e-16;
    CK(k_car_update_a(h->lay, h->w, red, h->d_sc, eps, cg_loop, h->st));
    CK(k_car_update_b(h->lay, h->w, red, h->d_sc, h->opt.max_cg, cg_loop, h->st));
    return IPM_OK;
  }
  if (h->opt.krylov == 1) {
    // conjugate residuals: w = K z, then the two update kernels
    GSpec k;
    k.mapin = MAPIN_BETA;
    k.mapout = MAPOUT_K;
    k.cr = true;
    ipm_status s = run_g(h, h->opt.precision == IPM_MIXED, k);
    if (s != IPM_OK) return s;
    Reduce red{h->d_partials, h->d_counter};
    ProfScope ps(h, 3);
    CK(k_cr_update_a(h->lay, h->w, red, h->d_sc, cg_loop, h->st));
    CK(k_cr_update_b(h->lay, h->w, red, h->d_sc, h->opt.max_cg, cg_loop, h->st));
    return IPM_OK;
  }
  GSpec k;
  k.mapin = MAPIN_PCG;
  k.mapout = MAPOUT_K;
  k.pcg = true;
  ipm_status s = run_g(h, h->opt.precision == IPM_MIXED, k);
  if (s != IPM_OK) return s;
  Reduce red{h->d_partials, h->d_counter};
  const bool refine = h->opt.precision == IPM_MIXED && h->opt.refine_every > 0;
  {
    ProfScope ps(h, 3);
    CK(k_pcg_update(h->lay, h->w, red, h->d_sc, h->opt.max_cg, refine ? h->opt.refine_every : 0, cg_loop, h->st));
  }
  if (refine) {
    // q = K x with FP64 products, then r = rhs - q (kernels return at once unless asked)
    GSpec g;
    g.mapin = MAPIN_BETA;
    g.src = h->w.x;
    g.mapout = MAPOUT_K;
    g.p_in = h->w.x;
    g.q_out = h->w.q;
    g.refine = true;
    if ((s = run_g(h, false, g)) != IPM_OK) return s;
    ProfScope ps(h, 3);
    CK(k_refine(h->lay, h->w, red, h->d_sc, cg_loop, h->st));
  }
  return IPM_OK;
}

ipm_status queue_step(sdft_ipm* h) {
  Reduce red{h->d_partials, h->d_counter};
  {
    ProfScope ps(h, kProfStep);
    CK(k_step_length(h->lay, h->w, red, h->d_sc, h->opt.tau, h->opt.sigma_rule == 2 ? 1 : 0, h->st));
  }
  ProfScope ps(h, kProfStep);
  CK(k_step_update(h->lay, h->w, red, h->d_sc, h->opt.sigma, h->opt.sigma_slow, h->opt.sigma_rule,
                   h->opt.sigma_min, h->st));
  return IPM_OK;
}

// Queue, on the stream h->st that is being captured, the whole IPM loop:
//   WHILE (c_ipm):  G beta -> certificate (writes c_ipm) -> prepare (writes c_cg)
//                   WHILE (c_cg): K p passes -> pcg_update (writes c_cg)
//                   step length -> step update
ipm_status capture_solve_loop(sdft_ipm* h) {
  ipm_status s = make_cond(h, &h->c_ipm, 1u);
  if (s != IPM_OK) return s;
  return add_while(h, h->c_ipm, h->cap[1], [h]() -> ipm_status {
    ipm_status r = make_cond(h, &h->c_cg, 0u);
    if (r != IPM_OK) return r;
    if ((r = queue_residual_and_test(h, LoopCtl{h->c_ipm, 1})) != IPM_OK) return r;
    if ((r = queue_prepare(h, LoopCtl{h->c_cg, 1})) != IPM_OK) return r;
    r = add_while(h, h->c_cg, h->cap[2], [h]() -> ipm_status {
      return queue_pcg_iteration(h, LoopCtl{h->c_cg, 1});
    });
    if (r != IPM_OK) return r;
    return queue_step(h);
  });
}

// The solve loop of one handle as a graph of its own (the start point is set
// before each launch, outside the graph).
ipm_status build_graph(sdft_ipm* h) {
  if (h->gexec) { cudaGraphExecDestroy(h->gexec); h->gexec = nullptr; }
  if (h->graph) { cudaGraphDestroy(h->graph); h->graph = nullptr; }
  h->graph_valid = false;
  CK(cudaStreamBeginCapture(h->cap[0], cudaStreamCaptureModeRelaxed));
  ipm_status s;
  {
    StreamSwap sw(h, h->cap[0]);
    s = capture_solve_loop(h);
  }
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(h->cap[0], &g);
  if (s != IPM_OK) { if (g) cudaGraphDestroy(g); return s; }
  CK(e);
  h->graph = g;
  CK(cudaGraphInstantiate(&h->gexec, h->graph, 0));
  h->graph_valid = true;
  return IPM_OK;
}

ipm_status fill_result(sdft_ipm* h, ipm_result* res, double seconds) {
  const DevScalars& sc = *h->h_sc;
  ipm_status final_status = sc.ipm_status == 0 ? IPM_OK : (sc.ipm_status == 4 ? IPM_MAXITER : IPM_NUMERICAL);
  if (final_status == IPM_OK && sc.cg_cap_hit) final_status = IPM_KRYLOV_MAXITER;
  if (sc.wait_expired) final_status = IPM_TIMEOUT;
  if (res) {
    res->status = final_status;
    res->ipm_iters = sc.ipm_it;
    res->cg_iters_total = sc.cg_total;
    res->cg_iters_max = sc.cg_max;
    res->primal = sc.primal;
    res->dual = sc.dual;
    res->rel_gap = sc.gap;
    res->mu = sc.mu;
    res->lambda = sc.lambda;
    res->lambda_max = sc.cmax;
    res->kkt_products = sc.cg_total + sc.gb_products + sc.refinements;
    res->exact_products = sc.gb_products;
    res->seconds = seconds;
    res->refinements = sc.refinements;
  }
  if (final_status == IPM_NUMERICAL) h->err = "non-finite value or breakdown of positive definiteness";
  if (final_status == IPM_MAXITER) h->err = "IPM iteration cap reached before gap_tol";
  if (final_status == IPM_TIMEOUT) h->err = "a bounded device-side wait expired (staged K operands)";
  return final_status;
}

}  // namespace

extern "C" {

ipm_status ipm_solve(sdft_ipm* h, ipm_result* res) {
  if (!h) return fail_arg(nullptr, "handle is NULL");
  const auto t0 = std::chrono::steady_clock::now();
  const Layout& L = h->lay;
  const ipm_options& o = h->opt;
  Reduce red{h->d_partials, h->d_counter};
  ipm_status s;
  PdlScope pdl(o.pdl != 0);
  {
    ProfScope ps(h, 4);
    if (h->point_set) CK(k_mu(L, h->w, red, h->d_sc, o.sigma, incremental_gb(h), h->st));
    else CK(k_init_point(L, h->w, red, h->d_sc, o.sigma, incremental_gb(h), h->st));
  }
  h->point_set = false;
  const LoopCtl none{0, 0};
  if (o.use_graph && !h->prof) {
    if (!h->graph_valid && (s = build_graph(h)) != IPM_OK) return s;
    CK(cudaGraphLaunch(h->gexec, h->st));
  } else {
    // host-driven loop: the same kernels, the host reads the device decisions
    for (;;) {
      if ((s = queue_residual_and_test(h, none)) != IPM_OK) return s;
      if ((s = read_scalars(h)) != IPM_OK) return s;
      if (h->h_sc->ipm_done) break;
      if ((s = queue_prepare(h, none)) != IPM_OK) return s;
      for (;;) {
        for (int c = 0; c < o.cg_chunk; ++c)
          if ((s = queue_pcg_iteration(h, none)) != IPM_OK) return s;
        if ((s = read_scalars(h)) != IPM_OK) return s;
        if (h->h_sc->cg_done) break;
      }
      if ((s = queue_step(h)) != IPM_OK) return s;
    }
  }
  if ((s = read_scalars(h)) != IPM_OK) return s;
  prof_collect(h);
  h->sigma_ready = true;
  return fill_result(h, res, std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count());
}

ipm_status gapply(sdft_ipm* h, const double* p, double* q) {
  if (!h || !p || !q) return fail_arg(h, "NULL argument");
  if (!aligned16(p) || !aligned16(q)) return fail_arg(h, "p and q must be 16-byte aligned");
  GSpec g;
  g.src = p;
  g.dst = q;
  PdlScope pdl(h->opt.pdl != 0);
  ipm_status s = run_g(h, h->opt.precision == IPM_MIXED, g);
  if (s != IPM_OK) return s;
  CK(cudaStreamSynchronize(h->st));
  prof_collect(h);
  return IPM_OK;
}

ipm_status kkt_apply(sdft_ipm* h, const double* p, double* q) {
  if (!h || !p || !q) return fail_arg(h, "NULL argument");
  if (!h->sigma_ready) return fail_arg(h, "Sigma is not set: call ipm_set_sigma or ipm_solve first");
  if (!aligned16(p) || !aligned16(q)) return fail_arg(h, "p and q must be 16-byte aligned");
  GSpec g;
  g.mapin = MAPIN_BETA;
  g.src = p;
  g.mapout = MAPOUT_K;
  g.p_in = p;
  g.q_out = q;
  g.stall_log2 = h->stall_log2;
  h->stall_log2 = 0;
  const bool fp32 = h->opt.precision == IPM_MIXED;
  // a last pass that stages its operands on an mbarrier reports an expired wait
  const bool staged = h->lay.d >= 2 && (fp32 ? h->pass32 : h->pass64).row_fwd_k.kstage == 2;
  int* flag = &h->d_sc->wait_expired;
  if (staged) CK(cudaMemsetAsync(flag, 0, sizeof(int), h->st));
  PdlScope pdl(h->opt.pdl != 0);
  ipm_status s = run_g(h, fp32, g);
  if (s != IPM_OK) return s;
  if (staged) CK(cudaMemcpyAsync(&h->h_sc->wait_expired, flag, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  prof_collect(h);
  if (staged && h->h_sc->wait_expired) {
    h->err = "a bounded device-side wait expired (staged K operands)";
    return IPM_TIMEOUT;
  }
  return IPM_OK;
}

ipm_status ipm_test_stage_stall(sdft_ipm* h, int wait_log2) {
  if (!h) return fail_arg(nullptr, "handle is NULL");
  if (wait_log2 < 8 || wait_log2 > 24) return fail_arg(h, "wait_log2 must be in 8..24");
  const PassCfg& f = (h->opt.precision == IPM_MIXED ? h->pass32 : h->pass64).row_fwd_k;
  if (h->lay.d < 2 || f.kstage != 2) return fail_arg(h, "the last pass does not stage its operands in shared memory");
  h->stall_log2 = wait_log2;
  return IPM_OK;
}

ipm_status precond_apply(sdft_ipm* h, const double* r, double* z) {
  if (!h || !r || !z) return fail_arg(h, "NULL argument");
  if (!h->sigma_ready) return fail_arg(h, "Sigma is not set: call ipm_set_sigma or ipm_solve first");
  {
    ProfScope ps(h, 4);
    CK(k_precond(h->lay, h->w, r, z, h->d_sc, h->st));
  }
  CK(cudaStreamSynchronize(h->st));
  prof_collect(h);
  return IPM_OK;
}

ipm_status ipm_set_sigma(sdft_ipm* h, const double* s1, const double* nu1, const double* s2, const double* nu2) {
  if (!h || !s1 || !nu1 || !s2 || !nu2) return fail_arg(h, "NULL argument");
  {
    ProfScope ps(h, 4);
    CK(k_sigma_coef(h->lay, s1, nu1, s2, nu2, h->w, h->d_sc, h->opt.precond_rho, h->st));
  }
  CK(cudaStreamSynchronize(h->st));
  h->sigma_ready = true;
  return IPM_OK;
}

ipm_status ipm_set_point(sdft_ipm* h, const double* const wv[6]) {
  if (!h || !wv) return fail_arg(h, "NULL argument");
  for (int i = 0; i < 6; ++i)
    if (!wv[i]) return fail_arg(h, "NULL vector in the point");
  double* dst[6] = {h->w.beta, h->w.z, h->w.s1, h->w.s2, h->w.nu1, h->w.nu2};
  const size_t bytes = 2 * (size_t)h->lay.H * sizeof(double);
  for (int i = 0; i < 6; ++i) {
    CK(cudaMemcpyAsync(dst[i], wv[i], bytes, cudaMemcpyDefault, h->st));
    ProfScope ps(h, 4);
    CK(k_clear_ghosts(h->lay, dst[i], 1, h->d_sc, h->st));
  }
  CK(cudaStreamSynchronize(h->st));
  h->point_set = true;
  return IPM_OK;
}

ipm_status ipm_get_point(sdft_ipm* h, double* const wv[6]) {
  if (!h || !wv) return fail_arg(h, "NULL argument");
  const double* src[6] = {h->w.beta, h->w.z, h->w.s1, h->w.s2, h->w.nu1, h->w.nu2};
  const size_t bytes = 2 * (size_t)h->lay.H * sizeof(double);
  for (int i = 0; i < 6; ++i) {
    if (!wv[i]) return fail_arg(h, "NULL vector in the point");
    CK(cudaMemcpyAsync(wv[i], src[i], bytes, cudaMemcpyDefault, h->st));
  }
  CK(cudaStreamSynchronize(h->st));
  return IPM_OK;
}

ipm_status ipm_get_spectrum(sdft_ipm* h, double* v_half) {
  if (!h || !v_half) return fail_arg(h, "NULL argument");
  {
    ProfScope ps(h, 4);
    CK(k_unpack(h->lay, h->w.beta, h->d_tmp, h->d_sc, h->st));
  }
  CK(cudaMemcpyAsync(v_half, h->d_tmp, 2 * (size_t)h->lay.H * sizeof(double), cudaMemcpyDefault, h->st));
  CK(cudaStreamSynchronize(h->st));
  return IPM_OK;
}

ipm_status ipm_pack_beta(sdft_ipm* h, const double* v_half, double* beta) {
  if (!h || !v_half || !beta) return fail_arg(h, "NULL argument");
  {
    ProfScope ps(h, 4);
    CK(k_pack(h->lay, v_half, beta, h->d_sc, h->st));
  }
  CK(cudaStreamSynchronize(h->st));
  return IPM_OK;
}

ipm_status ipm_unpack_beta(sdft_ipm* h, const double* beta, double* v_half) {
  if (!h || !v_half || !beta) return fail_arg(h, "NULL argument");
  {
    ProfScope ps(h, 4);
    CK(k_unpack(h->lay, beta, v_half, h->d_sc, h->st));
  }
  CK(cudaStreamSynchronize(h->st));
  return IPM_OK;
}

ipm_status ipm_profile_enable(sdft_ipm* h, int on) {
  if (!h) return fail_arg(nullptr, "handle is NULL");
  prof_collect(h);
  h->prof = on != 0;
  for (int k = 0; k < kProfClasses; ++k) { h->prof_count[k] = 0; h->prof_ms[k] = 0; }
  ipm_status s = read_scalars(h);
  if (s != IPM_OK) return s;
  h->launch_base = h->h_sc->launches;
  return IPM_OK;
}

ipm_status ipm_profile_get(sdft_ipm* h, int k, int64_t* launches, double* ms) {
  if (!h || k < 0 || k >= kProfClasses) return fail_arg(h, "bad kernel class");
  prof_collect(h);
  if (k == 5) {
    ipm_status s = read_scalars(h);
    if (s != IPM_OK) return s;
    if (launches) *launches = (int64_t)(h->h_sc->launches - h->launch_base);
    if (ms) *ms = 0.0;
    return IPM_OK;
  }
  if (launches) *launches = h->prof_count[k];
  if (ms) *ms = h->prof_ms[k];
  return IPM_OK;
}

int ipm_describe(const sdft_ipm* h, char* buf, int len) {
  if (!h || !buf || len <= 0) return 0;
  std::string out = "{";
  auto one = [&](const char* name, const PassCfg& c) {
    char tmp[256];
    snprintf(tmp, sizeof(tmp), "\"%s\": {\"L\": %d, \"E\": %d, \"P\": %d, \"threads\": %d, \"blocks\": %u, "
             "\"smem\": %zu, \"engine\": \"%s\", \"kstage\": %d}", name, c.plan.L, c.E, 1 << c.lgP, c.threads,
             c.grid.x * c.grid.y, c.kstage == 2 ? c.smem_staged : c.smem, c.reg ? "register" : "shared", c.kstage);
    if (out.size() > 1) out += ", ";
    out += tmp;
  };
  for (int t = 0; t < 2; ++t) {
    const PassSet& ps = t ? h->pass32 : h->pass64;
    const std::string pre = t ? "fp32_" : "fp64_";
    one((pre + "middle").c_str(), ps.mid);
    if (h->lay.d >= 2) one((pre + "row").c_str(), ps.row_fwd);
    if (h->lay.d >= 2) one((pre + "row_k").c_str(), ps.row_fwd_k);
    if (h->lay.d >= 2) one((pre + "row_first").c_str(), ps.row_inv);
    if (h->lay.d >= 2) one((pre + "row_first_beta").c_str(), ps.row_inv_beta);
    if (h->lay.d == 3) one((pre + "col").c_str(), ps.col_fwd);
  }
  out += "}";
  snprintf(buf, (size_t)len, "%s", out.c_str());
  return (int)out.size();
}

const char* ipm_last_error(const sdft_ipm* h) {
  if (!h) return g_create_error.c_str();
  return h->err.c_str();
}

void ipm_destroy(sdft_ipm* h) {
  if (!h) return;
  if (h->st) cudaStreamSynchronize(h->st);
  else cudaDeviceSynchronize();
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->graph) cudaGraphDestroy(h->graph);
  for (cudaStream_t c : h->cap)
    if (c) cudaStreamDestroy(c);
  for (auto& e : h->prof_live) { cudaEventDestroy(e.a); cudaEventDestroy(e.b); }
  for (auto e : h->ev_pool) cudaEventDestroy(e);
  for (void* p : h->allocs) cudaFree(p);
  if (h->h_sc) cudaFreeHost(h->h_sc);
  delete h;
}

}  // extern "C"

namespace sdft {
// Message returned by ipm_last_error(NULL) (used by entry points without a handle).
void record_error(const char* msg) { g_create_error = msg; }
}  // namespace sdft

// ---------------------------------------------------------------------------
// Batched solve: many independent problems, one graph launch.  Each problem is
// a full handle; the batch graph forks one branch per problem (start point +
// its nested IPM / PCG WHILE loops) and joins them, so the problems' kernels run
// concurrently and the whole batch needs a single launch and a single wait.
// ---------------------------------------------------------------------------
struct sdft_ipm_batch {
  std::vector<sdft_ipm*> members;
  cudaStream_t st = nullptr;       // caller's stream
  cudaStream_t cap = nullptr;      // capture origin
  std::vector<cudaEvent_t> ev;     // join events (one per member) + the fork event
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  bool valid = false;
  std::string err;
};

namespace {

ipm_status batch_fail(sdft_ipm_batch* b, const std::string& msg, ipm_status st) {
  if (b) b->err = msg;
  g_create_error = msg;
  return st;
}

#define CKB(call)                                                                                   \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess) return batch_fail(b, std::string(#call) + ": " + cudaGetErrorString(e_), \
                                             IPM_ERR_CUDA);                                         \
  } while (0)

ipm_status build_batch_graph(sdft_ipm_batch* b) {
  if (b->gexec) { cudaGraphExecDestroy(b->gexec); b->gexec = nullptr; }
  if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
  b->valid = false;
  const int count = (int)b->members.size();
  CKB(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed));
  ipm_status s = IPM_OK;
  CKB(cudaEventRecord(b->ev[count], b->cap));          // fork point
  for (int i = 0; i < count && s == IPM_OK; ++i) {
    sdft_ipm* h = b->members[i];
    CKB(cudaStreamWaitEvent(h->cap[0], b->ev[count], 0));
    PdlScope pdl(h->opt.pdl != 0);
    {
      StreamSwap sw(h, h->cap[0]);
      Reduce red{h->d_partials, h->d_counter};
      cudaError_t e = k_init_point(h->lay, h->w, red, h->d_sc, h->opt.sigma, incremental_gb(h), h->st);
      if (e != cudaSuccess) s = batch_fail(b, std::string("init: ") + cudaGetErrorString(e), IPM_ERR_CUDA);
      if (s == IPM_OK) s = capture_solve_loop(h);
      if (s != IPM_OK && b->err.empty()) b->err = h->err;
    }
    if (s == IPM_OK) {
      CKB(cudaEventRecord(b->ev[i], h->cap[0]));
      CKB(cudaStreamWaitEvent(b->cap, b->ev[i], 0));    // join
    }
  }
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(b->cap, &g);
  if (s != IPM_OK) { if (g) cudaGraphDestroy(g); return s; }
  CKB(e);
  b->graph = g;
  CKB(cudaGraphInstantiate(&b->gexec, b->graph, 0));
  b->valid = true;
  return IPM_OK;
}

}  // namespace

extern "C" {

ipm_status ipm_create_batch(sdft_ipm_batch** out, int count, const int* ndims, const int64_t* dims,
                            const uint8_t* const* masks, const double* const* ys, const double* lambdas,
                            const ipm_options* opt, void* stream) {
  g_create_error.clear();
  if (!out) return fail_arg(nullptr, "out must not be NULL");
  *out = nullptr;
  if (count < 1 || !ndims || !dims || !masks || !ys || !lambdas)
    return fail_arg(nullptr, "count must be positive and every array non-NULL");
  sdft_ipm_batch* b = new sdft_ipm_batch();
  b->st = (cudaStream_t)stream;
  for (int i = 0; i < count; ++i) {
    sdft_ipm* h = nullptr;
    ipm_status s = ipm_create(&h, ndims[i], dims + 3 * (size_t)i, masks[i], ys[i], lambdas[i], opt, stream);
    if (s != IPM_OK) {
      const std::string msg = "problem " + std::to_string(i) + ": " + g_create_error;
      ipm_destroy_batch(b);
      g_create_error = msg;
      return s;
    }
    b->members.push_back(h);
  }
  cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  b->ev.resize(count + 1, nullptr);
  for (int i = 0; i <= count && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&b->ev[i], cudaEventDisableTiming);
  if (e != cudaSuccess) {
    g_create_error = std::string("batch streams/events: ") + cudaGetErrorString(e);
    ipm_destroy_batch(b);
    return IPM_ERR_CUDA;
  }
  *out = b;
  return IPM_OK;
}

ipm_status ipm_solve_batch(sdft_ipm_batch* b, ipm_result* results) {
  if (!b) return fail_arg(nullptr, "batch is NULL");
  const auto t0 = std::chrono::steady_clock::now();
  ipm_status s;
  if (!b->valid && (s = build_batch_graph(b)) != IPM_OK) return s;
  CKB(cudaGraphLaunch(b->gexec, b->st));
  CKB(cudaStreamSynchronize(b->st));
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  ipm_status worst = IPM_OK;
  for (size_t i = 0; i < b->members.size(); ++i) {
    sdft_ipm* h = b->members[i];
    if ((s = read_scalars(h)) != IPM_OK) return batch_fail(b, h->err, s);
    h->point_set = false;
    h->sigma_ready = true;
    const ipm_status si = fill_result(h, results ? &results[i] : nullptr, secs);
    if (si != IPM_OK && (worst == IPM_OK || worst == IPM_KRYLOV_MAXITER)) worst = si;
  }
  if (worst != IPM_OK) b->err = "at least one problem did not reach gap_tol (see its result)";
  return worst;
}

sdft_ipm* ipm_batch_member(sdft_ipm_batch* b, int i) {
  if (!b || i < 0 || i >= (int)b->members.size()) return nullptr;
  return b->members[i];
}

int ipm_batch_size(const sdft_ipm_batch* b) { return b ? (int)b->members.size() : 0; }

const char* ipm_batch_last_error(const sdft_ipm_batch* b) { return b ? b->err.c_str() : g_create_error.c_str(); }

void ipm_destroy_batch(sdft_ipm_batch* b) {
  if (!b) return;
  if (b->st) cudaStreamSynchronize(b->st);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (cudaEvent_t e : b->ev)
    if (e) cudaEventDestroy(e);
  if (b->cap) cudaStreamDestroy(b->cap);
  for (sdft_ipm* h : b->members) ipm_destroy(h);
  delete b;
}

}  // extern "C"

namespace sdft {
// Internal view of a handle for the warm-start code (warmstart.cu).
bool handle_view(sdft_ipm* h, HandleView* v) {
  if (!h || !v) return false;
  v->lay = h->lay;
  v->w = h->w;
  v->sc = h->d_sc;
  v->st = h->st;
  v->partials = h->d_partials;
  v->counter = h->d_counter;
  return true;
}
// The next ipm_solve starts from the point now in the handle's vectors.
void handle_point_set(sdft_ipm* h) { h->point_set = true; }
}  // namespace sdft
