// C-ABI of libxfft: context, setup pipeline and solver orchestration (see include/xfft.h).
//
// Solver loop (Algorithm 1, read as standard preconditioned CG on A u = -b):
//   f = -(b + A u0); z = P^-1 f; rr = f^T z; d = z
//   repeat: q = A d; alpha = rr / <q, d>; u += alpha d; f -= alpha q;
//           z = P^-1 f; rr' = f^T z; beta = rr'/rr; d = z + beta d
// until sqrt(rr / |Y|) <= tol ||<sigma(u)>_Y|| (eq. stoppingCriterion).
// Every scalar stays on the device; the host only polls the per-RHS activity flags.
//
// FP32_REFINED: iterative refinement.  The residual r = -(b + A u) of the FP64 iterate u is
// evaluated with the FP64 kernels and tested against the stopping rule; otherwise an FP32
// PCG solves A delta = r to a relative reduction inner_tol and u += delta.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <thread>
#include <type_traits>
#include <unordered_map>
#include <vector>

#include "../../include/xfft.h"
#include "xfft_kernels.h"

using namespace xfft;

static thread_local std::string g_err;

static xfft_status fail(xfft_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

#define CU(...)                                                                             \
  do {                                                                                      \
    cudaError_t e_ = (__VA_ARGS__);                                                         \
    if (e_ != cudaSuccess)                                                                  \
      return fail(e_ == cudaErrorMemoryAllocation ? XFFT_ENOMEM : XFFT_ECUDA,              \
                  std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e_));              \
  } while (0)

// device loop memory: one LoopState (padded to kLoopStride bytes) per loop of a graph
constexpr int kMaxBatch = 64;
constexpr size_t kLoopStride = 64;
constexpr size_t kLoopBytes = kLoopStride * kMaxBatch;

struct xfft_ctx;
static cudaError_t dalloc_bytes(xfft_ctx* c, void** p, size_t bytes);
static void dfree_bytes(xfft_ctx* c, void* p);

// Device allocations of a context go through these two: they keep the context's byte count
// (option max_device_bytes) and the size of every live block.
template <typename T>
static cudaError_t dalloc(xfft_ctx* c, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  return dalloc_bytes(c, (void**)p, count * sizeof(T));
}

template <typename T>
static void dfree(xfft_ctx* c, T*& p) {
  if (p) dfree_bytes(c, (void*)p);
  p = nullptr;
}

struct xfft_ctx {
  GridDev g;
  xfft_options opt;
  cudaStream_t stream;
  // microstructure
  bool have_micro = false;
  PhaseDev ph;
  double tau = 0.0;
  double* Ls = nullptr;
  double* Lin = nullptr;  // device copy of a host level set
  float* kcache = nullptr;  // cached FP32 cut-tet element matrices (kCutPacked x ncut)
  double* sig_keep = nullptr;  // [64][6] stress integrals of the last residual phase per RHS
  uint16_t* code = nullptr;
  int* cutcount = nullptr;
  int* enr_flag = nullptr;
  int* enr_id = nullptr;
  int* enr_nodes = nullptr;
  int* scan_tmp = nullptr;
  int* d_tot = nullptr;
  float* scale = nullptr;
  bool has_scale = false;
  int nX = -1, ncut = -1;
  int* cut_ip = nullptr;
  double* cut_dp = nullptr;
  float* cut_fp = nullptr;
  int4* cut_n4 = nullptr;
  int4* cut_e4 = nullptr;
  double* cut_r64 = nullptr;
  float* cut_r32 = nullptr;
  double* D = nullptr;
  double* isD = nullptr;
  float* isF = nullptr;
  // device-driven CG loops (a conditional while graph per inner solve), keyed by their arguments
  struct CgGraph {
    bool valid = false;
    bool dbl = false;
    int n_rhs = 0, crit = 0, maxit = 0, pe = 0;
    double tol = 0.0;
    long long limit = -1;
    const void* p[6] = {};
    cudaGraphExec_t exec = nullptr;
  } cg_graphs[4];
  int cg_next = 0;
  bool devloop_ok = true;            // false once a conditional graph could not be built
  unsigned char* loopmem = nullptr;  // device: LoopState, act pointers, RHS counts
  unsigned char* h_loop = nullptr;   // pinned host staging of loopmem
  cudaEvent_t ev_fork = nullptr;
  std::vector<cudaEvent_t> ev_join;
  double step0 = 0.0;  // step of the basic / Barzilai-Borwein schemes
  // block enriched preconditioner: off-diagonal block entries and the inverse blocks
  double* Doff = nullptr;
  double* eb64 = nullptr;
  float* eb32 = nullptr;
  FftPlan* fft = nullptr;
  // solver workspace
  int cap_rhs = 0;
  long long cap_stride = 0;
  int cap_prec = -1;
  double* v64[6] = {};  // u f d z q d' (FP64)
  float* v32[6] = {};   // u f d z q d' (FP32); d and d' alternate as old / new direction
  void* spec = nullptr;
  size_t spec_bytes = 0;
  RhsState* st = nullptr;
  int* act = nullptr;
  int* outer_mask = nullptr;
  double* eps_d = nullptr;
  double* partials = nullptr;
  size_t partials_count = 0;
  double* red_out = nullptr;
  int* h_act = nullptr;          // pinned
  RhsState* h_st = nullptr;      // pinned
  // checkpoint of the six unit load cases (scaled DOFs, FP64)
  double* U6 = nullptr;
  bool have6 = false;
  double C6[36];
  double* dscale = nullptr;
  float* dscale_f = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // tracing
  struct PE {
    int kind, nlaunch;
    cudaEvent_t a, b;
  };
  bool prof = false;
  std::vector<PE> pend;
  std::vector<cudaEvent_t> evpool;
  double pms[16] = {};
  long long plaunch[16] = {};
  unsigned long long* punits = nullptr;  // device, 16 counters
  // device memory owned by the context (option max_device_bytes)
  std::unordered_map<void*, size_t> blocks;
  size_t bytes = 0;
  // Euclidean Barzilai-Borwein steps: <d, d>, <A d, A d> partial sums
  double* bbpart = nullptr;
  // launch shapes picked by the tuner (0: defaults): the FP32 cut-tet kernel's grid and
  // right-hand sides per launch, the FP32 preconditioner's right-hand sides per FFT pass group
  int cut_blocks = 0, cut_rpl = 0, prec_group = 0;
  bool tuned = false;
};

static cudaError_t dalloc_bytes(xfft_ctx* c, void** p, size_t bytes) {
  *p = nullptr;
  if (c->opt.max_device_bytes > 0 && c->bytes + bytes > (size_t)c->opt.max_device_bytes)
    return cudaErrorMemoryAllocation;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return e;
  }
  c->blocks[*p] = bytes;
  c->bytes += bytes;
  return cudaSuccess;
}

static void dfree_bytes(xfft_ctx* c, void* p) {
  auto it = c->blocks.find(p);
  if (it != c->blocks.end()) {
    c->bytes -= it->second;
    c->blocks.erase(it);
  }
  cudaFree(p);
}

static xfft_status noalloc_prepare(cudaStream_t stream);

static cudaEvent_t prof_event(xfft_ctx* c) {
  if (!c->evpool.empty()) {
    cudaEvent_t e = c->evpool.back();
    c->evpool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Brackets a group of kernel launches with events on the context's stream (tracing only).
struct ProfScope {
  xfft_ctx* c;
  int kind, n;
  cudaEvent_t a = nullptr;
  ProfScope(xfft_ctx* c_, int kind_, int n_) : c(c_), kind(kind_), n(n_) {
    if (c->prof) {
      a = prof_event(c);
      cudaEventRecord(a, c->stream);
    }
  }
  ~ProfScope() {
    if (c->prof && a) {
      cudaEvent_t b = prof_event(c);
      cudaEventRecord(b, c->stream);
      c->pend.push_back({kind, n, a, b});
    }
  }
};

// fold finished event pairs into the totals (synchronises the stream)
static cudaError_t prof_flush(xfft_ctx* c) {
  if (c->pend.empty()) return cudaSuccess;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return e;
  for (auto& pe : c->pend) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, pe.a, pe.b);
    c->pms[pe.kind] += ms;
    c->plaunch[pe.kind] += pe.nlaunch;
    c->evpool.push_back(pe.a);
    c->evpool.push_back(pe.b);
  }
  c->pend.clear();
  return cudaSuccess;
}

static unsigned long long* punit(xfft_ctx* c, int kind) { return c->prof ? c->punits + kind : nullptr; }

static CutData cutdata(const xfft_ctx* c) {
  CutData cd;
  cd.ip = c->cut_ip;
  cd.dp = c->cut_dp;
  cd.fp = c->cut_fp;
  cd.ncut = c->ncut;
  cd.n4 = c->cut_n4;
  cd.e4 = c->cut_e4;
  cd.r64 = c->cut_r64;
  cd.r32 = c->cut_r32;
  return cd;
}

static long long stride_of(const xfft_ctx* c) { return 3LL * (c->g.N + c->nX); }

static bool good_len(int n) {
  if (n < 4 || n > 1024 || (n & 1)) return false;
  int m = n;
  for (int p : {2, 3, 5})
    while (m % p == 0) m /= p;
  return m == 1;
}

extern "C" const char* xfft_last_error(void) { return g_err.c_str(); }

extern "C" const char* xfft_status_string(xfft_status s) {
  switch (s) {
    case XFFT_OK: return "ok";
    case XFFT_EINVAL: return "invalid argument";
    case XFFT_ENOMEM: return "out of memory";
    case XFFT_ECUDA: return "CUDA error";
    case XFFT_ENOTCONV: return "not converged";
    case XFFT_EBREAKDOWN: return "CG breakdown";
    case XFFT_ETIMEOUT: return "device wait timed out";
    case XFFT_EUNSUPPORTED: return "unsupported";
    case XFFT_ESTATE: return "invalid call order";
  }
  return "unknown status";
}

extern "C" xfft_status xfft_default_options(xfft_options* opt) {
  if (!opt) return fail(XFFT_EINVAL, "opt is NULL");
  opt->precision = XFFT_FP64;
  opt->tol = 1e-10;
  opt->maxit = 10000;
  opt->snap_tau = 0.0;
  opt->enr_precond = XFFT_ENR_IDENTITY;
  opt->inner_tol = 1e-5;
  opt->max_refine = 20;
  opt->poll_every = 8;
  opt->scheme = XFFT_SCHEME_CG;
  opt->step = 0.0;
  opt->cut_cache = 0;
  opt->bb_rule = XFFT_BB1;
  opt->bb_cycle = 1;
  opt->enrichment = 1;
  opt->max_device_bytes = 0;
  opt->spin_limit_ns = -1;
  opt->autotune = 1;
  opt->residual_update = 1;
  return XFFT_OK;
}

extern "C" xfft_status xfft_create(xfft_ctx** out, const xfft_grid* grid, const xfft_options* opt,
                                   void* stream) {
  if (!out || !grid) return fail(XFFT_EINVAL, "NULL argument");
  *out = nullptr;
  for (int a = 0; a < 3; ++a) {
    if (!good_len(grid->n[a]))
      return fail(XFFT_EINVAL, "grid size must be even, 2^a 3^b 5^c and in [4, 1024]");
    if (!(grid->len[a] > 0.0)) return fail(XFFT_EINVAL, "cell lengths must be positive");
  }
  const long long N = (long long)grid->n[0] * grid->n[1] * grid->n[2];
  if (N > (1LL << 28)) return fail(XFFT_EUNSUPPORTED, "more than 2^28 voxels");
  xfft_options o;
  xfft_default_options(&o);
  if (opt) o = *opt;
  if (o.precision != XFFT_FP64 && o.precision != XFFT_FP32_REFINED)
    return fail(XFFT_EINVAL, "unknown precision");
  if (o.enr_precond != XFFT_ENR_IDENTITY && o.enr_precond != XFFT_ENR_BLOCK3)
    return fail(XFFT_EINVAL, "unknown enriched preconditioner");
  if (o.scheme != XFFT_SCHEME_CG && o.scheme != XFFT_SCHEME_BASIC && o.scheme != XFFT_SCHEME_BB &&
      o.scheme != XFFT_SCHEME_NLCG)
    return fail(XFFT_EINVAL, "unknown iteration scheme");
  if (o.cut_cache != 0 && o.cut_cache != 1) return fail(XFFT_EINVAL, "cut_cache must be 0 or 1");
  if (o.bb_rule < XFFT_BB1 || o.bb_rule > XFFT_BB2_EUCLID || o.bb_cycle < 1)
    return fail(XFFT_EINVAL, "unknown Barzilai-Borwein rule or bb_cycle < 1");
  if (o.enrichment != 0 && o.enrichment != 1) return fail(XFFT_EINVAL, "enrichment must be 0 or 1");
  if (o.max_device_bytes < 0) return fail(XFFT_EINVAL, "max_device_bytes must be >= 0");
  if (o.autotune != 0 && o.autotune != 1) return fail(XFFT_EINVAL, "autotune must be 0 or 1");
  if (o.residual_update != 0 && o.residual_update != 1) return fail(XFFT_EINVAL, "residual_update must be 0 or 1");
  if (!(o.tol > 0.0) || o.maxit < 1 || o.poll_every < 1 || o.max_refine < 1 || !(o.inner_tol > 0.0))
    return fail(XFFT_EINVAL, "invalid options");
  xfft_ctx* c = new xfft_ctx();
  c->opt = o;
  c->stream = (cudaStream_t)stream;
  GridDev& g = c->g;
  g.n0 = grid->n[0];
  g.n1 = grid->n[1];
  g.n2 = grid->n[2];
  g.N = N;
  for (int a = 0; a < 3; ++a) g.h[a] = grid->len[a] / grid->n[a];
  g.vol_tet = g.h[0] * g.h[1] * g.h[2] / 6.0;
  g.volY = grid->len[0] * grid->len[1] * grid->len[2];
  cudaError_t e = cudaSuccess;
  c->fft = fft_plan_create(g, &e);
  if (!c->fft || e != cudaSuccess) {
    delete c;
    return fail(XFFT_ECUDA, std::string("FFT plan: ") + cudaGetErrorString(e));
  }
  if ((e = cudaEventCreate(&c->ev0)) != cudaSuccess || (e = cudaEventCreate(&c->ev1)) != cudaSuccess ||
      (e = cudaMallocHost((void**)&c->h_act, 64 * sizeof(int))) != cudaSuccess ||
      (e = cudaMallocHost((void**)&c->h_st, 64 * sizeof(RhsState))) != cudaSuccess ||
      (e = cudaMalloc((void**)&c->punits, 16 * sizeof(unsigned long long))) != cudaSuccess ||
      (e = cudaMemset(c->punits, 0, 16 * sizeof(unsigned long long))) != cudaSuccess ||
      (e = cudaMalloc((void**)&c->loopmem, kLoopBytes)) != cudaSuccess ||
      (e = cudaMallocHost((void**)&c->h_loop, kLoopBytes)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming)) != cudaSuccess) {
    xfft_destroy(c);
    return fail(XFFT_ECUDA, cudaGetErrorString(e));
  }
  c->ev_join.assign(1, nullptr);
  if ((e = cudaEventCreateWithFlags(&c->ev_join[0], cudaEventDisableTiming)) != cudaSuccess) {
    xfft_destroy(c);
    return fail(XFFT_ECUDA, cudaGetErrorString(e));
  }
  *out = c;
  return XFFT_OK;
}

static void drop_graphs(xfft_ctx* c) {
  for (auto& g : c->cg_graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g = xfft_ctx::CgGraph();
  }
}

static void free_micro(xfft_ctx* c) {
  drop_graphs(c);
  c->tuned = false;
  c->cut_blocks = c->cut_rpl = c->prec_group = 0;
  dfree(c, c->Ls);
  dfree(c, c->Lin);
  dfree(c, c->kcache);
  dfree(c, c->code);
  dfree(c, c->cutcount);
  dfree(c, c->enr_flag);
  dfree(c, c->enr_id);
  dfree(c, c->enr_nodes);
  dfree(c, c->scan_tmp);
  dfree(c, c->d_tot);
  dfree(c, c->scale);
  dfree(c, c->cut_ip);
  dfree(c, c->cut_dp);
  dfree(c, c->cut_fp);
  dfree(c, c->cut_n4);
  dfree(c, c->cut_e4);
  dfree(c, c->cut_r64);
  dfree(c, c->cut_r32);
  dfree(c, c->D);
  dfree(c, c->isD);
  dfree(c, c->isF);
  dfree(c, c->Doff);
  dfree(c, c->eb64);
  dfree(c, c->eb32);
  dfree(c, c->U6);
  dfree(c, c->dscale);
  dfree(c, c->dscale_f);
  c->have_micro = false;
  c->have6 = false;
  c->nX = c->ncut = -1;
}

static void free_work(xfft_ctx* c) {
  drop_graphs(c);
  for (int k = 0; k < 6; ++k) {
    dfree(c, c->v64[k]);
    dfree(c, c->v32[k]);
  }
  if (c->spec) dfree_bytes(c, c->spec);
  c->spec = nullptr;
  dfree(c, c->st);
  dfree(c, c->act);
  dfree(c, c->outer_mask);
  dfree(c, c->eps_d);
  dfree(c, c->sig_keep);
  dfree(c, c->partials);
  dfree(c, c->red_out);
  dfree(c, c->bbpart);
  c->cap_rhs = 0;
  c->cap_stride = 0;
  c->cap_prec = -1;
}

extern "C" void xfft_destroy(xfft_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  free_micro(c);
  free_work(c);
  fft_plan_destroy(c->fft);
  if (c->h_act) cudaFreeHost(c->h_act);
  if (c->h_st) cudaFreeHost(c->h_st);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  for (auto& pe : c->pend) {
    cudaEventDestroy(pe.a);
    cudaEventDestroy(pe.b);
  }
  for (auto e : c->evpool) cudaEventDestroy(e);
  if (c->punits) cudaFree(c->punits);
  if (c->loopmem) cudaFree(c->loopmem);
  if (c->h_loop) cudaFreeHost(c->h_loop);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  for (auto e : c->ev_join)
    if (e) cudaEventDestroy(e);
  for (auto& kv : c->blocks) cudaFree(kv.first);  // anything a failed call left behind
  delete c;
}

extern "C" xfft_status xfft_get_tuning(const xfft_ctx* c, int* cut_blocks, int* cut_rhs_per_launch,
                                       int* prec_rhs_per_group) {
  if (!c || !cut_blocks || !cut_rhs_per_launch || !prec_rhs_per_group) return fail(XFFT_EINVAL, "NULL argument");
  if (!c->have_micro) return fail(XFFT_ESTATE, "xfft_set_microstructure first");
  *cut_blocks = c->cut_blocks > 0 ? c->cut_blocks : apply_cut_blocks(c->ncut);
  *cut_rhs_per_launch = c->cut_rpl > 0 ? c->cut_rpl : 8;
  *prec_rhs_per_group = c->prec_group > 0 ? c->prec_group : 64;
  return XFFT_OK;
}

extern "C" int xfft_num_enriched(const xfft_ctx* c) { return c && c->have_micro ? c->nX : -1; }
extern "C" int xfft_num_cut_tets(const xfft_ctx* c) { return c && c->have_micro ? c->ncut : -1; }

// ---------------------------------------------------------------- microstructure setup
extern "C" xfft_status xfft_set_microstructure(xfft_ctx* c, const double* L, const double lame_minus[2],
                                               const double lame_plus[2], const float* voxel_scale,
                                               int ptrs_on_device) {
  if (!c || !L || !lame_minus || !lame_plus) return fail(XFFT_EINVAL, "NULL argument");
  const double lame[4] = {lame_minus[0], lame_minus[1], lame_plus[0], lame_plus[1]};
  return xfft_set_microstructure_phases(c, 1, L, lame, voxel_scale, ptrs_on_device);
}

extern "C" xfft_status xfft_set_microstructure_phases(xfft_ctx* c, int n_levelsets, const double* L,
                                                      const double* lame, const float* voxel_scale,
                                                      int ptrs_on_device) {
  if (!c || !L || !lame) return fail(XFFT_EINVAL, "NULL argument");
  if (n_levelsets < 1 || n_levelsets > XFFT_MAX_LEVELSETS)
    return fail(XFFT_EINVAL, "n_levelsets must be 1 .. XFFT_MAX_LEVELSETS");
  const int nph = n_levelsets + 1;
  for (int p = 0; p < nph; ++p)
    if (!(lame[2 * p + 1] > 0.0) || !(3.0 * lame[2 * p] + 2.0 * lame[2 * p + 1] > 0.0))
      return fail(XFFT_EINVAL, "Lame constants must give a positive definite stiffness");
  free_micro(c);
  const GridDev& g = c->g;
  const long long N = g.N;
  cudaStream_t s = c->stream;
  CU(cudaEventRecord(c->ev0, s));
  for (int p = 0; p < kMaxPhases; ++p) {
    c->ph.lam[p] = p < nph ? lame[2 * p] : 0.0;
    c->ph.mu[p] = p < nph ? lame[2 * p + 1] : 0.0;
  }
  c->ph.nph = nph;
  c->tau = c->opt.snap_tau > 0.0 ? c->opt.snap_tau : 1e-6 * std::min(g.h[0], std::min(g.h[1], g.h[2]));
  CU(dalloc(c, &c->Ls, (size_t)n_levelsets * N));
  CU(dalloc(c, &c->code, N));
  CU(dalloc(c, &c->cutcount, N));
  CU(dalloc(c, &c->enr_flag, N));
  CU(dalloc(c, &c->enr_id, N));
  CU(dalloc(c, &c->scan_tmp, scan_tmp_ints(N)));
  CU(dalloc(c, &c->d_tot, 16));
  const double* Ldev = L;
  if (!ptrs_on_device) {
    CU(dalloc(c, &c->Lin, (size_t)n_levelsets * N));
    CU(cudaMemcpyAsync(c->Lin, L, n_levelsets * N * sizeof(double), cudaMemcpyHostToDevice, s));
    Ldev = c->Lin;
  }
  if (voxel_scale) {
    CU(dalloc(c, &c->scale, N));
    CU(cudaMemcpyAsync(c->scale, voxel_scale, N * sizeof(float),
                       ptrs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    c->has_scale = true;
  } else {
    c->has_scale = false;
  }
  // step of the basic and Barzilai-Borwein schemes, s0 = 2 / (C_- + C_+) (eq. stepsize): the
  // extreme stiffness eigenvalues (2 mu, 3 lambda + 2 mu per phase) times the extreme scales
  c->step0 = c->opt.step;
  if (c->opt.scheme != XFFT_SCHEME_CG && !(c->step0 > 0.0)) {
    double smin = 1.0, smax = 1.0;
    if (voxel_scale) {
      std::vector<float> hs(N);
      CU(cudaMemcpyAsync(hs.data(), c->scale, N * sizeof(float), cudaMemcpyDeviceToHost, s));
      CU(cudaStreamSynchronize(s));
      smin = smax = hs[0];
      for (long long i = 1; i < N; ++i) {
        smin = std::min(smin, (double)hs[i]);
        smax = std::max(smax, (double)hs[i]);
      }
    }
    double ev[2 * kMaxPhases];
    for (int p = 0; p < nph; ++p) {
      ev[2 * p] = 2.0 * lame[2 * p + 1];
      ev[2 * p + 1] = 3.0 * lame[2 * p] + 2.0 * lame[2 * p + 1];
    }
    const double cmin = *std::min_element(ev, ev + 2 * nph) * smin;
    const double cmax = *std::max_element(ev, ev + 2 * nph) * smax;
    c->step0 = 2.0 / (cmin + cmax);
  }
  ProfScope ps_setup(c, XFFT_PROF_SETUP, 15);
  CU(launch_count_nonfinite(Ldev, (long long)n_levelsets * N, c->has_scale ? c->scale : nullptr, N,
                            c->d_tot + 4, s));
  CU(launch_snap_classify(Ldev, c->Ls, n_levelsets, c->code, c->cutcount, c->enr_flag, c->d_tot + 3,
                          g, c->tau, c->opt.enrichment ? 0 : 1, s));
  // enriched ids (scan of node flags) and cut-tet offsets (scan of per-voxel counts)
  CU(launch_scan(c->enr_flag, c->enr_id, N, c->d_tot + 0, c->scan_tmp, s));
  CU(launch_scan(c->cutcount, c->cutcount, N, c->d_tot + 1, c->scan_tmp, s));
  int tot[8];
  CU(cudaMemcpyAsync(tot, c->d_tot, 8 * sizeof(int), cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  if (tot[4] > 0) return fail(XFFT_EINVAL, "the level set holds NaN or Inf values");
  if (tot[5] > 0) return fail(XFFT_EINVAL, "the voxel scale holds NaN or Inf values");
  if (tot[3] > 0) return fail(XFFT_EINVAL, "a tet is cut by two interfaces (one interface per element)");
  c->nX = tot[0];
  c->ncut = tot[1];
  CU(dalloc(c, &c->enr_nodes, c->nX));
  CU(dalloc(c, &c->cut_ip, (size_t)kCutInts * c->ncut));
  CU(dalloc(c, &c->cut_dp, (size_t)kCutReals * c->ncut));
  CU(dalloc(c, &c->cut_fp, (size_t)kCutReals * c->ncut));
  {
    int* chunk_tmp = nullptr;
    CU(dalloc(c, &chunk_tmp, 2 * (size_t)chunk_ints(c->ncut)));
    const cudaError_t eb = launch_build_lists(c->code, c->cutcount, c->enr_flag, c->enr_id, c->enr_nodes,
                                              c->cut_ip, c->ncut, g, c->d_tot + 8, c->scan_tmp, chunk_tmp,
                                              chunk_tmp + chunk_ints(c->ncut), s);
    CU(cudaStreamSynchronize(s));
    dfree(c, chunk_tmp);
    CU(eb);
  }
  CutData cd = cutdata(c);
  CU(launch_cut_geometry(c->Ls, n_levelsets, cd, c->cut_dp, c->cut_ip, g, s));
  CU(launch_cut_eids(c->cut_ip, c->enr_id, c->ncut, s));
  CU(dalloc(c, &c->D, 3 * (size_t)c->nX));
  CU(dalloc(c, &c->isD, 3 * (size_t)c->nX));
  CU(dalloc(c, &c->isF, 3 * (size_t)c->nX));
  const bool blk = c->opt.enr_precond == XFFT_ENR_BLOCK3;
  if (blk) {
    CU(dalloc(c, &c->Doff, 3 * (size_t)c->nX));
    CU(dalloc(c, &c->eb64, 6 * (size_t)c->nX));
    CU(dalloc(c, &c->eb32, 6 * (size_t)c->nX));
  }
  CU(launch_cut_scaling(cd, c->D, blk ? c->Doff : nullptr, c->nX, g, s));
  CU(launch_finish_scaling(c->D, c->isD, c->isF, c->nX, s));
  if (blk) {
    int* bad = c->d_tot + 2;
    CU(cudaMemsetAsync(bad, 0, sizeof(int), s));
    CU(launch_block_inverse(c->D, c->Doff, c->isD, c->eb64, c->eb32, c->nX, bad, s));
    int hbad = 0;
    CU(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (hbad) return fail(XFFT_EBREAKDOWN, "an enriched 3x3 block is not positive definite");
  }
  CU(launch_cut_to_float(c->cut_dp, c->cut_fp, (long long)kCutReals * c->ncut, s));
  CU(dalloc(c, &c->cut_n4, c->ncut));
  CU(dalloc(c, &c->cut_e4, c->ncut));
  CU(dalloc(c, &c->cut_r64, (size_t)kRec * c->ncut));
  CU(dalloc(c, &c->cut_r32, (size_t)kRec * c->ncut));
  CU(launch_cut_records(cd, c->isD, c->nX, g, c->ph, c->has_scale ? c->scale : nullptr, c->cut_n4,
                        c->cut_e4, c->cut_r64, c->cut_r32, s));
  if (c->opt.precision == XFFT_FP32_REFINED && c->opt.cut_cache && c->ncut > 0) {
    CU(dalloc(c, &c->kcache, (size_t)kCutPacked * c->ncut));
    CU(launch_cut_matrix(cd, c->isD, c->nX, g, c->ph, c->has_scale ? c->scale : nullptr, c->kcache, s));
  }
  CU(cudaEventRecord(c->ev1, s));
  CU(cudaStreamSynchronize(s));
  {
    const xfft_status ps = noalloc_prepare(s);
    if (ps != XFFT_OK) return ps;
  }
  c->have_micro = true;
  c->have6 = false;
  return XFFT_OK;
}

// ---------------------------------------------------------------- workspace
static bool bb_euclid(const xfft_ctx* c) {
  return c->opt.scheme == XFFT_SCHEME_BB &&
         (c->opt.bb_rule == XFFT_BB1_EUCLID || c->opt.bb_rule == XFFT_BB2_EUCLID);
}

static FinArgs fin_args(const xfft_ctx* c, int mode, int crit, double tol, int maxit, int nparts,
                        int nparts_used, int parity) {
  FinArgs fa;
  fa.scheme = c->opt.scheme;
  fa.step0 = c->step0;
  fa.mode = mode;
  fa.crit = crit;
  fa.tol = tol;
  fa.volY = c->g.volY;
  fa.maxit = maxit;
  fa.nparts = nparts;
  fa.nparts_used = nparts_used;
  fa.set_rel = 0;
  fa.inner_floor = 0.0;
  fa.parity = parity;
  fa.bb_rule = c->opt.bb_rule;
  fa.bb_cycle = c->opt.bb_cycle;
  fa.bbpart = nullptr;
  fa.sig_base = nullptr;
  fa.sig_keep = nullptr;
  return fa;
}

static xfft_status ensure_work(xfft_ctx* c, int n_rhs, int prec) {
  const long long stride = stride_of(c);
  if (c->cap_rhs >= n_rhs && c->cap_stride == stride && c->cap_prec == prec) return XFFT_OK;
  free_work(c);
  const size_t tot = (size_t)n_rhs * stride;
  if (prec == XFFT_FP64) {
    for (int k = 0; k < 6; ++k) CU(dalloc(c, &c->v64[k], tot));
  } else {
    CU(dalloc(c, &c->v64[0], tot));  // u (FP64 iterate)
    CU(dalloc(c, &c->v64[4], tot));  // FP64 residual
    for (int k = 0; k < 6; ++k) CU(dalloc(c, &c->v32[k], tot));
  }
  c->spec_bytes = (size_t)n_rhs * fft_spectrum_elems(c->fft) * (prec == XFFT_FP64 ? 16 : 8);
  CU(dalloc_bytes(c, &c->spec, c->spec_bytes));
  CU(dalloc(c, &c->st, 64));
  CU(dalloc(c, &c->act, 64));
  CU(dalloc(c, &c->outer_mask, 64));
  CU(dalloc(c, &c->eps_d, 6 * 64));
  CU(dalloc(c, &c->sig_keep, 6 * 64));
  const int na = apply_uncut_blocks(c->g) + apply_cut_blocks_max(c->ncut);
  const int np =
      std::max(precondition_blocks(c->fft, c->nX, true), precondition_blocks(c->fft, c->nX, false));
  const int ng = grad_blocks_uncut(c->g) + grad_blocks_cut(c->ncut);
  const int nparts = std::max(na, np);
  c->partials_count = std::max((size_t)n_rhs * 7 * nparts, (size_t)kGradValues * ng);
  CU(dalloc(c, &c->partials, c->partials_count));
  CU(dalloc(c, &c->red_out, 64));
  if (bb_euclid(c)) CU(dalloc(c, &c->bbpart, (size_t)n_rhs * 2 * kBBParts));
  c->cap_rhs = n_rhs;
  c->cap_stride = stride;
  c->cap_prec = prec;
  return XFFT_OK;
}

// the cut-tet kernel's grid of a launch (its partial slots are reserved for the largest tuned
// grid): the tuned grid for the FP32 kernel, the default for the FP64 and double-word kernels
static int cut_blocks_of(const xfft_ctx* c, bool fp32 = true) {
  return fp32 && c->cut_blocks > 0 ? c->cut_blocks : apply_cut_blocks(c->ncut);
}

static int nparts_of(const xfft_ctx* c) {
  return std::max(apply_uncut_blocks(c->g) + apply_cut_blocks_max(c->ncut),
                  std::max(precondition_blocks(c->fft, c->nX, true), precondition_blocks(c->fft, c->nX, false)));
}

static ApplyArgs apply_args(const xfft_ctx* c, const double* eps, const int* active) {
  ApplyArgs a;
  a.g = c->g;
  a.ph = c->ph;
  a.code = c->code;
  a.scale = c->has_scale ? c->scale : nullptr;
  a.eps = eps;
  a.active = active;
  a.stride = stride_of(c);
  a.nX = c->nX;
  a.partials = c->partials;
  a.nparts = nparts_of(c);
  a.part_offset_cut = apply_uncut_blocks(c->g);
  a.units_uncut = nullptr;
  a.units_cut = nullptr;
  a.want_sig = 1;
  a.kcache = c->kcache;
  a.fz = nullptr;
  a.fdnew = nullptr;
  a.fu = nullptr;
  a.st = nullptr;
  a.cut_blocks = c->cut_blocks;
  a.cut_rpl = c->cut_rpl;
  return a;
}

template <typename T>
static const T* isd_of(const xfft_ctx* c);
template <>
const double* isd_of<double>(const xfft_ctx* c) {
  return c->isD;
}
template <>
const float* isd_of<float>(const xfft_ctx* c) {
  return c->isF;
}

// inverse enriched blocks (block enriched preconditioner) or nullptr (identity)
template <typename T>
static const T* enr_block_of(const xfft_ctx* c);
template <>
const double* enr_block_of<double>(const xfft_ctx* c) {
  return c->opt.enr_precond == XFFT_ENR_BLOCK3 ? c->eb64 : nullptr;
}
template <>
const float* enr_block_of<float>(const xfft_ctx* c) {
  return c->opt.enr_precond == XFFT_ENR_BLOCK3 ? c->eb32 : nullptr;
}

// q = A d (+ b(eps)); finalisation `mode` (0 or 1) on the apply partials
// T: storage type of the vectors; A: arithmetic type of the kernels (T, or dw on FP64 data)
template <typename T, typename A = T>
static xfft_status do_apply(xfft_ctx* c, const T* d, T* q, const double* eps_dev, int n_rhs,
                            const int* active, int fin_mode, double tol, int crit, int maxit,
                            const T* fz = nullptr, T* fdnew = nullptr, T* fu = nullptr, int parity = 0,
                            int want_sig = -1, bool sig_add = false) {
  static_assert(std::is_same<typename Store<A>::type, T>::value, "arithmetic/storage mismatch");
  ApplyArgs a = apply_args(c, eps_dev, active);
  a.fz = fz;
  a.fdnew = fdnew;
  a.fu = fu;
  a.st = c->st;
  // the relative stopping rule of the inner FP32 solve needs no stress integrals
  a.want_sig = want_sig >= 0 ? want_sig : (fin_mode == 1 && crit == 1) ? 0 : 1;
  const bool dbl = sizeof(T) == 8;
  const bool dwa = std::is_same<A, dw>::value;
  const int ku = dwa ? XFFT_PROF_APPLY_UNCUT_DW : dbl ? XFFT_PROF_APPLY_UNCUT_F64 : XFFT_PROF_APPLY_UNCUT_F32;
  const int kc = dwa ? XFFT_PROF_APPLY_CUT_DW : dbl ? XFFT_PROF_APPLY_CUT_F64 : XFFT_PROF_APPLY_CUT_F32;
  a.units_uncut = punit(c, ku);
  a.units_cut = punit(c, kc);
  if (dbl || dwa) a.cut_blocks = a.cut_rpl = 0;  // the tuned shape is that of the FP32 kernel
  {
    ProfScope ps(c, ku, 1);
    CU(launch_apply_uncut<A>(d, q, a, n_rhs, c->stream));
  }
  {
    ProfScope ps(c, kc, 1);
    CU(launch_apply_cut<A>(fz ? fdnew : d, q, isd_of<T>(c), cutdata(c), a, n_rhs, c->stream));
  }
  if (fin_mode >= 0) {
    FinArgs fa = fin_args(c, fin_mode, crit, tol, maxit, a.nparts,
                          apply_uncut_blocks(c->g) + cut_blocks_of(c, !(dbl || dwa)), parity);
    if (fin_mode == 0) {  // a residual phase: record its stress integrals (base of a later update)
      fa.sig_keep = c->sig_keep;
      fa.sig_base = sig_add ? c->sig_keep : nullptr;
    }
    if (fin_mode == 1 && bb_euclid(c) && c->bbpart) {
      ProfScope ps(c, XFFT_PROF_VECTOR, 1);
      CU(launch_bb_dots<T>(fz ? fdnew : d, q, active, stride_of(c), n_rhs, c->bbpart, c->stream));
      fa.bbpart = c->bbpart;
    }
    ProfScope ps(c, XFFT_PROF_FINALIZE, 1);
    CU(launch_finalize(c->st, c->partials, fa, n_rhs, c->act, c->stream));
  }
  return XFFT_OK;
}

template <typename T>
static xfft_status do_prec(xfft_ctx* c, T* f, T* z, int n_rhs, const int* active, int fin_mode,
                           double tol, int crit, int maxit, int set_rel = 0, const T* qfuse = nullptr,
                           int parity = 0) {
  const int nparts = nparts_of(c);
  {
    const int kp = sizeof(T) == 8 ? XFFT_PROF_PREC_F64 : XFFT_PROF_PREC_F32;
    ProfScope ps(c, kp, 6);
    CU(launch_precondition<T>(c->fft, f, z, c->spec, stride_of(c), c->nX, active, c->partials, nparts,
                              n_rhs, c->stream, punit(c, kp), qfuse, qfuse ? c->st : nullptr,
                              enr_block_of<T>(c), sizeof(T) == 4 ? c->prec_group : 0));
  }
  if (fin_mode >= 0) {
    ProfScope ps(c, XFFT_PROF_FINALIZE, 1);
    FinArgs fa = fin_args(c, fin_mode, crit, tol, maxit, nparts,
                          precondition_blocks(c->fft, c->nX, sizeof(T) == 8), parity);
    fa.set_rel = set_rel;
    fa.inner_floor = c->opt.inner_tol;
    CU(launch_finalize(c->st, c->partials, fa, n_rhs, c->act, c->stream));
  }
  return XFFT_OK;
}

// ---------------------------------------------------------------- launch-shape tuner
// The FP32 cut-tet kernel's grid (its blocks loop over the cut list) and the right-hand sides
// per launch (all six in one launch, or three per launch) are picked by timing each candidate
// on the context's own microstructure: a warm-up and three timed launches of the FP32 apply of
// the inner CG iterations, CUDA events on the context's stream.  The choice is cached per grid
// and cut-tet / enriched-node counts for the process, so a repeated microstructure is not
// timed again.  The partial-sum rows keep room for the largest candidate grid
// (apply_cut_blocks_max), so the finalisation reads the slots the chosen grid writes.
struct TuneEntry {
  int n0, n1, n2, ncut, nX, blocks, rpl, group;
};
static std::mutex g_tune_mu;
static std::vector<TuneEntry> g_tune_cache;

static xfft_status autotune(xfft_ctx* c) {
  if (c->tuned || !c->opt.autotune || c->opt.precision != XFFT_FP32_REFINED || c->opt.cut_cache ||
      c->ncut < 4 * kThreads || c->prof || c->cap_rhs < 6)
    return XFFT_OK;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (const auto& t : g_tune_cache)
      if (t.n0 == c->g.n0 && t.n1 == c->g.n1 && t.n2 == c->g.n2 && t.ncut == c->ncut && t.nX == c->nX) {
        c->cut_blocks = t.blocks;
        c->cut_rpl = t.rpl;
        c->prec_group = t.group;
        c->tuned = true;
        return XFFT_OK;
      }
  }
  const int n_rhs = 6;
  float* d = c->v32[2];
  float* q = c->v32[4];
  CU(cudaMemsetAsync(d, 0, (size_t)n_rhs * stride_of(c) * sizeof(float), c->stream));
  const int bmax = apply_cut_blocks_max(c->ncut);
  std::vector<int> blocks;
  for (int w : {152, 304, 608, 912, 1216, 1824, 2432})
    if (w <= bmax) blocks.push_back(w);
  if (std::find(blocks.begin(), blocks.end(), bmax) == blocks.end()) blocks.push_back(bmax);
  struct Ev {
    cudaEvent_t e = nullptr;
    ~Ev() {
      if (e) cudaEventDestroy(e);
    }
  } t0, t1;
  CU(cudaEventCreate(&t0.e));
  CU(cudaEventCreate(&t1.e));
  double best = 1e30;
  int bb = 0, br = 0;
  for (int rpl : {6, 3}) {
    for (int nb : blocks) {
      c->cut_blocks = nb;
      c->cut_rpl = rpl;
      ApplyArgs a = apply_args(c, nullptr, nullptr);
      a.want_sig = 0;
      CU(launch_apply_cut<float>(d, q, c->isF, cutdata(c), a, n_rhs, c->stream));
      CU(cudaEventRecord(t0.e, c->stream));
      for (int k = 0; k < 3; ++k) CU(launch_apply_cut<float>(d, q, c->isF, cutdata(c), a, n_rhs, c->stream));
      CU(cudaEventRecord(t1.e, c->stream));
      CU(cudaEventSynchronize(t1.e));
      float ms = 0.f;
      CU(cudaEventElapsedTime(&ms, t0.e, t1.e));
      if (ms < best) {
        best = ms;
        bb = nb;
        br = rpl;
      }
    }
  }
  c->cut_blocks = bb;
  c->cut_rpl = br;
  // the preconditioner: 6, 3, 2 or 1 right-hand sides per group of FFT passes
  {
    float* f = c->v32[1];
    float* z = c->v32[3];
    CU(cudaMemsetAsync(f, 0, (size_t)n_rhs * stride_of(c) * sizeof(float), c->stream));
    double bestp = 1e30;
    int bg = 0;
    for (int G : {6, 3, 2, 1}) {
      auto run = [&]() {
        return launch_precondition<float>(c->fft, f, z, c->spec, stride_of(c), c->nX, nullptr, c->partials,
                                          nparts_of(c), n_rhs, c->stream, nullptr, nullptr, nullptr,
                                          enr_block_of<float>(c), G == 6 ? 0 : G);
      };
      CU(run());
      CU(cudaEventRecord(t0.e, c->stream));
      for (int k = 0; k < 3; ++k) CU(run());
      CU(cudaEventRecord(t1.e, c->stream));
      CU(cudaEventSynchronize(t1.e));
      float ms = 0.f;
      CU(cudaEventElapsedTime(&ms, t0.e, t1.e));
      if (ms < bestp) {
        bestp = ms;
        bg = G == 6 ? 0 : G;
      }
    }
    c->prec_group = bg;
  }
  c->tuned = true;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache.push_back({c->g.n0, c->g.n1, c->g.n2, c->ncut, c->nX, bb, br, c->prec_group});
  return XFFT_OK;
}

static xfft_status poll_active(xfft_ctx* c, int n_rhs, int* nactive) {
  CU(cudaMemcpyAsync(c->h_act, c->act, n_rhs * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  if (c->prof && c->pend.size() > 2048) CU(prof_flush(c));
  int k = 0;
  for (int r = 0; r < n_rhs; ++r) k += c->h_act[r] != 0;
  *nactive = k;
  return XFFT_OK;
}

static xfft_status read_states(xfft_ctx* c, int n_rhs) {
  CU(cudaMemcpyAsync(c->h_st, c->st, n_rhs * sizeof(RhsState), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  return XFFT_OK;
}

#define TRY(...)                      \
  do {                                \
    xfft_status s_ = (__VA_ARGS__);   \
    if (s_ != XFFT_OK) return s_;     \
  } while (0)

// CG iterations of type T.  On entry f is the negative residual, z = P^-1 f with the state
// finalised in mode 3, the state's alpha = beta = 0 and dA = 0.  Each iteration:
//   d_new = z + beta d_old, u += alpha d_old (fused into the stencil and a tail kernel),
//   q = A d_new, alpha = rr / <q, d_new>,
//   f -= alpha q, z = P^-1 f (fused into the first FFT pass), beta = rr'/rr.
// The last u += alpha d of each right-hand side is applied after the loop.
// One CG iteration (Algorithm 1) for all right-hand sides: d_new = z + beta d_old and
// u += alpha d_old (fused into the stencil), q = A d_new with <d, q>, alpha; f -= alpha q fused
// into the preconditioner's first pass, z = P^-1 f with f^T z, beta and the stopping rule.
template <typename T>
static xfft_status cg_iter(xfft_ctx* c, int it, T* u, T* f, T* const* dbuf, T* z, T* q, int n_rhs,
                           double tol, int crit, int maxit) {
  const long long stride = stride_of(c);
  T* dold = dbuf[it & 1];
  T* dnew = dbuf[(it + 1) & 1];
  const int par = (it + 1) & 1;
  {
    ProfScope ps(c, XFFT_PROF_VECTOR, 1);
    CU(launch_cg_update_tail<T>(z, dold, dnew, u, c->st, 3 * c->g.N, stride, n_rhs, c->stream));
  }
  TRY(do_apply<T>(c, dold, q, nullptr, n_rhs, c->act, 1, tol, crit, maxit, z, dnew, u, par));
  TRY(do_prec<T>(c, f, z, n_rhs, c->act, 2, tol, crit, maxit, 0, q, par));
  return XFFT_OK;
}

// One inner CG solve of a context (the FP64 solver's whole solve, or one FP32 inner solve of the
// refinement) as a loop argument set.
struct LoopArgs {
  xfft_ctx* c = nullptr;
  bool dbl = false;
  void *u = nullptr, *f = nullptr, *dA = nullptr, *dB = nullptr, *z = nullptr, *q = nullptr;
  int n_rhs = 0;
  double tol = 0.0;
  int crit = 0, maxit = 0;
};

// iterations per round of a device-driven loop: poll_every rounded up to an even count, so that
// the two direction buffers are in the same roles at the start of every round
static int loop_pe(const xfft_ctx* c) { return c->opt.poll_every + (c->opt.poll_every & 1); }

template <typename T>
static xfft_status loop_round(const LoopArgs& L, int pe) {
  T* dbuf[2] = {(T*)L.dA, (T*)L.dB};
  for (int j = 0; j < pe; ++j)
    TRY(cg_iter<T>(L.c, j, (T*)L.u, (T*)L.f, dbuf, (T*)L.z, (T*)L.q, L.n_rhs, L.tol, L.crit, L.maxit));
  return XFFT_OK;
}

static xfft_status loop_finish(const LoopArgs& L) {
  ProfScope ps(L.c, XFFT_PROF_VECTOR, 1);
  const long long stride = stride_of(L.c);
  if (L.dbl)
    CU(launch_cg_finish<double>((double*)L.u, (double*)L.dA, (double*)L.dB, L.c->st, stride, L.n_rhs,
                                L.c->stream));
  else
    CU(launch_cg_finish<float>((float*)L.u, (float*)L.dA, (float*)L.dB, L.c->st, stride, L.n_rhs,
                               L.c->stream));
  return XFFT_OK;
}

static bool graph_stream(const xfft_ctx* c) {
  return !c->prof && c->stream != nullptr && c->stream != cudaStreamLegacy && c->stream != cudaStreamPerThread;
}

// The device-driven loops of the inner solves `items` (one or several contexts) as one graph:
// for each item an independent conditional while loop whose body is loop_pe(c) iterations on its
// context's stream.  lm: device LoopState per item (kLoopStride bytes apart).  Returns
// XFFT_EUNSUPPORTED when the graph cannot be built (the caller then polls on the host).
static xfft_status build_device_loop(const std::vector<LoopArgs>& items, unsigned char* lm,
                                     long long limit_ns, cudaGraphExec_t* exec) {
  const int n = (int)items.size();
  xfft_status body_status = XFFT_OK;
  std::vector<LoopSpec> loops;
  loops.reserve(n);
  for (int i = 0; i < n; ++i) {
    const LoopArgs L = items[i];
    LoopSpec sp;
    sp.stream = L.c->stream;
    sp.body = [L, &body_status](cudaStream_t) -> cudaError_t {
      const xfft_status s = L.dbl ? loop_round<double>(L, loop_pe(L.c)) : loop_round<float>(L, loop_pe(L.c));
      if (s != XFFT_OK) {
        body_status = s;
        return cudaErrorUnknown;
      }
      return cudaSuccess;
    };
    sp.act = L.c->act;
    sp.nr = L.n_rhs;
    sp.st = reinterpret_cast<LoopState*>(lm + kLoopStride * i);
    sp.max_rounds = (unsigned)(L.maxit / loop_pe(L.c) + 2);
    sp.limit_ns = limit_ns;
    loops.push_back(std::move(sp));
  }
  const cudaError_t e = build_loop_graph(loops, exec);
  if (body_status != XFFT_OK) return body_status;
  if (e != cudaSuccess) {
    cudaGetLastError();  // clear a sticky launch-configuration error of the failed build
    return fail(XFFT_EUNSUPPORTED, std::string("device-driven loop: ") + cudaGetErrorString(e));
  }
  return XFFT_OK;
}

// whether any of the n loop states in lm_host (copied back from the device) timed out
static bool loops_timed_out(const unsigned char* lm_host, int n) {
  for (int i = 0; i < n; ++i)
    if (reinterpret_cast<const LoopState*>(lm_host + kLoopStride * i)->timed_out) return true;
  return false;
}

// Launch a built device loop graph on master: master after every item's earlier work, every
// item after the graph.
static xfft_status run_device_loop(const std::vector<LoopArgs>& items, cudaStream_t master,
                                   cudaGraphExec_t exec, cudaEvent_t fork, const std::vector<cudaEvent_t>& joins,
                                   const std::vector<char>* finish = nullptr) {
  for (size_t i = 0; i < items.size(); ++i) {
    xfft_ctx* c = items[i].c;
    if (c->stream == master) continue;
    CU(cudaEventRecord(joins[i], c->stream));
    CU(cudaStreamWaitEvent(master, joins[i], 0));
  }
  CU(cudaGraphLaunch(exec, master));
  CU(cudaEventRecord(fork, master));
  for (const auto& L : items)
    if (L.c->stream != master) CU(cudaStreamWaitEvent(L.c->stream, fork, 0));
  for (size_t i = 0; i < items.size(); ++i)
    if (!finish || (*finish)[i]) TRY(loop_finish(items[i]));
  return XFFT_OK;
}

// One context's inner solve: the device-driven loop (cached per argument set) when the stream
// allows graphs, else convergence polls on the host every poll_every iterations.  *timed_out is
// set when the loop's device-time limit (option spin_limit_ns) ended it.
static xfft_status cg_loop(const LoopArgs& L, bool* timed_out) {
  xfft_ctx* c = L.c;
  *timed_out = false;
  if (graph_stream(c) && c->devloop_ok) {
    const void* key[6] = {L.u, L.f, L.dA, L.dB, L.z, L.q};
    xfft_ctx::CgGraph* hit = nullptr;
    for (auto& g : c->cg_graphs)
      if (g.valid && g.dbl == L.dbl && g.n_rhs == L.n_rhs && g.crit == L.crit && g.maxit == L.maxit &&
          g.pe == loop_pe(c) && g.tol == L.tol && g.limit == c->opt.spin_limit_ns &&
          std::equal(key, key + 6, g.p))
        hit = &g;
    if (!hit) {
      cudaGraphExec_t exec = nullptr;
      const std::vector<LoopArgs> items{L};
      const xfft_status s = build_device_loop(items, c->loopmem, c->opt.spin_limit_ns, &exec);
      if (s == XFFT_EUNSUPPORTED) {
        c->devloop_ok = false;
      } else {
        TRY(s);
        hit = &c->cg_graphs[c->cg_next];
        c->cg_next = (c->cg_next + 1) % 4;
        if (hit->exec) cudaGraphExecDestroy(hit->exec);
        *hit = xfft_ctx::CgGraph();
        hit->valid = true;
        hit->dbl = L.dbl;
        hit->n_rhs = L.n_rhs;
        hit->crit = L.crit;
        hit->maxit = L.maxit;
        hit->pe = loop_pe(c);
        hit->tol = L.tol;
        hit->limit = c->opt.spin_limit_ns;
        std::copy(key, key + 6, hit->p);
        hit->exec = exec;
      }
    }
    if (hit) {
      TRY(run_device_loop({L}, c->stream, hit->exec, c->ev_fork, c->ev_join));
      CU(cudaMemcpyAsync(c->h_loop, c->loopmem, sizeof(LoopState), cudaMemcpyDeviceToHost, c->stream));
      CU(cudaStreamSynchronize(c->stream));
      *timed_out = loops_timed_out(c->h_loop, 1);
      return XFFT_OK;
    }
  }
  // host-polled loop (tracing on, legacy streams, or no conditional graphs)
  const int pe = c->opt.poll_every;
  for (int it = 0; it <= L.maxit; ++it) {
    if (it % pe == 0) {
      int na = 0;
      TRY(poll_active(c, L.n_rhs, &na));
      if (na == 0) break;
    }
    if (L.dbl) {
      double* dbuf[2] = {(double*)L.dA, (double*)L.dB};
      TRY(cg_iter<double>(c, it, (double*)L.u, (double*)L.f, dbuf, (double*)L.z, (double*)L.q, L.n_rhs,
                          L.tol, L.crit, L.maxit));
    } else {
      float* dbuf[2] = {(float*)L.dA, (float*)L.dB};
      TRY(cg_iter<float>(c, it, (float*)L.u, (float*)L.f, dbuf, (float*)L.z, (float*)L.q, L.n_rhs, L.tol,
                         L.crit, L.maxit));
    }
  }
  return loop_finish(L);
}

__global__ void k_copy_act_to_mask(const int* act, int* mask, int n) {
  const int r = threadIdx.x;
  if (r < n) mask[r] = act[r];
}

struct SolveResult {
  int iters[64];
  double res[64];
  double sig[64][6];
  int status[64];
  int refine_steps;
};

// The phases of a solve for n_rhs strains (device eps_d filled), shared by the single-context
// solve and the lockstep batch: the FP64 solver is one residual phase and one inner solve; the
// FP32-refined solver repeats (residual of the FP64 iterate, check, inner FP32 solve of the
// correction).  The FP64 solution (scaled enriched DOFs) ends in c->v64[0].
struct SolveRun {
  xfft_ctx* c = nullptr;
  int n_rhs = 0;
  SolveResult* R = nullptr;
  int ref = 0;
  bool done = false;
  int pending[64];
  int hmask[64];
};

static xfft_status run_begin(SolveRun& s, xfft_ctx* c, int n_rhs, SolveResult* R) {
  s.c = c;
  s.n_rhs = n_rhs;
  s.R = R;
  s.ref = 0;
  s.done = false;
  for (int r = 0; r < 64; ++r) {
    s.pending[r] = r < n_rhs ? 1 : 0;
    s.hmask[r] = 0;
  }
  for (int r = 0; r < n_rhs; ++r) {
    R->iters[r] = 0;
    R->res[r] = 0.0;
    R->status[r] = 0;
    for (int k = 0; k < 6; ++k) R->sig[r][k] = 0.0;
  }
  R->refine_steps = 0;
  CU(cudaMemsetAsync(c->v64[0], 0, (size_t)n_rhs * stride_of(c) * sizeof(double), c->stream));
  return XFFT_OK;
}

// A residual update instead of a recomputation (option residual_update): after the first
// recomputed residual of the FP64 iterate, when every right-hand side still iterating has a
// residual (stopping-rule measure of the last residual phase) below 100 tol.  The update adds
// the FP32 operator applied to the last correction delta; its rounding, about 1e-7 of |A delta|
// times the stencil's cancellation, is then well below 1e-2 tol.
static bool residual_update_ok(const SolveRun& s) {
  const xfft_ctx* c = s.c;
  if (!c->opt.residual_update || s.ref < 2) return false;
  for (int r = 0; r < s.n_rhs; ++r)
    if (s.pending[r] && !(s.R->res[r] <= 100.0 * c->opt.tol)) return false;
  return true;
}

// enqueue the residual phase: the residual f of the current iterate, z = P^-1 f and the stopping
// rule (finalisation mode 3)
static xfft_status run_residual(SolveRun& s) {
  xfft_ctx* c = s.c;
  cudaStream_t st = c->stream;
  const long long stride = stride_of(c);
  const size_t tot = (size_t)s.n_rhs * stride;
  const double tol = c->opt.tol;
  if (c->opt.precision == XFFT_FP64) {
    double *u = c->v64[0], *f = c->v64[1], *d = c->v64[2], *z = c->v64[3], *q = c->v64[4];
    {
      ProfScope ps(c, XFFT_PROF_VECTOR, 1);
      CU(launch_init_state(c->st, c->act, s.n_rhs, nullptr, st));
    }
    TRY(do_apply<double>(c, u, q, c->eps_d, s.n_rhs, c->act, 0, tol, 0, c->opt.maxit));
    {
      ProfScope ps(c, XFFT_PROF_VECTOR, 1);
      CU(launch_scale_copy<double, double>(q, f, -1.0, stride, s.n_rhs, c->act, st));
    }
    TRY(do_prec<double>(c, f, z, s.n_rhs, c->act, 3, tol, 0, c->opt.maxit));
    CU(cudaMemsetAsync(d, 0, tot * sizeof(double), st));
    return XFFT_OK;
  }
  double* u = c->v64[0];
  double* r64 = c->v64[4];
  float *f = c->v32[1], *d = c->v32[2], *z = c->v32[3], *q = c->v32[4];
  for (int r = 0; r < 64; ++r) s.hmask[r] = r < s.n_rhs ? s.pending[r] : 0;
  CU(cudaMemcpyAsync(c->outer_mask, s.hmask, 64 * sizeof(int), cudaMemcpyHostToDevice, st));
  {
    ProfScope ps(c, XFFT_PROF_VECTOR, 1);
    CU(launch_init_state(c->st, c->act, s.n_rhs, c->outer_mask, st));
  }
  if (s.ref == 0) {
    // u = 0: the residual is -b; FP32 suffices for the first inner solve because every later
    // check recomputes the residual of the accumulated iterate in FP64
    CU(cudaMemsetAsync(d, 0, tot * sizeof(float), st));
    TRY(do_apply<float>(c, d, q, c->eps_d, s.n_rhs, c->act, 0, tol, 0, c->opt.maxit));
    ProfScope ps(c, XFFT_PROF_VECTOR, 1);
    CU(launch_scale_copy<float, float>(q, f, -1.0, stride, s.n_rhs, c->act, st));
  } else if (residual_update_ok(s)) {
    // residual update (option residual_update): r64 = A u + b of the previous residual phase
    // plus A delta of the last inner solve's correction (still in v32[0]), applied in FP32 with
    // its stress integrals added to the previous ones
    TRY(do_apply<float>(c, c->v32[0], q, nullptr, s.n_rhs, c->act, 0, tol, 0, c->opt.maxit, nullptr, nullptr,
                        nullptr, 0, 1, true));
    ProfScope ps(c, XFFT_PROF_VECTOR, 1);
    CU(launch_add_to_double<float>(r64, q, stride, s.n_rhs, c->act, st));
    CU(launch_scale_copy<double, float>(r64, f, -1.0, stride, s.n_rhs, c->act, st));
  } else {
    // residual of the accumulated FP64 iterate in double-word arithmetic (about 48 bits, far
    // below the FP32 rounding it corrects) and the stopping rule
    TRY((do_apply<double, dw>(c, u, r64, c->eps_d, s.n_rhs, c->act, 0, tol, 0, c->opt.maxit)));
    ProfScope ps(c, XFFT_PROF_VECTOR, 1);
    CU(launch_scale_copy<double, float>(r64, f, -1.0, stride, s.n_rhs, c->act, st));
  }
  TRY(do_prec<float>(c, f, z, s.n_rhs, c->act, 3, tol, 0, c->opt.maxit, 1));
  return XFFT_OK;
}

static void fill_result(SolveRun& s, int r, const RhsState& st) {
  double sn = 0.0;
  for (int k = 0; k < 6; ++k) {
    s.R->sig[r][k] = st.sig[k];
    sn += st.sig[k] * st.sig[k];
  }
  const double vol = s.c->g.volY;
  s.R->res[r] = sn > 0 ? sqrt(std::max(st.rr, 0.0) / vol) / (sqrt(sn) / vol) : 0.0;
}

// read the residual phase's states: done, or an inner solve is needed
static xfft_status run_check(SolveRun& s, bool* need_inner) {
  xfft_ctx* c = s.c;
  TRY(read_states(c, s.n_rhs));
  *need_inner = false;
  if (c->opt.precision == XFFT_FP64) {
    for (int r = 0; r < s.n_rhs; ++r) *need_inner |= c->h_st[r].active != 0;
    if (!*need_inner) {  // converged (or broke down) at the start
      for (int r = 0; r < s.n_rhs; ++r) {
        fill_result(s, r, c->h_st[r]);
        s.R->status[r] = c->h_st[r].converged ? 0 : (c->h_st[r].status ? c->h_st[r].status : 4);
      }
      s.done = true;
    }
    return XFFT_OK;
  }
  int still = 0;
  for (int r = 0; r < s.n_rhs; ++r) {
    if (!s.pending[r]) continue;
    const RhsState& st = c->h_st[r];
    fill_result(s, r, st);
    if (st.converged) {
      s.pending[r] = 0;
      s.R->status[r] = 0;
    } else if (st.status == 5) {
      s.pending[r] = 0;
      s.R->status[r] = 5;
    } else {
      ++still;
    }
  }
  if (still == 0) {
    s.done = true;
  } else if (s.ref == c->opt.max_refine) {
    for (int r = 0; r < s.n_rhs; ++r)
      if (s.pending[r]) s.R->status[r] = 4;
    s.done = true;
  } else {
    if (s.ref > 0) s.R->refine_steps++;
    *need_inner = true;
  }
  return XFFT_OK;
}

// the loop arguments of a run's inner solves (the same in every refinement round)
static LoopArgs run_loop_args(const SolveRun& s) {
  xfft_ctx* c = s.c;
  LoopArgs L;
  L.c = c;
  L.n_rhs = s.n_rhs;
  L.maxit = c->opt.maxit;
  if (c->opt.precision == XFFT_FP64) {
    L.dbl = true;
    L.u = c->v64[0];
    L.f = c->v64[1];
    L.dA = c->v64[2];
    L.dB = c->v64[5];
    L.z = c->v64[3];
    L.q = c->v64[4];
    L.tol = c->opt.tol;
    L.crit = 0;
  } else {
    L.dbl = false;
    L.u = c->v32[0];
    L.f = c->v32[1];
    L.dA = c->v32[2];
    L.dB = c->v32[5];
    L.z = c->v32[3];
    L.q = c->v32[4];
    L.tol = 0.5;
    L.crit = 1;
  }
  return L;
}

// enqueue what precedes the inner solve and return its loop arguments
static xfft_status run_inner_pre(SolveRun& s, LoopArgs* L) {
  xfft_ctx* c = s.c;
  *L = run_loop_args(s);
  if (c->opt.precision == XFFT_FP64) return XFFT_OK;
  const size_t tot = (size_t)s.n_rhs * stride_of(c);
  // inner FP32 PCG on A delta = r (relative reduction inner_tol); the act flags of the refining
  // RHS were set by the mode-3 finalisation
  {
    ProfScope ps(c, XFFT_PROF_VECTOR, 2);
    k_copy_act_to_mask<<<1, 64, 0, c->stream>>>(c->act, c->outer_mask, s.n_rhs);
    CU(cudaGetLastError());
    CU(cudaMemsetAsync(c->v32[0], 0, tot * sizeof(float), c->stream));
    CU(cudaMemsetAsync(c->v32[2], 0, tot * sizeof(float), c->stream));
  }
  return XFFT_OK;
}

// after the inner solve (its last u += alpha d applied): results or the next refinement round
static xfft_status run_inner_post(SolveRun& s, bool timed_out) {
  xfft_ctx* c = s.c;
  TRY(read_states(c, s.n_rhs));
  if (c->opt.precision == XFFT_FP64) {
    for (int r = 0; r < s.n_rhs; ++r) {
      const RhsState& st = c->h_st[r];
      s.R->iters[r] = st.iters;
      fill_result(s, r, st);
      s.R->status[r] = st.converged ? 0 : (st.status ? st.status : (timed_out && st.active ? 6 : 4));
    }
    s.done = true;
    return XFFT_OK;
  }
  for (int r = 0; r < s.n_rhs; ++r) {
    if (s.hmask[r]) s.R->iters[r] += c->h_st[r].iters;
    if (s.hmask[r] && c->h_st[r].status == 5) {  // breakdown inside the inner solve
      s.pending[r] = 0;
      s.R->status[r] = 5;
    }
  }
  {
    ProfScope ps(c, XFFT_PROF_VECTOR, 1);
    CU(launch_add_to_double<float>(c->v64[0], c->v32[0], stride_of(c), s.n_rhs, c->outer_mask, c->stream));
  }
  if (timed_out) {
    for (int r = 0; r < s.n_rhs; ++r)
      if (s.pending[r] && c->h_st[r].active) {
        s.pending[r] = 0;
        s.R->status[r] = 6;
      }
  }
  s.ref += 1;
  for (int r = 0; r < s.n_rhs; ++r)
    if (s.pending[r]) return XFFT_OK;
  s.done = true;
  return XFFT_OK;
}

// Solve for n_rhs strains (device eps_d already filled); the FP64 solution (scaled enriched
// DOFs) ends in c->v64[0].
static xfft_status solve_core(xfft_ctx* c, int n_rhs, SolveResult* R) {
  SolveRun s;
  TRY(run_begin(s, c, n_rhs, R));
  while (!s.done) {
    TRY(run_residual(s));
    bool need = false;
    TRY(run_check(s, &need));
    if (!need) break;
    LoopArgs L;
    TRY(run_inner_pre(s, &L));
    bool timed_out = false;
    TRY(cg_loop(L, &timed_out));
    TRY(run_inner_post(s, timed_out));
  }
  return XFFT_OK;
}

__global__ void k_unscale_enr(const double* __restrict__ u, const double* __restrict__ isD,
                              double* __restrict__ out, long long stride, long long N, int nX) {
  const int rhs = blockIdx.y;
  const long long n = 3LL * nX;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[rhs * n + i] = u[rhs * stride + 3 * N + i] * isD[i];
}

static xfft_status upload_eps(xfft_ctx* c, int n_rhs, const double* eps_host) {
  CU(cudaMemcpyAsync(c->eps_d, eps_host, 6 * n_rhs * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  return XFFT_OK;
}

static xfft_status finish_stats(xfft_ctx* c, const SolveResult& R, int n_rhs, float ms_solve,
                                xfft_stats* stats) {
  if (!stats) return XFFT_OK;
  memset(stats, 0, sizeof(*stats));
  stats->n_rhs = n_rhs;
  for (int r = 0; r < n_rhs; ++r) {
    stats->iters[r] = R.iters[r];
    stats->final_res[r] = R.res[r];
  }
  stats->refine_steps = R.refine_steps;
  stats->n_fe = (int)c->g.N;
  stats->n_x = c->nX;
  stats->n_cut_tets = c->ncut;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, c->ev0, c->ev1);
  stats->ms_setup = ms;
  stats->ms_solve = ms_solve;
  return XFFT_OK;
}

static xfft_status status_of(const SolveResult& R, int n_rhs) {
  xfft_status st = XFFT_OK;
  for (int r = 0; r < n_rhs; ++r) {
    if (R.status[r] == 5) return fail(XFFT_EBREAKDOWN, "CG breakdown");
    if (R.status[r] == 6) st = XFFT_ETIMEOUT;
    if (R.status[r] == 4 && st == XFFT_OK) st = XFFT_ENOTCONV;
  }
  if (st == XFFT_ENOTCONV) g_err = "maximum number of iterations reached";
  if (st == XFFT_ETIMEOUT) g_err = "the device-driven iteration loop reached its time limit (spin_limit_ns)";
  return st;
}

extern "C" xfft_status xfft_solve(xfft_ctx* c, int n_rhs, const double* eps_bar, double* u_std,
                                  double* u_enr, double* voxel_stress, double* mean_stress,
                                  xfft_stats* stats, int ptrs_on_device) {
  if (!c || !eps_bar) return fail(XFFT_EINVAL, "NULL argument");
  if (!c->have_micro) return fail(XFFT_ESTATE, "xfft_set_microstructure first");
  if (n_rhs < 1 || n_rhs > 64) return fail(XFFT_EINVAL, "n_rhs must be in [1, 64]");
  TRY(ensure_work(c, n_rhs, c->opt.precision));
  TRY(autotune(c));
  cudaStream_t s = c->stream;
  TRY(upload_eps(c, n_rhs, eps_bar));
  cudaEvent_t e0, e1;
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  CU(cudaEventRecord(e0, s));
  SolveResult R;
  xfft_status rs = solve_core(c, n_rhs, &R);
  if (rs != XFFT_OK) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rs;
  }
  CU(cudaEventRecord(e1, s));
  const GridDev& g = c->g;
  const long long stride = stride_of(c);
  const double* u = c->v64[0];
  const cudaMemcpyKind kind = ptrs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (u_std) {
    for (int r = 0; r < n_rhs; ++r)
      CU(cudaMemcpyAsync(u_std + (size_t)r * 3 * g.N, u + r * stride, 3 * g.N * sizeof(double), kind, s));
  }
  if (u_enr && c->nX > 0) {
    double* tmp = c->v64[4];  // free after the solve (residual / q buffer)
    long long nb = (3LL * c->nX + 255) / 256;
    if (nb > 4096) nb = 4096;
    {
      ProfScope ps(c, XFFT_PROF_POST, 1);
      k_unscale_enr<<<dim3((unsigned)nb, n_rhs), 256, 0, s>>>(u, c->isD, tmp, stride, g.N, c->nX);
      CU(cudaGetLastError());
    }
    CU(cudaMemcpyAsync(u_enr, tmp, (size_t)n_rhs * 3 * c->nX * sizeof(double), kind, s));
  }
  if (voxel_stress) {
    double* out = voxel_stress;
    double* tmp = nullptr;
    if (!ptrs_on_device) {
      CU(dalloc(c, &tmp, (size_t)n_rhs * 6 * g.N));
      out = tmp;
    }
    ApplyArgs a = apply_args(c, c->eps_d, nullptr);
    {
      ProfScope ps(c, XFFT_PROF_POST, 2);
      CU(launch_voxel_stress(u, c->isD, cutdata(c), a, out, n_rhs, s));
    }
    if (tmp) {
      CU(cudaMemcpyAsync(voxel_stress, tmp, (size_t)n_rhs * 6 * g.N * sizeof(double),
                         cudaMemcpyDeviceToHost, s));
      CU(cudaStreamSynchronize(s));
      dfree(c, tmp);
    }
  }
  CU(cudaStreamSynchronize(s));
  if (mean_stress)
    for (int r = 0; r < n_rhs; ++r)
      for (int k = 0; k < 6; ++k) mean_stress[6 * r + k] = R.sig[r][k] / g.volY;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  finish_stats(c, R, n_rhs, ms, stats);
  return status_of(R, n_rhs);
}

// C_eff, the six-case checkpoint and the stats of a finished six-case solve
static xfft_status finish_six(xfft_ctx* c, const SolveResult& R, double C_eff[36], xfft_stats* stats,
                              float msolve) {
  const long long stride = stride_of(c);
  if (!c->U6) CU(dalloc(c, &c->U6, 6 * (size_t)stride));
  CU(cudaMemcpyAsync(c->U6, c->v64[0], 6 * (size_t)stride * sizeof(double), cudaMemcpyDeviceToDevice,
                     c->stream));
  CU(cudaStreamSynchronize(c->stream));
  // C_eff[i][k] = <sigma_i>(E_k)
  for (int i = 0; i < 6; ++i)
    for (int k = 0; k < 6; ++k) C_eff[i * 6 + k] = R.sig[k][i] / c->g.volY;
  memcpy(c->C6, C_eff, sizeof(c->C6));
  finish_stats(c, R, 6, msolve, stats);
  xfft_status st = status_of(R, 6);
  if (st == XFFT_OK) c->have6 = true;
  return st;
}

extern "C" xfft_status xfft_effective_stiffness(xfft_ctx* c, double C_eff[36], xfft_stats* stats) {
  if (!c || !C_eff) return fail(XFFT_EINVAL, "NULL argument");
  if (!c->have_micro) return fail(XFFT_ESTATE, "xfft_set_microstructure first");
  double eps[36];
  for (int k = 0; k < 36; ++k) eps[k] = (k % 7 == 0) ? 1.0 : 0.0;
  c->have6 = false;
  TRY(ensure_work(c, 6, c->opt.precision));
  TRY(autotune(c));
  TRY(upload_eps(c, 6, eps));
  cudaEvent_t e0, e1;
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  CU(cudaEventRecord(e0, c->stream));
  SolveResult R;
  xfft_status rs = solve_core(c, 6, &R);
  CU(cudaEventRecord(e1, c->stream));
  if (rs != XFFT_OK) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rs;
  }
  CU(cudaEventSynchronize(e1));
  float msolve = 0.f;
  cudaEventElapsedTime(&msolve, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return finish_six(c, R, C_eff, stats, msolve);
}

// The threaded form of the batch (contexts on the legacy stream, or tracing on): each context's
// xfft_effective_stiffness from its own host thread.
static xfft_status batch_threaded(int n, xfft_ctx* const* ctxs, double* C_eff, xfft_stats* stats, int dev) {
  std::vector<xfft_status> st(n, XFFT_OK);
  std::vector<std::string> msg(n);
  std::vector<std::thread> th;
  th.reserve(n);
  for (int i = 0; i < n; ++i) {
    th.emplace_back([&, i]() {
      if (cudaSetDevice(dev) != cudaSuccess) {
        st[i] = XFFT_ECUDA;
        msg[i] = "cudaSetDevice in a batch thread";
        return;
      }
      st[i] = xfft_effective_stiffness(ctxs[i], C_eff + 36 * (size_t)i, stats ? stats + i : nullptr);
      if (st[i] != XFFT_OK) msg[i] = g_err;
    });
  }
  for (auto& t : th) t.join();
  for (int i = 0; i < n; ++i)
    if (st[i] != XFFT_OK && st[i] != XFFT_ENOTCONV)
      return fail(st[i], "context " + std::to_string(i) + ": " + msg[i]);
  for (int i = 0; i < n; ++i)
    if (st[i] != XFFT_OK) return fail(st[i], "context " + std::to_string(i) + ": " + msg[i]);
  return XFFT_OK;
}

// Resources of one lockstep batch call: a master stream, fork / join events, loop memory.
struct BatchRes {
  cudaStream_t master = nullptr;
  cudaEvent_t fork = nullptr, t0 = nullptr, t1 = nullptr;
  std::vector<cudaEvent_t> joins;
  unsigned char* lm = nullptr;
  unsigned char* lm_host = nullptr;
  ~BatchRes() {
    if (master) cudaStreamSynchronize(master);
    for (auto e : joins)
      if (e) cudaEventDestroy(e);
    if (fork) cudaEventDestroy(fork);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (lm) cudaFree(lm);
    if (lm_host) cudaFreeHost(lm_host);
    if (master) cudaStreamDestroy(master);
  }
};

extern "C" xfft_status xfft_batch_effective_stiffness(int n, xfft_ctx* const* ctxs, double* C_eff,
                                                      xfft_stats* stats) {
  if (n < 1 || !ctxs || !C_eff) return fail(XFFT_EINVAL, "n >= 1 contexts and C_eff required");
  if (n > kMaxBatch) return fail(XFFT_EINVAL, "at most 64 contexts per batch");
  bool lockstep = true;
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i]) return fail(XFFT_EINVAL, "NULL context");
    if (!ctxs[i]->have_micro) return fail(XFFT_ESTATE, "xfft_set_microstructure first");
    for (int k = 0; k < i; ++k)
      if (ctxs[k] == ctxs[i]) return fail(XFFT_EINVAL, "a context appears twice in the batch");
    lockstep = lockstep && graph_stream(ctxs[i]) && ctxs[i]->devloop_ok;
  }
  int dev = 0;
  CU(cudaGetDevice(&dev));
  if (!lockstep) return batch_threaded(n, ctxs, C_eff, stats, dev);
  // Lockstep: the residual phases of all contexts on their own streams, then ONE device-driven
  // loop graph over every context still iterating, until every context is done.
  BatchRes B;
  CU(cudaStreamCreateWithFlags(&B.master, cudaStreamNonBlocking));
  CU(cudaEventCreateWithFlags(&B.fork, cudaEventDisableTiming));
  CU(cudaEventCreate(&B.t0));
  CU(cudaEventCreate(&B.t1));
  B.joins.assign(n, nullptr);
  for (int i = 0; i < n; ++i) CU(cudaEventCreateWithFlags(&B.joins[i], cudaEventDisableTiming));
  CU(cudaMalloc((void**)&B.lm, kLoopBytes));
  CU(cudaMallocHost((void**)&B.lm_host, kLoopBytes));
  double eps[36];
  for (int k = 0; k < 36; ++k) eps[k] = (k % 7 == 0) ? 1.0 : 0.0;
  std::vector<SolveRun> runs(n);
  std::vector<SolveResult> Rs(n);
  long long limit = -1;
  for (int i = 0; i < n; ++i) {
    xfft_ctx* c = ctxs[i];
    c->have6 = false;
    TRY(ensure_work(c, 6, c->opt.precision));
    TRY(autotune(c));
    TRY(upload_eps(c, 6, eps));
    if (c->opt.spin_limit_ns >= 0 && (limit < 0 || c->opt.spin_limit_ns < limit)) limit = c->opt.spin_limit_ns;
  }
  CU(cudaEventRecord(B.t0, B.master));
  for (int i = 0; i < n; ++i) {
    CU(cudaStreamWaitEvent(ctxs[i]->stream, B.t0, 0));
    TRY(run_begin(runs[i], ctxs[i], 6, &Rs[i]));
  }
  // one graph of n independent device loops, built at the first inner solve and launched in
  // every round; a context without an inner solve in a round has its activity flags cleared, so
  // its loop ends after one round of early-exiting kernels and its state stays as it was
  std::vector<LoopArgs> all(n);
  for (int i = 0; i < n; ++i) all[i] = run_loop_args(runs[i]);
  struct ExecGuard {
    cudaGraphExec_t e = nullptr;
    ~ExecGuard() {
      if (e) cudaGraphExecDestroy(e);
    }
  } G;
  bool graph_ok = true;
  for (;;) {
    for (auto& r : runs)
      if (!r.done) TRY(run_residual(r));
    std::vector<char> part(n, 0);
    int nin = 0;
    for (int i = 0; i < n; ++i) {
      SolveRun& r = runs[i];
      if (r.done) continue;
      bool need = false;
      TRY(run_check(r, &need));
      if (!need) continue;
      LoopArgs L;
      TRY(run_inner_pre(r, &L));
      part[i] = 1;
      ++nin;
    }
    if (nin == 0) break;
    if (graph_ok && !G.e) {
      const xfft_status bs = build_device_loop(all, B.lm, limit, &G.e);
      if (bs == XFFT_EUNSUPPORTED) graph_ok = false;
      else TRY(bs);
    }
    bool timed_out = false;
    if (graph_ok) {
      for (int i = 0; i < n; ++i)
        if (!part[i]) CU(cudaMemsetAsync(ctxs[i]->act, 0, 64 * sizeof(int), ctxs[i]->stream));
      TRY(run_device_loop(all, B.master, G.e, B.fork, B.joins, &part));
      CU(cudaMemcpyAsync(B.lm_host, B.lm, kLoopStride * n, cudaMemcpyDeviceToHost, B.master));
      CU(cudaStreamSynchronize(B.master));
      for (int i = 0; i < n; ++i)
        if (part[i] && reinterpret_cast<const LoopState*>(B.lm_host + kLoopStride * i)->timed_out) timed_out = true;
    } else {
      for (int i = 0; i < n; ++i) {  // no conditional graphs: each context's own loop
        if (!part[i]) continue;
        ctxs[i]->devloop_ok = false;
        bool to = false;
        TRY(cg_loop(all[i], &to));
        timed_out = timed_out || to;
      }
    }
    for (int i = 0; i < n; ++i)
      if (part[i]) TRY(run_inner_post(runs[i], timed_out));
  }
  for (int i = 0; i < n; ++i) {
    CU(cudaEventRecord(B.joins[i], ctxs[i]->stream));
    CU(cudaStreamWaitEvent(B.master, B.joins[i], 0));
  }
  CU(cudaEventRecord(B.t1, B.master));
  CU(cudaEventSynchronize(B.t1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, B.t0, B.t1);
  xfft_status first = XFFT_OK;
  std::string msg;
  for (int i = 0; i < n; ++i) {
    const xfft_status st = finish_six(ctxs[i], Rs[i], C_eff + 36 * (size_t)i, stats ? stats + i : nullptr, ms);
    if (st != XFFT_OK && (first == XFFT_OK || (first == XFFT_ENOTCONV && st != XFFT_ENOTCONV))) {
      first = st;
      msg = "context " + std::to_string(i) + ": " + g_err;
    }
  }
  if (first != XFFT_OK) return fail(first, msg);
  return XFFT_OK;
}

extern "C" xfft_status xfft_grad(xfft_ctx* c, const double dL_dCeff[36], double dL_dlame[4],
                                 float* dL_dscale, double C_energy[36], int ptrs_on_device) {
  if (c && c->have_micro && c->ph.nph != 2)
    return fail(XFFT_EINVAL, "more than two phases: use xfft_grad_phases");
  return xfft_grad_phases(c, dL_dCeff, dL_dlame, dL_dscale, C_energy, ptrs_on_device);
}

extern "C" xfft_status xfft_grad_phases(xfft_ctx* c, const double dL_dCeff[36], double* dL_dlame,
                                        float* dL_dscale, double C_energy[36], int ptrs_on_device) {
  if (!c || !dL_dCeff || !dL_dlame) return fail(XFFT_EINVAL, "NULL argument");
  if (!c->have_micro || !c->have6) return fail(XFFT_ESTATE, "xfft_effective_stiffness first");
  TRY(ensure_work(c, 6, c->cap_prec >= 0 ? c->cap_prec : c->opt.precision));
  const GridDev& g = c->g;
  cudaStream_t s = c->stream;
  GradArgs a;
  a.g = g;
  a.ph = c->ph;
  a.code = c->code;
  a.scale = c->has_scale ? c->scale : nullptr;
  a.stride = stride_of(c);
  a.nX = c->nX;
  for (int k = 0; k < 36; ++k) a.G[k] = dL_dCeff[k];
  a.partials = c->partials;
  a.nparts = grad_blocks_uncut(g) + grad_blocks_cut(c->ncut);
  a.part_offset_cut = grad_blocks_uncut(g);
  if (!c->dscale) CU(dalloc(c, &c->dscale, g.N));
  {
    ProfScope ps(c, XFFT_PROF_GRAD, 3);
    // the mixed-precision gradient splits U into float pairs in the solve's float work vectors
    // (free between solves; at least 6 * stride floats each)
    const bool f32 = c->opt.precision == XFFT_FP32_REFINED && c->cap_prec == XFFT_FP32_REFINED && c->v32[0] &&
                     c->v32[1] && c->cap_rhs >= 6;
    CU(launch_grad(c->U6, c->isD, cutdata(c), a, c->dscale, f32 ? c->v32[0] : nullptr, f32 ? c->v32[1] : nullptr, s));
    CU(launch_reduce_partials(c->partials, kGradValues, a.nparts, a.nparts, c->red_out, s));
  }
  double red[kGradValues];
  CU(cudaMemcpyAsync(red, c->red_out, sizeof(red), cudaMemcpyDeviceToHost, s));
  if (dL_dscale) {
    ProfScope ps(c, XFFT_PROF_GRAD, 1);
    if (ptrs_on_device) {
      CU(launch_scale_copy<double, float>(c->dscale, dL_dscale, 1.0, g.N, 1, nullptr, s));
    } else {
      if (!c->dscale_f) CU(dalloc(c, &c->dscale_f, g.N));
      CU(launch_scale_copy<double, float>(c->dscale, c->dscale_f, 1.0, g.N, 1, nullptr, s));
      CU(cudaMemcpyAsync(dL_dscale, c->dscale_f, g.N * sizeof(float), cudaMemcpyDeviceToHost, s));
    }
  }
  CU(cudaStreamSynchronize(s));
  for (int p = 0; p < c->ph.nph; ++p) {
    dL_dlame[2 * p] = red[p];                   // lambda_p
    dL_dlame[2 * p + 1] = red[kMaxPhases + p];  // mu_p
  }
  if (C_energy) {
    int idx = 0;
    for (int k = 0; k < 6; ++k)
      for (int l = k; l < 6; ++l, ++idx) {
        C_energy[k * 6 + l] = red[2 * kMaxPhases + idx];
        C_energy[l * 6 + k] = red[2 * kMaxPhases + idx];
      }
  }
  return XFFT_OK;
}

// ---------------------------------------------------------------- step-level entry points
template <typename T>
static xfft_status stage_in(xfft_ctx* c, const double* src, T* dst, size_t count, int on_dev,
                            double* scratch64) {
  // dst (device, type T) <- src (double, host or device)
  const double* dsrc = src;
  if (!on_dev) {
    CU(cudaMemcpyAsync(scratch64, src, count * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    dsrc = scratch64;
  }
  CU(launch_scale_copy<double, T>(dsrc, dst, 1.0, (long long)count, 1, nullptr, c->stream));
  return XFFT_OK;
}

template <typename T>
static xfft_status stage_out(xfft_ctx* c, const T* src, double* dst, size_t count, int on_dev,
                             double* scratch64) {
  double* ddst = on_dev ? dst : scratch64;
  CU(launch_scale_copy<T, double>(src, ddst, 1.0, (long long)count, 1, nullptr, c->stream));
  if (!on_dev)
    CU(cudaMemcpyAsync(dst, scratch64, count * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  return XFFT_OK;
}

template <typename T, typename A = T>
static xfft_status apply_entry(xfft_ctx* c, int n_rhs, const double* d, const double* eps_bar, double* q,
                               double* sigma_int, int on_dev) {
  const long long stride = stride_of(c);
  const size_t tot = (size_t)n_rhs * stride;
  double* scratch = nullptr;
  T* dd = nullptr;
  T* qq = nullptr;
  cudaError_t ea = dalloc(c, &scratch, tot);
  if (ea == cudaSuccess) ea = dalloc(c, &dd, tot);
  if (ea == cudaSuccess) ea = dalloc(c, &qq, tot);
  xfft_status st = XFFT_OK;
  if (ea != cudaSuccess)
    st = fail(ea == cudaErrorMemoryAllocation ? XFFT_ENOMEM : XFFT_ECUDA, cudaGetErrorString(ea));
  if (st == XFFT_OK) st = stage_in<T>(c, d, dd, tot, on_dev, scratch);
  if (st == XFFT_OK && eps_bar) st = upload_eps(c, n_rhs, eps_bar);
  if (st == XFFT_OK)
    st = do_apply<T, A>(c, dd, qq, eps_bar ? c->eps_d : nullptr, n_rhs, nullptr, -1, 0, 0, 0, nullptr,
                        nullptr, nullptr, 0, (sigma_int || eps_bar) ? 1 : 0);
  if (st == XFFT_OK) st = stage_out<T>(c, qq, q, tot, on_dev, scratch);
  if (st == XFFT_OK && sigma_int) {
    const int nparts = nparts_of(c);
    const int used = apply_uncut_blocks(c->g) + cut_blocks_of(c, sizeof(T) == 4);
    cudaError_t e = launch_reduce_partials(c->partials, 7 * n_rhs, nparts, used, c->red_out, c->stream);
    double red[7 * 64];
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(red, c->red_out, 7 * n_rhs * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) st = fail(XFFT_ECUDA, cudaGetErrorString(e));
    for (int r = 0; r < n_rhs && st == XFFT_OK; ++r)
      for (int k = 0; k < 6; ++k) sigma_int[6 * r + k] = red[7 * r + 1 + k];
  }
  cudaError_t e = cudaStreamSynchronize(c->stream);
  dfree(c, scratch);
  dfree(c, dd);
  dfree(c, qq);
  if (st == XFFT_OK && e != cudaSuccess) st = fail(XFFT_ECUDA, cudaGetErrorString(e));
  return st;
}

extern "C" xfft_status xfft_apply(xfft_ctx* c, int n_rhs, const double* d, const double* eps_bar,
                                  double* q, double* sigma_int, int precision, int ptrs_on_device) {
  if (!c || !d || !q) return fail(XFFT_EINVAL, "NULL argument");
  if (!c->have_micro) return fail(XFFT_ESTATE, "xfft_set_microstructure first");
  if (n_rhs < 1 || n_rhs > 64) return fail(XFFT_EINVAL, "n_rhs must be in [1, 64]");
  TRY(ensure_work(c, std::max(n_rhs, c->cap_rhs), c->cap_prec >= 0 ? c->cap_prec : c->opt.precision));
  if (precision == XFFT_FP64) return apply_entry<double>(c, n_rhs, d, eps_bar, q, sigma_int, ptrs_on_device);
  if (precision == XFFT_DW)
    return apply_entry<double, dw>(c, n_rhs, d, eps_bar, q, sigma_int, ptrs_on_device);
  if (precision == XFFT_FP32_REFINED)
    return apply_entry<float>(c, n_rhs, d, eps_bar, q, sigma_int, ptrs_on_device);
  return fail(XFFT_EINVAL, "precision must be XFFT_FP64, XFFT_FP32_REFINED or XFFT_DW");
}

template <typename T>
static xfft_status prec_entry(xfft_ctx* c, int n_rhs, const double* f, double* z, double* rr, int on_dev) {
  const long long stride = stride_of(c);
  const size_t tot = (size_t)n_rhs * stride;
  double* scratch = nullptr;
  T* ff = nullptr;
  T* zz = nullptr;
  void* spec_save = c->spec;
  void* spec = nullptr;
  cudaError_t ea = dalloc(c, &scratch, tot);
  if (ea == cudaSuccess) ea = dalloc(c, &ff, tot);
  if (ea == cudaSuccess) ea = dalloc(c, &zz, tot);
  if (ea == cudaSuccess) ea = dalloc_bytes(c, &spec, (size_t)n_rhs * fft_spectrum_elems(c->fft) * sizeof(T) * 2);
  xfft_status st = XFFT_OK;
  if (ea != cudaSuccess)
    st = fail(ea == cudaErrorMemoryAllocation ? XFFT_ENOMEM : XFFT_ECUDA, cudaGetErrorString(ea));
  else
    c->spec = spec;
  if (st == XFFT_OK) st = stage_in<T>(c, f, ff, tot, on_dev, scratch);
  if (st == XFFT_OK) st = do_prec<T>(c, ff, zz, n_rhs, nullptr, -1, 0, 0, 0);
  if (st == XFFT_OK) st = stage_out<T>(c, zz, z, tot, on_dev, scratch);
  if (st == XFFT_OK && rr) {
    const int nparts = nparts_of(c);
    cudaError_t e = launch_reduce_partials(c->partials, n_rhs, nparts,
                                           precondition_blocks(c->fft, c->nX, sizeof(T) == 8), c->red_out,
                                           c->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(rr, c->red_out, n_rhs * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) st = fail(XFFT_ECUDA, cudaGetErrorString(e));
  }
  cudaError_t e = cudaStreamSynchronize(c->stream);
  c->spec = spec_save;
  if (spec) dfree_bytes(c, spec);
  dfree(c, scratch);
  dfree(c, ff);
  dfree(c, zz);
  if (st == XFFT_OK && e != cudaSuccess) st = fail(XFFT_ECUDA, cudaGetErrorString(e));
  return st;
}

extern "C" xfft_status xfft_precondition(xfft_ctx* c, int n_rhs, const double* f, double* z, double* rr,
                                         int precision, int ptrs_on_device) {
  if (!c || !f || !z) return fail(XFFT_EINVAL, "NULL argument");
  if (!c->have_micro) return fail(XFFT_ESTATE, "xfft_set_microstructure first");
  if (n_rhs < 1 || n_rhs > 64) return fail(XFFT_EINVAL, "n_rhs must be in [1, 64]");
  TRY(ensure_work(c, std::max(n_rhs, c->cap_rhs), c->cap_prec >= 0 ? c->cap_prec : c->opt.precision));
  return precision == XFFT_FP64 ? prec_entry<double>(c, n_rhs, f, z, rr, ptrs_on_device)
                                : prec_entry<float>(c, n_rhs, f, z, rr, ptrs_on_device);
}

extern "C" xfft_status xfft_get_setup(xfft_ctx* c, int* enr_nodes, double* D0, unsigned short* tet_code) {
  if (!c) return fail(XFFT_EINVAL, "NULL argument");
  if (!c->have_micro) return fail(XFFT_ESTATE, "xfft_set_microstructure first");
  cudaStream_t s = c->stream;
  if (enr_nodes && c->nX > 0)
    CU(cudaMemcpyAsync(enr_nodes, c->enr_nodes, c->nX * sizeof(int), cudaMemcpyDeviceToHost, s));
  if (D0 && c->nX > 0) {
    // device layout [component][j]; API layout [j][component]
    std::vector<double> tmp(3 * (size_t)c->nX);
    CU(cudaMemcpyAsync(tmp.data(), c->D, tmp.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    for (int j = 0; j < c->nX; ++j)
      for (int k = 0; k < 3; ++k) D0[3 * (size_t)j + k] = tmp[(size_t)k * c->nX + j];
  }
  if (tet_code)
    CU(cudaMemcpyAsync(tet_code, c->code, c->g.N * sizeof(uint16_t), cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  return XFFT_OK;
}

extern "C" xfft_status xfft_profile(xfft_ctx* c, int enable) {
  if (!c) return fail(XFFT_EINVAL, "NULL argument");
  CU(prof_flush(c));
  c->prof = enable != 0;
  if (enable) {
    for (int k = 0; k < 16; ++k) {
      c->pms[k] = 0.0;
      c->plaunch[k] = 0;
    }
    CU(cudaMemsetAsync(c->punits, 0, 16 * sizeof(unsigned long long), c->stream));
    CU(cudaStreamSynchronize(c->stream));
  }
  return XFFT_OK;
}

extern "C" xfft_status xfft_profile_read(xfft_ctx* c, double ms[16], long long launches[16],
                                         long long units[16]) {
  if (!c) return fail(XFFT_EINVAL, "NULL argument");
  CU(prof_flush(c));
  unsigned long long u[16];
  CU(cudaMemcpyAsync(u, c->punits, sizeof(u), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  for (int k = 0; k < 16; ++k) {
    if (ms) ms[k] = c->pms[k];
    if (launches) launches[k] = c->plaunch[k];
    if (units) units[k] = (long long)u[k];
  }
  return XFFT_OK;
}

// ---------------------------------------------------------------- allocation-free apply
// Reduction scratch of xfft_apply_noalloc: 7 partial-sum rows per right-hand side.  Host code
// must not pass g_noalloc_scratch itself to a kernel (in host code the name is only a host-side
// stand-in); its device address is looked up once per device with cudaGetSymbolAddress.
static __device__ __align__(256) double g_noalloc_scratch[XFFT_NOALLOC_MAX_RHS * 7 * XFFT_NOALLOC_MAX_PARTS];

static std::mutex g_noalloc_mu;
static double* g_noalloc_ptr[64] = {};

// Device address of the scratch array on the current device, looked up once per device.
// stream: when the address is not cached yet and this stream is being captured, the lookup
// (which may initialise the module on the device) is refused with XFFT_ESTATE.
static xfft_status noalloc_scratch(double** out, cudaStream_t stream) {
  int dev = 0;
  CU(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(XFFT_EUNSUPPORTED, "device index above 63");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (stream && cudaStreamIsCapturing(stream, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
      return fail(XFFT_ESTATE,
                  "xfft_apply_noalloc: the scratch address of this device is not known yet; make "
                  "one call (or xfft_set_microstructure) before capturing the stream");
    void* p = nullptr;
    CU(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return XFFT_OK;
}

// called by xfft_set_microstructure (which runs outside any capture): resolves the scratch
// address of the current device so that xfft_apply_noalloc needs no set-up of its own
static xfft_status noalloc_prepare(cudaStream_t stream) {
  double* p = nullptr;
  return noalloc_scratch(&p, stream);
}

extern "C" xfft_status xfft_apply_noalloc(xfft_ctx* c, int n_rhs, const double* d, double* q,
                                          double* dAd_sig) {
  if (!c || !d || !q) return fail(XFFT_EINVAL, "NULL argument");
  if (!c->have_micro) return fail(XFFT_ESTATE, "xfft_set_microstructure first");
  if (n_rhs < 1 || n_rhs > XFFT_NOALLOC_MAX_RHS)
    return fail(XFFT_EINVAL, "n_rhs must be in [1, XFFT_NOALLOC_MAX_RHS]");
  const int nparts = apply_uncut_blocks(c->g) + apply_cut_blocks(c->ncut);
  if (nparts > XFFT_NOALLOC_MAX_PARTS)
    return fail(XFFT_EINVAL, "grid too large for the fixed scratch of xfft_apply_noalloc");
  double* scratch = nullptr;
  TRY(noalloc_scratch(&scratch, c->stream));
  ApplyArgs a;
  a.g = c->g;
  a.ph = c->ph;
  a.code = c->code;
  a.scale = c->has_scale ? c->scale : nullptr;
  a.eps = nullptr;
  a.active = nullptr;
  a.stride = stride_of(c);
  a.nX = c->nX;
  a.partials = scratch;
  a.nparts = nparts;
  a.part_offset_cut = apply_uncut_blocks(c->g);
  a.units_uncut = nullptr;
  a.units_cut = nullptr;
  a.want_sig = 1;
  a.kcache = c->kcache;
  a.fz = nullptr;
  a.fdnew = nullptr;
  a.fu = nullptr;
  a.st = nullptr;
  CU(launch_apply<double>(d, q, c->isD, cutdata(c), a, n_rhs, c->stream));
  if (dAd_sig) CU(launch_reduce_partials(scratch, 7 * n_rhs, nparts, nparts, dAd_sig, c->stream));
  return XFFT_OK;
}
