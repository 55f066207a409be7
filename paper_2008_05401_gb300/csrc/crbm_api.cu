// C ABI of the CRBM-aided Monte Carlo library (declarations and contracts in
// include/crbm.h).  Host side: contexts, models (row-sum tables of the CRBM
// filters), jobs laid out in caller-owned device memory, and kernel launches.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdlib>
#include <map>
#include <tuple>
#include <cstdio>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "crbm.h"
#include "crbm_device.cuh"
#include "crbm_kernels.h"

using namespace crbm;

namespace {

struct Model {
  bool live = false;
  int kind = 0, K = 0, k = 0;
  int edge = 0, ncls = 1;    // LCRBM: edge unshared kernels per side, 2 edge + 1 classes (FP64 tables only)
  double vb = 0.0;
  std::vector<double> hb;
  double* d_f64 = nullptr;   // forward FP64 row-sum table, then the backward one
  float* d_f32 = nullptr;    // fd, bd, fh, fl
  float4* d_q = nullptr;     // fd4, fh4, fl4 (filter-interleaved, K <= 4)
  size_t nlut = 0, nq = 0;
  float hb32[kMaxK] = {}, hb_hi[kMaxK] = {}, hb_lo[kMaxK] = {};
  float vb32 = 0.f;
  float c0h = 0.f, c0v = 0.f, c1 = 0.f, csp = 0.f, cdf = 0.f;
  // tensor-core form (Ising, K <= 4, k <= 5): filter-digit operand images
  uint4* d_tc = nullptr;
  size_t tc_bytes = 0;
  float tq2 = 0.f, tq1 = 0.f, tq0 = 0.f, tc0h = 0.f, tc0v = 0.f, tc1 = 0.f, tcft = 0.f;
};

struct Layout {
  size_t bits, T, F, Fb, Lb, lp, E, ot, os, acc, rec, step, sched, eps, total;
};

struct Job {
  bool live = false;
  int model = -1, kind = 0, L = 0, N = 0, Wd = 0, n = 0, nc = 1, tiles = 0;
  int tpc = 0;   // Kitaev: threads of each chain's group (chains per CTA follow per launch)
  double J[3] = {1.0, 1.0, 1.0};
  uint64_t seed = 0, cid_base = 0, step = 0;
  unsigned char* mem = nullptr;
  size_t bytes = 0;
  Layout lay{};
  cudaStream_t stream = nullptr;
  std::vector<double> T;   // host copy of the temperatures
  // F and log pi of every chain are FP64 values (bounds 0) and, for the
  // Kitaev kind, eps holds the spectra of the current lattices: true after an
  // evaluation or a tempering cycle, false after proposals (mode 0)
  bool exact = false;
  bool fexact = false;       // F of every chain is an FP64 value (bound 0)
  // log pi, F and E_phys of every chain are the FP64 path's values (after an
  // FP64 evaluation or an FP64 run; false after a mixed run, whose F carries
  // an FP32 bound and, for the Kitaev kind, whose log pi a double-FP32 one)
  bool f64vals = false;
  // optional E_phys trace in caller-owned device memory (crbm_set_trace)
  double* trace = nullptr;
  uint64_t trace_base = 0;
  int64_t trace_cap = 0;
};

Layout make_layout(int kind, int L, int n) {
  Layout y{};
  size_t off = 0;
  auto take = [&](size_t b) {
    const size_t o = off;
    off += (b + 255) & ~size_t(255);
    return o;
  };
  const size_t Wd = ((size_t)L * L + 31) / 32;
  y.bits = take((size_t)n * Wd * 4);
  y.T = take((size_t)n * 8);
  y.F = take((size_t)n * 8);
  y.Fb = take((size_t)n * 8);
  y.Lb = take((size_t)n * 8);
  y.lp = take((size_t)n * 8);
  y.E = take((size_t)n * 8);
  y.ot = take((size_t)n * 8 * kNobs);
  y.os = take((size_t)n * 8 * kNobs);
  y.acc = take((size_t)n * 8);
  y.rec = take((size_t)n * 16);
  y.step = take(8);
  y.sched = take(16);     // work-queue counter of the tensor-core kernel's launches led by this job
  y.eps = take(kind == kKitaev ? (size_t)n * L * L * 8 : 0);
  y.total = n > 0 ? off : 0;   // an empty job needs no device memory
  return y;
}

bool valid_L(int kind, int L) {
  if (kind == kIsing) return (L >= 2 && L <= 32) || (L % 32 == 0 && L <= 256);
  if (kind == kKitaev) return L >= 2 && L <= 12;
  return false;
}

// Chains per CTA of an Ising job: about two 4-site units per thread, a power
// of two in [1, 32].  (A Kitaev job's follow from its group size per launch.)
int chains_per_tile(int kind, int L) {
  if (kind == kKitaev) return 1;
  const int nblk = (L * L + 3) / 4;
  int nc = 1;
  while (nc < kThreads / 8 && (nc * 2) * nblk <= 2 * kThreads) nc *= 2;
  return nc;
}

}  // namespace

struct crbm_ctx {
  int device = 0;
  size_t budget = 0, used = 0;
  std::vector<Model> models;
  std::vector<Job> jobs;
  std::string err;
  int* d_err = nullptr;
  // non-blocking stream of the context's own copies and evaluation launches,
  // so that job set-up never waits for other streams' work
  cudaStream_t own = nullptr;
  // side streams and events of a batch whose jobs need launches of different
  // CTA sizes: the launches fork from the caller's stream and join it again,
  // so they run side by side
  static constexpr int kSide = 7;
  cudaStream_t side[kSide] = {};
  cudaEvent_t fork = nullptr, join[kSide] = {};
  struct Graph {
    bool live = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<int> jobs;
    uint64_t steps = 0;   // proposals per replay
    int precision = 0;
  };
  std::vector<Graph> graphs;
  // chains per CTA chosen by crbm_tune for (kind, L, K, k)
  std::map<std::tuple<int, int, int, int>, int> tuned;
  // proposals of eligible jobs (crbm_step_tc.cu) run on the tensor-core form;
  // tc_ok: the device grants its shared memory
  bool use_tc = true, tc_ok = false;
  int sms = 1;                          // SMs of the device: persistent grid size
  long long wait_limit = 1ll << 28;     // cycles before a device-side wait gives up
  // device buffer of crbm_read_energies' FP64 re-evaluation (a copy of one
  // job's memory), grown on demand
  unsigned char* scratch = nullptr;
  size_t scratch_bytes = 0;
};

static int fail(crbm_ctx* c, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return code;
}

static int cuda_fail(crbm_ctx* c, cudaError_t e, const char* where) {
  return fail(c, CRBM_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define CK(call, where)                                  \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where); \
  } while (0)

static Job* get_job(crbm_ctx* ctx, int id) {
  if (!ctx || id < 0 || id >= (int)ctx->jobs.size() || !ctx->jobs[id].live) return nullptr;
  return &ctx->jobs[id];
}

static JobDev make_jobdev(const crbm_ctx* ctx, const Job& j) {
  const Model& m = ctx->models[j.model];
  JobDev d;
  memset(&d, 0, sizeof d);
  d.kind = j.kind;
  d.L = j.L;
  d.N = j.N;
  d.Wd = j.Wd;
  d.P = j.Wd + 1;
  d.K = m.K;
  d.k = m.k;
  d.n_chains = j.n;
  d.nc = j.nc;
  d.vb = m.vb;
  d.lc_edge = m.edge;
  d.ncls = m.ncls;
  d.nhex = m.edge ? j.L * (j.L - 1) : j.N;
  for (int f = 0; f < m.K; ++f) {
    d.hb[f] = m.hb[f];
    d.hb32[f] = m.hb32[f];
    d.hb_hi[f] = m.hb_hi[f];
    d.hb_lo[f] = m.hb_lo[f];
  }
  for (int i = 0; i < 3; ++i) d.J[i] = j.J[i];
  d.vb32 = m.vb32;
  d.c0h = m.c0h;
  d.c0v = m.c0v;
  d.c1 = m.c1;
  d.csp = m.csp;
  d.cdf = m.cdf;
  d.f64 = m.d_f64;
  d.b64 = m.d_f64 + m.nlut;
  if (m.d_f32) {                 // an LCRBM has FP64 tables only
    d.fd = m.d_f32;
    d.bd = m.d_f32 + m.nlut;
    d.fh = m.d_f32 + 2 * m.nlut;
    d.fl = m.d_f32 + 3 * m.nlut;
  }
  if (m.d_tc) {
    d.tcw = m.d_tc;
    d.tq2 = m.tq2;
    d.tq1 = m.tq1;
    d.tq0 = m.tq0;
    d.tc0h = m.tc0h;
    d.tc0v = m.tc0v;
    d.tc1 = m.tc1;
    d.tcft = m.tcft;
  }
  if (m.d_q) {
    d.fd4 = m.d_q;
    d.fh4 = m.d_q + m.nq;
    d.fl4 = m.d_q + 2 * m.nq;
  }
  d.seed = j.seed;
  for (int r = 0; r < 10; ++r) {
    d.rk[2 * r] = (uint32_t)j.seed + (uint32_t)r * 0x9E3779B9u;
    d.rk[2 * r + 1] = (uint32_t)(j.seed >> 32) + (uint32_t)r * 0xBB67AE85u;
  }
  d.cid_base = j.cid_base;
  d.step = (unsigned long long*)(j.mem + j.lay.step);
  unsigned char* b = j.mem;
  d.bits = (uint32_t*)(b + j.lay.bits);
  d.T = (const double*)(b + j.lay.T);
  d.F = (double*)(b + j.lay.F);
  d.Fb = (double*)(b + j.lay.Fb);
  d.Lb = (double*)(b + j.lay.Lb);
  d.logpi = (double*)(b + j.lay.lp);
  d.Ephys = (double*)(b + j.lay.E);
  d.obs_t = (double*)(b + j.lay.ot);
  d.obs = (double*)(b + j.lay.os);
  d.acc = (unsigned long long*)(b + j.lay.acc);
  d.rec = (unsigned long long*)(b + j.lay.rec);
  d.eps = (double*)(b + j.lay.eps);
  d.trace = j.trace;
  d.trace_base = j.trace_base;
  d.trace_cap = j.trace_cap;
  return d;
}

// Launch the fused kernel for a set of jobs (same kind and filter shape);
// mode 1 = evaluate.  The threads of a chain's group (Ising: the job's chains
// per 256-thread CTA; Kitaev: the job's group size) -- and so its per-chain
// reduction order and every bit of its results -- depend only on the job, so
// it gives the same results alone or batched.  A Kitaev launch takes CTAs of
// the largest group size among its jobs, each job as many chains per CTA as
// its groups fill: small matrices alone run in small CTAs, a batch of mixed
// sizes in one launch.  The jobs' tiles are laid out by decreasing lattice
// side, so that the longest tiles start first and the short ones fill the end.
static int launch_group(crbm_ctx* ctx, std::vector<int> ids, int S, int g, int correct, int prec,
                        int mode, int nt, cudaStream_t st, const Job* partner = nullptr) {
  if (!partner)
    std::stable_sort(ids.begin(), ids.end(), [&](int a, int b) { return ctx->jobs[a].L > ctx->jobs[b].L; });
  const bool kitaev = !ids.empty() && ctx->jobs[ids[0]].kind == kKitaev;
  bool multi = false;
  if (kitaev) {
    // one chain per CTA of its group size when every job has the same;
    // otherwise CTAs of 256 threads holding several groups (proposals only:
    // the other modes run one job at a time)
    nt = 32;
    for (int id : ids) nt = std::max(nt, ctx->jobs[id].tpc);
    for (int id : ids) multi = multi || ctx->jobs[id].tpc != nt;
    if (multi) {
      if (mode != 0) return fail(ctx, CRBM_EINVAL, "jobs of different group sizes in a mode-%d launch", mode);
      nt = kThreads;
    }
  }
  LaunchParams p;
  memset(&p, 0, sizeof p);
  p.n_jobs = (int)ids.size();
  p.S = S;
  p.g = g;
  p.correct = correct;
  p.mode = mode;
  p.err = ctx->d_err;
  p.wait_limit = ctx->wait_limit;
  size_t smem = 0;
  int tiles = 0, kind = -1, K = 0, k = 0;
  bool generic = false;
  for (size_t i = 0; i < ids.size(); ++i) {
    const Job& j = ctx->jobs[ids[i]];
    const Model& m = ctx->models[j.model];
    kind = j.kind;
    p.tile_begin[i] = tiles;
    p.job[i] = make_jobdev(ctx, j);
    const int nc = kitaev ? nt / j.tpc : j.nc;
    p.job[i].nc = nc;
    tiles += kitaev ? (j.n + nc - 1) / nc : j.tiles;
    if (m.edge && prec != kFP64) return fail(ctx, CRBM_EINVAL, "LCRBM models run in CRBM_FP64 only");
    int KC, kC;
    specialisation(m.K, m.k, KC, kC);
    if (m.edge) {
      KC = kC = 0;                // the class tables are read by the runtime-shape code
      generic = true;
    }
    const size_t b = smem_bytes(j.kind, prec, j.L, m.K, m.k, nc, KC, m.ncls);
    if (b > smem) smem = b;
    K = m.K;
    k = m.k;
  }
  p.tile_begin[ids.size()] = tiles;
  if (partner) p.job[ids.size()] = make_jobdev(ctx, *partner);    // tempering: the physical chains
  if (tiles == 0) return CRBM_OK;
  if (generic) {
    // every job of the launch runs the runtime-shape variant: size its shared memory so
    smem = 0;
    for (size_t i = 0; i < ids.size(); ++i) {
      const Job& j = ctx->jobs[ids[i]];
      const Model& m = ctx->models[j.model];
      smem = std::max(smem, smem_bytes(j.kind, prec, j.L, m.K, m.k, p.job[i].nc, 0, m.ncls));
    }
  }
  CK(launch_step(kind, prec, K, k, nt, p, tiles, smem, st, generic, multi), "kernel launch");
  return CRBM_OK;
}

// Whether the proposals of job j run on the tensor-core form: a property of
// the job alone (kind, precision, lattice, filter bank), so that its results
// are the same alone or batched.
static bool on_tc(const crbm_ctx* ctx, const Job& j, int prec, int mode) {
  const Model& m = ctx->models[j.model];
  return ctx->use_tc && ctx->tc_ok && (mode == 0 || mode == 1) && m.d_tc && !m.edge &&
         tc_supported(j.kind, prec, j.L, m.K, m.k);
}

// One persistent launch of the tensor-core kernel for the given jobs (any of
// the four sides): a tile of 128 / L chains per work item, the jobs ordered by
// decreasing L so that the longest items go first; the work-queue counter is
// the first job's.
static int launch_tc_group(crbm_ctx* ctx, std::vector<int> ids, int S, int g, int correct, int mode,
                           cudaStream_t st) {
  std::stable_sort(ids.begin(), ids.end(), [&](int a, int b) { return ctx->jobs[a].L > ctx->jobs[b].L; });
  LaunchParams p;
  memset(&p, 0, sizeof p);
  p.n_jobs = (int)ids.size();
  p.S = S;
  p.g = g;
  p.correct = correct;
  p.mode = mode;                 // 0: proposals, 1: evaluation of the current lattices
  p.err = ctx->d_err;
  p.wait_limit = ctx->wait_limit;
  int tiles = 0;
  size_t smem = 0;
  for (size_t i = 0; i < ids.size(); ++i) {
    const Job& j = ctx->jobs[ids[i]];
    const Model& m = ctx->models[j.model];
    p.tile_begin[i] = tiles;
    p.job[i] = make_jobdev(ctx, j);
    const int ch = tc_chains_per_cta(j.L);
    tiles += (j.n + ch - 1) / ch;
    smem = std::max(smem, tc_smem_bytes(j.L, m.K, m.k));
  }
  p.tile_begin[ids.size()] = tiles;
  p.total_items = tiles;
  if (tiles == 0 || (S == 0 && mode == 0)) return CRBM_OK;
  const Job& lead = ctx->jobs[ids[0]];
  p.queue = (int*)(lead.mem + lead.lay.sched);
  CK(launch_tc(p, std::min(tiles, ctx->sms), smem, st), "kernel launch");
  return CRBM_OK;
}

static int launch_jobs(crbm_ctx* ctx, const std::vector<int>& ids, int S, int g, int correct, int prec, int mode,
                       cudaStream_t st, const Job* partner = nullptr) {
  // parts: (CTA size, jobs); CTA size -1 = the tensor-core form (one persistent launch for every side)
  std::vector<std::pair<int, std::vector<int>>> parts;
  for (int nt : {-1, 256, 128, 64, 32}) {
    std::vector<int> part;
    for (int id : ids) {
      const Job& j = ctx->jobs[id];
      if (j.n == 0) continue;
      const bool tc = !partner && on_tc(ctx, j, prec, mode);
      if (nt < 0 ? tc : (!tc && threads_for(j.kind, j.N) == nt)) part.push_back(id);
    }
    if (!part.empty()) parts.emplace_back(nt, part);
  }
  auto launch_part = [&](const std::pair<int, std::vector<int>>& pt, cudaStream_t s) {
    return pt.first < 0 ? launch_tc_group(ctx, pt.second, S, g, correct, mode, s)
                        : launch_group(ctx, pt.second, S, g, correct, prec, mode, pt.first, s, partner);
  };
  if (parts.size() <= 1) {
    for (auto& pt : parts) {
      const int rc = launch_part(pt, st);
      if (rc) return rc;
    }
    return CRBM_OK;
  }
  // several CTA sizes: the first launch on st, the others on side streams
  // forked from st and joined back into it
  if (parts.size() > (size_t)crbm_ctx::kSide + 1) return fail(ctx, CRBM_EINVAL, "too many kernel kinds in one batch");
  CK(cudaEventRecord(ctx->fork, st), "fork event");
  for (size_t i = 1; i < parts.size(); ++i) CK(cudaStreamWaitEvent(ctx->side[i - 1], ctx->fork, 0), "fork wait");
  int rc = CRBM_OK;
  for (size_t i = 0; i < parts.size() && rc == CRBM_OK; ++i) rc = launch_part(parts[i], i == 0 ? st : ctx->side[i - 1]);
  for (size_t i = 1; i < parts.size(); ++i) {
    CK(cudaEventRecord(ctx->join[i - 1], ctx->side[i - 1]), "join event");
    CK(cudaStreamWaitEvent(st, ctx->join[i - 1], 0), "join wait");
  }
  return rc;
}

extern "C" {

int crbm_create(crbm_ctx** out, int device, size_t hbm_budget_bytes) {
  if (!out) return CRBM_EINVAL;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return CRBM_EINVAL;
  crbm_ctx* ctx = new crbm_ctx();
  ctx->device = device;
  ctx->budget = hbm_budget_bytes;
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(ctx->d_err, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->own, cudaStreamNonBlocking);
  for (int i = 0; i < crbm_ctx::kSide && e == cudaSuccess; ++i) {
    e = cudaStreamCreateWithFlags(&ctx->side[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->join[i], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) {
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, device);
    if (ctx->sms < 1) ctx->sms = 1;
    e = set_smem_limits((size_t)optin);
    if (e == cudaSuccess && (size_t)optin >= tc_smem_bytes(128, 4, 5)) {
      e = tc_set_smem_limit();
      ctx->tc_ok = e == cudaSuccess;
    }
  }
  if (e != cudaSuccess) {
    if (ctx->d_err) cudaFree(ctx->d_err);
    delete ctx;
    return CRBM_ECUDA;
  }
  *out = ctx;
  return CRBM_OK;
}

int crbm_destroy(crbm_ctx* ctx) {
  if (!ctx) return CRBM_EINVAL;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  for (auto& m : ctx->models) {
    if (m.d_f64) cudaFree(m.d_f64);
    if (m.d_f32) cudaFree(m.d_f32);
    if (m.d_q) cudaFree(m.d_q);
    if (m.d_tc) cudaFree(m.d_tc);
  }
  if (ctx->d_err) cudaFree(ctx->d_err);
  if (ctx->scratch) cudaFree(ctx->scratch);
  for (auto& gr : ctx->graphs) {
    if (gr.exec) cudaGraphExecDestroy(gr.exec);
    if (gr.graph) cudaGraphDestroy(gr.graph);
  }
  if (ctx->own) cudaStreamDestroy(ctx->own);
  for (int i = 0; i < crbm_ctx::kSide; ++i) {
    if (ctx->side[i]) cudaStreamDestroy(ctx->side[i]);
    if (ctx->join[i]) cudaEventDestroy(ctx->join[i]);
  }
  if (ctx->fork) cudaEventDestroy(ctx->fork);
  delete ctx;
  return CRBM_OK;
}

const char* crbm_last_error(const crbm_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

// fp16 bit pattern of an integer |v| <= 2048 (exact).
static uint16_t half_of_int(int v) {
  if (v == 0) return 0;
  const uint16_t sgn = v < 0 ? 0x8000u : 0u;
  unsigned a = (unsigned)(v < 0 ? -v : v);
  int e = 0;
  while ((a >> (e + 1)) != 0u) ++e;                    // 2^e <= a < 2^(e+1), e <= 11
  const unsigned man = e <= 10 ? ((a << (10 - e)) & 0x3FFu) : 0u;
  return (uint16_t)(sgn | (unsigned)((e + 15) << 10) | man);
}

// Operand images and error constants of the tensor-core form (Ising, K <= 4,
// k <= 5; crbm_step_tc.cu).  Every weight becomes W ~ qf (c2 2^22 + c1 2^11 + c0)
// with qf = 2^e, |W / qf| <= 2^31, balanced digits c0, c1 in [-1024, 1023]
// and |c2| <= 513, all exact in fp16.  Images (K-major, no swizzle: element
// (row kk, column n) at (kk/8) LBO + (n/8) 128 + (n%8) 16 + (kk%8) 2):
//   hidden / free energy, per kernel row a: K=16 x N=96, LBO 1536, column
//     n = e*32 + f*8 + jj holds digit e (c2, c1, c0) of W[f][a][kk - jj];
//   visible, per (a, K-step j < J = ceil(3K / 2)): K=16 x N=48, LBO 768; row kk
//     is column c = kk % 8 of group G = 2j + kk / 8 of a V buffer (filter
//     f = G / 3, slot s = G % 3: hidden columns 8 (s - 1) + c of the tile's
//     16), column n = e*16 + jj holds digit e of W[f][a][jj + 8 - 8s - c]
//     (zero for f >= K).
static int build_tc(crbm_ctx* ctx, Model& m, int K, int k, const double* W, double v_bias, const double* h_bias,
                    double sh, double sv, double common, bool alloc) {
  double maxw = 0.0, maxhb = 0.0;
  for (int i = 0; i < K * k * k; ++i) maxw = std::fmax(maxw, std::fabs(W[i]));
  for (int f = 0; f < K; ++f) maxhb = std::fmax(maxhb, std::fabs(h_bias[f]));
  const int e0 = (maxw > 0.0 ? (int)std::ceil(std::log2(maxw)) : -60) - 31;
  const double qf = std::ldexp(1.0, e0);
  auto bal = [](long long x, long long& rest) {
    long long r = ((x % 2048) + 2048) % 2048;
    if (r >= 1024) r -= 2048;
    rest = (x - r) / 2048;
    return r;
  };
  std::vector<int> dg((size_t)3 * K * k * k);      // digits e = 0, 1, 2 (c2, c1, c0) of W[f][a][b]
  double t1 = 0.0, t1v = 0.0;
  for (int f = 0; f < K; ++f) {
    double tf = 0.0;
    for (int ab = 0; ab < k * k; ++ab) {
      const size_t idx = (size_t)f * k * k + ab;
      const long long wi = std::llround(W[idx] / qf);
      long long w1, w2;
      const long long c0 = bal(wi, w1), c1 = bal(w1, w2);
      dg[0 * (size_t)K * k * k + idx] = (int)w2;
      dg[1 * (size_t)K * k * k + idx] = (int)c1;
      dg[2 * (size_t)K * k * k + idx] = (int)c0;
      tf += qf * (2048.0 * (double)std::llabs(c1) + (double)std::llabs(c0));   // |q1 c1-sum + q0 c0-sum|
    }
    t1 = std::fmax(t1, tf);
    t1v += tf;
  }
  auto digit = [&](int e, int f, int a, int b) { return dg[((size_t)e * K + f) * k * k + (size_t)a * k + b]; };
  const int J = (3 * K + 1) / 2;
  const size_t bh = (size_t)k * 3072, bytes = bh + (size_t)k * J * 1536;
  std::vector<uint16_t> img(bytes / 2, 0);
  for (int a = 0; a < k; ++a)
    for (int kk = 0; kk < 16; ++kk)
      for (int n = 0; n < 96; ++n) {
        const int e = n / 32, f = (n / 8) % 4, jj = n % 8, b = kk - jj;
        if (f >= K || b < 0 || b >= k) continue;
        const size_t off = (size_t)a * 3072 + (kk / 8) * 1536 + (n / 8) * 128 + (n % 8) * 16 + (kk % 8) * 2;
        img[off / 2] = half_of_int(digit(e, f, a, b));
      }
  for (int a = 0; a < k; ++a)
    for (int j = 0; j < J; ++j) {
      const size_t aj = bh + (size_t)(a * J + j) * 1536;
      for (int kk = 0; kk < 16; ++kk) {
        const int G = 2 * j + kk / 8, f = G / 3, s = G % 3, c = kk % 8;
        if (f >= K) continue;
        for (int n = 0; n < 48; ++n) {
          const int e = n / 16, jj = n % 16, b = jj + 8 - 8 * s - c;
          if (b >= 0 && b < k)
            img[(aj + (kk / 8) * 768 + (n / 8) * 128 + (n % 8) * 16 + (kk % 8) * 2) / 2] = half_of_int(digit(e, f, a, b));
        }
      }
    }
  m.tq2 = (float)std::ldexp(qf, 22);
  m.tq1 = (float)std::ldexp(qf, 11);
  m.tq0 = (float)qf;
  // decisions (decide32 units of 2^-32): x = fl(c2-sum q2 + fl(c1-sum q1 +
  // fl(c0-sum q0 + b32))) (three fused multiply-adds; the products are exact)
  // is within quantisation (k^2 or K k^2) qf / 2, the two inner roundings
  // 2^-24 (|c0 part| + |b|) + 2^-24 (|c1 part| + |c0 part| + |b|) <= 2^-24
  // (2 T1 + 2 |b|) and the outer one 2^-24 |x| (budgeted 2^-23 |x|) of the
  // exact pre-activation, the FP64 path's own sum within 2^-50 S; slope of
  // sigma <= 1/4; factor 2 of safety
  const double u24 = std::ldexp(1.0, -24), u50 = std::ldexp(1.0, -50);
  const double eqh = 0.5 * k * k * qf, eqv = 0.5 * K * k * k * qf;
  m.tc0h = (float)std::ldexp(2.0 * (common + 0.25 * (eqh + 2.0 * u24 * t1 + 2.0 * u24 * maxhb + u50 * sh)) + 1e-14, 32);
  m.tc0v = (float)std::ldexp(
      2.0 * (common + 0.25 * (eqv + 2.0 * u24 * t1v + 2.0 * u24 * std::fabs(v_bias) + u50 * sv)) + 1e-14, 32);
  m.tc1 = (float)std::ldexp(2.0 * (std::ldexp(1.0, -25) + 0.25 * 2.0 * u24), 32);
  // free energy, per unit beyond the 2^-23 |x| the kernel sums: quantisation
  // k^2 qf / 2, the two inner roundings 2^-24 (2 T1 + 2 |hb|) (budgeted
  // 3 2^-24 |hb|); factor 1.5
  m.tcft = (float)(1.5 * (0.5 * k * k * qf + 2.0 * u24 * t1 + 3.0 * u24 * maxhb + u50 * sh));
  if (alloc) CK(cudaMalloc(&m.d_tc, bytes), "cudaMalloc tensor-core images");
  else if (!m.d_tc || m.tc_bytes != bytes) return fail(ctx, CRBM_EINVAL, "tensor-core image size changed");
  m.tc_bytes = bytes;
  CK(cudaMemcpy(m.d_tc, img.data(), bytes, cudaMemcpyHostToDevice), "tensor-core image copy");
  return CRBM_OK;
}

// Host tables and error constants of a model from its parameters, copied to
// the device (into new buffers when alloc, else into the model's own).
static int build_model(crbm_ctx* ctx, Model& m, int kind, int K, int k, const double* W, double v_bias,
                       const double* h_bias, bool alloc) {
  m.kind = kind;
  m.K = K;
  m.k = k;
  m.vb = v_bias;
  m.hb.assign(h_bias, h_bias + K);
  // Row-sum tables: lut[f][a][code] = sum over set bits b of code of W[f][a][b],
  // summed in increasing b (the FP64 order of every pre-activation); the
  // backward table is indexed by the raw window of a hidden row, whose bit
  // k-1-b is the unit seen through tap b.
  const int T = 1 << k;
  const size_t nlut = (size_t)K * k * T;
  if (nlut > 4096) return fail(ctx, CRBM_EINVAL, "K*k*2^k = %zu exceeds 4096 table entries", nlut);
  std::vector<double> fwd(nlut), bwd(nlut);
  for (int f = 0; f < K; ++f)
    for (int a = 0; a < k; ++a)
      for (int c = 0; c < T; ++c) {
        double s = 0.0;
        for (int b = 0; b < k; ++b)
          if ((c >> b) & 1) s += W[((size_t)f * k + a) * k + b];
        fwd[((size_t)f * k + a) * T + c] = s;
      }
  for (int f = 0; f < K; ++f)
    for (int a = 0; a < k; ++a)
      for (int w = 0; w < T; ++w) {
        int rev = 0;
        for (int b = 0; b < k; ++b)
          if ((w >> b) & 1) rev |= 1 << (k - 1 - b);
        bwd[((size_t)f * k + a) * T + w] = fwd[((size_t)f * k + a) * T + rev];
      }
  // S_h, S_v: largest possible |partial sum| of a hidden / visible pre-activation
  double sh = 0.0, sv = std::fabs(v_bias);
  for (int f = 0; f < K; ++f) {
    double sf = std::fabs(h_bias[f]);
    for (int a = 0; a < k; ++a) {
      double mx = 0.0;
      for (int c = 0; c < T; ++c) mx = std::fmax(mx, std::fabs(fwd[((size_t)f * k + a) * T + c]));
      sf += mx;
      sv += mx;
    }
    sh = std::fmax(sh, sf);
  }
  // hi/lo split for the FP32 free energy: hi on a 2^-gbits grid such that every
  // partial sum of hi terms is exact in FP32; lo = the FP32-rounded remainder.
  const int gbits = 23 - (int)std::ceil(std::log2(std::fmax(sh, sv) + 1.0));
  auto split = [&](double x, float& hi, float& lo) {
    const double h = std::ldexp(std::nearbyint(std::ldexp(x, gbits)), -gbits);
    hi = (float)h;
    lo = (float)(x - h);
  };
  std::vector<float> t32(4 * nlut);
  for (size_t i = 0; i < nlut; ++i) {
    t32[i] = (float)fwd[i];
    t32[nlut + i] = (float)bwd[i];
    split(fwd[i], t32[2 * nlut + i], t32[3 * nlut + i]);
  }
  for (int f = 0; f < K; ++f) {
    m.hb32[f] = (float)h_bias[f];
    split(h_bias[f], m.hb_hi[f], m.hb_lo[f]);
  }
  m.vb32 = (float)v_bias;
  // Certified FP32 error constants.  Assumed bounds of the special-function
  // approximations (checked exhaustively on the device by the test-suite):
  // ex2 relative 2^-22, rcp relative 2^-23, lg2 absolute 2^-22 on [1, 2].
  const double u24 = std::ldexp(1.0, -24), ex2 = std::ldexp(1.0, -22), rcp = std::ldexp(1.0, -23),
               lg2 = std::ldexp(1.0, -22);
  // decisions: |p32 - p64| <= 0.25 ex2 + 2^-24 + rcp + |u32 - u| + 0.25 dx + 2^-25 |x|,
  // dx <= (terms + 1) 2^-24 S; factor 2 of safety
  const double common = 0.25 * ex2 + u24 + rcp + std::ldexp(1.0, -25) + std::ldexp(1.0, -33);
  // (decide32 compares in units of 2^-32: the constants are scaled by 2^32)
  m.c0h = (float)std::ldexp(2.0 * (common + 0.25 * (k + 1) * u24 * sh) + 1e-14, 32);
  m.c0v = (float)std::ldexp(2.0 * (common + 0.25 * ((double)K * k + 1) * u24 * sv) + 1e-14, 32);
  m.c1 = (float)std::ldexp(2.0 * std::ldexp(1.0, -25), 32);
  // free energy, per softplus term: 0.5 ex2 + 2^-24 (1 + e) + ln2 lg2 + 2^-23 ln2
  // (ln 2 product) + error of the FP32 sum of k + 1 lo terms; factor 1.5 of safety
  const double lo1 = std::ldexp(1.0, -(gbits + 1));
  const double elo = (k + 2) * u24 * (k + 1) * lo1;
  m.csp = (float)(1.5 * (0.5 * ex2 + u24 + 0.69314718055994531 * lg2 + 0.7 * std::ldexp(1.0, -23)) + elo);
  // the second-level (df64) free energy's pre-activation: hi sums exact, the
  // lo entries rounded (2^-24 lo1 each) and summed in FP32, against the FP64
  // path's sum of k + 1 terms (its own rounding (k + 1) 2^-52 S); factor 2
  m.cdf = (float)(2.0 * (elo + (k + 1) * u24 * lo1 + (k + 1) * std::ldexp(1.0, -52) * std::fmax(sh, sv)));
  // filter-interleaved copies (entry (a*T + code)*4 + f), zero for f >= K
  const size_t nq = (size_t)k * T;
  std::vector<float> q4(3 * nq * 4, 0.0f);
  if (K <= 4) {
    for (int f = 0; f < K; ++f)
      for (size_t e = 0; e < nq; ++e) {
        const size_t src = (size_t)f * nq + e;
        q4[(0 * nq + e) * 4 + f] = t32[src];
        q4[(1 * nq + e) * 4 + f] = t32[2 * nlut + src];
        q4[(2 * nq + e) * 4 + f] = t32[3 * nlut + src];
      }
  }
  m.nlut = nlut;
  m.nq = nq;
  if (kind == kIsing && K <= 4 && k <= 5) {
    const int rc = build_tc(ctx, m, K, k, W, v_bias, h_bias, sh, sv, common, alloc);
    if (rc) return rc;
  }
  if (alloc) CK(cudaMalloc(&m.d_q, 3 * nq * sizeof(float4)), "cudaMalloc tables");
  CK(cudaMemcpy(m.d_q, q4.data(), 3 * nq * sizeof(float4), cudaMemcpyHostToDevice), "table copy");
  if (alloc) {
    CK(cudaMalloc(&m.d_f64, 2 * nlut * sizeof(double)), "cudaMalloc tables");
    CK(cudaMalloc(&m.d_f32, 4 * nlut * sizeof(float)), "cudaMalloc tables");
  }
  CK(cudaMemcpy(m.d_f64, fwd.data(), nlut * sizeof(double), cudaMemcpyHostToDevice), "table copy");
  CK(cudaMemcpy(m.d_f64 + nlut, bwd.data(), nlut * sizeof(double), cudaMemcpyHostToDevice), "table copy");
  CK(cudaMemcpy(m.d_f32, t32.data(), 4 * nlut * sizeof(float), cudaMemcpyHostToDevice), "table copy");
  return CRBM_OK;
}

int crbm_load_model(crbm_ctx* ctx, int kind, int K, int k, const double* W, double v_bias,
                    const double* h_bias, int* model_id) {
  if (!ctx) return CRBM_EINVAL;
  if (kind != kIsing && kind != kKitaev) return fail(ctx, CRBM_EINVAL, "unknown model kind %d", kind);
  if (K < 1 || K > kMaxK) return fail(ctx, CRBM_EINVAL, "K=%d outside [1,%d]", K, kMaxK);
  if (k < 1 || k > kMaxk) return fail(ctx, CRBM_EINVAL, "k=%d outside [1,%d]", k, kMaxk);
  if (!W || !h_bias || !model_id) return fail(ctx, CRBM_EINVAL, "null pointer");
  for (int i = 0; i < K * k * k; ++i)
    if (!std::isfinite(W[i])) return fail(ctx, CRBM_EINVAL, "non-finite weight");
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  Model m;
  const int rc = build_model(ctx, m, kind, K, k, W, v_bias, h_bias, true);
  if (rc) return rc;
  m.live = true;
  ctx->models.push_back(m);
  *model_id = (int)ctx->models.size() - 1;
  return CRBM_OK;
}

int crbm_load_lcrbm(crbm_ctx* ctx, int kind, int K, int k, int edge, const double* W, double v_bias,
                    const double* h_bias, int* model_id) {
  if (!ctx) return CRBM_EINVAL;
  if (kind != kKitaev) return fail(ctx, CRBM_EINVAL, "the LCRBM serves the open-boundary Kitaev model only");
  if (K < 1 || K > kMaxK) return fail(ctx, CRBM_EINVAL, "K=%d outside [1,%d]", K, kMaxK);
  if (k < 1 || k > kMaxk) return fail(ctx, CRBM_EINVAL, "k=%d outside [1,%d]", k, kMaxk);
  if (edge < 1 || edge > 6) return fail(ctx, CRBM_EINVAL, "edge=%d outside [1,6]", edge);
  if (!W || !h_bias || !model_id) return fail(ctx, CRBM_EINVAL, "null pointer");
  const int ncls = 2 * edge + 1, T = 1 << k;
  const size_t per = (size_t)K * k * T, nlut = (size_t)ncls * per;
  if (nlut > 4096)
    return fail(ctx, CRBM_EINVAL, "(2 edge + 1) K k 2^k = %zu exceeds 4096 table entries", nlut);
  for (int i = 0; i < ncls * K * k * k; ++i)
    if (!std::isfinite(W[i])) return fail(ctx, CRBM_EINVAL, "non-finite weight");
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  // per class c the tables of the periodic CRBM: fwd[((c K + f) k + a) 2^k + code]
  // sums W[c][f][a][b] over the set bits b of code in increasing b; bwd is
  // indexed by the raw (reversed) window
  std::vector<double> fwd(nlut), bwd(nlut);
  for (int c = 0; c < ncls; ++c)
    for (int f = 0; f < K; ++f)
      for (int a = 0; a < k; ++a)
        for (int code = 0; code < T; ++code) {
          double acc = 0.0;
          for (int b = 0; b < k; ++b)
            if ((code >> b) & 1) acc += W[(((size_t)c * K + f) * k + a) * k + b];
          fwd[(((size_t)c * K + f) * k + a) * T + code] = acc;
        }
  for (size_t e = 0; e < nlut; ++e) {
    const int w = (int)(e % T);
    int rev = 0;
    for (int b = 0; b < k; ++b)
      if ((w >> b) & 1) rev |= 1 << (k - 1 - b);
    bwd[e] = fwd[e - w + rev];
  }
  Model m;
  m.kind = kind;
  m.K = K;
  m.k = k;
  m.edge = edge;
  m.ncls = ncls;
  m.vb = v_bias;
  m.hb.assign(h_bias, h_bias + K);
  m.nlut = nlut;
  CK(cudaMalloc(&m.d_f64, 2 * nlut * sizeof(double)), "cudaMalloc tables");
  CK(cudaMemcpy(m.d_f64, fwd.data(), nlut * sizeof(double), cudaMemcpyHostToDevice), "table copy");
  CK(cudaMemcpy(m.d_f64 + nlut, bwd.data(), nlut * sizeof(double), cudaMemcpyHostToDevice), "table copy");
  m.live = true;
  ctx->models.push_back(m);
  *model_id = (int)ctx->models.size() - 1;
  return CRBM_OK;
}

int crbm_update_model(crbm_ctx* ctx, int model_id, const double* W, double v_bias, const double* h_bias) {
  if (!ctx) return CRBM_EINVAL;
  if (model_id < 0 || model_id >= (int)ctx->models.size() || !ctx->models[model_id].live)
    return fail(ctx, CRBM_EINVAL, "bad model id %d", model_id);
  Model& m = ctx->models[model_id];
  if (m.edge) return fail(ctx, CRBM_EINVAL, "model %d is an LCRBM: load a new one instead", model_id);
  if (!W || !h_bias) return fail(ctx, CRBM_EINVAL, "null pointer");
  for (int i = 0; i < m.K * m.k * m.k; ++i)
    if (!std::isfinite(W[i])) return fail(ctx, CRBM_EINVAL, "non-finite weight");
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  // the tables are read by every launch of the model's jobs: wait until none runs
  CK(cudaDeviceSynchronize(), "device synchronize");
  const int rc = build_model(ctx, m, m.kind, m.K, m.k, W, v_bias, h_bias, false);
  if (rc) return rc;
  for (auto& j : ctx->jobs)
    if (j.live && j.model == model_id) j.exact = j.fexact = false;
  return CRBM_OK;
}

size_t crbm_job_bytes(int kind, int L, int n_chains, int precision) {
  if (!valid_L(kind, L) || n_chains < 0 || (precision != CRBM_FP64 && precision != CRBM_MIXED)) return 0;
  return make_layout(kind, L, n_chains).total;
}

// F (in `prec`), log pi, E and observables (FP64) of a job's current lattices.
static int evaluate(crbm_ctx* ctx, int id, int prec = kFP64) {
  int rc = launch_jobs(ctx, {id}, 0, 1, 1, prec, 1, ctx->own);
  if (rc) return rc;
  CK(cudaStreamSynchronize(ctx->own), "evaluate");
  ctx->jobs[id].exact = true;
  ctx->jobs[id].fexact = (prec == kFP64);
  ctx->jobs[id].f64vals = (prec == kFP64);
  return CRBM_OK;
}

int crbm_init_chains(crbm_ctx* ctx, int model_id, int L, int n_chains, const double* T,
                     const double* J, uint64_t seed, uint64_t chain_id_base, int init,
                     const uint32_t* init_bits, void* dev_mem, size_t dev_bytes, int* job_id) {
  if (!ctx) return CRBM_EINVAL;
  if (!job_id) return fail(ctx, CRBM_EINVAL, "null job_id");
  if (model_id < 0 || model_id >= (int)ctx->models.size() || !ctx->models[model_id].live)
    return fail(ctx, CRBM_EINVAL, "bad model id %d", model_id);
  const Model& m = ctx->models[model_id];
  if (!valid_L(m.kind, L)) return fail(ctx, CRBM_EINVAL, "lattice side L=%d not supported", L);
  if (m.k > L) return fail(ctx, CRBM_EINVAL, "kernel side k=%d exceeds L=%d", m.k, L);
  if (m.edge && L < 2 * m.edge)
    return fail(ctx, CRBM_EINVAL, "L=%d has fewer than the 2 x %d edge columns of the LCRBM", L, m.edge);
  if (n_chains < 0) return fail(ctx, CRBM_EINVAL, "n_chains < 0");
  if (chain_id_base + (uint64_t)n_chains > (1ull << 32)) return fail(ctx, CRBM_EINVAL, "chain ids must stay below 2^32");
  if (n_chains > 0 && (!T || !J)) return fail(ctx, CRBM_EINVAL, "null T or J");
  if (init != 0 && init != 1) return fail(ctx, CRBM_EINVAL, "init must be 0 or 1");
  if (init == 1 && n_chains > 0 && !init_bits) return fail(ctx, CRBM_EINVAL, "null init_bits");
  for (int c = 0; c < n_chains; ++c)
    if (!(T[c] > 0.0) || !std::isfinite(T[c])) return fail(ctx, CRBM_EINVAL, "temperature of chain %d not > 0", c);
  const Layout lay = make_layout(m.kind, L, n_chains);
  if (n_chains > 0 && (!dev_mem || dev_bytes < lay.total))
    return fail(ctx, CRBM_ENOMEM, "dev_mem holds %zu bytes, job needs %zu", dev_bytes, lay.total);
  if (((uintptr_t)dev_mem & 255) != 0) return fail(ctx, CRBM_EINVAL, "dev_mem must be 256-byte aligned");
  if (ctx->budget && ctx->used + lay.total > ctx->budget)
    return fail(ctx, CRBM_ENOMEM, "job of %zu bytes exceeds the HBM budget (%zu of %zu used)", lay.total,
                ctx->used, ctx->budget);
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  Job j;
  j.live = true;
  j.model = model_id;
  j.kind = m.kind;
  j.L = L;
  j.N = L * L;
  j.Wd = (j.N + 31) / 32;
  j.n = n_chains;
  j.nc = chains_per_tile(m.kind, L);
  if (m.kind == kKitaev) j.tpc = kitaev_group_threads(j.N);
  {
    // crbm_tune's choice: chains per CTA (Ising) or the group size (Kitaev)
    const auto it = ctx->tuned.find(std::make_tuple(m.kind, L, m.K, m.k));
    if (it != ctx->tuned.end()) (m.kind == kKitaev ? j.tpc : j.nc) = it->second;
  }
  j.tiles = (n_chains + j.nc - 1) / j.nc;
  if (m.kind == kIsing) {
    j.J[0] = n_chains > 0 ? J[0] : 1.0;
  } else if (n_chains > 0) {
    for (int i = 0; i < 3; ++i) j.J[i] = J[i];
  }
  j.seed = seed;
  j.cid_base = chain_id_base;
  j.step = 0;
  j.mem = (unsigned char*)dev_mem;
  j.bytes = lay.total;
  j.lay = lay;
  j.stream = nullptr;
  if (n_chains > 0) j.T.assign(T, T + n_chains);
  if (n_chains > 0) {
    unsigned char* b = j.mem;
    cudaStream_t o = ctx->own;
    CK(cudaMemcpyAsync(b + lay.T, T, (size_t)n_chains * 8, cudaMemcpyHostToDevice, o), "copy T");
    if (init == 1)
      CK(cudaMemcpyAsync(b + lay.bits, init_bits, (size_t)n_chains * j.Wd * 4, cudaMemcpyHostToDevice, o),
         "copy init_bits");
    else
      CK(launch_random_init((uint32_t*)(b + lay.bits), n_chains, j.N, j.Wd, seed, chain_id_base, o),
         "random init");
    CK(cudaMemsetAsync(b + lay.os, 0, (size_t)n_chains * 8 * kNobs, o), "zero sums");
    CK(cudaMemsetAsync(b + lay.acc, 0, (size_t)n_chains * 8, o), "zero accepts");
    CK(cudaMemsetAsync(b + lay.rec, 0, (size_t)n_chains * 16, o), "zero recomputes");
    CK(cudaMemsetAsync(b + lay.step, 0, 8, o), "zero step");
    CK(cudaMemsetAsync(b + lay.sched, 0, 16, o), "zero work queue");
  }
  ctx->jobs.push_back(j);
  const int id = (int)ctx->jobs.size() - 1;
  if (n_chains > 0) {
    const int rc = evaluate(ctx, id);
    if (rc) {
      ctx->jobs[id].live = false;
      return rc;
    }
  }
  ctx->used += lay.total;
  *job_id = id;
  return CRBM_OK;
}

static int check_run_args(crbm_ctx* ctx, int64_t S, int g, int correct, int precision) {
  if (S < 0) return fail(ctx, CRBM_EINVAL, "S < 0");
  if (g < 1 || g > 64) return fail(ctx, CRBM_EINVAL, "g=%d outside [1,64]", g);
  if (correct != 0 && correct != 1) return fail(ctx, CRBM_EINVAL, "correct must be 0 or 1");
  if (precision != CRBM_FP64 && precision != CRBM_MIXED) return fail(ctx, CRBM_EINVAL, "bad precision");
  return CRBM_OK;
}

static int check_batch(crbm_ctx* ctx, int n_jobs, const int* job_ids, uint64_t total_steps,
                       std::vector<int>& ids) {
  if (n_jobs < 1 || n_jobs > kMaxJobs || !job_ids) return fail(ctx, CRBM_EINVAL, "n_jobs=%d outside [1,%d]", n_jobs, kMaxJobs);
  int kind = -1, Kb = 0, kb = 0;
  for (int i = 0; i < n_jobs; ++i) {
    Job* j = get_job(ctx, job_ids[i]);
    if (!j) return fail(ctx, CRBM_EINVAL, "bad job id %d", job_ids[i]);
    for (int x : ids)
      if (x == job_ids[i]) return fail(ctx, CRBM_EINVAL, "job %d listed twice", x);
    if (kind >= 0 && j->kind != kind) return fail(ctx, CRBM_EINVAL, "jobs of different model kinds in one batch");
    const Model& mj = ctx->models[j->model];
    if (kind >= 0 && (mj.K != Kb || mj.k != kb))
      return fail(ctx, CRBM_EINVAL, "jobs of one batch must share the filter-bank shape (K, k)");
    kind = j->kind;
    Kb = mj.K;
    kb = mj.k;
    if (j->step + total_steps > (1ull << 32)) return fail(ctx, CRBM_EINVAL, "step counter would pass 2^32");
    ids.push_back(job_ids[i]);
  }
  return CRBM_OK;
}

// Enqueue S proposals of the jobs on st, in launches of at most 2^20 proposals.
static int enqueue_runs(crbm_ctx* ctx, const std::vector<int>& ids, int64_t S, int g, int correct, int precision,
                        cudaStream_t st) {
  int64_t left = S;
  while (left > 0) {
    const int chunk = (int)(left < (1 << 20) ? left : (1 << 20));
    const int rc = launch_jobs(ctx, ids, chunk, g, correct, precision, 0, st);
    if (rc) return rc;
    left -= chunk;
  }
  return CRBM_OK;
}

int crbm_run_batch(crbm_ctx* ctx, int n_jobs, const int* job_ids, int64_t S, int g, int correct,
                   int precision, void* cuda_stream) {
  if (!ctx) return CRBM_EINVAL;
  int rc = check_run_args(ctx, S, g, correct, precision);
  if (rc) return rc;
  std::vector<int> ids;
  if ((rc = check_batch(ctx, n_jobs, job_ids, (uint64_t)S, ids))) return rc;
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if ((rc = enqueue_runs(ctx, ids, S, g, correct, precision, st))) return rc;
  for (int id : ids) {
    ctx->jobs[id].step += (uint64_t)S;
    ctx->jobs[id].stream = st;
    if (S > 0) {
      ctx->jobs[id].exact = false;
      ctx->jobs[id].fexact = ctx->jobs[id].f64vals = (precision == kFP64);
    }
  }
  return CRBM_OK;
}

int crbm_graph_create(crbm_ctx* ctx, int n_jobs, const int* job_ids, int64_t S, int g, int correct, int precision,
                      int repeats, int* graph_id) {
  if (!ctx) return CRBM_EINVAL;
  if (!graph_id) return fail(ctx, CRBM_EINVAL, "null graph_id");
  if (repeats < 1) return fail(ctx, CRBM_EINVAL, "repeats must be >= 1");
  int rc = check_run_args(ctx, S, g, correct, precision);
  if (rc) return rc;
  std::vector<int> ids;
  if ((rc = check_batch(ctx, n_jobs, job_ids, 0, ids))) return rc;
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  // the graph reads and advances the jobs' device step counters: make sure
  // earlier work on the jobs' streams has finished before capturing
  for (int id : ids) CK(cudaStreamSynchronize(ctx->jobs[id].stream), "stream sync");
  crbm_ctx::Graph gr;
  CK(cudaStreamBeginCapture(ctx->own, cudaStreamCaptureModeThreadLocal), "begin capture");
  for (int r = 0; r < repeats && rc == CRBM_OK; ++r) rc = enqueue_runs(ctx, ids, S, g, correct, precision, ctx->own);
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(ctx->own, &graph);
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(ctx, e, "end capture");
  cudaGraphExec_t exec = nullptr;
  const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
  if (ei != cudaSuccess) {
    cudaGraphDestroy(graph);
    return cuda_fail(ctx, ei, "graph instantiate");
  }
  gr.live = true;
  gr.graph = graph;
  gr.exec = exec;
  gr.jobs = ids;
  gr.steps = (uint64_t)S * (uint64_t)repeats;
  gr.precision = precision;
  ctx->graphs.push_back(gr);
  *graph_id = (int)ctx->graphs.size() - 1;
  return CRBM_OK;
}

int crbm_graph_launch(crbm_ctx* ctx, int graph_id, void* cuda_stream) {
  if (!ctx) return CRBM_EINVAL;
  if (graph_id < 0 || graph_id >= (int)ctx->graphs.size() || !ctx->graphs[graph_id].live)
    return fail(ctx, CRBM_EINVAL, "bad graph id %d", graph_id);
  crbm_ctx::Graph& gr = ctx->graphs[graph_id];
  for (int id : gr.jobs)
    if (ctx->jobs[id].step + gr.steps > (1ull << 32)) return fail(ctx, CRBM_EINVAL, "step counter would pass 2^32");
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  CK(cudaGraphLaunch(gr.exec, st), "graph launch");
  for (int id : gr.jobs) {
    ctx->jobs[id].step += gr.steps;
    ctx->jobs[id].stream = st;
    if (gr.steps > 0) {
      ctx->jobs[id].exact = false;
      ctx->jobs[id].fexact = ctx->jobs[id].f64vals = (gr.precision == kFP64);
    }
  }
  return CRBM_OK;
}

int crbm_graph_destroy(crbm_ctx* ctx, int graph_id) {
  if (!ctx) return CRBM_EINVAL;
  if (graph_id < 0 || graph_id >= (int)ctx->graphs.size() || !ctx->graphs[graph_id].live)
    return fail(ctx, CRBM_EINVAL, "bad graph id %d", graph_id);
  crbm_ctx::Graph& gr = ctx->graphs[graph_id];
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  for (int id : gr.jobs) CK(cudaStreamSynchronize(ctx->jobs[id].stream), "stream sync");
  cudaGraphExecDestroy(gr.exec);
  cudaGraphDestroy(gr.graph);
  gr = crbm_ctx::Graph();
  return CRBM_OK;
}

int crbm_pt_run(crbm_ctx* ctx, int phys_job, int rbm_job, int64_t cycles, int g, int precision,
                void* cuda_stream) {
  if (!ctx) return CRBM_EINVAL;
  int rc = check_run_args(ctx, cycles, g, 0, precision);
  if (rc) return rc;
  Job* x = get_job(ctx, phys_job);
  Job* y = get_job(ctx, rbm_job);
  if (!x || !y) return fail(ctx, CRBM_EINVAL, "bad job id");
  if (x == y) return fail(ctx, CRBM_EINVAL, "the physical and the RBM job must differ");
  if (x->model != y->model) return fail(ctx, CRBM_EINVAL, "both jobs must use the same model");
  if (x->L != y->L || x->n != y->n) return fail(ctx, CRBM_EINVAL, "both jobs need the same L and number of chains");
  for (int i = 0; i < 3; ++i)
    if (x->J[i] != y->J[i]) return fail(ctx, CRBM_EINVAL, "both jobs need the same couplings J");
  if (x->T != y->T) return fail(ctx, CRBM_EINVAL, "both jobs need the same temperatures, chain by chain");
  for (const Job* j : {x, y})
    if (j->step + (uint64_t)cycles > (1ull << 32)) return fail(ctx, CRBM_EINVAL, "step counter would pass 2^32");
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  if (cycles == 0 || x->n == 0) return CRBM_OK;
  // the exchanges need FP64 log pi (and Kitaev spectra) of the physical chains,
  // and in CRBM_FP64 also FP64 F (the mixed path carries F's certified bound)
  if (!x->exact || (precision == kFP64 && !x->fexact)) {
    if ((rc = crbm_sync(ctx, phys_job))) return rc;
    if ((rc = evaluate(ctx, phys_job))) return rc;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const JobDev xd = make_jobdev(ctx, *x);
  for (int64_t c = 0; c < cycles; ++c) {
    // RBM proposals and their swaps with the physical chains, then the
    // temperature exchanges, observables and the cycle counter
    if ((rc = launch_jobs(ctx, {rbm_job}, 1, g, 0, precision, 2, st, x))) return rc;
    CK(launch_pt_exchange(xd, 0, true, st), "exchange launch");
  }
  for (Job* j : {x, y}) {
    j->step += (uint64_t)cycles;
    j->stream = st;
    j->exact = true;
    j->fexact = j->fexact && precision == kFP64;
    j->f64vals = j->fexact;
  }
  return CRBM_OK;
}

int crbm_local_run(crbm_ctx* ctx, int job_id, int64_t sweeps, int exchange, int precision, void* cuda_stream) {
  if (!ctx) return CRBM_EINVAL;
  int rc = check_run_args(ctx, sweeps, 1, 1, precision);
  if (rc) return rc;
  if (exchange != 0 && exchange != 1) return fail(ctx, CRBM_EINVAL, "exchange must be 0 or 1");
  Job* j = get_job(ctx, job_id);
  if (!j) return fail(ctx, CRBM_EINVAL, "bad job id %d", job_id);
  if (j->kind == kIsing && j->L % 2) return fail(ctx, CRBM_EINVAL, "checkerboard sweeps need an even L (L=%d)", j->L);
  if (j->step + (uint64_t)sweeps > (1ull << 32)) return fail(ctx, CRBM_EINVAL, "step counter would pass 2^32");
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  if (sweeps == 0 || j->n == 0) return CRBM_OK;
  // the temperature exchange needs FP64 log pi (and Kitaev spectra) of every chain
  if (exchange && !j->exact) {
    if ((rc = crbm_sync(ctx, job_id))) return rc;
    if ((rc = evaluate(ctx, job_id))) return rc;
  }
  // Ising sweeps have no precision choice (integer counts, FP64 thresholds);
  // with the exchange the Kitaev spectra must come from the FP64 stage
  const int prec = (j->kind == kIsing || exchange) ? (int)kFP64 : precision;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (!exchange) {
    int64_t left = sweeps;
    while (left > 0) {
      const int chunk = (int)(left < (1 << 20) ? left : (1 << 20));
      if ((rc = launch_jobs(ctx, {job_id}, chunk, 1, 1, prec, 3, st))) return rc;
      left -= chunk;
    }
  } else {
    const JobDev xd = make_jobdev(ctx, *j);
    for (int64_t c = 0; c < sweeps; ++c) {
      if ((rc = launch_jobs(ctx, {job_id}, 1, 1, 0, prec, 3, st))) return rc;
      CK(launch_pt_exchange(xd, -1, false, st), "exchange launch");
    }
  }
  j->step += (uint64_t)sweeps;
  j->stream = st;
  j->exact = (prec == kFP64);
  j->fexact = true;       // each launch ends with the FP64 free energy
  j->f64vals = j->exact || j->kind == kIsing;
  return CRBM_OK;
}

int crbm_set_trace(crbm_ctx* ctx, int job_id, double* dev_trace, int64_t capacity_steps) {
  Job* j = get_job(ctx, job_id);
  if (!j) return ctx ? fail(ctx, CRBM_EINVAL, "bad job id %d", job_id) : CRBM_EINVAL;
  if (dev_trace && capacity_steps < 1) return fail(ctx, CRBM_EINVAL, "capacity_steps must be >= 1");
  if (((uintptr_t)dev_trace & 7) != 0) return fail(ctx, CRBM_EINVAL, "dev_trace must be 8-byte aligned");
  j->trace = dev_trace;
  j->trace_base = j->step;
  j->trace_cap = dev_trace ? capacity_steps : 0;
  return CRBM_OK;
}

int crbm_autocorr(crbm_ctx* ctx, const double* dev_series, int n_series, int64_t length, double c,
                  double* tau, int64_t* window, void* cuda_stream) {
  if (!ctx) return CRBM_EINVAL;
  if (n_series < 0 || length < 0) return fail(ctx, CRBM_EINVAL, "negative size");
  if (!(c > 0.0)) return fail(ctx, CRBM_EINVAL, "window constant c must be > 0");
  if (n_series == 0) return CRBM_OK;
  if (!dev_series || !tau || !window) return fail(ctx, CRBM_EINVAL, "null pointer");
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  double* d_tau = nullptr;
  long long* d_w = nullptr;
  CK(cudaMallocAsync(&d_tau, (size_t)n_series * 8, st), "cudaMallocAsync");
  CK(cudaMallocAsync(&d_w, (size_t)n_series * 8, st), "cudaMallocAsync");
  cudaError_t e = launch_tau(dev_series, n_series, (long long)length, c, d_tau, d_w, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(tau, d_tau, (size_t)n_series * 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(window, d_w, (size_t)n_series * 8, cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(d_tau, st);
  cudaFreeAsync(d_w, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "autocorrelation");
  return CRBM_OK;
}

// For callers that must not allocate device memory during the call (for
// instance a serving loop that has handed its whole HBM budget to jobs, where
// an allocation could fail or force the allocator to trim): the results pass
// through a fixed 256 KiB device array instead of stream-ordered buffers.
int crbm_autocorr_noalloc(crbm_ctx* ctx, const double* dev_series, int n_series, int64_t length, double c,
                          double* tau, int64_t* window, void* cuda_stream) {
  if (!ctx) return CRBM_EINVAL;
  if (n_series < 0 || length < 0) return fail(ctx, CRBM_EINVAL, "negative size");
  if (n_series > CRBM_AUTOCORR_NOALLOC_MAX_SERIES)
    return fail(ctx, CRBM_EINVAL, "n_series=%d exceeds the no-allocation limit %d", n_series,
                CRBM_AUTOCORR_NOALLOC_MAX_SERIES);
  if (!(c > 0.0)) return fail(ctx, CRBM_EINVAL, "window constant c must be > 0");
  if (n_series == 0) return CRBM_OK;
  if (!dev_series || !tau || !window) return fail(ctx, CRBM_EINVAL, "null pointer");
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  CK(launch_tau_noalloc(dev_series, n_series, (long long)length, c, tau, window, (cudaStream_t)cuda_stream),
     "autocorrelation (no allocation)");
  return CRBM_OK;
}

int crbm_train_epochs(crbm_ctx* ctx, int n_problems, const crbm_train_problem* problems, int batch, double lr,
                      double b1, double b2, double eps, void* cuda_stream) {
  if (!ctx) return CRBM_EINVAL;
  if (n_problems < 0 || (n_problems > 0 && !problems)) return fail(ctx, CRBM_EINVAL, "bad problem list");
  if (batch < 1 || batch > 64) return fail(ctx, CRBM_EINVAL, "batch=%d outside [1,64]", batch);
  if (!(lr >= 0.0) || !(b1 >= 0.0 && b1 < 1.0) || !(b2 >= 0.0 && b2 < 1.0) || !(eps > 0.0))
    return fail(ctx, CRBM_EINVAL, "bad ADAM hyper-parameters");
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
  for (int i = 0; i < n_problems; ++i) {
    const crbm_train_problem& q = problems[i];
    if (q.L < 2 || q.L > 32) return fail(ctx, CRBM_EINVAL, "problem %d: L=%d outside [2,32]", i, q.L);
    if (q.K < 1 || q.K > kMaxK || q.k < 1 || q.k > kMaxk || q.k > q.L)
      return fail(ctx, CRBM_EINVAL, "problem %d: filter shape (%d,%d) out of range", i, q.K, q.k);
    if (q.n_samples < 0) return fail(ctx, CRBM_EINVAL, "problem %d: n_samples < 0", i);
    if (!q.theta || !q.adam_m || !q.adam_v || !q.adam_t || (q.n_samples > 0 && (!q.samples || !q.targets || !q.order)))
      return fail(ctx, CRBM_EINVAL, "problem %d: null pointer", i);
    if (train_smem_bytes(q, batch) > (size_t)optin)
      return fail(ctx, CRBM_EINVAL, "problem %d needs %zu bytes of shared memory", i, train_smem_bytes(q, batch));
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  for (int i0 = 0; i0 < n_problems; i0 += CRBM_TRAIN_MAX_PROBLEMS) {
    const int n = n_problems - i0 < CRBM_TRAIN_MAX_PROBLEMS ? n_problems - i0 : CRBM_TRAIN_MAX_PROBLEMS;
    CK(launch_train(problems + i0, n, batch, lr, b1, b2, eps, st), "trainer launch");
  }
  return CRBM_OK;
}


int crbm_probe_peaks(crbm_ctx* ctx, double* fp32_tflops, double* fp64_tflops) {
  if (!ctx) return CRBM_EINVAL;
  if (!fp32_tflops || !fp64_tflops) return fail(ctx, CRBM_EINVAL, "null pointer");
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  CK(probe_fma_peaks(ctx->device, fp32_tflops, fp64_tflops, ctx->own), "peak probe");
  return CRBM_OK;
}

int crbm_set_wait_limit(crbm_ctx* ctx, int64_t cycles) {
  if (!ctx) return CRBM_EINVAL;
  if (cycles < 1000 || cycles > (1ll << 40)) return fail(ctx, CRBM_EINVAL, "wait limit %lld outside [1000, 2^40]",
                                                         (long long)cycles);
  ctx->wait_limit = (long long)cycles;
  return CRBM_OK;
}

int crbm_probe_wait(crbm_ctx* ctx, int64_t limit_cycles, int arrive, void* cuda_stream) {
  if (!ctx) return CRBM_EINVAL;
  if (limit_cycles < 1000 || limit_cycles > (1ll << 40))
    return fail(ctx, CRBM_EINVAL, "limit %lld outside [1000, 2^40]", (long long)limit_cycles);
  if (arrive != 0 && arrive != 1) return fail(ctx, CRBM_EINVAL, "arrive must be 0 or 1");
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  CK(launch_wait_probe((long long)limit_cycles, arrive, ctx->d_err, (cudaStream_t)cuda_stream), "probe launch");
  return CRBM_OK;
}

int crbm_run(crbm_ctx* ctx, int job_id, int64_t S, int g, int correct, int precision, void* cuda_stream) {
  return crbm_run_batch(ctx, 1, &job_id, S, g, correct, precision, cuda_stream);
}

int crbm_tune(crbm_ctx* ctx, int model_id, int L, int precision, int* best_nc, double* best_ms) {
  if (!ctx) return CRBM_EINVAL;
  if (model_id < 0 || model_id >= (int)ctx->models.size() || !ctx->models[model_id].live)
    return fail(ctx, CRBM_EINVAL, "bad model id %d", model_id);
  const Model& m = ctx->models[model_id];
  if (m.edge) return fail(ctx, CRBM_EINVAL, "model %d is an LCRBM: nothing to tune", model_id);
  if (!valid_L(m.kind, L) || m.k > L) return fail(ctx, CRBM_EINVAL, "lattice side L=%d not supported", L);
  if (precision != CRBM_FP64 && precision != CRBM_MIXED) return fail(ctx, CRBM_EINVAL, "bad precision");
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
  const int N = L * L, nblk = (N + 3) / 4;
  std::vector<int> cand;
  if (m.kind == kIsing) {
    for (int nc = 1; nc <= kThreads / 8; nc *= 2)
      if ((nc == 1 || (nc / 2) * nblk < 8 * kThreads) &&
          smem_bytes(m.kind, precision, L, m.K, m.k, nc, m.K == 4 ? 4 : 0) <= 100 * 1024)
        cand.push_back(nc);
  } else {
    // group sizes 256 / nc threads (at least a warp); timed alone, a job runs
    // one chain per CTA of its group size
    for (int nc = 1; nc <= kThreads / 32; nc *= 2) cand.push_back(nc);
  }
  // a temporary job large enough for every candidate to fill the GPU
  const int n_chains = 4 * sms * cand.back();
  const Layout lay = make_layout(m.kind, L, n_chains);
  unsigned char* mem = nullptr;
  CK(cudaMalloc(&mem, lay.total), "cudaMalloc tuning job");
  std::vector<double> T(n_chains, 2.0);
  CK(cudaMemsetAsync(mem, 0, lay.total, ctx->own), "zero tuning job");
  CK(cudaMemcpyAsync(mem + lay.T, T.data(), (size_t)n_chains * 8, cudaMemcpyHostToDevice, ctx->own), "copy T");
  CK(launch_random_init((uint32_t*)(mem + lay.bits), n_chains, N, (N + 31) / 32, 12345, 0, ctx->own), "init");
  Job j;
  j.live = true;
  j.model = model_id;
  j.kind = m.kind;
  j.L = L;
  j.N = N;
  j.Wd = (N + 31) / 32;
  j.n = n_chains;
  j.seed = 12345;
  j.mem = mem;
  j.bytes = lay.total;
  j.lay = lay;
  j.stream = ctx->own;
  ctx->jobs.push_back(j);
  const int id = (int)ctx->jobs.size() - 1;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int best = cand[0], rc = CRBM_OK;
  float best_t = 1e30f;
  for (int nc : cand) {
    Job& jj = ctx->jobs[id];
    if (m.kind == kKitaev) {
      jj.tpc = kThreads / nc;
      jj.nc = 1;
      jj.tiles = n_chains;
    } else {
      jj.nc = nc;
      jj.tiles = (n_chains + nc - 1) / nc;
    }
    if ((rc = launch_jobs(ctx, {id}, 0, 1, 1, kFP64, 1, ctx->own))) break;        // F, log pi of the state
    if ((rc = launch_jobs(ctx, {id}, 2, 1, 1, precision, 0, ctx->own))) break;    // warm-up
    cudaEventRecord(e0, ctx->own);
    if ((rc = launch_jobs(ctx, {id}, 4, 1, 1, precision, 0, ctx->own))) break;
    cudaEventRecord(e1, ctx->own);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= (float)n_chains;       // per chain: candidates run different numbers of CTAs per SM
    if (ms < best_t) {
      best_t = ms;
      best = nc;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(ctx->own);
  ctx->jobs[id].live = false;
  cudaFree(mem);
  if (rc) return rc;
  ctx->tuned[std::make_tuple(m.kind, L, m.K, m.k)] = m.kind == kKitaev ? kThreads / best : best;
  if (best_nc) *best_nc = best;
  if (best_ms) *best_ms = (double)best_t * 1e3 / 4.0;     // microseconds per chain-proposal
  return CRBM_OK;
}

int crbm_set_tensor_cores(crbm_ctx* ctx, int enable) {
  if (!ctx) return CRBM_EINVAL;
  if (enable != 0 && enable != 1) return fail(ctx, CRBM_EINVAL, "enable must be 0 or 1");
  ctx->use_tc = enable == 1;
  return CRBM_OK;
}

int crbm_sync(crbm_ctx* ctx, int job_id) {
  Job* j = get_job(ctx, job_id);
  if (!j) return ctx ? fail(ctx, CRBM_EINVAL, "bad job id %d", job_id) : CRBM_EINVAL;
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  CK(cudaStreamSynchronize(j->stream), "stream sync");
  int h = 0;
  CK(cudaMemcpyAsync(&h, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->own), "read error flag");
  CK(cudaStreamSynchronize(ctx->own), "read error flag");
  if (h == 0) return CRBM_OK;
  // reported once: the flag is cleared so that the context stays usable
  CK(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->own), "clear error flag");
  CK(cudaStreamSynchronize(ctx->own), "clear error flag");
  if (h == kErrTimeout) return fail(ctx, CRBM_ETIMEOUT, "a device-side wait reached its cycle limit");
  return fail(ctx, CRBM_EINVAL, "device reported configuration error %d", h);
}

static int read_back(crbm_ctx* ctx, Job* j, void* dst, size_t off, size_t bytes) {
  if (!dst || bytes == 0) return CRBM_OK;
  CK(cudaMemcpyAsync(dst, j->mem + off, bytes, cudaMemcpyDeviceToHost, ctx->own), "device to host copy");
  CK(cudaStreamSynchronize(ctx->own), "device to host copy");
  return CRBM_OK;
}

int crbm_read_energies(crbm_ctx* ctx, int job_id, double* logpi, double* F_crbm, double* E_phys) {
  Job* j = get_job(ctx, job_id);
  if (!j) return ctx ? fail(ctx, CRBM_EINVAL, "bad job id %d", job_id) : CRBM_EINVAL;
  int rc = crbm_sync(ctx, job_id);
  if (rc) return rc;
  const size_t b = (size_t)j->n * 8;
  if (!j->f64vals && j->n > 0 && (logpi || F_crbm || E_phys)) {
    // the stored values of a mixed run are within their certified bounds of
    // the FP64 ones (the decisions are the FP64 path's either way); the values
    // returned here are the FP64 path's: a copy of the job's memory is
    // evaluated in FP64 (Eq. 13 for F), the job itself is left as it is
    const Job jc = *j;
    if (ctx->scratch_bytes < jc.bytes) {
      if (ctx->scratch) CK(cudaFree(ctx->scratch), "cudaFree");
      ctx->scratch = nullptr;
      ctx->scratch_bytes = 0;
      CK(cudaMalloc(&ctx->scratch, jc.bytes), "cudaMalloc (FP64 read-back copy)");
      ctx->scratch_bytes = jc.bytes;
    }
    CK(cudaMemcpyAsync(ctx->scratch, jc.mem, jc.bytes, cudaMemcpyDeviceToDevice, ctx->own), "copy job memory");
    Job tmp = jc;
    tmp.mem = ctx->scratch;
    tmp.stream = ctx->own;
    tmp.trace = nullptr;
    tmp.trace_cap = 0;
    ctx->jobs.push_back(tmp);
    const int tid = (int)ctx->jobs.size() - 1;
    rc = launch_jobs(ctx, {tid}, 0, 1, 1, kFP64, 1, ctx->own);
    ctx->jobs.pop_back();       // the launch holds its own copy of the job's pointers
    if (rc) return rc;
    for (auto [dst, off] : {std::make_pair(logpi, jc.lay.lp), std::make_pair(F_crbm, jc.lay.F),
                            std::make_pair(E_phys, jc.lay.E)})
      if (dst) CK(cudaMemcpyAsync(dst, ctx->scratch + off, b, cudaMemcpyDeviceToHost, ctx->own), "device to host copy");
    CK(cudaStreamSynchronize(ctx->own), "FP64 re-evaluation");
    return CRBM_OK;
  }
  if ((rc = read_back(ctx, j, logpi, j->lay.lp, b))) return rc;
  if ((rc = read_back(ctx, j, F_crbm, j->lay.F, b))) return rc;
  return read_back(ctx, j, E_phys, j->lay.E, b);
}

int crbm_read_observables(crbm_ctx* ctx, int job_id, double* sums, int64_t* accepts, int64_t* recomputes) {
  Job* j = get_job(ctx, job_id);
  if (!j) return ctx ? fail(ctx, CRBM_EINVAL, "bad job id %d", job_id) : CRBM_EINVAL;
  int rc = crbm_sync(ctx, job_id);
  if (rc) return rc;
  if ((rc = read_back(ctx, j, sums, j->lay.os, (size_t)j->n * 8 * kNobs))) return rc;
  if ((rc = read_back(ctx, j, accepts, j->lay.acc, (size_t)j->n * 8))) return rc;
  return read_back(ctx, j, recomputes, j->lay.rec, (size_t)j->n * 16);
}

int crbm_read_state(crbm_ctx* ctx, int job_id, uint32_t* bits, uint64_t* step) {
  Job* j = get_job(ctx, job_id);
  if (!j) return ctx ? fail(ctx, CRBM_EINVAL, "bad job id %d", job_id) : CRBM_EINVAL;
  int rc = crbm_sync(ctx, job_id);
  if (rc) return rc;
  if (step) *step = j->step;
  return read_back(ctx, j, bits, j->lay.bits, (size_t)j->n * j->Wd * 4);
}

int crbm_read_states(crbm_ctx* ctx, int n_jobs, const int* job_ids, uint32_t* const* bits, uint64_t* steps,
                     double* const* sums) {
  if (!ctx) return CRBM_EINVAL;
  if (n_jobs < 0 || n_jobs > kMaxJobs) return fail(ctx, CRBM_EINVAL, "n_jobs must be 0..%d", kMaxJobs);
  if (n_jobs > 0 && !job_ids) return fail(ctx, CRBM_EINVAL, "null job_ids");
  for (int i = 0; i < n_jobs; ++i)
    if (!get_job(ctx, job_ids[i])) return fail(ctx, CRBM_EINVAL, "bad job id %d", job_ids[i]);
  if (n_jobs == 0) return CRBM_OK;
  // every job's stream, then the error flag once (crbm_sync of the first job
  // reads it after its own stream; the others are synchronised before)
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  for (int i = 1; i < n_jobs; ++i) CK(cudaStreamSynchronize(ctx->jobs[job_ids[i]].stream), "stream sync");
  int rc = crbm_sync(ctx, job_ids[0]);
  if (rc) return rc;
  for (int i = 0; i < n_jobs; ++i) {
    Job& j = ctx->jobs[job_ids[i]];
    if (steps) steps[i] = j.step;
    if (j.n == 0) continue;
    if (bits && bits[i])
      CK(cudaMemcpyAsync(bits[i], j.mem + j.lay.bits, (size_t)j.n * j.Wd * 4, cudaMemcpyDeviceToHost, ctx->own),
         "device to host copy");
    if (sums && sums[i])
      CK(cudaMemcpyAsync(sums[i], j.mem + j.lay.os, (size_t)j.n * 8 * kNobs, cudaMemcpyDeviceToHost, ctx->own),
         "device to host copy");
  }
  CK(cudaStreamSynchronize(ctx->own), "device to host copy");
  return CRBM_OK;
}

int crbm_write_state(crbm_ctx* ctx, int job_id, const uint32_t* bits, uint64_t step, int precision) {
  Job* j = get_job(ctx, job_id);
  if (!j) return ctx ? fail(ctx, CRBM_EINVAL, "bad job id %d", job_id) : CRBM_EINVAL;
  if (!bits && j->n > 0) return fail(ctx, CRBM_EINVAL, "null bits");
  if (step >= (1ull << 32)) return fail(ctx, CRBM_EINVAL, "step must stay below 2^32");
  if (precision != CRBM_FP64 && precision != CRBM_MIXED) return fail(ctx, CRBM_EINVAL, "bad precision");
  int rc = crbm_sync(ctx, job_id);
  if (rc) return rc;
  j->step = step;
  if (j->n == 0) return CRBM_OK;
  CK(cudaMemcpyAsync(j->mem + j->lay.bits, bits, (size_t)j->n * j->Wd * 4, cudaMemcpyHostToDevice, ctx->own),
     "copy bits");
  const unsigned long long st = step;
  CK(cudaMemcpyAsync(j->mem + j->lay.step, &st, 8, cudaMemcpyHostToDevice, ctx->own), "copy step");
  return evaluate(ctx, job_id, precision);
}

int crbm_write_states(crbm_ctx* ctx, int n_jobs, const int* job_ids, const uint32_t* const* bits,
                      const uint64_t* steps, int precision) {
  if (!ctx) return CRBM_EINVAL;
  if (n_jobs < 0 || n_jobs > kMaxJobs) return fail(ctx, CRBM_EINVAL, "n_jobs must be 0..%d", kMaxJobs);
  if (n_jobs > 0 && (!job_ids || !bits || !steps)) return fail(ctx, CRBM_EINVAL, "null job_ids, bits or steps");
  if (precision != CRBM_FP64 && precision != CRBM_MIXED) return fail(ctx, CRBM_EINVAL, "bad precision");
  std::vector<int> ids;
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  for (int i = 0; i < n_jobs; ++i) {
    Job* j = get_job(ctx, job_ids[i]);
    if (!j) return fail(ctx, CRBM_EINVAL, "bad job id %d", job_ids[i]);
    for (int q = 0; q < i; ++q)
      if (job_ids[q] == job_ids[i]) return fail(ctx, CRBM_EINVAL, "job %d listed twice", job_ids[i]);
    if (!bits[i] && j->n > 0) return fail(ctx, CRBM_EINVAL, "null bits for job %d", job_ids[i]);
    if (steps[i] >= (1ull << 32)) return fail(ctx, CRBM_EINVAL, "step must stay below 2^32");
  }
  for (int i = 0; i < n_jobs; ++i) {
    const int rc = crbm_sync(ctx, job_ids[i]);
    if (rc) return rc;
  }
  // the steps stay in host memory until the copies have run (synchronised below)
  std::vector<unsigned long long> st(steps, steps + n_jobs);
  for (int i = 0; i < n_jobs; ++i) {
    Job& j = ctx->jobs[job_ids[i]];
    j.step = steps[i];
    if (j.n == 0) continue;
    CK(cudaMemcpyAsync(j.mem + j.lay.bits, bits[i], (size_t)j.n * j.Wd * 4, cudaMemcpyHostToDevice, ctx->own),
       "copy bits");
    CK(cudaMemcpyAsync(j.mem + j.lay.step, &st[i], 8, cudaMemcpyHostToDevice, ctx->own), "copy step");
    ids.push_back(job_ids[i]);
  }
  if (ids.empty()) return CRBM_OK;
  // one evaluation launch per (model kind, filter shape): the table kernel
  // takes jobs of every side of a shape in one launch
  std::vector<bool> done(ids.size(), false);
  for (size_t a = 0; a < ids.size(); ++a) {
    if (done[a]) continue;
    const Job& ja = ctx->jobs[ids[a]];
    const Model& ma = ctx->models[ja.model];
    std::vector<int> grp;
    for (size_t b = a; b < ids.size(); ++b) {
      const Job& jb = ctx->jobs[ids[b]];
      const Model& mb = ctx->models[jb.model];
      if (!done[b] && jb.kind == ja.kind && mb.K == ma.K && mb.k == ma.k) {
        grp.push_back(ids[b]);
        done[b] = true;
      }
    }
    const int rc = launch_jobs(ctx, grp, 0, 1, 1, precision, 1, ctx->own);
    if (rc) return rc;
  }
  CK(cudaStreamSynchronize(ctx->own), "evaluate");
  for (int id : ids) {
    ctx->jobs[id].exact = true;
    ctx->jobs[id].fexact = (precision == kFP64);
    ctx->jobs[id].f64vals = (precision == kFP64);
  }
  return CRBM_OK;
}

int crbm_release(crbm_ctx* ctx, int job_id) {
  Job* j = get_job(ctx, job_id);
  if (!j) return ctx ? fail(ctx, CRBM_EINVAL, "bad job id %d", job_id) : CRBM_EINVAL;
  for (size_t gi = 0; gi < ctx->graphs.size(); ++gi)
    if (ctx->graphs[gi].live)
      for (int id : ctx->graphs[gi].jobs)
        if (id == job_id) return fail(ctx, CRBM_EBUSY, "job %d is part of live graph %zu", job_id, gi);
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  CK(cudaStreamSynchronize(j->stream), "stream sync");
  ctx->used -= j->bytes;
  j->live = false;
  return CRBM_OK;
}

}  // extern "C"
