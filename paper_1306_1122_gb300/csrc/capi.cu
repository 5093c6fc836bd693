// capi.cu -- the C ABI (include/dbie.h): contexts, validation, staging, and the host drivers of
// evaluation, the on-device lambda search and the adjoint.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "dbie.h"
#include "kernels.h"

using namespace dbie;

#ifndef DBIE_FF_SPLIT_TARGET_PCT
#define DBIE_FF_SPLIT_TARGET_PCT 200   // the same for the float-float re-evaluation pass
#endif
#ifndef DBIE_SPLIT_TARGET_PCT
#define DBIE_SPLIT_TARGET_PCT 200
#endif

namespace {

thread_local std::string g_err;

dbie_status fail(dbie_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

#define CUDA_TRY(expr)                                                                       \
  do {                                                                                       \
    cudaError_t e_ = (expr);                                                                 \
    if (e_ != cudaSuccess) {                                                                 \
      return fail(e_ == cudaErrorMemoryAllocation ? DBIE_ENOMEM : DBIE_ECUDA,                \
                  std::string(#expr) + ": " + cudaGetErrorString(e_));                       \
    }                                                                                        \
  } while (0)

#define DBIE_TRY(expr)                      \
  do {                                      \
    dbie_status s_ = (expr);                \
    if (s_ != DBIE_OK) return s_;           \
  } while (0)

// Growable device buffer (contents are not preserved when it grows).
struct DBuf {
  void* p = nullptr;
  size_t cap = 0;
  template <typename T>
  T* as() const { return static_cast<T*>(p); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
};

dbie_status ensure(DBuf& b, size_t bytes) {
  if (bytes <= b.cap && b.p) return DBIE_OK;
  b.release();
  const size_t nb = std::max<size_t>(bytes, 256);
  CUDA_TRY(cudaMalloc(&b.p, nb));
  b.cap = nb;
  return DBIE_OK;
}

// Small per-pass control block on the device.
struct Misc {
  PlanHdr plan;
  int32_t item_off[2];
  int32_t q_cnt[1];
  int32_t work;
  int32_t near_cnt;
  int32_t bad;
  int32_t pad[2];
};

struct SolveBufs {
  DBuf probs, ppos, lam0, sd, si, q_cnt_pass, item_off, ctrl, out, res, codes, corr;
  DBuf qpos[2], qlam[2], q_cnt[2], act[2], near[2];
  DBuf msc, fout, fq_cnt_pass, fitem_off;            // certified decisions
  DBuf fpos[2], flam[2], fq_cnt[2], ref[2];
  DBuf dout, dq_cnt_pass, ditem_off;                  // its difference level
  DBuf dpos[2], dlam[2], dlam0[2], dq_cnt[2];
  cudaGraphExec_t exec = nullptr;
  std::vector<unsigned char> key;   // launch arguments the cached graph was captured with
  std::vector<cudaEvent_t> ev;      // profiling events inside the graph (6 per round)
  void release() {
    for (DBuf* b : {&probs, &ppos, &lam0, &sd, &si, &q_cnt_pass, &item_off, &ctrl, &out, &res,
                    &codes, &corr, &msc, &fout, &fq_cnt_pass, &fitem_off, &dout, &dq_cnt_pass,
                    &ditem_off})
      b->release();
    for (int s = 0; s < 2; ++s)
      for (DBuf* b : {&qpos[s], &qlam[s], &q_cnt[s], &act[s], &near[s], &fpos[s], &flam[s],
                      &fq_cnt[s], &ref[s], &dpos[s], &dlam[s], &dlam0[s], &dq_cnt[s]})
        b->release();
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    ev.clear();
  }
};

// Device control words of a solve: plan, counters, statistics.
struct SolveCtrl {
  PlanHdr plan;
  int32_t work;
  int32_t round;
  int32_t act_cnt[2];
  int32_t near_cnt[2];
  int32_t bad;
  int32_t pad;
  unsigned long long stat_queries;
  double stat_pairs;
  // certified decisions: the float-float re-evaluation pass of each round
  PlanHdr fplan;
  int32_t fwork;
  int32_t ref_cnt[2];
  int32_t pad2;
  unsigned long long stat_ties;
  double stat_ff_pairs;
  // and its difference level
  PlanHdr dplan;
  int32_t dwork;
  int32_t pad3;
  unsigned long long stat_difs;
  double stat_dif_pairs;
};

int device_sm_count(int dev) {
  int n = 0;
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

// Persistent grid size of a kernel: resident CTAs per SM times SMs.
struct GridCache {
  std::mutex mu;
  std::vector<std::pair<const void*, int>> entries;
};
GridCache g_grids;

int persistent_grid(const KernelRef& k, int dev) {
  {
    std::lock_guard<std::mutex> lk(g_grids.mu);
    for (auto& e : g_grids.entries)
      if (e.first == k.fn) return e.second;
  }
  if (k.smem > 48 * 1024)
    cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k.fn, k.nt, k.smem);
  if (per_sm < 1) per_sm = 1;
  const int g = per_sm * device_sm_count(dev);
  std::lock_guard<std::mutex> lk(g_grids.mu);
  g_grids.entries.push_back({k.fn, g});
  return g;
}

}  // namespace

struct dbie_ctx {
  int device = 0;
  int32_t nx = 0, ny = 0;
  double x0 = 0, y0 = 0, hx = 1, hy = 1, dA = 1;
  int64_t npix = 0;
  int32_t ntiles = 0;
  int sm_count = 1;
  DBuf t32, t64, tff, prob, err, misc;
  DBuf st_in, st_out, st_aux;     // host-memory staging
  DBuf qpos, qlam, near_list, out, ptiles;
  DBuf qlam0, dmsc;                // dbie_eval_difference: reference lambdas, bound sums
  DBuf trace;                     // DBIE_TRACE_ITEMS builds: item timeline of the last pass
  int64_t trace_items = 0;
  DBuf tv32, tv64, probv;         // noise-variance tiles and their problem descriptor
  DBuf b0raw;                     // the magnetogram as given (3 x npix float32), for restaging
  DBuf vtmp;                      // per-quadrature-point adjoint before the gather to nodes
  int quad_g = 0;                 // 0: pixel centres (Eq. 16); g: nine-node elements (Eq. 15)
  bool pxe = false;               // pixel-exact near field on the pixel-centre rule
  DBuf pxe_corr, pxe_pos, pxe_list, pxe_w, pxe_part, pxe_bins;   // its per-call scratch
  QuadInfo qi{};
  int64_t nquad = 0;              // quadrature points: npix, or (elements x g)^2
  int32_t qnx = 0, qny = 0;       // quadrature-point grid
  SolveBufs sb;
  int cfg[NVAR][2] = {};   // tuned launch configuration per variant / tied
  int vjp_cfg = 0;
  cudaStream_t cap_stream = nullptr;  // stream used only to capture graphs
  int32_t* pinned = nullptr;          // pinned host words for polling
  bool profiling = false;
  dbie_stats stats{};
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;  // eval/vjp launches to time
  std::vector<double> pending_pairs;
  std::vector<cudaEvent_t> free_events;
};

namespace {

dbie_options resolved(const dbie_ctx* c, const dbie_options* o) {
  dbie_options r;
  dbie_default_options(&r);
  if (o) r = *o;
  if (!(r.simplex_step > 0)) r.simplex_step = 1.0 / (std::max(c->nx, c->ny) * c->hx);
  if (!(r.g_scale > 0)) r.g_scale = c->hx / 6.0;
  if (r.near_z < 0) r.near_z = 2.0 * c->hx;
  return r;
}

dbie_status check_opts(const dbie_options& o) {
  if (!(o.tol >= 0) || !std::isfinite(o.tol)) return fail(DBIE_EINVAL, "tol must be >= 0");
  if (o.max_iter < 0) return fail(DBIE_EINVAL, "max_iter must be >= 0");
  if (o.lambda_mode != DBIE_LAMBDA_PER_COMPONENT && o.lambda_mode != DBIE_LAMBDA_TIED)
    return fail(DBIE_EINVAL, "lambda_mode must be DBIE_LAMBDA_PER_COMPONENT or DBIE_LAMBDA_TIED");
  if (o.precision != DBIE_PREC_MIXED && o.precision != DBIE_PREC_FP64 &&
      o.precision != DBIE_PREC_FLOAT_FLOAT)
    return fail(DBIE_EINVAL, "precision must be DBIE_PREC_MIXED, DBIE_PREC_FP64 or "
                             "DBIE_PREC_FLOAT_FLOAT");
  if (o.method != DBIE_METHOD_SIMPLEX && o.method != DBIE_METHOD_QUASI_NEWTON)
    return fail(DBIE_EINVAL, "method must be DBIE_METHOD_SIMPLEX or DBIE_METHOD_QUASI_NEWTON");
  if (!(o.certify >= 0) || !std::isfinite(o.certify))
    return fail(DBIE_EINVAL, "certify must be finite and >= 0");
  if (!(o.certify_ref >= 0) || !std::isfinite(o.certify_ref))
    return fail(DBIE_EINVAL, "certify_ref must be finite and >= 0");
  if (!std::isfinite(o.simplex_step) || !std::isfinite(o.w_g) || !std::isfinite(o.g_scale) ||
      !std::isfinite(o.near_z) || !std::isfinite(o.eps_f) || !std::isfinite(o.eps_g))
    return fail(DBIE_EINVAL, "options must be finite");
  return DBIE_OK;
}

// The float-float form serves field evaluation (B, grad B, f, g) only.
dbie_status no_float_float(const dbie_options& o, const char* fn) {
  if (o.precision == DBIE_PREC_FLOAT_FLOAT)
    return fail(DBIE_EINVAL, std::string(fn) + ": DBIE_PREC_FLOAT_FLOAT is available in dbie_eval "
                                               "(without dBdlam) only");
  return DBIE_OK;
}

dbie_status check_mem(int32_t mem_kind) {
  if (mem_kind != DBIE_MEM_HOST && mem_kind != DBIE_MEM_DEVICE)
    return fail(DBIE_EINVAL, "mem_kind must be DBIE_MEM_HOST or DBIE_MEM_DEVICE");
  return DBIE_OK;
}

dbie_status host_points_ok(const float* xyz, int64_t n) {
  for (int64_t i = 0; i < n; ++i) {
    const float x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
    if (!std::isfinite(x) || !std::isfinite(y) || !std::isfinite(z) || !(z > 0.f))
      return fail(DBIE_EINVAL, "point " + std::to_string(i) + " is not finite or has z <= 0");
  }
  return DBIE_OK;
}

dbie_status host_finite(const float* a, int64_t n, const char* what) {
  for (int64_t i = 0; i < n; ++i)
    if (!std::isfinite(a[i])) return fail(DBIE_EINVAL, std::string(what) + " has a non-finite value");
  return DBIE_OK;
}
dbie_status host_finite(const double* a, int64_t n, const char* what) {
  for (int64_t i = 0; i < n; ++i)
    if (!std::isfinite(a[i])) return fail(DBIE_EINVAL, std::string(what) + " has a non-finite value");
  return DBIE_OK;
}

// Reads and clears the device error word (synchronises the stream).
dbie_status check_device_error(dbie_ctx* c, cudaStream_t s) {
  CUDA_TRY(cudaStreamSynchronize(s));
  unsigned e = 0;
  CUDA_TRY(cudaMemcpy(&e, c->err.p, sizeof(unsigned), cudaMemcpyDeviceToHost));
  if (e) {
    CUDA_TRY(cudaMemset(c->err.p, 0, sizeof(unsigned)));
    char buf[128];
    std::snprintf(buf, sizeof buf, "a bounded device wait gave up (error word 0x%x)", e);
    return fail(DBIE_ETIMEOUT, buf);
  }
  return DBIE_OK;
}

cudaEvent_t take_event(dbie_ctx* c) {
  if (!c->free_events.empty()) {
    cudaEvent_t e = c->free_events.back();
    c->free_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void resolve_pending(dbie_ctx* c) {
  for (size_t i = 0; i < c->pending.size(); ++i) {
    float ms = 0.f;
    if (cudaEventSynchronize(c->pending[i].second) == cudaSuccess &&
        cudaEventElapsedTime(&ms, c->pending[i].first, c->pending[i].second) == cudaSuccess) {
      c->stats.kernel_ms += ms;
      c->stats.launches += 1;
      c->stats.pair_evals += c->pending_pairs[i];
    } else {
      (void)cudaGetLastError();
    }
    c->free_events.push_back(c->pending[i].first);
    c->free_events.push_back(c->pending[i].second);
  }
  c->pending.clear();
  c->pending_pairs.clear();
}

dbie_status launch_kernel(const KernelRef& k, int grid, void* args, cudaStream_t s) {
  void* argv[1] = {args};
  CUDA_TRY(cudaLaunchKernel(k.fn, dim3(grid), dim3(k.nt), argv, k.smem, s));
  return DBIE_OK;
}

int var_of(bool grad, bool dlam) {
  return grad ? (dlam ? VAR_OBJL : VAR_OBJ) : (dlam ? VAR_VL : VAR_V);
}

// rows < 0: from this context's quadrature-point grid (aligned groups of 4 on one row).
KernelRef g1_ref(dbie_ctx* c, int var, bool tied, bool fp64, int rows = -1) {
  if (fp64) return g1_ref_f64(var, tied);
  const bool r = rows < 0 ? (c->qnx % 4 == 0) : rows != 0;
  if (c->quad_g != 0) return g1_ref_f32_split(var, tied, r);   // element Gauss points
  return g1_ref_f32(var, tied, c->cfg[var][tied ? 1 : 0], r);
}

// One pair-sum pass over n queries of this context (single problem): pack, plan, sweep,
// near-field correction.  Results are in c->out as item chunks described by c->misc.
dbie_status pass_single(dbie_ctx* c, int var, bool fp64, const dbie_options& o, int64_t n,
                        const float* d_xyz, const float* d_lamf, const double* d_lamd,
                        cudaStream_t s, bool tied = false, bool ffp = false) {
  Misc* m = c->misc.as<Misc>();
  DBIE_TRY(ensure(c->qpos, sizeof(float4) * n));
  DBIE_TRY(ensure(c->qlam, sizeof(Lam4) * n));
  // (the noise variance sums positive terms: FP32 is accurate there without a near field)
  const bool near_on = !fp64 && !ffp && o.near_z > 0 && var != VAR_NV;
  if (near_on) DBIE_TRY(ensure(c->near_list, sizeof(int32_t) * n));
  CUDA_TRY(cudaMemsetAsync(&m->near_cnt, 0, sizeof(int32_t), s));
  launch_pack_eval(n, d_xyz, d_lamf, d_lamd, c->qpos.as<float4>(), c->qlam.as<Lam4>(),
                   c->near_list.as<int32_t>(), &m->near_cnt, near_on ? 1 : 0, o.near_z, s);
  const KernelRef k = ffp ? g1_ref_ff(var, tied) : g1_ref(c, var, tied, fp64);
  const int grid = persistent_grid(k, c->device);
  const int64_t nblk = (n + k.qper - 1) / k.qper;
  const int64_t target = std::max<int64_t>(1, (int64_t)grid * DBIE_SPLIT_TARGET_PCT / 100);
  int64_t nsplit = 1;
  if (nblk < target) nsplit = std::min<int64_t>((target + nblk - 1) / nblk, c->ntiles);
  const int64_t nitems = nblk * nsplit;
  if (nitems > INT32_MAX / 2) return fail(DBIE_EINVAL, "too many points for one call");
  const int nsum = 3 * nsum_per_comp(var);
  DBIE_TRY(ensure(c->out, sizeof(double) * nitems * nsum * k.qper));
  launch_plan_single(&m->plan, m->item_off, m->q_cnt, &m->work, (int)nitems, (int)nsplit, k.qper,
                     (int)n, s);
  G1Args a{};
  a.probs = var == VAR_NV ? c->probv.as<ProbDesc>() : c->prob.as<ProbDesc>();
  a.nprob = 1;
  // Fault injection for tests of the bounded waits: the CTA that takes work item 0 never issues
  // its tile copies, its waits expire after their time limit and the call reports DBIE_ETIMEOUT.
  if (const char* fi = std::getenv("DBIE_FAULT_INJECT")) a.fault = std::atoi(fi) == 1 ? 1 : 0;
  a.plan = &m->plan;
  a.item_off = m->item_off;
  a.q_cnt = m->q_cnt;
  a.work = &m->work;
  a.qpos = c->qpos.as<float4>();
  a.qlam = c->qlam.as<Lam4>();
  a.out = c->out.as<double>();
  a.err = c->err.as<unsigned>();
#if DBIE_TRACE_ITEMS
  DBIE_TRY(ensure(c->trace, sizeof(unsigned long long) * 3 * nitems));
  CUDA_TRY(cudaMemsetAsync(c->trace.p, 0, sizeof(unsigned long long) * 3 * nitems, s));
  a.trace = c->trace.as<unsigned long long>();
  c->trace_items = nitems;
#endif
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (c->profiling) {
    e0 = take_event(c);
    e1 = take_event(c);
    CUDA_TRY(cudaEventRecord(e0, s));
  }
  DBIE_TRY(launch_kernel(k, grid, &a, s));
  if (c->profiling) {
    CUDA_TRY(cudaEventRecord(e1, s));
    c->pending.push_back({e0, e1});
    c->pending_pairs.push_back((double)n * (double)c->nquad);
  }
  if (near_on)
    launch_nearfield(var, tied, c->prob.as<ProbDesc>(), c->near_list.as<int32_t>(), &m->near_cnt,
                     c->qpos.as<float4>(), c->qlam.as<Lam4>(), &m->plan, m->item_off,
                     c->out.as<double>(), 2 * c->sm_count, s);
  CUDA_TRY(cudaGetLastError());
  return DBIE_OK;
}

struct Staging {  // host-memory calls: where each argument lives on the device
  size_t off = 0;
  char* base = nullptr;
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = reinterpret_cast<T*>(base + off);
    off += count * sizeof(T);
    return p;
  }
};

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// ------------------------------------------------------------------------ autotuning ----
// Chosen launch configuration per (device, kernel, variant, boundary size class), kept in memory
// and, when $DBIE_TUNE_CACHE names a file, appended to it as "key cfg" lines.
struct TuneCache {
  std::mutex mu;
  std::vector<std::pair<std::string, int>> entries;
  bool loaded = false;
};
TuneCache g_tune;

std::string tune_key(int dev, const char* kernel, int var, int tied, int64_t units) {
  cudaDeviceProp p;
  cudaGetDeviceProperties(&p, dev);
  int bucket = 0;
  while ((int64_t(1) << bucket) < units) ++bucket;
  std::string name(p.name);
  for (char& ch : name)
    if (ch == ' ') ch = '_';
  return name + "/" + kernel + "/v" + std::to_string(var) + "/t" + std::to_string(tied) + "/2^" +
         std::to_string(bucket);
}

int tune_lookup(const std::string& key) {
  std::lock_guard<std::mutex> lk(g_tune.mu);
  if (!g_tune.loaded) {
    g_tune.loaded = true;
    if (const char* path = std::getenv("DBIE_TUNE_CACHE")) {
      if (FILE* f = std::fopen(path, "r")) {
        char k[512];
        int v;
        while (std::fscanf(f, "%511s %d", k, &v) == 2)
          if (v >= 0 && v < NCFG) g_tune.entries.push_back({k, v});
        std::fclose(f);
      }
    }
  }
  for (auto it = g_tune.entries.rbegin(); it != g_tune.entries.rend(); ++it)
    if (it->first == key) return it->second;
  return -1;
}

void tune_store(const std::string& key, int cfg) {
  std::lock_guard<std::mutex> lk(g_tune.mu);
  g_tune.entries.push_back({key, cfg});
  if (const char* path = std::getenv("DBIE_TUNE_CACHE")) {
    if (FILE* f = std::fopen(path, "a")) {
      std::fprintf(f, "%s %d\n", key.c_str(), cfg);
      std::fclose(f);
    }
  }
}

// Minimum over `reps` launches of the timed pair-sum kernel of fn() (profiling events).
template <typename Fn>
dbie_status time_min(dbie_ctx* c, int reps, Fn fn, double* best_ms) {
  *best_ms = 1e30;
  for (int r = 0; r < reps; ++r) {
    c->pending.clear();
    c->pending_pairs.clear();
    const dbie_stats saved = c->stats;
    c->stats = dbie_stats{};
    DBIE_TRY(fn());
    resolve_pending(c);
    if (c->stats.launches > 0) *best_ms = std::min(*best_ms, c->stats.kernel_ms);
    c->stats = saved;
  }
  return DBIE_OK;
}

}  // namespace

// =====================================================================================
extern "C" {

const char* dbie_last_error(void) { return g_err.c_str(); }

const char* dbie_version(void) { return "dbie-gb300 0.2 (sm_103a)"; }

void dbie_default_options(dbie_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof *o);
  o->eps_f = 1e-3;
  o->eps_g = 1e-4;
  o->tol = 1e-6;
  o->certify = 0.02;
  o->certify_ref = 0.02;
  o->max_iter = 50;
  o->lambda_mode = DBIE_LAMBDA_PER_COMPONENT;
  o->simplex_step = 0.0;
  o->w_g = 1.0;
  o->g_scale = 0.0;
  o->precision = DBIE_PREC_MIXED;
  o->near_z = -1.0;
}

void dbie_destroy(dbie_ctx* c) {
  if (!c) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  for (DBuf* b : {&c->t32, &c->t64, &c->tff, &c->prob, &c->err, &c->misc, &c->st_in, &c->st_out,
                  &c->st_aux, &c->qpos, &c->qlam, &c->near_list, &c->out, &c->ptiles, &c->tv32,
                  &c->tv64, &c->probv, &c->b0raw, &c->vtmp, &c->pxe_corr, &c->pxe_pos,
                  &c->pxe_list, &c->pxe_w, &c->pxe_part, &c->pxe_bins, &c->trace, &c->qlam0,
                  &c->dmsc})
    b->release();
  c->sb.release();
  for (auto& pr : c->pending) {
    cudaEventDestroy(pr.first);
    cudaEventDestroy(pr.second);
  }
  for (cudaEvent_t e : c->free_events) cudaEventDestroy(e);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->pinned) cudaFreeHost(c->pinned);
  cudaSetDevice(prev);
  delete c;
}

// Problem descriptor of the context's current quadrature (problem-specific search fields 0).
static ProbDesc desc_of(const dbie_ctx* c) {
  ProbDesc pd{};
  pd.tiles32 = c->t32.as<float>();
  pd.tiles64 = c->t64.as<double>();
  pd.tilesff = c->tff.as<float>();
  pd.ntiles = c->ntiles;
  pd.nx = c->qnx;
  pd.ny = c->qny;
  pd.quad_g = c->quad_g;
  pd.near_w = c->quad_g == 0 ? NEAR_W : std::max(1, (NEAR_W * c->quad_g + 1) / 2);
  pd.nf32 = c->quad_g == 0 ? NFIELD : NFIELD_SPLIT;
  for (int a = 0; a < MAX_GAUSS; ++a) pd.gx[a] = c->qi.gx[a];
  pd.x0 = c->x0; pd.y0 = c->y0; pd.hx = c->hx; pd.hy = c->hy;
  pd.area = c->dA;
  return pd;
}

// Quadrature-point tiles from the stored magnetogram: pixel centres with b = B0 dA / 2 pi, or the
// Gauss points of the nine-node elements with the interpolated, weighted field.
static dbie_status restage(dbie_ctx* c, cudaStream_t s) {
  const float* B0 = c->b0raw.as<float>();
  if (c->quad_g == 0)
    launch_stage_boundary(B0, B0 + c->npix, B0 + 2 * c->npix, c->nx, c->ny, c->x0, c->y0, c->hx,
                          c->hy, c->dA / TWO_PI, c->ntiles, c->t32.as<float>(),
                          c->t64.as<double>(), s);
  else
    launch_stage_q9(B0, c->nx, c->ny, c->x0, c->y0, c->hx, c->hy, c->qi, c->ntiles,
                    c->t32.as<float>(), c->t64.as<double>(), s);
  launch_stage_ff(c->t64.as<double>(), c->ntiles, c->tff.as<float>(), s);
  CUDA_TRY(cudaGetLastError());
  return DBIE_OK;
}

// Pixel-exact near field of one call: on for this context and options (near_z > 0 bounds it).
static bool pxe_on(const dbie_ctx* c, const dbie_options& o) { return c->pxe && o.near_z > 0; }

// Correction of B and grad B (12 per point, c->pxe_corr) at n points packed as float4 (problem 0).
static dbie_status pxe_correct(dbie_ctx* c, int64_t n, const float4* pos, bool fp64,
                               const dbie_options& o, cudaStream_t s) {
  DBIE_TRY(ensure(c->pxe_corr, sizeof(double) * 12 * n));
  launch_pxe_corr(fp64, c->prob.as<ProbDesc>(), n, pos, o.near_z, c->pxe_corr.as<double>(),
                  16 * c->sm_count, s);
  CUDA_TRY(cudaGetLastError());
  return DBIE_OK;
}

// gB0 += the transpose of the correction at n points with weights w (full: 12 per point,
// else 3 = gB).
static dbie_status pxe_adjoint(dbie_ctx* c, int64_t n, const float4* pos, const double* w,
                               bool full, bool fp64, const dbie_options& o, double* gB0,
                               cudaStream_t s) {
  DBIE_TRY(ensure(c->pxe_list, sizeof(int32_t) * (n + 1)));
  const int nchunk = pxe_adjoint_chunks(n, c->npix, c->sm_count);
  DBIE_TRY(ensure(c->pxe_part, sizeof(double) * 3 * (size_t)c->npix * (nchunk + 1)));
  DBIE_TRY(ensure(c->pxe_bins, sizeof(int32_t) * (3 * (size_t)pxe_bins(c->nx, c->ny) + 1 + n)));
  int32_t* list = c->pxe_list.as<int32_t>();
  CUDA_TRY(launch_pxe_adjoint(fp64, full, c->prob.as<ProbDesc>(), n, c->nx, c->ny, pos, o.near_z,
                              w, list, list + n, c->pxe_bins.as<int32_t>(), nchunk,
                              c->pxe_part.as<double>(), gB0, s));
  return DBIE_OK;
}

static dbie_status stage_boundary(dbie_ctx* c, const float* Bx, const float* By, const float* Bz,
                                  int32_t mem_kind, cudaStream_t s) {
  const float* src[3] = {Bx, By, Bz};
  const int64_t npix = c->npix;
  float* raw = c->b0raw.as<float>();
  if (mem_kind == DBIE_MEM_HOST) {
    for (int p = 0; p < 3; ++p) DBIE_TRY(host_finite(src[p], npix, "magnetogram"));
    for (int p = 0; p < 3; ++p)
      CUDA_TRY(cudaMemcpyAsync(raw + p * npix, src[p], sizeof(float) * npix,
                               cudaMemcpyHostToDevice, s));
    DBIE_TRY(restage(c, s));
    CUDA_TRY(cudaStreamSynchronize(s));   // the caller may free its arrays after the call
  } else {
    Misc* m = c->misc.as<Misc>();
    CUDA_TRY(cudaMemsetAsync(&m->bad, 0, sizeof(int32_t), s));
    for (int p = 0; p < 3; ++p) launch_count_bad(src[p], npix, 0, &m->bad, s);
    int32_t bad = 0;
    CUDA_TRY(cudaMemcpyAsync(&bad, &m->bad, sizeof bad, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (bad) return fail(DBIE_EINVAL, "magnetogram has a non-finite value");
    for (int p = 0; p < 3; ++p)
      CUDA_TRY(cudaMemcpyAsync(raw + p * npix, src[p], sizeof(float) * npix,
                               cudaMemcpyDeviceToDevice, s));
    DBIE_TRY(restage(c, s));
  }
  return DBIE_OK;
}

// Variance tiles for the noise propagation (device sigma arrays or NULL = sigma0).
static dbie_status stage_variance(dbie_ctx* c, const float* sx, const float* sy, const float* sz,
                                  double sigma0, cudaStream_t s) {
  if (!c->probv.p) {
    DBIE_TRY(ensure(c->tv32, sizeof(float) * NFIELD * TILE * (size_t)c->ntiles));
    DBIE_TRY(ensure(c->tv64, sizeof(double) * NFIELD * TILE * (size_t)c->ntiles));
    DBIE_TRY(ensure(c->probv, sizeof(ProbDesc)));
    ProbDesc pd{};
    pd.tiles32 = c->tv32.as<float>();
    pd.tiles64 = c->tv64.as<double>();
    pd.ntiles = c->ntiles;
    pd.nx = c->nx; pd.ny = c->ny;
    pd.x0 = c->x0; pd.y0 = c->y0; pd.hx = c->hx; pd.hy = c->hy;
    CUDA_TRY(cudaMemcpyAsync(c->probv.p, &pd, sizeof pd, cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaStreamSynchronize(s));   // pd is a host temporary
  }
  launch_stage_variance(sx, sy, sz, sigma0, c->nx, c->ny, c->x0, c->y0, c->hx, c->hy,
                        c->dA / TWO_PI, c->ntiles, c->tv32.as<float>(), c->tv64.as<double>(), s);
  CUDA_TRY(cudaGetLastError());
  return DBIE_OK;
}

dbie_status dbie_create(dbie_ctx** out, int32_t nx, int32_t ny, double x0, double y0, double hx,
                        double hy, double pixel_area, const float* Bx, const float* By,
                        const float* Bz, int32_t mem_kind, void* stream) {
  if (!out) return fail(DBIE_EINVAL, "out is NULL");
  *out = nullptr;
  DBIE_TRY(check_mem(mem_kind));
  if (nx < 1 || ny < 1) return fail(DBIE_EINVAL, "nx and ny must be >= 1");
  if ((int64_t)nx * ny > (int64_t)1 << 30) return fail(DBIE_EINVAL, "magnetogram too large");
  if (!(hx > 0) || !(hy > 0) || !std::isfinite(hx) || !std::isfinite(hy))
    return fail(DBIE_EINVAL, "hx and hy must be finite and > 0");
  if (!(pixel_area > 0) || !std::isfinite(pixel_area))
    return fail(DBIE_EINVAL, "pixel_area must be finite and > 0");
  if (!std::isfinite(x0) || !std::isfinite(y0)) return fail(DBIE_EINVAL, "x0, y0 must be finite");
  if (!Bx || !By || !Bz) return fail(DBIE_EINVAL, "Bx, By, Bz must not be NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  dbie_ctx* c = new dbie_ctx();
  cudaGetDevice(&c->device);
  c->sm_count = device_sm_count(c->device);
  c->nx = nx; c->ny = ny; c->x0 = x0; c->y0 = y0; c->hx = hx; c->hy = hy; c->dA = pixel_area;
  c->npix = (int64_t)nx * ny;
  c->nquad = c->npix;
  c->qnx = nx;
  c->qny = ny;
  c->ntiles = (int32_t)((c->npix + TILE - 1) / TILE);
  auto bail = [&](dbie_status st) { std::string m = g_err; dbie_destroy(c); g_err = m; return st; };
  dbie_status st;
  if ((st = ensure(c->t32, sizeof(float) * NFIELD * TILE * (size_t)c->ntiles)) != DBIE_OK) return bail(st);
  if ((st = ensure(c->t64, sizeof(double) * NFIELD * TILE * (size_t)c->ntiles)) != DBIE_OK) return bail(st);
  if ((st = ensure(c->tff, sizeof(float) * 2 * NFIELD * TILE * (size_t)c->ntiles)) != DBIE_OK) return bail(st);
  if ((st = ensure(c->b0raw, sizeof(float) * 3 * (size_t)c->npix)) != DBIE_OK) return bail(st);
  if ((st = ensure(c->prob, sizeof(ProbDesc))) != DBIE_OK) return bail(st);
  if ((st = ensure(c->err, sizeof(unsigned))) != DBIE_OK) return bail(st);
  if ((st = ensure(c->misc, sizeof(Misc))) != DBIE_OK) return bail(st);
  if (cudaMemsetAsync(c->err.p, 0, sizeof(unsigned), s) != cudaSuccess ||
      cudaMemsetAsync(c->misc.p, 0, sizeof(Misc), s) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaHostAlloc((void**)&c->pinned, 64, cudaHostAllocDefault) != cudaSuccess)
    return bail(fail(DBIE_ECUDA, "context set-up failed"));
  const ProbDesc pd = desc_of(c);
  if (cudaMemcpyAsync(c->prob.p, &pd, sizeof pd, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return bail(fail(DBIE_ECUDA, "copy of the problem descriptor failed"));
  if ((st = stage_boundary(c, Bx, By, Bz, mem_kind, s)) != DBIE_OK) return bail(st);
  if (cudaStreamSynchronize(s) != cudaSuccess) return bail(fail(DBIE_ECUDA, "create: sync failed"));
  *out = c;
  return DBIE_OK;
}

dbie_status dbie_set_boundary(dbie_ctx* c, const float* Bx, const float* By, const float* Bz,
                              int32_t mem_kind, void* stream) {
  if (!c) return fail(DBIE_EINVAL, "ctx is NULL");
  DBIE_TRY(check_mem(mem_kind));
  if (!Bx || !By || !Bz) return fail(DBIE_EINVAL, "Bx, By, Bz must not be NULL");
  CUDA_TRY(cudaSetDevice(c->device));
  return stage_boundary(c, Bx, By, Bz, mem_kind, static_cast<cudaStream_t>(stream));
}

// Gauss-Legendre rule with m points on [-1, 1]: roots of P_m by Newton's method (P_m and its
// derivative from the three-term recurrence), weights 2 / ((1 - x^2) P_m'(x)^2), ascending.
static void gauss_rule(int m, double* x, double* w) {
  for (int i = 0; i < (m + 1) / 2; ++i) {
    double t = std::cos(3.14159265358979323846 * (i + 0.75) / (m + 0.5));
    double d = 1.0;
    for (int it = 0; it < 64; ++it) {
      double p_prev = 1.0, p = t;
      for (int k = 2; k <= m; ++k) {
        const double pk = ((2 * k - 1) * t * p - (k - 1) * p_prev) / k;
        p_prev = p;
        p = pk;
      }
      d = m * (t * p - p_prev) / (t * t - 1.0);
      const double step = p / d;
      t -= step;
      if (std::fabs(step) <= 1e-16 * std::fabs(t) + 1e-300) {
        // one more evaluation at the converged root for the weight
        p_prev = 1.0; p = t;
        for (int k = 2; k <= m; ++k) {
          const double pk = ((2 * k - 1) * t * p - (k - 1) * p_prev) / k;
          p_prev = p;
          p = pk;
        }
        d = m * (t * p - p_prev) / (t * t - 1.0);
        break;
      }
    }
    const double wt = 2.0 / ((1.0 - t * t) * d * d);
    x[m - 1 - i] = t;     // t > 0 first: fill from the top
    w[m - 1 - i] = wt;
    x[i] = -t;
    w[i] = wt;
  }
  if (m % 2 == 1) x[m / 2] = 0.0;
}

dbie_status dbie_set_quadrature(dbie_ctx* c, int32_t order, void* stream) {
  if (!c) return fail(DBIE_EINVAL, "ctx is NULL");
  if (order < DBIE_QUAD_PIXEL_EXACT || order > MAX_GAUSS)
    return fail(DBIE_EINVAL, "order must be -1 (pixel-exact near field), 0 (pixel centres) or "
                             "1.." + std::to_string(MAX_GAUSS));
  const bool pxe = order == DBIE_QUAD_PIXEL_EXACT;
  if (pxe) order = 0;
  if (order > 0 && (c->nx < 3 || c->ny < 3 || c->nx % 2 == 0 || c->ny % 2 == 0))
    return fail(DBIE_EINVAL, "nine-node elements need odd nx, ny >= 3");
  CUDA_TRY(cudaSetDevice(c->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CUDA_TRY(cudaStreamSynchronize(s));   // no pass of the old quadrature may still read the tiles
  c->quad_g = order;
  c->pxe = pxe;
  c->qi = QuadInfo{};
  c->qi.g = order;
  if (order > 0) {
    gauss_rule(order, c->qi.gx, c->qi.gw);
    c->qnx = (c->nx - 1) / 2 * order;
    c->qny = (c->ny - 1) / 2 * order;
  } else {
    c->qnx = c->nx;
    c->qny = c->ny;
  }
  c->nquad = (int64_t)c->qnx * c->qny;
  if (c->nquad > (int64_t)1 << 30) return fail(DBIE_EINVAL, "too many quadrature points");
  c->ntiles = (int32_t)((c->nquad + TILE - 1) / TILE);
  DBIE_TRY(ensure(c->t32, sizeof(float) * (order > 0 ? NFIELD_SPLIT : NFIELD) * TILE *
                              (size_t)c->ntiles));
  DBIE_TRY(ensure(c->t64, sizeof(double) * NFIELD * TILE * (size_t)c->ntiles));
  DBIE_TRY(ensure(c->tff, sizeof(float) * 2 * NFIELD * TILE * (size_t)c->ntiles));
  c->sb.release();   // cached solve graphs hold the old tile pointers
  const ProbDesc pd = desc_of(c);
  CUDA_TRY(cudaMemcpyAsync(c->prob.p, &pd, sizeof pd, cudaMemcpyHostToDevice, s));
  DBIE_TRY(restage(c, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  return DBIE_OK;
}

dbie_status dbie_eval(dbie_ctx* c, int64_t n, const float* xyz, const float* lambda,
                      const dbie_options* opt, int32_t mem_kind, double* B, double* gradB,
                      double* dBdlam, double* fgphi, void* stream) {
  if (!c) return fail(DBIE_EINVAL, "ctx is NULL");
  DBIE_TRY(check_mem(mem_kind));
  if (n < 0) return fail(DBIE_EINVAL, "n must be >= 0");
  if (n > ((int64_t)1 << 31) - 1) return fail(DBIE_EINVAL, "n too large");
  if (n > 0 && (!xyz || !lambda || !B))
    return fail(DBIE_EINVAL, "xyz, lambda and B must not be NULL");
  const dbie_options o = resolved(c, opt);
  DBIE_TRY(check_opts(o));
  if (n == 0) return DBIE_OK;
  CUDA_TRY(cudaSetDevice(c->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool fp64 = o.precision == DBIE_PREC_FP64;
  const bool ffp = o.precision == DBIE_PREC_FLOAT_FLOAT;
  if (ffp && dBdlam) DBIE_TRY(no_float_float(o, "dbie_eval with dBdlam"));
  const int var = var_of(gradB || fgphi, dBdlam != nullptr);
  const float* d_xyz = xyz;
  const float* d_lam = lambda;
  double *dB = B, *dG = gradB, *dL = dBdlam, *dF = fgphi;
  if (mem_kind == DBIE_MEM_HOST) {
    DBIE_TRY(host_points_ok(xyz, n));
    DBIE_TRY(host_finite(lambda, 3 * n, "lambda"));
    DBIE_TRY(ensure(c->st_in, 2 * align256(sizeof(float) * 3 * n)));
    DBIE_TRY(ensure(c->st_out, 4 * align256(sizeof(double) * 9 * n)));
    Staging si{0, c->st_in.as<char>()}, so{0, c->st_out.as<char>()};
    float* t_xyz = si.take<float>(3 * n);
    float* t_lam = si.take<float>(3 * n);
    CUDA_TRY(cudaMemcpyAsync(t_xyz, xyz, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(t_lam, lambda, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, s));
    d_xyz = t_xyz;
    d_lam = t_lam;
    dB = so.take<double>(3 * n);
    dG = gradB ? so.take<double>(9 * n) : nullptr;
    dL = dBdlam ? so.take<double>(3 * n) : nullptr;
    dF = fgphi ? so.take<double>(3 * n) : nullptr;
  }
  DBIE_TRY(pass_single(c, var, fp64, o, n, d_xyz, d_lam, nullptr, s, false, ffp));
  const bool pxe = pxe_on(c, o);
  if (pxe) DBIE_TRY(pxe_correct(c, n, c->qpos.as<float4>(), fp64, o, s));
  Misc* m = c->misc.as<Misc>();
  launch_finalize_eval(var, n, &m->plan, m->item_off, c->out.as<double>(), c->qpos.as<float4>(),
                       c->qlam.as<Lam4>(), o.g_scale, o.w_g, dB, dG, dL, nullptr, dF,
                       pxe ? c->pxe_corr.as<double>() : nullptr, s);
  CUDA_TRY(cudaGetLastError());
  if (mem_kind == DBIE_MEM_HOST) {
    CUDA_TRY(cudaMemcpyAsync(B, dB, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s));
    if (gradB) CUDA_TRY(cudaMemcpyAsync(gradB, dG, sizeof(double) * 9 * n, cudaMemcpyDeviceToHost, s));
    if (dBdlam) CUDA_TRY(cudaMemcpyAsync(dBdlam, dL, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s));
    if (fgphi) CUDA_TRY(cudaMemcpyAsync(fgphi, dF, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s));
    DBIE_TRY(check_device_error(c, s));
  }
  return DBIE_OK;
}

dbie_status dbie_eval_difference(dbie_ctx* c, int64_t n, const float* xyz,
                                 const double* lambda, const double* lambda_ref, int32_t tied,
                                 double* dS, double* dS_bound, void* stream) {
  if (!c) return fail(DBIE_EINVAL, "ctx is NULL");
  if (n < 0) return fail(DBIE_EINVAL, "n must be >= 0");
  if (n > ((int64_t)1 << 31) - 1) return fail(DBIE_EINVAL, "n too large");
  if (n > 0 && (!xyz || !lambda || !lambda_ref || !dS))
    return fail(DBIE_EINVAL, "xyz, lambda, lambda_ref and dS must not be NULL");
  if (n == 0) return DBIE_OK;
  CUDA_TRY(cudaSetDevice(c->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Misc* m = c->misc.as<Misc>();
  DBIE_TRY(ensure(c->qpos, sizeof(float4) * n));
  DBIE_TRY(ensure(c->qlam, sizeof(Lam4) * n));
  DBIE_TRY(ensure(c->qlam0, sizeof(Lam4) * n));
  launch_pack_eval(n, xyz, nullptr, lambda_ref, c->qpos.as<float4>(), c->qlam0.as<Lam4>(), nullptr,
                   nullptr, 0, 0.0, s);
  launch_pack_eval(n, xyz, nullptr, lambda, c->qpos.as<float4>(), c->qlam.as<Lam4>(), nullptr,
                   nullptr, 0, 0.0, s);
  const KernelRef k = g1_ref_dif(tied != 0);
  const int grid = persistent_grid(k, c->device);
  const int64_t nblk = (n + k.qper - 1) / k.qper;
  const int64_t target = std::max<int64_t>(1, (int64_t)grid * DBIE_SPLIT_TARGET_PCT / 100);
  int64_t nsplit = 1;
  if (nblk < target) nsplit = std::min<int64_t>((target + nblk - 1) / nblk, c->ntiles);
  const int64_t nitems = nblk * nsplit;
  if (nitems > INT32_MAX / 2) return fail(DBIE_EINVAL, "too many points for one call");
  DBIE_TRY(ensure(c->out, sizeof(double) * nitems * 12 * k.qper));
  launch_plan_single(&m->plan, m->item_off, m->q_cnt, &m->work, (int)nitems, (int)nsplit, k.qper,
                     (int)n, s);
  G1Args a{};
  a.probs = c->prob.as<ProbDesc>();
  a.nprob = 1;
  a.plan = &m->plan;
  a.item_off = m->item_off;
  a.q_cnt = m->q_cnt;
  a.work = &m->work;
  a.qpos = c->qpos.as<float4>();
  a.qlam = c->qlam.as<Lam4>();
  a.qlam0 = c->qlam0.as<Lam4>();
  a.out = c->out.as<double>();
  a.err = c->err.as<unsigned>();
  DBIE_TRY(launch_kernel(k, grid, &a, s));
  double* msc = nullptr;
  if (dS_bound) {
    DBIE_TRY(ensure(c->dmsc, sizeof(double) * 18 * n));
    msc = c->dmsc.as<double>();
    launch_msc(c->prob.as<ProbDesc>(), n, c->qpos.as<float4>(), msc, msc + 15 * n,
               (int)std::min<int64_t>((n + 127) / 128, 32LL * c->sm_count), s);
  }
  launch_dif_debug(n, &m->plan, m->item_off, c->out.as<double>(), c->qlam.as<Lam4>(),
                   c->qlam0.as<Lam4>(), msc, msc ? msc + 15 * n : nullptr, tied ? 1 : 3, dS,
                   dS_bound, s);
  CUDA_TRY(cudaGetLastError());
  return DBIE_OK;
}

dbie_status dbie_objective(dbie_ctx* c, int64_t n, const float* xyz, const float* lambda,
                           const dbie_options* opt, int32_t mem_kind, double* fgphi, double* dphi,
                           void* stream) {
  if (!c) return fail(DBIE_EINVAL, "ctx is NULL");
  DBIE_TRY(check_mem(mem_kind));
  if (n < 0) return fail(DBIE_EINVAL, "n must be >= 0");
  if (n > ((int64_t)1 << 31) - 1) return fail(DBIE_EINVAL, "n too large");
  if (!fgphi && !dphi) return fail(DBIE_EINVAL, "fgphi and dphi are both NULL");
  if (n > 0 && (!xyz || !lambda)) return fail(DBIE_EINVAL, "xyz and lambda must not be NULL");
  const dbie_options o = resolved(c, opt);
  DBIE_TRY(check_opts(o));
  DBIE_TRY(no_float_float(o, "dbie_objective"));
  if (n == 0) return DBIE_OK;
  CUDA_TRY(cudaSetDevice(c->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool fp64 = o.precision == DBIE_PREC_FP64;
  const float* d_xyz = xyz;
  const float* d_lam = lambda;
  double *dF = fgphi, *dD = dphi;
  if (mem_kind == DBIE_MEM_HOST) {
    DBIE_TRY(host_points_ok(xyz, n));
    DBIE_TRY(host_finite(lambda, 3 * n, "lambda"));
    DBIE_TRY(ensure(c->st_in, 2 * align256(sizeof(float) * 3 * n)));
    DBIE_TRY(ensure(c->st_out, 2 * align256(sizeof(double) * 3 * n)));
    Staging si{0, c->st_in.as<char>()}, so{0, c->st_out.as<char>()};
    float* t_xyz = si.take<float>(3 * n);
    float* t_lam = si.take<float>(3 * n);
    CUDA_TRY(cudaMemcpyAsync(t_xyz, xyz, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(t_lam, lambda, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, s));
    d_xyz = t_xyz;
    d_lam = t_lam;
    dF = fgphi ? so.take<double>(3 * n) : nullptr;
    dD = dphi ? so.take<double>(3 * n) : nullptr;
  }
  DBIE_TRY(pass_single(c, VAR_OBJN, fp64, o, n, d_xyz, d_lam, nullptr, s));
  const bool pxe = pxe_on(c, o);
  if (pxe) DBIE_TRY(pxe_correct(c, n, c->qpos.as<float4>(), fp64, o, s));
  Misc* m = c->misc.as<Misc>();
  launch_finalize_objective(n, &m->plan, m->item_off, c->out.as<double>(), c->qpos.as<float4>(),
                            c->qlam.as<Lam4>(), o.g_scale, o.w_g, dF, dD, nullptr,
                            pxe ? c->pxe_corr.as<double>() : nullptr, s);
  CUDA_TRY(cudaGetLastError());
  if (mem_kind == DBIE_MEM_HOST) {
    if (fgphi) CUDA_TRY(cudaMemcpyAsync(fgphi, dF, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s));
    if (dphi) CUDA_TRY(cudaMemcpyAsync(dphi, dD, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s));
    DBIE_TRY(check_device_error(c, s));
  }
  return DBIE_OK;
}

// Per-quadrature-point adjoint sums (item chunks of 3 sums) -> dL/dB0 per node: scaled by
// dA / 2 pi at pixel centres, or gathered through the nine-node shape functions.
static dbie_status finalize_adjoint(dbie_ctx* c, const PlanHdr* plan, double* gB0, int accumulate,
                                    cudaStream_t s) {
  if (c->quad_g == 0) {
    launch_finalize_vjp(c->npix, plan, c->out.as<double>(), c->dA / TWO_PI, gB0, accumulate, s);
  } else {
    DBIE_TRY(ensure(c->vtmp, sizeof(double) * 3 * (size_t)c->nquad));
    launch_finalize_vjp(c->nquad, plan, c->out.as<double>(), 1.0, c->vtmp.as<double>(), 0, s);
    launch_q9_gather(c->vtmp.as<double>(), c->nx, c->ny, c->hx, c->hy, c->qi, gB0, accumulate, s);
  }
  CUDA_TRY(cudaGetLastError());
  return DBIE_OK;
}

dbie_status dbie_vjp(dbie_ctx* c, int64_t n, const float* xyz, const double* lambda,
                     const double* gB, const dbie_options* opt, int32_t mem_kind, double* gB0,
                     double* glam, int32_t accumulate, void* stream) {
  if (!c) return fail(DBIE_EINVAL, "ctx is NULL");
  DBIE_TRY(check_mem(mem_kind));
  if (n < 0) return fail(DBIE_EINVAL, "n must be >= 0");
  if (n > ((int64_t)1 << 31) - 1) return fail(DBIE_EINVAL, "n too large");
  if (!gB0) return fail(DBIE_EINVAL, "gB0 must not be NULL");
  if (n > 0 && (!xyz || !lambda || !gB)) return fail(DBIE_EINVAL, "xyz, lambda, gB must not be NULL");
  const dbie_options o = resolved(c, opt);
  DBIE_TRY(check_opts(o));
  DBIE_TRY(no_float_float(o, "dbie_vjp"));
  CUDA_TRY(cudaSetDevice(c->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool fp64 = o.precision == DBIE_PREC_FP64;
  const int64_t npix = c->npix;
  const float* d_xyz = xyz;
  const double *d_lam = lambda, *d_gB = gB;
  double *d_gB0 = gB0, *d_glam = glam;
  if (mem_kind == DBIE_MEM_HOST) {
    if (n > 0) {
      DBIE_TRY(host_points_ok(xyz, n));
      DBIE_TRY(host_finite(lambda, 3 * n, "lambda"));
      DBIE_TRY(host_finite(gB, 3 * n, "gB"));
    }
    DBIE_TRY(ensure(c->st_in, align256(sizeof(float) * 3 * n) + 2 * align256(sizeof(double) * 3 * n)));
    DBIE_TRY(ensure(c->st_out, align256(sizeof(double) * 3 * npix) + align256(sizeof(double) * 3 * n)));
    Staging si{0, c->st_in.as<char>()}, so{0, c->st_out.as<char>()};
    float* t_xyz = si.take<float>(3 * n);
    double* t_lam = si.take<double>(3 * n);
    double* t_gB = si.take<double>(3 * n);
    if (n > 0) {
      CUDA_TRY(cudaMemcpyAsync(t_xyz, xyz, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, s));
      CUDA_TRY(cudaMemcpyAsync(t_lam, lambda, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s));
      CUDA_TRY(cudaMemcpyAsync(t_gB, gB, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s));
    }
    d_xyz = t_xyz; d_lam = t_lam; d_gB = t_gB;
    d_gB0 = so.take<double>(3 * npix);
    d_glam = glam ? so.take<double>(3 * n) : nullptr;
    if (accumulate)
      CUDA_TRY(cudaMemcpyAsync(d_gB0, gB0, sizeof(double) * 3 * npix, cudaMemcpyHostToDevice, s));
  }
  if (n == 0) {
    if (!accumulate) CUDA_TRY(cudaMemsetAsync(d_gB0, 0, sizeof(double) * 3 * npix, s));
  } else {
    // Adjoint sweep: pixels in registers, point tiles through shared memory.
    const int nptiles = (int)((n + TILE - 1) / TILE);
    DBIE_TRY(ensure(c->ptiles, (size_t)nptiles * VJP_NFIELD * TILE * (fp64 ? 8 : 4)));
    launch_pack_vjp(n, d_xyz, d_lam, d_gB, 0, nptiles, c->ptiles.as<float>(),
                    c->ptiles.as<double>(), fp64 ? 1 : 0, s);
    const KernelRef k = (!fp64 && c->quad_g != 0) ? vjp_ref_split(false)
                                                   : vjp_ref(fp64, false, c->vjp_cfg);
    const int grid = persistent_grid(k, c->device);
    const int64_t nq = c->nquad;   // quadrature points (pixels, or element Gauss points)
    const int64_t nblk = (nq + k.qper - 1) / k.qper;
    const int64_t target = 2LL * grid;
    int64_t nsplit = 1;
    if (nblk < target) nsplit = std::min<int64_t>((target + nblk - 1) / nblk, nptiles);
    const int64_t nitems = nblk * nsplit;
    DBIE_TRY(ensure(c->out, sizeof(double) * nitems * 3 * k.qper));
    Misc* m = c->misc.as<Misc>();
    launch_plan_single(&m->plan, m->item_off, m->q_cnt, &m->work, (int)nitems, (int)nsplit,
                       k.qper, (int)nq, s);
    VjpArgs a{};
    a.ptiles32 = c->ptiles.as<float>();
    a.ptiles64 = c->ptiles.as<double>();
    a.nptiles = nptiles;
    a.npix = (int32_t)nq;
    a.btiles32 = c->t32.as<float>();
    a.btiles64 = c->t64.as<double>();
    a.plan = &m->plan;
    a.work = &m->work;
    a.out = c->out.as<double>();
    a.err = c->err.as<unsigned>();
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (c->profiling) {
      e0 = take_event(c);
      e1 = take_event(c);
      CUDA_TRY(cudaEventRecord(e0, s));
    }
    DBIE_TRY(launch_kernel(k, grid, &a, s));
    if (c->profiling) {
      CUDA_TRY(cudaEventRecord(e1, s));
      c->pending.push_back({e0, e1});
      c->pending_pairs.push_back((double)n * (double)nq);
    }
    DBIE_TRY(finalize_adjoint(c, &m->plan, d_gB0, accumulate ? 1 : 0, s));
    if (pxe_on(c, o)) {
      DBIE_TRY(ensure(c->pxe_pos, sizeof(float4) * n));
      launch_pack_points(n, d_xyz, 0, c->pxe_pos.as<float4>(), s);
      DBIE_TRY(pxe_adjoint(c, n, c->pxe_pos.as<float4>(), d_gB, false, fp64, o, d_gB0, s));
    }
    if (d_glam) {
      // dL/dlambda_p = gB_p * z lambda_p Sl_p, from a value + dB/dlambda pass.
      DBIE_TRY(pass_single(c, VAR_VL, fp64, o, n, d_xyz, nullptr, d_lam, s));
      launch_finalize_eval(VAR_VL, n, &m->plan, m->item_off, c->out.as<double>(),
                           c->qpos.as<float4>(), c->qlam.as<Lam4>(), o.g_scale, o.w_g, nullptr,
                           nullptr, d_glam, d_gB, nullptr, nullptr, s);
      CUDA_TRY(cudaGetLastError());
    }
  }
  if (mem_kind == DBIE_MEM_HOST) {
    CUDA_TRY(cudaMemcpyAsync(gB0, d_gB0, sizeof(double) * 3 * npix, cudaMemcpyDeviceToHost, s));
    if (glam && n > 0)
      CUDA_TRY(cudaMemcpyAsync(glam, d_glam, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s));
    DBIE_TRY(check_device_error(c, s));
  }
  return DBIE_OK;
}

// ------------------------------------------------------------------ second order ----
// Common argument checks and host staging of (xyz, lambda[, gB]) for the second-order calls.
struct PtArgs {
  const float* xyz = nullptr;
  const double* lam = nullptr;
  const double* gB = nullptr;
};
static dbie_status stage_points(dbie_ctx* c, int64_t n, const float* xyz, const double* lambda,
                                const double* gB, int32_t mem_kind, size_t out_bytes,
                                cudaStream_t s, PtArgs& d, Staging& so) {
  d.xyz = xyz;
  d.lam = lambda;
  d.gB = gB;
  if (mem_kind != DBIE_MEM_HOST) return DBIE_OK;
  DBIE_TRY(host_points_ok(xyz, n));
  DBIE_TRY(host_finite(lambda, 3 * n, "lambda"));
  if (gB) DBIE_TRY(host_finite(gB, 3 * n, "gB"));
  DBIE_TRY(ensure(c->st_in, align256(sizeof(float) * 3 * n) + 2 * align256(sizeof(double) * 3 * n)));
  DBIE_TRY(ensure(c->st_out, out_bytes));
  Staging si{0, c->st_in.as<char>()};
  so = Staging{0, c->st_out.as<char>()};
  float* t_xyz = si.take<float>(3 * n);
  double* t_lam = si.take<double>(3 * n);
  CUDA_TRY(cudaMemcpyAsync(t_xyz, xyz, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(t_lam, lambda, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s));
  d.xyz = t_xyz;
  d.lam = t_lam;
  if (gB) {
    double* t_gB = si.take<double>(3 * n);
    CUDA_TRY(cudaMemcpyAsync(t_gB, gB, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s));
    d.gB = t_gB;
  }
  return DBIE_OK;
}

static dbie_status check_n(int64_t n) {
  if (n < 0) return fail(DBIE_EINVAL, "n must be >= 0");
  if (n > ((int64_t)1 << 31) - 1) return fail(DBIE_EINVAL, "n too large");
  return DBIE_OK;
}

dbie_status dbie_hessian(dbie_ctx* c, int64_t n, const float* xyz, const double* lambda,
                         const dbie_options* opt, int32_t mem_kind, double* phi, double* grad,
                         double* hess, void* stream) {
  if (!c) return fail(DBIE_EINVAL, "ctx is NULL");
  DBIE_TRY(check_mem(mem_kind));
  DBIE_TRY(check_n(n));
  if (!phi && !grad && !hess) return fail(DBIE_EINVAL, "phi, grad and hess are all NULL");
  if (n > 0 && (!xyz || !lambda)) return fail(DBIE_EINVAL, "xyz and lambda must not be NULL");
  const dbie_options o = resolved(c, opt);
  DBIE_TRY(check_opts(o));
  DBIE_TRY(no_float_float(o, "dbie_hessian"));
  if (n == 0) return DBIE_OK;
  CUDA_TRY(cudaSetDevice(c->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool fp64 = o.precision == DBIE_PREC_FP64;
  const bool tied = o.lambda_mode == DBIE_LAMBDA_TIED;
  PtArgs d;
  Staging so;
  DBIE_TRY(stage_points(c, n, xyz, lambda, nullptr, mem_kind,
                        align256(sizeof(double) * n) + align256(sizeof(double) * 3 * n) +
                            align256(sizeof(double) * 9 * n),
                        s, d, so));
  double *dP = phi, *dG = grad, *dH = hess;
  if (mem_kind == DBIE_MEM_HOST) {
    dP = phi ? so.take<double>(n) : nullptr;
    dG = grad ? so.take<double>(3 * n) : nullptr;
    dH = hess ? so.take<double>(9 * n) : nullptr;
  }
  DBIE_TRY(pass_single(c, VAR_HESS, fp64, o, n, d.xyz, nullptr, d.lam, s, tied));
  const bool pxe = pxe_on(c, o);
  if (pxe) DBIE_TRY(pxe_correct(c, n, c->qpos.as<float4>(), fp64, o, s));
  Misc* m = c->misc.as<Misc>();
  launch_finalize_hessian(n, &m->plan, m->item_off, c->out.as<double>(), c->qpos.as<float4>(),
                          c->qlam.as<Lam4>(), tied ? 1 : 3, o.g_scale, o.w_g, dP, dG, dH,
                          pxe ? c->pxe_corr.as<double>() : nullptr, s);
  CUDA_TRY(cudaGetLastError());
  if (mem_kind == DBIE_MEM_HOST) {
    if (phi) CUDA_TRY(cudaMemcpyAsync(phi, dP, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    if (grad) CUDA_TRY(cudaMemcpyAsync(grad, dG, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s));
    if (hess) CUDA_TRY(cudaMemcpyAsync(hess, dH, sizeof(double) * 9 * n, cudaMemcpyDeviceToHost, s));
    DBIE_TRY(check_device_error(c, s));
  }
  return DBIE_OK;
}

dbie_status dbie_vjp_implicit(dbie_ctx* c, int64_t n, const float* xyz, const double* lambda,
                              const double* gB, const dbie_options* opt, int32_t mem_kind,
                              double* gB0, double* v, int32_t* flags, int32_t accumulate,
                              void* stream) {
  if (!c) return fail(DBIE_EINVAL, "ctx is NULL");
  DBIE_TRY(check_mem(mem_kind));
  DBIE_TRY(check_n(n));
  if (!gB0) return fail(DBIE_EINVAL, "gB0 must not be NULL");
  if (n > 0 && (!xyz || !lambda || !gB)) return fail(DBIE_EINVAL, "xyz, lambda, gB must not be NULL");
  const dbie_options o = resolved(c, opt);
  DBIE_TRY(check_opts(o));
  DBIE_TRY(no_float_float(o, "dbie_vjp_implicit"));
  CUDA_TRY(cudaSetDevice(c->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool fp64 = o.precision == DBIE_PREC_FP64;
  const bool tied = o.lambda_mode == DBIE_LAMBDA_TIED;
  const int64_t npix = c->npix;
  PtArgs d;
  Staging so;
  DBIE_TRY(stage_points(c, n, xyz, lambda, gB, mem_kind,
                        align256(sizeof(double) * 3 * npix) + align256(sizeof(double) * 3 * n) +
                            align256(sizeof(int32_t) * n),
                        s, d, so));
  double *d_gB0 = gB0, *d_v = v;
  int32_t* d_fl = flags;
  if (mem_kind == DBIE_MEM_HOST) {
    d_gB0 = so.take<double>(3 * npix);
    d_v = v ? so.take<double>(3 * n) : nullptr;
    d_fl = flags ? so.take<int32_t>(n) : nullptr;
    if (accumulate)
      CUDA_TRY(cudaMemcpyAsync(d_gB0, gB0, sizeof(double) * 3 * npix, cudaMemcpyHostToDevice, s));
  }
  if (n == 0) {
    if (!accumulate) CUDA_TRY(cudaMemsetAsync(d_gB0, 0, sizeof(double) * 3 * npix, s));
  } else {
    // 1. Hessian pass at lambda (ten sums per component) -> 2. per-point H, v and the adjoint
    // weights, written as point records -> 3. seven-weight adjoint sweep over the pixels.
    DBIE_TRY(pass_single(c, VAR_HESS, fp64, o, n, d.xyz, nullptr, d.lam, s, tied));
    const bool pxe = pxe_on(c, o);
    if (pxe) {
      DBIE_TRY(pxe_correct(c, n, c->qpos.as<float4>(), fp64, o, s));
      DBIE_TRY(ensure(c->pxe_w, sizeof(double) * 12 * n));
    }
    Misc* m = c->misc.as<Misc>();
    const int nptiles = (int)((n + TILE - 1) / TILE);
    DBIE_TRY(ensure(c->ptiles, (size_t)nptiles * VJP7_NFIELD * TILE * (fp64 ? 8 : 4)));
    launch_implicit_weights(n, nptiles, &m->plan, m->item_off, c->out.as<double>(),
                            c->qpos.as<float4>(), c->qlam.as<Lam4>(), d.gB, tied ? 1 : 3,
                            o.g_scale, o.w_g, c->ptiles.as<float>(), c->ptiles.as<double>(),
                            fp64 ? 1 : 0, d_v, d_fl, pxe ? c->pxe_corr.as<double>() : nullptr,
                            pxe ? c->pxe_w.as<double>() : nullptr, s);
    CUDA_TRY(cudaGetLastError());
    const KernelRef k = (!fp64 && c->quad_g != 0) ? vjp7_ref_split(tied) : vjp7_ref(fp64, tied);
    const int grid = persistent_grid(k, c->device);
    const int64_t nq = c->nquad;   // quadrature points (pixels, or element Gauss points)
    const int64_t nblk = (nq + k.qper - 1) / k.qper;
    const int64_t target = 2LL * grid;
    int64_t nsplit = 1;
    if (nblk < target) nsplit = std::min<int64_t>((target + nblk - 1) / nblk, nptiles);
    const int64_t nitems = nblk * nsplit;
    // (the Hessian pass's partial sums were consumed by the weights kernel above; the stream
    // orders the reuse of c->out and of the plan block)
    DBIE_TRY(ensure(c->out, sizeof(double) * nitems * 3 * k.qper));
    launch_plan_single(&m->plan, m->item_off, m->q_cnt, &m->work, (int)nitems, (int)nsplit,
                       k.qper, (int)nq, s);
    VjpArgs a{};
    a.ptiles32 = c->ptiles.as<float>();
    a.ptiles64 = c->ptiles.as<double>();
    a.nptiles = nptiles;
    a.npix = (int32_t)nq;
    a.btiles32 = c->t32.as<float>();
    a.btiles64 = c->t64.as<double>();
    a.plan = &m->plan;
    a.work = &m->work;
    a.out = c->out.as<double>();
    a.err = c->err.as<unsigned>();
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (c->profiling) {
      e0 = take_event(c);
      e1 = take_event(c);
      CUDA_TRY(cudaEventRecord(e0, s));
    }
    DBIE_TRY(launch_kernel(k, grid, &a, s));
    if (c->profiling) {
      CUDA_TRY(cudaEventRecord(e1, s));
      c->pending.push_back({e0, e1});
      c->pending_pairs.push_back((double)n * (double)nq);
    }
    DBIE_TRY(finalize_adjoint(c, &m->plan, d_gB0, accumulate ? 1 : 0, s));
    if (pxe)
      DBIE_TRY(pxe_adjoint(c, n, c->qpos.as<float4>(), c->pxe_w.as<double>(), true, fp64, o,
                           d_gB0, s));
  }
  if (mem_kind == DBIE_MEM_HOST) {
    CUDA_TRY(cudaMemcpyAsync(gB0, d_gB0, sizeof(double) * 3 * npix, cudaMemcpyDeviceToHost, s));
    if (v && n > 0) CUDA_TRY(cudaMemcpyAsync(v, d_v, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s));
    if (flags && n > 0)
      CUDA_TRY(cudaMemcpyAsync(flags, d_fl, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
    DBIE_TRY(check_device_error(c, s));
  }
  return DBIE_OK;
}

dbie_status dbie_noise_var(dbie_ctx* c, int64_t n, const float* xyz, const double* lambda,
                           const float* sigma_x, const float* sigma_y, const float* sigma_z,
                           double sigma0, const dbie_options* opt, int32_t mem_kind, double* var,
                           void* stream) {
  if (!c) return fail(DBIE_EINVAL, "ctx is NULL");
  DBIE_TRY(check_mem(mem_kind));
  DBIE_TRY(check_n(n));
  if (n > 0 && (!xyz || !lambda || !var))
    return fail(DBIE_EINVAL, "xyz, lambda and var must not be NULL");
  if (!std::isfinite(sigma0)) return fail(DBIE_EINVAL, "sigma0 must be finite");
  if (c->quad_g != 0 || c->pxe)
    return fail(DBIE_EINVAL, "the noise variance needs the pixel-centre rule (dbie_set_quadrature 0)");
  const dbie_options o = resolved(c, opt);
  DBIE_TRY(check_opts(o));
  DBIE_TRY(no_float_float(o, "dbie_noise_var"));
  if (n == 0) return DBIE_OK;
  CUDA_TRY(cudaSetDevice(c->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool fp64 = o.precision == DBIE_PREC_FP64;
  const float* sg[3] = {sigma_x, sigma_y, sigma_z};
  const float* d_sg[3] = {sigma_x, sigma_y, sigma_z};
  const int64_t npix = c->npix;
  if (mem_kind == DBIE_MEM_HOST) {
    for (int p = 0; p < 3; ++p)
      if (sg[p]) DBIE_TRY(host_finite(sg[p], npix, "sigma"));
    DBIE_TRY(ensure(c->st_aux, 3 * align256(sizeof(float) * npix)));
    Staging sa{0, c->st_aux.as<char>()};
    for (int p = 0; p < 3; ++p) {
      float* t = sa.take<float>(npix);
      if (sg[p]) {
        CUDA_TRY(cudaMemcpyAsync(t, sg[p], sizeof(float) * npix, cudaMemcpyHostToDevice, s));
        d_sg[p] = t;
      }
    }
  }
  if (mem_kind == DBIE_MEM_DEVICE) {
    Misc* m = c->misc.as<Misc>();
    CUDA_TRY(cudaMemsetAsync(&m->bad, 0, sizeof(int32_t), s));
    for (int p = 0; p < 3; ++p)
      if (sg[p]) launch_count_bad(sg[p], npix, 0, &m->bad, s);
    int32_t bad = 0;
    CUDA_TRY(cudaMemcpyAsync(&bad, &m->bad, sizeof bad, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (bad) return fail(DBIE_EINVAL, "sigma has a non-finite value");
  }
  DBIE_TRY(stage_variance(c, d_sg[0], d_sg[1], d_sg[2], sigma0, s));
  PtArgs d;
  Staging so;
  DBIE_TRY(stage_points(c, n, xyz, lambda, nullptr, mem_kind, align256(sizeof(double) * 3 * n), s,
                        d, so));
  double* d_var = mem_kind == DBIE_MEM_HOST ? so.take<double>(3 * n) : var;
  DBIE_TRY(pass_single(c, VAR_NV, fp64, o, n, d.xyz, nullptr, d.lam, s,
                       o.lambda_mode == DBIE_LAMBDA_TIED));
  Misc* m = c->misc.as<Misc>();
  launch_finalize_nv(n, &m->plan, m->item_off, c->out.as<double>(), c->qpos.as<float4>(), d_var, s);
  CUDA_TRY(cudaGetLastError());
  if (mem_kind == DBIE_MEM_HOST) {
    CUDA_TRY(cudaMemcpyAsync(var, d_var, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s));
    DBIE_TRY(check_device_error(c, s));
  }
  return DBIE_OK;
}

// -------------------------------------------------------------------------- solve ----
static dbie_status solve_impl(int32_t nprob, dbie_ctx* const* ctxs, const int64_t* n,
                              const float* const* xyz, const dbie_options* opt,
                              const double* const* lam_init, int32_t mem_kind,
                              const dbie_solve_out* out, cudaStream_t s) {
  dbie_ctx* c = ctxs[0];
  CUDA_TRY(cudaSetDevice(c->device));
  const dbie_options o = resolved(c, opt);
  DBIE_TRY(check_opts(o));
  DBIE_TRY(no_float_float(o, "dbie_solve"));
  const bool fp64 = o.precision == DBIE_PREC_FP64;
  const bool tied = o.lambda_mode == DBIE_LAMBDA_TIED;
  const int dim = tied ? 1 : 3;
  // one pair-sum kernel serves every problem: the FP32 tile layout must agree
  for (int p = 1; p < nprob; ++p)
    if ((ctxs[p]->quad_g != 0) != (c->quad_g != 0))
      return fail(DBIE_EINVAL, "a batched solve needs all contexts on pixel centres or all on "
                               "nine-node elements");
  // Per-problem offsets.
  std::vector<int64_t> pt_off(nprob + 1, 0);
  for (int p = 0; p < nprob; ++p) pt_off[p + 1] = pt_off[p] + n[p];
  const int64_t N = pt_off[nprob];
  if (N == 0) return DBIE_OK;
  if (N > ((int64_t)1 << 31) / 4 - 1) return fail(DBIE_EINVAL, "too many points for one solve");
  const int64_t Qcap = (int64_t)(dim + 1) * N;
  SolveBufs& b = c->sb;
  int codes_stride = 0;
  for (int p = 0; p < nprob; ++p)
    if (out[p].codes) codes_stride = std::max(codes_stride, (int)out[p].codes_stride);
  codes_stride = std::min(codes_stride, std::max(o.max_iter, 1));

  const bool qn = o.method == DBIE_METHOD_QUASI_NEWTON;
  const int var = qn ? VAR_OBJN : VAR_OBJ;            // quasi-Newton needs the gradient sums
  // certified decisions: mixed-precision simplex with a positive near-tie band
  const bool cert = !fp64 && !qn && o.certify > 0;
  const int nsum = 3 * nsum_per_comp(var);
  bool rows_all = true;   // one kernel for all problems: rows only if every grid allows it
  for (int p = 0; p < nprob; ++p) rows_all &= ctxs[p]->qnx % 4 == 0;
  const KernelRef k = g1_ref(c, var, tied, fp64, rows_all ? 1 : 0);
  const int grid = persistent_grid(k, c->device);
  // Split a round's queries over tile ranges until the items cover this many CTAs (percent of
  // the persistent grid): more items balance the queue, fewer items mean fewer partial sums.
  const int target = (int)((int64_t)grid * DBIE_SPLIT_TARGET_PCT / 100);
  const int64_t items_cap = std::max<int64_t>((Qcap + k.qper - 1) / k.qper + nprob, 2LL * target) + 1;
  // float-float re-evaluation pass (at most 2 queries per point and round)
  const KernelRef kf = g1_ref_ff(VAR_OBJ, tied);
  const int grid_ff = cert ? persistent_grid(kf, c->device) : 0;
  const int target_ff = std::max(1, (int)((int64_t)grid_ff * DBIE_FF_SPLIT_TARGET_PCT / 100));
  const int64_t fitems_cap = std::max<int64_t>((2 * N + kf.qper - 1) / kf.qper + nprob,
                                               2LL * target_ff) + 1;
  // difference level of the re-evaluation (values near the point's float-float reference)
  const bool dif_on = cert && o.certify_ref > 0;
  const KernelRef kd = g1_ref_dif(tied);
  const int grid_dif = dif_on ? persistent_grid(kd, c->device) : 0;
  const int target_dif = std::max(1, (int)((int64_t)grid_dif * DBIE_FF_SPLIT_TARGET_PCT / 100));
  const int64_t ditems_cap = std::max<int64_t>((2 * N + kd.qper - 1) / kd.qper + nprob,
                                               2LL * target_dif) + 1;

  DBIE_TRY(ensure(b.probs, sizeof(ProbDesc) * nprob));
  DBIE_TRY(ensure(b.ppos, sizeof(float4) * N));
  DBIE_TRY(ensure(b.sd, sizeof(double) * D_NFIELDS * N));
  DBIE_TRY(ensure(b.si, sizeof(int32_t) * I_NFIELDS * N));
  DBIE_TRY(ensure(b.q_cnt_pass, sizeof(int32_t) * nprob));
  DBIE_TRY(ensure(b.item_off, sizeof(int32_t) * (nprob + 1)));
  DBIE_TRY(ensure(b.ctrl, sizeof(SolveCtrl)));
  DBIE_TRY(ensure(b.out, sizeof(double) * items_cap * nsum * k.qper));
  DBIE_TRY(ensure(b.res, align256(sizeof(double) * 8 * N) + align256(sizeof(int32_t) * 3 * N)));
  if (codes_stride) DBIE_TRY(ensure(b.codes, (size_t)codes_stride * N));
  for (int sd = 0; sd < 2; ++sd) {
    DBIE_TRY(ensure(b.qpos[sd], sizeof(float4) * Qcap));
    DBIE_TRY(ensure(b.qlam[sd], sizeof(Lam4) * Qcap));
    DBIE_TRY(ensure(b.q_cnt[sd], sizeof(int32_t) * nprob));
    DBIE_TRY(ensure(b.act[sd], sizeof(int32_t) * N));
    if (!fp64) DBIE_TRY(ensure(b.near[sd], sizeof(int32_t) * Qcap));
  }
  if (cert) {
    DBIE_TRY(ensure(b.msc, sizeof(double) * 18 * N));
    DBIE_TRY(ensure(b.fout, sizeof(double) * fitems_cap * 12 * kf.qper));
    DBIE_TRY(ensure(b.fq_cnt_pass, sizeof(int32_t) * nprob));
    DBIE_TRY(ensure(b.fitem_off, sizeof(int32_t) * (nprob + 1)));
    for (int sd = 0; sd < 2; ++sd) {
      DBIE_TRY(ensure(b.fpos[sd], sizeof(float4) * 2 * N));
      DBIE_TRY(ensure(b.flam[sd], sizeof(Lam4) * 2 * N));
      DBIE_TRY(ensure(b.fq_cnt[sd], sizeof(int32_t) * nprob));
      DBIE_TRY(ensure(b.ref[sd], sizeof(int32_t) * N));
    }
  }
  if (dif_on) {
    DBIE_TRY(ensure(b.dout, sizeof(double) * ditems_cap * 12 * kd.qper));
    DBIE_TRY(ensure(b.dq_cnt_pass, sizeof(int32_t) * nprob));
    DBIE_TRY(ensure(b.ditem_off, sizeof(int32_t) * (nprob + 1)));
    for (int sd = 0; sd < 2; ++sd) {
      DBIE_TRY(ensure(b.dpos[sd], sizeof(float4) * 2 * N));
      DBIE_TRY(ensure(b.dlam[sd], sizeof(Lam4) * 2 * N));
      DBIE_TRY(ensure(b.dlam0[sd], sizeof(Lam4) * 2 * N));
      DBIE_TRY(ensure(b.dq_cnt[sd], sizeof(int32_t) * nprob));
    }
  }
  bool any_init = false;
  for (int p = 0; p < nprob; ++p) any_init |= (lam_init && lam_init[p]);
  if (any_init) DBIE_TRY(ensure(b.lam0, sizeof(double) * 3 * N));

  // Problems and points.
  // Descriptor slot of each problem: largest (points x pixels) first, so that the dynamic item
  // queue hands out the longest work first and the round ends evenly (LPT order).
  std::vector<int> order(nprob), slot_of(nprob);
  for (int p = 0; p < nprob; ++p) order[p] = p;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b2) {
    return (double)n[a] * ctxs[a]->nquad > (double)n[b2] * ctxs[b2]->nquad;
  });
  for (int q = 0; q < nprob; ++q) slot_of[order[q]] = q;
  std::vector<ProbDesc> pds(nprob);
  for (int p = 0; p < nprob; ++p) {
    dbie_ctx* cp = ctxs[p];
    ProbDesc& pd = pds[slot_of[p]];
    pd = desc_of(cp);
    const dbie_options op = resolved(cp, opt);   // size- and spacing-dependent defaults
    pd.step = op.simplex_step;
    pd.g_scale = op.g_scale;
    pd.near_z = (!fp64 && op.near_z > 0) ? op.near_z : 0.0;
    pd.pxe_z = pxe_on(cp, op) ? op.near_z : 0.0;
    pd.q_off = (int64_t)(dim + 1) * pt_off[p];
    pd.qff_off = 2 * pt_off[p];
    pd.pt_off = pt_off[p];
    pd.npts = n[p];
  }
  CUDA_TRY(cudaMemcpyAsync(b.probs.p, pds.data(), sizeof(ProbDesc) * nprob, cudaMemcpyHostToDevice, s));
  SolveCtrl* ctrl = b.ctrl.as<SolveCtrl>();
  CUDA_TRY(cudaMemsetAsync(ctrl, 0, sizeof(SolveCtrl), s));
  for (int p = 0; p < nprob; ++p) {
    if (n[p] == 0) continue;
    const float* src = xyz[p];
    const float* dsrc = src;
    if (mem_kind == DBIE_MEM_HOST) {
      DBIE_TRY(host_points_ok(src, n[p]));
      DBIE_TRY(ensure(c->st_in, sizeof(float) * 3 * n[p]));
      CUDA_TRY(cudaMemcpyAsync(c->st_in.p, src, sizeof(float) * 3 * n[p], cudaMemcpyHostToDevice, s));
      dsrc = c->st_in.as<float>();
    } else {
      launch_count_bad(src, n[p], 1, &ctrl->bad, s);
    }
    launch_pack_points(n[p], dsrc, slot_of[p], b.ppos.as<float4>() + pt_off[p], s);
    if (any_init) {
      double* dst = b.lam0.as<double>() + 3 * pt_off[p];
      if (lam_init[p]) {
        if (mem_kind == DBIE_MEM_HOST) DBIE_TRY(host_finite(lam_init[p], 3 * n[p], "lambda_init"));
        CUDA_TRY(cudaMemcpyAsync(dst, lam_init[p], sizeof(double) * 3 * n[p],
                                 mem_kind == DBIE_MEM_HOST ? cudaMemcpyHostToDevice
                                                           : cudaMemcpyDeviceToDevice, s));
      } else {
        CUDA_TRY(cudaMemsetAsync(dst, 0, sizeof(double) * 3 * n[p], s));
      }
    }
    if (mem_kind == DBIE_MEM_HOST) CUDA_TRY(cudaStreamSynchronize(s));  // staging reuse
  }
  if (mem_kind == DBIE_MEM_DEVICE) {
    CUDA_TRY(cudaMemcpyAsync(c->pinned, &ctrl->bad, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (c->pinned[0]) return fail(DBIE_EINVAL, "a point is not finite or has z <= 0");
  }
  for (int sd = 0; sd < 2; ++sd) CUDA_TRY(cudaMemsetAsync(b.q_cnt[sd].p, 0, sizeof(int32_t) * nprob, s));
  if (cert) {
    for (int sd = 0; sd < 2; ++sd)
      CUDA_TRY(cudaMemsetAsync(b.fq_cnt[sd].p, 0, sizeof(int32_t) * nprob, s));
    if (dif_on)
      for (int sd = 0; sd < 2; ++sd)
        CUDA_TRY(cudaMemsetAsync(b.dq_cnt[sd].p, 0, sizeof(int32_t) * nprob, s));
    // the error bounds' lambda-independent absolute-value sums of every point
    launch_msc(b.probs.as<ProbDesc>(), N, b.ppos.as<float4>(), b.msc.as<double>(),
               b.msc.as<double>() + 15 * N,
               (int)std::min<int64_t>((N + 127) / 128, 32LL * c->sm_count), s);
    CUDA_TRY(cudaGetLastError());
  }
  if (codes_stride) CUDA_TRY(cudaMemsetAsync(b.codes.p, 0, (size_t)codes_stride * N, s));
  // Pixel-exact near field: the lambda-independent corrections of every point, once per solve.
  bool pxe_any = false;
  for (int q = 0; q < nprob; ++q) pxe_any |= pds[q].pxe_z > 0;
  if (pxe_any) {
    DBIE_TRY(ensure(b.corr, sizeof(double) * 12 * N));
    launch_pxe_corr(fp64, b.probs.as<ProbDesc>(), N, b.ppos.as<float4>(), -1.0,
                    b.corr.as<double>(), 16 * c->sm_count, s);
    CUDA_TRY(cudaGetLastError());
  }

  // Kernel arguments.
  char* rb = b.res.as<char>();
  double* res_B = reinterpret_cast<double*>(rb);
  double* res_lam = res_B + 3 * N;
  double* res_f = res_lam + 3 * N;
  double* res_g = res_f + N;
  int32_t* res_i = reinterpret_cast<int32_t*>(rb + align256(sizeof(double) * 8 * N));
  SolveArgs sa[2];
  bool near_on = false;
  for (int q = 0; q < nprob; ++q) near_on |= pds[q].near_z > 0;
  for (int cur = 0; cur < 2; ++cur) {
    SolveArgs& a = sa[cur];
    a = SolveArgs{};
    a.probs = b.probs.as<ProbDesc>();
    a.nprob = nprob;
    a.N = N;
    a.ppos = b.ppos.as<float4>();
    a.sd = b.sd.as<double>();
    a.si = b.si.as<int32_t>();
    const int nx_ = cur ^ 1;
    a.cur = RoundBuf{b.qpos[cur].as<float4>(), b.qlam[cur].as<Lam4>(), b.q_cnt[cur].as<int32_t>(),
                     b.act[cur].as<int32_t>(), &ctrl->act_cnt[cur], b.near[cur].as<int32_t>(),
                     &ctrl->near_cnt[cur], b.fpos[cur].as<float4>(), b.flam[cur].as<Lam4>(),
                     b.fq_cnt[cur].as<int32_t>(), b.ref[cur].as<int32_t>(), &ctrl->ref_cnt[cur],
                     b.dpos[cur].as<float4>(), b.dlam[cur].as<Lam4>(), b.dlam0[cur].as<Lam4>(),
                     b.dq_cnt[cur].as<int32_t>()};
    a.nxt = RoundBuf{b.qpos[nx_].as<float4>(), b.qlam[nx_].as<Lam4>(), b.q_cnt[nx_].as<int32_t>(),
                     b.act[nx_].as<int32_t>(), &ctrl->act_cnt[nx_], b.near[nx_].as<int32_t>(),
                     &ctrl->near_cnt[nx_], b.fpos[nx_].as<float4>(), b.flam[nx_].as<Lam4>(),
                     b.fq_cnt[nx_].as<int32_t>(), b.ref[nx_].as<int32_t>(), &ctrl->ref_cnt[nx_],
                     b.dpos[nx_].as<float4>(), b.dlam[nx_].as<Lam4>(), b.dlam0[nx_].as<Lam4>(),
                     b.dq_cnt[nx_].as<int32_t>()};
    a.out = b.out.as<double>();
    a.plan = &ctrl->plan;
    a.item_off = b.item_off.as<int32_t>();
    a.o = SolveOpts{o.eps_f, o.eps_g, o.tol, o.w_g, cert ? o.certify : 0.0, o.max_iter, dim,
                    near_on ? 1 : 0, 0, dif_on ? o.certify_ref : 0.0};
    a.res_B = res_B;
    a.res_lam = res_lam;
    a.res_f = res_f;
    a.res_g = res_g;
    a.res_iters = res_i;
    a.res_status = res_i + N;
    a.res_nfev = res_i + 2 * N;
    a.codes = codes_stride ? b.codes.as<char>() : nullptr;
    a.codes_stride = codes_stride;
    a.err = c->err.as<unsigned>();
    a.corr = pxe_any ? b.corr.as<double>() : nullptr;
    if (cert) {
      a.msc = b.msc.as<double>();
      a.fout = b.fout.as<double>();
      a.fplan = &ctrl->fplan;
      a.fitem_off = b.fitem_off.as<int32_t>();
      a.stat_ties = &ctrl->stat_ties;
      a.msc0 = b.msc.as<double>() + 15 * N;
    }
    if (dif_on) {
      a.dout = b.dout.as<double>();
      a.dplan = &ctrl->dplan;
      a.ditem_off = b.ditem_off.as<int32_t>();
      a.stat_difs = &ctrl->stat_difs;
    }
  }
  // Initial simplex and its queries go to side 0.
  SolveArgs a0 = sa[1];  // "next" of the side-1 round is side 0
  const int nm_grid = (int)std::min<int64_t>((N + 127) / 128, 8LL * c->sm_count);
  (qn ? launch_bfgs_init : launch_solve_init)(a0, any_init ? b.lam0.as<double>() : nullptr,
                    (int)std::min<int64_t>((N + 255) / 256, 8LL * c->sm_count), s);
  CUDA_TRY(cudaGetLastError());

  // One re-evaluation pass of a round (float-float, or differences when lam0 is given): plan
  // the queued values, run the pair sums, with profiling events ev_at and ev_at + 1 around it.
  auto record_reeval = [&](cudaStream_t cs, const KernelRef& kr, int grid_r, int target_r,
                           const DBuf& cnt, const DBuf& cnt_pass, const DBuf& item_off_r,
                           PlanHdr* plan_r, int32_t* work_r, double* stat_pairs_r,
                           const DBuf& qpos_r, const DBuf& qlam_r, const DBuf* qlam0_r,
                           const DBuf& out_r, int ev_at) -> dbie_status {
    PlanArgs pp{};
    pp.probs = b.probs.as<ProbDesc>();
    pp.nprob = nprob;
    pp.qper = kr.qper;
    pp.target_items = target_r;
    pp.nsplit_cap = 1 << 20;
    pp.q_cnt_cur = cnt.as<int32_t>();
    pp.q_cnt_pass = cnt_pass.as<int32_t>();
    pp.item_off = item_off_r.as<int32_t>();
    pp.plan = plan_r;
    pp.work = work_r;
    pp.stat_pairs = stat_pairs_r;
    launch_plan_round(pp, cs);
    G1Args ga{};
    ga.probs = b.probs.as<ProbDesc>();
    ga.nprob = nprob;
    ga.plan = plan_r;
    ga.item_off = item_off_r.as<int32_t>();
    ga.q_cnt = cnt_pass.as<int32_t>();
    ga.work = work_r;
    ga.qpos = qpos_r.as<float4>();
    ga.qlam = qlam_r.as<Lam4>();
    ga.qlam0 = qlam0_r ? qlam0_r->as<Lam4>() : nullptr;
    ga.out = out_r.as<double>();
    ga.err = c->err.as<unsigned>();
    if (c->profiling)
      CUDA_TRY(cudaEventRecordWithFlags(b.ev[ev_at], cs, cudaEventRecordExternal));
    DBIE_TRY(launch_kernel(kr, grid_r, &ga, cs));
    if (c->profiling)
      CUDA_TRY(cudaEventRecordWithFlags(b.ev[ev_at + 1], cs, cudaEventRecordExternal));
    return DBIE_OK;
  };
  // One simplex round = plan, pair sums (objective variant), near-field correction, step.
  constexpr int K = 4;  // rounds per graph launch (even: the ping-pong side returns to 0)
  auto record_rounds = [&](cudaStream_t cs) -> dbie_status {
    for (int r = 0; r < K; ++r) {
      const int cur = r & 1;
      PlanArgs pa{};
      pa.probs = b.probs.as<ProbDesc>();
      pa.nprob = nprob;
      pa.qper = k.qper;
      pa.target_items = target;
      pa.nsplit_cap = 1 << 20;
      pa.q_cnt_cur = b.q_cnt[cur].as<int32_t>();
      pa.q_cnt_pass = b.q_cnt_pass.as<int32_t>();
      pa.item_off = b.item_off.as<int32_t>();
      pa.plan = &ctrl->plan;
      pa.work = &ctrl->work;
      pa.q_cnt_nxt = b.q_cnt[cur ^ 1].as<int32_t>();
      pa.act_cnt_nxt = &ctrl->act_cnt[cur ^ 1];
      pa.near_cnt_nxt = &ctrl->near_cnt[cur ^ 1];
      if (cert) {
        pa.fq_cnt_nxt = b.fq_cnt[cur ^ 1].as<int32_t>();
        pa.ref_cnt_nxt = &ctrl->ref_cnt[cur ^ 1];
      }
      if (dif_on) pa.dq_cnt_nxt = b.dq_cnt[cur ^ 1].as<int32_t>();
      pa.round_ctr = &ctrl->round;
      pa.stat_queries = &ctrl->stat_queries;
      pa.stat_pairs = &ctrl->stat_pairs;
      launch_plan_round(pa, cs);
      G1Args ga{};
      ga.probs = b.probs.as<ProbDesc>();
      ga.nprob = nprob;
      ga.plan = &ctrl->plan;
      ga.item_off = b.item_off.as<int32_t>();
      ga.q_cnt = b.q_cnt_pass.as<int32_t>();
      ga.work = &ctrl->work;
      ga.qpos = b.qpos[cur].as<float4>();
      ga.qlam = b.qlam[cur].as<Lam4>();
      ga.out = b.out.as<double>();
      ga.err = c->err.as<unsigned>();
      // External event records become event-record nodes of the graph (plain records inside a
      // capture only order work and are never timestamped).
      if (c->profiling) CUDA_TRY(cudaEventRecordWithFlags(b.ev[6 * r], cs, cudaEventRecordExternal));
      DBIE_TRY(launch_kernel(k, grid, &ga, cs));
      if (c->profiling)
        CUDA_TRY(cudaEventRecordWithFlags(b.ev[6 * r + 1], cs, cudaEventRecordExternal));
      if (near_on)
        launch_nearfield(var, tied, b.probs.as<ProbDesc>(), b.near[cur].as<int32_t>(),
                         &ctrl->near_cnt[cur], b.qpos[cur].as<float4>(), b.qlam[cur].as<Lam4>(),
                         &ctrl->plan, b.item_off.as<int32_t>(), b.out.as<double>(),
                         2 * c->sm_count, cs);
      (qn ? launch_bfgs_step : launch_nm_step)(sa[cur], nm_grid, cs);
      if (cert) {
        // the near-tied values of this round in float-float, then those queued as differences
        // from the points' references, then the waiting steps again
        DBIE_TRY(record_reeval(cs, kf, grid_ff, target_ff, b.fq_cnt[cur], b.fq_cnt_pass,
                               b.fitem_off, &ctrl->fplan, &ctrl->fwork, &ctrl->stat_ff_pairs,
                               b.fpos[cur], b.flam[cur], nullptr, b.fout, 6 * r + 2));
        if (dif_on)
          DBIE_TRY(record_reeval(cs, kd, grid_dif, target_dif, b.dq_cnt[cur], b.dq_cnt_pass,
                                 b.ditem_off, &ctrl->dplan, &ctrl->dwork, &ctrl->stat_dif_pairs,
                                 b.dpos[cur], b.dlam[cur], &b.dlam0[cur], b.dout, 6 * r + 4));
        launch_nm_refine(sa[cur], nm_grid, cs);
      }
    }
    CUDA_TRY(cudaGetLastError());
    return DBIE_OK;
  };
  if (c->profiling && b.ev.size() != 6 * K) {
    for (cudaEvent_t e : b.ev) cudaEventDestroy(e);
    b.ev.assign(6 * K, nullptr);
    for (auto& e : b.ev) CUDA_TRY(cudaEventCreate(&e));
  }
  // Capture (or reuse) the graph of K rounds; the key is every launch argument.
  std::vector<unsigned char> key(sizeof sa + sizeof(KernelRef) + 3 * sizeof(int));
  {
    unsigned char* kp = key.data();
    std::memcpy(kp, sa, sizeof sa);
    std::memcpy(kp + sizeof sa, &k, sizeof k);
    const int extra[3] = {grid, nm_grid, (c->profiling ? 1 : 0) | (qn ? 2 : 0) | (cert ? 4 : 0)};
    std::memcpy(kp + sizeof sa + sizeof k, extra, sizeof extra);
  }
  if (!b.exec || b.key != key) {
    if (b.exec) cudaGraphExecDestroy(b.exec);
    b.exec = nullptr;
    CUDA_TRY(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    dbie_status st = record_rounds(c->cap_stream);
    cudaGraph_t graph = nullptr;
    cudaError_t ce = cudaStreamEndCapture(c->cap_stream, &graph);
    if (st != DBIE_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (ce != cudaSuccess) return fail(DBIE_ECUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
    ce = cudaGraphInstantiate(&b.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) return fail(DBIE_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ce));
    b.key = key;
  }
  // Rounds a point can take: the simplex spends at most 3 per iteration; the quasi-Newton search
  // at most 31 line-search trials (alpha = 1 ... 2^-30) per accepted step.
  // A certified step waits at most once per value it compares (4 vertices, the trial and the
  // reflected point), each re-evaluation removing one bound; twice with the difference level
  // (a difference value that ties again goes to float-float).
  const int max_rounds = (qn ? 31 : (dif_on ? 39 : (cert ? 21 : 3))) * o.max_iter + (cert ? 26 : 8);
  const int max_launches = max_rounds / K + 2;
  int launches = 0;
  for (;;) {
    CUDA_TRY(cudaGraphLaunch(b.exec, s));
    CUDA_TRY(cudaMemcpyAsync(c->pinned, &ctrl->act_cnt[0], sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    c->pinned[1] = 0;
    if (cert)
      CUDA_TRY(cudaMemcpyAsync(c->pinned + 1, &ctrl->ref_cnt[0], sizeof(int32_t),
                               cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    ++launches;
    if (c->profiling) {
      for (int r = 0; r < K; ++r) {
        float ms = 0.f;
        const cudaError_t te = cudaEventElapsedTime(&ms, b.ev[6 * r], b.ev[6 * r + 1]);
        float ms_ff = 0.f, ms_dif = 0.f;
        const cudaError_t tf = cert ? cudaEventElapsedTime(&ms_ff, b.ev[6 * r + 2], b.ev[6 * r + 3])
                                    : cudaSuccess;
        const cudaError_t td =
            dif_on ? cudaEventElapsedTime(&ms_dif, b.ev[6 * r + 4], b.ev[6 * r + 5]) : cudaSuccess;
        if (te == cudaSuccess && tf == cudaSuccess && td == cudaSuccess) {
          c->stats.kernel_ms += ms;
          c->stats.objective_ms += ms;
          c->stats.refine_ms += ms_ff;
          c->stats.dif_ms += ms_dif;
          c->stats.launches += 1;
        } else {
          (void)cudaGetLastError();  // timing unavailable: not an error of the solve
          if (std::getenv("DBIE_DEBUG"))
            std::fprintf(stderr, "dbie: graph event timing failed: %s\n", cudaGetErrorString(te));
        }
      }
    }
    DBIE_TRY(check_device_error(c, s));
    if (c->pinned[0] == 0 && c->pinned[1] == 0) break;
    if (launches >= max_launches) return fail(DBIE_EINTERNAL, "lambda-search rounds did not terminate");
  }
  // Certified B: the final field of every point whose error bound does not certify 1e-5
  // relative (the cancellation-dominated points) again, in float-float at lambda* (side 0 is the
  // current side after an even number of rounds).
  if (cert) {
    const KernelRef kv = g1_ref_ff(VAR_V, tied);
    CUDA_TRY(cudaMemsetAsync(b.fq_cnt[0].p, 0, sizeof(int32_t) * nprob, s));
    CUDA_TRY(cudaMemsetAsync(&ctrl->ref_cnt[0], 0, sizeof(int32_t), s));
    launch_certb_flag(sa[0], 1e-5, (int)std::min<int64_t>((N + 127) / 128, 8LL * c->sm_count), s);
    PlanArgs pf{};
    pf.probs = b.probs.as<ProbDesc>();
    pf.nprob = nprob;
    pf.qper = kv.qper;
    pf.target_items = std::max(1, 2 * persistent_grid(kv, c->device));
    pf.nsplit_cap = 1 << 20;
    pf.q_cnt_cur = b.fq_cnt[0].as<int32_t>();
    pf.q_cnt_pass = b.fq_cnt_pass.as<int32_t>();
    pf.item_off = b.fitem_off.as<int32_t>();
    pf.plan = &ctrl->fplan;
    pf.work = &ctrl->fwork;
    launch_plan_round(pf, s);
    G1Args gf{};
    gf.probs = b.probs.as<ProbDesc>();
    gf.nprob = nprob;
    gf.plan = &ctrl->fplan;
    gf.item_off = b.fitem_off.as<int32_t>();
    gf.q_cnt = b.fq_cnt_pass.as<int32_t>();
    gf.work = &ctrl->fwork;
    gf.qpos = b.fpos[0].as<float4>();
    gf.qlam = b.flam[0].as<Lam4>();
    gf.out = b.fout.as<double>();
    gf.err = c->err.as<unsigned>();
    DBIE_TRY(launch_kernel(kv, persistent_grid(kv, c->device), &gf, s));
    launch_certb_apply(sa[0], nm_grid, s);
    CUDA_TRY(cudaGetLastError());
    DBIE_TRY(check_device_error(c, s));
  }
  // Statistics and outputs.
  SolveCtrl hc;
  CUDA_TRY(cudaMemcpy(&hc, ctrl, sizeof hc, cudaMemcpyDeviceToHost));
  c->stats.rounds += hc.round;
  c->stats.queries += (int64_t)hc.stat_queries;
  c->stats.ties += (int64_t)hc.stat_ties;
  c->stats.refine_pairs += hc.stat_ff_pairs;
  c->stats.difs += (int64_t)hc.stat_difs;
  c->stats.dif_pairs += hc.stat_dif_pairs;
  if (cert) c->stats.b_refined += hc.ref_cnt[0];
  if (c->profiling) {
    c->stats.pair_evals += hc.stat_pairs;
    c->stats.objective_pairs += hc.stat_pairs;
  }
  const cudaMemcpyKind kind = mem_kind == DBIE_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  for (int p = 0; p < nprob; ++p) {
    const int64_t np = n[p], off = pt_off[p];
    if (np == 0) continue;
    const dbie_solve_out& so = out[p];
    CUDA_TRY(cudaMemcpyAsync(so.B, res_B + 3 * off, sizeof(double) * 3 * np, kind, s));
    CUDA_TRY(cudaMemcpyAsync(so.lambda, res_lam + 3 * off, sizeof(double) * 3 * np, kind, s));
    if (so.f) CUDA_TRY(cudaMemcpyAsync(so.f, res_f + off, sizeof(double) * np, kind, s));
    if (so.g) CUDA_TRY(cudaMemcpyAsync(so.g, res_g + off, sizeof(double) * np, kind, s));
    if (so.iters) CUDA_TRY(cudaMemcpyAsync(so.iters, res_i + off, sizeof(int32_t) * np, kind, s));
    if (so.status) CUDA_TRY(cudaMemcpyAsync(so.status, res_i + N + off, sizeof(int32_t) * np, kind, s));
    if (so.nfev) CUDA_TRY(cudaMemcpyAsync(so.nfev, res_i + 2 * N + off, sizeof(int32_t) * np, kind, s));
    if (so.codes && so.codes_stride > 0) {
      const int w = std::min<int>(so.codes_stride, codes_stride);
      if (mem_kind == DBIE_MEM_HOST) std::memset(so.codes, 0, (size_t)so.codes_stride * np);
      else CUDA_TRY(cudaMemsetAsync(so.codes, 0, (size_t)so.codes_stride * np, s));
      if (w > 0)
        CUDA_TRY(cudaMemcpy2DAsync(so.codes, so.codes_stride, b.codes.as<char>() + off * codes_stride,
                                   codes_stride, w, np, kind, s));
    }
  }
  CUDA_TRY(cudaStreamSynchronize(s));
  return DBIE_OK;
}

dbie_status dbie_solve(dbie_ctx* c, int64_t n, const float* xyz, const dbie_options* opt,
                       const double* lambda_init, int32_t mem_kind, const dbie_solve_out* out,
                       void* stream) {
  if (!c) return fail(DBIE_EINVAL, "ctx is NULL");
  DBIE_TRY(check_mem(mem_kind));
  if (n < 0) return fail(DBIE_EINVAL, "n must be >= 0");
  if (!out) return fail(DBIE_EINVAL, "out must not be NULL");
  if (n > 0 && (!xyz || !out->B || !out->lambda))
    return fail(DBIE_EINVAL, "xyz, out->B and out->lambda are required");
  const double* li[1] = {lambda_init};
  return solve_impl(1, &c, &n, &xyz, opt, li, mem_kind, out, static_cast<cudaStream_t>(stream));
}

dbie_status dbie_solve_batched(int32_t nprob, dbie_ctx* const* ctxs, const int64_t* n,
                               const float* const* xyz, const dbie_options* opt,
                               const double* const* lambda_init, int32_t mem_kind,
                               const dbie_solve_out* out, void* stream) {
  if (nprob < 1) return fail(DBIE_EINVAL, "nprob must be >= 1");
  if (!ctxs || !n || !xyz || !out) return fail(DBIE_EINVAL, "ctxs, n, xyz, out must not be NULL");
  DBIE_TRY(check_mem(mem_kind));
  for (int p = 0; p < nprob; ++p) {
    if (!ctxs[p]) return fail(DBIE_EINVAL, "ctxs[" + std::to_string(p) + "] is NULL");
    if (ctxs[p]->device != ctxs[0]->device) return fail(DBIE_EINVAL, "contexts on different devices");
    if (n[p] < 0) return fail(DBIE_EINVAL, "n[" + std::to_string(p) + "] < 0");
    if (n[p] > 0 && !xyz[p]) return fail(DBIE_EINVAL, "xyz[" + std::to_string(p) + "] is NULL");
    if (n[p] > 0 && (!out[p].B || !out[p].lambda))
      return fail(DBIE_EINVAL, "out[p].B and out[p].lambda are required");
  }
  return solve_impl(nprob, ctxs, n, xyz, opt, lambda_init, mem_kind, out,
                    static_cast<cudaStream_t>(stream));
}

#if DBIE_TRACE_ITEMS
// Debugging aid of DBIE_TRACE_ITEMS builds (not part of the ABI): copies the item timeline of the
// context's last single pair-sum pass (3 uint64 per item: start ns, end ns, SM | CTA << 16) to
// host memory and returns the item count, or -1.
int64_t dbie_debug_item_trace(dbie_ctx* c, unsigned long long* dst, int64_t max_items) {
  if (!c || !dst || !c->trace.p) return -1;
  const int64_t n = std::min<int64_t>(max_items, c->trace_items);
  if (cudaMemcpy(dst, c->trace.p, sizeof(unsigned long long) * 3 * n, cudaMemcpyDeviceToHost) !=
      cudaSuccess)
    return -1;
  return n;
}
#endif

dbie_status dbie_set_profiling(dbie_ctx* c, int32_t enable) {
  if (!c) return fail(DBIE_EINVAL, "ctx is NULL");
  c->profiling = enable != 0;
  return DBIE_OK;
}

dbie_status dbie_get_stats(dbie_ctx* c, dbie_stats* st, int32_t reset) {
  if (!c || !st) return fail(DBIE_EINVAL, "ctx and stats must not be NULL");
  CUDA_TRY(cudaSetDevice(c->device));
  resolve_pending(c);
  *st = c->stats;
  if (reset) c->stats = dbie_stats{};
  return DBIE_OK;
}

dbie_status dbie_autotune(dbie_ctx* c, void* stream) {
  if (!c) return fail(DBIE_EINVAL, "ctx is NULL");
  CUDA_TRY(cudaSetDevice(c->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // Synthetic queries over the context's own boundary: points above the field of view at
  // 1..16 pixels, lambda of the order of 1 / (box size); a fixed linear congruential sequence.
  const int64_t n = std::min<int64_t>(131072, std::max<int64_t>(8192, 16LL * c->sm_count * 128));
  std::vector<float> xyz(3 * n), lamf(3 * n);
  std::vector<double> lamd(3 * n), gB(3 * n);
  uint64_t st = 0x9E3779B97F4A7C15ull;
  auto rnd = [&]() {
    st = st * 6364136223846793005ull + 1442695040888963407ull;
    return (double)(st >> 11) * (1.0 / 9007199254740992.0);
  };
  const double L = std::max(c->nx * c->hx, c->ny * c->hy);
  for (int64_t i = 0; i < n; ++i) {
    xyz[3 * i] = (float)(c->x0 + rnd() * (c->nx - 1) * c->hx);
    xyz[3 * i + 1] = (float)(c->y0 + rnd() * (c->ny - 1) * c->hy);
    xyz[3 * i + 2] = (float)(c->hx * (1.0 + 15.0 * rnd()));
    for (int p = 0; p < 3; ++p) {
      lamd[3 * i + p] = (rnd() - 0.5) * 4.0 / L;
      lamf[3 * i + p] = (float)lamd[3 * i + p];
      gB[3 * i + p] = rnd() - 0.5;
    }
  }
  DBuf buf;
  const size_t bytes = align256(12 * n) * 2 + align256(24 * n) * 2 + align256(24 * c->npix);
  CUDA_TRY(cudaMalloc(&buf.p, bytes));
  buf.cap = bytes;
  Staging sg{0, buf.as<char>()};
  float* d_xyz = sg.take<float>(3 * n);
  float* d_lamf = sg.take<float>(3 * n);
  double* d_lamd = sg.take<double>(3 * n);
  double* d_gB = sg.take<double>(3 * n);
  double* d_gB0 = sg.take<double>(3 * c->npix);
  cudaError_t ce = cudaMemcpyAsync(d_xyz, xyz.data(), 12 * n, cudaMemcpyHostToDevice, s);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(d_lamf, lamf.data(), 12 * n, cudaMemcpyHostToDevice, s);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(d_lamd, lamd.data(), 24 * n, cudaMemcpyHostToDevice, s);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(d_gB, gB.data(), 24 * n, cudaMemcpyHostToDevice, s);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  if (ce != cudaSuccess) {
    buf.release();
    return fail(DBIE_ECUDA, std::string("autotune staging: ") + cudaGetErrorString(ce));
  }
  dbie_options o;
  dbie_default_options(&o);
  o = resolved(c, &o);
  const bool prof = c->profiling;
  c->profiling = true;
  dbie_status status = DBIE_OK;
  const int pairs[9][2] = {{VAR_OBJ, 0},  {VAR_OBJ, 1},  {VAR_V, 0},    {VAR_VL, 0},
                           {VAR_OBJL, 0}, {VAR_OBJN, 0}, {VAR_OBJN, 1}, {VAR_HESS, 0},
                           {VAR_NV, 0}};
  if (c->quad_g == 0) status = stage_variance(c, nullptr, nullptr, nullptr, 1.0, s);
  for (const auto& vt : pairs) {
    if (status != DBIE_OK) break;
    const int var = vt[0], tied = vt[1];
    if (var == VAR_NV && c->quad_g != 0) continue;   // noise variance: pixel-centre rule only
    const std::string key = tune_key(c->device, "g1", var, tied, c->nquad);
    const int cached = tune_lookup(key);
    if (cached >= 0) {
      c->cfg[var][tied] = cached;
      continue;
    }
    int best = 0;
    double best_ms = 1e30;
    for (int cfg = 0; cfg < NCFG && status == DBIE_OK; ++cfg) {
      c->cfg[var][tied] = cfg;
      double ms = 0;
      status = time_min(c, 3, [&]() {
        return pass_single(c, var, false, o, n, d_xyz, d_lamf, nullptr, s, tied != 0);
      }, &ms);
      if (ms < best_ms) { best_ms = ms; best = cfg; }
    }
    c->cfg[var][tied] = best;
    if (status == DBIE_OK) tune_store(key, best);
  }
  {
    const std::string key = tune_key(c->device, "vjp", 0, 0, c->nquad);
    const int cached = tune_lookup(key);
    if (cached >= 0) {
      c->vjp_cfg = cached;
    } else {
      int best = 0;
      double best_ms = 1e30;
      for (int cfg = 0; cfg < NCFG && status == DBIE_OK; ++cfg) {
        c->vjp_cfg = cfg;
        double ms = 0;
        status = time_min(c, 3, [&]() {
          return dbie_vjp(c, n, d_xyz, d_lamd, d_gB, &o, DBIE_MEM_DEVICE, d_gB0, nullptr, 0, s);
        }, &ms);
        if (ms < best_ms) { best_ms = ms; best = cfg; }
      }
      c->vjp_cfg = best;
      if (status == DBIE_OK) tune_store(key, best);
    }
  }
  c->profiling = prof;
  cudaStreamSynchronize(s);
  buf.release();
  return status;
}

dbie_status dbie_set_config(dbie_ctx* c, const int32_t* cfg_in) {
  if (!c || !cfg_in) return fail(DBIE_EINVAL, "ctx and cfg_in must not be NULL");
  for (int i = 0; i < 2 * NVAR + 1; ++i)
    if (cfg_in[i] < 0 || cfg_in[i] >= NCFG) return fail(DBIE_EINVAL, "configuration index out of range");
  for (int v = 0; v < NVAR; ++v)
    for (int t = 0; t < 2; ++t) c->cfg[v][t] = cfg_in[2 * v + t];
  c->vjp_cfg = cfg_in[2 * NVAR];
  return DBIE_OK;
}

dbie_status dbie_get_config(dbie_ctx* c, int32_t* cfg_out) {
  if (!c || !cfg_out) return fail(DBIE_EINVAL, "ctx and cfg_out must not be NULL");
  for (int v = 0; v < NVAR; ++v)
    for (int t = 0; t < 2; ++t) cfg_out[2 * v + t] = c->cfg[v][t];
  cfg_out[2 * NVAR] = c->vjp_cfg;
  return DBIE_OK;
}

}  // extern "C"
