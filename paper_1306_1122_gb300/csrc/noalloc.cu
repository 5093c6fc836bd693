// noalloc.cu -- dbie_eval_noalloc: field evaluation that allocates no memory.
//
// Who needs it: callers that may not allocate device memory while they run -- code that
// executes inside another framework's memory pool or arena (where a cudaMalloc would bypass
// the pool's accounting and can fail or fragment it), real-time loops where an allocation's
// implicit device synchronisation would stall the pipeline, and plugin hosts that forbid
// allocations from third-party libraries.  dbie_create allocates the context's copies and
// scratch, so such callers cannot use dbie_eval; this entry point takes the magnetogram and the
// points directly and keeps all of its scratch in one fixed file-scope device array.
//
// The array (kScratchBytes) is part of the library image: every GPU that loads the library holds
// it until the process exits.  All calls share it and it keeps the previous call's contents, so
// the counters that must start at zero are cleared by every call, and calls whose work overlaps
// on the GPU (different streams, or several host threads) race on it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "dbie.h"
#include "kernels.h"

using namespace dbie;

namespace {

constexpr int64_t kMaxPixels = 65536;          // largest magnetogram (nx * ny)
constexpr int64_t kMaxPoints = 65536;          // largest point count per call
constexpr size_t kScratchBytes = 16u << 20;    // 16 MiB

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct Ctl {  // counters and plan of one call (cleared by every call)
  PlanHdr plan;
  int32_t item_off[2];
  int32_t q_cnt[1];
  int32_t work;
  int32_t near_cnt;
  uint32_t err;
  int32_t pad[2];
};

constexpr size_t align256(size_t b) { return (b + 255) & ~size_t(255); }
constexpr int64_t kMaxTiles = (kMaxPixels + TILE - 1) / TILE;
constexpr size_t kOffCtl = 0;
constexpr size_t kOffProb = align256(sizeof(Ctl));
constexpr size_t kOffT32 = kOffProb + align256(sizeof(ProbDesc));
constexpr size_t kOffT64 = kOffT32 + align256(sizeof(float) * NFIELD * TILE * kMaxTiles);
constexpr size_t kOffQpos = kOffT64 + align256(sizeof(double) * NFIELD * TILE * kMaxTiles);
constexpr size_t kOffQlam = kOffQpos + align256(sizeof(float4) * kMaxPoints);
constexpr size_t kOffNear = kOffQlam + align256(sizeof(Lam4) * kMaxPoints);
constexpr size_t kOffOut = kOffNear + align256(sizeof(int32_t) * kMaxPoints);
// Largest queries-per-CTA over the launch configurations (the call uses configuration 0).
constexpr int64_t max_qper() {
  int64_t m = 0;
  for (int c = 0; c < NCFG; ++c) m = std::max<int64_t>(m, (int64_t)cfg_of(c).p * cfg_of(c).nt);
  return m;
}
// The output region must hold at least one split of the largest call (3 sums per query, the
// query count rounded up to whole CTAs); with less, nsplit would be forced below 1.
static_assert(kOffOut < kScratchBytes, "scratch layout does not fit");
static_assert(kScratchBytes - kOffOut >= sizeof(double) * 3 * (kMaxPoints + max_qper()),
              "scratch output region cannot hold one split of the largest call");

thread_local std::string t_err;
std::mutex g_mu;
void* g_addr[64] = {};    // device address of g_scratch, per device (set up on first use)
int g_grid[64] = {};      // persistent grid of the value kernel, per device

dbie_status err(dbie_status s, const std::string& m) {
  t_err = m;
  std::fprintf(stderr, "dbie_eval_noalloc: %s\n", m.c_str());
  return s;
}

}  // namespace

extern "C" dbie_status dbie_eval_noalloc(int32_t nx, int32_t ny, double x0, double y0, double hx,
                                         double hy, double pixel_area, const float* Bx,
                                         const float* By, const float* Bz, int64_t n,
                                         const float* xyz, const float* lambda, double* B,
                                         void* stream) {
  if (nx < 1 || ny < 1 || (int64_t)nx * ny > kMaxPixels)
    return err(DBIE_EINVAL, "nx * ny must be in [1, 65536]");
  if (n < 0 || n > kMaxPoints) return err(DBIE_EINVAL, "n must be in [0, 65536]");
  if (!(hx > 0) || !(hy > 0) || !(pixel_area > 0) || !std::isfinite(hx) || !std::isfinite(hy) ||
      !std::isfinite(pixel_area) || !std::isfinite(x0) || !std::isfinite(y0))
    return err(DBIE_EINVAL, "grid spacing and pixel area must be finite and > 0");
  if (!Bx || !By || !Bz) return err(DBIE_EINVAL, "Bx, By, Bz must not be NULL");
  if (n > 0 && (!xyz || !lambda || !B)) return err(DBIE_EINVAL, "xyz, lambda, B must not be NULL");
  if (n == 0) return DBIE_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
    return err(DBIE_ECUDA, "no usable current device");

  // Set-up, once per device, with that device current: the device address of the scratch array
  // (host code may not use the symbol itself) and the value kernel's resident grid.
  const KernelRef k = g1_ref_f32(VAR_V, false, 0, false);
  char* base = nullptr;
  int grid = 0;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
      if (e != cudaSuccess || !p)
        return err(DBIE_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      int per_sm = 0, sms = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k.fn, k.nt, k.smem) !=
              cudaSuccess ||
          cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return err(DBIE_ECUDA, "occupancy query failed");
      g_grid[dev] = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
      g_addr[dev] = p;
    }
    base = static_cast<char*>(g_addr[dev]);
    grid = g_grid[dev];
  }
  Ctl* ctl = reinterpret_cast<Ctl*>(base + kOffCtl);
  ProbDesc* prob = reinterpret_cast<ProbDesc*>(base + kOffProb);
  float* t32 = reinterpret_cast<float*>(base + kOffT32);
  double* t64 = reinterpret_cast<double*>(base + kOffT64);
  float4* qpos = reinterpret_cast<float4*>(base + kOffQpos);
  Lam4* qlam = reinterpret_cast<Lam4*>(base + kOffQlam);
  int32_t* near = reinterpret_cast<int32_t*>(base + kOffNear);
  double* out = reinterpret_cast<double*>(base + kOffOut);

  const int64_t npix = (int64_t)nx * ny;
  const int ntiles = (int)((npix + TILE - 1) / TILE);
  const int64_t nblk = (n + k.qper - 1) / k.qper;
  const int64_t max_items = (int64_t)((kScratchBytes - kOffOut) / (sizeof(double) * 3 * k.qper));
  if (nblk > max_items) return err(DBIE_EINTERNAL, "scratch output region too small for this call");
  int64_t nsplit = 1;
  const int64_t target = 2LL * grid;
  if (nblk < target) nsplit = std::min<int64_t>((target + nblk - 1) / nblk, ntiles);
  nsplit = std::max<int64_t>(1, std::min<int64_t>(nsplit, max_items / nblk));
  const int64_t nitems = nblk * nsplit;

  // Same defaults as dbie_eval with opt = NULL: FP64 near field for z <= 2 hx.
  const double near_z = 2.0 * hx;
  ProbDesc pd{};
  pd.tiles32 = t32;
  pd.tiles64 = t64;
  pd.ntiles = ntiles;
  pd.nx = nx;
  pd.ny = ny;
  pd.near_w = NEAR_W;
  pd.x0 = x0; pd.y0 = y0; pd.hx = hx; pd.hy = hy;
  // Everything that must start at zero (counters, error word) is cleared here.
  if (cudaMemsetAsync(ctl, 0, sizeof(Ctl), s) != cudaSuccess ||
      cudaMemcpyAsync(prob, &pd, sizeof pd, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return err(DBIE_ECUDA, "control block set-up failed");
  launch_stage_boundary(Bx, By, Bz, nx, ny, x0, y0, hx, hy, pixel_area / TWO_PI, ntiles, t32, t64, s);
  launch_pack_eval(n, xyz, lambda, nullptr, qpos, qlam, near, &ctl->near_cnt, 1, near_z, s);
  launch_plan_single(&ctl->plan, ctl->item_off, ctl->q_cnt, &ctl->work, (int)nitems, (int)nsplit,
                     k.qper, (int)n, s);
  G1Args a{};
  a.probs = prob;
  a.nprob = 1;
  a.plan = &ctl->plan;
  a.item_off = ctl->item_off;
  a.q_cnt = ctl->q_cnt;
  a.work = &ctl->work;
  a.qpos = qpos;
  a.qlam = qlam;
  a.out = out;
  a.err = &ctl->err;
  void* argv[1] = {&a};
  cudaError_t e = cudaLaunchKernel(k.fn, dim3(grid), dim3(k.nt), argv, k.smem, s);
  if (e != cudaSuccess) return err(DBIE_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
  int sms = 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  launch_nearfield(VAR_V, false, prob, near, &ctl->near_cnt, qpos, qlam, &ctl->plan,
                   ctl->item_off, out, 2 * sms, s);
  launch_finalize_eval(VAR_V, n, &ctl->plan, ctl->item_off, out, qpos, qlam, hx / 6.0, 1.0, B,
                       nullptr, nullptr, nullptr, nullptr, nullptr, s);
  e = cudaGetLastError();
  if (e != cudaSuccess) return err(DBIE_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
  // Synchronous: report a bounded-wait timeout of this call's kernels.
  uint32_t word = 0;
  if (cudaMemcpyAsync(&word, &ctl->err, sizeof word, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return err(DBIE_ECUDA, "synchronisation failed");
  if (word) return err(DBIE_ETIMEOUT, "a bounded device wait gave up");
  return DBIE_OK;
}
