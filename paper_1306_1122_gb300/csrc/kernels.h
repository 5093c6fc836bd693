// kernels.h -- host-side interface to the device kernels (launch wrappers and kernel lookup).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "solve.cuh"

namespace dbie {

// Launch configurations of the pair-sum kernels: points (or pixels) per thread, CTA size, and a
// minimum number of resident CTAs per SM (a register cap; 1 = none).  The autotuner picks one.
// The two capped shapes depend on the variant: the Hessian pass (30 compensated sums, ~250
// registers uncapped) is capped at 3 or 4 CTAs of 128 threads (168 or 128 registers), the others
// at 6 or 7 (80 or 72 registers).
constexpr int NCFG = 6;
constexpr int NSTAGE = 3;
struct LaunchCfg { int p, nt, minb; };
__host__ __device__ constexpr LaunchCfg cfg_of(int c, int var = -1) {
  return c == 0 ? LaunchCfg{1, 128, 1}
       : c == 1 ? LaunchCfg{2, 128, 1}
       : c == 2 ? LaunchCfg{1, 256, 1}
       : c == 3 ? LaunchCfg{1, 128, var == VAR_HESS ? 3 : 6}
       : c == 4 ? LaunchCfg{1, 64, 1}
                : LaunchCfg{1, 128, var == VAR_HESS ? 4 : 7};
}

struct KernelRef {
  const void* fn;     // __global__ function
  int nt;             // threads per CTA
  int qper;           // queries (or pixels) per CTA = nt * points per thread
  size_t smem;        // dynamic shared memory bytes
};

// rows: every aligned group of 4 quadrature points lies on one row (row length % 4 == 0)
KernelRef g1_ref_f32(int var, bool tied, int cfg, bool rows);   // pairsum_f32_*.cu
KernelRef g1_ref_f64(int var, bool tied);            // pairsum_f64.cu
KernelRef g1_ref_ff(int var, bool tied);             // pairsum_ff.cu (VAR_V, VAR_OBJ)
KernelRef g1_ref_dif(bool tied);                     // pairsum_dif.cu (objective sums)
void launch_stage_ff(const double* t64, int ntiles, float* tff, cudaStream_t s);
KernelRef vjp_ref(bool fp64, bool tied, int cfg);    // vjp.cu
KernelRef vjp7_ref(bool fp64, bool tied);            // vjp.cu (seven-weight adjoint)
// FP32 form over element Gauss points with float-pair positions (pairsum_f32_split.cu)
KernelRef g1_ref_f32_split(int var, bool tied, bool rows);
KernelRef vjp_ref_split(bool tied);
KernelRef vjp7_ref_split(bool tied);

// Gauss rule of the nine-node elements (Eq. 15): g points per side, abscissae and weights.
struct QuadInfo {
  int g;
  double gx[MAX_GAUSS], gw[MAX_GAUSS];
};

// aux.cu
void launch_stage_q9(const float* B0, int nx, int ny, double x0, double y0, double hx, double hy,
                     const QuadInfo& qi, int ntiles, float* t32, double* t64, cudaStream_t s);
void launch_q9_gather(const double* T, int nx, int ny, double hx, double hy, const QuadInfo& qi,
                      double* gB0, int accumulate, cudaStream_t s);
void launch_stage_boundary(const float* Bx, const float* By, const float* Bz, int nx, int ny,
                           double x0, double y0, double hx, double hy, double scale,
                           int ntiles, float* t32, double* t64, cudaStream_t s);
void launch_pack_eval(int64_t n, const float* xyz, const float* lam_f, const double* lam_d,
                      float4* qpos, Lam4* qlam, int32_t* near_list, int32_t* near_cnt,
                      int near_on, double near_z, cudaStream_t s);
void launch_plan_single(PlanHdr* plan, int32_t* item_off, int32_t* q_cnt, int32_t* work,
                        int nitems, int nsplit, int qper, int qcount, cudaStream_t s);
void launch_nearfield(int var, bool tied, const ProbDesc* probs, const int32_t* near_list,
                      const int32_t* near_cnt, const float4* qpos, const Lam4* qlam,
                      const PlanHdr* plan, const int32_t* item_off, double* out, int grid,
                      cudaStream_t s);
void launch_pack_vjp(int64_t n, const float* xyz, const double* lam, const double* gB, int tied,
                     int nptiles, float* p32, double* p64, int fp64, cudaStream_t s);
void launch_finalize_vjp(int64_t npix, const PlanHdr* plan, const double* out, double scale,
                         double* gB0, int accumulate, cudaStream_t s);

// pxe.cu (pixel-exact near field)
void launch_pxe_corr(bool fp64, const ProbDesc* probs, int64_t n, const float4* pos, double zmax,
                     double* corr, int grid, cudaStream_t s);
// chunks of near points per pixel; the partial buffer holds (nchunk + 1) * npix * 3 doubles (the
// extra part: the window pairs of the mixed form), the bin buffer 3 * pxe_bins + 1 + n int32
int pxe_adjoint_chunks(int64_t n, int64_t npix, int sm_count);
int64_t pxe_bins(int nx, int ny);
cudaError_t launch_pxe_adjoint(bool fp64, bool full, const ProbDesc* prob, int64_t n, int nx,
                               int ny, const float4* pos, double zmax, const double* w,
                               int32_t* list, int32_t* cnt, int32_t* bins, int nchunk,
                               double* part, double* gB0, cudaStream_t s);

void launch_count_bad(const float* a, int64_t n, int mode, int32_t* cnt, cudaStream_t s);
void launch_pack_points(int64_t n, const float* xyz, int pidx, float4* ppos, cudaStream_t s);

// solve.cu
// corr (nullable): per query the pixel-exact correction of B (3) and grad B (9), added after the
// sums are assembled.
void launch_finalize_eval(int var, int64_t n, const PlanHdr* plan, const int32_t* item_off,
                          const double* out, const float4* qpos, const Lam4* qlam, double g_scale,
                          double w_g, double* B, double* gradB, double* dBdl,
                          const double* gB_for_glam, double* fgphi, const double* corr,
                          cudaStream_t s);
void launch_finalize_objective(int64_t n, const PlanHdr* plan, const int32_t* item_off,
                               const double* out, const float4* qpos, const Lam4* qlam,
                               double g_scale, double w_g, double* fgphi, double* dphi, double* B,
                               const double* corr, cudaStream_t s);
// second_order.cu
void launch_finalize_hessian(int64_t n, const PlanHdr* plan, const int32_t* item_off,
                             const double* out, const float4* qpos, const Lam4* qlam, int dim,
                             double g_scale, double w_g, double* phi, double* grad, double* hess,
                             const double* corr, cudaStream_t s);
// corr as above; pxe_w (nullable, with corr): per point the 12 weights of the transposed
// correction, gB_p - dW/dB_p and -dW/d(dB_p/dx_j) with W = v . grad_lambda Phi (at 4 p + m).
void launch_implicit_weights(int64_t n, int nptiles, const PlanHdr* plan, const int32_t* item_off,
                             const double* out, const float4* qpos, const Lam4* qlam,
                             const double* gB, int dim, double g_scale, double w_g, float* p32,
                             double* p64, int fp64, double* v_out, int32_t* flags,
                             const double* corr, double* pxe_w, cudaStream_t s);
void launch_finalize_nv(int64_t n, const PlanHdr* plan, const int32_t* item_off, const double* out,
                        const float4* qpos, double* var, cudaStream_t s);
void launch_stage_variance(const float* sx, const float* sy, const float* sz, double sigma0,
                           int nx, int ny, double x0, double y0, double hx, double hy, double w,
                           int ntiles, float* t32, double* t64, cudaStream_t s);

void launch_bfgs_init(const SolveArgs& a, const double* lam_init, int grid, cudaStream_t s);
void launch_bfgs_step(const SolveArgs& a, int grid, cudaStream_t s);
void launch_solve_init(const SolveArgs& a, const double* lam_init, int grid, cudaStream_t s);
void launch_plan_round(const PlanArgs& a, cudaStream_t s);
void launch_nm_step(const SolveArgs& a, int grid, cudaStream_t s);
void launch_nm_refine(const SolveArgs& a, int grid, cudaStream_t s);
void launch_msc(const ProbDesc* probs, int64_t N, const float4* ppos, double* msc, double* msc0,
                int grid, cudaStream_t s);
void launch_dif_debug(int64_t n, const PlanHdr* plan, const int32_t* item_off, const double* out,
                      const Lam4* qlam, const Lam4* qlam0, const double* msc, const double* msc0,
                      int dim, double* dS, double* dS_bound, cudaStream_t s);
void launch_certb_flag(const SolveArgs& a, double rel, int grid, cudaStream_t s);
void launch_certb_apply(const SolveArgs& a, int grid, cudaStream_t s);

}  // namespace dbie
