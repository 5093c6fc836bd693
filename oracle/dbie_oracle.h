/*
 * dbie_oracle.h -- FP64 CPU oracle for the DBIE quadrature (TEST INFRASTRUCTURE ONLY).
 *
 * Plain, slow, obviously-correct restatement of the direct boundary integral equation of
 * Wang, Yan & Tan (Solar Phys., arXiv 1306.1122), Sect. 2.1, Eqs. 6, 8, 9, 13, 14, 16, and of the
 * per-point Downhill Simplex (Nelder & Mead 1965) search for the pseudo-force-free factor lambda.
 * Only tests, the package's smoke check and the benchmark's CPU-baseline leg may call this
 * library; the product path never does. It shares no code with the CUDA path.
 */
#ifndef DBIE_ORACLE_H
#define DBIE_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Bottom boundary (Eq. 3): an nx-by-ny magnetogram, pixel (i, j) centred at
 * (x0 + i*hx, y0 + j*hy, 0), row-major storage index j*nx + i, pixel area dA.
 * The field vanishes outside the magnetogram (Sect. 2.1). */
typedef struct {
  int32_t nx, ny;
  double x0, y0, hx, hy, dA;
  const float *Bx, *By, *Bz;
} orc_boundary;

/* Options of the lambda search (Sect. 2.1, Eqs. 8-12). */
typedef struct {
  double eps_f, eps_g;   /* stopping thresholds of Eq. 12 */
  double tol;            /* simplex value-spread tolerance */
  int32_t max_iter;      /* maximum number of simplex iterations */
  int32_t lambda_mode;   /* 0: three factors (lx, ly, lz) per point, 1: one shared factor */
  double simplex_step;   /* edge of the initial simplex */
  double w_g;            /* objective Phi = f + w_g * g */
  double g_scale;        /* Delta V_i / Delta sigma_i of Eq. 9 */
  int32_t deriv;         /* 0: analytic derivative at fixed lambda, 1: forward difference */
  double fd_delta;       /* difference step for deriv = 1 */
  int32_t method;        /* 0: Downhill Simplex (the paper), 1: quasi-Newton (orc_bfgs) from
                            lambda_init + simplex_step (1, 1, 1): Phi is even in each lambda_p,
                            so lambda = 0 itself is a stationary point */
  int32_t quad_order;    /* 0: midpoint rule at pixel centres (Eq. 16); g >= 1: nine-node
                            elements with g x g Gauss points each (Eq. 15, orc_field_q9);
                            -1: pixel-exact near field for z <= pxe_near_z (orc_field_pxe);
                            the simplex only */
  double pxe_near_z;
} orc_options;

/* Field and its derivatives at one point for a given lambda triple:
 *   B[p], G[p][j] = d B_p / d x_j (j = x, y, z), dBdl[p] = d B_p / d lambda_p. */
void orc_field(const orc_boundary* bd, double xi, double yi, double zi, const double lam[3],
               double B[3], double G[9], double dBdl[3]);

/* Same, with the spatial derivatives by first-order forward differences of step delta
 * taken at the same lambda (the zeroth-order rule of Eq. 13). */
void orc_field_fd(const orc_boundary* bd, double xi, double yi, double zi, const double lam[3],
                  double delta, double B[3], double G[9]);

/* As orc_field, plus the lambda-derivatives of the spatial derivatives:
 *   dGdl[p][j] = d^2 B_p / (d x_j d lambda_p). */
void orc_field_dl(const orc_boundary* bd, double xi, double yi, double zi, const double lam[3],
                  double B[3], double G[9], double dBdl[3], double dGdl[9]);

/* Force-freeness f (Eq. 8), divergence measure g (Eq. 9), J = curl B (Eq. 14), D = div B. */
void orc_objective(const double B[3], const double G[9], double g_scale, double w_g,
                   double* f, double* g, double* phi, double J[3], double* D);

/* Phi = f + w_g g and its gradient with respect to (lambda_x, lambda_y, lambda_z), by the chain
 * rule through B and its spatial derivatives (lambda_p moves only component p). */
void orc_objective_grad(const double B[3], const double G[9], const double dBdl[3],
                        const double dGdl[9], double g_scale, double w_g, double* f, double* g,
                        double* phi, double dphi[3]);

/* Generic Downhill Simplex in n dimensions (n <= 3).  fun(ctx, x, &flag) returns the
 * objective and sets flag != 0 when the point meets the problem's own stopping test. */
typedef double (*orc_fun)(void* ctx, const double* x, int32_t* flag);
typedef struct {
  double x[3];        /* best vertex */
  double fx;          /* its value */
  int32_t iters;      /* simplex iterations performed */
  int32_t nfev;       /* objective evaluations */
  int32_t status;     /* 0 converged, 1 iteration limit */
  int32_t ncodes;     /* number of step codes written */
} orc_nm_result;
void orc_nelder_mead(int32_t n, const double x0[3], double step, double tol, int32_t max_iter,
                     orc_fun fun, void* ctx, orc_nm_result* res, char* codes, int32_t codes_cap);
/* Same, from an explicit initial simplex sim[(n+1)*n]. */
void orc_nelder_mead_sim(int32_t n, const double* sim, double tol, int32_t max_iter,
                         orc_fun fun, void* ctx, orc_nm_result* res, char* codes, int32_t codes_cap);

/* Quasi-Newton (BFGS, Armijo backtracking) search for lambda at one point; not in the paper:
 * an alternative to the Downhill Simplex that uses the exact gradient of Phi.
 *   x_{k+1} = x_k + a d_k, d_k = -H_k grad Phi, a = 1, 1/2, 1/4, ... until
 *   Phi(x_k + a d_k) <= Phi(x_k) + 1e-4 a grad . d_k (at most 30 halvings), then the BFGS update
 *   of the inverse Hessian H (skipped unless s.y > 1e-12 |s||y|).  H_0 = I step / |grad Phi_0|
 *   (first step of length `step` along -grad), reset the same way when d is not a descent
 *   direction.  Stops on Eq. 12, on a decrease below tol, on grad = 0, when the line search
 *   fails, or after max_iter accepted steps. */
typedef double (*orc_fun_grad)(void* ctx, const double* x, double* grad, int32_t* flag);
void orc_bfgs(int32_t n, const double x0[3], double step, double tol, int32_t max_iter,
              orc_fun_grad fun, void* ctx, orc_nm_result* res);

/* Eq. 15: the boundary as nine-node biquadratic elements.  Element (ex, ey) spans nodes
 * 2ex..2ex+2 by 2ey..2ey+2 (nx, ny odd, >= 3), centred on node (2ex+1, 2ey+1) at (xc, yc); local
 * coordinates xi = (x - xc) / hx, eta = (y - yc) / hy in [-1, 1]; shape functions
 * N = L_a(xi) L_b(eta) with L_-1 = xi (xi - 1) / 2, L_0 = 1 - xi^2, L_+1 = xi (xi + 1) / 2;
 * Jacobian hx hy; each element integral by order x order Gauss-Legendre points.  The weights a_ik
 * of Eq. 16 then follow per node (orc_node_weights_q9) and B_i = sum_k a_ik B_k.  dA is not used.
 * gauss_legendre: nodes x[m] and weights w[m] on [-1, 1] (Newton's method on P_m). */
void orc_gauss_legendre(int32_t m, double* x, double* w);
/* Per node k (row-major, npix entries each): a_ik and its derivatives at fixed lambda,
 * out[5 k + 0..4] = {a, da/dx_i, da/dy_i, da/dz_i, da/dlambda}. */
void orc_node_weights_q9(const orc_boundary* bd, double xi, double yi, double zi, double lam,
                         int32_t order, double* out);
void orc_field_q9(const orc_boundary* bd, double xi, double yi, double zi, const double lam[3],
                  int32_t order, double B[3], double G[9], double dBdl[3]);
void orc_eval_many_q9(const orc_boundary* bd, int64_t n, const double* xyz, const double* lam,
                      int32_t order, double* B, double* G, double* dBdl, int32_t nthreads);
/* Transpose with the element weights: gB0[k][p] = sum_i gB_pi a_ik(lambda_pi). */
void orc_vjp_q9(const orc_boundary* bd, int64_t n, const double* xyz, const double* lam,
                const double* gB, int32_t order, double* gB0, int32_t nthreads);

/* Pixel-exact near field (the exact near-field integration of the lambda = 0 kernel):
 * for a point with z <= near_z the boundary is read as constant on each pixel rectangle
 * (hx x hy around the pixel centre), and the lambda = 0 part of the kernel, K0 = z / (2 pi r^3),
 * is integrated exactly over every pixel (the closed-form solid angle, orc_rect_exact), while the
 * lambda-dependent remainder z [lambda r sin(lambda r) + cos(lambda r) - 1] / (2 pi r^3) stays on
 * the midpoint rule of Eq. 16.  So B = B_midpoint(lambda) + sum_k B0_k (int_pixel K0 - dA K0(c_k)),
 * a correction that does not depend on lambda.  Points above near_z take the midpoint rule.
 * orc_rect_exact: the integral of K0 over [xa, xb] x [ya, yb] (corner minus point coordinates)
 * and its derivatives with respect to the point (out[1..3]: x_i, y_i, z_i).
 * orc_pxe_correction: the correction of B (3) and of dB_p/dx_j (9) at one point, whatever z. */
void orc_rect_exact(double xa, double xb, double ya, double yb, double z, double out[4]);
void orc_pxe_correction(const orc_boundary* bd, double xi, double yi, double zi, double dB[3],
                        double dG[9]);
void orc_field_pxe(const orc_boundary* bd, double xi, double yi, double zi, const double lam[3],
                   double near_z, double B[3], double G[9], double dBdl[3]);
void orc_eval_many_pxe(const orc_boundary* bd, int64_t n, const double* xyz, const double* lam,
                       double near_z, double* B, double* G, double* dBdl, int32_t nthreads);
void orc_vjp_pxe(const orc_boundary* bd, int64_t n, const double* xyz, const double* lam,
                 const double* gB, double near_z, double* gB0, int32_t nthreads);

/* Second order, by hyper-dual numbers through the whole quadrature (no difference step; not in
 * the paper).  At one point and lambda: Phi, its gradient grad[q] = dPhi/dlambda_q, the Hessian
 * H[3q+r] = d^2 Phi / dlambda_q dlambda_r and dBdl[p] = dB_p/dlambda_p.  lambda_mode = 1 (one
 * shared lambda): grad[0], H[0] and dBdl[p] = dB_p/dlambda are the derivatives along the shared
 * lambda, the other entries 0.  pxe_near_z > 0: B and grad B carry the pixel-exact correction
 * (orc_pxe_correction) at points with z <= pxe_near_z; <= 0: the midpoint rule. */
void orc_hessian(const orc_boundary* bd, double xi, double yi, double zi, const double lam[3],
                 int32_t lambda_mode, double g_scale, double w_g, double pxe_near_z, double* phi,
                 double grad[3], double H[9], double dBdl[3]);
void orc_hessian_many(const orc_boundary* bd, int64_t n, const double* xyz, const double* lam,
                      int32_t lambda_mode, double g_scale, double w_g, double pxe_near_z,
                      double* phi, double* grad, double* H, double* dBdl, int32_t nthreads);

/* Gradient of L(B) with respect to the magnetogram THROUGH the lambda search: lambda* is taken as
 * a stationary point of Phi (grad_lambda Phi = 0), so d(lambda*) / dB0 = -H^-1 d(grad_lambda Phi) / dB0
 * and, for gB = dL/dB (n, 3),
 *   gB0[k][p] = sum_i gB_pi a_ik(lambda_pi) - d/dB0_pk sum_i v_i . grad_lambda Phi_i,
 *   v_i = H_i^-1 dL/dlambda_i,  dL/dlambda_p = gB_p dB_p/dlambda_p (summed over p when tied).
 * v_out (n, 3, nullable) gets v per component; flags (n, nullable) is 1 where H is not positive
 * definite (that point keeps only the fixed-lambda term).  pxe_near_z as for orc_hessian: the
 * weights a_ik then include the pixel-exact correction at the points with z <= pxe_near_z. */
void orc_implicit_vjp(const orc_boundary* bd, int64_t n, const double* xyz, const double* lam,
                      const double* gB, int32_t lambda_mode, double g_scale, double w_g,
                      double pxe_near_z, double* gB0, double* v_out, int32_t* flags,
                      int32_t nthreads);

/* Noise propagation at fixed lambda: with independent zero-mean noise of standard deviation
 * s_p[k] on pixel k of component p (sx, sy, sz are (ny, nx); a NULL array means sigma0), B is
 * linear in B0 (Eq. 16), so Var B_p(r_i) = sum_k a_ik(lambda_pi)^2 s_p[k]^2.  var is (n, 3). */
void orc_noise_var(const orc_boundary* bd, int64_t n, const double* xyz, const double* lam,
                   const float* sx, const float* sy, const float* sz, double sigma0, double* var,
                   int32_t nthreads);

/* Batched entry points over n points (OpenMP over points when nthreads > 1). */
void orc_objective_many(const orc_boundary* bd, int64_t n, const double* xyz, const double* lam,
                        double g_scale, double w_g, double pxe_near_z, double* fgphi,
                        double* dphi, int32_t nthreads);
void orc_eval_many(const orc_boundary* bd, int64_t n, const double* xyz, const double* lam,
                   int32_t deriv, double fd_delta, double* B, double* G, double* dBdl,
                   int32_t nthreads);
void orc_solve_many(const orc_boundary* bd, int64_t n, const double* xyz, const orc_options* opt,
                    const double* lam0, double* lam, double* B, double* f, double* g,
                    double* phi, int32_t* iters, int32_t* nfev, int32_t* status,
                    char* codes, int32_t codes_stride, int32_t nthreads);
/* Boundary adjoint: gB0[k][p] = sum_i gB[i][p] * a_ik(lambda_pi), the transpose of Eq. 16. */
void orc_vjp(const orc_boundary* bd, int64_t n, const double* xyz, const double* lam,
             const double* gB, double* gB0, int32_t nthreads);

#ifdef __cplusplus
}
#endif
#endif
