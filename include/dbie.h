/*
 * dbie.h -- C ABI of the GB300 DBIE library (libdbie.so).
 *
 * The library evaluates the direct boundary integral equation (DBIE) of Wang, Yan & Tan
 * (Solar Phys., arXiv 1306.1122) for non-linear force-free coronal fields:
 *
 *   Eq. 6 / Eq. 16   B_p(r_i) = sum_k a_ik(lambda_pi) B_p0,k,  p = x, y, z,
 *                    a_ik = z_i [lambda r sin(lambda r) + cos(lambda r)] / (2 pi r^3) * dA,
 *                    r^2 = (x_k - x_i)^2 + (y_k - y_i)^2 + z_i^2,
 *
 * summed over every pixel k of the bottom-boundary magnetogram (Eq. 3; zero field outside it),
 * with the pixel-centre (midpoint) rule.  lambda_pi is the pseudo-force-free factor of point i
 * and component p (Sect. 2.1).  On top of the quadrature the library runs the paper's per-point
 * Downhill Simplex search for lambda (Sect. 2.1), minimising f (Eq. 8) and g (Eq. 9) with the
 * spatial derivatives of B taken at fixed lambda (the zeroth-order rule of Eq. 13), and the
 * adjoint of Eq. 16 for gradients.
 *
 * Conventions shared by every entry point:
 *  - Coordinates (x, y, z) and pixel spacings are in one length unit; lambda in 1/length;
 *    magnetic fields in any unit (the map is linear in B0).
 *  - Arrays of points are row-major (n, 3) float32: x, y, z per point; z must be > 0.
 *  - Magnetogram components are row-major (ny, nx) float32: element j*nx + i is the pixel
 *    centred at (x0 + i*hx, y0 + j*hy).
 *  - mem_kind says where EVERY pointer argument of that call lives: DBIE_MEM_HOST (ordinary or
 *    pinned host memory; the call copies in and out and returns when results are in place) or
 *    DBIE_MEM_DEVICE (device memory of the current CUDA device; the call is asynchronous on
 *    `stream` unless stated otherwise).
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).
 *  - The caller owns every buffer it passes; the library never frees caller memory.  The
 *    context owns copies of the boundary and its own scratch; dbie_destroy frees them.
 *  - Errors are returned as dbie_status; no exception crosses the ABI.  Argument errors are
 *    detected on the host before any launch.  dbie_last_error() gives a thread-local message.
 *    Device-side waits are bounded: a wait that does not complete sets an error word that the
 *    next synchronising call reports as DBIE_ETIMEOUT.
 */
#ifndef DBIE_H
#define DBIE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dbie_ctx dbie_ctx; /* opaque; created by dbie_create, owned by the library */

typedef enum {
  DBIE_OK = 0,
  DBIE_EINVAL = 1,     /* invalid argument (null pointer, n < 0, z <= 0, non-finite input ...) */
  DBIE_ENOMEM = 2,     /* device or host allocation failed */
  DBIE_ECUDA = 3,      /* a CUDA call failed; message from dbie_last_error() */
  DBIE_ETIMEOUT = 4,   /* a bounded device-side wait gave up (kernel returned early) */
  DBIE_EINTERNAL = 5   /* inconsistent internal state */
} dbie_status;

enum { DBIE_MEM_HOST = 0, DBIE_MEM_DEVICE = 1 };
enum { DBIE_PREC_MIXED = 0, DBIE_PREC_FP64 = 1, DBIE_PREC_FLOAT_FLOAT = 2 };
enum { DBIE_LAMBDA_PER_COMPONENT = 0, DBIE_LAMBDA_TIED = 1 };
/* Per-point result status of dbie_solve. */
enum { DBIE_PT_CONVERGED = 0, DBIE_PT_MAXITER = 1 };
/* Lambda search method of dbie_solve. */
enum { DBIE_METHOD_SIMPLEX = 0, DBIE_METHOD_QUASI_NEWTON = 1 };

/* Options of the lambda search (Sect. 2.1, Eqs. 8-12) and of the arithmetic.
 * Fill with dbie_default_options() and override fields. */
typedef struct {
  double eps_f;        /* Eq. 12 threshold on f (default 1e-3) */
  double eps_g;        /* Eq. 12 threshold on g (default 1e-4) */
  double tol;          /* stop when the simplex value spread max Phi - min Phi <= tol (1e-6) */
  int32_t max_iter;    /* maximum simplex iterations per point (default 50) */
  int32_t lambda_mode; /* DBIE_LAMBDA_PER_COMPONENT (lx, ly, lz; the paper) or DBIE_LAMBDA_TIED */
  double simplex_step; /* initial simplex edge; <= 0 selects 1 / (max(nx, ny) * hx) */
  double w_g;          /* objective Phi = f + w_g * g (default 1) */
  double g_scale;      /* Delta V_i / Delta sigma_i of Eq. 9; <= 0 selects hx / 6 */
  int32_t precision;   /* DBIE_PREC_MIXED (FP32 pair terms, compensated sums, FP64 near field
                          and FP64 reductions), DBIE_PREC_FP64 (FP64 throughout), or
                          DBIE_PREC_FLOAT_FLOAT (every pair term and sum as a pair of floats,
                          about 48 significant bits, on the FP32 pipe: FP64-grade sums at a
                          fraction of the FP64 pipe's cost; dbie_eval only, without dBdlam;
                          other entry points return DBIE_EINVAL) */
  int32_t method;      /* DBIE_METHOD_SIMPLEX (the paper's Downhill Simplex, default) or
                          DBIE_METHOD_QUASI_NEWTON (BFGS with Armijo backtracking on the exact
                          gradient dPhi/dlambda; not in the paper).  For the quasi-Newton method
                          max_iter counts accepted steps, tol bounds the decrease of Phi per step,
                          and the search starts at lambda_init + simplex_step (1, 1, 1) (Phi is even
                          in every lambda_p, so lambda_init = 0 itself is a stationary point). */
  double near_z;       /* mixed precision: points with z <= near_z get their near-field pixels
                          (a 7 x 7 window) summed in FP64; with DBIE_QUAD_PIXEL_EXACT also the
                          height up to which the exact near-field integration applies (both
                          precisions); < 0 selects 2 * hx, 0 disables */
  double certify;      /* mixed precision, Downhill Simplex: certified decisions.  Every simplex
                          comparison whose two Phi values differ by no more than `certify` times
                          the sum of their error bounds (a worst-case bound of the FP32-term sums,
                          from the point's absolute-value sums) re-evaluates those values in the
                          float-float form before the step is taken, so that the search takes the
                          decisions of sums accurate to ~1e-13 (those of the FP64 form up to its
                          own rounding); at the end, every point whose final B the bound does not
                          certify to 1e-5 relative (the cancellation-dominated points) gets its B
                          again in float-float at lambda*.  0 disables; default 0.02 (the largest measured gap of a
                          decision that the FP32-term sums flipped was 0.009 times that sum of
                          bounds).  Not used by the FP64 form or the quasi-Newton search. */
  double certify_ref;  /* certified decisions, second level: once a point has a float-float value
                          (its reference), near-tied values of that point that lie close to the
                          reference in lambda are first re-evaluated as the reference's sums plus
                          the difference sums of dbie_eval_difference, whose error bound shrinks
                          with |lambda - lambda_ref|; such a value is near-tied again when it is
                          within certify_ref times that bound (plus the other value's radius), and
                          then goes to float-float.  Without a reference, a near tie of two
                          mixed-form values re-evaluates the one with the larger bound in
                          float-float first.  0 disables the level (every near tie in
                          float-float); default 0.02 (the mixed form's band: on 16,384 ll128 and
                          2,048 ar512 points the search took the FP64 form's step sequence on
                          every point with it). */
} dbie_options;

/* Per-point outputs of dbie_solve; every pointer may be NULL except B and lambda. */
typedef struct {
  double* B;           /* (n, 3): field at the converged lambda */
  double* lambda;      /* (n, 3): |lambda*| per component (the kernel is even in lambda) */
  int32_t* iters;      /* (n): simplex iterations */
  int32_t* status;     /* (n): DBIE_PT_CONVERGED or DBIE_PT_MAXITER */
  double* f;           /* (n): Eq. 8 at lambda* */
  double* g;           /* (n): Eq. 9 at lambda* */
  int32_t* nfev;       /* (n): objective evaluations of the search.  With one shared lambda, a
                          reflection of the worst vertex through a best vertex at lambda = 0 is
                          counted but not computed: it is the worst vertex's mirror image, where
                          Phi (even in lambda) has that vertex's value */
  char* codes;         /* (n, codes_stride): simplex step codes R/E/O/I/S, NUL-padded */
  int32_t codes_stride;
  int32_t reserved0;
} dbie_solve_out;

/* Timing of the pair-sum kernels recorded while profiling is on (see dbie_set_profiling). */
typedef struct {
  int64_t launches;        /* pair-sum kernel launches timed */
  double kernel_ms;        /* summed CUDA-event time of those launches */
  double pair_evals;       /* point x pixel pairs they evaluated */
  double objective_pairs;  /* pairs of the 12-sum objective launches of dbie_solve */
  double objective_ms;     /* CUDA-event time of those launches */
  int64_t rounds;          /* simplex rounds run by dbie_solve calls */
  int64_t queries;         /* objective evaluations (points x trial lambdas) */
  int64_t ties;            /* certified decisions: near ties sent to float-float re-evaluation */
  double refine_pairs;     /* their point x pixel pairs (float-float form) */
  double refine_ms;        /* CUDA-event time of the float-float passes (while profiling) */
  int64_t b_refined;       /* certified decisions: points whose final B the error bound did not
                              certify to 1e-5 relative, re-evaluated in float-float at lambda* */
  int64_t difs;            /* certified decisions: near-tied values re-evaluated as differences
                              from the point's float-float reference (certify_ref) */
  double dif_pairs;        /* their point x pixel pairs */
  double dif_ms;           /* CUDA-event time of the difference passes (while profiling) */
} dbie_stats;

/* Fill `opt` with the defaults listed above. */
void dbie_default_options(dbie_options* opt);

/* Create a context holding one magnetogram (Eq. 3, Eq. 16 with a_ik's dA = pixel_area).
 *   nx, ny >= 1; hx, hy > 0; pixel_area > 0 (usually hx * hy); Bx, By, Bz: (ny, nx) float32,
 *   finite.  The boundary is copied (and pre-scaled by pixel_area / 2 pi) into the context; the
 *   caller may free its arrays after the call returns.  Synchronises `stream`.
 *   Errors: DBIE_EINVAL for bad sizes, null or non-finite data; DBIE_ENOMEM; DBIE_ECUDA. */
dbie_status dbie_create(dbie_ctx** out, int32_t nx, int32_t ny, double x0, double y0, double hx,
                        double hy, double pixel_area, const float* Bx, const float* By,
                        const float* Bz, int32_t mem_kind, void* stream);

/* Replace the magnetogram values of an existing context (same grid).  Used when B0 is a
 * variable (gradients through dbie_vjp).  Asynchronous for device memory. */
dbie_status dbie_set_boundary(dbie_ctx* ctx, const float* Bx, const float* By, const float* Bz,
                              int32_t mem_kind, void* stream);

/* Quadrature of the boundary integral for every later call on this context:
 *   order = 0: the midpoint rule at pixel centres, a_ik = K(r_ik) pixel_area (Eq. 16; default);
 *   order = g (1..8): Eq. 15's nine-node biquadratic elements.  Element (ex, ey) spans pixel
 *     centres 2ex..2ex+2 by 2ey..2ey+2 (nx, ny odd and >= 3: the nodes are the pixel centres and
 *     the integration domain is the rectangle they span), shape functions are products of the
 *     quadratic Lagrange polynomials on the element's local coordinates in [-1, 1], the Jacobian
 *     is hx hy, and each element integral uses g x g Gauss-Legendre points (pixel_area is not
 *     used).  The pair sums then run over the ((nx-1)/2 g) x ((ny-1)/2 g) Gauss points, each
 *     carrying the interpolated field times its weights; adjoints are gathered back to the
 *     nodes.  dbie_noise_var needs order 0.
 *   order = DBIE_QUAD_PIXEL_EXACT (-1): the midpoint rule plus the exact near-field integration
 *     of the lambda = 0 kernel (the closed-form solid angle of each pixel rectangle, Eq. 6 at
 *     lambda = 0).  At points with z <= opt->near_z the magnetogram is read as constant on each
 *     hx x hy pixel, z / (2 pi r^3) is integrated exactly over every pixel, and the
 *     lambda-dependent remainder z [lambda r sin(lambda r) + cos(lambda r) - 1] / (2 pi r^3)
 *     stays on the midpoint rule; this removes the midpoint rule's lattice error at small z.
 *     The correction of B and grad B does not depend on lambda (a solve computes it once per
 *     point), and it enters every call that returns B, grad B, Phi or an adjoint; dB/dlambda and
 *     the other lambda-derivatives are the midpoint rule's.  opt->near_z = 0 turns it off for a
 *     call.  dbie_noise_var is not available in this mode.
 * Restages the stored magnetogram; synchronises `stream`.  DBIE_EINVAL for an order outside
 * -1..8 or even / too small nx, ny with order > 0. */
#define DBIE_QUAD_PIXEL_EXACT (-1)
dbie_status dbie_set_quadrature(dbie_ctx* ctx, int32_t order, void* stream);

/* Evaluate Eq. 16 at n points for given lambda (n, 3) float32, and optionally
 *   gradB  (n, 9): gradB[9i + 3p + j] = d B_p / d x_j at fixed lambda (Eq. 13, delta -> 0),
 *   dBdlam (n, 3): d B_p / d lambda_p,
 *   fgphi  (n, 3): f (Eq. 8), g (Eq. 9), Phi = f + w_g g (needs gradB's sums; opt gives g_scale, w_g).
 * B is required when n > 0, the others may be NULL.  opt may be NULL (defaults; precision and near_z are
 * read from it).  n = 0 is a no-op.  With precision DBIE_PREC_FLOAT_FLOAT the sums agree with the
 * FP64 ones to about 1e-13 of their absolute-value sums (angles lambda r of 12,000 rad and more take
 * FP64 sine and cosine); dBdlam is then not available (DBIE_EINVAL). */
dbie_status dbie_eval(dbie_ctx* ctx, int64_t n, const float* xyz, const float* lambda,
                      const dbie_options* opt, int32_t mem_kind, double* B, double* gradB,
                      double* dBdlam, double* fgphi, void* stream);

/* Change of the 12 objective sums of Eq. 16 (per component p: S0 = sum u b / r^3, S1 = sum w b / r^3,
 * Sx, Sy = sum w b (x - x_k) / r^3, (y - y_k); u = theta sin(theta) + cos(theta),
 * w = lambda^2 cos(theta) - 3 u / r^2, theta = lambda_p r, b = B0_p dA / (2 pi); B_p = z S0,
 * dB_p/dx = z Sx, dB_p/dy = z Sy, dB_p/dz = S0 + z^2 S1) between lambda_ref and lambda, at n points.
 * Not in the paper: the re-evaluation step of certified simplex decisions.  The pair terms' changes
 * come from angle-sum identities (sin and cos of (lambda + lambda_ref) r / 2 and of
 * (lambda - lambda_ref) r / 2) in FP32, so their error is proportional to |lambda - lambda_ref|;
 * summed over 8-pixel FP32 blocks and then in float-float.  dS (n, 12): dS[12 i + 4 p + s] for
 * s = S0, S1, Sx, Sy.  dS_bound (n, 12) or NULL: a worst-case bound of each entry's error
 * (polynomial in |lambda - lambda_ref| and |lambda| + |lambda_ref| over sum |B0_p| dA / (2 pi r^j),
 * j = 0..5, plus 1e-12 of the sums at lambda_ref).  Device memory only: xyz (n, 3) float32,
 * lambda and lambda_ref (n, 3) float64; tied != 0 reads component 0 of each lambda for all three
 * components.  Every quadrature rule of the context (the pixel-exact near field adds nothing: it
 * does not depend on lambda).  Asynchronous on stream; n = 0 is a no-op. */
dbie_status dbie_eval_difference(dbie_ctx* ctx, int64_t n, const float* xyz, const double* lambda,
                                 const double* lambda_ref, int32_t tied, double* dS,
                                 double* dS_bound, void* stream);

/* f (Eq. 8), g (Eq. 9), Phi = f + w_g g (fgphi, (n, 3)) and the exact gradient dPhi/dlambda_p
 * (dphi, (n, 3); lambda_p moves component p of B and its spatial derivatives) at n points for
 * given lambda (n, 3) float32.  Either output may be NULL, not both.  Not in the paper: the
 * gradient used by the quasi-Newton search, exposed for callers' own optimisers. */
dbie_status dbie_objective(dbie_ctx* ctx, int64_t n, const float* xyz, const float* lambda,
                           const dbie_options* opt, int32_t mem_kind, double* fgphi, double* dphi,
                           void* stream);

/* Solve for lambda point by point (Sect. 2.1): Nelder-Mead on Phi(lambda) = f + w_g g from the
 * simplex lambda_init + simplex_step * e_j (lambda_init (n, 3) float64, NULL = 0), stopping on
 * Eq. 12, on the value spread tol, or after max_iter iterations.  The whole iteration runs on
 * the device (no host round trip per evaluation).  Synchronous: returns when outputs are
 * written.  out->B and out->lambda are required. */
dbie_status dbie_solve(dbie_ctx* ctx, int64_t n, const float* xyz, const dbie_options* opt,
                       const double* lambda_init, int32_t mem_kind, const dbie_solve_out* out,
                       void* stream);

/* Solve nprob independent problems (each its own context and point set) in one persistent
 * pair-sum launch per simplex round, with per-problem compaction of converged points.
 * Arrays of length nprob: ctxs, n, xyz, out (lambda_init may be NULL or hold NULL entries).
 * All contexts must live on the current device.  Synchronous. */
dbie_status dbie_solve_batched(int32_t nprob, dbie_ctx* const* ctxs, const int64_t* n,
                               const float* const* xyz, const dbie_options* opt,
                               const double* const* lambda_init, int32_t mem_kind,
                               const dbie_solve_out* out, void* stream);

/* Gradients at fixed lambda (n, 3) float64 for an upstream gradient gB = dL/dB (n, 3) float64:
 *   gB0  ((ny*nx), 3) float64: dL/dB0_pk = sum_i gB_pi a_ik(lambda_pi), the transpose of Eq. 16,
 *        computed by recomputing a_ik (no n x N matrix is stored); accumulate != 0 adds to gB0;
 *   glam (n, 3) float64 or NULL: dL/dlambda_p = gB_p dB_p/dlambda_p.
 * opt may be NULL (precision is read from it). */
dbie_status dbie_vjp(dbie_ctx* ctx, int64_t n, const float* xyz, const double* lambda,
                     const double* gB, const dbie_options* opt, int32_t mem_kind, double* gB0,
                     double* glam, int32_t accumulate, void* stream);

/* Second order at fixed lambda (n, 3) float64 (not in the paper): Phi = f + w_g g (phi, (n)),
 * its gradient dPhi/dlambda (grad, (n, 3)) and its Hessian d2Phi / dlambda_q dlambda_r (hess,
 * (n, 9), row-major 3 x 3), from one pass of ten pair sums per component (the objective sums, their
 * first lambda-derivatives and the second-derivative sums sum sin(lambda r) b,
 * sum cos(lambda r) (x_i - x_k) b / r and the same in y).  With lambda_mode = DBIE_LAMBDA_TIED,
 * lambda_x is the shared lambda and grad[0], hess[0] are the derivatives along it (other entries
 * 0).  Any of phi, grad, hess may be NULL, not all. */
dbie_status dbie_hessian(dbie_ctx* ctx, int64_t n, const float* xyz, const double* lambda,
                         const dbie_options* opt, int32_t mem_kind, double* phi, double* grad,
                         double* hess, void* stream);

/* Gradient of a loss L(B) with respect to the magnetogram THROUGH the lambda search (not in the
 * paper).  lambda (n, 3) float64 is taken as a stationary point of Phi (the result of dbie_solve),
 * so by implicit differentiation of grad_lambda Phi(lambda*; B0) = 0,
 *   gB0[k][p] = sum_i gB_pi a_ik(lambda_pi)  -  d/dB0_pk sum_i v_i . grad_lambda Phi_i,
 *   v_i = H_i^-1 dL/dlambda_i,  dL/dlambda_p = gB_p dB_p/dlambda_p (summed over p when tied),
 * H_i the lambda-Hessian of dbie_hessian.  The second term is a transposed pair sum of seven kernel
 * functions per component (no n x N matrix is stored).  gB (n, 3) float64 = dL/dB; gB0
 * ((ny*nx), 3) float64 (accumulate != 0 adds to it); v (n, 3) and flags (n) int32 may be NULL:
 * flags[i] = 1 where H_i is not positive definite (Cholesky fails), and that point contributes
 * only its fixed-lambda term (v_i = 0).  Points the search stopped early (Eq. 12 threshold or
 * max_iter) are not exactly stationary; the formula is applied to them as they are. */
dbie_status dbie_vjp_implicit(dbie_ctx* ctx, int64_t n, const float* xyz, const double* lambda,
                              const double* gB, const dbie_options* opt, int32_t mem_kind,
                              double* gB0, double* v, int32_t* flags, int32_t accumulate,
                              void* stream);

/* Noise propagation at fixed lambda (n, 3) float64 (not in the paper): with independent
 * zero-mean noise of standard deviation sigma_p on pixel k of component p, B is linear in B0
 * (Eq. 16), so var[i][p] = Var B_p(r_i) = sum_k a_ik(lambda_pi)^2 sigma_p[k]^2.  sigma_x, sigma_y,
 * sigma_z: (ny, nx) float32 maps (where mem_kind says), each may be NULL for the constant sigma0.
 * var (n, 3) float64.  Mixed precision sums the positive FP32 terms without a near field. */
dbie_status dbie_noise_var(dbie_ctx* ctx, int64_t n, const float* xyz, const double* lambda,
                           const float* sigma_x, const float* sigma_y, const float* sigma_z,
                           double sigma0, const dbie_options* opt, int32_t mem_kind, double* var,
                           void* stream);

/* Field evaluation that allocates no memory (no counterpart in the paper: an interface for
 * callers that may not allocate device memory while they run -- code inside another framework's
 * memory pool or arena, real-time loops that cannot take an allocation's implicit device
 * synchronisation, plugin hosts that forbid allocations by third-party libraries).
 *   Computes B (n, 3) float64 as dbie_eval does with opt = NULL (mixed precision, FP64 near field
 *   for z <= 2 hx; pixel-centre quadrature only), for the magnetogram (nx, ny, x0, y0, hx, hy, pixel_area, Bx, By, Bz: device
 *   float32, row-major (ny, nx)) at the points xyz (n, 3) device float32 with lambda (n, 3)
 *   device float32.  No context is needed.  All pointers are device memory.
 *   Limits: nx * ny <= 65536 and n <= 65536; larger sizes return DBIE_EINVAL.
 *   Scratch: one fixed 16 MiB array in the library's device image; every GPU that loads the
 *   library holds it until the process exits.  No cudaMalloc or cudaFree is made.
 *   The first call on a device looks up that array's device address (cudaGetSymbolAddress) with
 *   the device current; make that first call before any stream capture.
 *   All calls share the array and it keeps the previous call's contents (the call clears what
 *   must start at zero); calls that overlap on the GPU (other streams, other host threads) race.
 *   Synchronises `stream` before returning.  Device inputs are not validated.  Error messages
 *   go to stderr (dbie_last_error() is not updated by this function). */
dbie_status dbie_eval_noalloc(int32_t nx, int32_t ny, double x0, double y0, double hx, double hy,
                              double pixel_area, const float* Bx, const float* By,
                              const float* Bz, int64_t n, const float* xyz, const float* lambda,
                              double* B, void* stream);

/* Turn CUDA-event timing of the pair-sum kernels on or off, and read or reset the counters. */
dbie_status dbie_set_profiling(dbie_ctx* ctx, int32_t enable);
dbie_status dbie_get_stats(dbie_ctx* ctx, dbie_stats* stats, int32_t reset);

/* Pick launch parameters (CTA size, points per thread) for this device by timing candidates on
 * the context's boundary; results are cached per (device, variant, boundary size class) in
 * memory and in the file named by $DBIE_TUNE_CACHE when set.  Synchronises `stream`. */
dbie_status dbie_autotune(dbie_ctx* ctx, void* stream);

/* Launch configuration indices in use (after dbie_autotune): cfg_out[2 * variant + tied] for the
 * pair-sum variants value, value+dlambda, objective, objective+dlambda, objective+gradient,
 * objective+Hessian and noise variance (14 entries), then the adjoint kernel's (cfg_out[14]).
 * cfg_out must hold 15 int32. */
dbie_status dbie_get_config(dbie_ctx* ctx, int32_t* cfg_out);
/* Set the same 15 indices (each in [0, 6)); DBIE_EINVAL if one is out of range. */
dbie_status dbie_set_config(dbie_ctx* ctx, const int32_t* cfg_in);

/* Release the context and everything it owns.  NULL is a no-op. */
void dbie_destroy(dbie_ctx* ctx);

/* Message of the last error on this thread ("" if none). */
const char* dbie_last_error(void);

/* Library version string. */
const char* dbie_version(void);

#ifdef __cplusplus
}
#endif
#endif /* DBIE_H */
