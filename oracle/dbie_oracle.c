/*
 * dbie_oracle.c -- FP64 CPU oracle for the DBIE quadrature (TEST INFRASTRUCTURE ONLY).
 *
 * Restates, in the plainest form, what the paper (Wang, Yan & Tan, arXiv 1306.1122) computes:
 *   Eq. 6 / Eq. 16  B_p(r_i) = sum_k a_ik(lambda_pi) B_p0,k,
 *                   a_ik = z_i [lambda r sin(lambda r) + cos(lambda r)] / (2 pi r^3) * dA,
 *                   r^2 = (x_k - x_i)^2 + (y_k - y_i)^2 + z_i^2  (midpoint rule at pixel centres);
 *   Eq. 13          spatial derivatives of B at fixed lambda (zeroth-order rule), taken
 *                   analytically (the delta -> 0 limit) or by first-order forward differences;
 *   Eq. 14          J = curl B;
 *   Eq. 8, Eq. 9    f = |J x B| / (|J| |B|),  g = |div B| dV / (|B| dSigma);
 *   Sect. 2.1       Downhill Simplex (Nelder & Mead 1965) over (lambda_x, lambda_y, lambda_z),
 *                   with the standard coefficients (reflection 1, expansion 2, contraction 1/2,
 *                   shrink 1/2) and the outside/inside contraction rule of Lagarias et al. (1998).
 * Sums are taken in row-major pixel order with Neumaier compensation, so results are
 * deterministic.  Built with -ffp-contract=off: no fused multiply-adds.
 *
 * Only tests, the smoke check and the benchmark's CPU-baseline leg use this file.
 */
#include "dbie_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static const double TWO_PI = 6.283185307179586476925286766559;

/* Neumaier (improved Kahan-Babuska) compensated sum. */
typedef struct { double s, c; } nsum;
static void nsum_add(nsum* a, double v) {
  double t = a->s + v;
  if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
  else a->c += (v - t) + a->s;
  a->s = t;
}
static double nsum_get(const nsum* a) { return a->s + a->c; }

static const float* comp_ptr(const orc_boundary* bd, int p) {
  return p == 0 ? bd->Bx : (p == 1 ? bd->By : bd->Bz);
}

/* Eq. 6 / Eq. 16 and the analytic derivatives of the weight a_ik at fixed lambda (Eq. 13):
 *   a        = z u / (2 pi r^3) dA,            u = lambda r sin(lambda r) + cos(lambda r)
 *   da/dx_i  = z (x_i - x_k) psi / (2 pi) dA,  psi = (du/dr / r^3 - 3 u / r^4) / r
 *   da/dy_i  = z (y_i - y_k) psi / (2 pi) dA,  du/dr = lambda^2 r cos(lambda r)
 *   da/dz_i  = (u / r^3 + z^2 psi) / (2 pi) dA
 *   da/dlam  = z lambda cos(lambda r) / (2 pi r) dA. */
void orc_field(const orc_boundary* bd, double xi, double yi, double zi, const double lam[3],
               double B[3], double G[9], double dBdl[3]) {
  for (int p = 0; p < 3; ++p) {
    const float* B0 = comp_ptr(bd, p);
    const double l = lam[p];
    nsum sb = {0, 0}, sx = {0, 0}, sy = {0, 0}, sz = {0, 0}, sl = {0, 0};
    for (int j = 0; j < bd->ny; ++j) {
      const double yk = bd->y0 + j * bd->hy;
      for (int i = 0; i < bd->nx; ++i) {
        const double xk = bd->x0 + i * bd->hx;
        const double b0 = (double)B0[(int64_t)j * bd->nx + i];
        const double dx = xi - xk, dy = yi - yk;
        const double r = sqrt(dx * dx + dy * dy + zi * zi);
        const double lr = l * r;
        const double u = lr * sin(lr) + cos(lr);
        const double dudr = l * l * r * cos(lr);
        const double r3 = r * r * r;
        const double psi = (dudr / r3 - 3.0 * u / (r3 * r)) / r;
        const double w = bd->dA / TWO_PI;
        const double a = zi * u / r3 * w;
        const double ax = zi * dx * psi * w;
        const double ay = zi * dy * psi * w;
        const double az = (u / r3 + zi * zi * psi) * w;
        const double al = zi * l * cos(lr) / r * w;
        nsum_add(&sb, a * b0);
        nsum_add(&sx, ax * b0);
        nsum_add(&sy, ay * b0);
        nsum_add(&sz, az * b0);
        nsum_add(&sl, al * b0);
      }
    }
    B[p] = nsum_get(&sb);
    if (G) {
      G[3 * p + 0] = nsum_get(&sx);
      G[3 * p + 1] = nsum_get(&sy);
      G[3 * p + 2] = nsum_get(&sz);
    }
    if (dBdl) dBdl[p] = nsum_get(&sl);
  }
}

/* Eq. 13 read literally: first-order forward differences of B with lambda held at its value at r_i. */
void orc_field_fd(const orc_boundary* bd, double xi, double yi, double zi, const double lam[3],
                  double delta, double B[3], double G[9]) {
  double B1[3];
  orc_field(bd, xi, yi, zi, lam, B, NULL, NULL);
  orc_field(bd, xi + delta, yi, zi, lam, B1, NULL, NULL);
  for (int p = 0; p < 3; ++p) G[3 * p + 0] = (B1[p] - B[p]) / delta;
  orc_field(bd, xi, yi + delta, zi, lam, B1, NULL, NULL);
  for (int p = 0; p < 3; ++p) G[3 * p + 1] = (B1[p] - B[p]) / delta;
  orc_field(bd, xi, yi, zi + delta, lam, B1, NULL, NULL);
  for (int p = 0; p < 3; ++p) G[3 * p + 2] = (B1[p] - B[p]) / delta;
}

/* Eq. 14: J = curl B; Eq. 8: f = |J x B| / (|J||B|) (0 when |J||B| = 0);
 * Eq. 9: g = |div B| g_scale / |B| (0 when |B| = 0); Phi = f + w_g g. */
void orc_objective(const double B[3], const double G[9], double g_scale, double w_g,
                   double* f, double* g, double* phi, double J[3], double* D) {
  double Jx = G[3 * 2 + 1] - G[3 * 1 + 2];  /* dBz/dy - dBy/dz */
  double Jy = G[3 * 0 + 2] - G[3 * 2 + 0];  /* dBx/dz - dBz/dx */
  double Jz = G[3 * 1 + 0] - G[3 * 0 + 1];  /* dBy/dx - dBx/dy */
  double div = G[0] + G[4] + G[8];
  double cx = Jy * B[2] - Jz * B[1];
  double cy = Jz * B[0] - Jx * B[2];
  double cz = Jx * B[1] - Jy * B[0];
  double nJ = sqrt(Jx * Jx + Jy * Jy + Jz * Jz);
  double nB = sqrt(B[0] * B[0] + B[1] * B[1] + B[2] * B[2]);
  double nC = sqrt(cx * cx + cy * cy + cz * cz);
  double fv = (nJ * nB > 0.0) ? nC / (nJ * nB) : 0.0;
  double gv = (nB > 0.0) ? fabs(div) * g_scale / nB : 0.0;
  if (f) *f = fv;
  if (g) *g = gv;
  if (phi) *phi = fv + w_g * gv;
  if (J) { J[0] = Jx; J[1] = Jy; J[2] = Jz; }
  if (D) *D = div;
}

/* ---------------------------------------------------------------- Downhill Simplex ---- */

/* Stable ordering of the n+1 vertices by value (ties keep their current order). */
static void nm_sort(int n, double sim[4][3], double fs[4], int32_t fl[4]) {
  for (int a = 1; a <= n; ++a) {
    for (int b = a; b > 0 && fs[b] < fs[b - 1]; --b) {
      double t = fs[b]; fs[b] = fs[b - 1]; fs[b - 1] = t;
      int32_t tf = fl[b]; fl[b] = fl[b - 1]; fl[b - 1] = tf;
      for (int d = 0; d < n; ++d) { t = sim[b][d]; sim[b][d] = sim[b - 1][d]; sim[b - 1][d] = t; }
    }
  }
}

void orc_nelder_mead_sim(int32_t n, const double* sim0, double tol, int32_t max_iter,
                         orc_fun fun, void* ctx, orc_nm_result* res, char* codes, int32_t codes_cap) {
  const double rho = 1.0, chi = 2.0, psi = 0.5, sigma = 0.5;
  double sim[4][3] = {{0}}, fs[4], xr[3], xe[3], xc[3];
  int32_t fl[4], flr, fle, flc;
  int32_t nfev = 0, iters = 0, status = 0, nc = 0;
  for (int v = 0; v <= n; ++v) {
    for (int d = 0; d < n; ++d) sim[v][d] = sim0[v * n + d];
    fs[v] = fun(ctx, sim[v], &fl[v]);
    nfev++;
  }
  nm_sort(n, sim, fs, fl);
  for (;;) {
    /* Stopping tests: Eq. 12 at the best vertex, the simplex value spread, the iteration cap. */
    if (fl[0]) { status = 0; break; }
    if (fs[n] - fs[0] <= tol) { status = 0; break; }
    if (iters >= max_iter) { status = 1; break; }
    iters++;
    double c[3] = {0, 0, 0};
    for (int d = 0; d < n; ++d) {
      double s = 0.0;
      for (int v = 0; v < n; ++v) s += sim[v][d];
      c[d] = s / n;
    }
    for (int d = 0; d < n; ++d) xr[d] = (1.0 + rho) * c[d] - rho * sim[n][d];
    double fr = fun(ctx, xr, &flr); nfev++;
    char code;
    int shrink = 0;
    if (fr < fs[0]) {
      for (int d = 0; d < n; ++d) xe[d] = (1.0 + rho * chi) * c[d] - rho * chi * sim[n][d];
      double fe = fun(ctx, xe, &fle); nfev++;
      if (fe < fr) {
        for (int d = 0; d < n; ++d) sim[n][d] = xe[d];
        fs[n] = fe; fl[n] = fle; code = 'E';
      } else {
        for (int d = 0; d < n; ++d) sim[n][d] = xr[d];
        fs[n] = fr; fl[n] = flr; code = 'R';
      }
    } else if (fr < fs[n - 1]) {
      for (int d = 0; d < n; ++d) sim[n][d] = xr[d];
      fs[n] = fr; fl[n] = flr; code = 'R';
    } else if (fr < fs[n]) {
      /* outside contraction */
      for (int d = 0; d < n; ++d) xc[d] = (1.0 + psi * rho) * c[d] - psi * rho * sim[n][d];
      double fc = fun(ctx, xc, &flc); nfev++;
      if (fc <= fr) {
        for (int d = 0; d < n; ++d) sim[n][d] = xc[d];
        fs[n] = fc; fl[n] = flc; code = 'O';
      } else {
        shrink = 1;
      }
    } else {
      /* inside contraction */
      for (int d = 0; d < n; ++d) xc[d] = (1.0 - psi) * c[d] + psi * sim[n][d];
      double fc = fun(ctx, xc, &flc); nfev++;
      if (fc < fs[n]) {
        for (int d = 0; d < n; ++d) sim[n][d] = xc[d];
        fs[n] = fc; fl[n] = flc; code = 'I';
      } else {
        shrink = 1;
      }
    }
    if (shrink) {
      for (int v = 1; v <= n; ++v) {
        for (int d = 0; d < n; ++d) sim[v][d] = sim[0][d] + sigma * (sim[v][d] - sim[0][d]);
        fs[v] = fun(ctx, sim[v], &fl[v]); nfev++;
      }
      code = 'S';
    }
    if (codes && nc < codes_cap) codes[nc] = code;
    nc++;
    nm_sort(n, sim, fs, fl);
  }
  for (int d = 0; d < 3; ++d) res->x[d] = d < n ? sim[0][d] : 0.0;
  res->fx = fs[0];
  res->iters = iters;
  res->nfev = nfev;
  res->status = status;
  res->ncodes = nc < codes_cap ? nc : codes_cap;
  if (codes && nc < codes_cap) codes[nc] = '\0';
}

void orc_nelder_mead(int32_t n, const double x0[3], double step, double tol, int32_t max_iter,
                     orc_fun fun, void* ctx, orc_nm_result* res, char* codes, int32_t codes_cap) {
  double sim[12] = {0};
  for (int v = 0; v <= n; ++v)
    for (int d = 0; d < n; ++d) sim[v * n + d] = x0[d] + ((v == d + 1) ? step : 0.0);
  orc_nelder_mead_sim(n, sim, tol, max_iter, fun, ctx, res, codes, codes_cap);
}

/* The per-point objective of Sect. 2.1: Phi(lambda) = f + w_g g at point r_i. */
typedef struct {
  const orc_boundary* bd;
  const orc_options* opt;
  double x, y, z;
} dbie_point_ctx;

static void expand_lambda(const orc_options* opt, const double* x, double lam[3]) {
  if (opt->lambda_mode == 1) { lam[0] = lam[1] = lam[2] = x[0]; }
  else { lam[0] = x[0]; lam[1] = x[1]; lam[2] = x[2]; }
}

static void eval_point(const dbie_point_ctx* pc, const double lam[3], double B[3], double* f,
                       double* g, double* phi) {
  double G[9];
  if (pc->opt->deriv == 1) orc_field_fd(pc->bd, pc->x, pc->y, pc->z, lam, pc->opt->fd_delta, B, G);
  else orc_field(pc->bd, pc->x, pc->y, pc->z, lam, B, G, NULL);
  orc_objective(B, G, pc->opt->g_scale, pc->opt->w_g, f, g, phi, NULL, NULL);
}

static double dbie_phi(void* ctx, const double* x, int32_t* flag) {
  const dbie_point_ctx* pc = (const dbie_point_ctx*)ctx;
  double lam[3], B[3], f, g, phi;
  expand_lambda(pc->opt, x, lam);
  eval_point(pc, lam, B, &f, &g, &phi);
  *flag = (f <= pc->opt->eps_f && g <= pc->opt->eps_g) ? 1 : 0;
  return phi;
}

void orc_eval_many(const orc_boundary* bd, int64_t n, const double* xyz, const double* lam,
                   int32_t deriv, double fd_delta, double* B, double* G, double* dBdl,
                   int32_t nthreads) {
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads > 0 ? nthreads : 1)
#endif
  for (int64_t i = 0; i < n; ++i) {
    double Gi[9];
    if (deriv == 1) {
      orc_field_fd(bd, xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], lam + 3 * i, fd_delta, B + 3 * i, Gi);
      if (dBdl) { double tmp[3]; orc_field(bd, xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], lam + 3 * i, tmp, NULL, dBdl + 3 * i); }
    } else {
      orc_field(bd, xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], lam + 3 * i, B + 3 * i, Gi,
                dBdl ? dBdl + 3 * i : NULL);
    }
    if (G) memcpy(G + 9 * i, Gi, sizeof Gi);
  }
}

void orc_solve_many(const orc_boundary* bd, int64_t n, const double* xyz, const orc_options* opt,
                    const double* lam0, double* lam, double* B, double* f, double* g,
                    double* phi, int32_t* iters, int32_t* nfev, int32_t* status,
                    char* codes, int32_t codes_stride, int32_t nthreads) {
  const int dim = opt->lambda_mode == 1 ? 1 : 3;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
#endif
  for (int64_t i = 0; i < n; ++i) {
    dbie_point_ctx pc = {bd, opt, xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2]};
    double x0[3] = {0, 0, 0};
    if (lam0) for (int d = 0; d < dim; ++d) x0[d] = lam0[3 * i + d];
    orc_nm_result r;
    orc_nelder_mead(dim, x0, opt->simplex_step, opt->tol, opt->max_iter, dbie_phi, &pc, &r,
                    codes ? codes + i * (int64_t)codes_stride : NULL, codes ? codes_stride : 0);
    /* The kernel depends on lambda^2 only, so |lambda| is reported (Sect. 2.1: lambda is not unique). */
    double lb[3];
    expand_lambda(opt, r.x, lb);
    double Bi[3], fi, gi, phii;
    eval_point(&pc, lb, Bi, &fi, &gi, &phii);
    for (int p = 0; p < 3; ++p) { lam[3 * i + p] = fabs(lb[p]); B[3 * i + p] = Bi[p]; }
    if (f) f[i] = fi;
    if (g) g[i] = gi;
    if (phi) phi[i] = phii;
    if (iters) iters[i] = r.iters;
    if (nfev) nfev[i] = r.nfev;
    if (status) status[i] = r.status;
  }
}

/* Transpose of Eq. 16: for every pixel k and component p, sum over points i of gB_pi a_ik. */
void orc_vjp(const orc_boundary* bd, int64_t n, const double* xyz, const double* lam,
             const double* gB, double* gB0, int32_t nthreads) {
  const int64_t nb = (int64_t)bd->nx * bd->ny;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads > 0 ? nthreads : 1)
#endif
  for (int64_t k = 0; k < nb; ++k) {
    const int i_ = (int)(k % bd->nx), j_ = (int)(k / bd->nx);
    const double xk = bd->x0 + i_ * bd->hx, yk = bd->y0 + j_ * bd->hy;
    const double w = bd->dA / TWO_PI;
    for (int p = 0; p < 3; ++p) {
      nsum s = {0, 0};
      for (int64_t i = 0; i < n; ++i) {
        const double dx = xyz[3 * i] - xk, dy = xyz[3 * i + 1] - yk, zi = xyz[3 * i + 2];
        const double r = sqrt(dx * dx + dy * dy + zi * zi);
        const double lr = lam[3 * i + p] * r;
        const double u = lr * sin(lr) + cos(lr);
        const double a = zi * u / (r * r * r) * w;
        nsum_add(&s, gB[3 * i + p] * a);
      }
      gB0[3 * k + p] = nsum_get(&s);
    }
  }
}
