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

/* The lambda-derivatives of the weight's spatial derivatives, term by term:
 *   d/dlam (da/dx_i) = z (x_i - x_k) dpsi/dlam w,  d/dlam (da/dy_i) = z (y_i - y_k) dpsi/dlam w,
 *   d/dlam (da/dz_i) = (dphi/dlam + z^2 dpsi/dlam) w,
 *   dphi/dlam = lambda cos(lambda r) / r,
 *   dpsi/dlam = (2 lambda cos(lambda r) - lambda^2 r sin(lambda r) - 3 lambda cos(lambda r)) / r^3
 * (the last from differentiating psi = (lambda^2 cos(lambda r) - 3 u / r^2) / r^3 with
 * du/dlam = lambda r^2 cos(lambda r)). */
void orc_field_dl(const orc_boundary* bd, double xi, double yi, double zi, const double lam[3],
                  double B[3], double G[9], double dBdl[3], double dGdl[9]) {
  orc_field(bd, xi, yi, zi, lam, B, G, dBdl);
  for (int p = 0; p < 3; ++p) {
    const float* B0 = comp_ptr(bd, p);
    const double l = lam[p];
    nsum sx = {0, 0}, sy = {0, 0}, sz = {0, 0};
    for (int j = 0; j < bd->ny; ++j) {
      const double yk = bd->y0 + j * bd->hy;
      for (int i = 0; i < bd->nx; ++i) {
        const double xk = bd->x0 + i * bd->hx;
        const double b0 = (double)B0[(int64_t)j * bd->nx + i];
        const double dx = xi - xk, dy = yi - yk;
        const double r = sqrt(dx * dx + dy * dy + zi * zi);
        const double lr = l * r;
        const double r3 = r * r * r;
        const double dphi = l * cos(lr) / r;
        const double dpsi = (2.0 * l * cos(lr) - l * l * r * sin(lr) - 3.0 * l * cos(lr)) / r3;
        const double w = bd->dA / TWO_PI;
        nsum_add(&sx, zi * dx * dpsi * w * b0);
        nsum_add(&sy, zi * dy * dpsi * w * b0);
        nsum_add(&sz, (dphi + zi * zi * dpsi) * w * b0);
      }
    }
    dGdl[3 * p + 0] = nsum_get(&sx);
    dGdl[3 * p + 1] = nsum_get(&sy);
    dGdl[3 * p + 2] = nsum_get(&sz);
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

/* Gradient of Phi = f + w_g g with respect to lambda_q: lambda_q moves B_q (by dBdl[q]) and row q
 * of the gradient matrix (by dGdl[q][.]); the derivatives of |J x B|, |J|, |B| and |div B| follow
 * by the chain rule.  At |J x B| = 0 or |div B| = 0 (kinks of f and g) the one-sided part is 0. */
void orc_objective_grad(const double B[3], const double G[9], const double dBdl[3],
                        const double dGdl[9], double g_scale, double w_g, double* f, double* g,
                        double* phi, double dphi[3]) {
  double J[3], D;
  orc_objective(B, G, g_scale, w_g, f, g, phi, J, &D);
  const double C[3] = {J[1] * B[2] - J[2] * B[1], J[2] * B[0] - J[0] * B[2],
                       J[0] * B[1] - J[1] * B[0]};
  const double nJ = sqrt(J[0] * J[0] + J[1] * J[1] + J[2] * J[2]);
  const double nB = sqrt(B[0] * B[0] + B[1] * B[1] + B[2] * B[2]);
  const double nC = sqrt(C[0] * C[0] + C[1] * C[1] + C[2] * C[2]);
  for (int q = 0; q < 3; ++q) {
    double dB[3] = {0, 0, 0}, dG[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    dB[q] = dBdl[q];
    for (int j = 0; j < 3; ++j) dG[3 * q + j] = dGdl[3 * q + j];
    const double dJ[3] = {dG[3 * 2 + 1] - dG[3 * 1 + 2], dG[3 * 0 + 2] - dG[3 * 2 + 0],
                          dG[3 * 1 + 0] - dG[3 * 0 + 1]};
    const double dD = dG[0] + dG[4] + dG[8];
    /* dC = dJ x B + J x dB */
    const double dC[3] = {dJ[1] * B[2] - dJ[2] * B[1] + J[1] * dB[2] - J[2] * dB[1],
                          dJ[2] * B[0] - dJ[0] * B[2] + J[2] * dB[0] - J[0] * dB[2],
                          dJ[0] * B[1] - dJ[1] * B[0] + J[0] * dB[1] - J[1] * dB[0]};
    double df = 0.0, dg = 0.0;
    if (nJ * nB > 0.0) {
      const double JdJ = J[0] * dJ[0] + J[1] * dJ[1] + J[2] * dJ[2];
      const double BdB = B[0] * dB[0] + B[1] * dB[1] + B[2] * dB[2];
      const double CdC = C[0] * dC[0] + C[1] * dC[1] + C[2] * dC[2];
      df = (nC > 0.0 ? CdC / (nC * nJ * nB) : 0.0) - (*f) * (JdJ / (nJ * nJ) + BdB / (nB * nB));
    }
    if (nB > 0.0) {
      const double BdB = B[0] * dB[0] + B[1] * dB[1] + B[2] * dB[2];
      const double sgn = D > 0.0 ? 1.0 : (D < 0.0 ? -1.0 : 0.0);
      dg = g_scale * (sgn * dD / nB - fabs(D) * BdB / (nB * nB * nB));
    }
    dphi[q] = df + w_g * dg;
  }
}

/* ---------------------------------------------------------------------- quasi-Newton ---- */

void orc_bfgs(int32_t n, const double x0[3], double step, double tol, int32_t max_iter,
              orc_fun_grad fun, void* ctx, orc_nm_result* res) {
  double x[3] = {0, 0, 0}, gr[3] = {0, 0, 0}, H[9], xt[3] = {0, 0, 0}, gt[3] = {0, 0, 0};
  double d[3] = {0, 0, 0};
  int32_t flag = 0, flagt = 0, nfev = 0, iters = 0, status = 0;
  for (int i = 0; i < n; ++i) x[i] = x0[i];
  double F = fun(ctx, x, gr, &flag);
  nfev++;
  double gn = 0.0;
  for (int i = 0; i < n; ++i) gn += gr[i] * gr[i];
  gn = sqrt(gn);
  for (int i = 0; i < 9; ++i) H[i] = 0.0;
  if (gn > 0.0)
    for (int i = 0; i < n; ++i) H[3 * i + i] = step / gn;
  for (;;) {
    if (flag) { status = 0; break; }
    if (!(gn > 0.0)) { status = 0; break; }
    if (iters >= max_iter) { status = 1; break; }
    double gd = 0.0;
    for (int i = 0; i < n; ++i) {
      double s = 0.0;
      for (int j = 0; j < n; ++j) s += H[3 * i + j] * gr[j];
      d[i] = -s;
    }
    for (int i = 0; i < n; ++i) gd += gr[i] * d[i];
    if (!(gd < 0.0)) {  /* not a descent direction: restart from the scaled gradient */
      for (int i = 0; i < 9; ++i) H[i] = 0.0;
      for (int i = 0; i < n; ++i) H[3 * i + i] = step / gn;
      gd = 0.0;
      for (int i = 0; i < n; ++i) { d[i] = -(H[3 * i + i] * gr[i]); gd += gr[i] * d[i]; }
    }
    double a = 1.0, Ft = 0.0;
    int accepted = 0;
    for (int ls = 0; ls <= 30; ++ls) {
      for (int i = 0; i < n; ++i) xt[i] = x[i] + a * d[i];
      Ft = fun(ctx, xt, gt, &flagt);
      nfev++;
      if (Ft <= F + 1e-4 * a * gd) { accepted = 1; break; }
      a = 0.5 * a;
    }
    if (!accepted) { status = 0; break; }
    iters++;
    double s[3] = {0, 0, 0}, y[3] = {0, 0, 0}, sy = 0.0, ss = 0.0, yy = 0.0;
    for (int i = 0; i < n; ++i) {
      s[i] = xt[i] - x[i];
      y[i] = gt[i] - gr[i];
      sy += s[i] * y[i];
      ss += s[i] * s[i];
      yy += y[i] * y[i];
    }
    if (sy > 1e-12 * sqrt(ss) * sqrt(yy)) {
      const double rho = 1.0 / sy;
      double Hy[3] = {0, 0, 0}, yHy = 0.0;
      for (int i = 0; i < n; ++i) {
        double t = 0.0;
        for (int j = 0; j < n; ++j) t += H[3 * i + j] * y[j];
        Hy[i] = t;
      }
      for (int i = 0; i < n; ++i) yHy += y[i] * Hy[i];
      const double c2 = rho * rho * yHy + rho;
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
          H[3 * i + j] = H[3 * i + j] - rho * (s[i] * Hy[j] + Hy[i] * s[j]) + c2 * s[i] * s[j];
    }
    const double dec = F - Ft;
    for (int i = 0; i < n; ++i) { x[i] = xt[i]; gr[i] = gt[i]; }
    F = Ft;
    flag = flagt;
    gn = 0.0;
    for (int i = 0; i < n; ++i) gn += gr[i] * gr[i];
    gn = sqrt(gn);
    if (dec <= tol) { status = 0; break; }
  }
  for (int i = 0; i < 3; ++i) res->x[i] = i < n ? x[i] : 0.0;
  res->fx = F;
  res->iters = iters;
  res->nfev = nfev;
  res->status = status;
  res->ncodes = 0;
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

static void pxe_terms(const orc_boundary* bd, double xi, double yi, double zi, double pxe_near_z,
                      double dB[3], double dG[9]);

/* The per-point objective of Sect. 2.1: Phi(lambda) = f + w_g g at point r_i. */
typedef struct {
  const orc_boundary* bd;
  const orc_options* opt;
  double x, y, z;
  double cB[3], cG[9];    /* pixel-exact correction of B and grad B (quad_order -1), else 0 */
} dbie_point_ctx;

static void add_correction(const dbie_point_ctx* pc, double B[3], double G[9]) {
  for (int p = 0; p < 3; ++p) B[p] += pc->cB[p];
  for (int q = 0; q < 9; ++q) G[q] += pc->cG[q];
}

static void expand_lambda(const orc_options* opt, const double* x, double lam[3]) {
  if (opt->lambda_mode == 1) { lam[0] = lam[1] = lam[2] = x[0]; }
  else { lam[0] = x[0]; lam[1] = x[1]; lam[2] = x[2]; }
}

static void eval_point(const dbie_point_ctx* pc, const double lam[3], double B[3], double* f,
                       double* g, double* phi) {
  double G[9];
  if (pc->opt->quad_order > 0) orc_field_q9(pc->bd, pc->x, pc->y, pc->z, lam, pc->opt->quad_order, B, G, NULL);
  else if (pc->opt->deriv == 1) orc_field_fd(pc->bd, pc->x, pc->y, pc->z, lam, pc->opt->fd_delta, B, G);
  else orc_field(pc->bd, pc->x, pc->y, pc->z, lam, B, G, NULL);
  if (pc->opt->quad_order == -1) add_correction(pc, B, G);
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

/* Phi and its lambda-gradient at point pc (tied mode: the sum over the three components). */
static double dbie_phi_grad(void* ctx, const double* x, double* grad, int32_t* flag) {
  const dbie_point_ctx* pc = (const dbie_point_ctx*)ctx;
  double lam[3], B[3], G[9], dBdl[3], dGdl[9], f, g, phi, dphi[3];
  expand_lambda(pc->opt, x, lam);
  orc_field_dl(pc->bd, pc->x, pc->y, pc->z, lam, B, G, dBdl, dGdl);
  if (pc->opt->quad_order == -1) add_correction(pc, B, G);
  orc_objective_grad(B, G, dBdl, dGdl, pc->opt->g_scale, pc->opt->w_g, &f, &g, &phi, dphi);
  if (pc->opt->lambda_mode == 1) grad[0] = dphi[0] + dphi[1] + dphi[2];
  else { grad[0] = dphi[0]; grad[1] = dphi[1]; grad[2] = dphi[2]; }
  *flag = (f <= pc->opt->eps_f && g <= pc->opt->eps_g) ? 1 : 0;
  return phi;
}

void orc_objective_many(const orc_boundary* bd, int64_t n, const double* xyz, const double* lam,
                        double g_scale, double w_g, double pxe_near_z, double* fgphi,
                        double* dphi, int32_t nthreads) {
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads > 0 ? nthreads : 1)
#endif
  for (int64_t i = 0; i < n; ++i) {
    double B[3], G[9], dBdl[3], dGdl[9], f, g, phi, cB[3], cG[9];
    orc_field_dl(bd, xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], lam + 3 * i, B, G, dBdl, dGdl);
    pxe_terms(bd, xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], pxe_near_z, cB, cG);
    for (int p = 0; p < 3; ++p) B[p] += cB[p];
    for (int q = 0; q < 9; ++q) G[q] += cG[q];
    orc_objective_grad(B, G, dBdl, dGdl, g_scale, w_g, &f, &g, &phi, dphi + 3 * i);
    fgphi[3 * i] = f;
    fgphi[3 * i + 1] = g;
    fgphi[3 * i + 2] = phi;
  }
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
    dbie_point_ctx pc;
    memset(&pc, 0, sizeof pc);
    pc.bd = bd;
    pc.opt = opt;
    pc.x = xyz[3 * i];
    pc.y = xyz[3 * i + 1];
    pc.z = xyz[3 * i + 2];
    if (opt->quad_order == -1 && pc.z <= opt->pxe_near_z)
      orc_pxe_correction(bd, pc.x, pc.y, pc.z, pc.cB, pc.cG);
    double x0[3] = {0, 0, 0};
    if (lam0) for (int d = 0; d < dim; ++d) x0[d] = lam0[3 * i + d];
    orc_nm_result r;
    if (opt->method == 1) {
      /* Phi is even in every lambda_p, so lambda = 0 is a stationary point: the gradient search
       * starts one step away from it along (1, 1, 1). */
      for (int d = 0; d < dim; ++d) x0[d] += opt->simplex_step;
      orc_bfgs(dim, x0, opt->simplex_step, opt->tol, opt->max_iter, dbie_phi_grad, &pc, &r);
    }
    else
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

/* ------------------------------------------------------ second order: hyper-dual numbers ---- */
/* x = v + a e1 + b e2 + c e1 e2 with e1^2 = e2^2 = 0 (hyper-dual numbers, Fike & Alonso 2011).
 * A function evaluated at x0 + s1 e1 + s2 e2 returns its value, its derivatives along s1 (a) and
 * s2 (b) and the second derivative s1^T Hess s2 (c), exactly and without a difference step. */
typedef struct { double v, a, b, c; } hd;

static hd hd_k(double v) { hd r = {v, 0.0, 0.0, 0.0}; return r; }
static hd hd_add(hd x, hd y) { hd r = {x.v + y.v, x.a + y.a, x.b + y.b, x.c + y.c}; return r; }
static hd hd_sub(hd x, hd y) { hd r = {x.v - y.v, x.a - y.a, x.b - y.b, x.c - y.c}; return r; }
static hd hd_scl(hd x, double s) { hd r = {x.v * s, x.a * s, x.b * s, x.c * s}; return r; }
static hd hd_mul(hd x, hd y) {
  hd r = {x.v * y.v, x.v * y.a + x.a * y.v, x.v * y.b + x.b * y.v,
          x.v * y.c + x.a * y.b + x.b * y.a + x.c * y.v};
  return r;
}
/* phi(x) for a scalar function with phi = g0, phi' = g1, phi'' = g2 at x.v. */
static hd hd_chain(hd x, double g0, double g1, double g2) {
  hd r = {g0, g1 * x.a, g1 * x.b, g1 * x.c + g2 * x.a * x.b};
  return r;
}
static hd hd_sin(hd x) { return hd_chain(x, sin(x.v), cos(x.v), -sin(x.v)); }
static hd hd_cos(hd x) { return hd_chain(x, cos(x.v), -sin(x.v), -cos(x.v)); }
static hd hd_inv(hd x) {
  const double i = 1.0 / x.v;
  return hd_chain(x, i, -i * i, 2.0 * i * i * i);
}
static hd hd_div(hd x, hd y) { return hd_mul(x, hd_inv(y)); }
static hd hd_abs(hd x) { return x.v < 0.0 ? hd_scl(x, -1.0) : x; }
/* |x| of a 3-vector; at |x| = 0 (a kink) the derivative parts are taken as 0. */
static hd hd_norm3(const hd x[3]) {
  const hd q = hd_add(hd_add(hd_mul(x[0], x[0]), hd_mul(x[1], x[1])), hd_mul(x[2], x[2]));
  if (!(q.v > 0.0)) return hd_k(0.0);
  const double s = sqrt(q.v);
  return hd_chain(q, s, 0.5 / s, -0.25 / (s * q.v));
}

typedef struct { nsum v, a, b, c; } hsum;
static void hsum_add(hsum* s, hd x) {
  nsum_add(&s->v, x.v);
  nsum_add(&s->a, x.a);
  nsum_add(&s->b, x.b);
  nsum_add(&s->c, x.c);
}
static hd hsum_get(const hsum* s) {
  hd r = {nsum_get(&s->v), nsum_get(&s->a), nsum_get(&s->b), nsum_get(&s->c)};
  return r;
}

/* The weight a_ik of Eq. 16 and its spatial derivatives at fixed lambda (the terms of orc_field)
 * for one pixel, with lambda a hyper-dual number: w4 = {a, da/dx_i, da/dy_i, da/dz_i}.
 * dx = x_i - x_k, dy = y_i - y_k, w = dA / 2 pi. */
static void weights_hd(double dx, double dy, double zi, hd l, double w, hd w4[4]) {
  const double r = sqrt(dx * dx + dy * dy + zi * zi);
  const double r3 = r * r * r;
  const hd lr = hd_scl(l, r);
  const hd s = hd_sin(lr), c = hd_cos(lr);
  const hd u = hd_add(hd_mul(lr, s), c);
  const hd dudr = hd_scl(hd_mul(hd_mul(l, l), c), r);
  const hd psi = hd_scl(hd_sub(hd_scl(dudr, 1.0 / r3), hd_scl(u, 3.0 / (r3 * r))), 1.0 / r);
  w4[0] = hd_scl(u, zi / r3 * w);
  w4[1] = hd_scl(psi, zi * dx * w);
  w4[2] = hd_scl(psi, zi * dy * w);
  w4[3] = hd_scl(hd_add(hd_scl(u, 1.0 / r3), hd_scl(psi, zi * zi)), w);
}

/* B_p and row p of the gradient matrix (Eq. 16 and Eq. 13 at fixed lambda), each component at
 * its own hyper-dual lambda_p. */
static void field_hd(const orc_boundary* bd, double xi, double yi, double zi, const hd lam[3],
                     hd B[3], hd G[9]) {
  const double w = bd->dA / TWO_PI;
  for (int p = 0; p < 3; ++p) {
    const float* B0 = comp_ptr(bd, p);
    hsum s[4];
    memset(s, 0, sizeof s);
    for (int j = 0; j < bd->ny; ++j) {
      const double yk = bd->y0 + j * bd->hy;
      for (int i = 0; i < bd->nx; ++i) {
        const double xk = bd->x0 + i * bd->hx;
        const double b0 = (double)B0[(int64_t)j * bd->nx + i];
        hd w4[4];
        weights_hd(xi - xk, yi - yk, zi, lam[p], w, w4);
        for (int q = 0; q < 4; ++q) hsum_add(&s[q], hd_scl(w4[q], b0));
      }
    }
    B[p] = hsum_get(&s[0]);
    for (int j = 0; j < 3; ++j) G[3 * p + j] = hsum_get(&s[1 + j]);
  }
}

/* Eq. 14, Eq. 8 and Eq. 9 in hyper-dual arithmetic, Phi = f + w_g g, with the degenerate cases of
 * orc_objective (f = 0 when |J||B| = 0, g = 0 when |B| = 0). */
static hd objective_hd(const hd B[3], const hd G[9], double g_scale, double w_g) {
  const hd J[3] = {hd_sub(G[3 * 2 + 1], G[3 * 1 + 2]), hd_sub(G[3 * 0 + 2], G[3 * 2 + 0]),
                   hd_sub(G[3 * 1 + 0], G[3 * 0 + 1])};
  const hd D = hd_add(hd_add(G[0], G[4]), G[8]);
  const hd C[3] = {hd_sub(hd_mul(J[1], B[2]), hd_mul(J[2], B[1])),
                   hd_sub(hd_mul(J[2], B[0]), hd_mul(J[0], B[2])),
                   hd_sub(hd_mul(J[0], B[1]), hd_mul(J[1], B[0]))};
  const hd nJ = hd_norm3(J), nB = hd_norm3(B), nC = hd_norm3(C);
  const hd f = (nJ.v * nB.v > 0.0) ? hd_div(nC, hd_mul(nJ, nB)) : hd_k(0.0);
  const hd g = (nB.v > 0.0) ? hd_scl(hd_div(hd_abs(D), nB), g_scale) : hd_k(0.0);
  return hd_add(f, hd_scl(g, w_g));
}

static void pxe_pixel_weights(const orc_boundary* bd, double xi, double yi, double zi, int i, int j,
                              double c[4]);

/* The pixel-exact correction (orc_pxe_correction) of B and grad B at a point with
 * z <= pxe_near_z (pxe_near_z <= 0: none); it does not depend on lambda. */
static void pxe_terms(const orc_boundary* bd, double xi, double yi, double zi, double pxe_near_z,
                      double dB[3], double dG[9]) {
  memset(dB, 0, 3 * sizeof(double));
  memset(dG, 0, 9 * sizeof(double));
  if (pxe_near_z > 0.0 && zi <= pxe_near_z) orc_pxe_correction(bd, xi, yi, zi, dB, dG);
}
static void field_hd_pxe(const orc_boundary* bd, double xi, double yi, double zi, const hd lam[3],
                         const double dB[3], const double dG[9], hd B[3], hd G[9]) {
  field_hd(bd, xi, yi, zi, lam, B, G);
  for (int p = 0; p < 3; ++p) B[p].v += dB[p];
  for (int q = 0; q < 9; ++q) G[q].v += dG[q];
}

void orc_hessian(const orc_boundary* bd, double xi, double yi, double zi, const double lam[3],
                 int32_t lambda_mode, double g_scale, double w_g, double pxe_near_z, double* phi,
                 double grad[3], double H[9], double dBdl[3]) {
  hd lh[3], B[3], G[9];
  double cB[3], cG[9];
  pxe_terms(bd, xi, yi, zi, pxe_near_z, cB, cG);
  for (int q = 0; q < 9; ++q) H[q] = 0.0;
  for (int q = 0; q < 3; ++q) grad[q] = dBdl[q] = 0.0;
  if (lambda_mode == 1) {
    for (int p = 0; p < 3; ++p) { lh[p].v = lam[p]; lh[p].a = 1.0; lh[p].b = 1.0; lh[p].c = 0.0; }
    field_hd_pxe(bd, xi, yi, zi, lh, cB, cG, B, G);
    const hd ph = objective_hd(B, G, g_scale, w_g);
    *phi = ph.v;
    grad[0] = ph.a;
    H[0] = ph.c;
    for (int p = 0; p < 3; ++p) dBdl[p] = B[p].a;
    return;
  }
  for (int j = 0; j < 3; ++j)
    for (int k = j; k < 3; ++k) {
      for (int p = 0; p < 3; ++p) {
        lh[p].v = lam[p];
        lh[p].a = p == j ? 1.0 : 0.0;
        lh[p].b = p == k ? 1.0 : 0.0;
        lh[p].c = 0.0;
      }
      field_hd_pxe(bd, xi, yi, zi, lh, cB, cG, B, G);
      const hd ph = objective_hd(B, G, g_scale, w_g);
      H[3 * j + k] = H[3 * k + j] = ph.c;
      if (j == k) {
        grad[j] = ph.a;
        dBdl[j] = B[j].a;
        *phi = ph.v;
      }
    }
}

void orc_hessian_many(const orc_boundary* bd, int64_t n, const double* xyz, const double* lam,
                      int32_t lambda_mode, double g_scale, double w_g, double pxe_near_z,
                      double* phi, double* grad, double* H, double* dBdl, int32_t nthreads) {
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
#endif
  for (int64_t i = 0; i < n; ++i)
    orc_hessian(bd, xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], lam + 3 * i, lambda_mode, g_scale,
                w_g, pxe_near_z, phi + i, grad + 3 * i, H + 9 * i, dBdl + 3 * i);
}

/* Solve H v = r for a symmetric m x m matrix (m <= 3) by Cholesky; returns 0 when H is not
 * positive definite (a pivot <= 0). */
static int chol_solve(int m, const double* H, const double* r, double* v) {
  double L[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, y[3] = {0, 0, 0};
  for (int j = 0; j < m; ++j) {
    double d = H[3 * j + j];
    for (int k = 0; k < j; ++k) d -= L[3 * j + k] * L[3 * j + k];
    if (!(d > 0.0)) return 0;
    L[3 * j + j] = sqrt(d);
    for (int i = j + 1; i < m; ++i) {
      double e = H[3 * i + j];
      for (int k = 0; k < j; ++k) e -= L[3 * i + k] * L[3 * j + k];
      L[3 * i + j] = e / L[3 * j + j];
    }
  }
  for (int i = 0; i < m; ++i) {
    double e = r[i];
    for (int k = 0; k < i; ++k) e -= L[3 * i + k] * y[k];
    y[i] = e / L[3 * i + i];
  }
  for (int i = m - 1; i >= 0; --i) {
    double e = y[i];
    for (int k = i + 1; k < m; ++k) e -= L[3 * k + i] * v[k];
    v[i] = e / L[3 * i + i];
  }
  return 1;
}

void orc_implicit_vjp(const orc_boundary* bd, int64_t n, const double* xyz, const double* lam,
                      const double* gB, int32_t lambda_mode, double g_scale, double w_g,
                      double pxe_near_z, double* gB0, double* v_out, int32_t* flags,
                      int32_t nthreads) {
  const int m = lambda_mode == 1 ? 1 : 3;
  const double w = bd->dA / TWO_PI;
  double* vp = (double*)calloc((size_t)(n > 0 ? n : 1) * 3, sizeof(double));
  hd* q = (hd*)calloc((size_t)(n > 0 ? n : 1) * 12, sizeof(hd));
  int32_t* fl = (int32_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
  /* per point: H, dL/dlambda, v = H^-1 dL/dlambda, and B, grad B moving along v (e1) */
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
#endif
  for (int64_t i = 0; i < n; ++i) {
    const double xi = xyz[3 * i], yi = xyz[3 * i + 1], zi = xyz[3 * i + 2];
    double phi, grad[3], H[9], dBdl[3], gl[3] = {0, 0, 0}, v[3] = {0, 0, 0};
    orc_hessian(bd, xi, yi, zi, lam + 3 * i, lambda_mode, g_scale, w_g, pxe_near_z, &phi, grad, H,
                dBdl);
    if (lambda_mode == 1) gl[0] = gB[3 * i] * dBdl[0] + gB[3 * i + 1] * dBdl[1] + gB[3 * i + 2] * dBdl[2];
    else for (int p = 0; p < 3; ++p) gl[p] = gB[3 * i + p] * dBdl[p];
    if (!chol_solve(m, H, gl, v)) { fl[i] = 1; v[0] = v[1] = v[2] = 0.0; }
    for (int p = 0; p < 3; ++p) vp[3 * i + p] = lambda_mode == 1 ? v[0] : v[p];
    hd lh[3], B[3], G[9];
    double cB[3], cG[9];
    pxe_terms(bd, xi, yi, zi, pxe_near_z, cB, cG);
    for (int p = 0; p < 3; ++p) { lh[p] = hd_k(lam[3 * i + p]); lh[p].a = vp[3 * i + p]; }
    field_hd_pxe(bd, xi, yi, zi, lh, cB, cG, B, G);
    for (int p = 0; p < 3; ++p) q[12 * i + p] = B[p];
    for (int e = 0; e < 9; ++e) q[12 * i + 3 + e] = G[e];
    if (v_out) for (int p = 0; p < 3; ++p) v_out[3 * i + p] = vp[3 * i + p];
    if (flags) flags[i] = fl[i];
  }
  /* per pixel and component: the fixed-lambda adjoint minus d/dB0_pk of v . grad_lambda Phi,
   * the latter as the e1 e2 part of Phi with e2 seeded on the pixel's weights */
  const int64_t nb = (int64_t)bd->nx * bd->ny;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads > 0 ? nthreads : 1)
#endif
  for (int64_t k = 0; k < nb; ++k) {
    const int i_ = (int)(k % bd->nx), j_ = (int)(k / bd->nx);
    const double xk = bd->x0 + i_ * bd->hx, yk = bd->y0 + j_ * bd->hy;
    for (int p = 0; p < 3; ++p) {
      nsum s = {0, 0};
      for (int64_t i = 0; i < n; ++i) {
        hd l = hd_k(lam[3 * i + p]);
        l.a = vp[3 * i + p];
        hd w4[4];
        weights_hd(xyz[3 * i] - xk, xyz[3 * i + 1] - yk, xyz[3 * i + 2], l, w, w4);
        if (pxe_near_z > 0.0 && xyz[3 * i + 2] <= pxe_near_z) {
          double c[4];
          pxe_pixel_weights(bd, xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], i_, j_, c);
          for (int e = 0; e < 4; ++e) w4[e].v += c[e];
        }
        double t = gB[3 * i + p] * w4[0].v;
        if (!fl[i]) {
          hd B[3], G[9];
          for (int e = 0; e < 3; ++e) B[e] = q[12 * i + e];
          for (int e = 0; e < 9; ++e) G[e] = q[12 * i + 3 + e];
          B[p].b = w4[0].v;
          B[p].c = w4[0].a;
          for (int j = 0; j < 3; ++j) {
            G[3 * p + j].b = w4[1 + j].v;
            G[3 * p + j].c = w4[1 + j].a;
          }
          t -= objective_hd(B, G, g_scale, w_g).c;
        }
        nsum_add(&s, t);
      }
      gB0[3 * k + p] = nsum_get(&s);
    }
  }
  free(vp);
  free(q);
  free(fl);
}

void orc_noise_var(const orc_boundary* bd, int64_t n, const double* xyz, const double* lam,
                   const float* sx, const float* sy, const float* sz, double sigma0, double* var,
                   int32_t nthreads) {
  const float* sg[3] = {sx, sy, sz};
  const double w = bd->dA / TWO_PI;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads > 0 ? nthreads : 1)
#endif
  for (int64_t i = 0; i < n; ++i) {
    const double xi = xyz[3 * i], yi = xyz[3 * i + 1], zi = xyz[3 * i + 2];
    for (int p = 0; p < 3; ++p) {
      nsum s = {0, 0};
      for (int j = 0; j < bd->ny; ++j) {
        const double yk = bd->y0 + j * bd->hy;
        for (int ii = 0; ii < bd->nx; ++ii) {
          const double xk = bd->x0 + ii * bd->hx;
          const double dx = xi - xk, dy = yi - yk;
          const double r = sqrt(dx * dx + dy * dy + zi * zi);
          const double lr = lam[3 * i + p] * r;
          const double a = zi * (lr * sin(lr) + cos(lr)) / (r * r * r) * w;
          const double sd = sg[p] ? (double)sg[p][(int64_t)j * bd->nx + ii] : sigma0;
          nsum_add(&s, a * a * sd * sd);
        }
      }
      var[3 * i + p] = nsum_get(&s);
    }
  }
}

/* ------------------------------------------------------ Eq. 15: nine-node elements ---- */

void orc_gauss_legendre(int32_t m, double* x, double* w) {
  /* Roots of the Legendre polynomial P_m by Newton's method from the Chebyshev-like guesses
   * cos(pi (i + 3/4) / (m + 1/2)); P_m and P_m' by the three-term recurrence;
   * w = 2 / ((1 - x^2) P_m'(x)^2). */
  const double PI = 3.14159265358979323846;
  for (int i = 0; i < m; ++i) {
    double t = cos(PI * (i + 0.75) / (m + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = t;
      for (int k = 2; k <= m; ++k) {
        const double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = m * (t * p1 - p0) / (t * t - 1.0);
      const double dt = p1 / dp;
      t -= dt;
      if (fabs(dt) < 1e-16) break;
    }
    {
      double p0 = 1.0, p1 = t;
      for (int k = 2; k <= m; ++k) {
        const double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = m * (t * p1 - p0) / (t * t - 1.0);
    }
    x[m - 1 - i] = t;   /* ascending order */
    w[m - 1 - i] = 2.0 / ((1.0 - t * t) * dp * dp);
  }
}

/* 1-D quadratic Lagrange polynomials on the nodes -1, 0, 1. */
static double lagr2(int a, double t) {
  return a == 0 ? 0.5 * t * (t - 1.0) : (a == 1 ? 1.0 - t * t : 0.5 * t * (t + 1.0));
}

void orc_node_weights_q9(const orc_boundary* bd, double xi, double yi, double zi, double lam,
                         int32_t order, double* out) {
  double gx[16], gw[16];
  orc_gauss_legendre(order, gx, gw);
  const int64_t np = (int64_t)bd->nx * bd->ny;
  for (int64_t k = 0; k < 5 * np; ++k) out[k] = 0.0;
  const int nex = (bd->nx - 1) / 2, ney = (bd->ny - 1) / 2;
  const double jac = bd->hx * bd->hy;
  for (int ey = 0; ey < ney; ++ey)
    for (int ex = 0; ex < nex; ++ex) {
      const double xc = bd->x0 + (2 * ex + 1) * bd->hx, yc = bd->y0 + (2 * ey + 1) * bd->hy;
      /* integral over the element of K (and its derivatives) times each shape function */
      for (int jb = 0; jb < 3; ++jb)
        for (int ia = 0; ia < 3; ++ia) {
          const int64_t node = (int64_t)(2 * ey + jb) * bd->nx + (2 * ex + ia);
          for (int gb = 0; gb < order; ++gb)
            for (int ga = 0; ga < order; ++ga) {
              const double s = gx[ga], t = gx[gb];
              const double xk = xc + s * bd->hx, yk = yc + t * bd->hy;
              const double dx = xi - xk, dy = yi - yk;
              const double r = sqrt(dx * dx + dy * dy + zi * zi);
              const double lr = lam * r;
              const double u = lr * sin(lr) + cos(lr);
              const double dudr = lam * lam * r * cos(lr);
              const double r3 = r * r * r;
              const double psi = (dudr / r3 - 3.0 * u / (r3 * r)) / r;
              const double c = lagr2(ia, s) * lagr2(jb, t) * gw[ga] * gw[gb] * jac / TWO_PI;
              out[5 * node + 0] += zi * u / r3 * c;
              out[5 * node + 1] += zi * dx * psi * c;
              out[5 * node + 2] += zi * dy * psi * c;
              out[5 * node + 3] += (u / r3 + zi * zi * psi) * c;
              out[5 * node + 4] += zi * lam * cos(lr) / r * c;
            }
        }
    }
}

void orc_field_q9(const orc_boundary* bd, double xi, double yi, double zi, const double lam[3],
                  int32_t order, double B[3], double G[9], double dBdl[3]) {
  const int64_t np = (int64_t)bd->nx * bd->ny;
  double* a = (double*)malloc(sizeof(double) * 5 * (size_t)np);
  for (int p = 0; p < 3; ++p) {
    const float* B0 = comp_ptr(bd, p);
    orc_node_weights_q9(bd, xi, yi, zi, lam[p], order, a);
    nsum s[5];
    memset(s, 0, sizeof s);
    for (int64_t k = 0; k < np; ++k)
      for (int q = 0; q < 5; ++q) nsum_add(&s[q], a[5 * k + q] * (double)B0[k]);
    B[p] = nsum_get(&s[0]);
    if (G)
      for (int j = 0; j < 3; ++j) G[3 * p + j] = nsum_get(&s[1 + j]);
    if (dBdl) dBdl[p] = nsum_get(&s[4]);
  }
  free(a);
}

void orc_eval_many_q9(const orc_boundary* bd, int64_t n, const double* xyz, const double* lam,
                      int32_t order, double* B, double* G, double* dBdl, int32_t nthreads) {
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
#endif
  for (int64_t i = 0; i < n; ++i)
    orc_field_q9(bd, xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], lam + 3 * i, order, B + 3 * i,
                 G ? G + 9 * i : NULL, dBdl ? dBdl + 3 * i : NULL);
}

void orc_vjp_q9(const orc_boundary* bd, int64_t n, const double* xyz, const double* lam,
                const double* gB, int32_t order, double* gB0, int32_t nthreads) {
  const int64_t np = (int64_t)bd->nx * bd->ny;
  /* a_ik for every point and component (n x 3 x np), then the transposed sums in point order */
  double* A = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * 3 * (size_t)np);
#ifdef _OPENMP
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : 1)
#endif
  {
    double* a = (double*)malloc(sizeof(double) * 5 * (size_t)np);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
    for (int64_t i = 0; i < n; ++i)
      for (int p = 0; p < 3; ++p) {
        orc_node_weights_q9(bd, xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], lam[3 * i + p], order, a);
        for (int64_t k = 0; k < np; ++k) A[((size_t)i * 3 + p) * np + k] = a[5 * k];
      }
    free(a);
  }
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
#endif
  for (int64_t k = 0; k < np; ++k)
    for (int p = 0; p < 3; ++p) {
      nsum s = {0, 0};
      for (int64_t i = 0; i < n; ++i) nsum_add(&s, gB[3 * i + p] * A[((size_t)i * 3 + p) * np + k]);
      gB0[3 * k + p] = nsum_get(&s);
    }
  free(A);
}

/* ------------------------------------- pixel-exact near field (piecewise-constant B0) ---- */
/* Exact integral of K0 = z / (2 pi r^3) (the lambda = 0 kernel) over the rectangle
 * [xa, xb] x [ya, yb], given in corner-minus-point coordinates, and its derivatives with respect
 * to the point (x_i, y_i, z_i).  With F(a, b) = arctan(a b / (z R)), R = sqrt(a^2 + b^2 + z^2),
 * the integral is the solid angle over 2 pi,
 *   (1 / 2 pi) [F(xb, yb) - F(xa, yb) - F(xb, ya) + F(xa, ya)],
 * and dF/da = b z / (R (a^2 + z^2)), dF/db = a z / (R (b^2 + z^2)),
 * dF/dz = -a b (R^2 + z^2) / (R (a^2 + z^2) (b^2 + z^2)); a corner coordinate a = x_c - x_i
 * moves as -x_i. */
void orc_rect_exact(double xa, double xb, double ya, double yb, double z, double out[4]) {
  const double cx[2] = {xa, xb}, cy[2] = {ya, yb};
  double v = 0, gx = 0, gy = 0, gz = 0;
  for (int u = 0; u < 2; ++u)
    for (int w = 0; w < 2; ++w) {
      const double s = (u == w) ? 1.0 : -1.0;
      const double a = cx[u], b = cy[w];
      const double R = sqrt(a * a + b * b + z * z);
      v += s * atan(a * b / (z * R));
      gx -= s * (b * z / (R * (a * a + z * z)));
      gy -= s * (a * z / (R * (b * b + z * z)));
      gz -= s * (a * b * (R * R + z * z) / (R * (a * a + z * z) * (b * b + z * z)));
    }
  out[0] = v / TWO_PI;
  out[1] = gx / TWO_PI;
  out[2] = gy / TWO_PI;
  out[3] = gz / TWO_PI;
}

/* Weights of pixel (i, j) in the pixel-exact correction at a point: the exact integral of K0
 * over the pixel minus the midpoint rule's dA K0 at its centre, for B (c[0]) and for the
 * derivatives with respect to the point's x, y, z (c[1..3]); dK0/dx_i = -3 z dx / (2 pi r^5),
 * dK0/dz = (1 / r^3 - 3 z^2 / r^5) / (2 pi). */
static void pxe_pixel_weights(const orc_boundary* bd, double xi, double yi, double zi, int i, int j,
                              double c[4]) {
  const double hx = bd->hx, hy = bd->hy, dA = bd->dA;
  const double xk = bd->x0 + i * hx, yk = bd->y0 + j * hy;
  const double dx = xi - xk, dy = yi - yk;
  const double r2 = dx * dx + dy * dy + zi * zi, r = sqrt(r2), r3 = r2 * r, r5 = r3 * r2;
  double e[4];
  orc_rect_exact(xk - 0.5 * hx - xi, xk + 0.5 * hx - xi, yk - 0.5 * hy - yi, yk + 0.5 * hy - yi,
                 zi, e);
  c[0] = e[0] - dA * zi / (TWO_PI * r3);
  c[1] = e[1] - dA * (-3.0 * zi * dx / (TWO_PI * r5));
  c[2] = e[2] - dA * (-3.0 * zi * dy / (TWO_PI * r5));
  c[3] = e[3] - dA * ((1.0 / r3 - 3.0 * zi * zi / r5) / TWO_PI);
}

void orc_pxe_correction(const orc_boundary* bd, double xi, double yi, double zi, double dB[3],
                        double dG[9]) {
  nsum sB[3], sG[9];
  memset(sB, 0, sizeof sB);
  memset(sG, 0, sizeof sG);
  for (int j = 0; j < bd->ny; ++j)
    for (int i = 0; i < bd->nx; ++i) {
      double c[4];
      pxe_pixel_weights(bd, xi, yi, zi, i, j, c);
      for (int p = 0; p < 3; ++p) {
        const double b0 = (double)comp_ptr(bd, p)[(int64_t)j * bd->nx + i];
        nsum_add(&sB[p], c[0] * b0);
        for (int q = 0; q < 3; ++q) nsum_add(&sG[3 * p + q], c[1 + q] * b0);
      }
    }
  for (int p = 0; p < 3; ++p) {
    dB[p] = nsum_get(&sB[p]);
    for (int q = 0; q < 3; ++q) dG[3 * p + q] = nsum_get(&sG[3 * p + q]);
  }
}

void orc_field_pxe(const orc_boundary* bd, double xi, double yi, double zi, const double lam[3],
                   double near_z, double B[3], double G[9], double dBdl[3]) {
  double Gl[9];
  orc_field(bd, xi, yi, zi, lam, B, Gl, dBdl);
  if (zi <= near_z) {
    double dB[3], dG[9];
    orc_pxe_correction(bd, xi, yi, zi, dB, dG);
    for (int p = 0; p < 3; ++p) B[p] += dB[p];
    for (int q = 0; q < 9; ++q) Gl[q] += dG[q];
  }
  if (G) memcpy(G, Gl, sizeof Gl);
}

void orc_eval_many_pxe(const orc_boundary* bd, int64_t n, const double* xyz, const double* lam,
                       double near_z, double* B, double* G, double* dBdl, int32_t nthreads) {
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
#endif
  for (int64_t i = 0; i < n; ++i)
    orc_field_pxe(bd, xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], lam + 3 * i, near_z, B + 3 * i,
                  G ? G + 9 * i : NULL, dBdl ? dBdl + 3 * i : NULL);
}

void orc_vjp_pxe(const orc_boundary* bd, int64_t n, const double* xyz, const double* lam,
                 const double* gB, double near_z, double* gB0, int32_t nthreads) {
  /* the midpoint adjoint plus, for every point with z <= near_z, its pixel weights c[0] times gB */
  orc_vjp(bd, n, xyz, lam, gB, gB0, nthreads);
  const int64_t nb = (int64_t)bd->nx * bd->ny;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads > 0 ? nthreads : 1)
#endif
  for (int64_t k = 0; k < nb; ++k) {
    const int i = (int)(k % bd->nx), j = (int)(k / bd->nx);
    nsum s[3];
    memset(s, 0, sizeof s);
    for (int64_t q = 0; q < n; ++q) {
      if (!(xyz[3 * q + 2] <= near_z)) continue;
      double c[4];
      pxe_pixel_weights(bd, xyz[3 * q], xyz[3 * q + 1], xyz[3 * q + 2], i, j, c);
      for (int p = 0; p < 3; ++p) nsum_add(&s[p], gB[3 * q + p] * c[0]);
    }
    for (int p = 0; p < 3; ++p) gB0[3 * k + p] += nsum_get(&s[p]);
  }
}
