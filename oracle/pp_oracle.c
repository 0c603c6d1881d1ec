/*
 * pp_oracle.c -- plain FP64 CPU oracle of the positivity-preserving
 * fifth-order finite-volume compact-WENO scheme (Guo, Xiong & Shi).
 *
 * TEST INFRASTRUCTURE ONLY: only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this code.  It shares no code with
 * the CUDA implementation.  It is deliberately written step by step in the
 * order of the paper, with serial Thomas solves and no blocking or fusion.
 *
 * Readings of points where the paper is silent, garbled or ambiguous (the
 * same readings are listed with their reasons in the design notes):
 *  - plus-side reconstruction: mirror image of the minus-side row about the
 *    face; the smoothness indicators are reversed (beta2, beta1, beta0).
 *  - non-periodic lines: the first and last unknown of each system are
 *    closed by the explicit fifth-order WENO-Z reconstruction using two
 *    ghost cells; transmissive ghosts copy the boundary cell, reflective
 *    ghosts mirror the interior with the normal momentum negated; the
 *    exterior state at a boundary face is the boundary condition applied to
 *    the limited interior face state.
 *  - HLLC: S_M has rho_r in its denominator's first term, S_R is a max, and
 *    the right star flux uses S_R (the printed formulas carry typos).
 *  - limiter: rho_min is the minimum of the three listed densities, theta_1
 *    is evaluated only when rho_min < eps; e is the specific internal
 *    energy; theta_2 = 0 if the cell average itself has e <= eps.  Both
 *    thresholds carry a round-off allowance (a bound on the rounding of the
 *    rescaled states) so that the limited states are in G in floating point;
 *    with the exact-arithmetic thresholds a face with large kinetic energy
 *    can land at e < 0 after rounding.
 *  - Gauss-Lobatto end weight omega_hat_1 = 1/12 (M = 4 points) by default.
 *  - 2-D: dimension by dimension, L = L_x + L_y, HLLC at face centres with
 *    the tangential momentum carried by the contact.
 *  - Lax-Friedrichs flux (named in Sec. 3 as a way to control the
 *    oscillations of the near-vacuum double rarefaction): the local form,
 *    the dissipation coefficient being the larger |u| + a of the two face
 *    states; an alternative to HLLC selected per grid.
 *  - characteristic-wise reconstruction (Sec. 2.3), selected per grid: the
 *    eigenvectors of a row come from the Roe average of the two cells
 *    adjacent to the row's face (cells j, j+1 for U^-_{j+1/2}; cells k-1, k
 *    for U^+_{k-1/2}); the weights of field k use that face's l^(k) on all
 *    five cells of the stencil; bounded lines close the first and last
 *    unknown with WENO5-Z on the same characteristic variables; the cyclic
 *    block system is solved with a Woodbury correction; 2-D lines use the
 *    4 x 4 eigensystem with the shear field (0, 0, 1, v).
 */
#include "pp_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

static double sq(double x) { return x * x; }

/* ------------------------------------------------------------------------ */
/* Sec. 2.2: smoothness indicators (the classical Jiang-Shu beta_k).         */
/* ------------------------------------------------------------------------ */
void orc_smoothness(const double *u, double *beta) {
  /* u[0..4] = ubar_{j-2} .. ubar_{j+2} */
  beta[0] = 13.0 / 12.0 * sq(u[0] - 2.0 * u[1] + u[2]) + 0.25 * sq(u[0] - 4.0 * u[1] + 3.0 * u[2]);
  beta[1] = 13.0 / 12.0 * sq(u[1] - 2.0 * u[2] + u[3]) + 0.25 * sq(u[1] - u[3]);
  beta[2] = 13.0 / 12.0 * sq(u[2] - 2.0 * u[3] + u[4]) + 0.25 * sq(3.0 * u[2] - 4.0 * u[3] + u[4]);
}

/* Sec. 2.2, eq. (weight): WENO-Z nonlinear weights. */
void orc_wenoz_weights(const double *beta, const double *c, double eps, double *w) {
  double tau5 = fabs(beta[2] - beta[0]);
  double alpha[3], sum = 0.0;
  for (int k = 0; k < 3; ++k) {
    alpha[k] = c[k] * (1.0 + sq(tau5 / (beta[k] + eps)));
    sum += alpha[k];
  }
  for (int k = 0; k < 3; ++k) w[k] = alpha[k] / sum;
}

/* ------------------------------------------------------------------------ */
/* Tridiagonal solves (Sec. 2.2: "a tri-diagonal system is solved").         */
/* ------------------------------------------------------------------------ */
int orc_thomas(long n, const double *sub, const double *diag, const double *sup,
               const double *rhs, double *x, int reverse) {
  if (n <= 0) return 0;
  double *cp = (double *)malloc(sizeof(double) * (size_t)n);
  double *dp = (double *)malloc(sizeof(double) * (size_t)n);
  if (!cp || !dp) { free(cp); free(dp); return -1; }
  int rc = 0;
  if (!reverse) {
    /* forward elimination i = 0 .. n-1, back substitution n-1 .. 0 */
    for (long i = 0; i < n; ++i) {
      double piv = diag[i] - (i > 0 ? sub[i] * cp[i - 1] : 0.0);
      if (piv == 0.0) { rc = -1; break; }
      cp[i] = (i < n - 1 ? sup[i] : 0.0) / piv;
      dp[i] = (rhs[i] - (i > 0 ? sub[i] * dp[i - 1] : 0.0)) / piv;
    }
    if (rc == 0) {
      x[n - 1] = dp[n - 1];
      for (long i = n - 2; i >= 0; --i) x[i] = dp[i] - cp[i] * x[i + 1];
    }
  } else {
    /* the same algorithm on the reversed ordering: eliminate i = n-1 .. 0 */
    for (long i = n - 1; i >= 0; --i) {
      double piv = diag[i] - (i < n - 1 ? sup[i] * cp[i + 1] : 0.0);
      if (piv == 0.0) { rc = -1; break; }
      cp[i] = (i > 0 ? sub[i] : 0.0) / piv;
      dp[i] = (rhs[i] - (i < n - 1 ? sup[i] * dp[i + 1] : 0.0)) / piv;
    }
    if (rc == 0) {
      x[0] = dp[0];
      for (long i = 1; i < n; ++i) x[i] = dp[i] - cp[i] * x[i - 1];
    }
  }
  free(cp);
  free(dp);
  return rc;
}

/*
 * Cyclic system A x = r with A = T + u v^T (Sherman-Morrison).
 * Natural order: the corner entries are A[0][n-1] = sub[0] and
 * A[n-1][0] = sup[n-1].  With g = -diag[0]:
 *   u = (g, 0, .., 0, sup[n-1]),  v = (1, 0, .., 0, sub[0]/g),
 *   T = A - u v^T  (diag[0] - g, diag[n-1] - sup[n-1] sub[0] / g, no corners),
 *   x = y - (v.y)/(1 + v.z) z  with  T y = r,  T z = u.
 * Reverse order applies the same construction to the reversed system, so
 * that the Thomas eliminations run from i = n-1 downward.
 */
int orc_cyclic(long n, const double *sub, const double *diag, const double *sup,
               const double *rhs, double *x, int reverse) {
  if (n < 3) return -1;
  size_t bytes = sizeof(double) * (size_t)n;
  double *d2 = (double *)malloc(bytes), *u = (double *)malloc(bytes);
  double *y = (double *)malloc(bytes), *z = (double *)malloc(bytes);
  if (!d2 || !u || !y || !z) { free(d2); free(u); free(y); free(z); return -1; }
  memcpy(d2, diag, bytes);
  memset(u, 0, bytes);
  long f = reverse ? n - 1 : 0;  /* first row eliminated */
  long l = reverse ? 0 : n - 1;  /* last row eliminated */
  /* corner couplings in the elimination ordering */
  double corner_f = reverse ? sup[n - 1] : sub[0];   /* row f couples x[l] */
  double corner_l = reverse ? sub[0] : sup[n - 1];   /* row l couples x[f] */
  double g = -diag[f];
  d2[f] = diag[f] - g;
  d2[l] = diag[l] - corner_l * corner_f / g;
  u[f] = g;
  u[l] = corner_l;
  int rc = orc_thomas(n, sub, d2, sup, rhs, y, reverse);
  if (rc == 0) rc = orc_thomas(n, sub, d2, sup, u, z, reverse);
  if (rc == 0) {
    double vy = y[f] + corner_f / g * y[l];
    double vz = z[f] + corner_f / g * z[l];
    double den = 1.0 + vz;
    if (den == 0.0) rc = -1;
    else {
      double fac = vy / den;
      for (long i = 0; i < n; ++i) x[i] = y[i] - fac * z[i];
    }
  }
  free(d2); free(u); free(y); free(z);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.2: compact-WENO reconstruction of a scalar line.                   */
/* ------------------------------------------------------------------------ */
static const double C_COMPACT[3] = {0.2, 0.5, 0.3};   /* optimal c_k, eq. (weight) */
static const double D_WENO5[3] = {0.1, 0.6, 0.3};     /* explicit WENO5 linear weights */

/* explicit fifth-order WENO-Z value u^-_{j+1/2} from u5 = ubar_{j-2..j+2} */
static double weno5z_minus(const double *u5, double eps, int linear) {
  double beta[3], w[3];
  orc_smoothness(u5, beta);
  if (linear) { w[0] = D_WENO5[0]; w[1] = D_WENO5[1]; w[2] = D_WENO5[2]; }
  else orc_wenoz_weights(beta, D_WENO5, eps, w);
  double q0 = (2.0 * u5[0] - 7.0 * u5[1] + 11.0 * u5[2]) / 6.0;
  double q1 = (-u5[1] + 5.0 * u5[2] + 2.0 * u5[3]) / 6.0;
  double q2 = (2.0 * u5[2] + 5.0 * u5[3] - u5[4]) / 6.0;
  return w[0] * q0 + w[1] * q1 + w[2] * q2;
}

/* mirror image: u^+_{j-1/2} from the same five cells */
static double weno5z_plus(const double *u5, double eps, int linear) {
  double r5[5] = {u5[4], u5[3], u5[2], u5[1], u5[0]};
  return weno5z_minus(r5, eps, linear);
}

int orc_recon_scalar(long n, const double *ext, int periodic, double eps_weno,
                     int linear, double *um, double *up) {
  if (n < 3) return -1;
  size_t bytes = sizeof(double) * (size_t)n;
  double *sub = (double *)malloc(bytes), *dia = (double *)malloc(bytes);
  double *sup = (double *)malloc(bytes), *rhs = (double *)malloc(bytes);
  double *wm = (double *)malloc(3 * bytes), *wp = (double *)malloc(3 * bytes);
  if (!sub || !dia || !sup || !rhs || !wm || !wp) {
    free(sub); free(dia); free(sup); free(rhs); free(wm); free(wp);
    return -1;
  }
  const double *u = ext + 2;  /* u[j] = ubar_j, valid for j = -2 .. n+1 */

  /* weights of every cell: minus side from (beta0, beta1, beta2), plus side
   * from the mirrored stencil, i.e. (beta2, beta1, beta0) */
  for (long j = 0; j < n; ++j) {
    double beta[3], brev[3];
    orc_smoothness(u + j - 2, beta);
    brev[0] = beta[2]; brev[1] = beta[1]; brev[2] = beta[0];
    if (linear) {
      for (int k = 0; k < 3; ++k) wm[3 * j + k] = wp[3 * j + k] = C_COMPACT[k];
    } else {
      orc_wenoz_weights(beta, C_COMPACT, eps_weno, wm + 3 * j);
      orc_wenoz_weights(brev, C_COMPACT, eps_weno, wp + 3 * j);
    }
  }

  /* minus system, eq. (CWENO-FV): row j couples x_{j-1}, x_j, x_{j+1} with
   * x_j = u~_{j+1/2} */
  for (long j = 0; j < n; ++j) {
    const double *w = wm + 3 * j;
    sub[j] = (2.0 * w[0] + w[1]) / 3.0;
    dia[j] = (w[0] + 2.0 * (w[1] + w[2])) / 3.0;
    sup[j] = w[2] / 3.0;
    rhs[j] = w[0] / 6.0 * u[j - 1] + (5.0 * (w[0] + w[1]) + w[2]) / 6.0 * u[j] +
             (w[1] + 5.0 * w[2]) / 6.0 * u[j + 1];
  }
  int rc;
  if (periodic) {
    rc = orc_cyclic(n, sub, dia, sup, rhs, um, 0);
  } else {
    /* closure rows: first and last unknown from explicit WENO5-Z */
    sub[0] = 0.0; dia[0] = 1.0; sup[0] = 0.0; rhs[0] = weno5z_minus(u - 2, eps_weno, linear);
    sub[n - 1] = 0.0; dia[n - 1] = 1.0; sup[n - 1] = 0.0;
    rhs[n - 1] = weno5z_minus(u + n - 3, eps_weno, linear);
    rc = orc_thomas(n, sub, dia, sup, rhs, um, 0);
  }

  /* plus system: mirror of eq. (CWENO-FV) about the face; row k couples
   * y_{k-1}, y_k, y_{k+1} with y_k = u~^+_{k-1/2}; eliminated from the right */
  if (rc == 0) {
    for (long k = 0; k < n; ++k) {
      const double *w = wp + 3 * k;
      sub[k] = w[2] / 3.0;
      dia[k] = (w[0] + 2.0 * (w[1] + w[2])) / 3.0;
      sup[k] = (2.0 * w[0] + w[1]) / 3.0;
      rhs[k] = (w[1] + 5.0 * w[2]) / 6.0 * u[k - 1] + (5.0 * (w[0] + w[1]) + w[2]) / 6.0 * u[k] +
               w[0] / 6.0 * u[k + 1];
    }
    if (periodic) {
      rc = orc_cyclic(n, sub, dia, sup, rhs, up, 1);
    } else {
      sub[0] = 0.0; dia[0] = 1.0; sup[0] = 0.0; rhs[0] = weno5z_plus(u - 2, eps_weno, linear);
      sub[n - 1] = 0.0; dia[n - 1] = 1.0; sup[n - 1] = 0.0;
      rhs[n - 1] = weno5z_plus(u + n - 3, eps_weno, linear);
      rc = orc_thomas(n, sub, dia, sup, rhs, up, 1);
    }
  }
  free(sub); free(dia); free(sup); free(rhs); free(wm); free(wp);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Sec. 1 and Sec. 2.4: Euler physics and the HLLC flux.                     */
/* ------------------------------------------------------------------------ */
static double kinetic(int nv, const double *U) {
  /* rho |u|^2 / 2 */
  double m2 = U[1] * U[1] + (nv == 4 ? U[2] * U[2] : 0.0);
  return 0.5 * m2 / U[0];
}

static double pressure(int nv, double gamma, const double *U) {
  return (gamma - 1.0) * (U[nv - 1] - kinetic(nv, U));
}

void orc_hllc_batch(int nv, double gamma, long n, const double *Ul, const double *Ur, double *F) {
  for (long i = 0; i < n; ++i) orc_hllc(nv, gamma, Ul + i * nv, Ur + i * nv, F + i * nv);
}

void orc_flux(int nv, double gamma, const double *U, double *F) {
  double rho = U[0], un = U[1] / rho, p = pressure(nv, gamma, U), E = U[nv - 1];
  F[0] = U[1];
  F[1] = U[1] * un + p;
  if (nv == 4) F[2] = U[2] * un;
  F[nv - 1] = un * (E + p);
}

void orc_hllc(int nv, double gamma, const double *Ul, const double *Ur, double *F) {
  double rl = Ul[0], rr = Ur[0];
  double ul = Ul[1] / rl, ur = Ur[1] / rr;
  double vl = nv == 4 ? Ul[2] / rl : 0.0, vr = nv == 4 ? Ur[2] / rr : 0.0;
  double El = Ul[nv - 1], Er = Ur[nv - 1];
  double pl = pressure(nv, gamma, Ul), pr = pressure(nv, gamma, Ur);
  double al = sqrt(gamma * pl / rl), ar = sqrt(gamma * pr / rr);   /* eq. (sspeed) */
  double Hl = (El + pl) / rl, Hr = (Er + pr) / rr;

  /* eq. (acoustic ws): Roe-type averages and Batten's wave speeds */
  double Rrho = sqrt(rr / rl);
  double ut = (ul + ur * Rrho) / (1.0 + Rrho);
  double vt = (vl + vr * Rrho) / (1.0 + Rrho);
  double Ht = (Hl + Hr * Rrho) / (1.0 + Rrho);
  double at = sqrt((gamma - 1.0) * (Ht - 0.5 * (ut * ut + vt * vt)));
  double SL = fmin(ul - al, ut - at);
  double SR = fmax(ur + ar, ut + at);

  /* eq. (contact-v) */
  double SM = (rr * ur * (SR - ur) - rl * ul * (SL - ul) + pl - pr) /
              (rr * (SR - ur) - rl * (SL - ul));

  double Fl[4], Fr[4];
  if (SL > 0.0) {
    orc_flux(nv, gamma, Ul, F);
  } else if (SM > 0.0) {
    /* F*_l = F_l + S_L (U*_l - U_l), eq. (star-l) */
    double Us[4];
    double ps = rl * (ul - SL) * (ul - SM) + pl;
    Us[0] = rl * (SL - ul) / (SL - SM);
    Us[1] = ((SL - ul) * rl * ul + (ps - pl)) / (SL - SM);
    if (nv == 4) Us[2] = Us[0] * vl;
    Us[nv - 1] = ((SL - ul) * El - pl * ul + ps * SM) / (SL - SM);
    orc_flux(nv, gamma, Ul, Fl);
    for (int k = 0; k < nv; ++k) F[k] = Fl[k] + SL * (Us[k] - Ul[k]);
  } else if (SR >= 0.0) {
    /* F*_r = F_r + S_R (U*_r - U_r), right star state by symmetry */
    double Us[4];
    double ps = rr * (ur - SR) * (ur - SM) + pr;
    Us[0] = rr * (SR - ur) / (SR - SM);
    Us[1] = ((SR - ur) * rr * ur + (ps - pr)) / (SR - SM);
    if (nv == 4) Us[2] = Us[0] * vr;
    Us[nv - 1] = ((SR - ur) * Er - pr * ur + ps * SM) / (SR - SM);
    orc_flux(nv, gamma, Ur, Fr);
    for (int k = 0; k < nv; ++k) F[k] = Fr[k] + SR * (Us[k] - Ur[k]);
  } else {
    orc_flux(nv, gamma, Ur, F);
  }
}

/* Sec. 3 (double rarefaction remark): the Lax-Friedrichs flux, here its
 * local form with the largest signal speed |u| + a of the two face states */
void orc_llf(int nv, double gamma, const double *Ul, const double *Ur, double *F) {
  double Fl[4], Fr[4];
  orc_flux(nv, gamma, Ul, Fl);
  orc_flux(nv, gamma, Ur, Fr);
  double al = fabs(Ul[1] / Ul[0]) + sqrt(gamma * pressure(nv, gamma, Ul) / Ul[0]);
  double ar = fabs(Ur[1] / Ur[0]) + sqrt(gamma * pressure(nv, gamma, Ur) / Ur[0]);
  double alpha = fmax(al, ar);
  for (int k = 0; k < nv; ++k) F[k] = 0.5 * (Fl[k] + Fr[k]) - 0.5 * alpha * (Ur[k] - Ul[k]);
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.3: characteristic-wise compact-WENO reconstruction of a line.      */
/* ------------------------------------------------------------------------ */
/* Solve M X = Y in place for m x m matrix M (row-major) and ncol columns of
 * Y ([m][ncol], overwritten with X): Gaussian elimination with partial
 * pivoting.  Returns -1 on a zero pivot. */
static int dense_solve(int m, double *M, int ncol, double *Y) {
  for (int k = 0; k < m; ++k) {
    int p = k;
    for (int i = k + 1; i < m; ++i)
      if (fabs(M[i * m + k]) > fabs(M[p * m + k])) p = i;
    if (M[p * m + k] == 0.0) return -1;
    if (p != k) {
      for (int c = 0; c < m; ++c) { double t = M[k * m + c]; M[k * m + c] = M[p * m + c]; M[p * m + c] = t; }
      for (int c = 0; c < ncol; ++c) { double t = Y[k * ncol + c]; Y[k * ncol + c] = Y[p * ncol + c]; Y[p * ncol + c] = t; }
    }
    for (int i = k + 1; i < m; ++i) {
      double f = M[i * m + k] / M[k * m + k];
      for (int c = k; c < m; ++c) M[i * m + c] -= f * M[k * m + c];
      for (int c = 0; c < ncol; ++c) Y[i * ncol + c] -= f * Y[k * ncol + c];
    }
  }
  for (int k = m - 1; k >= 0; --k)
    for (int c = 0; c < ncol; ++c) {
      double s = Y[k * ncol + c];
      for (int j = k + 1; j < m; ++j) s -= M[k * m + j] * Y[j * ncol + c];
      Y[k * ncol + c] = s / M[k * m + k];
    }
  return 0;
}

/* Sec. 2.3: Roe average of two conserved states and the left / right
 * eigenvectors of the flux Jacobian there (eqs. (eigen), (reigenv),
 * (leigenv)); nv = 4 adds the tangential velocity v: eigenvalues u - a, u,
 * u, u + a with the shear eigenvector (0, 0, 1, v). */
void orc_roe_eigen(int nv, double gamma, const double *Ua, const double *Ub, double *Lm, double *Rm) {
  double sa = sqrt(Ua[0]), sb = sqrt(Ub[0]);
  double pa = pressure(nv, gamma, Ua), pb = pressure(nv, gamma, Ub);
  double u = (Ua[1] / sa + Ub[1] / sb) / (sa + sb);
  double v = nv == 4 ? (Ua[2] / sa + Ub[2] / sb) / (sa + sb) : 0.0;
  double H = ((Ua[nv - 1] + pa) / sa + (Ub[nv - 1] + pb) / sb) / (sa + sb);
  double q2 = u * u + v * v;
  double a = sqrt((gamma - 1.0) * (H - 0.5 * q2));
  double c1 = (gamma - 1.0) / (a * a), c2 = 0.5 * q2 * c1;
  if (nv == 3) {
    double R[9] = {1.0, 1.0, 1.0,
                   u - a, u, u + a,
                   H - u * a, 0.5 * u * u, H + u * a};
    double L[9] = {0.5 * (c2 + u / a), 0.5 * (-c1 * u - 1.0 / a), 0.5 * c1,
                   1.0 - c2, c1 * u, -c1,
                   0.5 * (c2 - u / a), 0.5 * (-c1 * u + 1.0 / a), 0.5 * c1};
    memcpy(Rm, R, sizeof R);
    memcpy(Lm, L, sizeof L);
  } else {
    double R[16] = {1.0, 1.0, 0.0, 1.0,
                    u - a, u, 0.0, u + a,
                    v, v, 1.0, v,
                    H - u * a, 0.5 * q2, v, H + u * a};
    double L[16] = {0.5 * (c2 + u / a), 0.5 * (-c1 * u - 1.0 / a), -0.5 * c1 * v, 0.5 * c1,
                    1.0 - c2, c1 * u, c1 * v, -c1,
                    -v, 0.0, 1.0, 0.0,
                    0.5 * (c2 - u / a), 0.5 * (-c1 * u + 1.0 / a), -0.5 * c1 * v, 0.5 * c1};
    memcpy(Rm, R, sizeof R);
    memcpy(Lm, L, sizeof L);
  }
}

/* Block tridiagonal system with m x m blocks and ncol right-hand sides:
 *   A[i] x[i-1] + B[i] x[i] + C[i] x[i+1] = r[i],  i = 0..n-1
 * A, B, C are [n][m][m] (A[0], C[n-1] ignored), r and x [n][m][ncol].
 * Block Thomas elimination; reverse = 1 eliminates from i = n-1 downward. */
int orc_block_thomas(long n, int m, const double *A, const double *B, const double *C,
                     const double *r, int ncol, double *x, int reverse) {
  const long mm = (long)m * m, mc = (long)m * ncol;
  double *Y = (double *)malloc(sizeof(double) * (size_t)(n * mm));   /* Bp^{-1} (next block) */
  double *g = (double *)malloc(sizeof(double) * (size_t)(n * mc));
  double Bp[16], T[16 * 5];
  if (!Y || !g) { free(Y); free(g); return -1; }
  int rc = 0;
  for (long s = 0; s < n && rc == 0; ++s) {
    long i = reverse ? n - 1 - s : s;         /* row being eliminated */
    long ip = reverse ? i + 1 : i - 1;        /* previously eliminated neighbour */
    const double *lo = reverse ? C + i * mm : A + i * mm;   /* couples the previous row */
    const double *hi = reverse ? A + i * mm : C + i * mm;   /* couples the next row */
    /* Bp = B_i - lo Y_prev, rhs = r_i - lo g_prev */
    for (int a = 0; a < m; ++a) {
      for (int b = 0; b < m; ++b) {
        double t = B[i * mm + a * m + b];
        if (s > 0) for (int k = 0; k < m; ++k) t -= lo[a * m + k] * Y[ip * mm + k * m + b];
        Bp[a * m + b] = t;
      }
    }
    /* T = [hi | rhs] with m + ncol columns, solved against Bp */
    int w = m + ncol;
    for (int a = 0; a < m; ++a) {
      for (int b = 0; b < m; ++b) T[a * w + b] = hi[a * m + b];
      for (int c = 0; c < ncol; ++c) {
        double t = r[i * mc + a * ncol + c];
        if (s > 0) for (int k = 0; k < m; ++k) t -= lo[a * m + k] * g[ip * mc + k * ncol + c];
        T[a * w + m + c] = t;
      }
    }
    rc = dense_solve(m, Bp, w, T);
    for (int a = 0; a < m; ++a) {
      for (int b = 0; b < m; ++b) Y[i * mm + a * m + b] = T[a * w + b];
      for (int c = 0; c < ncol; ++c) g[i * mc + a * ncol + c] = T[a * w + m + c];
    }
  }
  /* back substitution: x_i = g_i - Y_i x_next */
  for (long s = n - 1; s >= 0 && rc == 0; --s) {
    long i = reverse ? n - 1 - s : s;
    long in = reverse ? i - 1 : i + 1;
    for (int a = 0; a < m; ++a)
      for (int c = 0; c < ncol; ++c) {
        double t = g[i * mc + a * ncol + c];
        if (s < n - 1) for (int k = 0; k < m; ++k) t -= Y[i * mm + a * m + k] * x[in * mc + k * ncol + c];
        x[i * mc + a * ncol + c] = t;
      }
  }
  free(Y); free(g);
  return rc;
}

/* Cyclic block tridiagonal system (A[0] couples x[n-1], C[n-1] couples
 * x[0]), one right-hand side: Woodbury correction of a block Thomas solve.
 * With G = -B[0], T = T' + U V^T where U = (G, 0, .., 0, C[n-1]) and
 * V^T = (I, 0, .., 0, G^{-1} A[0]); T' has B'[0] = B[0] - G and
 * B'[n-1] = B[n-1] - C[n-1] G^{-1} A[0] and no corners.  Then
 * x = y - Z (I + V^T Z)^{-1} V^T y with T' y = r, T' Z = U. */
int orc_block_cyclic(long n, int m, const double *A, const double *B, const double *C,
                     const double *r, double *x, int reverse) {
  const long mm = (long)m * m;
  double *Bm = (double *)malloc(sizeof(double) * (size_t)(n * mm));
  double *Um = (double *)calloc((size_t)(n * mm), sizeof(double));
  double *Z = (double *)malloc(sizeof(double) * (size_t)(n * mm));
  double *y = (double *)malloc(sizeof(double) * (size_t)(n * m));
  if (!Bm || !Um || !Z || !y) { free(Bm); free(Um); free(Z); free(y); return -1; }
  double G[16], GiA[16], Gc[16];
  for (int k = 0; k < mm; ++k) { G[k] = -B[k]; Gc[k] = G[k]; GiA[k] = A[k]; }
  int rc = dense_solve(m, Gc, m, GiA);     /* GiA = G^{-1} A[0] */
  memcpy(Bm, B, sizeof(double) * (size_t)(n * mm));
  for (int k = 0; k < mm; ++k) Bm[k] = B[k] - G[k];
  for (int a = 0; a < m; ++a)
    for (int b = 0; b < m; ++b) {
      double t = 0.0;
      for (int k = 0; k < m; ++k) t += C[(n - 1) * mm + a * m + k] * GiA[k * m + b];
      Bm[(n - 1) * mm + a * m + b] -= t;
    }
  for (int k = 0; k < mm; ++k) { Um[k] = G[k]; Um[(n - 1) * mm + k] = C[(n - 1) * mm + k]; }
  if (rc == 0) rc = orc_block_thomas(n, m, A, Bm, C, r, 1, y, reverse);
  if (rc == 0) rc = orc_block_thomas(n, m, A, Bm, C, Um, m, Z, reverse);
  if (rc == 0) {
    /* S = I + V^T Z (m x m), t = V^T y */
    double S[16], t[4];
    for (int a = 0; a < m; ++a) {
      for (int b = 0; b < m; ++b) {
        double s = (a == b ? 1.0 : 0.0) + Z[a * m + b];
        for (int k = 0; k < m; ++k) s += GiA[a * m + k] * Z[(n - 1) * mm + k * m + b];
        S[a * m + b] = s;
      }
      double s = y[a];
      for (int k = 0; k < m; ++k) s += GiA[a * m + k] * y[(n - 1) * m + k];
      t[a] = s;
    }
    rc = dense_solve(m, S, 1, t);
    for (long i = 0; i < n && rc == 0; ++i)
      for (int a = 0; a < m; ++a) {
        double s = y[i * m + a];
        for (int k = 0; k < m; ++k) s -= Z[i * mm + a * m + k] * t[k];
        x[i * m + a] = s;
      }
  }
  free(Bm); free(Um); free(Z); free(y);
  return rc;
}

/* The characteristic-wise reconstruction of Sec. 2.3, steps 1-4, on one line
 * of nv conserved variables.  ext is [nv][n+4] with two ghost cells per
 * side; um, up are [nv][n] like the component-wise form.
 * Minus system: unknown j is U~_{j+1/2}; its row is the scalar row of
 * eq. (CWENO-FV) for every characteristic field k, multiplied by the left
 * eigenvector l^(k) at the Roe average of cells j and j+1 (eq. (cha-1)),
 * the weights coming from the characteristic variables l^(k) ubar_i of the
 * five cells j-2..j+2; eq. (1DEuler-FVC) is the resulting block system.
 * Plus system: unknown k is U~^+_{k-1/2} at the Roe average of cells k-1
 * and k, with the mirrored row and indicators of the component-wise form.
 * Bounded lines close the first and last unknown with the explicit WENO5-Z
 * value of each characteristic variable (same face eigenvectors). */
int orc_recon_char(int nv, long n, const double *ext, int periodic, double gamma,
                   double eps_weno, int linear, double *um, double *up) {
  if (n < 3) return -1;
  const long s = n + 4, mm = (long)nv * nv;
  double *A = (double *)calloc((size_t)(n * mm), sizeof(double));
  double *B = (double *)calloc((size_t)(n * mm), sizeof(double));
  double *C = (double *)calloc((size_t)(n * mm), sizeof(double));
  double *r = (double *)calloc((size_t)(n * nv), sizeof(double));
  double *x = (double *)malloc(sizeof(double) * (size_t)(n * nv));
  if (!A || !B || !C || !r || !x) { free(A); free(B); free(C); free(r); free(x); return -1; }
  int rc = 0;
  for (int side = 0; side < 2 && rc == 0; ++side) {
    for (long j = 0; j < n; ++j) {
      /* step 1: eigenvectors at the row's face (j+1/2 minus, j-1/2 plus) */
      double Ua[4], Ub[4], Lm[16], Rm[16];
      long ca = side == 0 ? j : j - 1;
      for (int v = 0; v < nv; ++v) { Ua[v] = ext[v * s + ca + 2]; Ub[v] = ext[v * s + ca + 3]; }
      orc_roe_eigen(nv, gamma, Ua, Ub, Lm, Rm);
      /* characteristic variables of the five cells j-2..j+2 */
      double w5[4][5];
      for (int k = 0; k < nv; ++k)
        for (int q = 0; q < 5; ++q) {
          double t = 0.0;
          for (int v = 0; v < nv; ++v) t += Lm[k * nv + v] * ext[v * s + j + q];
          w5[k][q] = t;
        }
      int closure = !periodic && (j == 0 || j == n - 1);
      for (int k = 0; k < nv; ++k) {
        const double *lk = Lm + k * nv;
        if (closure) {
          double val = side == 0 ? weno5z_minus(w5[k], eps_weno, linear)
                                 : weno5z_plus(w5[k], eps_weno, linear);
          for (int v = 0; v < nv; ++v) B[j * mm + k * nv + v] = lk[v];
          r[j * nv + k] = val;
          continue;
        }
        /* step 2: weights of field k (mirrored indicators on the plus side) */
        double beta[3], bw[3], w[3];
        orc_smoothness(w5[k], beta);
        if (side == 0) { bw[0] = beta[0]; bw[1] = beta[1]; bw[2] = beta[2]; }
        else { bw[0] = beta[2]; bw[1] = beta[1]; bw[2] = beta[0]; }
        if (linear) { w[0] = C_COMPACT[0]; w[1] = C_COMPACT[1]; w[2] = C_COMPACT[2]; }
        else orc_wenoz_weights(bw, C_COMPACT, eps_weno, w);
        /* step 3: the scalar row's coefficients */
        double a, b, c, dm, dc, dp;   /* on x_{j-1}, x_j, x_{j+1}; on ubar_{j-1}, ubar_j, ubar_{j+1} */
        if (side == 0) {
          a = (2.0 * w[0] + w[1]) / 3.0; b = (w[0] + 2.0 * (w[1] + w[2])) / 3.0; c = w[2] / 3.0;
          dm = w[0] / 6.0; dc = (5.0 * (w[0] + w[1]) + w[2]) / 6.0; dp = (w[1] + 5.0 * w[2]) / 6.0;
        } else {
          a = w[2] / 3.0; b = (w[0] + 2.0 * (w[1] + w[2])) / 3.0; c = (2.0 * w[0] + w[1]) / 3.0;
          dm = (w[1] + 5.0 * w[2]) / 6.0; dc = (5.0 * (w[0] + w[1]) + w[2]) / 6.0; dp = w[0] / 6.0;
        }
        /* step 4: block row = coefficient x l^(k) */
        for (int v = 0; v < nv; ++v) {
          A[j * mm + k * nv + v] = a * lk[v];
          B[j * mm + k * nv + v] = b * lk[v];
          C[j * mm + k * nv + v] = c * lk[v];
        }
        r[j * nv + k] = dm * w5[k][1] + dc * w5[k][2] + dp * w5[k][3];
      }
    }
    rc = periodic ? orc_block_cyclic(n, nv, A, B, C, r, x, side)
                  : orc_block_thomas(n, nv, A, B, C, r, 1, x, side);
    double *out = side == 0 ? um : up;
    for (long j = 0; j < n; ++j)
      for (int v = 0; v < nv; ++v) out[v * n + j] = x[j * nv + v];
    memset(A, 0, sizeof(double) * (size_t)(n * mm));
    memset(B, 0, sizeof(double) * (size_t)(n * mm));
    memset(C, 0, sizeof(double) * (size_t)(n * mm));
  }
  free(A); free(B); free(C); free(r); free(x);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.4: the positivity-preserving limiter, steps 1-4.                    */
/* ------------------------------------------------------------------------ */

/* Unit round-off of FP64. */
#define ORC_U 1.1102230246251565e-16

/* g(W) = rho E - |m|^2 / 2 - eps rho^2; for rho > 0, e(W) >= eps iff g >= 0 */
static double energy_form(int nv, double eps, const double *w) {
  double m2 = w[1] * w[1] + (nv == 4 ? w[2] * w[2] : 0.0);
  return w[0] * w[nv - 1] - 0.5 * m2 - eps * w[0] * w[0];
}

/* Round-off allowance of g along the segment from ubar to w: every state
 * (1-t) ubar + t w is formed with an error of a few ulps of |ubar| + |w| per
 * component, which moves the bilinear form g by at most a small multiple of
 * u [(|E|+|E_w|)(|rho|+|rho_w|) + (|m|+|m_w|)^2].  Requiring g >= eta rather
 * than g >= 0 keeps the rounded limited states inside G. */
static double energy_allowance(int nv, const double *ubar, const double *w) {
  double sm = 0.0;
  for (int k = 1; k < nv - 1; ++k) sm += (fabs(ubar[k]) + fabs(w[k])) * (fabs(ubar[k]) + fabs(w[k]));
  return 16.0 * ORC_U *
         ((fabs(ubar[nv - 1]) + fabs(w[nv - 1])) * (fabs(ubar[0]) + fabs(w[0])) + sm);
}

/* root t in (0, 1] of g((1-t) ubar + t w) = eta, a quadratic
 * A t^2 + B t + (C - eta) = 0 with C - eta > 0 at t = 0 and < 0 at t = 1;
 * the cancellation-free form 2C'/(-B + sqrt(B^2 - 4AC')) is the root in (0,1) */
static double energy_root(int nv, double eps, double eta, const double *ubar, const double *w) {
  double dr = w[0] - ubar[0], dE = w[nv - 1] - ubar[nv - 1];
  double dm1 = w[1] - ubar[1], dm2 = nv == 4 ? w[2] - ubar[2] : 0.0;
  double m1 = ubar[1], m2 = nv == 4 ? ubar[2] : 0.0;
  double A = dE * dr - 0.5 * (dm1 * dm1 + dm2 * dm2) - eps * dr * dr;
  double B = ubar[nv - 1] * dr + dE * ubar[0] - (m1 * dm1 + m2 * dm2) - 2.0 * eps * ubar[0] * dr;
  double C = ubar[nv - 1] * ubar[0] - 0.5 * (m1 * m1 + m2 * m2) - eps * ubar[0] * ubar[0] - eta;
  if (!(C > 0.0)) return 0.0;
  double D = B * B - 4.0 * A * C;
  if (D < 0.0) D = 0.0;
  double den = -B + sqrt(D);
  double t = den > 0.0 ? 2.0 * C / den : 0.0;
  if (!(t >= 0.0)) t = 0.0;
  if (t > 1.0) t = 1.0;
  return t;
}

int orc_limit_cell(int nv, double gamma, double wgl, double eps,
                   const double *ubar, double *um, double *up) {
  (void)gamma;
  int flags = 0;
  /* step 2: theta_1 from the minimum density over the two face values and
   * the interior point value rho_j(x^{1*}) implied by the quadrature; the
   * threshold carries the round-off allowance of forming the scaled values */
  double rho_star = (ubar[0] - wgl * up[0] - wgl * um[0]) / (1.0 - 2.0 * wgl);
  double rho_min = fmin(fmin(um[0], up[0]), rho_star);
  double eps_r = eps + 8.0 * ORC_U * (fabs(ubar[0]) + fabs(rho_min));
  double theta1 = 1.0;
  if (rho_min < eps_r) {
    theta1 = fmin(fmax((ubar[0] - eps_r) / (ubar[0] - rho_min), 0.0), 1.0);
    flags |= 1;
  }
  /* step 3, eq. (limiter-rho): rescale the density face values (theta_1 = 1
   * is the identity and is skipped, so unlimited cells stay bit-identical) */
  if (theta1 < 1.0) {
    um[0] = theta1 * (um[0] - ubar[0]) + ubar[0];
    up[0] = theta1 * (up[0] - ubar[0]) + ubar[0];
  }

  /* W^1 = U^-_{j+1/2}, W^2 = U^+_{j-1/2}, W^3 = interior point */
  double W[3][4];
  for (int k = 0; k < nv; ++k) {
    W[0][k] = um[k];
    W[1][k] = up[k];
    W[2][k] = (ubar[k] - wgl * up[k] - wgl * um[k]) / (1.0 - 2.0 * wgl);
  }
  /* step 4: theta_2 = min over the three points of t_eps; a point needs
   * limiting when e(W) < eps, i.e. g(W) < 0, checked with the allowance */
  double theta2 = 1.0;
  for (int a = 0; a < 3; ++a) {
    double eta = energy_allowance(nv, ubar, W[a]);
    if (energy_form(nv, eps, W[a]) < eta) {
      double t = energy_root(nv, eps, eta, ubar, W[a]);
      if (t < theta2) theta2 = t;
    }
  }
  if (theta2 < 1.0) {
    flags |= 2;
    for (int k = 0; k < nv; ++k) {
      um[k] = theta2 * (um[k] - ubar[k]) + ubar[k];
      up[k] = theta2 * (up[k] - ubar[k]) + ubar[k];
    }
  }
  return flags;
}

/* ------------------------------------------------------------------------ */
/* One grid line: ghost cells, reconstruction, limiter, HLLC, difference.    */
/* ------------------------------------------------------------------------ */
/* vars of a line: 0 = rho, 1 = normal momentum, (2 = tangential), nv-1 = E */
static void ghost(int nv, long n, double *ext /* [nv][n+4] */, int bclo, int bchi) {
  long s = n + 4;
  for (int v = 0; v < nv; ++v) {
    double *e = ext + v * s;   /* e[j+2] = ubar_j */
    for (int g = 1; g <= 2; ++g) {
      /* low side: cells -1, -2 */
      double lo, hi;
      if (bclo == ORC_BC_PERIODIC) lo = e[2 + n - g];
      else if (bclo == ORC_BC_TRANSMISSIVE) lo = e[2];
      else lo = (v == 1 ? -1.0 : 1.0) * e[2 + g - 1];
      if (bchi == ORC_BC_PERIODIC) hi = e[2 + g - 1];
      else if (bchi == ORC_BC_TRANSMISSIVE) hi = e[2 + n - 1];
      else hi = (v == 1 ? -1.0 : 1.0) * e[2 + n - g];
      e[2 - g] = lo;
      e[2 + n - 1 + g] = hi;
    }
  }
}

static void boundary_state(int nv, int bc, const double *in, double *out) {
  for (int k = 0; k < nv; ++k) out[k] = in[k];
  if (bc == ORC_BC_REFLECTIVE) out[1] = -in[1];
}

/* line[v*n + j] in, Lout[v*n + j] += -(F_{j+1/2} - F_{j-1/2})/h */
static int line_operator(const orc_grid *g, int nv, long n, const double *line, int bclo,
                         int bchi, double h, double eps, double *Lout, orc_counters *cnt,
                         double *smax) {
  long s = n + 4;
  int periodic = (bclo == ORC_BC_PERIODIC);
  double *ext = (double *)malloc(sizeof(double) * (size_t)(nv * s));
  double *um = (double *)malloc(sizeof(double) * (size_t)(nv * n));
  double *up = (double *)malloc(sizeof(double) * (size_t)(nv * n));
  double *fl = (double *)malloc(sizeof(double) * (size_t)(nv * (n + 1)));
  double *tm = (double *)malloc(sizeof(double) * (size_t)n);
  double *tp = (double *)malloc(sizeof(double) * (size_t)n);
  int rc = 0;
  if (!ext || !um || !up || !fl || !tm || !tp) rc = -1;

  if (rc == 0) {
    for (int v = 0; v < nv; ++v) memcpy(ext + v * s + 2, line + v * n, sizeof(double) * (size_t)n);
    ghost(nv, n, ext, bclo, bchi);
    if (g->recon) {
      /* characteristic-wise reconstruction, Sec. 2.3 */
      rc = orc_recon_char(nv, n, ext, periodic, g->gamma, g->eps_weno, g->linear_weights, um, up);
    } else {
      /* component-wise reconstruction of the conserved variables */
      for (int v = 0; v < nv && rc == 0; ++v) {
        rc = orc_recon_scalar(n, ext + v * s, periodic, g->eps_weno, g->linear_weights, tm, tp);
        for (long j = 0; j < n; ++j) { um[v * n + j] = tm[j]; up[v * n + j] = tp[j]; }
      }
    }
  }
  if (rc == 0 && g->limiter) {
    for (long j = 0; j < n; ++j) {
      double ub[4], a[4], b[4];
      for (int v = 0; v < nv; ++v) { ub[v] = line[v * n + j]; a[v] = um[v * n + j]; b[v] = up[v * n + j]; }
      int f = orc_limit_cell(nv, g->gamma, g->gl_weight, eps, ub, a, b);
      if (cnt) { if (f & 1) cnt->theta1_active++; if (f & 2) cnt->theta2_active++; }
      for (int v = 0; v < nv; ++v) { um[v * n + j] = a[v]; up[v * n + j] = b[v]; }
    }
  }
  if (rc == 0 && smax) {
    /* the largest |u| + a over the face values the fluxes use (the states
     * of the first-order steps in the proof of the theorem of Sec. 2.4;
     * boundary exteriors repeat an interior face's speed) */
    double s = 0.0;
    for (long j = 0; j < n; ++j) {
      for (int side = 0; side < 2; ++side) {
        const double *w = side ? up : um;
        double W[4];
        for (int v = 0; v < nv; ++v) W[v] = w[v * n + j];
        double p = pressure(nv, g->gamma, W);
        double a = sqrt(fmax(g->gamma * p / W[0], 0.0));
        double sp = fabs(W[1] / W[0]) + a;
        if (sp > s || sp != sp) s = sp;   /* a NaN speed stays */
      }
    }
    *smax = s;
  }
  if (rc == 0) {
    /* faces f = 0..n: face f lies between cells f-1 and f */
    for (long f = 0; f <= n; ++f) {
      double Ul[4], Ur[4], F[4];
      if (f == 0) {
        for (int v = 0; v < nv; ++v) Ur[v] = up[v * n + 0];
        if (periodic) { for (int v = 0; v < nv; ++v) Ul[v] = um[v * n + n - 1]; }
        else boundary_state(nv, bclo, Ur, Ul);
      } else if (f == n) {
        for (int v = 0; v < nv; ++v) Ul[v] = um[v * n + n - 1];
        if (periodic) { for (int v = 0; v < nv; ++v) Ur[v] = up[v * n + 0]; }
        else boundary_state(nv, bchi, Ul, Ur);
      } else {
        for (int v = 0; v < nv; ++v) { Ul[v] = um[v * n + f - 1]; Ur[v] = up[v * n + f]; }
      }
      if (g->flux) orc_llf(nv, g->gamma, Ul, Ur, F);
      else orc_hllc(nv, g->gamma, Ul, Ur, F);
      for (int v = 0; v < nv; ++v) fl[v * (n + 1) + f] = F[v];
    }
    /* eq. (1DEulerFV-b) */
    for (int v = 0; v < nv; ++v)
      for (long j = 0; j < n; ++j)
        Lout[v * n + j] += -(fl[v * (n + 1) + j + 1] - fl[v * (n + 1) + j]) / h;
  }
  free(ext); free(um); free(up); free(fl); free(tm); free(tp);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Whole grid.                                                               */
/* ------------------------------------------------------------------------ */
int orc_operator(const orc_grid *g, const double *U, double *L, double eps, orc_counters *cnt) {
  long nx = g->nx, ny = g->ndim == 2 ? g->ny : 1, ncell = nx * ny;
  int nv = g->ndim == 2 ? 4 : 3;
  memset(L, 0, sizeof(double) * (size_t)(nv * ncell));
  int rc = 0;
  long t1 = 0, t2 = 0;
  double sx = 0.0, sy = 0.0;   /* max |u| + a over the x / y face values */
  int snan = 0;

  /* x sweep: one line per row; normal momentum is m_x */
#pragma omp parallel for schedule(dynamic, 4) reduction(min : rc) reduction(+ : t1, t2) \
    reduction(max : sx) reduction(| : snan)
  for (long jy = 0; jy < ny; ++jy) {
    double *line = (double *)malloc(sizeof(double) * (size_t)(nv * nx));
    double *Lo = (double *)calloc((size_t)(nv * nx), sizeof(double));
    orc_counters c = {0, 0, 0, 0.0, 0};
    for (int v = 0; v < nv; ++v)
      for (long i = 0; i < nx; ++i) line[v * nx + i] = U[v * ncell + jy * nx + i];
    double sl = 0.0;
    int r = line_operator(g, nv, nx, line, g->bc[0], g->bc[1], g->dx, eps, Lo, &c, &sl);
    if (sl > sx) sx = sl;
    if (sl != sl) snan = 1;
    for (int v = 0; v < nv; ++v)
      for (long i = 0; i < nx; ++i) L[v * ncell + jy * nx + i] += Lo[v * nx + i];
    if (r < rc) rc = r;
    t1 += c.theta1_active; t2 += c.theta2_active;
    free(line); free(Lo);
  }
  if (g->ndim == 2) {
    /* y sweep: one line per column; line variables (rho, m_y, m_x, E) */
#pragma omp parallel for schedule(dynamic, 4) reduction(min : rc) reduction(+ : t1, t2) \
    reduction(max : sy) reduction(| : snan)
    for (long ix = 0; ix < nx; ++ix) {
      double *line = (double *)malloc(sizeof(double) * (size_t)(nv * ny));
      double *Lo = (double *)calloc((size_t)(nv * ny), sizeof(double));
      orc_counters c = {0, 0, 0, 0.0, 0};
      const int map[4] = {0, 2, 1, 3};  /* line var -> grid var */
      for (int v = 0; v < nv; ++v)
        for (long jy = 0; jy < ny; ++jy) line[v * ny + jy] = U[map[v] * ncell + jy * nx + ix];
      double sl = 0.0;
      int r = line_operator(g, nv, ny, line, g->bc[2], g->bc[3], g->dy, eps, Lo, &c, &sl);
      if (sl > sy) sy = sl;
      if (sl != sl) snan = 1;
      for (int v = 0; v < nv; ++v)
        for (long jy = 0; jy < ny; ++jy) L[map[v] * ncell + jy * nx + ix] += Lo[v * ny + jy];
      if (r < rc) rc = r;
      t1 += c.theta1_active; t2 += c.theta2_active;
      free(line); free(Lo);
    }
  }
  if (cnt) {
    cnt->theta1_active += t1;
    cnt->theta2_active += t2;
    /* the rate of the face values: sum over directions, as dt in 2-D */
    double fr = snan ? NAN : sx / g->dx + (g->ndim == 2 ? sy / g->dy : 0.0);
    if (fr > cnt->face_rate || fr != fr) cnt->face_rate = fr;
  }
  return rc;
}

/* The x-sweep part L_x on the listed rows and the y-sweep part L_y on the
 * listed columns (sampled checks of large grids): Lx_rows is [nr][nv][nx],
 * Ly_cols is [nc][nv][ny], both in grid variable order. */
int orc_operator_lines(const orc_grid *g, const double *U, double eps, long nr, const long *rows,
                       long nc, const long *cols, double *Lx_rows, double *Ly_cols) {
  long nx = g->nx, ny = g->ndim == 2 ? g->ny : 1, ncell = nx * ny;
  int nv = g->ndim == 2 ? 4 : 3;
  int rc = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(min : rc)
  for (long q = 0; q < nr + nc; ++q) {
    int is_row = q < nr;
    long idx = is_row ? rows[q] : cols[q - nr];
    long n = is_row ? nx : ny;
    const int mapx[4] = {0, 1, 2, 3}, mapy[4] = {0, 2, 1, 3};
    const int *map = is_row ? mapx : mapy;
    double *line = (double *)malloc(sizeof(double) * (size_t)(nv * n));
    double *Lo = (double *)calloc((size_t)(nv * n), sizeof(double));
    for (int v = 0; v < nv; ++v)
      for (long i = 0; i < n; ++i)
        line[v * n + i] = is_row ? U[map[v] * ncell + idx * nx + i] : U[map[v] * ncell + i * nx + idx];
    int r = is_row ? line_operator(g, nv, n, line, g->bc[0], g->bc[1], g->dx, eps, Lo, 0, 0)
                   : line_operator(g, nv, n, line, g->bc[2], g->bc[3], g->dy, eps, Lo, 0, 0);
    double *out = is_row ? Lx_rows + q * nv * nx : Ly_cols + (q - nr) * nv * ny;
    for (int v = 0; v < nv; ++v)
      for (long i = 0; i < n; ++i) out[map[v] * n + i] = Lo[v * n + i];
    if (r < rc) rc = r;
    free(line); free(Lo);
  }
  return rc;
}

double orc_max_rate(const orc_grid *g, const double *U) {
  long nx = g->nx, ny = g->ndim == 2 ? g->ny : 1, ncell = nx * ny;
  int nv = g->ndim == 2 ? 4 : 3;
  double rate = 0.0;
  for (long c = 0; c < ncell; ++c) {
    double W[4];
    for (int v = 0; v < nv; ++v) W[v] = U[v * ncell + c];
    double p = pressure(nv, g->gamma, W);
    if (!(W[0] > 0.0) || !(p > 0.0)) return -1.0;
    double a = sqrt(g->gamma * p / W[0]);
    double r = (fabs(W[1] / W[0]) + a) / g->dx;
    if (nv == 4) r += (fabs(W[2] / W[0]) + a) / g->dy;
    if (r > rate) rate = r;
  }
  return rate;
}

double orc_min_rho(const orc_grid *g, const double *U) {
  long ncell = g->nx * (g->ndim == 2 ? g->ny : 1);
  double m = U[0];
  for (long c = 1; c < ncell; ++c) m = fmin(m, U[c]);
  return m;
}

static double stage_eps(const orc_grid *g, const double *U) {
  /* Sec. 2.4 step 1: eps = min_j {1e-13, rho_bar_j} */
  return fmin(g->eps_pos, orc_min_rho(g, U));
}

int orc_rk3_step(const orc_grid *g, double *U, double dt, orc_counters *cnt) {
  long ncell = g->nx * (g->ndim == 2 ? g->ny : 1);
  int nv = g->ndim == 2 ? 4 : 3;
  long n = nv * ncell;
  double *U0 = (double *)malloc(sizeof(double) * (size_t)n);
  double *U1 = (double *)malloc(sizeof(double) * (size_t)n);
  double *L = (double *)malloc(sizeof(double) * (size_t)n);
  if (!U0 || !U1 || !L) { free(U0); free(U1); free(L); return -1; }
  memcpy(U0, U, sizeof(double) * (size_t)n);
  int rc = 0;
  /* eq. (RK3), stage 1: U1 = Un + dt L(Un) */
  rc = orc_operator(g, U0, L, stage_eps(g, U0), cnt);
  if (rc == 0) {
    for (long i = 0; i < n; ++i) U1[i] = U0[i] + dt * L[i];
    /* stage 2: U2 = 3/4 Un + 1/4 U1 + 1/4 dt L(U1) */
    rc = orc_operator(g, U1, L, stage_eps(g, U1), cnt);
  }
  if (rc == 0) {
    for (long i = 0; i < n; ++i) U1[i] = 0.75 * U0[i] + 0.25 * U1[i] + 0.25 * dt * L[i];
    /* stage 3: U^{n+1} = 1/3 Un + 2/3 U2 + 2/3 dt L(U2) */
    rc = orc_operator(g, U1, L, stage_eps(g, U1), cnt);
  }
  if (rc == 0) {
    for (long i = 0; i < n; ++i) U[i] = U0[i] / 3.0 + 2.0 / 3.0 * U1[i] + 2.0 / 3.0 * dt * L[i];
  }
  free(U0); free(U1); free(L);
  return rc;
}

int orc_advance(const orc_grid *g, double *U, double cfl, double t0, double t_final,
                long max_steps, double *t_out, long *steps_out, double *dt_last,
                orc_counters *cnt) {
  long ncell = g->nx * (g->ndim == 2 ? g->ny : 1);
  long nval = (g->ndim == 2 ? 4 : 3) * ncell;
  double *Un = g->face_cfl > 0.0 ? (double *)malloc(sizeof(double) * (size_t)nval) : NULL;
  if (g->face_cfl > 0.0 && !Un) return -1;
  double t = t0;
  long steps = 0;
  int rc = 0;
  double dt = 0.0;
  double frate_prev = 0.0;   /* face rate of the last accepted step */
  if (g->face_cfl > 0.0) cfl = fmin(cfl, g->face_cfl);
  while (t < t_final) {
    if (steps >= max_steps) { rc = -2; break; }
    double rate = orc_max_rate(g, U);
    if (!(rate > 0.0)) { rc = -1; break; }
    /* eq. (CFL-CD) on the states the scheme's first-order steps use: with
     * the check on, the rate also covers the limited face values of the
     * last accepted step, and a step whose own face values exceed the bound
     * is redone from U^n with the time step their rate allows */
    double r_dt = g->face_cfl > 0.0 ? fmax(rate, frate_prev) : rate;
    int last = 0, tries = 0;
    if (Un) memcpy(Un, U, sizeof(double) * (size_t)nval);
    for (;;) {
      dt = cfl / r_dt;
      double rem = t_final - t;
      last = 0;
      if (dt >= rem) { dt = rem; last = 1; }
      orc_counters c = {0, 0, 0, 0.0, 0};
      if (orc_rk3_step(g, U, dt, &c) != 0) { rc = -1; break; }
      if (cnt) { cnt->theta1_active += c.theta1_active; cnt->theta2_active += c.theta2_active; }
      if (!(g->face_cfl > 0.0) || dt * c.face_rate <= g->face_cfl) {
        frate_prev = c.face_rate;
        if (cnt && (c.face_rate > cnt->face_rate || c.face_rate != c.face_rate)) cnt->face_rate = c.face_rate;
        break;
      }
      /* rejected: back to U^n; the observed rate exceeds face_cfl / dt >=
       * cfl / dt, so the next dt is strictly smaller */
      memcpy(U, Un, sizeof(double) * (size_t)nval);
      if (cnt) cnt->rejected++;
      if (++tries > 60) { rc = -1; break; }
      /* a stage that left G has no finite face rate: halve dt instead */
      r_dt = c.face_rate < INFINITY ? c.face_rate : 2.0 * cfl / dt;
    }
    if (rc) break;
    ++steps;
    t = last ? t_final : t + dt;
  }
  free(Un);
  if (t_out) *t_out = t;
  if (steps_out) *steps_out = steps;
  if (dt_last) *dt_last = dt;
  return rc;
}
