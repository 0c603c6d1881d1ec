/*
 * riemann_exact.c -- exact solution of the Riemann problem of the 1-D Euler
 * equations for an ideal gas (the classical construction: star pressure from
 * the sum of the two wave functions, Newton iteration with a bisection
 * cross-check, self-similar sampling, vacuum generation when the velocity
 * jump exceeds 2 (a_L + a_R) / (gamma - 1)).
 *
 * TEST INFRASTRUCTURE ONLY: a reference for the tests of the oracle and of
 * the GPU path on Riemann data (the paper compares with exact solutions in
 * its Sec. 3 examples); it is not a step of the scheme.
 * Primitive states are W = (rho, u, p).
 */
#include "pp_oracle.h"

#include <math.h>

static double sound(double gamma, const double *W) { return sqrt(gamma * W[2] / W[0]); }

/* wave function f_K(p) and its derivative for the side with state W */
static void wave_fn(double gamma, const double *W, double p, double *f, double *df) {
  double rho = W[0], pk = W[2], a = sound(gamma, W);
  if (p > pk) {
    /* shock: Rankine-Hugoniot */
    double A = 2.0 / ((gamma + 1.0) * rho);
    double B = (gamma - 1.0) / (gamma + 1.0) * pk;
    double q = sqrt(A / (p + B));
    *f = (p - pk) * q;
    *df = q * (1.0 - 0.5 * (p - pk) / (B + p));
  } else {
    /* rarefaction: isentropic, Riemann invariant */
    double e = (gamma - 1.0) / (2.0 * gamma);
    *f = 2.0 * a / (gamma - 1.0) * (pow(p / pk, e) - 1.0);
    *df = 1.0 / (rho * a) * pow(p / pk, -(gamma + 1.0) / (2.0 * gamma));
  }
}

static double total_fn(double gamma, const double *WL, const double *WR, double p, double *df) {
  double fl, dl, fr, dr;
  wave_fn(gamma, WL, p, &fl, &dl);
  wave_fn(gamma, WR, p, &fr, &dr);
  if (df) *df = dl + dr;
  return fl + fr + (WR[1] - WL[1]);
}

double orc_riemann_star_bisect(double gamma, const double *WL, const double *WR) {
  double lo = 0.0, hi = fmax(WL[2], WR[2]);
  while (total_fn(gamma, WL, WR, hi, 0) < 0.0) hi *= 2.0;
  if (total_fn(gamma, WL, WR, 0.0, 0) >= 0.0) return 0.0;   /* vacuum */
  for (int it = 0; it < 400; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (total_fn(gamma, WL, WR, mid, 0) < 0.0) lo = mid; else hi = mid;
  }
  return 0.5 * (lo + hi);
}

int orc_riemann_star(double gamma, const double *WL, const double *WR,
                     double *pstar, double *ustar, int *vacuum, int *iters) {
  double aL = sound(gamma, WL), aR = sound(gamma, WR);
  *iters = 0;
  if (2.0 * (aL + aR) / (gamma - 1.0) <= WR[1] - WL[1]) {
    *vacuum = 1;
    *pstar = 0.0;
    *ustar = 0.5 * (WL[1] + 2.0 * aL / (gamma - 1.0) + WR[1] - 2.0 * aR / (gamma - 1.0));
    return 0;
  }
  *vacuum = 0;
  /* starting value: two-rarefaction approximation (exact if both waves are
   * rarefactions) */
  double e = (gamma - 1.0) / (2.0 * gamma);
  double num = aL + aR - 0.5 * (gamma - 1.0) * (WR[1] - WL[1]);
  double den = aL / pow(WL[2], e) + aR / pow(WR[2], e);
  double p = pow(num / den, 1.0 / e);
  if (!(p > 0.0)) p = 1e-8 * fmin(WL[2], WR[2]);
  int ok = 0;
  for (int it = 1; it <= 100; ++it) {
    double df, f = total_fn(gamma, WL, WR, p, &df);
    double pn = p - f / df;
    if (pn <= 0.0) pn = 0.5 * p;
    *iters = it;
    if (fabs(pn - p) <= 1e-15 * 0.5 * (pn + p)) { p = pn; ok = 1; break; }
    p = pn;
  }
  if (!ok) p = orc_riemann_star_bisect(gamma, WL, WR);
  double fl, fr, d;
  wave_fn(gamma, WL, p, &fl, &d);
  wave_fn(gamma, WR, p, &fr, &d);
  *pstar = p;
  *ustar = 0.5 * (WL[1] + WR[1]) + 0.5 * (fr - fl);
  return ok ? 0 : 1;
}

/* left-going fan state at xi, from the left state */
static void fan_left(double gamma, const double *W, double xi, double *out) {
  double a = sound(gamma, W), g1 = gamma - 1.0, gp = gamma + 1.0;
  double c = 2.0 / gp * (a + 0.5 * g1 * (W[1] - xi));
  out[1] = 2.0 / gp * (a + 0.5 * g1 * W[1] + xi);
  out[0] = W[0] * pow(c / a, 2.0 / g1);
  out[2] = W[2] * pow(c / a, 2.0 * gamma / g1);
}

static void fan_right(double gamma, const double *W, double xi, double *out) {
  double a = sound(gamma, W), g1 = gamma - 1.0, gp = gamma + 1.0;
  double c = 2.0 / gp * (a - 0.5 * g1 * (W[1] - xi));
  out[1] = 2.0 / gp * (-a + 0.5 * g1 * W[1] + xi);
  out[0] = W[0] * pow(c / a, 2.0 / g1);
  out[2] = W[2] * pow(c / a, 2.0 * gamma / g1);
}

static void copy3(const double *a, double *b) { b[0] = a[0]; b[1] = a[1]; b[2] = a[2]; }

void orc_riemann_sample(double gamma, const double *WL, const double *WR, double xi, double *W) {
  double ps, us;
  int vac, it;
  orc_riemann_star(gamma, WL, WR, &ps, &us, &vac, &it);
  double aL = sound(gamma, WL), aR = sound(gamma, WR), g1 = gamma - 1.0, gp = gamma + 1.0;
  if (vac) {
    double sL = WL[1] + 2.0 * aL / g1, sR = WR[1] - 2.0 * aR / g1;
    if (xi <= WL[1] - aL) copy3(WL, W);
    else if (xi < sL) fan_left(gamma, WL, xi, W);
    else if (xi <= sR) { W[0] = 0.0; W[1] = xi; W[2] = 0.0; }
    else if (xi < WR[1] + aR) fan_right(gamma, WR, xi, W);
    else copy3(WR, W);
    return;
  }
  if (xi <= us) {
    double pr = ps / WL[2];
    if (ps > WL[2]) {
      double S = WL[1] - aL * sqrt(gp / (2.0 * gamma) * pr + g1 / (2.0 * gamma));
      if (xi <= S) copy3(WL, W);
      else { W[0] = WL[0] * (pr + g1 / gp) / (g1 / gp * pr + 1.0); W[1] = us; W[2] = ps; }
    } else {
      double sh = WL[1] - aL, as = aL * pow(pr, g1 / (2.0 * gamma)), st = us - as;
      if (xi <= sh) copy3(WL, W);
      else if (xi > st) { W[0] = WL[0] * pow(pr, 1.0 / gamma); W[1] = us; W[2] = ps; }
      else fan_left(gamma, WL, xi, W);
    }
  } else {
    double pr = ps / WR[2];
    if (ps > WR[2]) {
      double S = WR[1] + aR * sqrt(gp / (2.0 * gamma) * pr + g1 / (2.0 * gamma));
      if (xi >= S) copy3(WR, W);
      else { W[0] = WR[0] * (pr + g1 / gp) / (g1 / gp * pr + 1.0); W[1] = us; W[2] = ps; }
    } else {
      double sh = WR[1] + aR, as = aR * pow(pr, g1 / (2.0 * gamma)), st = us + as;
      if (xi >= sh) copy3(WR, W);
      else if (xi < st) { W[0] = WR[0] * pow(pr, 1.0 / gamma); W[1] = us; W[2] = ps; }
      else fan_right(gamma, WR, xi, W);
    }
  }
}

void orc_riemann_cell_averages(double gamma, const double *WL, const double *WR,
                               double x0, double x1, long n, double xd, double t,
                               int nsub, double *U) {
  /* 5-point Gauss-Legendre nodes and weights on [-1, 1] */
  static const double gx[5] = {-0.9061798459386640, -0.5384693101056831, 0.0,
                               0.5384693101056831, 0.9061798459386640};
  static const double gw[5] = {0.2369268850561891, 0.4786286704993665, 0.5688888888888889,
                               0.4786286704993665, 0.2369268850561891};
  double h = (x1 - x0) / (double)n;
  if (nsub < 1) nsub = 1;
  for (long j = 0; j < n; ++j) {
    double acc[3] = {0.0, 0.0, 0.0};
    double hs = h / nsub;
    for (int s = 0; s < nsub; ++s) {
      double a = x0 + j * h + s * hs, c = a + 0.5 * hs;
      for (int q = 0; q < 5; ++q) {
        double x = c + 0.5 * hs * gx[q], W[3];
        if (t > 0.0) orc_riemann_sample(gamma, WL, WR, (x - xd) / t, W);
        else copy3(x < xd ? WL : WR, W);
        double wq = 0.5 * gw[q] / nsub;
        acc[0] += wq * W[0];
        acc[1] += wq * W[0] * W[1];
        acc[2] += wq * (W[2] / (gamma - 1.0) + 0.5 * W[0] * W[1] * W[1]);
      }
    }
    U[0 * n + j] = acc[0];
    U[1 * n + j] = acc[1];
    U[2 * n + j] = acc[2];
  }
}
