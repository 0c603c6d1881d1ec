// char_recon.cu -- kernel of the characteristic-wise reconstruction
// (Sec. 2.3); the layout and the walk are described in char_recon.cuh.
#include "char_recon.cuh"
#include "physics.cuh"

namespace ppk {
namespace {

// Sec. 2.3: rows l^(k) of L, the left eigenvectors of the flux Jacobian at
// the Roe average of Ua and Ub (eqs. (eigen), (leigenv)), ordered by the
// eigenvalues u - a, u, (u,) u + a; in 2-D the third row is the shear field
// (-v, 0, 1, 0) and v enters the acoustic rows through |u|^2 and -c1 v / 2.
template <int NV>
__device__ __forceinline__ void roe_left(const double *Ua, const double *Ub, double gamma,
                                         double (&L)[NV][NV]) {
  const double sa = sqrt(Ua[0]), sb = sqrt(Ub[0]);
  const double isab = 1.0 / (sa + sb);
  const double pa = pressure<double, NV>(Ua, gamma), pb = pressure<double, NV>(Ub, gamma);
  const double u = (Ua[1] / sa + Ub[1] / sb) * isab;
  const double v = NV == 4 ? (Ua[2] / sa + Ub[2] / sb) * isab : 0.0;
  const double H = ((Ua[NV - 1] + pa) / sa + (Ub[NV - 1] + pb) / sb) * isab;
  const double q2 = u * u + v * v;
  const double a2 = (gamma - 1.0) * (H - 0.5 * q2);
  const double ia = 1.0 / sqrt(a2);
  const double c1 = (gamma - 1.0) / a2, c2 = 0.5 * q2 * c1;
  L[0][0] = 0.5 * (c2 + u * ia);
  L[0][1] = -0.5 * (c1 * u + ia);
  L[0][NV - 1] = 0.5 * c1;
  L[1][0] = 1.0 - c2;
  L[1][1] = c1 * u;
  L[1][NV - 1] = -c1;
  L[NV - 1][0] = 0.5 * (c2 - u * ia);
  L[NV - 1][1] = 0.5 * (ia - c1 * u);
  L[NV - 1][NV - 1] = 0.5 * c1;
  if constexpr (NV == 4) {
    L[0][2] = -0.5 * c1 * v;
    L[1][2] = c1 * v;
    L[3][2] = -0.5 * c1 * v;
    L[2][0] = -v;
    L[2][1] = 0.0;
    L[2][2] = 1.0;
    L[2][3] = 0.0;
  }
}

// X <- M^{-1} X for an NV x NV block M and NCOL columns: Gaussian
// elimination with partial pivoting, all indices fixed at compile time
template <int NV, int NCOL>
__device__ __forceinline__ void gauss_solve(double (&M)[NV][NV], double (&X)[NV][NCOL]) {
#pragma unroll
  for (int c = 0; c < NV; ++c) {
    double best = fabs(M[c][c]);
    int piv = c;
#pragma unroll
    for (int r = c + 1; r < NV; ++r) {
      const double m = fabs(M[r][c]);
      if (m > best) { best = m; piv = r; }
    }
#pragma unroll
    for (int r = c + 1; r < NV; ++r) {
      const bool sw = piv == r;
#pragma unroll
      for (int j = c; j < NV; ++j) {
        const double t = M[c][j];
        M[c][j] = sw ? M[r][j] : t;
        M[r][j] = sw ? t : M[r][j];
      }
#pragma unroll
      for (int j = 0; j < NCOL; ++j) {
        const double t = X[c][j];
        X[c][j] = sw ? X[r][j] : t;
        X[r][j] = sw ? t : X[r][j];
      }
    }
    const double inv = 1.0 / M[c][c];
#pragma unroll
    for (int r = c + 1; r < NV; ++r) {
      const double f = M[r][c] * inv;
#pragma unroll
      for (int j = c + 1; j < NV; ++j) M[r][j] -= f * M[c][j];
#pragma unroll
      for (int j = 0; j < NCOL; ++j) X[r][j] -= f * X[c][j];
    }
  }
#pragma unroll
  for (int c = NV - 1; c >= 0; --c) {
    const double inv = 1.0 / M[c][c];
#pragma unroll
    for (int j = 0; j < NCOL; ++j) {
      double s = X[c][j];
#pragma unroll
      for (int q = c + 1; q < NV; ++q) s -= M[c][q] * X[q][j];
      X[c][j] = s * inv;
    }
  }
}

// One thread per (line, side).  Position p of the walk is cell p (minus
// side, left to right) or cell n-1-p (plus side, right to left); in walk
// order both sides have the same rows (the plus row is the mirror image of
// the minus row), so "previous" and "next" below are in walk order.
// Periodic lines solve the cyclic system with the Woodbury correction
// T = T' + U V^T, G = -B_0: T' has B_0 - G at the first position and
// B_{n-1} - C_{n-1} G^{-1} A_0 at the last, U = (G, 0, .., 0, C_{n-1}),
// V^T = (I, 0, .., 0, G^{-1} A_0); the NV columns of U ride along as extra
// right-hand sides and x = y - Z (I + V^T Z)^{-1} V^T y at the end.
template <int NV, bool PER>
__global__ void __launch_bounds__(32) char_recon_kernel(const CharArgs a) {
  constexpr int NC = PER ? NV + 1 : 1;       // right-hand-side columns
  constexpr int ROW = NV * NV + NV * NC;     // scratch doubles per row: Y, g
  const long long line = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (line >= a.nlines) return;
  const int side = blockIdx.y;
  const int n = a.n;
  const int dir = side == 0 ? 1 : -1;
  const long long NL = a.nlines;
  const long long lbase = line * a.line_stride;
  double *scr = a.scr + (long long)side * ((long long)n * ROW + NV * NV) * NL + line;
  auto slot = [&](int p, int e) -> double & { return scr[((long long)p * ROW + e) * NL]; };
  auto wslot = [&](int e) -> double & { return scr[((long long)n * ROW + e) * NL]; };
  int gv[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) gv[k] = k == 0 ? 0 : (k == NV - 1 ? NV - 1 : (k == 1 ? a.vn : a.vt));

  // line variables of line cell i (ghost cells by the boundary condition)
  auto cell = [&](int i, double(&out)[NV]) {
    bool neg = false;
    if (i < 0 || i >= n) {
      if (PER) {
        i = (i % n + n) % n;
      } else {
        const int bc = i < 0 ? a.bclo : a.bchi;
        if (bc == 1) {
          i = i < 0 ? 0 : n - 1;
        } else {
          i = i < 0 ? -i - 1 : 2 * n - 1 - i;
          neg = true;
        }
      }
    }
    const double *src = a.U + lbase + (long long)i * a.cell_stride;
#pragma unroll
    for (int k = 0; k < NV; ++k) out[k] = src[gv[k] * a.ncell];
    if (neg) out[1] = -out[1];
  };
  auto cidx = [&](int p) { return side == 0 ? p : n - 1 - p; };

  double win[5][NV];   // walk offsets -2 .. +2 of the current position
#pragma unroll
  for (int q = 0; q < 4; ++q) cell(cidx(0) + (q - 2) * dir, win[q + 1]);

  double Yp[NV][NV], gp[NV][NC];   // the previous position's multipliers
#pragma unroll 1
  for (int p = 0; p < n; ++p) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int k = 0; k < NV; ++k) win[q][k] = win[q + 1][k];
    cell(cidx(p) + 2 * dir, win[4]);

    // step 1: eigenvectors at the unknown's face (this cell and the next)
    double L[NV][NV];
    roe_left<NV>(win[2], win[3], a.gamma, L);
    // characteristic variables of the five cells
    double cv[NV][5];
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        double t = 0.0;
#pragma unroll
        for (int m = 0; m < NV; ++m) t += L[k][m] * win[q][m];
        cv[k][q] = t;
      }
    // steps 2-3: per-field weights and scalar row (a on the previous
    // unknown, b on this one, c on the next); closure rows 0 x + 1 x + 0 x
    const bool closure = !PER && (p == 0 || p == n - 1);
    double ca[NV], cb[NV], cc[NV], cr[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      if (closure) {
        ca[k] = 0.0;
        cb[k] = 1.0;
        cc[k] = 0.0;
        cr[k] = weno5z_face<double>(cv[k][0], cv[k][1], cv[k][2], cv[k][3], cv[k][4], a.eps_weno);
      } else {
        double q0, q1, q2, w0, w1, w2;
        zratios<double>(cv[k][0], cv[k][1], cv[k][2], cv[k][3], cv[k][4], a.eps_weno, q0, q1, q2);
        zweights<double>(0.2, 0.5, 0.3, q0, q1, q2, w0, w1, w2);
        const Row<double> r = compact_row<double>(w0, w1, w2, cv[k][1], cv[k][2], cv[k][3]);
        ca[k] = r.a;
        cb[k] = r.b;
        cc[k] = r.c;
        cr[k] = r.r;
      }
    }
    // step 4: block row diag(ca, cb, cc) L, eliminated against the previous
    // position: Bp = B - A Y_prev, X = [C | r - A g_prev]
    double Bp[NV][NV], X[NV][NV + NC];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
#pragma unroll
      for (int j = 0; j < NV; ++j) {
        Bp[k][j] = cb[k] * L[k][j];
        X[k][j] = cc[k] * L[k][j];
      }
      X[k][NV] = cr[k];
#pragma unroll
      for (int j = 1; j < NC; ++j) X[k][NV + j] = 0.0;
    }
    if constexpr (PER) {
      if (p == 0) {
        // G = -B_0: B'_0 = B_0 - G = 2 B_0, Woodbury columns U_0 = G, and
        // G^{-1} A_0 for the last position and the final correction
        double Gm[NV][NV], GiA[NV][NV];
#pragma unroll
        for (int k = 0; k < NV; ++k)
#pragma unroll
          for (int j = 0; j < NV; ++j) {
            Gm[k][j] = -Bp[k][j];
            GiA[k][j] = ca[k] * L[k][j];
            X[k][NV + 1 + j] = Gm[k][j];
            Bp[k][j] = Bp[k][j] + Bp[k][j];
          }
        gauss_solve<NV, NV>(Gm, GiA);
#pragma unroll
        for (int k = 0; k < NV; ++k)
#pragma unroll
          for (int j = 0; j < NV; ++j) wslot(k * NV + j) = GiA[k][j];
      }
    }
    if (p > 0) {
#pragma unroll
      for (int k = 0; k < NV; ++k) {
#pragma unroll
        for (int j = 0; j < NV; ++j) {
          double t = 0.0;
#pragma unroll
          for (int m = 0; m < NV; ++m) t += L[k][m] * Yp[m][j];
          Bp[k][j] -= ca[k] * t;
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          double t = 0.0;
#pragma unroll
          for (int m = 0; m < NV; ++m) t += L[k][m] * gp[m][c];
          X[k][NV + c] -= ca[k] * t;
        }
      }
    }
    if constexpr (PER) {
      if (p == n - 1) {
        // B'_{n-1} = B_{n-1} - C_{n-1} G^{-1} A_0; the coupling to x_0 moves
        // into the Woodbury columns (U_{n-1} = C_{n-1})
        double GiA[NV][NV];
#pragma unroll
        for (int k = 0; k < NV; ++k)
#pragma unroll
          for (int j = 0; j < NV; ++j) GiA[k][j] = wslot(k * NV + j);
#pragma unroll
        for (int k = 0; k < NV; ++k)
#pragma unroll
          for (int j = 0; j < NV; ++j) {
            double t = 0.0;
#pragma unroll
            for (int m = 0; m < NV; ++m) t += X[k][m] * GiA[m][j];
            Bp[k][j] -= t;
          }
#pragma unroll
        for (int k = 0; k < NV; ++k)
#pragma unroll
          for (int j = 0; j < NV; ++j) {
            X[k][NV + 1 + j] += X[k][j];
            X[k][j] = 0.0;
          }
      }
    }
    gauss_solve<NV, NV + NC>(Bp, X);
#pragma unroll
    for (int k = 0; k < NV; ++k) {
#pragma unroll
      for (int j = 0; j < NV; ++j) {
        Yp[k][j] = X[k][j];
        slot(p, k * NV + j) = X[k][j];
      }
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        gp[k][c] = X[k][NV + c];
        slot(p, NV * NV + k * NC + c) = X[k][NV + c];
      }
    }
  }

  // back substitution x_p = g_p - Y_p x_{p+1}
  double *out = side == 0 ? a.Um : a.Up;
  double x[NV][NC];
#pragma unroll
  for (int k = 0; k < NV; ++k)
#pragma unroll
    for (int c = 0; c < NC; ++c) x[k][c] = gp[k][c];
#pragma unroll 1
  for (int p = n - 1; p >= 0; --p) {
    if (p < n - 1) {
      double Y[NV][NV], xn[NV][NC];
#pragma unroll
      for (int k = 0; k < NV; ++k) {
#pragma unroll
        for (int j = 0; j < NV; ++j) Y[k][j] = slot(p, k * NV + j);
#pragma unroll
        for (int c = 0; c < NC; ++c) xn[k][c] = x[k][c];
      }
#pragma unroll
      for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          double s = slot(p, NV * NV + k * NC + c);
#pragma unroll
          for (int j = 0; j < NV; ++j) s -= Y[k][j] * xn[j][c];
          x[k][c] = s;
        }
    }
    if (PER) {
#pragma unroll
      for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int c = 0; c < NC; ++c) slot(p, NV * NV + k * NC + c) = x[k][c];
    } else {
      double *dst = out + lbase + (long long)cidx(p) * a.cell_stride;
#pragma unroll
      for (int k = 0; k < NV; ++k) dst[gv[k] * a.ncell] = x[k][0];
    }
  }
  if constexpr (PER) {
    // S = I + Z_0 + G^{-1} A_0 Z_{n-1}, t = y_0 + G^{-1} A_0 y_{n-1};
    // x_p = y_p - Z_p S^{-1} t
    double S[NV][NV], t[NV][1], GiA[NV][NV];
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
      for (int j = 0; j < NV; ++j) GiA[k][j] = wslot(k * NV + j);
#pragma unroll
    for (int k = 0; k < NV; ++k) {
#pragma unroll
      for (int j = 0; j < NV; ++j) {
        double s = (k == j ? 1.0 : 0.0) + slot(0, NV * NV + k * NC + 1 + j);
#pragma unroll
        for (int m = 0; m < NV; ++m) s += GiA[k][m] * slot(n - 1, NV * NV + m * NC + 1 + j);
        S[k][j] = s;
      }
      double s = slot(0, NV * NV + k * NC);
#pragma unroll
      for (int m = 0; m < NV; ++m) s += GiA[k][m] * slot(n - 1, NV * NV + m * NC);
      t[k][0] = s;
    }
    gauss_solve<NV, 1>(S, t);
#pragma unroll 1
    for (int p = 0; p < n; ++p) {
      double *dst = out + lbase + (long long)cidx(p) * a.cell_stride;
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        double s = slot(p, NV * NV + k * NC);
#pragma unroll
        for (int j = 0; j < NV; ++j) s -= slot(p, NV * NV + k * NC + 1 + j) * t[j][0];
        dst[gv[k] * a.ncell] = s;
      }
    }
  }
}

}  // namespace

cudaError_t launch_char_recon(const CharArgs &a, int nv, bool periodic, cudaStream_t st) {
  const dim3 grid((unsigned)((a.nlines + 31) / 32), 2, 1);
  if (nv == 3) {
    if (periodic) char_recon_kernel<3, true><<<grid, 32, 0, st>>>(a);
    else char_recon_kernel<3, false><<<grid, 32, 0, st>>>(a);
  } else {
    if (periodic) char_recon_kernel<4, true><<<grid, 32, 0, st>>>(a);
    else char_recon_kernel<4, false><<<grid, 32, 0, st>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace ppk
