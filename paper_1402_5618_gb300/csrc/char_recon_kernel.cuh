// char_recon_kernel.cuh -- kernel of the characteristic-wise reconstruction
// (Sec. 2.3) in the arithmetic of the line: real = double is the plain
// form; real = float the mixed form, reading the FP32 hi parts of the state.
// The layout and the walk are described in char_recon.cuh.
#pragma once

#include "char_recon.cuh"
#include "physics.cuh"

namespace ppk {
namespace chr {

// Sec. 2.3: the Roe average of Ua and Ub, reduced to the four scalars the
// left eigenvectors depend on: u, v (2-D), 1/a and c1 = (gamma - 1)/a^2
template <typename real, int NV>
__device__ __forceinline__ void roe_scalars(const real *Ua, const real *Ub, real gamma,
                                            real (&rs)[4]) {
  const real one = real(1), half = real(0.5);
  const real sa = sqrt(Ua[0]), sb = sqrt(Ub[0]);
  const real isab = one / (sa + sb);
  const real pa = pressure<real, NV>(Ua, gamma), pb = pressure<real, NV>(Ub, gamma);
  const real u = (Ua[1] / sa + Ub[1] / sb) * isab;
  const real v = NV == 4 ? (Ua[2] / sa + Ub[2] / sb) * isab : real(0);
  const real H = ((Ua[NV - 1] + pa) / sa + (Ub[NV - 1] + pb) / sb) * isab;
  const real a2 = (gamma - one) * (H - half * (u * u + v * v));
  rs[0] = u;
  rs[1] = v;
  rs[2] = one / sqrt(a2);
  rs[3] = (gamma - one) / a2;
}

// rows l^(k) of L (eqs. (eigen), (leigenv)), ordered by the eigenvalues
// u - a, u, (u,) u + a; in 2-D the third row is the shear field
// (-v, 0, 1, 0) and v enters the acoustic rows through |u|^2 and -c1 v / 2
template <typename real, int NV>
__device__ __forceinline__ void left_from(const real (&rs)[4], real (&L)[NV][NV]) {
  const real one = real(1), half = real(0.5);
  const real u = rs[0], v = rs[1], ia = rs[2], c1 = rs[3];
  const real c2 = half * (u * u + v * v) * c1;
  L[0][0] = half * (c2 + u * ia);
  L[0][1] = -half * (c1 * u + ia);
  L[0][NV - 1] = half * c1;
  L[1][0] = one - c2;
  L[1][1] = c1 * u;
  L[1][NV - 1] = -c1;
  L[NV - 1][0] = half * (c2 - u * ia);
  L[NV - 1][1] = half * (ia - c1 * u);
  L[NV - 1][NV - 1] = half * c1;
  if constexpr (NV == 4) {
    L[0][2] = -half * c1 * v;
    L[1][2] = c1 * v;
    L[3][2] = -half * c1 * v;
    L[2][0] = -v;
    L[2][1] = real(0);
    L[2][2] = one;
    L[2][3] = real(0);
  }
}

// X <- M^{-1} X for an NV x NV block M and NCOL columns: Gaussian
// elimination with partial pivoting, all indices fixed at compile time; the
// pivots' reciprocals serve both passes (row c is final once column c is done)
template <typename real, int NV, int NCOL>
__device__ __forceinline__ void gauss_solve(real (&M)[NV][NV], real (&X)[NV][NCOL]) {
  real inv[NV];
#pragma unroll
  for (int c = 0; c < NV; ++c) {
    real best = fabs(M[c][c]);
    int piv = c;
#pragma unroll
    for (int r = c + 1; r < NV; ++r) {
      const real m = fabs(M[r][c]);
      if (m > best) { best = m; piv = r; }
    }
#pragma unroll
    for (int r = c + 1; r < NV; ++r) {
      const bool sw = piv == r;
#pragma unroll
      for (int j = c; j < NV; ++j) {
        const real t = M[c][j];
        M[c][j] = sw ? M[r][j] : t;
        M[r][j] = sw ? t : M[r][j];
      }
#pragma unroll
      for (int j = 0; j < NCOL; ++j) {
        const real t = X[c][j];
        X[c][j] = sw ? X[r][j] : t;
        X[r][j] = sw ? t : X[r][j];
      }
    }
    inv[c] = real(1) / M[c][c];
#pragma unroll
    for (int r = c + 1; r < NV; ++r) {
      const real f = M[r][c] * inv[c];
#pragma unroll
      for (int j = c + 1; j < NV; ++j) M[r][j] -= f * M[c][j];
#pragma unroll
      for (int j = 0; j < NCOL; ++j) X[r][j] -= f * X[c][j];
    }
  }
#pragma unroll
  for (int c = NV - 1; c >= 0; --c) {
#pragma unroll
    for (int j = 0; j < NCOL; ++j) {
      real s = X[c][j];
#pragma unroll
      for (int q = c + 1; q < NV; ++q) s -= M[c][q] * X[q][j];
      X[c][j] = s * inv[c];
    }
  }
}

// WENO-Z ratios of one characteristic field over its five-cell stencil v.
// FP32: the scaled ratios with eps lifted to the rounding floor of the
// indicators, FP32_BETA_FLOOR s^2 = 2^20 (u s)^2 with s = mag, the largest sum_m |l_m| |ubar_m|
// over the stencil: the size of the terms the characteristic variable is
// summed from, which bounds its rounding error even where the sum cancels
// (the same floor as the component-wise mixed form, taken on those terms).
template <typename real>
__device__ __forceinline__ void char_ratios(const real (&v)[5], real mag, real eps, real &q0,
                                            real &q1, real &q2, real &one) {
  if constexpr (sizeof(real) == 4) {
    const float c13 = 13.0f / 12.0f;
    const float b0 = c13 * sqr(v[0] - 2.0f * v[1] + v[2]) + 0.25f * sqr(v[0] - 4.0f * v[1] + 3.0f * v[2]);
    const float b1 = c13 * sqr(v[1] - 2.0f * v[2] + v[3]) + 0.25f * sqr(v[1] - v[3]);
    const float b2 = c13 * sqr(v[2] - 2.0f * v[3] + v[4]) + 0.25f * sqr(3.0f * v[2] - 4.0f * v[3] + v[4]);
    const float tau = fabsf(b2 - b0);
    const float e = fmaf(FP32_BETA_FLOOR * mag, mag, eps);
    const float d0 = b0 + e, d1 = b1 + e, d2 = b2 + e;
    const float dmin = fminf(fminf(d0, d1), d2);
    const float r = fminf(tau, dmin);
    const float sc = dmin / tau;
    one = tau <= dmin ? 1.0f : sc * sc;
    q0 = sqr(r / d0);
    q1 = sqr(r / d1);
    q2 = sqr(r / d2);
  } else {
    zratios<real>(v[0], v[1], v[2], v[3], v[4], eps, q0, q1, q2);
    one = real(1);
  }
}

// asynchronous copies global -> shared (cp.async): a per-thread ring in
// shared memory keeps several positions' loads of the serial walk in flight
template <int B>
__device__ __forceinline__ void cp_async(void *sdst, const void *gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  if constexpr (B == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gsrc) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// geometry of one line: its first cell's offset in the planes, cell stride,
// plane size, length and boundary kinds (a batched line from its problem)
struct LineGeo {
  long long base, cs, ncell;
  int n, bclo, bchi;
};

__device__ __forceinline__ LineGeo line_geo(const CharArgs &a, long long line) {
  LineGeo g;
  if (!a.lines) {
    g.base = line * a.line_stride;
    g.cs = a.cell_stride;
    g.ncell = a.ncell;
    g.n = a.n;
    g.bclo = a.bclo;
    g.bchi = a.bchi;
    return g;
  }
  const LineRef lr = a.lines[line];
  const ProbDesc pd = a.probs[lr.prob];
  g.ncell = pd.ncell;
  if (a.xdir == 1) {
    g.n = pd.nx; g.cs = 1; g.base = pd.off + (long long)lr.line * pd.nx;
    g.bclo = pd.bc[0]; g.bchi = pd.bc[1];
  } else if (a.xdir == 2) {   // a row of the problem's transposed planes: a y line
    g.n = pd.ny; g.cs = 1; g.base = pd.off + (long long)lr.line * pd.ny;
    g.bclo = pd.bc[2]; g.bchi = pd.bc[3];
  } else {
    g.n = pd.ny; g.cs = pd.nx; g.base = pd.off + lr.line;
    g.bclo = pd.bc[2]; g.bchi = pd.bc[3];
  }
  return g;
}

// ghost-aware read of the line variables of line cell i (both kernels)
template <typename real, int NV, bool PER>
__device__ __forceinline__ void line_cell(const LineGeo &g, const real *U, const int (&gv)[NV],
                                          int i, real (&out)[NV]) {
  const int n = g.n;
  bool neg = false;
  if (i < 0 || i >= n) {
    if (PER) {
      i = (i % n + n) % n;
    } else {
      const int bc = i < 0 ? g.bclo : g.bchi;
      if (bc == 1) {
        i = i < 0 ? 0 : n - 1;
      } else {
        i = i < 0 ? -i - 1 : 2 * n - 1 - i;
        neg = true;
      }
    }
  }
  const real *src = U + g.base + (long long)i * g.cs;
#pragma unroll
  for (int k = 0; k < NV; ++k) out[k] = src[gv[k] * g.ncell];
  if (neg) out[1] = -out[1];
}

template <int NV>
__device__ __forceinline__ void grid_vars(const CharArgs &a, int (&gv)[NV]) {
#pragma unroll
  for (int k = 0; k < NV; ++k) gv[k] = k == 0 ? 0 : (k == NV - 1 ? NV - 1 : (k == 1 ? a.vn : a.vt));
}

// Steps 1-3 at every face, all in parallel.  One block takes a tile of 32
// lines x 32 cells (plus the two-cell halo) into shared memory -- loaded
// along whichever of the two axes is contiguous in memory -- and computes
// the rows of both sides of every cell of the tile: the Roe scalars of the
// row's face, the characteristic variables of its five-cell stencil (walk
// order) and, per field k, the WENO-Z weights and the scalar row (a on the
// previous unknown of the walk, b on this one, c on the next, r the
// right-hand side; closure rows of bounded lines 0, 1, 0 and the explicit
// WENO5-Z value).  Output per row: the 4 Roe scalars and 4 NV coefficients,
// laid out [side][position][entry][line] so that both this kernel's stores
// and the serial walk's loads are contiguous over the lines of a warp.
constexpr int CT_L = 32, CT_C = 32;   // lines x cells of a tile

template <typename real, int NV, bool PER>
__global__ void __launch_bounds__(256) char_rows_kernel(const CharArgs a) {
  constexpr bool F32 = sizeof(real) == 4;
  constexpr int RC = 4 * NV + 4;
  constexpr int TW = CT_C + 4;        // cells of a tile row with the halo
  __shared__ real tile[NV][CT_L][TW + 1];
  __shared__ LineGeo sg[CT_L];
  const int NMAX = a.n;               // position stride of the rows buffer
  const long long NL = a.nlines;
  const long long line0 = (long long)blockIdx.x * CT_L;
  const int c0 = blockIdx.y * CT_C;
  const real *U = reinterpret_cast<const real *>(a.U);
  int gv[NV];
  grid_vars<NV>(a, gv);
  const int tid = threadIdx.x;
  if (tid < CT_L && line0 + tid < NL) sg[tid] = line_geo(a, line0 + tid);
  __syncthreads();
  const bool along_cells = a.lines ? a.xdir != 0 : a.cell_stride == 1;
  for (int idx = tid; idx < CT_L * TW; idx += blockDim.x) {
    const int ll = along_cells ? idx / TW : idx % CT_L;
    const int j = along_cells ? idx % TW : idx / CT_L;
    const int i = c0 - 2 + j;
    if (line0 + ll >= NL) continue;
    const LineGeo g = sg[ll];
    if (i < -2 || i > g.n + 1) continue;   // never read
    real v[NV];
    line_cell<real, NV, PER>(g, U, gv, i, v);
#pragma unroll
    for (int k = 0; k < NV; ++k) tile[k][ll][j] = v[k];
  }
  __syncthreads();
  const int ll = tid % CT_L;
  const long long line = line0 + ll;
  if (line >= NL) return;
  const int n = sg[ll].n;
  real *rows = reinterpret_cast<real *>(a.rows);
  const real gam = real(a.gamma), eps = real(a.eps_weno);
  for (int q = tid / CT_L; q < 2 * CT_C; q += blockDim.x / CT_L) {
    const int side = q / CT_C;
    const int c = c0 + q % CT_C;
    if (c >= n) continue;
    const int dir = side == 0 ? 1 : -1;
    const int p = side == 0 ? c : n - 1 - c;
    const int jc = c - c0 + 2;        // the cell's column in the tile
    real win[5][NV];
#pragma unroll
    for (int w = 0; w < 5; ++w)
#pragma unroll
      for (int k = 0; k < NV; ++k) win[w][k] = tile[k][ll][jc + (w - 2) * dir];
    real rs[4], L[NV][NV];
    roe_scalars<real, NV>(win[2], win[3], gam, rs);
    left_from<real, NV>(rs, L);
    const bool closure = !PER && (p == 0 || p == n - 1);
    real *dst = rows + ((long long)side * NMAX + p) * RC * NL + line;
#pragma unroll
    for (int e = 0; e < 4; ++e) dst[e * NL] = rs[e];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      real cv[5];
      real mag = real(0);
#pragma unroll
      for (int w = 0; w < 5; ++w) {
        real s0 = real(0), s1 = real(0);
#pragma unroll
        for (int m = 0; m < NV; ++m) {
          s0 += L[k][m] * win[w][m];
          if (F32) s1 += fabs(L[k][m]) * fabs(win[w][m]);
        }
        cv[w] = s0;
        if (F32) mag = fmax(mag, s1);
      }
      real q0, q1, q2, w0, w1, w2, one;
      char_ratios<real>(cv, mag, eps, q0, q1, q2, one);
      real fa, fb, fc, fr;
      if (closure) {
        zweights<real>(real(0.1), real(0.6), real(0.3), q0, q1, q2, w0, w1, w2, one);
        const real p0 = real(2) * cv[0] - real(7) * cv[1] + real(11) * cv[2];
        const real p1 = -cv[1] + real(5) * cv[2] + real(2) * cv[3];
        const real p2 = real(2) * cv[2] + real(5) * cv[3] - cv[4];
        fa = real(0);
        fb = real(1);
        fc = real(0);
        fr = (w0 * p0 + w1 * p1 + w2 * p2) * real(1.0 / 6.0);
      } else {
        zweights<real>(real(0.2), real(0.5), real(0.3), q0, q1, q2, w0, w1, w2, one);
        const Row<real> row = compact_row<real>(w0, w1, w2, cv[1], cv[2], cv[3]);
        fa = row.a;
        fb = row.b;
        fc = row.c;
        fr = row.r;
      }
      dst[(4 + 4 * k + 0) * NL] = fa;
      dst[(4 + 4 * k + 1) * NL] = fb;
      dst[(4 + 4 * k + 2) * NL] = fc;
      dst[(4 + 4 * k + 3) * NL] = fr;
    }
  }
}

// Step 4, the serial part: one thread per (line, side) walks the line in
// the elimination order.  Position p of the walk is cell p (minus side,
// left to right) or cell n-1-p (plus side, right to left); in walk order
// both sides have the same rows (the plus row is the mirror image of the
// minus row), so "previous" and "next" below are in walk order.  At each
// position the thread rebuilds L from the four Roe scalars, takes the row
// coefficients from char_rows_kernel, and runs one step of block Thomas.
// The walk is bound by the latency of its own loads (few chains per SM), so
// the row data of the next PD - 1 positions, and in the back substitution
// their multipliers, are in flight in a per-thread shared-memory ring.
// Periodic lines solve the cyclic system with the Woodbury correction
// T = T' + U V^T, G = -B_0: T' has B_0 - G at the first position and
// B_{n-1} - C_{n-1} G^{-1} A_0 at the last, U = (G, 0, .., 0, C_{n-1}),
// V^T = (I, 0, .., 0, G^{-1} A_0); the NV columns of U ride along as extra
// right-hand sides and x = y - Z (I + V^T Z)^{-1} V^T y at the end.
template <typename real, int NV, bool PER>
__global__ void __launch_bounds__(32) char_solve_kernel(const CharArgs a) {
  constexpr int NC = PER ? NV + 1 : 1;       // right-hand-side columns
  constexpr int ROW = NV * NV + NV * NC;     // scratch values per row: Y, g
  constexpr int RC = 4 * NV + 4;             // Roe scalars and row coefficients per position
  const long long line = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (line >= a.nlines) return;
  const int side = blockIdx.y;
  const LineGeo geo = line_geo(a, line);
  const int n = geo.n;
  const int NMAX = a.n;   // position stride of rows and scratch
  const long long NL = a.nlines;
  const long long lbase = geo.base;
  const real *rows = reinterpret_cast<const real *>(a.rows) + (long long)side * NMAX * RC * NL + line;
  real *scr = reinterpret_cast<real *>(a.scr) + (long long)side * ((long long)NMAX * ROW + NV * NV) * NL + line;
  auto slot = [&](int p, int e) -> real & { return scr[((long long)p * ROW + e) * NL]; };
  auto wslot = [&](int e) -> real & { return scr[((long long)NMAX * ROW + e) * NL]; };
  int gv[NV];
  grid_vars<NV>(a, gv);
  auto cidx = [&](int p) { return side == 0 ? p : n - 1 - p; };

  // ring of PD positions: [slot][entry][thread], conflict-free; as deep as
  // the 48 KB of static shared memory allows (periodic rows are longer)
  constexpr int PD = sizeof(real) == 4 ? (PER ? 8 : 16) : 4;
  constexpr int RING = RC > ROW ? RC : ROW;
  __shared__ real ring[PD][RING][32];
  const int tid = threadIdx.x;
  auto issue_row = [&](int p) {
#pragma unroll
    for (int e = 0; e < RC; ++e)
      cp_async<sizeof(real)>(&ring[p % PD][e][tid], &rows[((long long)p * RC + e) * NL]);
  };
#pragma unroll 1
  for (int j = 0; j < PD - 1; ++j) {
    if (j < n) issue_row(j);
    cp_async_commit();
  }

  real co[RC];
  real Yp[NV][NV], gp[NV][NC];   // the previous position's multipliers
#pragma unroll 1
  for (int p = 0; p < n; ++p) {
    if (p + PD - 1 < n) issue_row(p + PD - 1);
    cp_async_commit();
    cp_async_wait<PD - 1>();   // the group of position p has landed
#pragma unroll
    for (int e = 0; e < RC; ++e) co[e] = ring[p % PD][e][tid];
    real L[NV][NV];
    {
      const real rs[4] = {co[0], co[1], co[2], co[3]};
      left_from<real, NV>(rs, L);
    }
    real ca[NV], cb[NV], cc[NV], cr[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      ca[k] = co[4 + 4 * k];
      cb[k] = co[4 + 4 * k + 1];
      cc[k] = co[4 + 4 * k + 2];
      cr[k] = co[4 + 4 * k + 3];
    }
    // block row diag(ca, cb, cc) L, eliminated against the previous
    // position: Bp = B - A Y_prev, X = [C | r - A g_prev]
    real Bp[NV][NV], X[NV][NV + NC];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
#pragma unroll
      for (int j = 0; j < NV; ++j) {
        Bp[k][j] = cb[k] * L[k][j];
        X[k][j] = cc[k] * L[k][j];
      }
      X[k][NV] = cr[k];
#pragma unroll
      for (int j = 1; j < NC; ++j) X[k][NV + j] = real(0);
    }
    if constexpr (PER) {
      if (p == 0) {
        // G = -B_0: B'_0 = B_0 - G = 2 B_0, Woodbury columns U_0 = G, and
        // G^{-1} A_0 for the last position and the final correction
        real Gm[NV][NV], GiA[NV][NV];
#pragma unroll
        for (int k = 0; k < NV; ++k)
#pragma unroll
          for (int j = 0; j < NV; ++j) {
            Gm[k][j] = -Bp[k][j];
            GiA[k][j] = ca[k] * L[k][j];
            X[k][NV + 1 + j] = Gm[k][j];
            Bp[k][j] = Bp[k][j] + Bp[k][j];
          }
        gauss_solve<real, NV, NV>(Gm, GiA);
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
          real t = real(0);
#pragma unroll
          for (int m = 0; m < NV; ++m) t += L[k][m] * Yp[m][j];
          Bp[k][j] -= ca[k] * t;
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          real t = real(0);
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
        real GiA[NV][NV];
#pragma unroll
        for (int k = 0; k < NV; ++k)
#pragma unroll
          for (int j = 0; j < NV; ++j) GiA[k][j] = wslot(k * NV + j);
#pragma unroll
        for (int k = 0; k < NV; ++k)
#pragma unroll
          for (int j = 0; j < NV; ++j) {
            real t = real(0);
#pragma unroll
            for (int m = 0; m < NV; ++m) t += X[k][m] * GiA[m][j];
            Bp[k][j] -= t;
          }
#pragma unroll
        for (int k = 0; k < NV; ++k)
#pragma unroll
          for (int j = 0; j < NV; ++j) {
            X[k][NV + 1 + j] += X[k][j];
            X[k][j] = real(0);
          }
      }
    }
    gauss_solve<real, NV, NV + NC>(Bp, X);
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
  cp_async_wait<0>();

  // back substitution x_p = g_p - Y_p x_{p+1}; step b = n-2-p reads the
  // multipliers of position p through the same ring
  real *out = reinterpret_cast<real *>(side == 0 ? a.Um : a.Up);
  real x[NV][NC];
#pragma unroll
  for (int k = 0; k < NV; ++k)
#pragma unroll
    for (int c = 0; c < NC; ++c) x[k][c] = gp[k][c];
  auto issue_mult = [&](int b) {
    const int p = n - 2 - b;
#pragma unroll
    for (int e = 0; e < ROW; ++e) cp_async<sizeof(real)>(&ring[b % PD][e][tid], &slot(p, e));
  };
#pragma unroll 1
  for (int j = 0; j < PD - 1; ++j) {
    if (j < n - 1) issue_mult(j);
    cp_async_commit();
  }
#pragma unroll 1
  for (int p = n - 1; p >= 0; --p) {
    if (p < n - 1) {
      const int b = n - 2 - p;
      if (b + PD - 1 < n - 1) issue_mult(b + PD - 1);
      cp_async_commit();
      cp_async_wait<PD - 1>();
      real Yc[ROW];
#pragma unroll
      for (int e = 0; e < ROW; ++e) Yc[e] = ring[b % PD][e][tid];
      real xn[NV][NC];
#pragma unroll
      for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int c = 0; c < NC; ++c) xn[k][c] = x[k][c];
#pragma unroll
      for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          real s = Yc[NV * NV + k * NC + c];
#pragma unroll
          for (int j = 0; j < NV; ++j) s -= Yc[k * NV + j] * xn[j][c];
          x[k][c] = s;
        }
    }
    if (PER) {
#pragma unroll
      for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int c = 0; c < NC; ++c) slot(p, NV * NV + k * NC + c) = x[k][c];
    } else {
      real *dst = out + lbase + (long long)cidx(p) * geo.cs;
#pragma unroll
      for (int k = 0; k < NV; ++k) dst[gv[k] * geo.ncell] = x[k][0];
    }
  }
  cp_async_wait<0>();
  if constexpr (PER) {
    // S = I + Z_0 + G^{-1} A_0 Z_{n-1}, t = y_0 + G^{-1} A_0 y_{n-1};
    // x_p = y_p - Z_p S^{-1} t
    real S[NV][NV], t[NV][1], GiA[NV][NV];
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
      for (int j = 0; j < NV; ++j) GiA[k][j] = wslot(k * NV + j);
#pragma unroll
    for (int k = 0; k < NV; ++k) {
#pragma unroll
      for (int j = 0; j < NV; ++j) {
        real s = (k == j ? real(1) : real(0)) + slot(0, NV * NV + k * NC + 1 + j);
#pragma unroll
        for (int m = 0; m < NV; ++m) s += GiA[k][m] * slot(n - 1, NV * NV + m * NC + 1 + j);
        S[k][j] = s;
      }
      real s = slot(0, NV * NV + k * NC);
#pragma unroll
      for (int m = 0; m < NV; ++m) s += GiA[k][m] * slot(n - 1, NV * NV + m * NC);
      t[k][0] = s;
    }
    gauss_solve<real, NV, 1>(S, t);
#pragma unroll 1
    for (int p = 0; p < n; ++p) {
      real *dst = out + lbase + (long long)cidx(p) * geo.cs;
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        real s = slot(p, NV * NV + k * NC);
#pragma unroll
        for (int j = 0; j < NV; ++j) s -= slot(p, NV * NV + k * NC + 1 + j) * t[j][0];
        dst[gv[k] * geo.ncell] = s;
      }
    }
  }
}

// ---------------------------------------------------------------- FP32, few walks
// The same walk with four lanes per (line, side) chain, for launches with
// few chains (batch groups of long 1-D lines: a few hundred walks of up to
// 8192 positions, fewer than one warp per SM in the one-thread layout,
// where the chain's latency is the whole cost).  Lane j holds column j of
// the block being eliminated and the right-hand-side columns of unknown j:
// column j of Y (and of the Woodbury block on periodic lines); the g
// column is the same in every lane (every lane forms it from the same data
// with the same multipliers).  Per position the lanes solve
// B' [Y | g] = [C | r - A g_prev] together by Gaussian elimination with
// partial pivoting: lane c finds the pivot of column c in its own column
// and hands the exchange, the pivot's reciprocal and the multipliers to the
// other lanes; the back substitution takes the upper triangle's entries
// from their lanes.  A Y_prev needs column j of Y_prev only, which lane j
// already holds.  With three fields lane 3 carries right-hand sides only.
// The eight chains of a warp stay converged (full-warp shuffles over 4-lane
// segments): the warp walks as many positions as its longest chain, and a
// chain past its own end (a shorter batched line) computes on stale data
// and stores nothing.  A position costs about twice the one-thread walk's
// instructions per chain, so with many chains the one-thread walk is
// faster; the launch picks by the number of chains.

constexpr unsigned FULL = 0xffffffffu;
constexpr int LW = 4;   // lanes per chain (shuffle segment width)

// X <- M^{-1} X over the four lanes of a chain: M's column j and NR
// columns X[s] in lane j (lane ids below are within the chain's segment)
template <int NV, int NR>
__device__ __forceinline__ void lanes_solve(float (&M)[NV], float (&X)[NR][NV]) {
  float inv[NV];
  float U[NV][NV];   // U[c][q], q > c: row c of the factor, from lane q
#pragma unroll
  for (int c = 0; c < NV; ++c) {
    if (c < NV - 1) {
      int piv = c;
      float best = fabsf(M[c]);
#pragma unroll
      for (int r = c + 1; r < NV; ++r) {
        const float m = fabsf(M[r]);
        if (m > best) { best = m; piv = r; }
      }
      piv = __shfl_sync(FULL, piv, c, LW);
#pragma unroll
      for (int r = c + 1; r < NV; ++r) {
        const bool sw = piv == r;
        const float t = M[c];
        M[c] = sw ? M[r] : t;
        M[r] = sw ? t : M[r];
#pragma unroll
        for (int s = 0; s < NR; ++s) {
          const float u = X[s][c];
          X[s][c] = sw ? X[s][r] : u;
          X[s][r] = sw ? u : X[s][r];
        }
      }
    }
    const float iv = __shfl_sync(FULL, 1.0f / M[c], c, LW);
    inv[c] = iv;
#pragma unroll
    for (int r = c + 1; r < NV; ++r) {
      const float f = __shfl_sync(FULL, M[r] * iv, c, LW);
      M[r] -= f * M[c];
#pragma unroll
      for (int s = 0; s < NR; ++s) X[s][r] -= f * X[s][c];
    }
#pragma unroll
    for (int q = c + 1; q < NV; ++q) U[c][q] = __shfl_sync(FULL, M[c], q, LW);
  }
#pragma unroll
  for (int s = 0; s < NR; ++s)
#pragma unroll
    for (int c = NV - 1; c >= 0; --c) {
      float x = X[s][c];
#pragma unroll
      for (int q = c + 1; q < NV; ++q) x -= U[c][q] * X[s][q];
      X[s][c] = x * inv[c];
    }
}

template <int NV, bool PER>
__global__ void __launch_bounds__(64) char_solve_lanes_kernel(const CharArgs a) {
  constexpr int NC = PER ? NV + 1 : 1;       // right-hand-side columns of g
  constexpr int ROW = NV * NV + NV * NC;     // scratch values per row: Y, g
  constexpr int RC = 4 * NV + 4;             // Roe scalars and row coefficients per position
  constexpr int CH = 16;                     // chains per block
  constexpr int PD = 8;                      // positions in flight
  constexpr int NR = PER ? 3 : 2;            // right-hand sides per lane: Y col, (Z col,) g
  constexpr int SG = NR - 1;
  constexpr int RING = RC > ROW ? RC : ROW;
  // (a chain stride of 18 words instead of 16 takes the back substitution's
  // 4-way bank conflicts away but measured slower: 120 against 95 ms per
  // Riemann batch step)
  __shared__ float ring[PD][RING][CH];
  const int tid = threadIdx.x;
  const int ch = tid >> 2, j = tid & 3;
  const long long NL = a.nlines;
  const long long line_ = (long long)blockIdx.x * CH + ch;
  const bool live = line_ < NL;
  const long long line = live ? line_ : NL - 1;   // idle chains repeat the last line, store nothing
  const bool col = live && j < NV;                // lane owns a column of the block
  const int side = blockIdx.y;
  const LineGeo geo = line_geo(a, line);
  const int n = geo.n;
  const int nw = __reduce_max_sync(FULL, n);      // the warp's longest chain
  const int NMAX = a.n;                           // position stride of rows and scratch
  const long long lbase = geo.base;
  const float *rows = reinterpret_cast<const float *>(a.rows) + (long long)side * NMAX * RC * NL + line;
  float *scr = reinterpret_cast<float *>(a.scr) + (long long)side * ((long long)NMAX * ROW + NV * NV) * NL + line;
  auto slot = [&](int p, int e) -> float & { return scr[((long long)p * ROW + e) * NL]; };
  auto wslot = [&](int e) -> float & { return scr[((long long)NMAX * ROW + e) * NL]; };
  int gv[NV];
  grid_vars<NV>(a, gv);
  auto cidx = [&](int p) { return side == 0 ? p : n - 1 - p; };
  // lane j's entries of a row record, split four ways over the chain
  auto issue_row = [&](int p) {
#pragma unroll
    for (int q = 0; q < RC / 4; ++q) {
      const int e = j + 4 * q;
      cp_async<4>(&ring[p % PD][e][ch], &rows[((long long)p * RC + e) * NL]);
    }
  };
#pragma unroll 1
  for (int i = 0; i < PD - 1; ++i) {
    if (i < n) issue_row(i);
    cp_async_commit();
  }
  // k-th entry of this lane's column of an NV x NV matrix (no dynamic register index)
  auto colj = [&](const float (&Mk)[NV]) {
    float v = Mk[0];
#pragma unroll
    for (int q = 1; q < NV; ++q) v = j == q ? Mk[q] : v;
    return v;
  };

  float Yc[NV], Zc[NV], gc[NV], GiAc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) Yc[k] = Zc[k] = gc[k] = GiAc[k] = 0.0f;
#pragma unroll 1
  for (int p = 0; p < nw; ++p) {
    const bool act = live && p < n;
    __syncwarp();   // slot (p - 1) % PD is read by every lane before it is refilled
    if (p + PD - 1 < n) issue_row(p + PD - 1);
    cp_async_commit();
    cp_async_wait<PD - 1>();
    __syncwarp();   // the chain's four lanes' copies of position p have landed
    float co[RC];
#pragma unroll
    for (int e = 0; e < RC; ++e) co[e] = ring[p % PD][e][ch];
    float L[NV][NV];
    {
      const float rs[4] = {co[0], co[1], co[2], co[3]};
      left_from<float, NV>(rs, L);
    }
    float ca[NV], cb[NV], cc[NV], Lj[NV];
    float M[NV], X[NR][NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      ca[k] = co[4 + 4 * k];
      cb[k] = co[4 + 4 * k + 1];
      cc[k] = co[4 + 4 * k + 2];
      Lj[k] = colj(L[k]);
      M[k] = cb[k] * Lj[k];
      X[0][k] = cc[k] * Lj[k];
      X[SG][k] = co[4 + 4 * k + 3];
      if (PER) X[1][k] = 0.0f;
    }
    if constexpr (PER) {
      if (p == 0) {
        // G = -B_0: B'_0 = 2 B_0, Woodbury column j of U_0 = G, and column
        // j of G^{-1} A_0 for the last position and the final correction
        float Gm[NV], Aj[1][NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) {
          Gm[k] = -M[k];
          Aj[0][k] = ca[k] * Lj[k];
          X[1][k] = Gm[k];
          M[k] += M[k];
        }
        lanes_solve<NV, 1>(Gm, Aj);
#pragma unroll
        for (int k = 0; k < NV; ++k) {
          GiAc[k] = Aj[0][k];
          if (col) wslot(k * NV + j) = GiAc[k];
        }
      }
    }
    if (p > 0) {
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        float tY = 0.0f, tg = 0.0f, tz = 0.0f;
#pragma unroll
        for (int m = 0; m < NV; ++m) {
          tY += L[k][m] * Yc[m];
          tg += L[k][m] * gc[m];
          if (PER) tz += L[k][m] * Zc[m];
        }
        M[k] -= ca[k] * tY;
        X[SG][k] -= ca[k] * tg;
        if (PER) X[1][k] -= ca[k] * tz;
      }
    }
    if constexpr (PER) {
      if (p == n - 1) {
        // B'_{n-1} = B_{n-1} - C_{n-1} G^{-1} A_0; the coupling to x_0 moves
        // into the Woodbury columns (U_{n-1} = C_{n-1})
#pragma unroll
        for (int k = 0; k < NV; ++k) {
          float t = 0.0f;
#pragma unroll
          for (int m = 0; m < NV; ++m) t += cc[k] * L[k][m] * GiAc[m];
          M[k] -= t;
          X[1][k] += X[0][k];
          X[0][k] = 0.0f;
        }
      }
    }
    lanes_solve<NV, NR>(M, X);
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      Yc[k] = X[0][k];
      gc[k] = X[SG][k];
      if (PER) Zc[k] = X[1][k];
      if (col && act) {
        slot(p, k * NV + j) = Yc[k];
        if (PER) slot(p, NV * NV + k * NC + 1 + j) = Zc[k];
      }
    }
    if (act && j == 0) {
#pragma unroll
      for (int k = 0; k < NV; ++k) slot(p, NV * NV + k * NC) = gc[k];
    }
  }
  cp_async_wait<0>();
  __syncwarp();   // the chain's scratch rows, written by all four lanes, are read below

  // back substitution x_p = g_p - Y_p x_{p+1}; lane k (< NV) forms row k of
  // x_p from row k of (Y_p, g_p) and all of x_{p+1}; step b is position
  // n - 2 - b of each chain
  const int k = j < NV ? j : NV - 1;
  int gvk = gv[0];   // grid variable of field k, without a dynamic register index
#pragma unroll
  for (int q = 1; q < NV; ++q) gvk = k == q ? gv[q] : gvk;
  float *out = reinterpret_cast<float *>(side == 0 ? a.Um : a.Up);
  float x[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) x[c] = slot(n - 1, NV * NV + k * NC + c);
  auto issue_mult = [&](int b) {
    if (j >= NV) return;   // lane 3 of a three-field chain: nothing of its own
    const int p = n - 2 - b;
#pragma unroll
    for (int q = 0; q < NV; ++q) cp_async<4>(&ring[b % PD][k * NV + q][ch], &slot(p, k * NV + q));
#pragma unroll
    for (int c = 0; c < NC; ++c)
      cp_async<4>(&ring[b % PD][NV * NV + k * NC + c][ch], &slot(p, NV * NV + k * NC + c));
  };
  __syncwarp();
#pragma unroll 1
  for (int i = 0; i < PD - 1; ++i) {
    if (i < n - 1) issue_mult(i);
    cp_async_commit();
  }
  auto store_x = [&](int p) {
    if (!col) return;
    if (PER) {
#pragma unroll
      for (int c = 0; c < NC; ++c) slot(p, NV * NV + k * NC + c) = x[c];
    } else {
      out[lbase + (long long)cidx(p) * geo.cs + (long long)gvk * geo.ncell] = x[0];
    }
  };
  store_x(n - 1);
#pragma unroll 1
  for (int b = 0; b < nw - 1; ++b) {
    const int p = n - 2 - b;
    if (b + PD - 1 < n - 1) issue_mult(b + PD - 1);
    cp_async_commit();
    cp_async_wait<PD - 1>();   // this lane's own copies only: no exchange through the ring
    float Yr[NV], gr[NC];   // (lane 3 of a three-field chain reads values it never uses)
#pragma unroll
    for (int q = 0; q < NV; ++q) Yr[q] = ring[b % PD][k * NV + q][ch];
#pragma unroll
    for (int c = 0; c < NC; ++c) gr[c] = ring[b % PD][NV * NV + k * NC + c][ch];
    float xn[NV][NC];
#pragma unroll
    for (int q = 0; q < NV; ++q)
#pragma unroll
      for (int c = 0; c < NC; ++c) xn[q][c] = __shfl_sync(FULL, x[c], q, LW);
    if (p >= 0) {
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        float s = gr[c];
#pragma unroll
        for (int q = 0; q < NV; ++q) s -= Yr[q] * xn[q][c];
        x[c] = s;
      }
      store_x(p);
    }
  }
  cp_async_wait<0>();
  if constexpr (PER) {
    __syncwarp();   // every lane's rows of y and Z are in the scratch
    // S = I + Z_0 + G^{-1} A_0 Z_{n-1}, t = y_0 + G^{-1} A_0 y_{n-1};
    // x_p = y_p - Z_p S^{-1} t, row k in lane k
    float S[NV][NV], t[NV][1], GiA[NV][NV];
#pragma unroll
    for (int r = 0; r < NV; ++r)
#pragma unroll
      for (int q = 0; q < NV; ++q) GiA[r][q] = wslot(r * NV + q);
#pragma unroll
    for (int r = 0; r < NV; ++r) {
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        float s = (r == q ? 1.0f : 0.0f) + slot(0, NV * NV + r * NC + 1 + q);
#pragma unroll
        for (int m = 0; m < NV; ++m) s += GiA[r][m] * slot(n - 1, NV * NV + m * NC + 1 + q);
        S[r][q] = s;
      }
      float s = slot(0, NV * NV + r * NC);
#pragma unroll
      for (int m = 0; m < NV; ++m) s += GiA[r][m] * slot(n - 1, NV * NV + m * NC);
      t[r][0] = s;
    }
    gauss_solve<float, NV, 1>(S, t);
    if (col) {
#pragma unroll 4
      for (int p = 0; p < n; ++p) {
        float s = slot(p, NV * NV + k * NC);
#pragma unroll
        for (int q = 0; q < NV; ++q) s -= slot(p, NV * NV + k * NC + 1 + q) * t[q][0];
        out[lbase + (long long)cidx(p) * geo.cs + (long long)gvk * geo.ncell] = s;
      }
    }
  }
}

// Without a timed choice (CharArgs::layout < 0), FP32 launches with fewer
// lines than this take the four-lane walk (2048 lines: 4096 chains, fewer
// than one warp per SM in the one-thread layout; measured: the 4096^2
// grid's 8192 chains walk faster one thread each, 3.41 against 4.17 ms, the
// Riemann batch's groups of at most ~1700 chains faster four lanes each, 96
// against 149 ms per step)
constexpr long long LANES_BELOW = 2048;

template <typename real, int NV, bool PER>
cudaError_t launch_nv(const CharArgs &a, int part, cudaStream_t st) {
  if (part == 0) {
    const dim3 grid((unsigned)((a.nlines + CT_L - 1) / CT_L), (unsigned)((a.n + CT_C - 1) / CT_C), 1);
    char_rows_kernel<real, NV, PER><<<grid, 256, 0, st>>>(a);
  } else {
    if constexpr (sizeof(real) == 4) {
      if (a.layout == 1 || (a.layout < 0 && a.nlines < LANES_BELOW)) {
        char_solve_lanes_kernel<NV, PER><<<dim3((unsigned)((a.nlines + 15) / 16), 2, 1), 64, 0, st>>>(a);
        return cudaGetLastError();
      }
    }
    char_solve_kernel<real, NV, PER><<<dim3((unsigned)((a.nlines + 31) / 32), 2, 1), 32, 0, st>>>(a);
  }
  return cudaGetLastError();
}

// part 0: the parallel rows kernel; part 1: the serial block solve
template <typename real>
cudaError_t launch_char_recon_t(const CharArgs &a, int nv, bool periodic, int part, cudaStream_t st) {
  if (nv == 3) return periodic ? launch_nv<real, 3, true>(a, part, st) : launch_nv<real, 3, false>(a, part, st);
  return periodic ? launch_nv<real, 4, true>(a, part, st) : launch_nv<real, 4, false>(a, part, st);
}

}  // namespace chr
}  // namespace ppk
