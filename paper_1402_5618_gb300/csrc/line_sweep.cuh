// line_sweep.cuh -- the fused per-stage line operator of the FVCW scheme.
//
// One thread-block cluster of R CTAs owns one grid line of n cells; CTA r
// holds the contiguous segment [r*SEG, min((r+1)*SEG, n)) of it in shared
// memory and runs, in order:
//   load     cell averages of the segment plus a two-cell halo (ghost cells
//            from the boundary condition at the line ends);
//   weights  WENO-Z weights of every cell for both sides (Sec. 2.2, eq.
//            (weight)), kept in shared memory for the two passes below;
//   solve    for each conserved variable the minus and plus compact-WENO
//            systems (eq. (CWENO-FV)) by Thomas elimination in the stable
//            order (minus left to right, plus right to left), parallelised
//            exactly: every thread owns a chunk of M rows, the forward
//            elimination of a chunk is a projective map of the state (c', d')
//            carried in from the previous rows ((P, Q, D) with c' = P/Q,
//            d' = D/Q evolves linearly), the maps are composed by
//            warp-shuffle scans, across warps in shared memory and across the
//            cluster's CTAs through distributed shared memory; the back
//            substitution is an affine map per chunk, scanned the same way.
//            Periodic lines add the second right-hand side of the
//            Sherman-Morrison correction to the same sweep.
//   limit    Zhang-Shu limiter per cell (Sec. 2.4);
//   flux     HLLC at every face of the segment (the two segment-end faces
//            read the neighbour CTA's limited face value);
//   update   flux difference (eq. (1DEulerFV-b)) and either the x-sweep
//            output D = L_x, or the SSP-RK3 stage combination (eq. (RK3))
//            with L = D + L_y (2-D) / L (1-D), plus the grid-wide reductions
//            that fix the next stage's limiter epsilon and the next dt.
//
// real = double: the plain form (FP64 state and arithmetic).
// real = float: the mixed form -- FP32 line arithmetic, the state stored as
// FP32 hi + lo pairs combined with compensated (double-float) arithmetic,
// FP64 only for the limiter factors of cells that need limiting and for the
// Sherman-Morrison scalars.
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "batch_lines.cuh"
#include "dfloat.cuh"
#include "physics.cuh"

namespace cg = cooperative_groups;

namespace ppk {

constexpr int SEGC = 512;       // cells per CTA segment (all chunk lengths)

// device-side control block of one problem (time, dt, reductions, flags)
struct Ctl {
  double t, t_final, dt, cfl, dt_cap;
  long long step, step_limit;
  int active, done, err_steps, err_rate;
  double eps0;                         // limiter epsilon for stage 1
  unsigned long long minrho[3];        // min density after stage k (double bits; +inf init)
  unsigned long long rate;             // max rate after stage 3 (double bits)
  unsigned long long nviol;            // cells outside G
  unsigned long long first_bad;        // min flat index of a bad cell (~0 none)
  unsigned long long theta1, theta2;   // limiter activations
  double last_dt;
  double eps_pos;
  // eq. (CFL-CD) on the limited face values (face_cfl > 0): the largest
  // (|u| + a)/h over the face values of this step's stages per direction
  // (double bits; NaN propagates), the rate of the last accepted step, and
  // what a step that is redone restores
  unsigned long long frate[2];
  double face_cfl;
  double frate_prev;
  double t_prev;
  unsigned long long rate_n, minrho_n;
  long long nreject;
  int nrej_run;
};

enum { MODE_XSWEEP = 0, MODE_FINAL = 1, MODE_OPERATOR = 2 };

struct SweepArgs {
  // plain form: FP64 planes [nv][ncell]
  const double *U;    // stage input
  const double *U0;   // U^n
  double *Uout;       // FINAL: stage output
  // mixed form: FP32 hi / lo planes of the same states
  const float *Uh, *Ul, *U0h, *U0l;
  float *Uoh, *Uol;
  const void *Din;    // flux difference of the other direction (2-D), real
  void *Dout;         // x-sweep output, real
  double *Lout;       // OPERATOR: L (FP64 planes)
  long long ncell;    // cells per variable plane
  int n;              // cells per line
  int R;              // CTAs per line (cluster size)
  long long cell_stride, line_stride;
  int vn, vt;         // grid index of the normal / tangential momentum (vt < 0 in 1-D)
  int bclo, bchi;
  double h, h_other;  // cell size along the line / across (0 in 1-D)
  double ih;          // 1 / h (from the host: no FP64 division per thread)
  double ih_other;    // 1 / h_other (0 in 1-D)
  // FP32 copies for the mixed form's kernels (converting a double costs a
  // slot of GB300's FP64 pipe per warp): gamma, wgl, eps_weno, 1/h,
  // 1/h_other, gamma (gamma - 1), and the limiter epsilon of eps_fixed
  float gamma_f, wgl_f, eps_weno_f, ih_f, ih_other_f, gg1_f, eps_fixed_f;
  double gamma, wgl, eps_weno;
  int stage;          // 0, 1, 2
  double eps_fixed;   // > 0: fixed limiter epsilon, no control-block checks (operator evaluation)
  int limiter;
  int flux;           // 0 HLLC, 1 local Lax-Friedrichs
  int fcheck;         // 1: reduce the face speeds into ctl->frate[fdir]
  int fdir;           // 0: x faces, 1: y faces
  // face values U^-, U^+ computed by another kernel (planes of the line's
  // arithmetic in the state's layout); nullptr: the kernel reconstructs them
  const void *Fm_pre, *Fp_pre;
  Ctl *ctl;
  // batched launch: line table and problem descriptors (nullptr: one problem)
  const LineRef *lines;
  const ProbDesc *probs;
  int xdir;           // batched launch: 1 x lines, 0 y lines, 2 rows of the transposed planes
  long long nvals;    // batched mixed form: values per hi block (lo block follows)
};

// resolve the line a cluster works on: for a batched launch, take the
// problem's grid, boundaries, control block and its slice of every buffer
template <typename real, int NV>
__device__ __forceinline__ void bind_line(SweepArgs &a, long long &line) {
  if (!a.lines) return;
  LineRef lr = a.lines[line];
  const ProbDesc pd = a.probs[lr.prob];
  line = lr.line;
  a.ctl = a.ctl + lr.prob;
  a.ncell = pd.ncell;
  if (a.xdir == 1) {
    a.n = pd.nx; a.cell_stride = 1; a.line_stride = pd.nx;
    a.bclo = pd.bc[0]; a.bchi = pd.bc[1];
    a.h = pd.dx; a.h_other = NV == 4 ? pd.dy : 0.0; a.ih = pd.idx; a.ih_other = NV == 4 ? pd.idy : 0.0;
    a.ih_f = (float)a.ih; a.ih_other_f = (float)a.ih_other;
  } else if (a.xdir == 2) {   // a row of the problem's transposed planes: a y line
    a.n = pd.ny; a.cell_stride = 1; a.line_stride = pd.ny;
    a.bclo = pd.bc[2]; a.bchi = pd.bc[3];
    a.h = pd.dy; a.h_other = pd.dx; a.ih = pd.idy; a.ih_other = pd.idx;
    a.ih_f = (float)a.ih; a.ih_other_f = (float)a.ih_other;
  } else {
    a.n = pd.ny; a.cell_stride = pd.nx; a.line_stride = 1;
    a.bclo = pd.bc[2]; a.bchi = pd.bc[3];
    a.h = pd.dy; a.h_other = pd.dx; a.ih = pd.idy; a.ih_other = pd.idx;
    a.ih_f = (float)a.ih; a.ih_other_f = (float)a.ih_other;
  }
  const long long o = pd.off;
  if (a.U) a.U += o;
  if (a.U0) a.U0 += o;
  if (a.Uout) a.Uout += o;
  if (a.Uh) { a.Uh += o; a.Ul = a.Uh + a.nvals; }
  if (a.U0h) { a.U0h += o; a.U0l = a.U0h + a.nvals; }
  if (a.Uoh) { a.Uoh += o; a.Uol = a.Uoh + a.nvals; }
  if (a.Lout) a.Lout += o;
  if (a.Fm_pre) {   // face values of the characteristic-wise reconstruction, same layout
    a.Fm_pre = reinterpret_cast<const real *>(a.Fm_pre) + o;
    a.Fp_pre = reinterpret_cast<const real *>(a.Fp_pre) + o;
  }
}

// ---------------------------------------------------------------- maps
// Forward elimination map of a run of rows acting on the projective state
// (P, Q, D, Z): c' = P/Q, d' = D/Q and, on periodic lines, z' = Z/Q for the
// second right-hand side.  The map has the block form
//   [P;Q]' = G [P;Q],  D' = dP P + dQ Q + mu D,  Z' = zP P + zQ Q + mu Z.
template <typename real>
struct Fwd {
  real g00, g01, g10, g11, dP, dQ, mu, zP, zQ;
};

template <typename real>
__device__ __forceinline__ Fwd<real> fwd_identity() {
  Fwd<real> f;
  f.g00 = real(1); f.g01 = real(0); f.g10 = real(0); f.g11 = real(1);
  f.dP = real(0); f.dQ = real(0); f.mu = real(1); f.zP = real(0); f.zQ = real(0);
  return f;
}

// Y o X (X first)
template <typename real, bool PER>
__device__ __forceinline__ Fwd<real> fwd_compose(const Fwd<real> &Y, const Fwd<real> &X) {
  Fwd<real> f;
  f.g00 = Y.g00 * X.g00 + Y.g01 * X.g10;
  f.g01 = Y.g00 * X.g01 + Y.g01 * X.g11;
  f.g10 = Y.g10 * X.g00 + Y.g11 * X.g10;
  f.g11 = Y.g10 * X.g01 + Y.g11 * X.g11;
  f.dP = Y.dP * X.g00 + Y.dQ * X.g10 + Y.mu * X.dP;
  f.dQ = Y.dP * X.g01 + Y.dQ * X.g11 + Y.mu * X.dQ;
  f.mu = Y.mu * X.mu;
  if (PER) {
    f.zP = Y.zP * X.g00 + Y.zQ * X.g10 + Y.mu * X.zP;
    f.zQ = Y.zP * X.g01 + Y.zQ * X.g11 + Y.mu * X.zQ;
  } else {
    f.zP = real(0); f.zQ = real(0);
  }
  return f;
}

// row first, then the accumulated map (left multiplication by the row)
template <typename real, bool PER>
__device__ __forceinline__ void fwd_push_left(Fwd<real> &f, const Row<real> &w, real u) {
  Fwd<real> o = f;
  f.g00 = w.c * o.g10;
  f.g01 = w.c * o.g11;
  f.g10 = -w.a * o.g00 + w.b * o.g10;
  f.g11 = -w.a * o.g01 + w.b * o.g11;
  f.dP = w.r * o.g10 - w.a * o.dP;
  f.dQ = w.r * o.g11 - w.a * o.dQ;
  if (PER) {
    f.zP = u * o.g10 - w.a * o.zP;
    f.zQ = u * o.g11 - w.a * o.zQ;
  }
  f.mu = -w.a * o.mu;
}

// accumulated map first, then the row (right multiplication by the row)
template <typename real, bool PER>
__device__ __forceinline__ void fwd_push_right(Fwd<real> &f, const Row<real> &w, real u) {
  Fwd<real> o = f;
  f.g00 = -w.a * o.g01;
  f.g01 = w.c * o.g00 + w.b * o.g01;
  f.g10 = -w.a * o.g11;
  f.g11 = w.c * o.g10 + w.b * o.g11;
  f.dP = -w.a * o.dQ;
  f.dQ = w.c * o.dP + w.b * o.dQ + o.mu * w.r;
  if (PER) {
    f.zP = -w.a * o.zQ;
    f.zQ = w.c * o.zP + w.b * o.zQ + o.mu * u;
  }
  f.mu = -w.a * o.mu;
}

// power of two near 1/m (exact scaling, no division): 2^-(exponent of m)
__device__ __forceinline__ float pow2_inv(float m) {
  int e = (__float_as_int(m) >> 23) & 0xff;
  return (e > 0 && e < 254) ? __int_as_float((254 - e) << 23) : 1.0f;
}
__device__ __forceinline__ double pow2_inv(double m) {
  long long e = (__double_as_longlong(m) >> 52) & 0x7ff;
  return (e > 0 && e < 2046) ? __longlong_as_double((2046 - e) << 52) : 1.0;
}

// FP64 WENO-Z weights (w0, w2) of the minus side and (v0, v2) of the plus
// side (eq. (weight), linear weights 0.2, 0.5, 0.3, the plus side on the
// mirrored indicators) with one division for both: with d_k = beta_k + eps
// and D = d0 d1 d2, alpha_k D^2 = c_k (D^2 + tau^2 (D / d_k)^2), a common
// factor of each side's weights, and one reciprocal of the product of the
// two sides' sums normalises both.  (d, tau) are first scaled by a power of
// two near 1/max d (exact, the weights are homogeneous in them) so that the
// sixth powers stay in range.
__device__ __forceinline__ void zweights_both_fp64(double um2, double um1, double u0, double up1,
                                                   double up2, double eps, double &w0, double &w2,
                                                   double &v0, double &v2) {
  const double c13 = 13.0 / 12.0;
  const double b0 = c13 * sqr(um2 - 2.0 * um1 + u0) + 0.25 * sqr(um2 - 4.0 * um1 + 3.0 * u0);
  const double b1 = c13 * sqr(um1 - 2.0 * u0 + up1) + 0.25 * sqr(um1 - up1);
  const double b2 = c13 * sqr(u0 - 2.0 * up1 + up2) + 0.25 * sqr(3.0 * u0 - 4.0 * up1 + up2);
  double tau = fabs(b2 - b0);
  double d0 = b0 + eps, d1 = b1 + eps, d2 = b2 + eps;
  const double sc = pow2_inv(fmax(fmax(d0, d1), d2));
  d0 *= sc; d1 *= sc; d2 *= sc; tau *= sc;
  const double p01 = d0 * d1, p02 = d0 * d2, p12 = d1 * d2;
  const double D2 = sqr(p01 * d2), t2 = tau * tau;
  const double e0 = t2 * sqr(p12), e1 = t2 * sqr(p02), e2 = t2 * sqr(p01);
  // minus: (c0, c1, c2) on (e0, e1, e2); plus: the same c on (e2, e1, e0)
  const double am0 = 0.2 * (D2 + e0), am1 = 0.5 * (D2 + e1), am2 = 0.3 * (D2 + e2);
  const double ap0 = 0.2 * (D2 + e2), ap2 = 0.3 * (D2 + e0);
  const double sm = am0 + am1 + am2, sp = ap0 + am1 + ap2;
  const double inv = 1.0 / (sm * sp);
  const double ism = sp * inv, isp = sm * inv;
  w0 = am0 * ism;
  w2 = am2 * ism;
  v0 = ap0 * isp;
  v2 = ap2 * isp;
}

// rescale the map (its projective action is unchanged) so that the largest
// entry of G lies in [1, 2)
template <typename real>
__device__ __forceinline__ void fwd_normalise(Fwd<real> &f) {
  real m = fmax(fmax(fabs(f.g00), fabs(f.g01)), fmax(fabs(f.g10), fabs(f.g11)));
  if (m > real(0)) {
    real s = pow2_inv(m);
    f.g00 *= s; f.g01 *= s; f.g10 *= s; f.g11 *= s;
    f.dP *= s; f.dQ *= s; f.mu *= s; f.zP *= s; f.zQ *= s;
  }
}

// state (c', d', z') -> map -> state, renormalised to Q = 1
template <typename real, bool PER>
__device__ __forceinline__ void fwd_apply(const Fwd<real> &f, real &cp, real &dp, real &zp) {
  real P = f.g00 * cp + f.g01;
  real Q = f.g10 * cp + f.g11;
  real D = f.dP * cp + f.dQ + f.mu * dp;
  real Z = PER ? f.zP * cp + f.zQ + f.mu * zp : real(0);
  real iq = real(1) / Q;
  cp = P * iq;
  dp = D * iq;
  if (PER) zp = Z * iq;
}

template <typename real>
__device__ __forceinline__ real shfl_up_r(real v, int d, int width = 32) {
  return __shfl_up_sync(0xffffffffu, v, d, width);
}
template <typename real>
__device__ __forceinline__ real shfl_down_r(real v, int d, int width = 32) {
  return __shfl_down_sync(0xffffffffu, v, d, width);
}

template <typename real, bool PER, bool UP>
__device__ __forceinline__ Fwd<real> fwd_shfl(const Fwd<real> &f, int d, int width = 32) {
  Fwd<real> o;
#define PPK_SH(x) o.x = UP ? shfl_up_r(f.x, d, width) : shfl_down_r(f.x, d, width)
  PPK_SH(g00); PPK_SH(g01); PPK_SH(g10); PPK_SH(g11); PPK_SH(dP); PPK_SH(dQ); PPK_SH(mu);
  if (PER) { PPK_SH(zP); PPK_SH(zQ); } else { o.zP = real(0); o.zQ = real(0); }
#undef PPK_SH
  return o;
}

// back-substitution map of a run: x_first = A + B x_after (z alike, same B)
template <typename real>
struct Bwd {
  real A, B, Az;
};

// the run X followed (in back-substitution order) by the run Y:
// x_first(X) = X.A + X.B (Y.A + Y.B x_after(Y))
template <typename real>
__device__ __forceinline__ Bwd<real> bwd_compose(const Bwd<real> &X, const Bwd<real> &Y) {
  Bwd<real> r;
  r.A = X.A + X.B * Y.A;
  r.Az = X.Az + X.B * Y.Az;
  r.B = X.B * Y.B;
  return r;
}

// split cluster barrier: arrive (release this CTA's shared-memory writes to
// the cluster) and wait (acquire the other CTAs'), with independent work
// between the two halves
__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release;\n" ::: "memory");
}
__device__ __forceinline__ void cluster_arrive_relaxed() {   // publishes no data
  asm volatile("barrier.cluster.arrive.relaxed;\n" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire;\n" ::: "memory");
}

// ---------------------------------------------------------------- pairs
// The mixed form advances the minus (.x) and plus (.y) systems together with
// paired FP32 instructions (one instruction, two lanes' worth of FP32 work;
// each component rounds as the scalar fused multiply-add does).
__device__ __forceinline__ float2 p_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 p_set(float a) { return make_float2(a, a); }

// forward maps of both systems
struct Fwd2 {
  float2 g00, g01, g10, g11, dP, dQ, mu, zP, zQ;
};

__device__ __forceinline__ Fwd2 fwd2_pack(const Fwd<float> &m, const Fwd<float> &p) {
  Fwd2 f;
  f.g00 = make_float2(m.g00, p.g00); f.g01 = make_float2(m.g01, p.g01);
  f.g10 = make_float2(m.g10, p.g10); f.g11 = make_float2(m.g11, p.g11);
  f.dP = make_float2(m.dP, p.dP); f.dQ = make_float2(m.dQ, p.dQ);
  f.mu = make_float2(m.mu, p.mu); f.zP = make_float2(m.zP, p.zP); f.zQ = make_float2(m.zQ, p.zQ);
  return f;
}

__device__ __forceinline__ void fwd2_unpack(const Fwd2 &f, Fwd<float> &m, Fwd<float> &p) {
  m.g00 = f.g00.x; m.g01 = f.g01.x; m.g10 = f.g10.x; m.g11 = f.g11.x;
  m.dP = f.dP.x; m.dQ = f.dQ.x; m.mu = f.mu.x; m.zP = f.zP.x; m.zQ = f.zQ.x;
  p.g00 = f.g00.y; p.g01 = f.g01.y; p.g10 = f.g10.y; p.g11 = f.g11.y;
  p.dP = f.dP.y; p.dQ = f.dQ.y; p.mu = f.mu.y; p.zP = f.zP.y; p.zQ = f.zQ.y;
}

// Y o X (X first), both systems
template <bool PER>
__device__ __forceinline__ Fwd2 fwd2_compose(const Fwd2 &Y, const Fwd2 &X) {
  Fwd2 f;
  f.g00 = p_fma(Y.g01, X.g10, p_mul(Y.g00, X.g00));
  f.g01 = p_fma(Y.g01, X.g11, p_mul(Y.g00, X.g01));
  f.g10 = p_fma(Y.g11, X.g10, p_mul(Y.g10, X.g00));
  f.g11 = p_fma(Y.g11, X.g11, p_mul(Y.g10, X.g01));
  f.dP = p_fma(Y.mu, X.dP, p_fma(Y.dQ, X.g10, p_mul(Y.dP, X.g00)));
  f.dQ = p_fma(Y.mu, X.dQ, p_fma(Y.dQ, X.g11, p_mul(Y.dP, X.g01)));
  f.mu = p_mul(Y.mu, X.mu);
  if (PER) {
    f.zP = p_fma(Y.mu, X.zP, p_fma(Y.zQ, X.g10, p_mul(Y.zP, X.g00)));
    f.zQ = p_fma(Y.mu, X.zQ, p_fma(Y.zQ, X.g11, p_mul(Y.zP, X.g01)));
  } else {
    f.zP = p_set(0.0f); f.zQ = p_set(0.0f);
  }
  return f;
}

__device__ __forceinline__ void fwd2_normalise(Fwd2 &f) {
  float mx = fmaxf(fmaxf(fabsf(f.g00.x), fabsf(f.g01.x)), fmaxf(fabsf(f.g10.x), fabsf(f.g11.x)));
  float my = fmaxf(fmaxf(fabsf(f.g00.y), fabsf(f.g01.y)), fmaxf(fabsf(f.g10.y), fabsf(f.g11.y)));
  const float2 sc = make_float2(pow2_inv(mx), pow2_inv(my));   // 1 for 0, inf, nan
  f.g00 = p_mul(f.g00, sc); f.g01 = p_mul(f.g01, sc); f.g10 = p_mul(f.g10, sc);
  f.g11 = p_mul(f.g11, sc); f.dP = p_mul(f.dP, sc); f.dQ = p_mul(f.dQ, sc);
  f.mu = p_mul(f.mu, sc); f.zP = p_mul(f.zP, sc); f.zQ = p_mul(f.zQ, sc);
}

// back-substitution maps of both systems
struct Bwd2 {
  float2 A, B, Az;
};

__device__ __forceinline__ Bwd2 bwd2_compose(const Bwd2 &X, const Bwd2 &Y) {
  Bwd2 r;
  r.A = p_fma(X.B, Y.A, X.A);
  r.Az = p_fma(X.B, Y.Az, X.Az);
  r.B = p_mul(X.B, Y.B);
  return r;
}

// WENO-Z weights w0, w2 of the minus side (ratios q0, q1, q2, linear weights
// 0.2, 0.5, 0.3) and v0, v2 of the plus side (the same ratios reversed), in
// paired FP32; the middle term is common to both
__device__ __forceinline__ void zweights_pair(float q0, float q1, float q2, float one, float &w0,
                                              float &w2, float &v0, float &v2) {
  const float2 o2 = p_set(one);
  const float2 a0 = p_mul(p_set(0.2f), p_add(o2, make_float2(q0, q2)));
  const float a1 = 0.5f * (one + q1);
  const float2 a2 = p_mul(p_set(0.3f), p_add(o2, make_float2(q2, q0)));
  const float2 sum = p_add(p_add(a0, a2), p_set(a1));
  const float2 is = make_float2(1.0f / sum.x, 1.0f / sum.y);
  const float2 W0 = p_mul(a0, is), W2 = p_mul(a2, is);
  w0 = W0.x;
  w2 = W2.x;
  v0 = W0.y;
  v2 = W2.y;
}

// the compact row of both systems from their (w0, w2) and neighbour averages
__device__ __forceinline__ void row2(float2 w0, float2 w2, float2 up, float2 u0, float2 un,
                                     float2 &a, float2 &b, float2 &c, float2 &r) {
  const float2 th = p_set(1.0f / 3.0f), sx = p_set(1.0f / 6.0f);
  a = p_mul(p_add(p_set(1.0f), p_add(w0, p_neg(w2))), th);
  b = p_mul(p_add(p_set(2.0f), p_neg(w0)), th);
  c = p_mul(w2, th);
  const float2 k0 = p_fma(p_set(-4.0f), w2, p_set(5.0f));                 // 5 - 4 w2
  const float2 k1 = p_fma(p_set(4.0f), w2, p_add(p_set(1.0f), p_neg(w0)));  // 1 - w0 + 4 w2
  r = p_mul(p_fma(k1, un, p_fma(k0, u0, p_mul(w0, up))), sx);
}

// ---------------------------------------------------------------- smem
template <typename real, int NV, int WPV>
struct Exch {
  Fwd<real> warp_fwd[NV][2][WPV];
  real warp_in[NV][2][WPV][3];   // incoming (c', d', z') of each warp
  Fwd<real> seg_fwd[NV][2];
  Bwd<real> warp_bwd[NV][2][WPV];
  real warp_xn[NV][2][WPV][2];   // x, z after each warp
  Bwd<real> seg_bwd[NV][2];
  double sm[NV][2][6];           // y_f, z_f, y_l, z_l, -a0/b0 (periodic)
  // mixed form, the line's reference state R (difference form): per
  // variable the hi / lo pair of the median of five sampled cells, R in
  // FP32, the reference fluxes F(R), (u_R, v_R, p_R, E_R + p_R), whether
  // the sampled densities and energies lie within a factor 2 of R (gate)
  float rh[NV], rl[NV], rf[NV], rF[NV], rp[4];
  int rgate[NV];
  float rspread[NV];             // largest |sample - R| per variable (hi parts)
  float epsf;                    // mixed form: the limiter epsilon of this stage
};

// Segment planes in shared memory carry one pad word per 128 bytes: segment
// cell c (c >= -2) sits at pad(c) = c + (c >> PSH) of its plane.  Lanes of a
// warp then hit distinct banks both when each lane walks its own chunk of M
// cells (lane stride M) and when consecutive lanes take consecutive cells;
// a chunk (M divides 128 bytes) never straddles a pad word.
template <typename real, int NV, int M>
struct Smem {
  static constexpr int KC = SEGC / M;     // chunks per conserved variable
  static constexpr int WPV = KC / 32;     // warps per conserved variable
  static constexpr int SEG = SEGC;
  static constexpr int PSH = sizeof(real) == 4 ? 5 : 4;
  __host__ __device__ static constexpr int pad(int c) { return c + (c >> PSH); }
  static constexpr int UH = 3;                         // pad(-2) = -3
  static constexpr int UWP = UH + pad(SEG + 1) + 1;    // cells -2 .. SEG+1
  static constexpr int WP = pad(SEG - 1) + 1;          // cells 0 .. SEG-1
  static_assert(((32 * 4 / (int)sizeof(real)) % M) == 0, "a chunk must not straddle a pad word");
  static constexpr size_t u_off = 0;                                     // real Us[NV][UWP]
  static constexpr size_t w_off = u_off + sizeof(real) * NV * UWP;       // real Wt[NV][4][WP]
  static constexpr size_t fm_off = w_off + sizeof(real) * NV * 4 * WP;
  static constexpr size_t fp_off = fm_off + sizeof(real) * NV * WP;      // real Fm, Fp[NV][WP]
  static constexpr size_t fl_off = fp_off + sizeof(real) * NV * WP;      // real Fl[NV][SEG+2]
  static constexpr size_t rm_off = fl_off + sizeof(real) * NV * (SEG + 2);  // remote stencils
  static constexpr size_t ex_off = (rm_off + sizeof(real) * NV * 2 * 6 + 15) / 16 * 16;
  // mixed form: one byte per cell (its face values stored in full, not as
  // differences from R) and one per face (its flux stored as F - F(R))
  static constexpr size_t cf_off = ex_off + sizeof(Exch<real, NV, WPV>);
  static constexpr size_t ff_off = cf_off + SEG;
  static constexpr size_t bytes = (ff_off + SEG + 2 + 15) / 16 * 16;
};

// line-variable k -> grid variable
__device__ __forceinline__ int gvar(int k, int nv, int vn, int vt) {
  return k == 0 ? 0 : (k == nv - 1 ? nv - 1 : (k == 1 ? vn : vt));
}

__device__ __forceinline__ unsigned long long double_bits(double x) {
  return (unsigned long long)__double_as_longlong(x);
}
__device__ __forceinline__ double bits_double(unsigned long long b) {
  return __longlong_as_double((long long)b);
}

// grid-wide extrema on a few control-block words: every warp of every CTA
// reports, so an atomic whose value cannot change the word is skipped (the
// words only move one way during a launch; a stale read only costs an atomic)
__device__ __forceinline__ void atomic_max_bits(unsigned long long *w, unsigned long long v) {
  if (v > *reinterpret_cast<volatile unsigned long long *>(w)) atomicMax(w, v);
}
__device__ __forceinline__ void atomic_min_bits(unsigned long long *w, unsigned long long v) {
  if (v < *reinterpret_cast<volatile unsigned long long *>(w)) atomicMin(w, v);
}

// ---------------------------------------------------------------- kernel
// Resident CTAs per SM the kernel is compiled for: the mixed form is bound by
// latency, so it asks for three at M = 8 (85 registers a thread; the shared
// memory of three segments fits) and two at M = 16; the FP64 form is bound by
// the FP64 pipe and its shared memory allows one.
#ifndef PPK_MIXED_CTAS_M8
#define PPK_MIXED_CTAS_M8 3
#endif
// PRE: the face values come from another kernel (args.Fm_pre / Fp_pre) and
// the reconstruction phases are compiled out.
template <typename real, int NV, int M, bool PER, int MODE, bool PRE>
__global__ void __launch_bounds__(NV * (SEGC / M),
                                  sizeof(real) == 4 ? (M == 8 ? PPK_MIXED_CTAS_M8 : 2) : 1)
    line_sweep(SweepArgs args_in) {
  constexpr bool MIXED = sizeof(real) == 4;
  using S = Smem<real, NV, M>;
  constexpr int SEG = S::SEG;
  constexpr int KC = S::KC;
  constexpr int WPV = S::WPV;
  constexpr int T = NV * KC;
  constexpr int UW = SEG + 4;            // cells -2 .. SEG+1
  constexpr int UH = S::UH, UWP = S::UWP, WP = S::WP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  real *Us = reinterpret_cast<real *>(smem_raw + S::u_off);
  real *Wt = reinterpret_cast<real *>(smem_raw + S::w_off);
  real *Fm = reinterpret_cast<real *>(smem_raw + S::fm_off);
  real *Fp = reinterpret_cast<real *>(smem_raw + S::fp_off);
  real *Fl = reinterpret_cast<real *>(smem_raw + S::fl_off);
  real *Rm = reinterpret_cast<real *>(smem_raw + S::rm_off);
  Exch<real, NV, WPV> &ex = *reinterpret_cast<Exch<real, NV, WPV> *>(smem_raw + S::ex_off);

  cg::cluster_group cluster = cg::this_cluster();
  SweepArgs args = args_in;
  const int R = args.R;
  const int rank = (int)cluster.block_rank();
  long long line = blockIdx.x / R;
  bind_line<real, NV>(args, line);
  if (args.lines) {   // D buffers follow the state layout of the batch
    const long long o = args.probs[args_in.lines[blockIdx.x / R].prob].off;
    if (args.Din) args.Din = reinterpret_cast<const real *>(args.Din) + o;
    if (args.Dout) args.Dout = reinterpret_cast<real *>(args.Dout) + o;
  }
  const int n = args.n;
  const int lo = rank * SEG;
  const int hi = min(lo + SEG, n);
  const int tid = threadIdx.x;
  const int v = tid / KC;
  const int k = tid % KC;
  const int lane = tid & 31;
  const int w = k >> 5;
  Ctl *ctl = args.ctl;

  // a finished problem skips the launch (uniform over the grid)
  if (args.eps_fixed <= 0.0 && !ctl->active) return;

  const real eps_w = MIXED ? real(args.eps_weno_f) : real(args.eps_weno);
  const real gam = MIXED ? real(args.gamma_f) : real(args.gamma);
  const real wgl = MIXED ? real(args.wgl_f) : real(args.wgl);
  real eps_pos;
  if constexpr (MIXED) {
    // one thread takes the FP64 minimum; the others read it after the
    // load phase's barrier (the limiter comes later)
    if (tid == 0) {
      double e = args.eps_fixed > 0.0 ? args.eps_fixed
                 : (args.stage == 0 ? ctl->eps0
                                    : fmin(ctl->eps_pos, bits_double(ctl->minrho[args.stage - 1])));
      ex.epsf = (float)e;
    }
    eps_pos = real(0);   // set after the barrier
  } else {
    if (args.eps_fixed > 0.0) eps_pos = real(args.eps_fixed);
    else if (args.stage == 0) eps_pos = real(ctl->eps0);
    else eps_pos = real(fmin(ctl->eps_pos, bits_double(ctl->minrho[args.stage - 1])));
  }

  const long long lbase = line * args.line_stride;
  const long long cs = args.cell_stride;
  unsigned char *cfull = smem_raw + S::cf_off;   // mixed: cell's faces stored in full
  unsigned char *fdel = smem_raw + S::ff_off;    // mixed: face flux stored as F - F(R)

  // difference form possible: the reference samples load with the hi parts;
  // the lo parts, and the differences, only for lines that take the form
  const bool two = MIXED && !PRE && args.Ul != nullptr;
  float sh[5], sl[5];
  if constexpr (MIXED && !PRE) {
    if (two && tid < NV) {
      const int g = gvar(tid, NV, args.vn, args.vt);
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        const int i = (int)(((long long)(2 * q + 1) * n) / 10);
        const long long a = g * args.ncell + lbase + (long long)i * cs;
        sh[q] = args.Uh[a];
        sl[q] = args.Ul[a];
      }
    }
  }
  (void)sh; (void)sl;

  // ---------------------------------------------------------------- load
  // line cell i (any i; ghosts by the boundary condition): its address and
  // whether the ghost negates the value (reflective, normal momentum)
  auto cell_addr = [&](int kv, int i, bool &neg) -> long long {
    int g = gvar(kv, NV, args.vn, args.vt);
    neg = false;
    if (i < 0 || i >= n) {
      if (PER) {
        i = (i % n + n) % n;
      } else {
        int bc = i < 0 ? args.bclo : args.bchi;
        if (bc == 1) {
          i = i < 0 ? 0 : n - 1;
        } else {  // reflective mirror
          i = i < 0 ? -i - 1 : 2 * n - 1 - i;
          neg = kv == 1;
        }
      }
    }
    return g * args.ncell + lbase + (long long)i * cs;
  };
  auto cell_val = [&](int kv, int i) -> real {
    bool neg;
    const long long a = cell_addr(kv, i, neg);
    real x;
    if constexpr (MIXED) x = args.Uh[a];
    else x = args.U[a];
    return neg ? -x : x;
  };

  bool vec = false;
  int nq = 0;
  if constexpr (MIXED) {
    // contiguous line with 16-byte aligned segments: the segment's cells
    // come in as float4, only the halo and a ragged tail cell by cell
    vec = cs == 1 && !args.lines && ((lbase + lo) & 3) == 0 && (args.ncell & 3) == 0 &&
          ((reinterpret_cast<unsigned long long>(args.Uh) & 15) == 0);
    if (vec) {
      nq = (hi - lo) >> 2;
      for (int idx = tid; idx < NV * nq; idx += T) {
        int kv = idx / nq, q = idx - kv * nq;
        int g = gvar(kv, NV, args.vn, args.vt);
        const float4 x = *reinterpret_cast<const float4 *>(args.Uh + g * args.ncell + lbase + lo + 4 * q);
        real *d = Us + kv * UWP + UH + S::pad(4 * q);
        d[0] = x.x; d[1] = x.y; d[2] = x.z; d[3] = x.w;
      }
      const int nr = UW - 4 * nq;
      for (int idx = tid; idx < NV * nr; idx += T) {
        int kv = idx / nr, r = idx - kv * nr;
        int j = r < 2 ? r : 4 * nq + r;
        int i = lo - 2 + j;
        Us[kv * UWP + UH + S::pad(j - 2)] = (i < hi + 2) ? cell_val(kv, i) : real(0);
      }
    }
  }
  if (!vec) {
    for (int idx = tid; idx < NV * UW; idx += T) {
      int kv = idx / UW, j = idx % UW;
      int i = lo - 2 + j;
      Us[kv * UWP + UH + S::pad(j - 2)] = (i < hi + 2) ? cell_val(kv, i) : real(0);
    }
  }
  if (PER) {
    // stencils of the two "position 0" cells (minus: cell 0, plus: cell n-1)
    // for the Sherman-Morrison row at the far end of each system
    for (int idx = tid; idx < NV * 2 * 5; idx += T) {
      int kv = idx / 10, s = (idx / 5) % 2, j = idx % 5;
      int c0 = s == 0 ? 0 : n - 1;
      Rm[(kv * 2 + s) * 6 + j] = cell_val(kv, c0 - 2 + j);
    }
  }

  // ------------------------------------------------ reference state (mixed)
  // The mixed form reconstructs the differences ubar - R from a reference
  // state R of the line (shift invariance of eq. (CWENO-FV): every row's
  // coefficients and right-hand side weights sum to one, the indicators of
  // eq. (weight) see differences only) and evaluates the fluxes as F - F(R)
  // where the face states lie near R, so that FP32 rounding is relative to
  // |U - R| rather than |U|.  R: per variable the median of five sampled
  // cells (hi parts), the same in every CTA of the line.  The plain FP32 form
  // on the hi parts (R = 0) stays where the difference form cannot help:
  // lines whose sampled densities or energies spread beyond a factor 4 of R
  // (strong jumps, vacuum), and lines flat to FP32 precision (every
  // variable's samples within 2^-20 of its scale: R's magnitude, for the
  // momenta at least sqrt(rho_R E_R)).  A face whose states are farther than
  // half of R's density or energy from R is evaluated in full.  The
  // characteristic-wise path (PRE) takes its face values from outside and
  // keeps R = 0.  All in FP32: FP64 instructions here would cost each CTA
  // thousands of cycles on GB300's FP64 pipe while its other warps wait.
  bool dlt = false;
  if constexpr (MIXED && !PRE) {
    if (two && tid < NV) {
      const int kv = tid;
      // the median of the hi parts by rank (ties by index), picked by
      // unrolled selects (no run-time indexing of the arrays)
      float mh = 0.0f, ml = 0.0f;
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        int below = 0;
#pragma unroll
        for (int r = 0; r < 5; ++r) below += (sh[r] < sh[q]) || (sh[r] == sh[q] && r < q);
        if (below == 2) { mh = sh[q]; ml = sl[q]; }
      }
      bool gate = true;
      float spread = 0.0f;
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        if (kv == 0 || kv == NV - 1) gate = gate && sh[q] >= 0.25f * mh && sh[q] <= 4.0f * mh;
        spread = fmaxf(spread, fabsf(sh[q] - mh));
      }
      if (kv == 0 || kv == NV - 1) gate = gate && mh > 0.0f;
      ex.rh[kv] = mh;
      ex.rl[kv] = ml;
      ex.rf[kv] = mh + ml;
      ex.rgate[kv] = gate ? 1 : 0;
      ex.rspread[kv] = spread;
    }
  }
  __syncthreads();
  if constexpr (MIXED) eps_pos = ex.epsf;
  if constexpr (MIXED && !PRE) {
    if (two) {
      const float mom = sqrtf(fabsf(ex.rf[0] * ex.rf[NV - 1]));
      bool flat = true;
#pragma unroll
      for (int kv = 0; kv < NV; ++kv) {
        const float scale = (kv == 0 || kv == NV - 1) ? fabsf(ex.rf[kv]) : fmaxf(fabsf(ex.rf[kv]), mom);
        flat = flat && ex.rspread[kv] <= 9.5367432e-07f * scale;   // 2^-20
      }
      dlt = ex.rgate[0] && ex.rgate[NV - 1] && !flat;
    }
    if (dlt && tid == 0) {
      // F(R) and (u_R, v_R, p_R, E_R + p_R), FP32 (O(1) factors of the
      // difference terms; F(R) only meets fluxes of full-form faces)
      const float r0 = ex.rf[0], m = ex.rf[1], t = NV == 4 ? ex.rf[2] : 0.0f;
      const float E = ex.rf[NV - 1];
      const float ir = 1.0f / r0;
      const float u = m * ir, vv = t * ir;
      const float pr = (args.gamma_f - 1.0f) * (E - 0.5f * (m * u + t * vv));
      ex.rF[0] = m;
      ex.rF[1] = m * u + pr;
      if (NV == 4) ex.rF[2] = t * u;
      ex.rF[NV - 1] = (E + pr) * u;
      ex.rp[0] = u;
      ex.rp[1] = vv;
      ex.rp[2] = pr;
      ex.rp[3] = E + pr;
    }
    if (dlt) {
      // (hi - R_hi) + (lo - R_lo), exact where hi and R_hi are within a
      // factor of two of each other: each thread brings in the lo parts of
      // the cells it loaded (the same loops) and replaces their hi parts
      auto conv = [&](int kv, int slot, float l) {
        Us[slot] = (Us[slot] - ex.rh[kv]) + (l - ex.rl[kv]);
      };
      auto conv_cell = [&](int kv, int j) {
        const int i = lo - 2 + j;
        if (i >= hi + 2) return;
        bool neg;
        const long long a = cell_addr(kv, i, neg);
        const float l = args.Ul[a];
        conv(kv, kv * UWP + UH + S::pad(j - 2), neg ? -l : l);
      };
      if (vec) {
        for (int idx = tid; idx < NV * nq; idx += T) {
          const int kv = idx / nq, q = idx - kv * nq;
          const int g = gvar(kv, NV, args.vn, args.vt);
          const float4 y = *reinterpret_cast<const float4 *>(args.Ul + g * args.ncell + lbase + lo + 4 * q);
          const int b = kv * UWP + UH + S::pad(4 * q);
          conv(kv, b, y.x); conv(kv, b + 1, y.y); conv(kv, b + 2, y.z); conv(kv, b + 3, y.w);
        }
        const int nr = UW - 4 * nq;
        for (int idx = tid; idx < NV * nr; idx += T) {
          const int kv = idx / nr, r = idx - kv * nr;
          conv_cell(kv, r < 2 ? r : 4 * nq + r);
        }
      } else {
        for (int idx = tid; idx < NV * UW; idx += T) conv_cell(idx / UW, idx % UW);
      }
      if (PER) {
        for (int idx = tid; idx < NV * 2 * 5; idx += T) {
          const int kv = idx / 10, s = (idx / 5) % 2, j = idx % 5;
          bool neg;
          const long long a = cell_addr(kv, (s == 0 ? 0 : n - 1) - 2 + j, neg);
          const float l = args.Ul[a];
          const int o = (kv * 2 + s) * 6 + j;
          Rm[o] = (Rm[o] - ex.rh[kv]) + ((neg ? -l : l) - ex.rl[kv]);
        }
      }
      __syncthreads();
    }
  }
  (void)dlt;
  // epsilon of eq. (weight) for this thread's variable v.  The difference
  // form's indicators see U - R, but the rounding noise the FP32 stages
  // leave in the state scales with |U| wherever a line or a face took the
  // plain form; the floor therefore keeps the reference's share,
  // 2^20 u^2 (R^2 + max|U - R|^2) >= 2^19 u^2 max|U|^2 over the stencil
  real eps_v = eps_w;
  if constexpr (MIXED) {
    if (dlt) eps_v = eps_w + FP32_BETA_FLOOR * ex.rf[v] * ex.rf[v];
  }


  // face values computed outside (the characteristic-wise reconstruction):
  // U^- and U^+ of the segment's cells in the state's layout
  if constexpr (PRE) {
    const real *pm = reinterpret_cast<const real *>(args.Fm_pre);
    const real *pp = reinterpret_cast<const real *>(args.Fp_pre);
    for (int idx = tid; idx < NV * (hi - lo); idx += T) {
      const int kv = idx / (hi - lo), c = idx - kv * (hi - lo);
      const long long o = gvar(kv, NV, args.vn, args.vt) * args.ncell + lbase + (long long)(lo + c) * cs;
      Fm[kv * WP + S::pad(c)] = pm[o];
      Fp[kv * WP + S::pad(c)] = pp[o];
    }
  } else {
    // ---------------------------------------------------------------- rows
    const real *uv = Us + v * UWP + UH;         // u of segment cell c at uv[pad(c)], c in [-2, SEG+2)
    real *wt = Wt + v * 4 * WP;                 // wt[q*WP + pad(c)]: w0-, w2-, w0+, w2+
    const int s0 = lo + k * M;                  // first cell of this thread's chunk
    const int len = max(0, min(M, hi - s0));
    const int cb = S::pad(k * M);               // padded offset of the chunk's first cell
    const bool bounded = !PER;
    auto u_at = [&](int i) -> real { return uv[S::pad(i - lo)]; };

    // the chunk's cells with a two-cell halo, from shared memory into registers
    auto load_window = [&](real *win) {
      win[0] = uv[S::pad(k * M - 2)];
      win[1] = uv[S::pad(k * M - 1)];
  #pragma unroll
      for (int q = 0; q < M; ++q) win[q + 2] = uv[cb + q];
      win[M + 2] = uv[S::pad(k * M + M)];
      win[M + 3] = uv[S::pad(k * M + M + 1)];
    };

    // a, b of the unmodified position-0 row of side 0 (cell 0) or 1 (cell n-1),
    // needed by the Sherman-Morrison row at the far end of a periodic system
    auto far_row = [&](int side, real &a0, real &b0) {
      const real *y = Rm + (v * 2 + side) * 6 + 2;
      real q0, q1, q2, one, w0, w1, w2;
      zratios_any(y[-2], y[-1], y[0], y[1], y[2], eps_v, q0, q1, q2, one);
      if (side == 0) zweights(real(0.2), real(0.5), real(0.3), q0, q1, q2, w0, w1, w2, one);
      else zweights(real(0.2), real(0.5), real(0.3), q2, q1, q0, w0, w1, w2, one);
      Row<real> r = compact_row02(w0, w2, real(0), real(0), real(0));
      a0 = r.a;
      b0 = r.b;
    };

    // row of the periodic end cell i (0 or n-1), side 0 (minus) or 1 (plus),
    // from the stored weights; zr = the Sherman-Morrison right-hand side entry
    auto per_row = [&](int i, int side, real &zr) -> Row<real> {
      const real *o = wt + 2 * side * WP + S::pad(i - lo);
      const real xm = u_at(i - 1), x0 = u_at(i), xp = u_at(i + 1);
      Row<real> r = side == 0 ? compact_row02(o[0], o[WP], xm, x0, xp)
                              : compact_row02(o[0], o[WP], xp, x0, xm);
      const int first = side == 0 ? 0 : n - 1, last = side == 0 ? n - 1 : 0;
      zr = real(0);
      if (i == first) {          // T = A - u v^T with g = -b at position 0
        zr = -r.b;
        r.b = r.b + r.b;
        r.a = real(0);
      } else if (i == last) {    // corner removed, b reduced by c a0 / g
        real a0, b0;
        far_row(side, a0, b0);
        zr = r.c;
        r.b = r.b + r.c * a0 / b0;
        r.c = real(0);
      }
      return r;
    };

    // ------------------------------------------- weights + chunk maps (F1)
    // weights are stored for the elimination pass (F5); the rows come from the
    // register window.  The bounded closure cells store their explicit
    // WENO5-Z face values in the w0 slots instead (rows 0 x + 1 x + 0 x = f).
    Fwd<real> fm = fwd_identity<real>(), fp = fwd_identity<real>();
    {
      real win[M + 4];
      load_window(win);
  #pragma unroll
      for (int j = 0; j < M; ++j) {
        if (j < len) {
          const int i = s0 + j;
          real zm = real(0), zp = real(0);
          Row<real> rm, rp;
          if (bounded && (i == 0 || i == n - 1)) {
            real fmv = weno5z_face(win[j], win[j + 1], win[j + 2], win[j + 3], win[j + 4], eps_v);
            real fpv = weno5z_face(win[j + 4], win[j + 3], win[j + 2], win[j + 1], win[j], eps_v);
            wt[cb + j] = fmv;
            wt[2 * WP + cb + j] = fpv;
            rm.a = real(0); rm.b = real(1); rm.c = real(0); rm.r = fmv;
            rp.a = real(0); rp.b = real(1); rp.c = real(0); rp.r = fpv;
          } else {
            real w0, w2, v0, v2;
            if constexpr (MIXED) {
              real q0, q1, q2, one;
              zratios_any(win[j], win[j + 1], win[j + 2], win[j + 3], win[j + 4], eps_v, q0, q1, q2,
                          one);
              zweights_pair(q0, q1, q2, one, w0, w2, v0, v2);
            } else {
              zweights_both_fp64(win[j], win[j + 1], win[j + 2], win[j + 3], win[j + 4], eps_v, w0,
                                 w2, v0, v2);
            }
            wt[cb + j] = w0;
            wt[WP + cb + j] = w2;
            wt[2 * WP + cb + j] = v0;
            wt[3 * WP + cb + j] = v2;
            if (PER && (i == 0 || i == n - 1)) {
              rm = per_row(i, 0, zm);
              rp = per_row(i, 1, zp);
            } else {
              rm = compact_row02(w0, w2, win[j + 1], win[j + 2], win[j + 3]);
              rp = compact_row02(v0, v2, win[j + 3], win[j + 2], win[j + 1]);
            }
          }
          fwd_push_left<real, PER>(fm, rm, zm);
          fwd_push_right<real, PER>(fp, rp, zp);
        }
      }
    }
    fwd_normalise(fm);
    fwd_normalise(fp);

    // ------------------------------------------- warp inclusive scans (F2)
    // minus maps accumulate from the lower lanes, plus maps from the higher
    if constexpr (MIXED) {
      Fwd2 f2 = fwd2_pack(fm, fp);
      const float2 one2 = p_set(1.0f), zero2 = p_set(0.0f);
  #pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const bool am = lane >= d, ap = lane + d < 32;
        Fwd2 o;
        // every lane executes both shuffles; the select comes after
  #define PPK_SH2(fld, idv)                                                    \
    {                                                                          \
      const float tm_ = __shfl_up_sync(0xffffffffu, f2.fld.x, d);              \
      const float tp_ = __shfl_down_sync(0xffffffffu, f2.fld.y, d);            \
      o.fld.x = am ? tm_ : idv.x;                                              \
      o.fld.y = ap ? tp_ : idv.y;                                              \
    }
        PPK_SH2(g00, one2); PPK_SH2(g01, zero2); PPK_SH2(g10, zero2); PPK_SH2(g11, one2);
        PPK_SH2(dP, zero2); PPK_SH2(dQ, zero2); PPK_SH2(mu, one2);
        if (PER) { PPK_SH2(zP, zero2); PPK_SH2(zQ, zero2); } else { o.zP = zero2; o.zQ = zero2; }
  #undef PPK_SH2
        f2 = fwd2_compose<PER>(f2, o);   // with the identity where a lane has no partner
        fwd2_normalise(f2);
      }
      fwd2_unpack(f2, fm, fp);
    } else {
  #pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        Fwd<real> o = fwd_shfl<real, PER, true>(fm, d);
        if (lane >= d) { fm = fwd_compose<real, PER>(fm, o); fwd_normalise(fm); }
        Fwd<real> q = fwd_shfl<real, PER, false>(fp, d);
        if (lane + d < 32) { fp = fwd_compose<real, PER>(fp, q); fwd_normalise(fp); }
      }
    }
    if (lane == 31) ex.warp_fwd[v][0][w] = fm;
    if (lane == 0) ex.warp_fwd[v][1][w] = fp;
    __syncthreads();

    // ------------------------------------------- CTA segment maps (F3)
    if (tid < 2 * NV) {
      int vv = tid >> 1, sd = tid & 1;
      Fwd<real> sg = fwd_identity<real>();
      for (int ww = 0; ww < WPV; ++ww) {
        int wi = sd == 0 ? ww : WPV - 1 - ww;
        sg = fwd_compose<real, PER>(ex.warp_fwd[vv][sd][wi], sg);
        fwd_normalise(sg);
      }
      ex.seg_fwd[vv][sd] = sg;
    }
    cluster.sync();

    // ------------------------------------------- incoming states (F4)
    // The segment maps of the CTAs ahead of this one on each side (minus: the
    // lower ranks, applied in rank order; plus: the higher ranks, from the
    // last one down) applied to the zero state that enters a line end.
    // Mixed form (latency bound): composed by a tree over 16 lanes, lane q
    // holding rank q's map (the identity where rank q is not ahead), so the
    // remote reads happen at once.  FP64 form (bound by the FP64 pipe): one
    // thread per side and variable applies them in turn, the fewest FP64
    // operations.
    real cin = real(0), din = real(0), zin = real(0);
    int fvv = -1, fsd = 0;
    if constexpr (MIXED) {
      if (tid < 2 * NV * 16) {   // whole warps: T >= 2 NV 16 for M <= 16
        const int grp = tid >> 4, q = tid & 15;
        const int vv = grp >> 1, sd = grp & 1;
        Fwd<real> mq = fwd_identity<real>();
        if (q < R && (sd == 0 ? q < rank : q > rank)) {
          Exch<real, NV, WPV> *rx = cluster.map_shared_rank(&ex, q);
          mq = rx->seg_fwd[vv][sd];
        }
  #pragma unroll
        for (int d = 1; d < 16; d <<= 1) {
          Fwd<real> o = fwd_shfl<real, PER, false>(mq, d, 16);   // ranks q + d ...
          if ((q & (2 * d - 1)) == 0) {
            mq = sd == 0 ? fwd_compose<real, PER>(o, mq) : fwd_compose<real, PER>(mq, o);
            fwd_normalise(mq);
          }
        }
        if (q == 0) {
          fwd_apply<real, PER>(mq, cin, din, zin);
          fvv = vv;
          fsd = sd;
        }
      }
    } else {
      if (tid < 2 * NV) {
        const int vv = tid >> 1, sd = tid & 1;
        if (sd == 0) {
          for (int q = 0; q < rank; ++q) {
            Exch<real, NV, WPV> *rx = cluster.map_shared_rank(&ex, q);
            fwd_apply<real, PER>(rx->seg_fwd[vv][0], cin, din, zin);
          }
        } else {
          for (int q = R - 1; q > rank; --q) {
            Exch<real, NV, WPV> *rx = cluster.map_shared_rank(&ex, q);
            fwd_apply<real, PER>(rx->seg_fwd[vv][1], cin, din, zin);
          }
        }
        fvv = vv;
        fsd = sd;
      }
    }
    if (fvv >= 0) {   // the state entering each warp of this segment
      for (int ww = 0; ww < WPV; ++ww) {
        int wi = fsd == 0 ? ww : WPV - 1 - ww;
        ex.warp_in[fvv][fsd][wi][0] = cin;
        ex.warp_in[fvv][fsd][wi][1] = din;
        ex.warp_in[fvv][fsd][wi][2] = zin;
        fwd_apply<real, PER>(ex.warp_fwd[fvv][fsd][wi], cin, din, zin);
      }
    }
    __syncthreads();

    // the state after each lane's chunk (its inclusive map applied to the
    // warp's incoming state), handed to the next lane in elimination order
    real cpm, dpm, zpm, cpp, dpp, zpp;
    {
      const real cw = ex.warp_in[v][0][w][0], dw = ex.warp_in[v][0][w][1], zw = ex.warp_in[v][0][w][2];
      real c = cw, d = dw, z = zw;
      fwd_apply<real, PER>(fm, c, d, z);
      cpm = shfl_up_r(c, 1);
      dpm = shfl_up_r(d, 1);
      zpm = PER ? shfl_up_r(z, 1) : real(0);
      if (lane == 0) { cpm = cw; dpm = dw; zpm = zw; }
    }
    {
      const real cw = ex.warp_in[v][1][w][0], dw = ex.warp_in[v][1][w][1], zw = ex.warp_in[v][1][w][2];
      real c = cw, d = dw, z = zw;
      fwd_apply<real, PER>(fp, c, d, z);
      cpp = shfl_down_r(c, 1);
      dpp = shfl_down_r(d, 1);
      zpp = PER ? shfl_down_r(z, 1) : real(0);
      if (lane == 31) { cpp = cw; dpp = dw; zpp = zw; }
    }

    // ------------------------------------------- chunk elimination (F5)
    // Thomas elimination of the chunk from the incoming state, and the chunk's
    // back-substitution map x_first = A + B x_after accumulated in the same
    // pass: A = sum_j (prod_{l<j} -c'_l) d'_j, B = prod_l -c'_l.  The minus
    // system runs over the chunk's cells left to right, the plus system right
    // to left.  c', d' of a cell overwrite its two weights (read just before by
    // the same thread); z' stays in registers (periodic lines).
    // Mixed form: the recurrence runs on the projective state (P, Q, D, Z),
    // c' = P/Q, d' = D/Q, z' = Z/Q, mapped linearly by a row (P <- c Q,
    // Q <- b Q - a P, D <- r Q - a D), so consecutive rows depend on each other
    // through two multiply-adds and the reciprocals 1/Q are off that chain
    // (over one chunk Q changes by at most M factors b - a c': no rescaling).
    // FP64 form: the plain recurrence with one division per row, the fewest
    // FP64 operations.
    real zmv[PER ? M : 1], zpv[PER ? M : 1];
    Bwd<real> bm, bp;
    // a full chunk without a line-end cell: every row is a plain compact row
    const bool plain = len == M && s0 > 0 && s0 + M < n;
    bool done5 = false;
    if constexpr (MIXED) {
      if (plain) {   // both systems together in paired FP32, no guards
        float win[M + 4];
        load_window(win);
        float *om = wt + cb, *op = wt + 2 * WP + cb;
        float2 P = make_float2(cpm, cpp), Q = p_set(1.0f), D = make_float2(dpm, dpp);
        float2 Z = make_float2(zpm, zpp);
        float2 pi = p_set(1.0f), A = p_set(0.0f), Az = p_set(0.0f);
  #pragma unroll
        for (int jj = 0; jj < M; ++jj) {
          const int jm = jj, jp = M - 1 - jj;    // minus left to right, plus right to left
          float2 a, b, c, r;
          row2(make_float2(om[jm], op[jp]), make_float2(om[WP + jm], op[WP + jp]),
               make_float2(win[jm + 1], win[jp + 3]), make_float2(win[jm + 2], win[jp + 2]),
               make_float2(win[jm + 3], win[jp + 1]), a, b, c, r);
          const float2 na = p_neg(a);
          const float2 nq = p_fma(na, P, p_mul(b, Q));
          D = p_fma(na, D, p_mul(r, Q));
          if (PER) Z = p_mul(na, Z);            // zero right-hand side away from the ends
          P = p_mul(c, Q);
          Q = nq;
          const float2 iq = make_float2(1.0f / Q.x, 1.0f / Q.y);
          const float2 co = p_mul(P, iq), dd = p_mul(D, iq);
          om[jm] = co.x;
          om[WP + jm] = dd.x;
          op[jp] = co.y;
          op[WP + jp] = dd.y;
          A = p_fma(pi, dd, A);
          if (PER) {
            const float2 zz = p_mul(Z, iq);
            zmv[jm] = zz.x;
            zpv[jp] = zz.y;
            Az = p_fma(pi, zz, Az);
          }
          pi = p_mul(pi, p_neg(co));
        }
        bm.A = A.x; bm.Az = Az.x; bm.B = pi.x;
        bp.A = A.y; bp.Az = Az.y; bp.B = pi.y;
        done5 = true;
      }
    }
    if (!done5) {
      real win[M + 4];
      load_window(win);
      // projective state (mixed) or (c', -, d', z') (FP64) of each side
      real Pm = cpm, Qm = real(1), Dm = dpm, Zm = zpm;
      real Pp = cpp, Qp = real(1), Dp = dpp, Zp = zpp;
      real pim = real(1), Am = real(0), Azm = real(0);
      real pip = real(1), Ap = real(0), Azp = real(0);
      (void)Qm; (void)Qp;   // the FP64 chains carry no Q
      auto elim = [&](const Row<real> &r, real zr, real &P, real &Qs, real &D, real &Z,
                      real &co, real &dout, real &zo) {
        if constexpr (MIXED) {
          real nq = r.b * Qs - r.a * P;
          D = r.r * Qs - r.a * D;
          if (PER) Z = zr * Qs - r.a * Z;
          P = r.c * Qs;
          Qs = nq;
          real iq = real(1) / Qs;
          co = P * iq;
          dout = D * iq;
          zo = PER ? Z * iq : real(0);
        }
      };
      // the row of cell s0 + j of side sd (0 minus, 1 plus) and its z entry
      auto row_of = [&](int sd, int j, real &zr) -> Row<real> {
        const int i = s0 + j;
        const real *o = wt + 2 * sd * WP + cb + j;
        Row<real> r;
        zr = real(0);
        if (bounded && (i == 0 || i == n - 1)) {
          r.a = real(0); r.b = real(1); r.c = real(0); r.r = o[0];
        } else if (PER && (i == 0 || i == n - 1)) {
          r = per_row(i, sd, zr);
        } else if (sd == 0) {
          r = compact_row02(o[0], o[WP], win[j + 1], win[j + 2], win[j + 3]);
        } else {
          r = compact_row02(o[0], o[WP], win[j + 3], win[j + 2], win[j + 1]);
        }
        return r;
      };
      // c', d' (and z') of a row stored over its weights; the back map grows
      auto finish = [&](int sd, int j, real co, real dd, real zz) {
        real *o = wt + 2 * sd * WP + cb + j;
        o[0] = co;
        o[WP] = dd;
        if (sd == 0) {
          if (PER) zmv[j] = zz;
          Am += pim * dd;
          if (PER) Azm += pim * zz;
          pim *= -co;
        } else {
          if (PER) zpv[j] = zz;
          Ap += pip * dd;
          if (PER) Azp += pip * zz;
          pip *= -co;
        }
      };
  #pragma unroll
      for (int jj = 0; jj < M; ++jj) {
        const int jm = jj, jp = M - 1 - jj;    // minus left to right, plus right to left
        const bool am = jm < len, ap = jp < len;
        if constexpr (MIXED) {
          if (am) {
            real zr, co, dd, zz;
            const Row<real> r = row_of(0, jm, zr);
            elim(r, zr, Pm, Qm, Dm, Zm, co, dd, zz);
            finish(0, jm, co, dd, zz);
          }
          if (ap) {
            real zr, co, dd, zz;
            const Row<real> r = row_of(1, jp, zr);
            elim(r, zr, Pp, Qp, Dp, Zp, co, dd, zz);
            finish(1, jp, co, dd, zz);
          }
        } else {
          // FP64: one division for the pivots of both chains,
          // 1/(q_m q_p) times q_p and q_m
          real zrm = real(0), zrp = real(0);
          Row<real> rm, rp;
          rm.a = rm.c = rm.r = rp.a = rp.c = rp.r = real(0);
          rm.b = rp.b = real(1);
          if (am) rm = row_of(0, jm, zrm);
          if (ap) rp = row_of(1, jp, zrp);
          const real qm = am ? rm.b - rm.a * Pm : real(1);
          const real qp = ap ? rp.b - rp.a * Pp : real(1);
          const real inv = real(1) / (qm * qp);
          if (am) {
            const real ip = qp * inv;
            Dm = (rm.r - rm.a * Dm) * ip;
            if (PER) Zm = (zrm - rm.a * Zm) * ip;
            Pm = rm.c * ip;
            finish(0, jm, Pm, Dm, Zm);
          }
          if (ap) {
            const real ip = qm * inv;
            Dp = (rp.r - rp.a * Dp) * ip;
            if (PER) Zp = (zrp - rp.a * Zp) * ip;
            Pp = rp.c * ip;
            finish(1, jp, Pp, Dp, Zp);
          }
        }
      }
      bm.A = Am; bm.Az = Azm; bm.B = pim;
      bp.A = Ap; bp.Az = Azp; bp.B = pip;
    }

    // ------------------------------------------- backward scans (F6)
    // minus back maps accumulate from the higher lanes (its back substitution
    // runs right to left), plus maps from the lower lanes
    Bwd<real> bm_in = bm, bp_in = bp;
    if constexpr (MIXED) {
      Bwd2 b2;
      b2.A = make_float2(bm.A, bp.A);
      b2.B = make_float2(bm.B, bp.B);
      b2.Az = make_float2(bm.Az, bp.Az);
  #pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const bool am = lane + d < 32, ap = lane >= d;
        Bwd2 o;
        {
          float tm = __shfl_down_sync(0xffffffffu, b2.A.x, d), tp = __shfl_up_sync(0xffffffffu, b2.A.y, d);
          o.A = make_float2(am ? tm : 0.0f, ap ? tp : 0.0f);
        }
        {
          float tm = __shfl_down_sync(0xffffffffu, b2.B.x, d), tp = __shfl_up_sync(0xffffffffu, b2.B.y, d);
          o.B = make_float2(am ? tm : 1.0f, ap ? tp : 1.0f);
        }
        if (PER) {
          float tm = __shfl_down_sync(0xffffffffu, b2.Az.x, d), tp = __shfl_up_sync(0xffffffffu, b2.Az.y, d);
          o.Az = make_float2(am ? tm : 0.0f, ap ? tp : 0.0f);
        } else {
          o.Az = p_set(0.0f);
        }
        b2 = bwd2_compose(b2, o);   // with the identity where a lane has no partner
      }
      bm_in.A = b2.A.x; bm_in.B = b2.B.x; bm_in.Az = b2.Az.x;
      bp_in.A = b2.A.y; bp_in.B = b2.B.y; bp_in.Az = b2.Az.y;
    } else {
  #pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        Bwd<real> o;
        o.A = shfl_down_r(bm_in.A, d); o.B = shfl_down_r(bm_in.B, d);
        o.Az = PER ? shfl_down_r(bm_in.Az, d) : real(0);
        if (lane + d < 32) bm_in = bwd_compose(bm_in, o);
        Bwd<real> q;
        q.A = shfl_up_r(bp_in.A, d); q.B = shfl_up_r(bp_in.B, d);
        q.Az = PER ? shfl_up_r(bp_in.Az, d) : real(0);
        if (lane >= d) bp_in = bwd_compose(bp_in, q);
      }
    }
    if (lane == 0) ex.warp_bwd[v][0][w] = bm_in;
    if (lane == 31) ex.warp_bwd[v][1][w] = bp_in;
    __syncthreads();

    // ------------------------------------------- segment back maps (F7)
    if (tid < 2 * NV) {
      int vv = tid >> 1, sd = tid & 1;
      Bwd<real> sg;
      sg.A = real(0); sg.B = real(1); sg.Az = real(0);
      // minus: first cell of the segment = warp 0 o warp 1 o ...; plus: the
      // last warp's map is applied first
      for (int ww = WPV - 1; ww >= 0; --ww) {
        int wi = sd == 0 ? ww : WPV - 1 - ww;
        sg = bwd_compose(ex.warp_bwd[vv][sd][wi], sg);
      }
      ex.seg_bwd[vv][sd] = sg;
    }
    cluster.sync();
    // back substitution entering this segment from the far side: the back maps
    // of the CTAs behind it in that order (minus: the higher ranks, the last
    // acting first; plus: the lower ranks, rank 0 acting first); x = 0 after
    // the line end.  Mixed form: a tree over 16 lanes as in F4; FP64 form: one
    // thread per side and variable.
    {
      real xb = real(0), zb = real(0);
      int bvv = -1, bsd = 0;
      if constexpr (MIXED) {
        if (tid < 2 * NV * 16) {
          const int grp = tid >> 4, q = tid & 15;
          const int vv = grp >> 1, sd = grp & 1;
          Bwd<real> bq;
          bq.A = real(0); bq.B = real(1); bq.Az = real(0);
          if (q < R && (sd == 0 ? q > rank : q < rank)) {
            Exch<real, NV, WPV> *rx = cluster.map_shared_rank(&ex, q);
            bq = rx->seg_bwd[vv][sd];
          }
  #pragma unroll
          for (int d = 1; d < 16; d <<= 1) {
            Bwd<real> o;
            o.A = shfl_down_r(bq.A, d, 16);
            o.B = shfl_down_r(bq.B, d, 16);
            o.Az = PER ? shfl_down_r(bq.Az, d, 16) : real(0);
            if ((q & (2 * d - 1)) == 0) bq = sd == 0 ? bwd_compose(bq, o) : bwd_compose(o, bq);
          }
          if (q == 0) {
            xb = bq.A;
            zb = bq.Az;
            bvv = vv;
            bsd = sd;
          }
        }
      } else {
        if (tid < 2 * NV) {
          const int vv = tid >> 1, sd = tid & 1;
          if (sd == 0) {
            for (int q = R - 1; q > rank; --q) {
              Exch<real, NV, WPV> *rx = cluster.map_shared_rank(&ex, q);
              Bwd<real> b = rx->seg_bwd[vv][0];
              xb = b.A + b.B * xb;
              zb = b.Az + b.B * zb;
            }
          } else {
            for (int q = 0; q < rank; ++q) {
              Exch<real, NV, WPV> *rx = cluster.map_shared_rank(&ex, q);
              Bwd<real> b = rx->seg_bwd[vv][1];
              xb = b.A + b.B * xb;
              zb = b.Az + b.B * zb;
            }
          }
          bvv = vv;
          bsd = sd;
        }
      }
      if (bvv >= 0) {
        for (int ww = 0; ww < WPV; ++ww) {
          int wi = bsd == 0 ? WPV - 1 - ww : ww;
          ex.warp_xn[bvv][bsd][wi][0] = xb;
          ex.warp_xn[bvv][bsd][wi][1] = zb;
          Bwd<real> b = ex.warp_bwd[bvv][bsd][wi];
          xb = b.A + b.B * xb;
          zb = b.Az + b.B * zb;
        }
      }
    }
    __syncthreads();

    // ------------------------------------------- back substitution (F8)
    // minus from the chunk's last cell down, plus from its first cell up; c', d'
    // come from the weight slots, the solution goes to Fm / Fp.  The value
    // entering a chunk is the value leaving the neighbouring lane's chunk (its
    // inclusive back map applied to the warp's entering value).
    real xm, zm_, xp, zp_;
    {
      const real xn = ex.warp_xn[v][0][w][0], zn = ex.warp_xn[v][0][w][1];
      const real xo = bm_in.A + bm_in.B * xn, zo = bm_in.Az + bm_in.B * zn;
      xm = shfl_down_r(xo, 1);
      zm_ = PER ? shfl_down_r(zo, 1) : real(0);
      if (lane == 31) { xm = xn; zm_ = zn; }
    }
    {
      const real xn = ex.warp_xn[v][1][w][0], zn = ex.warp_xn[v][1][w][1];
      const real xo = bp_in.A + bp_in.B * xn, zo = bp_in.Az + bp_in.B * zn;
      xp = shfl_up_r(xo, 1);
      zp_ = PER ? shfl_up_r(zo, 1) : real(0);
      if (lane == 0) { xp = xn; zp_ = zn; }
    }
    real zmo[PER ? M : 1], zpo[PER ? M : 1];
    bool done8 = false;
    if constexpr (MIXED) {
      if (plain) {   // both systems together, no guards
        const float *om = wt + cb, *op = wt + 2 * WP + cb;
        float *dm = Fm + v * WP + cb, *dp = Fp + v * WP + cb;
        float2 x2 = make_float2(xm, xp), z2 = make_float2(zm_, zp_);
  #pragma unroll
        for (int jj = 0; jj < M; ++jj) {
          const int jm = M - 1 - jj, jp = jj;
          const float2 nc = make_float2(-om[jm], -op[jp]);
          x2 = p_fma(nc, x2, make_float2(om[WP + jm], op[WP + jp]));
          dm[jm] = x2.x;
          dp[jp] = x2.y;
          if (PER) {
            z2 = p_fma(nc, z2, make_float2(zmv[jm], zpv[jp]));
            zmo[jm] = z2.x;
            zpo[jp] = z2.y;
          }
        }
        done8 = true;
      }
    }
    if (!done8) {
      {
        const real *o = wt + cb;
        real *dst = Fm + v * WP + cb;
        real x = xm, z = zm_;
  #pragma unroll
        for (int jj = 0; jj < M; ++jj) {
          const int j = M - 1 - jj;
          if (j < len) {
            const real c = o[j];
            x = o[WP + j] - c * x;
            dst[j] = x;
            if (PER) {
              z = zmv[j] - c * z;
              zmo[j] = z;
            }
          }
        }
      }
      {
        const real *o = wt + 2 * WP + cb;
        real *dst = Fp + v * WP + cb;
        real x = xp, z = zp_;
  #pragma unroll
        for (int j = 0; j < M; ++j) {
          if (j < len) {
            const real c = o[j];
            x = o[WP + j] - c * x;
            dst[j] = x;
            if (PER) {
              z = zpv[j] - c * z;
              zpo[j] = z;
            }
          }
        }
      }
    }

    if (PER) {
      // Sherman-Morrison correction x = y - (v.y)/(1 + v.z) z, with
      // v = e_first + (corner_first / g) e_last and corner_first / g = -a0/b0
      // of the unmodified position-0 row; the scalars in FP64.  zmo, zpo are
      // indexed by the chunk's cells.
      real zm_last = real(0), zp_last = real(0);
  #pragma unroll
      for (int j = 0; j < M; ++j) {
        if (j == len - 1) { zm_last = zmo[j]; zp_last = zpo[j]; }
      }
      if (len > 0 && s0 == 0) {              // cell 0: minus first, plus last
        real a0, b0;
        far_row(0, a0, b0);
        ex.sm[v][0][4] = -(double)a0 / (double)b0;
        ex.sm[v][0][0] = Fm[v * WP + 0];
        ex.sm[v][0][1] = zmo[0];
        ex.sm[v][1][2] = Fp[v * WP + 0];
        ex.sm[v][1][3] = zpo[0];
      }
      if (len > 0 && s0 + len == n) {        // cell n-1: plus first, minus last
        real a0, b0;
        far_row(1, a0, b0);
        ex.sm[v][1][4] = -(double)a0 / (double)b0;
        ex.sm[v][1][0] = Fp[v * WP + S::pad(n - 1 - lo)];
        ex.sm[v][1][1] = zp_last;
        ex.sm[v][0][2] = Fm[v * WP + S::pad(n - 1 - lo)];
        ex.sm[v][0][3] = zm_last;
      }
      cluster.sync();
      {
        Exch<real, NV, WPV> *r0 = cluster.map_shared_rank(&ex, 0);
        Exch<real, NV, WPV> *rl = cluster.map_shared_rank(&ex, R - 1);
        double facm = (r0->sm[v][0][0] + r0->sm[v][0][4] * rl->sm[v][0][2]) /
                      (1.0 + r0->sm[v][0][1] + r0->sm[v][0][4] * rl->sm[v][0][3]);
        double facp = (rl->sm[v][1][0] + rl->sm[v][1][4] * r0->sm[v][1][2]) /
                      (1.0 + rl->sm[v][1][1] + rl->sm[v][1][4] * r0->sm[v][1][3]);
        real fm_ = real(facm), fp_ = real(facp);
  #pragma unroll
        for (int j = 0; j < M; ++j) {
          if (j < len) {
            Fm[v * WP + cb + j] -= fm_ * zmo[j];
            Fp[v * WP + cb + j] -= fp_ * zpo[j];
          }
        }
      }
    }
  }
  __syncthreads();

  // ---------------------------------------------------------------- limit
  unsigned int t1 = 0, t2 = 0;
  const real inv12 = real(1) / (real(1) - real(2) * wgl);
  // difference form: the face values hold U - R until a cell is limited,
  // then the limited values in full (cfull[c] = 1)
  float rf[NV];
#pragma unroll
  for (int kv = 0; kv < NV; ++kv) rf[kv] = dlt ? ex.rf[kv] : 0.0f;
  int anyfull = 0;   // this thread limited a cell (difference form)
  if constexpr (MIXED) {
    if (dlt)
      for (int c = tid; c < hi - lo; c += T) cfull[c] = 0;
  }
  if (args.limiter) {
    // FP32 pretest of every cell of this thread (a superset of the cells
    // the exact test limits: its thresholds carry twice the FP32 round-off
    // allowance, which covers the FP32 evaluation and, in the FP64 form, the
    // rounding of the inputs to FP32); the flagged cells (rare) are limited
    // exactly in a second loop, so the pretest loop carries no FP64 state
    static_assert(SEG <= 32 * T, "one mask bit per cell of a thread");
    unsigned int mask = 0;
    const float wgl_f = float(wgl), inv12_f = float(inv12), eps_f = float(eps_pos);
#pragma unroll 1
    for (int q = 0, c = tid; c < hi - lo; ++q, c += T) {
      float ub[NV], a[NV], b[NV];
#pragma unroll
      for (int kv = 0; kv < NV; ++kv) {
        ub[kv] = float(Us[kv * UWP + UH + S::pad(c)]) + rf[kv];
        a[kv] = float(Fm[kv * WP + S::pad(c)]) + rf[kv];
        b[kv] = float(Fp[kv * WP + S::pad(c)]) + rf[kv];
      }
      if (limit_need_mixed<NV>(ub, a, b, wgl_f, inv12_f, eps_f)) mask |= 1u << q;
    }
#pragma unroll 1
    while (mask) {
      const int q = __ffs(mask) - 1;
      mask &= mask - 1;
      const int c = tid + q * T;
      real ub[NV], a[NV], b[NV];
#pragma unroll
      for (int kv = 0; kv < NV; ++kv) {
        ub[kv] = Us[kv * UWP + UH + S::pad(c)];
        a[kv] = Fm[kv * WP + S::pad(c)];
        b[kv] = Fp[kv * WP + S::pad(c)];
      }
      if constexpr (MIXED) {
        if (dlt) {
          // the average as the plain form has it (the FP32 hi part, not
          // R + (ubar - R): exact relative to ubar however far it is from R)
          // and the face values in full
#pragma unroll
          for (int kv = 0; kv < NV; ++kv) {
            ub[kv] = args.Uh[gvar(kv, NV, args.vn, args.vt) * args.ncell + lbase + (long long)(lo + c) * cs];
            a[kv] += rf[kv];
            b[kv] += rf[kv];
          }
        }
      }
      int f;
      if constexpr (MIXED) f = limit_cell_mixed_fp64<NV>(ub, a, b, wgl, eps_pos);
      else f = limit_cell<real, NV>(ub, a, b, wgl, eps_pos, unit_roundoff<real>());
      if (f) {
#pragma unroll
        for (int kv = 0; kv < NV; ++kv) {
          Fm[kv * WP + S::pad(c)] = a[kv];
          Fp[kv * WP + S::pad(c)] = b[kv];
        }
        if constexpr (MIXED) {
          if (dlt) { cfull[c] = 1; anyfull = 1; }
        }
      }
      t1 += f & 1;
      t2 += (f >> 1) & 1;
    }
  }
  // ---------------------------------------------------------------- flux
  // HLLC (or local Lax-Friedrichs) at face f (between cells f-1 and f): the
  // left state is U^- of cell f-1, the right state U^+ of cell f; the two
  // segment-end faces read a neighbour CTA's value.  fsmax: the largest
  // |u| + a over this thread's face states
  real fsmax = real(0);
  auto face = [&](int f) {
    real Ul[NV], Ur[NV], F[NV];
    const real *srcL = nullptr;
    const real *srcR = nullptr;
    const unsigned char *cfL = cfull, *cfR = cfull;   // (difference form)
    int il = 0, ir = 0;
    // left state: U^- of cell f-1
    if (f == 0) {
      if (PER) {
        srcL = cluster.map_shared_rank(Fm, R - 1); il = (n - 1) - (R - 1) * SEG;
        cfL = cluster.map_shared_rank(cfull, R - 1);
      }
    } else if (f - 1 < lo) {
      srcL = cluster.map_shared_rank(Fm, rank - 1); il = f - 1 - (rank - 1) * SEG;
      cfL = cluster.map_shared_rank(cfull, rank - 1);
    } else { srcL = Fm; il = f - 1 - lo; }
    // right state: U^+ of cell f
    if (f == n) {
      if (PER) {
        srcR = cluster.map_shared_rank(Fp, 0); ir = 0;
        cfR = cluster.map_shared_rank(cfull, 0);
      }
    } else if (f >= hi) {
      srcR = cluster.map_shared_rank(Fp, rank + 1); ir = f - (rank + 1) * SEG;
      cfR = cluster.map_shared_rank(cfull, rank + 1);
    } else { srcR = Fp; ir = f - lo; }
    if (srcL) {
#pragma unroll
      for (int kv = 0; kv < NV; ++kv) Ul[kv] = srcL[kv * WP + S::pad(il)];
    }
    if (srcR) {
#pragma unroll
      for (int kv = 0; kv < NV; ++kv) Ur[kv] = srcR[kv * WP + S::pad(ir)];
    }
    real sf;
    if constexpr (MIXED) {
      if (dlt) {
        // stored values are U - R (or the limited U in full): both forms of
        // each state, the exterior of a boundary face by its condition
        float dl[NV], dr[NV];
        // flags of this CTA's cells only where one of them was limited
        const bool fulL = srcL && (cfL != cfull || anyfull) && cfL[il];
        const bool fulR = srcR && (cfR != cfull || anyfull) && cfR[ir];
        if (srcL) {
#pragma unroll
          for (int kv = 0; kv < NV; ++kv) {
            dl[kv] = fulL ? Ul[kv] - rf[kv] : Ul[kv];
            Ul[kv] = fulL ? Ul[kv] : Ul[kv] + rf[kv];
          }
        }
        if (srcR) {
#pragma unroll
          for (int kv = 0; kv < NV; ++kv) {
            dr[kv] = fulR ? Ur[kv] - rf[kv] : Ur[kv];
            Ur[kv] = fulR ? Ur[kv] : Ur[kv] + rf[kv];
          }
        }
        if (!srcL) {
#pragma unroll
          for (int kv = 0; kv < NV; ++kv) { Ul[kv] = Ur[kv]; dl[kv] = dr[kv]; }
          if (args.bclo == 2) { Ul[1] = -Ul[1]; dl[1] = -dr[1] - 2.0f * rf[1]; }
        }
        if (!srcR) {
#pragma unroll
          for (int kv = 0; kv < NV; ++kv) { Ur[kv] = Ul[kv]; dr[kv] = dl[kv]; }
          if (args.bchi == 2) { Ur[1] = -Ur[1]; dr[1] = -dl[1] - 2.0f * rf[1]; }
        }
        const bool near = !args.flux && !fulL && !fulR &&
                          fabsf(dl[0]) <= 0.5f * rf[0] && fabsf(dr[0]) <= 0.5f * rf[0] &&
                          fabsf(dl[NV - 1]) <= 0.5f * rf[NV - 1] &&
                          fabsf(dr[NV - 1]) <= 0.5f * rf[NV - 1];
        if (near) hllc_delta<NV>(Ul, Ur, dl, dr, rf, ex.rp, gam, F, sf);
        else if (args.flux) llf<real, NV>(Ul, Ur, gam, F, sf);
        else hllc<real, NV>(Ul, Ur, gam, F, sf);
        fdel[f - lo] = near ? 1 : 0;
        if (sf > fsmax || sf != sf) fsmax = sf;   // a NaN speed stays
#pragma unroll
        for (int kv = 0; kv < NV; ++kv) Fl[kv * (SEG + 2) + (f - lo)] = F[kv];
        return;
      }
    }
    if (!srcL) {  // boundary face 0: exterior = BC(interior)
#pragma unroll
      for (int kv = 0; kv < NV; ++kv) Ul[kv] = Ur[kv];
      if (args.bclo == 2) Ul[1] = -Ul[1];
    }
    if (!srcR) {
#pragma unroll
      for (int kv = 0; kv < NV; ++kv) Ur[kv] = Ul[kv];
      if (args.bchi == 2) Ur[1] = -Ur[1];
    }
    if (args.flux) llf<real, NV>(Ul, Ur, gam, F, sf);
    else hllc<real, NV>(Ul, Ur, gam, F, sf);
    if (sf > fsmax || sf != sf) fsmax = sf;   // a NaN speed stays
#pragma unroll
    for (int kv = 0; kv < NV; ++kv) Fl[kv * (SEG + 2) + (f - lo)] = F[kv];
  };
  if constexpr (MIXED) {
    // faces with both states in this CTA first, then (after the cluster
    // barrier completes) the two segment-end faces, on two warps; whether
    // any of this CTA's cells holds its face values in full
    anyfull = __syncthreads_or(anyfull);
    cluster_arrive();   // this CTA's limited face values, for the neighbours
    const bool lo_remote = PER || lo > 0, hi_remote = PER || hi < n;
#pragma unroll 1
    for (int pass = 0; pass < 2; ++pass) {   // one call site of the face code
      int f, fend;
      if (pass == 0) {
        f = lo + (lo_remote ? 1 : 0) + tid;
        fend = hi - (hi_remote ? 1 : 0);
      } else {
        cluster_wait();
        f = (tid == 0 && lo_remote) ? lo : ((tid == 32 && hi_remote) ? hi : hi + 1);
        fend = hi;
      }
      for (; f <= fend; f += T) face(f);
    }
  } else {
    // the FP64 form (one CTA per SM, bound by the FP64 pipe): a plain
    // barrier, then every face in one pass
    cluster.sync();
    for (int f = lo + tid; f <= hi; f += T) face(f);
  }
  __syncthreads();
  // the neighbours' face values are no longer read: arrive now, wait before
  // exit (a CTA's shared memory must outlive the neighbours' reads of it)
  cluster_arrive_relaxed();

  // ---------------------------------------------------------------- update
  // the stage's extrema in the line's arithmetic (converted once per warp)
  real mymin = real(sizeof(real) == 4 ? 3.0e38 : 1.0e300), mymax = real(0);
  unsigned int nbad = 0;
  unsigned long long firstbad = ~0ull;
  const real ih = MIXED ? real(args.ih_f) : real(args.ih);
  const double dt = (MODE == MODE_FINAL) ? ctl->dt : 0.0;
  const real *Din = reinterpret_cast<const real *>(args.Din);
  for (int c = tid; c < hi - lo; c += T) {
    int i = lo + c;
    long long addr = lbase + (long long)i * cs;
    real Lv[NV];
    // difference form: a face flux stored as F - F(R) next to one stored as F
    // (a limited or distant face state) is put on the same footing
    int fmix = 0;   // 1: only the left face is F - F(R), 2: only the right one
    if constexpr (MIXED) {
      if (dlt) fmix = (fdel[c] != fdel[c + 1]) ? (fdel[c] ? 2 : 1) : 0;
    }
#pragma unroll
    for (int kv = 0; kv < NV; ++kv) {
      real fa = Fl[kv * (SEG + 2) + c], fb = Fl[kv * (SEG + 2) + c + 1];
      if constexpr (MIXED) {
        if (fmix == 2) fb -= ex.rF[kv];
        else if (fmix == 1) fa -= ex.rF[kv];
      }
      Lv[kv] = (fa - fb) * ih;
      if (MODE != MODE_XSWEEP && Din) Lv[kv] += Din[gvar(kv, NV, args.vn, args.vt) * args.ncell + addr];
    }
    if (MODE == MODE_XSWEEP) {
      real *D = reinterpret_cast<real *>(args.Dout);
#pragma unroll
      for (int kv = 0; kv < NV; ++kv) D[gvar(kv, NV, args.vn, args.vt) * args.ncell + addr] = Lv[kv];
    } else if (MODE == MODE_OPERATOR) {
#pragma unroll
      for (int kv = 0; kv < NV; ++kv) args.Lout[gvar(kv, NV, args.vn, args.vt) * args.ncell + addr] = double(Lv[kv]);
    } else if constexpr (!MIXED) {
      double Ut[NV];
#pragma unroll
      for (int kv = 0; kv < NV; ++kv) {
        int g = gvar(kv, NV, args.vn, args.vt);
        double L = Lv[kv];
        double uk = args.U[g * args.ncell + addr];
        double un;
        if (args.stage == 0) un = uk + dt * L;
        else if (args.stage == 1) un = 0.75 * args.U0[g * args.ncell + addr] + 0.25 * uk + 0.25 * dt * L;
        else un = args.U0[g * args.ncell + addr] * (1.0 / 3.0) + 2.0 / 3.0 * uk + 2.0 / 3.0 * dt * L;
        args.Uout[g * args.ncell + addr] = un;
        Ut[kv] = un;   // line-variable order (no run-time register index)
      }
      // grid momenta: line variable 1 is the normal one (grid index vn)
      double rho = Ut[0], E = Ut[NV - 1];
      double mx = NV == 4 && args.vn != 1 ? Ut[2] : Ut[1];
      double my = NV == 4 ? (args.vn != 1 ? Ut[1] : Ut[2]) : 0.0;
      // one division per cell: 1/rho (1/h from the host)
      const double irho = 1.0 / rho;
      double e = (E - 0.5 * (mx * mx + my * my) * irho) * irho;
      bool ok = (rho > 0.0) && (e > 0.0) && isfinite(E) && isfinite(mx) && isfinite(my);
      if (!ok) {
        ++nbad;
        firstbad = min(firstbad, (unsigned long long)addr);
      } else {
        mymin = fmin(mymin, rho);
        double a = sqrt(args.gamma * (args.gamma - 1.0) * e);
        double rate;
        if (NV == 4) {
          const double ihx = args.vn == 1 ? args.ih : args.ih_other;
          const double ihy = args.vn == 1 ? args.ih_other : args.ih;
          rate = (fabs(mx) * irho + a) * ihx + (fabs(my) * irho + a) * ihy;
        } else {
          rate = (fabs(mx) * irho + a) * args.ih;
        }
        mymax = fmax(mymax, rate);
      }
    } else {
      // mixed form: compensated stage combination on hi + lo pairs
      const dfl dtd = {float(dt), float(dt - double(float(dt)))};
      const dfl third = {0.333333343f, -9.93410776e-09f};
      const dfl two3 = {0.666666687f, -1.98682155e-08f};
      float Th[NV], Tl[NV];
#pragma unroll
      for (int kv = 0; kv < NV; ++kv) {
        int g = gvar(kv, NV, args.vn, args.vt);
        long long a = g * args.ncell + addr;
        dfl uk = {args.Uh[a], args.Ul[a]};
        dfl s = df_add(uk, df_mul_f(dtd, Lv[kv]));          // U_k + dt L
        dfl un;
        if (args.stage == 0) {
          un = s;
        } else {
          dfl u0 = {args.U0h[a], args.U0l[a]};
          if (args.stage == 1) un = df_add(df_mul_f(u0, 0.75f), df_mul_f(s, 0.25f));
          else un = df_add(df_mul(u0, third), df_mul(s, two3));
        }
        args.Uoh[a] = un.hi;
        args.Uol[a] = un.lo;
        Th[kv] = un.hi;   // line-variable order (no run-time register index)
        Tl[kv] = un.lo;
      }
      float rho = Th[0], E = Th[NV - 1];
      float mx = NV == 4 && args.vn != 1 ? Th[2] : Th[1];
      float my = NV == 4 ? (args.vn != 1 ? Th[1] : Th[2]) : 0.0f;
      // g = rho E - |m|^2/2 with the compensated parts (its sign decides G)
      dfl rE = df_mul({Th[0], Tl[0]}, {Th[NV - 1], Tl[NV - 1]});
      dfl m2 = df_mul({Th[1], Tl[1]}, {Th[1], Tl[1]});
      if (NV == 4) m2 = df_add(m2, df_mul({Th[2], Tl[2]}, {Th[2], Tl[2]}));
      dfl gq = df_add(rE, {-0.5f * m2.hi, -0.5f * m2.lo});
      bool ok = (rho > 0.0f) && (gq.hi > 0.0f) && isfinite(E) && isfinite(mx) && isfinite(my);
      if (!ok) {
        ++nbad;
        firstbad = min(firstbad, (unsigned long long)addr);
      } else {
        mymin = fminf(mymin, rho);
        float e = gq.hi / (rho * rho);
        float a = sqrtf(args.gg1_f * e);
        float rate;
        if (NV == 4) {
          const float ihx = args.vn == 1 ? args.ih_f : args.ih_other_f;
          const float ihy = args.vn == 1 ? args.ih_other_f : args.ih_f;
          rate = (fabsf(mx / rho) + a) * ihx + (fabsf(my / rho) + a) * ihy;
        } else {
          rate = (fabsf(mx / rho) + a) * args.ih_f;
        }
        mymax = fmaxf(mymax, rate);
      }
    }
  }

  // ---------------------------------------------------------------- reduce
  // eq. (CFL-CD) checked on the face values: the stage's largest face rate
  // of this direction (max over the step's stages; NaN wins the bit max)
  // (in the line's arithmetic: FP64 instructions cost the FP32 form 1/64 of
  // an issue slot's worth each, and one conversion per warp suffices)
  if (MODE != MODE_OPERATOR && args.fcheck && args.eps_fixed <= 0.0) {
    real fr = fsmax * (MIXED ? real(args.ih_f) : real(args.ih));
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      const real o = shfl_down_r(fr, d);
      if (o > fr || o != o) fr = o;
    }
    if (lane == 0) atomic_max_bits(&ctl->frate[args.fdir], double_bits(double(fr)));
  }
  if (MODE == MODE_FINAL) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      mymin = fmin(mymin, shfl_down_r(mymin, d));
      mymax = fmax(mymax, shfl_down_r(mymax, d));
      nbad += __shfl_down_sync(0xffffffffu, nbad, d);
      t1 += __shfl_down_sync(0xffffffffu, t1, d);
      t2 += __shfl_down_sync(0xffffffffu, t2, d);
      unsigned long long fb = __shfl_down_sync(0xffffffffu, firstbad, d);
      firstbad = fb < firstbad ? fb : firstbad;
    }
    if (lane == 0) {
      atomic_min_bits(&ctl->minrho[args.stage], double_bits(double(mymin)));
      if (args.stage == 2) atomic_max_bits(&ctl->rate, double_bits(double(mymax)));
      if (nbad) {
        atomicAdd(&ctl->nviol, (unsigned long long)nbad);
        atomicMin(&ctl->first_bad, firstbad);
      }
      if (t1) atomicAdd(&ctl->theta1, (unsigned long long)t1);
      if (t2) atomicAdd(&ctl->theta2, (unsigned long long)t2);
    }
  } else if (MODE == MODE_XSWEEP) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      t1 += __shfl_down_sync(0xffffffffu, t1, d);
      t2 += __shfl_down_sync(0xffffffffu, t2, d);
    }
    if (lane == 0) {
      if (t1) atomicAdd(&ctl->theta1, (unsigned long long)t1);
      if (t2) atomicAdd(&ctl->theta2, (unsigned long long)t2);
    }
  }
  cluster_wait();
}

}  // namespace ppk
