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
};

enum { MODE_XSWEEP = 0, MODE_FINAL = 1, MODE_OPERATOR = 2 };

// one problem of a batch: its block of the concatenated state (values
// [off, off + nv*ncell), variable planes of ncell cells) and grid
struct ProbDesc {
  long long off, ncell;
  int nx, ny;
  double dx, dy;
  int bc[4];
};

// one line of a batched launch: problem index and line index inside it
struct LineRef {
  int prob, line;
};

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
  double gamma, wgl, eps_weno;
  int stage;          // 0, 1, 2
  double eps_fixed;   // > 0: fixed limiter epsilon, no control-block checks (operator evaluation)
  int limiter;
  Ctl *ctl;
  // batched launch: line table and problem descriptors (nullptr: one problem)
  const LineRef *lines;
  const ProbDesc *probs;
  int xdir;           // batched launch: 1 x lines, 0 y lines
  long long nvals;    // batched mixed form: values per hi block (lo block follows)
};

// resolve the line a cluster works on: for a batched launch, take the
// problem's grid, boundaries, control block and its slice of every buffer
template <int NV>
__device__ __forceinline__ void bind_line(SweepArgs &a, long long &line) {
  if (!a.lines) return;
  LineRef lr = a.lines[line];
  const ProbDesc pd = a.probs[lr.prob];
  line = lr.line;
  a.ctl = a.ctl + lr.prob;
  a.ncell = pd.ncell;
  if (a.xdir) {
    a.n = pd.nx; a.cell_stride = 1; a.line_stride = pd.nx;
    a.bclo = pd.bc[0]; a.bchi = pd.bc[1];
    a.h = pd.dx; a.h_other = NV == 4 ? pd.dy : 0.0;
  } else {
    a.n = pd.ny; a.cell_stride = pd.nx; a.line_stride = 1;
    a.bclo = pd.bc[2]; a.bchi = pd.bc[3];
    a.h = pd.dy; a.h_other = pd.dx;
  }
  const long long o = pd.off;
  if (a.U) a.U += o;
  if (a.U0) a.U0 += o;
  if (a.Uout) a.Uout += o;
  if (a.Uh) { a.Uh += o; a.Ul = a.Uh + a.nvals; }
  if (a.U0h) { a.U0h += o; a.U0l = a.U0h + a.nvals; }
  if (a.Uoh) { a.Uoh += o; a.Uol = a.Uoh + a.nvals; }
  if (a.Lout) a.Lout += o;
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
__device__ __forceinline__ real shfl_up_r(real v, int d) { return __shfl_up_sync(0xffffffffu, v, d); }
template <typename real>
__device__ __forceinline__ real shfl_down_r(real v, int d) { return __shfl_down_sync(0xffffffffu, v, d); }

template <typename real, bool PER, bool UP>
__device__ __forceinline__ Fwd<real> fwd_shfl(const Fwd<real> &f, int d) {
  Fwd<real> o;
#define PPK_SH(x) o.x = UP ? shfl_up_r(f.x, d) : shfl_down_r(f.x, d)
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
};

template <typename real, int NV, int M>
struct Smem {
  static constexpr int KC = SEGC / M;     // chunks per conserved variable
  static constexpr int WPV = KC / 32;     // warps per conserved variable
  static constexpr int SEG = SEGC;
  static constexpr size_t u_off = 0;                                    // real Us[NV][SEG+4]
  static constexpr size_t w_off = u_off + sizeof(real) * NV * (SEG + 4); // real Wt[NV][4][SEG]
  static constexpr size_t fm_off = w_off + sizeof(real) * NV * 4 * SEG;
  static constexpr size_t fp_off = fm_off + sizeof(real) * NV * SEG;    // real Fm, Fp[NV][SEG]
  static constexpr size_t fl_off = fp_off + sizeof(real) * NV * SEG;    // real Fl[NV][SEG+2]
  static constexpr size_t rm_off = fl_off + sizeof(real) * NV * (SEG + 2);  // remote stencils
  static constexpr size_t ex_off = (rm_off + sizeof(real) * NV * 2 * 6 + 15) / 16 * 16;
  static constexpr size_t bytes = ex_off + sizeof(Exch<real, NV, WPV>);
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

// ---------------------------------------------------------------- kernel
// the mixed form asks for two resident CTAs per SM (128 registers at M = 8)
template <typename real, int NV, int M, bool PER, int MODE>
__global__ void __launch_bounds__(NV * (SEGC / M), sizeof(real) == 4 ? 2 : 1)
    line_sweep(SweepArgs args_in) {
  constexpr bool MIXED = sizeof(real) == 4;
  using S = Smem<real, NV, M>;
  constexpr int SEG = S::SEG;
  constexpr int KC = S::KC;
  constexpr int WPV = S::WPV;
  constexpr int T = NV * KC;
  constexpr int UW = SEG + 4;
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
  bind_line<NV>(args, line);
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

  const real eps_w = real(args.eps_weno);
  const real gam = real(args.gamma);
  const real wgl = real(args.wgl);
  real eps_pos;
  if (args.eps_fixed > 0.0) eps_pos = real(args.eps_fixed);
  else if (args.stage == 0) eps_pos = real(ctl->eps0);
  else eps_pos = real(fmin(ctl->eps_pos, bits_double(ctl->minrho[args.stage - 1])));

  const long long lbase = line * args.line_stride;
  const long long cs = args.cell_stride;

  // ---------------------------------------------------------------- load
  auto cell_val = [&](int kv, int i) -> real {
    // line variable kv at line cell i (any i; ghosts by the boundary condition)
    int g = gvar(kv, NV, args.vn, args.vt);
    bool neg = false;
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
    long long a = g * args.ncell + lbase + (long long)i * cs;
    real x;
    if constexpr (MIXED) x = args.Uh[a];
    else x = args.U[a];
    return neg ? -x : x;
  };

  bool vec = false;
  if constexpr (MIXED) {
    // contiguous line with 16-byte aligned segments: the segment's cells
    // come in as float4, only the halo and a ragged tail cell by cell
    vec = cs == 1 && !args.lines && ((lbase + lo) & 3) == 0 && (args.ncell & 3) == 0 &&
          ((reinterpret_cast<unsigned long long>(args.Uh) & 15) == 0);
    if (vec) {
      const int nq = (hi - lo) >> 2;
      for (int idx = tid; idx < NV * nq; idx += T) {
        int kv = idx / nq, q = idx - kv * nq;
        int g = gvar(kv, NV, args.vn, args.vt);
        float4 x = *reinterpret_cast<const float4 *>(args.Uh + g * args.ncell + lbase + lo + 4 * q);
        real *d = Us + kv * UW + 2 + 4 * q;
        d[0] = x.x; d[1] = x.y; d[2] = x.z; d[3] = x.w;
      }
      const int nr = UW - 4 * nq;
      for (int idx = tid; idx < NV * nr; idx += T) {
        int kv = idx / nr, r = idx - kv * nr;
        int j = r < 2 ? r : 4 * nq + r;
        int i = lo - 2 + j;
        Us[kv * UW + j] = (i < hi + 2) ? cell_val(kv, i) : real(0);
      }
    }
  }
  if (!vec) {
    for (int idx = tid; idx < NV * UW; idx += T) {
      int kv = idx / UW, j = idx % UW;
      int i = lo - 2 + j;
      Us[kv * UW + j] = (i < hi + 2) ? cell_val(kv, i) : real(0);
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
  __syncthreads();

  // ---------------------------------------------------------------- rows
  const real *u = Us + v * UW + 2;            // u[i - lo], valid i - lo in [-2, hi-lo+2)
  real *wt = Wt + v * 4 * SEG;                // wt[q*SEG + c]: w0-, w2-, w0+, w2+
  const int s0 = lo + k * M;                  // first cell of this thread's chunk
  const int len = max(0, min(M, hi - s0));
  const bool bounded = !PER;

  // weights of cell i for both sides (stored), or the closure values
  auto weights_of = [&](int i) {
    const real *x = u + (i - lo);
    real *o = wt + (i - lo);
    if (bounded && (i == 0 || i == n - 1)) {
      o[0] = weno5z_face(x[-2], x[-1], x[0], x[1], x[2], eps_w);
      o[2 * SEG] = weno5z_face(x[2], x[1], x[0], x[-1], x[-2], eps_w);
      return;
    }
    real q0, q1, q2, one, w0, w1, w2;
    zratios_any(x[-2], x[-1], x[0], x[1], x[2], eps_w, q0, q1, q2, one);
    zweights(real(0.2), real(0.5), real(0.3), q0, q1, q2, w0, w1, w2, one);
    o[0] = w0;
    o[SEG] = w2;
    zweights(real(0.2), real(0.5), real(0.3), q2, q1, q0, w0, w1, w2, one);
    o[2 * SEG] = w0;
    o[3 * SEG] = w2;
  };

  // a, b of the unmodified position-0 row of side 0 (cell 0) or 1 (cell n-1),
  // needed by the Sherman-Morrison row at the far end of a periodic system
  auto far_row = [&](int side, real &a0, real &b0) {
    const real *y = Rm + (v * 2 + side) * 6 + 2;
    real q0, q1, q2, one, w0, w1, w2;
    zratios_any(y[-2], y[-1], y[0], y[1], y[2], eps_w, q0, q1, q2, one);
    if (side == 0) zweights(real(0.2), real(0.5), real(0.3), q0, q1, q2, w0, w1, w2, one);
    else zweights(real(0.2), real(0.5), real(0.3), q2, q1, q0, w0, w1, w2, one);
    Row<real> r = compact_row02(w0, w2, real(0), real(0), real(0));
    a0 = r.a;
    b0 = r.b;
  };

  // row of cell i, side 0 (minus: prev = i-1) or 1 (plus: prev = i+1), from
  // the stored weights; zr = the Sherman-Morrison right-hand side entry
  auto row_of = [&](int i, int side, real &zr) -> Row<real> {
    const real *x = u + (i - lo);
    const real *o = wt + (i - lo) + 2 * side * SEG;
    Row<real> r;
    zr = real(0);
    if (bounded && (i == 0 || i == n - 1)) {
      r.a = real(0); r.b = real(1); r.c = real(0); r.r = o[0];
      return r;
    }
    if (side == 0) r = compact_row02(o[0], o[SEG], x[-1], x[0], x[1]);
    else r = compact_row02(o[0], o[SEG], x[1], x[0], x[-1]);
    if (PER) {
      const int first = side == 0 ? 0 : n - 1, last = side == 0 ? n - 1 : 0;
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
    }
    return r;
  };

  // ------------------------------------------- weights + chunk maps (F1)
  // the chunk's cells and their two-cell halo come from shared memory once
  // into registers; weights are stored for the elimination pass (F5) and the
  // rows built from the registers
  Fwd<real> fm = fwd_identity<real>(), fp = fwd_identity<real>();
  {
    real win[M + 4];
#pragma unroll
    for (int q = 0; q < M + 4; ++q) win[q] = u[s0 - lo - 2 + q];
#pragma unroll
    for (int j = 0; j < M; ++j) {
      if (j < len) {
        const int i = s0 + j;
        real zm = real(0), zp = real(0);
        Row<real> rm, rp;
        if (bounded && (i == 0 || i == n - 1)) {
          weights_of(i);
          rm = row_of(i, 0, zm);
          rp = row_of(i, 1, zp);
        } else {
          real q0, q1, q2, one, w0, w1, w2, v0, v1, v2;
          zratios_any(win[j], win[j + 1], win[j + 2], win[j + 3], win[j + 4], eps_w, q0, q1, q2, one);
          zweights(real(0.2), real(0.5), real(0.3), q0, q1, q2, w0, w1, w2, one);
          zweights(real(0.2), real(0.5), real(0.3), q2, q1, q0, v0, v1, v2, one);
          real *o = wt + (i - lo);
          o[0] = w0;
          o[SEG] = w2;
          o[2 * SEG] = v0;
          o[3 * SEG] = v2;
          if (PER && (i == 0 || i == n - 1)) {
            rm = row_of(i, 0, zm);
            rp = row_of(i, 1, zp);
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
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    Fwd<real> o = fwd_shfl<real, PER, true>(fm, d);
    if (lane >= d) { fm = fwd_compose<real, PER>(fm, o); fwd_normalise(fm); }
    Fwd<real> q = fwd_shfl<real, PER, false>(fp, d);
    if (lane + d < 32) { fp = fwd_compose<real, PER>(fp, q); fwd_normalise(fp); }
  }
  Fwd<real> fm_ex = fwd_shfl<real, PER, true>(fm, 1);
  if (lane == 0) fm_ex = fwd_identity<real>();
  Fwd<real> fp_ex = fwd_shfl<real, PER, false>(fp, 1);
  if (lane == 31) fp_ex = fwd_identity<real>();
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
  if (tid < 2 * NV) {
    int vv = tid >> 1, sd = tid & 1;
    real cp = real(0), dp = real(0), zp = real(0);
    if (sd == 0) {
      for (int q = 0; q < rank; ++q) {
        Exch<real, NV, WPV> *rx = cluster.map_shared_rank(&ex, q);
        fwd_apply<real, PER>(rx->seg_fwd[vv][0], cp, dp, zp);
      }
    } else {
      for (int q = R - 1; q > rank; --q) {
        Exch<real, NV, WPV> *rx = cluster.map_shared_rank(&ex, q);
        fwd_apply<real, PER>(rx->seg_fwd[vv][1], cp, dp, zp);
      }
    }
    for (int ww = 0; ww < WPV; ++ww) {
      int wi = sd == 0 ? ww : WPV - 1 - ww;
      ex.warp_in[vv][sd][wi][0] = cp;
      ex.warp_in[vv][sd][wi][1] = dp;
      ex.warp_in[vv][sd][wi][2] = zp;
      fwd_apply<real, PER>(ex.warp_fwd[vv][sd][wi], cp, dp, zp);
    }
  }
  __syncthreads();

  real cpm = ex.warp_in[v][0][w][0], dpm = ex.warp_in[v][0][w][1], zpm = ex.warp_in[v][0][w][2];
  fwd_apply<real, PER>(fm_ex, cpm, dpm, zpm);
  real cpp = ex.warp_in[v][1][w][0], dpp = ex.warp_in[v][1][w][1], zpp = ex.warp_in[v][1][w][2];
  fwd_apply<real, PER>(fp_ex, cpp, dpp, zpp);

  // ------------------------------------------- chunk elimination (F5)
  // Thomas elimination of the chunk from the incoming state, keeping c', d'
  // (and z') per row for the back substitution, and the chunk's back
  // substitution map x_first = A + B x_after accumulated in the same pass:
  // A = sum_j (prod_{l<j} -c'_l) d'_j, B = prod_l -c'_l.
  // minus: position j <-> cell s0 + j; plus: position j <-> cell s0+len-1-j.
  real cmv[M], dmv[M], zmv[M], cpv[M], dpv[M], zpv[M];
  Bwd<real> bm, bp;
  {
    // the two sides' recurrences are independent: advance them together
    real pim = real(1), Am = real(0), Azm = real(0);
    real pip = real(1), Ap = real(0), Azp = real(0);
#pragma unroll
    for (int j = 0; j < M; ++j) {
      if (j < len) {
        real zrm, zrp;
        Row<real> rm = row_of(s0 + j, 0, zrm);
        Row<real> rp = row_of(s0 + len - 1 - j, 1, zrp);
        real ipm = real(1) / (rm.b - rm.a * cpm);
        real ipp = real(1) / (rp.b - rp.a * cpp);
        cpm = rm.c * ipm;
        cpp = rp.c * ipp;
        dpm = (rm.r - rm.a * dpm) * ipm;
        dpp = (rp.r - rp.a * dpp) * ipp;
        if (PER) {
          zpm = (zrm - rm.a * zpm) * ipm;
          zpp = (zrp - rp.a * zpp) * ipp;
        }
        cmv[j] = cpm; dmv[j] = dpm; zmv[j] = PER ? zpm : real(0);
        cpv[j] = cpp; dpv[j] = dpp; zpv[j] = PER ? zpp : real(0);
        Am += pim * dpm;
        Ap += pip * dpp;
        if (PER) { Azm += pim * zpm; Azp += pip * zpp; }
        pim *= -cpm;
        pip *= -cpp;
      }
    }
    bm.A = Am; bm.Az = Azm; bm.B = pim;
    bp.A = Ap; bp.Az = Azp; bp.B = pip;
  }

  // ------------------------------------------- backward scans (F6)
  Bwd<real> bm_in = bm, bp_in = bp;
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
  Bwd<real> bm_ex, bp_ex;
  bm_ex.A = shfl_down_r(bm_in.A, 1); bm_ex.B = shfl_down_r(bm_in.B, 1);
  bm_ex.Az = PER ? shfl_down_r(bm_in.Az, 1) : real(0);
  if (lane == 31) { bm_ex.A = real(0); bm_ex.B = real(1); bm_ex.Az = real(0); }
  bp_ex.A = shfl_up_r(bp_in.A, 1); bp_ex.B = shfl_up_r(bp_in.B, 1);
  bp_ex.Az = PER ? shfl_up_r(bp_in.Az, 1) : real(0);
  if (lane == 0) { bp_ex.A = real(0); bp_ex.B = real(1); bp_ex.Az = real(0); }
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
  if (tid < 2 * NV) {
    int vv = tid >> 1, sd = tid & 1;
    real x = real(0), z = real(0);
    if (sd == 0) {
      for (int q = R - 1; q > rank; --q) {
        Exch<real, NV, WPV> *rx = cluster.map_shared_rank(&ex, q);
        Bwd<real> b = rx->seg_bwd[vv][0];
        x = b.A + b.B * x;
        z = b.Az + b.B * z;
      }
      for (int ww = WPV - 1; ww >= 0; --ww) {
        ex.warp_xn[vv][0][ww][0] = x;
        ex.warp_xn[vv][0][ww][1] = z;
        Bwd<real> b = ex.warp_bwd[vv][0][ww];
        x = b.A + b.B * x;
        z = b.Az + b.B * z;
      }
    } else {
      for (int q = 0; q < rank; ++q) {
        Exch<real, NV, WPV> *rx = cluster.map_shared_rank(&ex, q);
        Bwd<real> b = rx->seg_bwd[vv][1];
        x = b.A + b.B * x;
        z = b.Az + b.B * z;
      }
      for (int ww = 0; ww < WPV; ++ww) {
        ex.warp_xn[vv][1][ww][0] = x;
        ex.warp_xn[vv][1][ww][1] = z;
        Bwd<real> b = ex.warp_bwd[vv][1][ww];
        x = b.A + b.B * x;
        z = b.Az + b.B * z;
      }
    }
  }
  __syncthreads();

  // ------------------------------------------- back substitution (F8)
  real zmo[M], zpo[M];
  {
    real xn = ex.warp_xn[v][0][w][0], zn = ex.warp_xn[v][0][w][1];
    real x = bm_ex.A + bm_ex.B * xn;
    real z = bm_ex.Az + bm_ex.B * zn;
#pragma unroll
    for (int jj = 0; jj < M; ++jj) {
      int j = M - 1 - jj;
      if (j < len) {
        x = dmv[j] - cmv[j] * x;
        if (PER) z = zmv[j] - cmv[j] * z;
        Fm[v * SEG + (s0 + j - lo)] = x;
        zmo[j] = z;
      }
    }
  }
  {
    real xn = ex.warp_xn[v][1][w][0], zn = ex.warp_xn[v][1][w][1];
    real x = bp_ex.A + bp_ex.B * xn;
    real z = bp_ex.Az + bp_ex.B * zn;
#pragma unroll
    for (int jj = 0; jj < M; ++jj) {
      int pos = M - 1 - jj;     // plus positions from the chunk's left-most cell
      if (pos < len) {
        x = dpv[pos] - cpv[pos] * x;
        if (PER) z = zpv[pos] - cpv[pos] * z;
        Fp[v * SEG + (s0 + len - 1 - pos - lo)] = x;
        zpo[pos] = z;
      }
    }
  }

  if (PER) {
    // Sherman-Morrison correction x = y - (v.y)/(1 + v.z) z, with
    // v = e_first + (corner_first / g) e_last and corner_first / g = -a0/b0
    // of the unmodified position-0 row; the scalars in FP64
    if (len > 0 && s0 == 0) {              // cell 0: minus first, plus last
      real a0, b0;
      far_row(0, a0, b0);
      ex.sm[v][0][4] = -(double)a0 / (double)b0;
      ex.sm[v][0][0] = Fm[v * SEG + 0];
      ex.sm[v][0][1] = zmo[0];
      ex.sm[v][1][2] = Fp[v * SEG + 0];
      ex.sm[v][1][3] = zpo[len - 1];
    }
    if (len > 0 && s0 + len == n) {        // cell n-1: plus first, minus last
      real a0, b0;
      far_row(1, a0, b0);
      ex.sm[v][1][4] = -(double)a0 / (double)b0;
      ex.sm[v][1][0] = Fp[v * SEG + (n - 1 - lo)];
      ex.sm[v][1][1] = zpo[0];
      ex.sm[v][0][2] = Fm[v * SEG + (n - 1 - lo)];
      ex.sm[v][0][3] = zmo[len - 1];
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
          Fm[v * SEG + (s0 + j - lo)] -= fm_ * zmo[j];
          Fp[v * SEG + (s0 + j - lo)] -= fp_ * zpo[len - 1 - j];
        }
      }
    }
  }
  __syncthreads();

  // ---------------------------------------------------------------- limit
  unsigned int t1 = 0, t2 = 0;
  if (args.limiter) {
    for (int c = tid; c < hi - lo; c += T) {
      real ub[NV], a[NV], b[NV];
#pragma unroll
      for (int kv = 0; kv < NV; ++kv) {
        ub[kv] = Us[kv * UW + c + 2];
        a[kv] = Fm[kv * SEG + c];
        b[kv] = Fp[kv * SEG + c];
      }
      int f;
      if constexpr (MIXED) f = limit_cell_mixed<NV>(ub, a, b, wgl, eps_pos);
      else f = limit_cell<real, NV>(ub, a, b, wgl, eps_pos, unit_roundoff<real>());
      if (f) {
#pragma unroll
        for (int kv = 0; kv < NV; ++kv) {
          Fm[kv * SEG + c] = a[kv];
          Fp[kv * SEG + c] = b[kv];
        }
      }
      t1 += f & 1;
      t2 += (f >> 1) & 1;
    }
  }
  cluster.sync();

  // ---------------------------------------------------------------- flux
  for (int f = lo + tid; f <= hi; f += T) {
    real Ul[NV], Ur[NV], F[NV];
    const real *srcL = nullptr;
    const real *srcR = nullptr;
    int il = 0, ir = 0;
    // left state: U^- of cell f-1
    if (f == 0) {
      if (PER) { srcL = cluster.map_shared_rank(Fm, R - 1); il = (n - 1) - (R - 1) * SEG; }
    } else if (f - 1 < lo) {
      srcL = cluster.map_shared_rank(Fm, rank - 1); il = f - 1 - (rank - 1) * SEG;
    } else { srcL = Fm; il = f - 1 - lo; }
    // right state: U^+ of cell f
    if (f == n) {
      if (PER) { srcR = cluster.map_shared_rank(Fp, 0); ir = 0; }
    } else if (f >= hi) {
      srcR = cluster.map_shared_rank(Fp, rank + 1); ir = f - (rank + 1) * SEG;
    } else { srcR = Fp; ir = f - lo; }
    if (srcL) {
#pragma unroll
      for (int kv = 0; kv < NV; ++kv) Ul[kv] = srcL[kv * SEG + il];
    }
    if (srcR) {
#pragma unroll
      for (int kv = 0; kv < NV; ++kv) Ur[kv] = srcR[kv * SEG + ir];
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
    hllc<real, NV>(Ul, Ur, gam, F);
#pragma unroll
    for (int kv = 0; kv < NV; ++kv) Fl[kv * (SEG + 2) + (f - lo)] = F[kv];
  }
  cluster.sync();   // neighbours' face values are no longer read after this

  // ---------------------------------------------------------------- update
  double mymin = 1.0e300, mymax = 0.0;
  unsigned int nbad = 0;
  unsigned long long firstbad = ~0ull;
  const real ih = real(1.0 / args.h);
  const double dt = (MODE == MODE_FINAL) ? ctl->dt : 0.0;
  const real *Din = reinterpret_cast<const real *>(args.Din);
  for (int c = tid; c < hi - lo; c += T) {
    int i = lo + c;
    long long addr = lbase + (long long)i * cs;
    real Lv[NV];
#pragma unroll
    for (int kv = 0; kv < NV; ++kv) {
      Lv[kv] = (Fl[kv * (SEG + 2) + c] - Fl[kv * (SEG + 2) + c + 1]) * ih;
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
        else un = args.U0[g * args.ncell + addr] / 3.0 + 2.0 / 3.0 * uk + 2.0 / 3.0 * dt * L;
        args.Uout[g * args.ncell + addr] = un;
        Ut[g] = un;
      }
      double rho = Ut[0];
      double mx = Ut[1], my = NV == 4 ? Ut[2] : 0.0, E = Ut[NV - 1];
      double e = E / rho - 0.5 * (mx * mx + my * my) / (rho * rho);
      bool ok = (rho > 0.0) && (e > 0.0) && isfinite(E) && isfinite(mx) && isfinite(my);
      if (!ok) {
        ++nbad;
        firstbad = min(firstbad, (unsigned long long)addr);
      } else {
        mymin = fmin(mymin, rho);
        double a = sqrt(args.gamma * (args.gamma - 1.0) * e);
        double rate;
        if (NV == 4) {
          double hx = args.vn == 1 ? args.h : args.h_other;
          double hy = args.vn == 1 ? args.h_other : args.h;
          rate = (fabs(mx / rho) + a) / hx + (fabs(my / rho) + a) / hy;
        } else {
          rate = (fabs(mx / rho) + a) / args.h;
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
        Th[g] = un.hi;
        Tl[g] = un.lo;
      }
      float rho = Th[0];
      float mx = Th[1], my = NV == 4 ? Th[2] : 0.0f, E = Th[NV - 1];
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
        mymin = fmin(mymin, (double)rho);
        float e = gq.hi / (rho * rho);
        float a = sqrtf(float(args.gamma * (args.gamma - 1.0)) * e);
        float rate;
        if (NV == 4) {
          float hx = float(args.vn == 1 ? args.h : args.h_other);
          float hy = float(args.vn == 1 ? args.h_other : args.h);
          rate = (fabsf(mx / rho) + a) / hx + (fabsf(my / rho) + a) / hy;
        } else {
          rate = (fabsf(mx / rho) + a) / float(args.h);
        }
        mymax = fmax(mymax, (double)rate);
      }
    }
  }

  // ---------------------------------------------------------------- reduce
  if (MODE == MODE_FINAL) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      mymin = fmin(mymin, __shfl_down_sync(0xffffffffu, mymin, d));
      mymax = fmax(mymax, __shfl_down_sync(0xffffffffu, mymax, d));
      nbad += __shfl_down_sync(0xffffffffu, nbad, d);
      t1 += __shfl_down_sync(0xffffffffu, t1, d);
      t2 += __shfl_down_sync(0xffffffffu, t2, d);
      unsigned long long fb = __shfl_down_sync(0xffffffffu, firstbad, d);
      firstbad = fb < firstbad ? fb : firstbad;
    }
    if (lane == 0) {
      atomicMin(&ctl->minrho[args.stage], double_bits(mymin));
      if (args.stage == 2) atomicMax(&ctl->rate, double_bits(mymax));
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
}

}  // namespace ppk
