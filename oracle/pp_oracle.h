/*
 * pp_oracle.h -- FP64 CPU oracle for the positivity-preserving fifth-order
 * finite-volume compact-WENO (FVCW) scheme of Guo, Xiong & Shi.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library
 * and its Python binding) may include, link or call this code; only the
 * tests, the smoke check and the CPU-baseline leg of the benchmark use it.
 * It shares no code with the GPU implementation.
 *
 * Layout of every state array: structure of arrays U[v][j][i] with i the
 * fastest (x) index, v = 0..nv-1:
 *   1-D (nv = 3): rho, m = rho*u, E                      (Sec. 1, eq. (1DEuler))
 *   2-D (nv = 4): rho, m_x, m_y, E   (dimension-by-dimension extension)
 */
#ifndef PP_ORACLE_H
#define PP_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_BC_PERIODIC = 0, ORC_BC_TRANSMISSIVE = 1, ORC_BC_REFLECTIVE = 2 };

typedef struct {
  int    ndim;           /* 1 or 2 */
  long   nx, ny;         /* ny = 1 when ndim == 1 */
  double dx, dy;         /* uniform cell sizes */
  double gamma;          /* ratio of specific heats */
  int    bc[4];          /* x-lo, x-hi, y-lo, y-hi (ORC_BC_*) */
  double gl_weight;      /* Gauss-Lobatto end weight omega_hat_1 (= omega_hat_M) */
  double eps_weno;       /* epsilon of the WENO-Z weights, eq. (weight) */
  double eps_pos;        /* cap of the limiter epsilon (1e-13), Sec. 2.4 step 1 */
  int    limiter;        /* 1: Zhang-Shu limiter on, 0: off (tests only) */
  int    linear_weights; /* 1: force omega_k = c_k (linear compact scheme, tests) */
  int    flux;           /* 0: HLLC (Sec. 2.4); 1: local Lax-Friedrichs (Sec. 3 remark) */
  int    recon;          /* 0: component-wise (conserved variables); 1: characteristic-wise (Sec. 2.3) */
  double face_cfl;       /* > 0: the bound omega_hat_1 of eq. (CFL-CD) checked on the limited face
                            values of every stage; orc_advance redoes a step that exceeds it
                            (0: no check, dt from the cell averages only) */
} orc_grid;

typedef struct {
  long theta1_active;    /* cells with theta_1 < 1 (density limited) */
  long theta2_active;    /* cells with theta_2 < 1 (internal energy limited) */
  long bad_cells;        /* cells whose average left the admissible set G */
  double face_rate;      /* max over the operator calls of sum over directions of
                            max (|u|+a)/h over the limited face values U^-, U^+ */
  long rejected;         /* orc_advance: steps redone with a smaller dt (face_cfl check) */
} orc_counters;

/* ---- scalar building blocks (Sec. 2.2) ---- */
/* Jiang-Shu smoothness indicators of the three 3-cell sub-stencils around
 * cell j; u5 = (u_{j-2}, u_{j-1}, u_j, u_{j+1}, u_{j+2}). */
void orc_smoothness(const double *u5, double *beta3);
/* WENO-Z weights, eq. (weight): omega_k = alpha_k / sum alpha,
 * alpha_k = c_k (1 + (tau5/(beta_k + eps))^2), tau5 = |beta_2 - beta_0|. */
void orc_wenoz_weights(const double *beta3, const double *c3, double eps, double *w3);

/* Thomas elimination of a tridiagonal system
 *   sub[i] x[i-1] + diag[i] x[i] + sup[i] x[i+1] = rhs[i],  i = 0..n-1
 * (sub[0], sup[n-1] ignored).  reverse = 0 eliminates from i = 0 upward,
 * reverse = 1 from i = n-1 downward.  Returns 0, or -1 on a zero pivot. */
int orc_thomas(long n, const double *sub, const double *diag, const double *sup,
               const double *rhs, double *x, int reverse);
/* Cyclic (periodic) tridiagonal system, sub[0] couples x[n-1] and sup[n-1]
 * couples x[0]; Sherman-Morrison correction of a Thomas solve. */
int orc_cyclic(long n, const double *sub, const double *diag, const double *sup,
               const double *rhs, double *x, int reverse);

/* Compact-WENO reconstruction of one scalar line of n cells.  ext holds
 * n + 4 cell averages: two ghost cells on each side, ext[j+2] = ubar_j.
 * periodic != 0 solves the cyclic systems; otherwise the first and last
 * unknowns are closed by the explicit fifth-order WENO-Z reconstruction.
 * um[j] = u^-_{j+1/2} (right face of cell j, from cell j),
 * up[j] = u^+_{j-1/2} (left face of cell j, from cell j).  Returns 0 or -1. */
int orc_recon_scalar(long n, const double *ext, int periodic, double eps_weno,
                     int linear_weights, double *um, double *up);

/* ---- characteristic-wise pieces (Sec. 2.3) ---- */
/* Left (Lm) and right (Rm) eigenvector matrices, row-major nv x nv, of the
 * flux Jacobian at the Roe average of the conserved states Ua and Ub; rows
 * of Lm are l^(k), columns of Rm are r^(k), ordered u - a, u, (u), u + a. */
void orc_roe_eigen(int nv, double gamma, const double *Ua, const double *Ub, double *Lm, double *Rm);
/* Block tridiagonal system with m x m blocks (m <= 4) and ncol <= 4
 * right-hand sides: A[i] x[i-1] + B[i] x[i] + C[i] x[i+1] = r[i]; A, B, C
 * [n][m][m], r and x [n][m][ncol]; block Thomas elimination (reverse = 1
 * from i = n-1 downward).  Returns 0, or -1 on a singular pivot block. */
int orc_block_thomas(long n, int m, const double *A, const double *B, const double *C,
                     const double *r, int ncol, double *x, int reverse);
/* Cyclic block tridiagonal system (A[0] couples x[n-1], C[n-1] couples
 * x[0]), one right-hand side; Woodbury correction of block Thomas solves. */
int orc_block_cyclic(long n, int m, const double *A, const double *B, const double *C,
                     const double *r, double *x, int reverse);
/* Characteristic-wise compact-WENO reconstruction of one line of nv conserved
 * variables: ext [nv][n+4] with two ghost cells per side, um / up [nv][n]
 * as in orc_recon_scalar. */
int orc_recon_char(int nv, long n, const double *ext, int periodic, double gamma,
                   double eps_weno, int linear_weights, double *um, double *up);

/* HLLC flux with Batten wave speeds (Sec. 2.4, eqs. (HLLC), (contact-v),
 * (star-l), (acoustic ws)).  nv = 3: (rho, m, E); nv = 4: (rho, m_n, m_t, E)
 * with the tangential momentum carried by the contact. */
void orc_hllc(int nv, double gamma, const double *Ul, const double *Ur, double *F);
/* Local Lax-Friedrichs flux (the alternative Sec. 3 names for the near-vacuum
 * double rarefaction): F = (F(Ul) + F(Ur))/2 - alpha (Ur - Ul)/2 with alpha
 * the larger |u| + a of the two states (u normal to the face). */
void orc_llf(int nv, double gamma, const double *Ul, const double *Ur, double *F);
/* n faces at once; Ul, Ur, F are [n][nv] (test convenience). */
void orc_hllc_batch(int nv, double gamma, long n, const double *Ul, const double *Ur, double *F);
/* Physical flux F(U) in the normal direction. */
void orc_flux(int nv, double gamma, const double *U, double *F);

/* Zhang-Shu limiter of one cell (Sec. 2.4, steps 1-4).  ubar, um (= U^-_{j+1/2})
 * and up (= U^+_{j-1/2}) hold nv conserved values; um and up are limited in
 * place.  Returns bit 0 set if theta_1 < 1, bit 1 set if theta_2 < 1. */
int orc_limit_cell(int nv, double gamma, double wgl, double eps,
                   const double *ubar, double *um, double *up);

/* ---- whole-grid operator and time stepping ---- */
/* Spatial operator L(U) = -(F_{j+1/2} - F_{j-1/2})/dx (+ y part in 2-D),
 * eq. (1DEuler-FVCW).  eps is the limiter epsilon.  Returns 0 or -1. */
int orc_operator(const orc_grid *g, const double *U, double *L, double eps,
                 orc_counters *cnt);
/* L_x on the listed rows ([nr][nv][nx]) and L_y on the listed columns
 * ([nc][nv][ny]), grid variable order; for sampled checks of large grids. */
int orc_operator_lines(const orc_grid *g, const double *U, double eps, long nr, const long *rows,
                       long nc, const long *cols, double *Lx_rows, double *Ly_cols);
/* max over cells of (|u|+a)/dx (+ (|v|+a)/dy); negative if a state is invalid */
double orc_max_rate(const orc_grid *g, const double *U);
/* min over cells of the density average */
double orc_min_rho(const orc_grid *g, const double *U);
/* One SSP-RK3 step, eq. (RK3), limiter at every stage.  Returns 0 or -1. */
int orc_rk3_step(const orc_grid *g, double *U, double dt, orc_counters *cnt);
/* March from t0 to t_final with dt = cfl / max rate at each step start.
 * With g->face_cfl > 0 the cfl is capped at face_cfl, the rate is max(rate
 * of the cell averages, face rate of the last accepted step), and a step
 * whose stages' face rate r gives
 * dt r > face_cfl is redone from U^n with dt = cfl / r (Zhang-Shu restart).
 * Returns 0, -1 on a failed stage, -2 if max_steps was reached. */
int orc_advance(const orc_grid *g, double *U, double cfl, double t0, double t_final,
                long max_steps, double *t_out, long *steps_out, double *dt_last,
                orc_counters *cnt);

/* ---- exact Riemann solver (test reference, not part of the scheme) ---- */
/* Star-region pressure and velocity; *vacuum = 1 if the data generate vacuum. */
int orc_riemann_star(double gamma, const double *WL, const double *WR,
                     double *pstar, double *ustar, int *vacuum, int *iters);
/* Same star pressure by bisection only (cross-check of the Newton solve). */
double orc_riemann_star_bisect(double gamma, const double *WL, const double *WR);
/* Primitive state (rho, u, p) of the self-similar solution at xi = x/t. */
void orc_riemann_sample(double gamma, const double *WL, const double *WR, double xi,
                        double *W);
/* Exact cell averages of (rho, m, E) at time t on n cells of [x0, x1] with the
 * initial jump at xd, by nq-point Gauss-Legendre quadrature per cell (sub-split
 * nsub times).  U is [3][n]. */
void orc_riemann_cell_averages(double gamma, const double *WL, const double *WR,
                               double x0, double x1, long n, double xd, double t,
                               int nsub, double *U);

int orc_num_threads(void);
void orc_set_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
