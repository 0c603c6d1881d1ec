/*
 * pp_cweno.h -- C ABI of the GB300 (sm_103a) implementation of the
 * positivity-preserving fifth-order finite-volume compact-WENO scheme for
 * the compressible Euler equations (Guo, Xiong & Shi).
 *
 * The problem is the one the paper states (Sec. 1, eq. (1DEuler); Sec. 2.1):
 * conservative Euler equations of an ideal gas with ratio of specific heats
 * gamma, cell averages on a uniform grid, an SSP-RK3 time integrator whose
 * stages apply the spatial operator of Sec. 2.2-2.4 (WENO-Z weights on the
 * compact candidate stencils, tridiagonal solves, Zhang-Shu limiter, HLLC
 * flux, flux difference) and a time step dt = cfl / max((|u|+a)/dx) taken
 * from the cell averages at the start of each step (eq. (CFL-CD)).
 * The 2-D form is a dimension-by-dimension extension (the paper is 1-D):
 * the same line operator is applied along x and y and the two flux
 * differences are added; dt = cfl / max((|u|+a)/dx + (|v|+a)/dy).
 *
 * State layout (every pointer in this API): float64 structure of arrays
 *   U[v][j][i], i = 0..nx-1 fastest, j = 0..ny-1 (ny = 1 in 1-D),
 *   1-D: v = 0..2 -> (rho, rho*u, E)
 *   2-D: v = 0..3 -> (rho, rho*u, rho*v, E)
 * A batch concatenates the problems' arrays in the order of the configs,
 * each problem in the layout above.
 *
 * Ownership: a handle owns all device memory it allocates; the caller's
 * buffers are only copied from / to and never retained.  All work is
 * enqueued on the CUDA stream given at creation (NULL = legacy default
 * stream).  Host pointers need not be pinned.
 *
 * Errors: every function returns PP_OK (0) or one of the PP_ERR_* codes
 * below; none aborts, traps or prints.  pp_cweno_strerror() names a code.
 * A handle that returned PP_ERR_CUDA may be unusable; destroy it.
 */
#ifndef PP_CWENO_H
#define PP_CWENO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pp_cweno_s *pp_cweno_t;

/* Boundary conditions of one grid side.  Periodic sides must pair. */
typedef enum {
  PP_BC_PERIODIC = 0,
  PP_BC_TRANSMISSIVE = 1, /* zero-gradient ("Neumann"): ghosts copy the boundary cell */
  PP_BC_REFLECTIVE = 2    /* mirror ghosts, normal momentum negated */
} pp_bc_t;

/* Arithmetic of the line operator. */
typedef enum {
  PP_PREC_FP64 = 0,  /* everything in FP64 */
  PP_PREC_MIXED = 1  /* reconstruction, solves and HLLC in FP32; limiter
                        factors near vacuum and the stage accumulation of
                        the conserved variables in FP64 */
} pp_prec_t;

/* Numerical flux at the faces. */
typedef enum {
  PP_FLUX_HLLC = 0,  /* HLLC, Sec. 2.4 */
  PP_FLUX_LLF = 1    /* local Lax-Friedrichs: (F(Ul) + F(Ur))/2 - alpha (Ur - Ul)/2 with
                        alpha = max(|u_l| + a_l, |u_r| + a_r); the more dissipative
                        alternative Sec. 3 names for near-vacuum rarefactions */
} pp_flux_t;

/* Variables the compact-WENO reconstruction works on. */
typedef enum {
  PP_RECON_COMPONENT = 0,      /* each conserved variable on its own: one scalar
                                  tridiagonal system per variable and side (Sec. 2.2) */
  PP_RECON_CHARACTERISTIC = 1  /* characteristic variables of the Roe average at each
                                  face: one block tridiagonal system per side, blocks
                                  diag(a, b, c) L (Sec. 2.3, eq. (1DEuler-FVC)),
                                  in the line arithmetic of either precision.
                                  Single problems and batches
                                  (PP_ERR_UNSUPPORTED for
                                  pp_cweno_operator_noalloc); needs
                                  2 (n (nv^2 + nv) + nv^2) values per line of
                                  scratch per sweep direction (periodic: nv^2 +
                                  nv (nv+1) per row; FP64, or FP32 for the mixed
                                  form), plus 2 (4 nv + 4) n values of row
                                  data; a batch sizes both per group of lines
                                  by the group's longest line; a mixed 2-D
                                  problem keeps both directions' (and a
                                  second set of face-value planes), its y
                                  reconstruction running on a second stream
                                  beside the x sweep */
} pp_recon_t;

enum {
  PP_OK = 0,
  PP_ERR_ARG = 1,          /* bad sizes, gamma <= 1, cfl <= 0, unpaired periodic sides, ... */
  PP_ERR_STATE = 2,        /* set_state input not in the admissible set G or not finite */
  PP_ERR_NONPHYSICAL = 3,  /* a step produced a cell outside G (see stats.first_bad_cell) */
  PP_ERR_STEPS = 4,        /* advance stopped at max_steps before t_final */
  PP_ERR_TIMEOUT = 5,      /* a bounded device-side wait gave up */
  PP_ERR_CUDA = 6,         /* a CUDA runtime call failed */
  PP_ERR_UNSUPPORTED = 7   /* configuration outside what this library supports */
};

typedef struct {
  int ndim;                /* 1 or 2 */
  int64_t nx, ny;          /* cells; ny is ignored (1) when ndim == 1; each >= 8 */
  double x0, x1, y0, y1;   /* domain [x0,x1] (x [y0,y1]) */
  double gamma;            /* > 1 */
  double cfl;              /* dt = cfl / max((|u|+a)/dx [+ (|v|+a)/dy]) */
  int bc[4];               /* pp_bc_t of x-lo, x-hi, y-lo, y-hi */
  int precision;           /* pp_prec_t */
  double gl_weight;        /* Gauss-Lobatto end weight omega_hat_1 of the limiter, Sec. 2.4 (1/12) */
  double eps_weno;         /* epsilon of the WENO-Z weights, eq. (weight) (1e-13); the mixed
                              form adds 2^20 (u max|ubar|)^2 over each 5-cell stencil
                              (u = 2^-24): the indicators' floor of FP32 rounding noise,
                              including the noise the FP32 stages accumulate in the state */
  double eps_pos;          /* cap of the limiter epsilon, Sec. 2.4 step 1 (1e-13) */
  int cfl_positivity_cap;  /* 1: enforce eq. (CFL-CD) of the theorem of Sec. 2.4 on the states
                              its first-order steps act on, the limited face values:
                              dt = min(cfl, gl_weight / 2) / max(rate of the cell averages,
                              face rate of the last accepted step), and a step whose stages'
                              face values have dt max((|u|+a)/dx [+ (|v|+a)/dy]) > gl_weight
                              is redone from U^n with dt = min(cfl, gl_weight / 2) / that
                              rate (half its dt if a stage had no finite rate); the
                              factor 1/2 is the first-order positivity CFL that brute
                              force supports (the Sec. 2.4 remark states 1).  Batches:
                              the same value for every problem */
  int limiter;             /* 1: Zhang-Shu limiter on (default); 0: off */
  int flux;                /* pp_flux_t: face flux (PP_FLUX_HLLC default) */
  int recon;               /* pp_recon_t: reconstructed variables (PP_RECON_COMPONENT default) */
} pp_cweno_config;

typedef struct {
  int64_t steps;           /* completed SSP-RK3 steps since set_state */
  int64_t stages;          /* completed stages */
  int64_t theta1_active;   /* cell-sweeps with theta_1 < 1 (density limited) */
  int64_t theta2_active;   /* cell-sweeps with theta_2 < 1 (internal energy limited) */
  int64_t violations;      /* cells found outside G after a stage */
  int64_t first_bad_cell;  /* flat cell index of one violation, -1 if none */
  double t;                /* simulation time */
  double last_dt;          /* last time step */
  double max_rate;         /* max (|u|+a)/dx (+(|v|+a)/dy) at the current state */
  double min_rho;          /* min density average at the current state */
  int64_t rejected;        /* checked steps redone with a smaller dt (cfl_positivity_cap) */
} pp_cweno_stats_t;

/* Fill *cfg with the defaults above (1-D, periodic, FP64, gamma 1.4, cfl 0.5). */
int pp_cweno_config_default(pp_cweno_config *cfg);

/* Create a solver for one problem; allocates device memory sized for it.
 * cuda_stream: a cudaStream_t or NULL.  On failure *out is NULL. */
int pp_cweno_create(const pp_cweno_config *cfg, void *cuda_stream, pp_cweno_t *out);

/* Create one handle for nprob independent problems advanced together (each
 * with its own time step).  All configs must share ndim, gamma, precision,
 * the limiter settings, the flux and the reconstruction (PP_ERR_ARG
 * otherwise); sizes, domains, boundaries and cfl may differ. */
int pp_cweno_create_batch(const pp_cweno_config *cfgs, int64_t nprob, void *cuda_stream,
                          pp_cweno_t *out);

/* Copy initial cell averages in (layout above; on_device != 0: U is a
 * device pointer), set t = t0 and the step count to 0, check every cell is
 * finite and in G, the admissible set rho > 0, p > 0 of Sec. 2.4
 * (PP_ERR_STATE otherwise), and take the first step's limiter epsilon
 * eps = min(eps_pos, min rho) (Sec. 2.4 limiter, step 1) and the first dt
 * (eq. (CFL-CD)) from it.  Synchronises the stream. */
int pp_cweno_set_state(pp_cweno_t h, const double *U, int on_device, double t0);

/* Copy the current state out; t and steps may be NULL.  Synchronises. */
int pp_cweno_get_state(pp_cweno_t h, double *U, int on_device, double *t, int64_t *steps);

/* One SSP-RK3 step (eq. (RK3), Sec. 2.5: three stages, each one evaluation
 * of the FVCW operator L with the positivity limiter of Sec. 2.4) with
 * dt = min(cfl-limited dt, dt_max), the cfl-limited dt being
 * cfl h / max(|u| + a) (eq. (CFL-CD)); *dt_taken may be NULL.
 * Synchronises.  Batch handles: every problem takes one step.  With
 * cfl_positivity_cap a step that fails the face check is redone (up to 64
 * attempts) until it is accepted. */
int pp_cweno_step(pp_cweno_t h, double dt_max, double *dt_taken);

/* March every problem with SSP-RK3 steps (eq. (RK3), Sec. 2.5; dt as in
 * pp_cweno_step) until its t reaches t_final (the last step is cut to
 * land on it), or until max_steps steps were taken (PP_ERR_STEPS).  Steps
 * are replayed from a captured CUDA graph; the host reads the device-side
 * progress flags once per replay.  *steps_taken (may be NULL) receives the
 * steps of this call (the maximum over problems for a batch). */
int pp_cweno_advance(pp_cweno_t h, double t_final, int64_t max_steps, int64_t *steps_taken);

/* Enqueue exactly nsteps steps on the handle's stream with no host
 * synchronisation and no stopping time (for timing); errors are reported by
 * the next synchronising call.  With cfl_positivity_cap a rejected step is
 * one of the nsteps (stats.rejected counts them). */
int pp_cweno_enqueue_steps(pp_cweno_t h, int64_t nsteps);

/* Evaluate the spatial operator once: L = L(U) (eq. (1DEulerFV-b); in 2-D
 * L_x + L_y) with limiter epsilon eps (eps <= 0: min(eps_pos, min rho)).
 * U and L are device pointers in the state layout; single-problem handles
 * only.  Synchronises. */
int pp_cweno_operator(pp_cweno_t h, const double *U_dev, double *L_dev, double eps);

/* Statistics; synchronises.  For a batch, sums and extrema over problems. */
int pp_cweno_stats(pp_cweno_t h, pp_cweno_stats_t *out);

/* Statistics of problem k of a batch (k = 0 for a single problem): its
 * steps, time, limiter counts and violations (first_bad_cell indexes the
 * problem's own cells); max_rate and min_rho are not filled (0).
 * Synchronises. */
int pp_cweno_problem_stats(pp_cweno_t h, int64_t k, pp_cweno_stats_t *out);

/* Number of problems in the handle and the cell count of problem k. */
int pp_cweno_num_problems(pp_cweno_t h, int64_t *nprob);
int pp_cweno_problem_cells(pp_cweno_t h, int64_t k, int64_t *ncell);

/* Rows per thread chunk of the line kernels chosen for this handle (8 or
 * 16: the serial Thomas run of a thread against the depth of the parallel
 * scans).  The first set_state of a handle times one sweep with each choice
 * on the handle's own data and keeps the faster: single problems over the x
 * sweep (cached per precision, dimension, grid size and periodicity),
 * batches over every x-line group of the batch. */
int pp_cweno_rows_per_chunk(pp_cweno_t h, int *m);

/* Kernel launches enqueued per step (for launch accounting). */
int pp_cweno_launches_per_step(pp_cweno_t h, int64_t *n);

/* Measurement: enqueue one step launch by launch with CUDA events on the
 * handle's stream between kernels, synchronise and return each kernel's
 * duration in ms (ms[0] the dt kernel, then the sweeps in launch order; a
 * characteristic-wise handle's sweep is preceded by its rows and block-solve
 * kernels, each timed on its own) in ms[0..*nk-1] (at most nmax entries). */
int pp_cweno_profile_step(pp_cweno_t h, float *ms, int nmax, int *nk);

/* Measurement: sustained fused multiply-add throughput of this GPU's CUDA
 * cores in GFLOP/s (2 flops per FMA), FP64 if fp64 != 0 else FP32, from a
 * dependent-chain-free kernel filling every SM.  Synchronises. */
int pp_cweno_fma_peak(int fp64, double *gflops);

/* The spatial operator of one FP64 problem with no device allocation at all
 * (the paper has no counterpart; this is a service of this library).
 *
 * For callers that cannot call cudaMalloc: code that runs while a CUDA graph
 * is being captured, inside a fixed memory budget or a pool that must not
 * grow, or in a loop that may not synchronise the device (cudaMalloc and
 * cudaFree can).  Such a caller passes its own U and L (device pointers,
 * FP64 planes in the state layout) and gets L = L(U) as pp_cweno_operator
 * computes it, with the same kernels; cfg describes the grid as for
 * pp_cweno_create and must select PP_PREC_FP64.  eps > 0 is the limiter
 * epsilon; eps <= 0 takes min(eps_pos, min rho) on the device, and then a
 * state with a cell outside G is not evaluated: the call still returns
 * PP_OK (it does not synchronise) and L is filled with NaN.  A pending
 * CUDA error left by the caller's own work is not cleared; the call then
 * returns PP_ERR_CUDA without launching anything.
 *
 * Scratch: the x-sweep flux difference and a control block live in one
 * fixed 32 MiB device array inside the library (every GPU that loads the
 * library holds it until exit), so a 2-D grid may have at most
 * (32 MiB - 256 B) / 32 B, about 1.05 million cells (1024 x 1023); larger
 * grids return PP_ERR_UNSUPPORTED.  1-D grids need no scratch beyond the
 * control block.  Every call shares the array: calls whose work overlaps on
 * the GPU (other streams, other host threads on the same device) race.  The
 * first call on a device resolves the array's device address and sets the
 * kernels' launch attributes with that device current; make it before any
 * stream capture.  The work is enqueued on cuda_stream (NULL = legacy
 * default stream) and the call returns without synchronising. */
int pp_cweno_operator_noalloc(const pp_cweno_config *cfg, const double *U_dev, double *L_dev,
                              double eps, void *cuda_stream);

/* Free all device memory of the handle (h may be NULL). */
int pp_cweno_destroy(pp_cweno_t h);

const char *pp_cweno_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* PP_CWENO_H */
