/*
 * elder.h -- C ABI of the GB300 implicit time step for the stochastic 3D
 * Elder-like density-driven flow problem (Litvinenko, Logashenko, Tempone,
 * Wittum, Keyes, arXiv:1906.01632).
 *
 * Model (Section 2.1): fluid mass conservation (eq. e_cont_eq), salt
 * transport (eq. e_tran_eq), Darcy law q = -(K/mu)(grad p - rho(c) g) with
 * g = (0,0,-g) (eq. e_Darcy_vel), scalar permeability (eq. e_scalar_perm),
 * linear density rho(c) = rho0 + (rho1-rho0) c (eq. e_lin_density), constant
 * viscosity, molecular diffusion phi*Dm (eq. e_mol_diff).
 * Discretisation and solver (Section 2.3, Section 5.1): vertex-centred finite
 * volumes on a structured hexahedral box, implicit Euler, Newton with line
 * search, BiCGStab preconditioned by a geometric-multigrid V-cycle whose
 * coarse matrices are the Jacobians of the discretised system on each grid.
 *
 * Conventions shared by every entry point
 * --------------------------------------
 *  - Grid: nodes (i,j,k), 0<=i<=nx, 0<=j<=ny, 0<=k<=nz, at x = i*Lx/nx,
 *    y = j*Ly/ny, z = k*Lz/nz; z points up (the top is z = Lz).
 *    N = (nx+1)(ny+1)(nz+1) nodes, C = nx*ny*nz cells.
 *  - Node arrays are [S][N] with n = i + (nx+1)*(j + (ny+1)*k) (x fastest);
 *    cell arrays are [S][C] with e = i + nx*(j + ny*k).
 *  - Pairs of unknowns/residual rows are interleaved [S][N][2] = (p, c).
 *  - All array arguments are DEVICE pointers owned by the caller unless a
 *    comment says "host"; the library never frees them.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *    stream-ordered; entry points that return per-sample status synchronise
 *    the stream before returning.
 *  - Every function returns an elder_status code; none throws.  After a
 *    failure, elder_last_error() describes it.  A context may be used by one
 *    host thread at a time.
 */
#ifndef ELDER_H
#define ELDER_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ELDER_OK = 0,
    ELDER_EINVAL = 1,    /* bad argument or unsupported grid              */
    ELDER_ENOMEM = 2,    /* device allocation failed                      */
    ELDER_ECUDA = 3,     /* a CUDA call failed                            */
    ELDER_ENOTCONV = 4,  /* at least one sample failed: see its status    */
    ELDER_ETIMEOUT = 5   /* a bounded device wait gave up                 */
} elder_status;

/* per-sample status of elder_step / elder_solve */
enum {
    ELDER_SAMPLE_OK = 0,
    ELDER_SAMPLE_NEWTON_MAXIT = 1,  /* Newton iteration cap reached        */
    ELDER_SAMPLE_KRYLOV_MAXIT = 2,  /* BiCGStab cap reached (elder_solve)  */
    ELDER_SAMPLE_BREAKDOWN = 3,     /* BiCGStab breakdown (rho or omega 0) */
    ELDER_SAMPLE_NONFINITE = 4,     /* NaN/Inf in a residual norm          */
    ELDER_SAMPLE_LINESEARCH = 5     /* no step length decreased ||R||      */
};

enum { ELDER_FP64 = 0, ELDER_MIXED = 1 };

/* multigrid smoothers (Section 5.1) */
enum { ELDER_SMOOTH_JACOBI = 0, ELDER_SMOOTH_ZLINE = 1, ELDER_SMOOTH_ILU = 2 };

/* Boundary-condition sets (Section 2.1 and the caption of Fig. 1):
 *  0 benchmark: c=1 on the closed top square [Lx/4,3Lx/4]x[Ly/4,3Ly/4],
 *    c=0 on the bottom, p=0 at the four top corners; no-flow elsewhere;
 *  1 paper variant: c=1 on the top square, c=0 on the rest of the top and
 *    on the bottom, p=0 on the four top edges;
 *  2 diffusion column test: c=1 on the whole top, c=0 on the bottom,
 *    p=0 at the four top corners;
 *  3 no c Dirichlet data, p=0 at the four top corners. */
typedef struct {
    int nx, ny, nz;           /* cells; for modes 0/1 nx, ny multiples of 4 */
    double Lx, Ly, Lz;        /* box size [m]                               */
    double rho0, rho1;        /* densities of water and brine [kg/m^3]      */
    double mu;                /* viscosity [Pa s]                           */
    double g;                 /* gravity [m/s^2], acting along -z           */
    double Dm;                /* molecular diffusion [m^2/s]                */
    int bc_mode;              /* see above                                  */
    int precision;            /* ELDER_FP64 or ELDER_MIXED                  */
    int max_samples;          /* largest S any call will pass               */
    /* Newton with line search (Section 2.3) */
    int newton_maxit;         /* iteration cap                              */
    double newton_tol_c;      /* converged: max|dc| <= tol_c ...            */
    double newton_tol_p;      /* ... and max|dp| <= tol_p at a full step    */
    int ls_max;               /* step halvings before the sample's line
                                 search fails (status LINESEARCH)           */
    /* BiCGStab (Section 5.1) */
    double lin_rtol;          /* relative residual target per Newton solve
                                 (default 1e-2: inexact Newton)             */
    int lin_maxit;            /* iteration cap                              */
    /* geometric multigrid V-cycle (Section 5.1) */
    int mg_levels;            /* 0 = coarsen as far as the grid allows      */
    int nu1, nu2;             /* pre/post smoothing sweeps (default 1, 0:
                                 V(1,0); the robust re-solve of failed
                                 samples uses at least one post-sweep)      */
    double omega;             /* damping of the point block-Jacobi smoother
                                 (default 0.5)                              */
    int coarse_K_harmonic;    /* 0 arithmetic, 1 harmonic mean of K         */
    int use_graphs;           /* 0: every kernel launched from the host;
                                 1: the BiCGStab iteration replayed as a
                                 captured CUDA graph, the host polling the
                                 per-sample flags between iterations;
                                 2 (default): the whole step is one captured
                                 graph whose Newton, BiCGStab and line-search
                                 loops are conditional while nodes driven by
                                 the per-sample flags on the device (the
                                 host launches it and reads the results
                                 once); used from a context's second step
                                 on (the first tunes block sizes), for the
                                 configured settings, outside profiling, and
                                 cached for the 4 most recent argument sets
                                 (array pointers, S, dt, Newton start)      */
    int autotune;             /* 1 (default): time the candidates (threads
                                 per block; for the multigrid residual and
                                 the z-line sweep also 1 or 2 samples per
                                 CTA) of the stencil kernels on the first
                                 step; 0: defaults (one sample per CTA);
                                 2: two samples per CTA without timing     */
    int newton_estimate;      /* also accept when the linear-convergence
                                 error estimate theta/(1-theta)|d| is within
                                 the Newton tolerances                      */
    int smoother;             /* ELDER_SMOOTH_JACOBI: damped 2x2 block
                                 Jacobi; ELDER_SMOOTH_ZLINE: damped block
                                 Jacobi over vertical grid lines (block
                                 tridiagonal solve per line, nz <= 128;
                                 the default); ELDER_SMOOTH_ILU: the
                                 multicolour block ILU_beta(0) of the
                                 paper's smoother ILU_beta (factors of each
                                 level's interior operator in the 8-colour
                                 node order, colour (i&1)+2(j&1)+4(k&1);
                                 fill outside the 27-point block pattern
                                 dropped, beta times it subtracted from the
                                 row's diagonal block; a sweep is x += omega
                                 (L U)^{-1}(b - A x), and (L U)^{-T} in the
                                 transposed solves).  The robust re-solve of
                                 failed samples always uses the z-line
                                 smoother (damping 0.5).                    */
    double omega_line;        /* damping of the z-line smoother (default
                                 0.95)                                      */
    int mixed_newton_maxit;   /* Newton iteration cap of the ELDER_MIXED
                                 solve only (0: newton_maxit).  A sample that
                                 reaches it is solved again in FP64 with
                                 newton_maxit; a cap of 1 forces that FP64
                                 re-solve from the host (failure-tier test) */
    double ilu_beta;          /* beta of ELDER_SMOOTH_ILU (default 0: block
                                 ILU(0); 1: modified ILU, whose pivots are
                                 nearly singular on this system because the
                                 pressure rows sum to about 0)              */
    double omega_ilu;         /* damping of the ILU sweep (default 1)       */
} elder_config;

/* Per-sample statistics of one elder_step call (host struct). */
typedef struct {
    int32_t status;           /* ELDER_SAMPLE_*                             */
    int32_t newton_iters;
    int32_t krylov_iters;     /* summed over the Newton iterations          */
    int32_t ls_cuts;          /* step halvings                              */
    double res0;              /* ||R(u^n)||_2 with Dirichlet data imposed   */
    double res;               /* ||R||_2 of the last iterate whose residual
                                 was evaluated: u^{n+1}, or its predecessor
                                 when Newton stopped on the size of the
                                 last full correction (whose residual is
                                 then not evaluated)                        */
    int32_t fp64_retry;       /* 0: solved by the configured solver; 1: the
                                 ELDER_MIXED solve failed and the step was
                                 solved again from u^n with the FP64 solver;
                                 2: that failed too and a last FP64 solve
                                 with robust settings was made (z-line
                                 smoother, Krylov rtol <= 1e-6 keeping its
                                 best iterate,
                                 >= 2000 Krylov and >= 50 Newton
                                 iterations, >= 16 step halvings)           */
    int32_t pad;
    /* FP64 salt-mass balance of the step: M = sum_e sum_corners phi_e
     * |scv| rho(c) c at u^n and at the returned state, and the salt that
     * entered through the c-Dirichlet nodes (dt times their net face
     * inflow); at convergence salt_mass - salt_mass0 = salt_inflow up to
     * the Newton tolerance. */
    double salt_mass0, salt_mass, salt_inflow;
} elder_stats;

typedef struct elder_ctx elder_ctx;

/* Fills *cfg with the benchmark problem of Table 1 on an nx*ny*nz grid and
 * default solver settings.  Dm = 3.565e-6 m^2/s, the classic Elder value:
 * Table 1 prints 0.565e-6, read as a dropped leading digit (both densities,
 * the viscosity, K and phi of the table are the classic Elder values too).
 * Returns ELDER_EINVAL for a NULL cfg. */
int elder_config_default(elder_config* cfg, int nx, int ny, int nz);

/* Creates a context: validates the grid, builds the multigrid hierarchy and
 * allocates all device workspace for up to cfg->max_samples samples on the
 * current device.  *out receives the handle (NULL on failure). */
int elder_create(const elder_config* cfg, elder_ctx** out);

/* Frees the context and its device workspace (NULL is accepted). */
int elder_destroy(elder_ctx* ctx);

/* Message of the last failure on ctx (or, when ctx is NULL, of the last
 * failed elder_create or context-free call of this thread); never NULL. */
const char* elder_last_error(const elder_ctx* ctx);

/* Number of nodes N and cells C of the context's grid (host outputs). */
int elder_sizes(const elder_ctx* ctx, int64_t* N, int64_t* C, int* levels);

/* Sample preprocessing (Section 2.2, eq. e_perm_Kozeny_Carman): per-cell
 * porosity and permeability for S samples.
 *  kind 0: params = xi [S][3] in [-1,1]^3, phi = 0.1*(1 + 0.3*(xi1 cos(pi
 *          x/Lx) + xi2 cos(pi y/Ly) + xi3 sin(2 pi z/Lz))/3) at cell centres;
 *  kind 1: params = Z [S][C] standard normals, phi = clip(0.1 exp(0.2 Z),
 *          0.05, 0.2);
 *  kind 2: params = xi [S][3], the paper's field eq. poro-paral3RVS.
 * K = K_mean * [phi^3/(1-phi)^2] / [0.1^3/0.9^2] (Kozeny-Carman normalised so
 * that K(0.1) = K_mean).  phi, K: [S][C] device outputs. */
int elder_fields(elder_ctx* ctx, int S, int kind, const double* params,
                 double K_mean, double* phi, double* K, void* stream);

/* Residual R(u; u_old) of the implicit Euler step (eqs. e_cont_eq,
 * e_tran_eq, box-method fluxes), FP64, for S samples.  R: [S][N][2] device
 * output; Dirichlet rows hold u - u_D.  Used by the parity tests. */
int elder_residual(elder_ctx* ctx, int S, const double* phi, const double* K,
                   const double* p, const double* c, const double* p_old,
                   const double* c_old, double dt, double* R, void* stream);

/* Jacobian dR/du at (p, c) on the finest grid in the library's storage:
 * J[S][27][N][4], slot s = (dx+1) + 3(dy+1) + 9(dz+1) for the neighbour at
 * offset (dx,dy,dz), block (row p|c, col p|c) = {pp, pc, cp, cc}; entries
 * of neighbours outside the grid are 0; Dirichlet rows are identity rows.
 * FP64 output regardless of precision (Section 5.1: "assembled as the
 * Jacobians of the discretized nonlinear systems"). */
int elder_jacobian(elder_ctx* ctx, int S, const double* phi, const double* K,
                   const double* p, const double* c, double dt, double* J,
                   void* stream);

/* One implicit Euler step for S samples (Sections 2.3 and 5.1): Newton with
 * line search on the FP64 residual, each Newton system solved by
 * multigrid-preconditioned BiCGStab (FP64, or FP32 multigrid and Krylov
 * storage with FP64 inner products in ELDER_MIXED).  In ELDER_MIXED a
 * sample whose Newton iteration fails is solved again from u^n with the
 * FP64 solver (packed into batches of at most 32 samples and at most 2^25
 * node-samples).
 *  phi, K: [S][C] inputs.  p, c: [S][N] in: u^n, out: u^{n+1}.
 *  dt: time step [s].  status, stats: HOST arrays of S entries (stats may
 *  be NULL), written after the stream is synchronised.  A failed sample
 *  keeps u^n.  Returns ELDER_ENOTCONV when any sample failed. */
int elder_step(elder_ctx* ctx, int S, const double* phi, const double* K,
               double* p, double* c, double dt, int32_t* status,
               elder_stats* stats, void* stream);

/* elder_step starting Newton from the linear extrapolation 2 u^n - u^{n-1}
 * (c clipped to [0, 1], Dirichlet values imposed) instead of u^n: the same
 * implicit Euler step (Sections 2.3 and 5.1) to the same Newton tolerance,
 * with fewer Newton iterations when the solution evolves smoothly (about
 * half an iteration per step on the 64x64x16 Sobol batch; elder_step_predicted
 * order 2 saves a little more).  p_prev, c_prev: [S][N] in: u^{n-1} (pass u^n on the first
 * step), out: u^n, so that repeated calls with the same four buffers march
 * in time.  p, c: in u^n, out u^{n+1}.  Re-solves of failed samples start
 * from u^n; a failed sample keeps u^n.  Other arguments as elder_step. */
int elder_step_extrapolated(elder_ctx* ctx, int S, const double* phi, const double* K,
                            double* p_prev, double* c_prev, double* p, double* c,
                            double dt, int32_t* status, elder_stats* stats,
                            void* stream);

/* elder_step starting Newton from a polynomial extrapolation of the last
 * states (c clipped to [0, 1], Dirichlet values imposed): order 1 the linear
 * 2 u^n - u^{n-1} (as elder_step_extrapolated), order 2 the quadratic
 * 3 u^n - 3 u^{n-1} + u^{n-2}.  The same implicit Euler step (Sections 2.3
 * and 5.1) to the same Newton tolerance.
 *  p_hist, c_hist: [order][S][N] history levels, in: (u^{n-1}[, u^{n-2}])
 *  (pass u^n in every level on the first step), out: (u^n[, u^{n-1}]), so
 *  that repeated calls with the same buffers march in time.  p, c: in u^n,
 *  out u^{n+1}.  Re-solves of failed samples start from u^n; a failed
 *  sample keeps u^n.  Other arguments as elder_step; order outside {1, 2}
 *  returns ELDER_EINVAL. */
int elder_step_predicted(elder_ctx* ctx, int S, const double* phi, const double* K, int order,
                         double* p_hist, double* c_hist, double* p, double* c, double dt,
                         int32_t* status, elder_stats* stats, void* stream);

/* Linearises at (p, c) and solves J x = rhs (transpose=0) or J^T x = rhs
 * (transpose=1) with the multigrid-preconditioned BiCGStab of elder_step,
 * to the relative residual rtol.  rhs, x: [S][N][2] device; x is output
 * only.  status: HOST [S].  The FP64 solver is used for rtol < 1e-6. */
int elder_solve(elder_ctx* ctx, int S, const double* phi, const double* K,
                const double* p, const double* c, double dt, int transpose,
                const double* rhs, double* x, double rtol, int32_t* status,
                void* stream);

/* One application of a multigrid smoother's preconditioner on the finest
 * level (Section 5.1), linearised at (p, c) with time step dt: z = P^{-1} r
 * (transpose = 0) or P^{-T} r (transpose = 1) on the interior unknowns of
 * the Jacobian (Dirichlet rows and columns replaced by the identity), with
 * P the 2x2 block diagonal (kind ELDER_SMOOTH_JACOBI), the block-tridiagonal
 * part along vertical grid lines (kind ELDER_SMOOTH_ZLINE, nz <= 128) or
 * L U of the multicolour block ILU_beta(0) factors with beta = cfg ilu_beta
 * (kind ELDER_SMOOTH_ILU; the transposed application uses the factors of
 * the untransposed operator).  Every kind needs no configuration: the
 * factors are formed for the call.  Computed in the context's multigrid
 * precision: FP64, or in ELDER_MIXED bfloat16 matrices and factors with
 * FP32 arithmetic and vectors.  r, z: [S][N][2] device (p, c interleaved);
 * Dirichlet components of r are ignored, those of z are 0.  Used by the
 * parity tests of the smoothers. */
int elder_smoother_apply(elder_ctx* ctx, int S, const double* phi, const double* K,
                         const double* p, const double* c, double dt, int kind,
                         int transpose, const double* r, double* z, void* stream);

/* Sample statistics over S fields c[S][N] (Section 3, eqs. pdestat and
 * numer_var, and the exceedance estimate of Section 3.3):
 * mean = sum_i w_i c_i, var = sum_i w_i (mean - c_i)^2,
 * p_exceed = sum_i w_i [c_i > threshold].  w: [S] device weights or NULL for
 * 1/S.  mean, var, p_exceed: [N] device outputs. */
int elder_moments(elder_ctx* ctx, int S, const double* c, const double* w,
                  double threshold, double* mean, double* var,
                  double* p_exceed, void* stream);

/* Discrete adjoint of n_steps implicit Euler steps of one sample from
 * (p0, c0): objective J = salt mass sum_e phi_e |scv| rho(c) c over the
 * cells whose centre lies below Lz/2 at the final time, and its gradients
 * with respect to per-cell phi and K (independent inputs).  Forward states
 * are kept every ckpt_every steps and recomputed in the reverse sweep.
 *  J_out: HOST double.  dJ_dphi, dJ_dK: [C] device outputs. */
int elder_grad(elder_ctx* ctx, int n_steps, const double* phi,
               const double* K, const double* p0, const double* c0, double dt,
               int ckpt_every, double* J_out, double* dJ_dphi, double* dJ_dK,
               void* stream);

/* Initial state of the benchmark problem (Section 2.1): c = its Dirichlet
 * value on c-Dirichlet nodes and 0 elsewhere; p = rho0 g (Lz - z), the
 * hydrostatic pressure of pure water, which only seeds Newton (p has no time
 * derivative).  p, c: [S][N] device outputs. */
int elder_initial_state(elder_ctx* ctx, int S, double* p, double* c,
                        void* stream);

/* ---- measurement (no counterpart in the paper) ------------------------ */

/* Kernel classes timed by elder_profile. */
enum {
    ELDER_K_SMOOTH = 0,     /* block-Jacobi sweeps with a nonzero iterate   */
    ELDER_K_SPMV = 1,       /* BiCGStab stencil products (+ inner products) */
    ELDER_K_MGRES = 2,      /* multigrid residuals b - A x                  */
    ELDER_K_RESIDUAL = 3,   /* FP64 Newton residual                         */
    ELDER_K_JACOBIAN = 4,   /* Jacobian assembly, all levels                */
    ELDER_K_SMOOTH0 = 5,    /* first sweep from a zero iterate              */
    ELDER_K_CLASSES = 6
};

/* on=1 resets the counters and brackets every launch of the classes above
 * with CUDA events on the launching stream (CUDA-graph replay is bypassed
 * while profiling); on=0 stops.  Event times are drained at the host
 * synchronisation points the step already has. */
int elder_profile(elder_ctx* ctx, int on);

/* Totals since elder_profile(ctx, 1) for one class: launches, summed event
 * time [ms], algorithmic DRAM bytes and FP64/FP32 flops of those launches.
 * Bytes = per-node model x nodes x samples active in the launch; the model
 * counts every array the kernel must touch once (neighbour reuse of a
 * vector is free).  Per node, with T the vector entry size (8 FP64, 4
 * mixed) and Mz the multigrid matrix entry size (8 FP64, 2 mixed):
 *   SMOOTH  108 Mz + 10 T + 1    SMOOTH0  8 T + 1 (+ 8 Mz z-line)
 *   SPMV    108 T  + 6 T + 1     MGRES    108 Mz + 6 T + 1
 *   RESIDUAL 49 + 16 C/N         JACOBIAN 108 T + 108 Mz + 4 T + 17 + 16 C/N
 * (the Jacobian writes the Krylov and the multigrid copies of J and the
 * inverse diagonal blocks; the residual reads p, c, c_old, phi, K and writes
 * R).  Flops: the FP64 residual counts 266 C/N + 75 of its factored face
 * form, the stencil products 216 + their vector terms.  Any output pointer
 * may be NULL.  Host outputs. */
int elder_profile_read(const elder_ctx* ctx, int kernel_class,
                       int64_t* launches, double* ms, double* bytes,
                       double* flops);

/* Number of kernels this library has launched in the process (graph
 * replays count every kernel node, the loop bodies of a device-controlled
 * step as often as they ran).  Host output. */
int elder_launch_count(int64_t* launches);

/* The autotuner's choice for one kernel class (ELDER_K_*): threads per
 * block and samples per CTA (1, or 2: each thread works on its node or line
 * in two samples, whose loads and recursions are independent).  For
 * ELDER_K_MGRES (the multigrid residual; candidates 128, 256, 512 threads)
 * and ELDER_K_SMOOTH0 (the z-line sweep from x = 0; candidates 64, 128, 256
 * threads) ms receives the measured milliseconds per launch of the 6
 * candidates [samples per CTA 1, 2][threads ascending], 0 when not tuned;
 * for the other classes 0.  Timed on the first step of a context (3
 * launches after a warm-up, CUDA events) on its level-0 operator with all
 * samples active.  Host outputs; any may be NULL. */
int elder_autotune_choice(const elder_ctx* ctx, int kernel_class, int* threads_per_block,
                          int* samples_per_cta, float* ms);

/* Device-controlled steps of ctx (use_graphs = 2): *cached receives the
 * number of captured step graphs held, *replays the steps run through them
 * since the context was created, and *note (may be NULL) the reason the
 * context fell back to host-driven steps ("" while it has not).  Host
 * outputs; the note stays valid until the next call on ctx. */
int elder_graph_status(const elder_ctx* ctx, int* cached, int64_t* replays, const char** note);

/* Threads per block chosen by the autotuner for the smoother, the Krylov
 * stencil product and the multigrid residual (256 until the first step has
 * run), and the measured milliseconds per launch of every candidate
 * (ms[3][3]: class x {128, 256, 512}, 0 when not tuned).  Host outputs; any
 * may be NULL. */
int elder_autotune_result(const elder_ctx* ctx, int* bs_smooth, int* bs_spmv,
                          int* bs_mgres, float* ms);

/* Measured arithmetic peak of the current device: kind 0 FP64 fused
 * multiply-adds, kind 1 FP32 fused multiply-adds.  A kernel of 8
 * independent FMA chains per thread on 8 resident blocks of 256 threads per
 * SM is timed with CUDA events on `stream` (best of 3 launches after a
 * warm-up); *gflops receives 2 x FMAs / time in GFLOP/s (host output).
 * Allocates and frees one small device buffer; synchronises the stream. */
int elder_measure_peak(int kind, double* gflops, void* stream);

/* ---- allocation-free entry point (no counterpart in the paper) -------- */

/* The residual of elder_residual plus its per-sample 2-norm, for callers
 * that may not allocate device memory at all: it needs no context (which
 * would allocate the solver workspace) and calls no cudaMalloc, cudaFree or
 * allocating library routine.  Typical callers: code running after another
 * runtime has taken over the device's memory pool, or a thread that may only
 * enqueue work.
 *  cfg: host pointer; its grid, physics constants and bc_mode are used
 *  (the Dirichlet sets are evaluated from the node indices).
 *  phi, K: [S][C]; p, c, p_old, c_old: [S][N] device inputs.
 *  R: [S][N][2] device output, the same values as elder_residual's.
 *  norms: [S] device output, ||R_s||_2.
 * Scratch: the per-block partial sums live in a file-scope device array of
 * 262144 doubles (2 MiB), which every GPU that loads the library holds until
 * the process exits.  S * ceil(N/256) must not exceed 262144, otherwise
 * ELDER_EINVAL is returned before anything is launched, as it is for
 * S > 65535 (samples run along the launch grid's y dimension).  The first
 * call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current.  With CUDA's lazy module
 * loading (the default since CUDA 12.2) that first lookup is also what
 * loads the library's device code and reserves the 2 MiB array on that
 * device, i.e. it may allocate device memory once.  So make the first call
 * on each device early: before another runtime takes the device's memory
 * and before any stream capture.  Later calls allocate nothing.
 * Every call shares the array and overwrites the entries it uses (nothing
 * in it has to start at zero); calls that overlap on the GPU race on it.
 * Errors: elder_last_error(NULL). */
int elder_residual_norms_static(const elder_config* cfg, int S,
                                const double* phi, const double* K,
                                const double* p, const double* c,
                                const double* p_old, const double* c_old,
                                double dt, double* R, double* norms,
                                void* stream);

/* ------------------------------------------------------------------------
 * gPC surrogate (Section 3: truncated expansion eq. PCEdecom2, projection
 * eq. PCEcoef, mean eq. PCEcoef2, variance eq. var, surrogate evaluation
 * eq. PCEpoint and the exceedance estimate; Appendix A: Legendre basis of
 * uniform variables on [-1, 1]).  Context-free; errors are reported through
 * elder_last_error(NULL).
 * ---------------------------------------------------------------------- */

/* q-point Gauss-Legendre rule on [-1, 1] (host): x[q] ascending, w[q]
 * summing to 2; exact for polynomials of degree <= 2q - 1.  Newton
 * iteration on the Legendre recurrence.  1 <= q <= 64, else ELDER_EINVAL. */
int elder_gauss_legendre(int q, double* x, double* w);

/* Truncated multi-index set J_{M,p} (host): rule 0 total degree <= p (rule
 * b of Section 3), rule 1 every degree <= p (rule c), rule 2
 * prod_j (beta_j + 1) <= p + 1 (the reading taken of rule a).  Sorted by
 * total degree, then lexicographically; the zero index comes first.  Writes
 * *n_terms; with beta != NULL also the indices, beta[t*M + j], when
 * capacity >= *n_terms (else ELDER_EINVAL).  1 <= M <= 8, 0 <= p <= 16. */
int elder_gpc_indices(int M, int p, int rule, int* n_terms, int32_t* beta, int capacity);

/* Expansion coefficients by quadrature projection (FP64):
 *   coef[t][n] = 0.5^M / Q_t * sum_i w[i] P_{beta_t}(theta_i) u[i][n],
 *   Q_t = prod_j 1 / (2 beta_tj + 1);
 * mean[n] = coef[0][n] and var[n] = sum_{t >= 1} Q_t coef[t][n]^2 (nullable).
 * Device arrays: beta [T][M] int32 with entries in [0, maxdeg] (beta[0] the
 * zero index for mean/var to be meaningful), theta [Nq][M], w [Nq],
 * u [Nq][N] (one field per quadrature point, e.g. c of a batched elder_step
 * run), coef [T][N], mean [N], var [N].  T <= 64, maxdeg <= 16 and
 * 8 (T Nq + T) <= 200 KiB; stream-ordered, no synchronisation. */
int elder_gpc_project(int M, int T, const int32_t* beta, int maxdeg, int Nq,
                      const double* theta, const double* w, int N, const double* u,
                      double* coef, double* mean, double* var, void* stream);

/* Exceedance probability from the surrogate: for each listed node n
 * (nodes[k], or n = k for k < n_pts when nodes is NULL), the fraction of the
 * Ns points theta [Ns][M] at which sum_t coef[t][n] P_{beta_t}(theta) is
 * above threshold.  On the tensor cores where the sizes allow it (see
 * elder_gpc_exceed_engine), else on the CUDA cores: the surrogate evaluated
 * in FP32 (coefficients rounded
 * to FP32, basis values by the FP32 Legendre recurrence, FP32 fused
 * multiply-adds in the order of t); its error is below about
 * 16 T 2^-24 sum_t |coef[t][n]| for degrees up to 8.  Device arrays:
 * beta [T][M], coef [T][N] (from elder_gpc_project), nodes [n_pts] int32 or
 * NULL, theta [Ns][M] (the caller draws the points), p_exceed [n_pts]
 * output (used as 64-bit counters until the last kernel converts them).
 * Stream-ordered, no synchronisation. */
int elder_gpc_exceed(int M, int T, const int32_t* beta, int maxdeg, int N,
                     const double* coef, int n_pts, const int32_t* nodes, int Ns,
                     const double* theta, double threshold, double* p_exceed,
                     void* stream);

/* elder_gpc_exceed with a choice of engine for the surrogate evaluation:
 *  1: the FP32 evaluation described above (CUDA cores);
 *  2: the tensor cores (M <= 4, maxdeg <= 8, T <= 36, else ELDER_EINVAL): the
 *     values of a tile of 128 nodes at a chunk of 128 points are one TF32
 *     matrix product (tcgen05) of the coefficients and the basis values, each
 *     FP32 factor split as hi + lo with hi exact in TF32 and the product
 *     formed as hi*hi + hi*lo + lo*hi with FP32 accumulation; its error stays
 *     below the FP32 engine's bound 16 T 2^-24 sum_t |coef[t][n]| for
 *     degrees up to 8.  Every internal wait of the kernel is bounded; if one
 *     gives up, every p_exceed entry of the call is NaN (one error flag per
 *     device: calls of this engine that overlap on the GPU race on it);
 *  0: engine 2 where it applies, else engine 1 (what elder_gpc_exceed does).
 * Other arguments as elder_gpc_exceed. */
int elder_gpc_exceed_engine(int engine, int M, int T, const int32_t* beta, int maxdeg, int N,
                            const double* coef, int n_pts, const int32_t* nodes, int Ns,
                            const double* theta, double threshold, double* p_exceed,
                            void* stream);

#ifdef __cplusplus
}
#endif
#endif /* ELDER_H */
