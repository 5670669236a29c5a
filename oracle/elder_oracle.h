/*
 * elder_oracle.h -- plain, slow FP64 CPU oracle for the implicit time step of
 * the 3D Elder-like density-driven flow problem (Litvinenko et al.,
 * arXiv:1906.01632).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the bench's
 * CPU-baseline leg may load this library.  It shares no code, header, table
 * or constant generator with the CUDA path in paper_1906_01632_gb300/.
 *
 * Model (Section 2.1): fluid mass conservation (eq. e_cont_eq), salt
 * transport (eq. e_tran_eq), Darcy law (eq. e_Darcy_vel) with scalar
 * permeability (eq. e_scalar_perm), linear density (eq. e_lin_density),
 * constant viscosity and molecular diffusion D = phi*Dm*I (eq. e_mol_diff).
 * Discretisation (Section 2.3): vertex-centred finite volumes (box method)
 * on a structured hexahedral box, implicit Euler, Newton with line search.
 *
 * Grid: nodes (i,j,k), 0<=i<=nx, at x=i*Lx/nx; z points up, the top is
 * z=Lz.  Node index n = i + (nx+1)*(j + (ny+1)*k); cell index
 * e = i + nx*(j + ny*k).  Linear-system unknowns are interleaved:
 * u[2n] = p_n, u[2n+1] = c_n; residual rows likewise.
 */
#ifndef ELDER_ORACLE_H
#define ELDER_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Boundary-condition sets (Section 2.1, Fig. 1 caption):
 *   0: c=1 on the closed top square [Lx/4,3Lx/4]x[Ly/4,3Ly/4], c=0 on the
 *      bottom, p=0 at the four top corners (the benchmark variant);
 *   1: paper variant: c=1 on the top square, c=0 on the rest of the top and
 *      on the bottom, p=0 on the four top edges;
 *   2: erfc column test: c=1 on the whole top, c=0 on the bottom, p=0 at the
 *      four top corners;
 *   3: no c Dirichlet nodes, p=0 at the four top corners (hydrostatic test). */
typedef struct {
    int nx, ny, nz;
    double Lx, Ly, Lz;
    double rho0, rho1, mu, g, Dm;
    int bc_mode;
} orc_problem;

typedef struct {
    int maxit;          /* Newton iteration cap                            */
    double tol_c;       /* converged when max|lambda*dc| <= tol_c ...      */
    double tol_p;       /* ... and max|lambda*dp| <= tol_p, with lambda=1  */
    double lin_rtol;    /* relative residual target of each linear solve   */
    int lin_maxit;      /* BiCGStab iteration cap                          */
    int ls_max;         /* maximum number of step halvings                 */
    int dense_max;      /* use dense LU when 2N <= dense_max               */
    int smoother;       /* multigrid smoother of the iterative solve:
                           0 damped 2x2-block Jacobi, 1 damped block Jacobi
                           over vertical grid lines (block-tridiagonal
                           solve per line), 2 multicolour block
                           ILU_beta(0) (orc_mcilu_factor, undamped); the
                           converged step does not depend on it            */
    double ilu_beta;    /* beta of smoother 2                              */
} orc_newton_opts;

typedef struct {
    int status;         /* 0 converged, 1 Newton cap, 2 linear failure     */
    int newton_iters;
    int lin_iters;      /* total linear iterations (0 with dense LU)       */
    int ls_cuts;        /* total step halvings                             */
    double res0, res;   /* 2-norm of R before the first and after the last */
} orc_step_info;

int  orc_num_nodes(const orc_problem* P);
int  orc_num_cells(const orc_problem* P);

/* Dirichlet data per node: pmask/cmask = 1 where p / c is prescribed, cval =
 * the prescribed c (p is always prescribed to 0). */
void orc_dirichlet(const orc_problem* P, unsigned char* pmask,
                   unsigned char* cmask, double* cval);

/* Initial state: c = Dirichlet value at c-Dirichlet nodes, else 0;
 * p = rho0*g*(Lz - z) (seeds Newton only: p has no time derivative). */
void orc_initial_state(const orc_problem* P, double* p, double* c);

/* Residual R(u^{n+1}; u^n) of the implicit Euler step (eqs. e_cont_eq,
 * e_tran_eq).  Rp, Rc: [N].  With apply_dirichlet=0 the raw FV balance is
 * returned at every node (used by the conservation pins). */
void orc_residual(const orc_problem* P, const double* phi, const double* K,
                  const double* p, const double* c, const double* p_old,
                  const double* c_old, double dt, int apply_dirichlet,
                  double* Rp, double* Rc);

/* Round-off scale of R: 2-norm over non-Dirichlet rows of the per-row sums
 * of the magnitudes of all terms of orc_residual (storage at both levels;
 * for each Darcy flux rho (K/mu)(|grad p| + [z] g rho) A, the size of the two
 * terms it cancels).  Newton treats ||R|| <= 2 eps times this as solved. */
double orc_residual_magnitude(const orc_problem* P, const double* phi,
                              const double* K, const double* p,
                              const double* c, const double* c_old, double dt);

/* Sparse pattern (CSR, 0-based, sorted columns) of the 2N x 2N Jacobian. */
int  orc_jac_nnz(const orc_problem* P);
void orc_jac_pattern(const orc_problem* P, int* rowptr, int* col);
/* Exact Jacobian dR/du at (p,c) with the current upwind branch. */
void orc_jacobian(const orc_problem* P, const double* phi, const double* K,
                  const double* p, const double* c, double dt,
                  const int* rowptr, const int* col, double* val);
/* CSR transpose. */
void orc_csr_transpose(int n, const int* rowptr, const int* col,
                       const double* val, int* trowptr, int* tcol,
                       double* tval);

/* Dense LU with partial pivoting; A (n*n, row-major) and b are overwritten,
 * b receives x.  Returns 0, or 1 on an exactly zero pivot. */
int orc_dense_solve(int n, double* A, double* b);
/* BiCGStab (right preconditioned by ILU(0)); x holds the initial guess.
 * Returns 0 when ||b-Ax|| <= rtol*||b||, else 1. */
int orc_bicgstab_ilu0(int n, const int* rowptr, const int* col,
                      const double* val, const double* b, double* x,
                      double rtol, int maxit, int* iters, double* relres);
/* Solve A x = b with the oracle's solver choice (dense when n<=dense_max). */
int orc_linear_solve(int n, const int* rowptr, const int* col,
                     const double* val, const double* b, double* x,
                     const orc_newton_opts* o, int* iters);

/* Multicolour block ILU_beta(0) (Section 5.1 names the multigrid smoother
 * ILU_beta without defining it).  Block matrices on the node grid are held
 * as [N][27][4]: entry [n][s] is the 2x2 block (n, n+d) of the neighbour at
 * offset d = (dx,dy,dz), s = (dx+1) + 3(dy+1) + 9(dz+1), entries (pp, pc,
 * cp, cc); blocks of neighbours outside the grid are 0.
 *
 * orc_mc_rank: rank[n] = position of node n in the multicolour order
 * (colour = (i&1) + 2(j&1) + 4(k&1), colours ascending, node index order
 * within a colour).
 * orc_csr_to_blocks: the block form B of a CSR matrix with the 27-point
 * block pattern (orc_jac_pattern, or its transpose).
 * orc_mcilu_factor: the factors F of A in that order, in A's block form:
 * slots whose neighbour has a smaller rank hold L (unit block diagonal
 * implied), the others U with the pivot blocks in slot 13.  Returns 0, or 1
 * when a pivot block is singular.
 * orc_mcilu_solve: z = (L U)^{-1} r, or (L U)^{-T} r when transpose = 1;
 * r, z: [N][2] (z may not alias r).
 * orc_smoother_apply: one application of a multigrid smoother's
 * preconditioner on the finest grid, linearised at (p, c) with time step dt:
 * z = P^{-1} r (transpose = 0) or P^{-T} r on the interior unknowns of the
 * Jacobian (Dirichlet rows and columns replaced by the identity; Dirichlet
 * components of r ignored, those of z set to 0), with P the 2x2 block
 * diagonal (kind 0), the block-tridiagonal part along vertical grid lines
 * (kind 1) or L U of the multicolour block ILU_beta(0) factors (kind 2).
 * Returns 0, or 1 on a singular pivot. */
void orc_mc_rank(const orc_problem* P, int* rank);
void orc_csr_to_blocks(const orc_problem* P, const int* rowptr, const int* col,
                       const double* val, double* B);
int orc_mcilu_factor(const orc_problem* P, const double* A, double beta, double* F);
void orc_mcilu_solve(const orc_problem* P, const double* F, int transpose,
                     const double* r, double* z);
int orc_smoother_apply(const orc_problem* P, const double* phi, const double* K,
                       const double* p, const double* c, double dt, int kind,
                       double beta, int transpose, const double* r, double* z);

/* One implicit Euler step by Newton with line search.  p, c: in u^n, out
 * u^{n+1}.  Returns info->status. */
int orc_newton_step(const orc_problem* P, const double* phi, const double* K,
                    double* p, double* c, double dt,
                    const orc_newton_opts* o, orc_step_info* info);

/* Sample statistics over S fields c[S][N] (eqs. pdestat, numer_var and the
 * exceedance estimate of Section 3.3).  w: [S] weights or NULL for 1/S. */
void orc_moments(int S, int N, const double* c, const double* w,
                 double threshold, double* mean, double* var, double* pexc);

/* Porosity / permeability per cell.
 * orc_fields_sobol: phi = 0.1*(1 + 0.3*(xi1*cos(pi x/Lx) + xi2*cos(pi y/Ly)
 *   + xi3*sin(2 pi z/Lz))/3) at cell centres;
 * orc_fields_lognormal: phi = clip(0.1*exp(0.2*Z), 0.05, 0.2);
 * both with normalised Kozeny-Carman K = K_mean * [phi^3/(1-phi)^2] /
 * [0.1^3/0.9^2] (eq. e_perm_Kozeny_Carman, normalised so K(E phi) = E K). */
void orc_fields_sobol(const orc_problem* P, const double* xi, double K_mean,
                      double* phi, double* K);
void orc_fields_lognormal(const orc_problem* P, const double* Z,
                          double K_mean, double* phi, double* K);
/* The paper's parallelepiped field with three RVs (eq. poro-paral3RVS). */
void orc_fields_paper3rv(const orc_problem* P, const double* xi,
                         double K_mean, double* phi, double* K);

/* Plume functional: salt mass in cells whose centre lies below Lz/2,
 * J = sum_e sum_corners phi_e |scv| rho(c_L) c_L. */
double orc_objective(const orc_problem* P, const double* phi,
                     const double* c);

/* Discrete adjoint gradient of J(u_N) over n_steps implicit Euler steps
 * w.r.t. per-cell phi and K (treated as independent inputs).  p0,c0: the
 * initial state (left untouched).  Forward states are all stored.
 * Returns 0 on success. */
int orc_adjoint_gradient(const orc_problem* P, const double* phi,
                         const double* K, const double* p0, const double* c0,
                         double dt, int n_steps, const orc_newton_opts* o,
                         double* J_out, double* dJ_dphi, double* dJ_dK);

#ifdef __cplusplus
}
#endif
#endif
