// kernels.h -- host-side launch wrappers of the Elder step kernels.
#pragma once

#include "common.cuh"

namespace elder {

// Per-sample Krylov scalars (BiCGStab of van der Vorst, Templates 2.3.8).
struct KScal {
    double rho, rho_old, alpha, omega;
    double bn2, rn2;
    double best_rn2;             // smallest ||r||^2 seen (x = 0 counts)
    double beta;                 // (rho/rho_old)(alpha/omega) of the next p update
    float alpha_f, omega_f, beta_f, pad_f;  // FP32 copies for the FP32 vector updates
    int active, iters, status;
    int improved;                // the last iteration lowered best_rn2
};

// BiCGStab scalars in the vector type: the FP32 solver reads the FP32
// copies, so that its vector kernels issue no FP64 instruction per element.
template <class T> __device__ __forceinline__ T ks_alpha(const KScal& k);
template <> __device__ __forceinline__ float ks_alpha<float>(const KScal& k) { return k.alpha_f; }
template <> __device__ __forceinline__ double ks_alpha<double>(const KScal& k) { return k.alpha; }
template <class T> __device__ __forceinline__ T ks_omega(const KScal& k);
template <> __device__ __forceinline__ float ks_omega<float>(const KScal& k) { return k.omega_f; }
template <> __device__ __forceinline__ double ks_omega<double>(const KScal& k) { return k.omega; }
template <class T> __device__ __forceinline__ T ks_beta(const KScal& k);
template <> __device__ __forceinline__ float ks_beta<float>(const KScal& k) { return k.beta_f; }
template <> __device__ __forceinline__ double ks_beta<double>(const KScal& k) { return k.beta; }

// Per-node contribution a.p b.p + a.c b.c to an FP64 inner product: FP64
// products for the FP64 solver; for the FP32 solver the two products are
// summed in FP32 and the sum is accumulated in FP64 (the vectors themselves
// carry FP32 rounding).
__device__ __forceinline__ double dot2(double ap, double ac, double bp, double bc)
{
    return ap * bp + ac * bc;
}
__device__ __forceinline__ double dot2(float ap, float ac, float bp, float bc)
{
    return (double)fmaf(ap, bp, ac * bc);
}

// Per-sample Newton state (Section 2.3: Newton with line search).
struct NScal {
    double rn, rt, lambda;       // ||R(u)||, ||R(u_trial)||, step length
    double res0;
    double dmax_p, dmax_c;       // max |lambda * delta| of the last step
    double rfloor, rfloor_t;     // round-off level of ||R(u)||, ||R(u_trial)||
    double dprev_p, dprev_c;     // max |delta| of the previous Newton step
    int full_prev;               // previous step was a full (lambda = 1) step
    int skip_res;                // this full step meets the stop: no trial residual
    int active;                  // still iterating
    int ls_active;               // line search still running
    int accepted;                // trial accepted in this Newton iteration
    int iters, ls_cuts, kiters, ls_count, status;
};

// Flux through the dual face of one edge, out of its lower node: mass and
// salt flux and the magnitudes of their terms.
// One quarter-face record of the residual: mass and salt flux from the
// edge's lower to its upper end, and the magnitudes of their terms.
struct alignas(8) QF {
    double m, F;
    float mm, Fm;
};

constexpr int kBS = 256;     // threads per block of the node kernels
constexpr int kMaxBS = 512;  // largest block of the autotuned stencil kernels
constexpr int kMinBS = 128;  // smallest block of the autotuned stencil kernels

inline int nblocks(int n, int bs = kBS) { return (n + bs - 1) / bs; }
// blocks of the BiCGStab x/r update (4 nodes per thread): its partials per sample
inline int bicg_xr_blocks(int n) { return nblocks((n + 3) / 4); }

// Process-wide count of kernel launches made by this library.
void count_launch(int n);
// Message returned by elder_last_error(NULL) after a failed context-free call.
void set_static_error(const char* msg);

// ---- assembly.cu ---------------------------------------------------------
void launch_residual(const Grid& G, const Phys& ph, const uint8_t* bc,
                     const double* cval, const double* phi, const double* K,
                     const double* p, const double* c, const double* p_old,
                     const double* c_old, V2<double>* R, double* partial,
                     double* act, const int* mask, int mask_stride, int S,
                     cudaStream_t st, QF* qf);
// Jacobian rows as T (JT) and/or as the multigrid type M (JM), and the inverse
// interior diagonal blocks (Dinv); null outputs are skipped.  cellT [S][C]
// and nodeT [S][N] are scratch for the inputs converted to T.
// inputs: 0 converts phi, K, p, c into cellT, nodeT first; 1 converts p, c
// only (cellT holds the step's coefficients); 2 converts nothing (nodeT
// written by launch_inject as well).
template <class T, class M>
void launch_jacobian(const Grid& G, const Phys& ph, const uint8_t* bc,
                     const double* phi, const double* K, const double* p,
                     const double* c, B4<T>* JT, B4<M>* JM, B4<T>* Dinv, V2<T>* cellT,
                     V2<T>* nodeT, const int* mask, int mask_stride, int S, cudaStream_t st,
                     int inputs = 0);
// (phi, K / mu) in T for every cell of S samples
template <class T>
void launch_cell_inputs(const Grid& G, double mu, const double* phi, const double* K,
                        V2<T>* cellT, int S, cudaStream_t st);
// coarse state by injection; nodeT (nullable) receives the coarse Jacobian's
// node inputs in T
template <class T>
void launch_inject(const Grid& Gf, const Grid& Gc, const double* pf, const double* cf,
                   double* pc, double* cc, V2<T>* nodeT, double rho0g, const int* mask,
                   int mask_stride, int S, cudaStream_t st);
void launch_average_cells(const Grid& Gf, const Grid& Gc, const double* phif,
                          const double* Kf, double* phic, double* Kc,
                          int harmonic, int S, cudaStream_t st);
template <class M>
void launch_coarse_inverse(const Grid& G, const uint8_t* bc, const B4<M>* J,
                           double* work, double* Ainv, const int* mask,
                           int mask_stride, int S, cudaStream_t st);
void launch_impose_dirichlet(const Grid& G, const uint8_t* bc,
                             const double* cval, double* p, double* c, int S,
                             cudaStream_t st);
void launch_initial_state(const Grid& G, double rho0g, const uint8_t* bc,
                          const double* cval, double* p, double* c, int S,
                          cudaStream_t st);
void launch_fields(const Grid& G, int kind, const double* params,
                   double K_mean, double* phi, double* K, int S,
                   cudaStream_t st);

// ---- linalg.cu -----------------------------------------------------------
// y = A x (or A^T x); mode 0: plain, 1: partial[0] = (a, y),
// 2: partial[0] = (y, a), partial[1] = (y, y), 3: plain and unmasked.
// Modes 0-2 mask the output at Dirichlet components.  partial layout
// [S][2][nblk].
template <class T>
void launch_spmv(const Grid& G, const B4<T>* J, const uint8_t* bc,
                 const V2<T>* x, V2<T>* y, int trans, int mode,
                 const V2<T>* a, double* partial, const int* mask,
                 int mask_stride, int S, cudaStream_t st, int bs = kBS);
// xo = x + omega Dinv (b - A x) (x == nullptr: xo = omega Dinv b); the
// matrix is stored as M (MgType<T>), vectors and Dinv as T
template <class T, class M>
void launch_smooth(const Grid& G, const B4<M>* J, const B4<T>* Dinv,
                   const uint8_t* bc, const V2<T>* b, const V2<T>* x,
                   V2<T>* xo, double omega, int trans, const int* mask,
                   int mask_stride, int S, cudaStream_t st, int bs = kBS);
// spc: samples per CTA (1 or 2), each thread forming its node's residual in
// spc samples
template <class T, class M>
void launch_mg_residual(const Grid& G, const B4<M>* J, const uint8_t* bc,
                        const V2<T>* b, const V2<T>* x, V2<T>* r, int trans,
                        const int* mask, int mask_stride, int S,
                        cudaStream_t st, int bs = kBS, int spc = 1);
template <class T>
void launch_restrict(const Grid& Gf, const Grid& Gc, const uint8_t* bcc,
                     const V2<T>* rf, V2<T>* bc_out, const int* mask,
                     int mask_stride, int S, cudaStream_t st);
template <class T>
void launch_prolong_add(const Grid& Gf, const Grid& Gc, const uint8_t* bcf,
                        const V2<T>* xc, V2<T>* xf, const int* mask,
                        int mask_stride, int S, cudaStream_t st);
template <class T>
void launch_coarse_apply(const Grid& G, const double* Ainv, const V2<T>* b,
                         V2<T>* x, int trans, const int* mask, int mask_stride,
                         int S, cudaStream_t st);

// BiCGStab pieces (all skip samples whose KScal.active == 0)
template <class T>
void launch_bicg_init(const Grid& G, const uint8_t* bc, const V2<T>* b,
                      V2<T>* x, V2<T>* r, V2<T>* rh, V2<T>* p, V2<T>* v,
                      double* partial, KScal* ks, int S, cudaStream_t st);
template <class T>
void launch_bicg_p(const Grid& G, const V2<T>* r, const V2<T>* v, V2<T>* p,
                   const KScal* ks, int S, cudaStream_t st);
template <class T>
void launch_bicg_s(const Grid& G, const V2<T>* r, const V2<T>* v, V2<T>* s,
                   double* partial, const KScal* ks, int S, cudaStream_t st);
template <class T>
void launch_bicg_xr(const Grid& G, const V2<T>* ph, const V2<T>* sh,
                    const V2<T>* s, const V2<T>* t, const V2<T>* rh, V2<T>* x,
                    V2<T>* r, double* partial, const KScal* ks, int S,
                    cudaStream_t st);
// stage: 0 init, 1 alpha, 2 omega, 3 end of iteration
void launch_bicg_finalize(int stage, const double* partial, int nblk,
                          KScal* ks, double rtol, int maxit, int S,
                          cudaStream_t st);

// Newton pieces
// which = 0: ||R(u)|| (also res0 and, from act, the round-off floor),
// which = 1: ||R(u_trial)||
void launch_norm_finalize(const double* partial, const double* act, int nblk,
                          NScal* ns, int which, int S, cudaStream_t st);
template <class T>
void launch_newton_rhs(const Grid& G, const V2<double>* R, V2<T>* b,
                       const NScal* ns, int S, cudaStream_t st);
template <class T>
void launch_newton_trial(const Grid& G, const double* p, const double* c,
                         const V2<T>* dx, double* pt, double* ct,
                         double* partial, const NScal* ns, int S,
                         cudaStream_t st);
void launch_newton_ls_finalize(const double* partial_res,
                               const double* partial_max, int nblk,
                               NScal* ns, int ls_max, int S, cudaStream_t st);
void launch_newton_accept(const Grid& G, double* p, double* c,
                          const double* pt, const double* ct,
                          V2<double>* R, const V2<double>* Rt,
                          const NScal* ns, int S, cudaStream_t st);
// Damped z-line block-Jacobi line solves; lines of at most kMaxLine nodes.
// mode 1: zero initial guess (x unused), x_out = omega L^{-1} b; mode 2: b
// is the masked residual b - A x of x, x_out = x + omega L^{-1} b.
constexpr int kMaxLine = 129;
constexpr int kLineBS = 128;
template <class T, class M>
void launch_smooth_zline(const Grid& G, const B4<M>* J, const B4<T>* Dinv, const uint8_t* bc,
                         const V2<T>* b, const V2<T>* x, V2<T>* xo, double omega, int trans,
                         const int* mask, int mstride, int S, cudaStream_t st, int mode);

// Block-LU factors of the vertical lines of a level's (non-transposed)
// operator, zMi and zC [S][N], and the line sweep that substitutes with
// them (mode 1: x = 0; mode 2: r is the masked residual of x).  Lines of at
// most kMaxLine nodes.
template <class T, class M>
void launch_zline_factor(const Grid& G, const B4<M>* J, const B4<T>* Dinv, const uint8_t* bc,
                         B4<T>* zMi, B4<T>* zC, const int* mask, int mstride, int S,
                         cudaStream_t st);
// bs threads per block; spc lines of different samples per thread (1 or 2)
template <class T, class M>
void launch_zline_apply(const Grid& G, const B4<M>* J, const B4<T>* zMi, const B4<T>* zC,
                        const uint8_t* bc, const V2<T>* r, const V2<T>* x, V2<T>* xo,
                        double omega, const int* mask, int mstride, int S, cudaStream_t st,
                        int mode, int bs = 128, int spc = 1);

// Multicolour block ILU_beta(0) smoother.  Colour c = (i&1) + 2(j&1) +
// 4(k&1); the factors are stored with the node axis in colour-blocked order:
// colour c at positions off[c] .. off[c+1]-1, its nodes in natural order;
// cnt_x[p] / cnt_y[p] count the nodes of index parity p along x / y.
struct IluLayout {
    int off[9];
    int cnt_x[2], cnt_y[2];
};
IluLayout ilu_layout(const Grid& G);
// Factors of a level's interior operator: F [S][27][N] (storage type M,
// colour-blocked node axis: L in the slots of smaller-colour neighbours, U
// in the others) and Fd [S][N] (inverse pivot blocks).  8 launches.
template <class T, class M>
void launch_ilu_factor(const Grid& G, const B4<M>* J, const B4<T>* Dinv, const uint8_t* bc,
                       B4<M>* F, B4<T>* Fd, double beta, const int* mask, int mstride, int S,
                       cudaStream_t st);
// One ILU sweep: x_out = x + omega (L U)^{-1} r (mode 2, r the masked
// residual of x) or x_out = omega (L U)^{-1} r (mode 1, x = 0, r = b); the
// transposed sweep applies (L U)^{-T}.  t: [S][N] scratch holding both
// triangular solves' results (t may be r).  16 launches, one per colour and
// solve.
template <class T, class M>
void launch_ilu_apply(const Grid& G, const B4<M>* F, const B4<T>* Fd, const uint8_t* bc,
                      const V2<T>* r, V2<T>* t, const V2<T>* x, V2<T>* xo, double omega,
                      int trans, int mode, const int* mask, int mstride, int S, cudaStream_t st,
                      int bs = kBS);

// Keeps the iterate of smallest residual: copies x into xbest for the
// samples whose last iteration improved it (keep == 1), or x <- xbest for
// the samples that did not converge (keep == 2).
template <class T>
void launch_bicg_keep(const Grid& G, V2<T>* x, V2<T>* xbest, const KScal* ks, int keep, int S,
                      cudaStream_t st);
void launch_newton_check(NScal* ns, const KScal* ks, double tol_p,
                         double tol_c, int maxit, int estimate, int S, cudaStream_t st);
// Before the trial residual of a full step: a sample whose correction
// already meets the stop of launch_newton_check is accepted without it.
void launch_newton_predict(const double* partial_max, int nblk, NScal* ns, double tol_p,
                           double tol_c, int estimate, int S, cudaStream_t st);
void launch_extrapolate(const Grid& G, int order, const double* p_n, const double* c_n,
                        const double* p1, const double* c1, const double* p2, const double* c2,
                        double* p, double* c, int S, cudaStream_t st);
void launch_newton_restore_failed(const Grid& G, double* p, double* c,
                                  const double* p_old, const double* c_old,
                                  const NScal* ns, int S, cudaStream_t st);

void launch_moments(int N, int S, const double* c, const double* w,
                    double threshold, double* mean, double* var,
                    double* pexc, cudaStream_t st);

// salt mass at u^n, u^{n+1} and the Dirichlet inflow; partial [S][3][nblk]
void launch_mass_balance(const Grid& G, const Phys& ph, const uint8_t* bc, const double* phi,
                         const double* K, const double* p, const double* c,
                         const double* c_old, double* partial, int S, cudaStream_t st);

// ---- adjoint pieces (assembly.cu) ----------------------------------------
void launch_objective(const Grid& G, const Phys& ph, const double* phi,
                      const double* c, double* partial, double* dJdphi,
                      V2<double>* dJdu, cudaStream_t st);
void launch_adjoint_theta(const Grid& G, const Phys& ph, const uint8_t* bc,
                          const double* phi, const double* K,
                          const double* p, const double* c,
                          const double* c_old, const V2<double>* lam,
                          double* dJdphi, double* dJdK, cudaStream_t st);
void launch_adjoint_prev_rhs(const Grid& G, const Phys& ph, const uint8_t* bc,
                             const double* phi, const double* c_old,
                             const V2<double>* lam, V2<double>* rhs,
                             cudaStream_t st);

// small helpers
void launch_sum_partials(const double* partial, int nblk, double* out,
                         int S, cudaStream_t st);
template <class T>
void launch_axpy_mask(const Grid& G, const uint8_t* bc, const V2<T>* x,
                      V2<T>* y, double a, int which, int S, cudaStream_t st);
template <class Ts, class Td>
void launch_convert(const V2<Ts>* x, V2<Td>* y, size_t n, cudaStream_t st);

}  // namespace elder
