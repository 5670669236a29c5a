/*
 * elder_oracle.c -- plain FP64 CPU oracle (test infrastructure only; see
 * elder_oracle.h).  Every function is written for clarity, element by
 * element, following the paper's model (Section 2.1) and discretisation
 * (Section 2.3, Section 5.1); none of it is tuned.
 */
#include "elder_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* grid helpers                                                             */
/* ------------------------------------------------------------------------ */

int orc_num_nodes(const orc_problem* P)
{
    return (P->nx + 1) * (P->ny + 1) * (P->nz + 1);
}

int orc_num_cells(const orc_problem* P) { return P->nx * P->ny * P->nz; }

static int node_id(const orc_problem* P, int i, int j, int k)
{
    return i + (P->nx + 1) * (j + (P->ny + 1) * k);
}

static double rho_of(const orc_problem* P, double c)
{
    /* eq. e_lin_density */
    return P->rho0 + (P->rho1 - P->rho0) * c;
}

/* Dirichlet sets of Section 2.1 / Fig. 1 (see the bc_mode list in the
 * header).  The top square is closed: 4*i in [nx, 3*nx]. */
void orc_dirichlet(const orc_problem* P, unsigned char* pmask,
                   unsigned char* cmask, double* cval)
{
    for (int k = 0; k <= P->nz; ++k)
        for (int j = 0; j <= P->ny; ++j)
            for (int i = 0; i <= P->nx; ++i) {
                int n = node_id(P, i, j, k);
                int top = (k == P->nz), bottom = (k == 0);
                int xedge = (i == 0 || i == P->nx);
                int yedge = (j == 0 || j == P->ny);
                int in_sq = (4 * i >= P->nx && 4 * i <= 3 * P->nx &&
                             4 * j >= P->ny && 4 * j <= 3 * P->ny);
                unsigned char pm = 0, cm = 0;
                double cv = 0.0;
                switch (P->bc_mode) {
                case 0:
                    pm = top && xedge && yedge;
                    if (top && in_sq) { cm = 1; cv = 1.0; }
                    else if (bottom) { cm = 1; cv = 0.0; }
                    break;
                case 1:
                    pm = top && (xedge || yedge);
                    if (top) { cm = 1; cv = in_sq ? 1.0 : 0.0; }
                    else if (bottom) { cm = 1; cv = 0.0; }
                    break;
                case 2:
                    pm = top && xedge && yedge;
                    if (top) { cm = 1; cv = 1.0; }
                    else if (bottom) { cm = 1; cv = 0.0; }
                    break;
                default:
                    pm = top && xedge && yedge;
                    break;
                }
                if (pmask) pmask[n] = pm;
                if (cmask) cmask[n] = cm;
                if (cval) cval[n] = cv;
            }
}

void orc_initial_state(const orc_problem* P, double* p, double* c)
{
    int N = orc_num_nodes(P);
    unsigned char* cm = (unsigned char*)malloc((size_t)N);
    double* cv = (double*)malloc(sizeof(double) * (size_t)N);
    orc_dirichlet(P, NULL, cm, cv);
    double hz = P->Lz / P->nz;
    for (int k = 0; k <= P->nz; ++k)
        for (int j = 0; j <= P->ny; ++j)
            for (int i = 0; i <= P->nx; ++i) {
                int n = node_id(P, i, j, k);
                p[n] = P->rho0 * P->g * (P->Lz - k * hz);
                c[n] = cm[n] ? cv[n] : 0.0;
            }
    free(cm);
    free(cv);
}

/* ------------------------------------------------------------------------ */
/* one sub-control-volume face of one hexahedron                            */
/* ------------------------------------------------------------------------ */

/* Corner L = a + 2b + 4cz of cell (i,j,k) is node (i+a, j+b, k+cz). */
static void cell_corners(const orc_problem* P, int i, int j, int k,
                         int nodes[8])
{
    for (int L = 0; L < 8; ++L)
        nodes[L] = node_id(P, i + (L & 1), j + ((L >> 1) & 1),
                           k + ((L >> 2) & 1));
}

/* Trilinear (Q1) shape functions of the unit cube and their derivative
 * along direction d (divided by the cell size h_d) at local point X[3]. */
static void q1_at(const double X[3], int d, double h_d, double N[8],
                  double dN[8])
{
    for (int L = 0; L < 8; ++L) {
        int a[3] = {L & 1, (L >> 1) & 1, (L >> 2) & 1};
        double f[3], df[3];
        for (int m = 0; m < 3; ++m) {
            f[m] = a[m] ? X[m] : 1.0 - X[m];
            df[m] = a[m] ? 1.0 : -1.0;
        }
        N[L] = f[0] * f[1] * f[2];
        double g = 1.0;
        for (int m = 0; m < 3; ++m) g *= (m == d) ? df[m] : f[m];
        dN[L] = g / h_d;
    }
}

/* The box method splits each hexahedron into 8 sub-control volumes and has
 * 12 sub-control-volume faces, one per cell edge.  The face of the edge
 * along direction d whose transverse local position is (s,t) lies in the
 * mid-plane of the edge; its integration point sits at 1/2 along d and at
 * 1/4 or 3/4 across, its area is a quarter of the cell cross-section and its
 * normal points from corner "a" (local coordinate 0 along d) to corner "b". */
typedef struct {
    int La, Lb;          /* local corners of the edge                  */
    double N[8], dN[8];  /* shape values and d-derivatives at the ip   */
    double A;            /* face area                                  */
    int d;
} scvf;

static void make_scvf(const orc_problem* P, int d, int s, int t, scvf* f)
{
    double h[3] = {P->Lx / P->nx, P->Ly / P->ny, P->Lz / P->nz};
    int t1 = (d == 0) ? 1 : 0;
    int t2 = (d == 2) ? 1 : 2;
    int ca[3] = {0, 0, 0};
    ca[t1] = s;
    ca[t2] = t;
    int cb[3] = {ca[0], ca[1], ca[2]};
    cb[d] = 1;
    f->La = ca[0] + 2 * ca[1] + 4 * ca[2];
    f->Lb = cb[0] + 2 * cb[1] + 4 * cb[2];
    double X[3];
    X[d] = 0.5;
    X[t1] = s ? 0.75 : 0.25;
    X[t2] = t ? 0.75 : 0.25;
    q1_at(X, d, h[d], f->N, f->dN);
    f->A = 0.25 * h[t1] * h[t2];
    f->d = d;
}

/* Flux quantities through one face (eq. e_Darcy_vel with g = (0,0,-g)). */
typedef struct {
    double rho_ip, qn, m, F, gradc, cup;
    int up;              /* local corner that supplies the upwind c */
} face_flux;

static void eval_face(const orc_problem* P, const scvf* f, double phi_e,
                      double K_e, const double pl[8], const double cl[8],
                      face_flux* out)
{
    double gradp = 0.0, gradc = 0.0, c_ip = 0.0, rhog = 0.0;
    for (int L = 0; L < 8; ++L) {
        gradp += pl[L] * f->dN[L];
        gradc += cl[L] * f->dN[L];
        c_ip += f->N[L] * cl[L];
    }
    /* Gravity: the Q1 interpolant of rho(c) times the z component of the
     * gravity vector (0,0,-g); horizontal faces see none. */
    if (f->d == 2) {
        double rho_interp = 0.0;
        for (int L = 0; L < 8; ++L) rho_interp += f->N[L] * rho_of(P, cl[L]);
        rhog = -P->g * rho_interp;
    }
    double rho_ip = rho_of(P, c_ip);
    double qn = -(K_e / P->mu) * (gradp - rhog);
    double m = rho_ip * qn * f->A;
    int up = (m >= 0.0) ? f->La : f->Lb;
    double cup = cl[up];
    out->rho_ip = rho_ip;
    out->qn = qn;
    out->m = m;
    out->gradc = gradc;
    out->cup = cup;
    out->up = up;
    out->F = cup * m - rho_ip * phi_e * P->Dm * gradc * f->A;
}

/* ------------------------------------------------------------------------ */
/* residual                                                                 */
/* ------------------------------------------------------------------------ */

void orc_residual(const orc_problem* P, const double* phi, const double* K,
                  const double* p, const double* c, const double* p_old,
                  const double* c_old, double dt, int apply_dirichlet,
                  double* Rp, double* Rc)
{
    (void)p_old; /* p has no time derivative */
    int N = orc_num_nodes(P);
    double vscv = (P->Lx / P->nx) * (P->Ly / P->ny) * (P->Lz / P->nz) / 8.0;
    memset(Rp, 0, sizeof(double) * (size_t)N);
    memset(Rc, 0, sizeof(double) * (size_t)N);
    scvf faces[12];
    int nf = 0;
    for (int d = 0; d < 3; ++d)
        for (int s = 0; s < 2; ++s)
            for (int t = 0; t < 2; ++t) make_scvf(P, d, s, t, &faces[nf++]);

    for (int k = 0; k < P->nz; ++k)
        for (int j = 0; j < P->ny; ++j)
            for (int i = 0; i < P->nx; ++i) {
                int e = i + P->nx * (j + P->ny * k);
                int nodes[8];
                cell_corners(P, i, j, k, nodes);
                double pl[8], cl[8];
                for (int L = 0; L < 8; ++L) {
                    pl[L] = p[nodes[L]];
                    cl[L] = c[nodes[L]];
                }
                /* lumped storage, implicit Euler (eqs. e_cont_eq/e_tran_eq) */
                for (int L = 0; L < 8; ++L) {
                    int n = nodes[L];
                    double rn = rho_of(P, c[n]), ro = rho_of(P, c_old[n]);
                    Rp[n] += phi[e] * vscv * (rn - ro) / dt;
                    Rc[n] += phi[e] * vscv * (rn * c[n] - ro * c_old[n]) / dt;
                }
                /* face fluxes: out of corner a, into corner b */
                for (int q = 0; q < 12; ++q) {
                    face_flux ff;
                    eval_face(P, &faces[q], phi[e], K[e], pl, cl, &ff);
                    int a = nodes[faces[q].La], b = nodes[faces[q].Lb];
                    Rp[a] += ff.m;
                    Rp[b] -= ff.m;
                    Rc[a] += ff.F;
                    Rc[b] -= ff.F;
                }
            }
    if (apply_dirichlet) {
        unsigned char* pm = (unsigned char*)malloc((size_t)N);
        unsigned char* cm = (unsigned char*)malloc((size_t)N);
        double* cv = (double*)malloc(sizeof(double) * (size_t)N);
        orc_dirichlet(P, pm, cm, cv);
        for (int n = 0; n < N; ++n) {
            if (pm[n]) Rp[n] = p[n];
            if (cm[n]) Rc[n] = c[n] - cv[n];
        }
        free(pm);
        free(cm);
        free(cv);
    }
}

/* Round-off scale of the residual: per node the sum of the magnitudes of
 * all terms that orc_residual adds up (storage at both time levels and every
 * face flux); Dirichlet rows get 0 (their residual u - u_D is exact).
 * Returns the 2-norm over all rows. */
double orc_residual_magnitude(const orc_problem* P, const double* phi,
                              const double* K, const double* p,
                              const double* c, const double* c_old, double dt)
{
    int N = orc_num_nodes(P);
    double vscv = (P->Lx / P->nx) * (P->Ly / P->ny) * (P->Lz / P->nz) / 8.0;
    double* ap = calloc((size_t)N, sizeof(double));
    double* ac = calloc((size_t)N, sizeof(double));
    scvf faces[12];
    int nf = 0;
    for (int d = 0; d < 3; ++d)
        for (int s = 0; s < 2; ++s)
            for (int t = 0; t < 2; ++t) make_scvf(P, d, s, t, &faces[nf++]);
    for (int k = 0; k < P->nz; ++k)
        for (int j = 0; j < P->ny; ++j)
            for (int i = 0; i < P->nx; ++i) {
                int e = i + P->nx * (j + P->ny * k);
                int nodes[8];
                cell_corners(P, i, j, k, nodes);
                double pl[8], cl[8];
                for (int L = 0; L < 8; ++L) {
                    pl[L] = p[nodes[L]];
                    cl[L] = c[nodes[L]];
                }
                for (int L = 0; L < 8; ++L) {
                    int n = nodes[L];
                    double rn = rho_of(P, c[n]), ro = rho_of(P, c_old[n]);
                    ap[n] += phi[e] * vscv * (fabs(rn) + fabs(ro)) / dt;
                    ac[n] += phi[e] * vscv * (fabs(rn * c[n]) + fabs(ro * c_old[n])) / dt;
                }
                for (int q = 0; q < 12; ++q) {
                    const scvf* f = &faces[q];
                    face_flux ff;
                    eval_face(P, f, phi[e], K[e], pl, cl, &ff);
                    /* the Darcy flux cancels grad p against rho g: its rounding
                     * scales with the size of both terms */
                    double gp = 0.0, gc = 0.0;
                    for (int L = 0; L < 8; ++L) {
                        gp += pl[L] * f->dN[L];
                        gc += cl[L] * f->dN[L];
                    }
                    double drive = fabs(gp) + (f->d == 2 ? P->g * ff.rho_ip : 0.0);
                    double mm = ff.rho_ip * (K[e] / P->mu) * drive * f->A;
                    double Fm = fabs(ff.cup) * mm +
                                ff.rho_ip * phi[e] * P->Dm * fabs(gc) * f->A;
                    int a = nodes[f->La], b = nodes[f->Lb];
                    ap[a] += mm;
                    ap[b] += mm;
                    ac[a] += Fm;
                    ac[b] += Fm;
                }
            }
    unsigned char* pm = malloc((size_t)N);
    unsigned char* cm = malloc((size_t)N);
    orc_dirichlet(P, pm, cm, NULL);
    double s2 = 0.0;
    for (int n = 0; n < N; ++n) {
        if (!pm[n]) s2 += ap[n] * ap[n];
        if (!cm[n]) s2 += ac[n] * ac[n];
    }
    free(ap); free(ac); free(pm); free(cm);
    return sqrt(s2);
}

/* ------------------------------------------------------------------------ */
/* Jacobian                                                                 */
/* ------------------------------------------------------------------------ */

int orc_jac_nnz(const orc_problem* P)
{
    int nnz = 0;
    for (int k = 0; k <= P->nz; ++k)
        for (int j = 0; j <= P->ny; ++j)
            for (int i = 0; i <= P->nx; ++i) {
                int cnt = 0;
                for (int dk = -1; dk <= 1; ++dk)
                    for (int dj = -1; dj <= 1; ++dj)
                        for (int di = -1; di <= 1; ++di) {
                            int ii = i + di, jj = j + dj, kk = k + dk;
                            if (ii >= 0 && ii <= P->nx && jj >= 0 &&
                                jj <= P->ny && kk >= 0 && kk <= P->nz)
                                ++cnt;
                        }
                nnz += 2 * 2 * cnt;
            }
    return nnz;
}

void orc_jac_pattern(const orc_problem* P, int* rowptr, int* col)
{
    int pos = 0;
    for (int k = 0; k <= P->nz; ++k)
        for (int j = 0; j <= P->ny; ++j)
            for (int i = 0; i <= P->nx; ++i) {
                int n = node_id(P, i, j, k);
                for (int v = 0; v < 2; ++v) {
                    rowptr[2 * n + v] = pos;
                    /* neighbours in ascending node order: k, then j, then i */
                    for (int dk = -1; dk <= 1; ++dk)
                        for (int dj = -1; dj <= 1; ++dj)
                            for (int di = -1; di <= 1; ++di) {
                                int ii = i + di, jj = j + dj, kk = k + dk;
                                if (ii < 0 || ii > P->nx || jj < 0 ||
                                    jj > P->ny || kk < 0 || kk > P->nz)
                                    continue;
                                int m = node_id(P, ii, jj, kk);
                                col[pos++] = 2 * m;
                                col[pos++] = 2 * m + 1;
                            }
                }
            }
    rowptr[2 * orc_num_nodes(P)] = pos;
}

static void csr_add(const int* rowptr, const int* col, double* val, int r,
                    int cidx, double v)
{
    for (int q = rowptr[r]; q < rowptr[r + 1]; ++q)
        if (col[q] == cidx) {
            val[q] += v;
            return;
        }
    /* not reached for a pattern built by orc_jac_pattern */
    abort();
}

void orc_jacobian(const orc_problem* P, const double* phi, const double* K,
                  const double* p, const double* c, double dt,
                  const int* rowptr, const int* col, double* val)
{
    int N = orc_num_nodes(P);
    double drho = P->rho1 - P->rho0;
    double vscv = (P->Lx / P->nx) * (P->Ly / P->ny) * (P->Lz / P->nz) / 8.0;
    memset(val, 0, sizeof(double) * (size_t)rowptr[2 * N]);
    scvf faces[12];
    int nf = 0;
    for (int d = 0; d < 3; ++d)
        for (int s = 0; s < 2; ++s)
            for (int t = 0; t < 2; ++t) make_scvf(P, d, s, t, &faces[nf++]);

    for (int k = 0; k < P->nz; ++k)
        for (int j = 0; j < P->ny; ++j)
            for (int i = 0; i < P->nx; ++i) {
                int e = i + P->nx * (j + P->ny * k);
                int nodes[8];
                cell_corners(P, i, j, k, nodes);
                double pl[8], cl[8];
                for (int L = 0; L < 8; ++L) {
                    pl[L] = p[nodes[L]];
                    cl[L] = c[nodes[L]];
                }
                /* storage derivatives (diagonal in the node) */
                for (int L = 0; L < 8; ++L) {
                    int n = nodes[L];
                    double dSp = phi[e] * vscv * drho / dt;
                    double dSc = phi[e] * vscv *
                                 (rho_of(P, c[n]) + drho * c[n]) / dt;
                    csr_add(rowptr, col, val, 2 * n, 2 * n + 1, dSp);
                    csr_add(rowptr, col, val, 2 * n + 1, 2 * n + 1, dSc);
                }
                for (int q = 0; q < 12; ++q) {
                    const scvf* f = &faces[q];
                    face_flux ff;
                    eval_face(P, f, phi[e], K[e], pl, cl, &ff);
                    int a = nodes[f->La], b = nodes[f->Lb];
                    double kmu = K[e] / P->mu;
                    for (int L = 0; L < 8; ++L) {
                        /* dm/dp_L and dm/dc_L */
                        double dm_dp = ff.rho_ip * (-kmu) * f->dN[L] * f->A;
                        double dqn_dc = 0.0;
                        if (f->d == 2) /* d(rho g_z)/dc_L = -g N_L drho */
                            dqn_dc = -kmu * (P->g * f->N[L] * drho);
                        double dm_dc = drho * f->N[L] * ff.qn * f->A +
                                       ff.rho_ip * dqn_dc * f->A;
                        double dF_dp = ff.cup * dm_dp;
                        double dF_dc = ff.cup * dm_dc +
                                       (L == ff.up ? ff.m : 0.0) -
                                       drho * f->N[L] * phi[e] * P->Dm *
                                           ff.gradc * f->A -
                                       ff.rho_ip * phi[e] * P->Dm * f->dN[L] *
                                           f->A;
                        int cp = 2 * nodes[L], cc = 2 * nodes[L] + 1;
                        csr_add(rowptr, col, val, 2 * a, cp, dm_dp);
                        csr_add(rowptr, col, val, 2 * a, cc, dm_dc);
                        csr_add(rowptr, col, val, 2 * b, cp, -dm_dp);
                        csr_add(rowptr, col, val, 2 * b, cc, -dm_dc);
                        csr_add(rowptr, col, val, 2 * a + 1, cp, dF_dp);
                        csr_add(rowptr, col, val, 2 * a + 1, cc, dF_dc);
                        csr_add(rowptr, col, val, 2 * b + 1, cp, -dF_dp);
                        csr_add(rowptr, col, val, 2 * b + 1, cc, -dF_dc);
                    }
                }
            }
    /* Dirichlet rows: R = u - u_D, so the row is the identity. */
    unsigned char* pm = (unsigned char*)malloc((size_t)N);
    unsigned char* cm = (unsigned char*)malloc((size_t)N);
    orc_dirichlet(P, pm, cm, NULL);
    for (int n = 0; n < N; ++n)
        for (int v = 0; v < 2; ++v) {
            if (!(v == 0 ? pm[n] : cm[n])) continue;
            int r = 2 * n + v;
            for (int q = rowptr[r]; q < rowptr[r + 1]; ++q)
                val[q] = (col[q] == r) ? 1.0 : 0.0;
        }
    free(pm);
    free(cm);
}

void orc_csr_transpose(int n, const int* rowptr, const int* col,
                       const double* val, int* trowptr, int* tcol,
                       double* tval)
{
    int nnz = rowptr[n];
    int* cnt = (int*)calloc((size_t)n + 1, sizeof(int));
    for (int q = 0; q < nnz; ++q) cnt[col[q] + 1]++;
    for (int r = 0; r < n; ++r) cnt[r + 1] += cnt[r];
    memcpy(trowptr, cnt, sizeof(int) * ((size_t)n + 1));
    for (int r = 0; r < n; ++r)
        for (int q = rowptr[r]; q < rowptr[r + 1]; ++q) {
            int dst = cnt[col[q]]++;
            tcol[dst] = r;
            tval[dst] = val[q];
        }
    free(cnt);
}

/* ------------------------------------------------------------------------ */
/* linear solvers                                                           */
/* ------------------------------------------------------------------------ */

int orc_dense_solve(int n, double* A, double* b)
{
    for (int k = 0; k < n; ++k) {
        int piv = k;
        double best = fabs(A[(size_t)k * n + k]);
        for (int r = k + 1; r < n; ++r)
            if (fabs(A[(size_t)r * n + k]) > best) {
                best = fabs(A[(size_t)r * n + k]);
                piv = r;
            }
        if (best == 0.0) return 1;
        if (piv != k) {
            for (int cidx = 0; cidx < n; ++cidx) {
                double tmp = A[(size_t)k * n + cidx];
                A[(size_t)k * n + cidx] = A[(size_t)piv * n + cidx];
                A[(size_t)piv * n + cidx] = tmp;
            }
            double tb = b[k];
            b[k] = b[piv];
            b[piv] = tb;
        }
        for (int r = k + 1; r < n; ++r) {
            double l = A[(size_t)r * n + k] / A[(size_t)k * n + k];
            if (l == 0.0) continue;
            for (int cidx = k; cidx < n; ++cidx)
                A[(size_t)r * n + cidx] -= l * A[(size_t)k * n + cidx];
            b[r] -= l * b[k];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        double s = b[r];
        for (int cidx = r + 1; cidx < n; ++cidx)
            s -= A[(size_t)r * n + cidx] * b[cidx];
        b[r] = s / A[(size_t)r * n + r];
    }
    return 0;
}

static void csr_matvec(int n, const int* rowptr, const int* col,
                       const double* val, const double* x, double* y)
{
    for (int r = 0; r < n; ++r) {
        double s = 0.0;
        for (int q = rowptr[r]; q < rowptr[r + 1]; ++q) s += val[q] * x[col[q]];
        y[r] = s;
    }
}

static double dot(int n, const double* a, const double* b)
{
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* ILU(0): incomplete LU restricted to the pattern of A (Saad, Iterative
 * Methods for Sparse Linear Systems, Alg. 10.4).  lu holds L (unit lower,
 * strictly below the diagonal) and U. */
static void ilu0(int n, const int* rowptr, const int* col, const double* val,
                 double* lu, int* diag)
{
    memcpy(lu, val, sizeof(double) * (size_t)rowptr[n]);
    int* pos = (int*)malloc(sizeof(int) * (size_t)n);
    for (int i = 0; i < n; ++i) pos[i] = -1;
    for (int i = 0; i < n; ++i) {
        for (int q = rowptr[i]; q < rowptr[i + 1]; ++q) {
            pos[col[q]] = q;
            if (col[q] == i) diag[i] = q;
        }
        for (int q = rowptr[i]; q < rowptr[i + 1] && col[q] < i; ++q) {
            int kk = col[q];
            lu[q] /= lu[diag[kk]];
            for (int r = diag[kk] + 1; r < rowptr[kk + 1]; ++r) {
                int jj = col[r];
                if (pos[jj] >= 0) lu[pos[jj]] -= lu[q] * lu[r];
            }
        }
        for (int q = rowptr[i]; q < rowptr[i + 1]; ++q) pos[col[q]] = -1;
    }
    free(pos);
}

static void ilu0_apply(int n, const int* rowptr, const int* col,
                       const double* lu, const int* diag, const double* r,
                       double* z)
{
    for (int i = 0; i < n; ++i) {
        double s = r[i];
        for (int q = rowptr[i]; q < diag[i]; ++q) s -= lu[q] * z[col[q]];
        z[i] = s;
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = z[i];
        for (int q = diag[i] + 1; q < rowptr[i + 1]; ++q) s -= lu[q] * z[col[q]];
        z[i] = s / lu[diag[i]];
    }
}

/* preconditioner z = M r */
typedef void (*precond_fn)(void* ctx, const double* r, double* z);

typedef struct {
    int n;
    const int *rowptr, *col;
    const double* lu;
    const int* diag;
} ilu_ctx;

static void ilu_precond(void* vctx, const double* r, double* z)
{
    ilu_ctx* c = (ilu_ctx*)vctx;
    ilu0_apply(c->n, c->rowptr, c->col, c->lu, c->diag, r, z);
}

static int bicgstab(int n, const int* rowptr, const int* col,
                    const double* val, const double* b, double* x, double rtol,
                    int maxit, precond_fn M, void* mctx, int* iters,
                    double* relres);

int orc_bicgstab_ilu0(int n, const int* rowptr, const int* col,
                      const double* val, const double* b, double* x,
                      double rtol, int maxit, int* iters, double* relres)
{
    double* lu = (double*)malloc(sizeof(double) * (size_t)rowptr[n]);
    int* diag = (int*)malloc(sizeof(int) * (size_t)n);
    ilu0(n, rowptr, col, val, lu, diag);
    ilu_ctx ic = {n, rowptr, col, lu, diag};
    int rc = bicgstab(n, rowptr, col, val, b, x, rtol, maxit, ilu_precond, &ic,
                      iters, relres);
    free(lu);
    free(diag);
    return rc;
}

/* BiCGStab of van der Vorst, right preconditioned (Barrett et al.,
 * Templates, Sec. 2.3.8); the method the paper names in Section 5.1. */
static int bicgstab(int n, const int* rowptr, const int* col,
                    const double* val, const double* b, double* x, double rtol,
                    int maxit, precond_fn M, void* mctx, int* iters,
                    double* relres)
{
    size_t sz = sizeof(double) * (size_t)n;
    double *r = malloc(sz), *rh = malloc(sz), *pv = malloc(sz), *v = malloc(sz),
           *s = malloc(sz), *t = malloc(sz), *ph = malloc(sz), *sh = malloc(sz);
    csr_matvec(n, rowptr, col, val, x, r);
    for (int i = 0; i < n; ++i) {
        r[i] = b[i] - r[i];
        rh[i] = r[i];
        pv[i] = v[i] = 0.0;
    }
    double bn = sqrt(dot(n, b, b));
    if (bn == 0.0) bn = 1.0;
    double rho_old = 1.0, alpha = 1.0, omega = 1.0;
    double rn = sqrt(dot(n, r, r));
    int it = 0, ok = (rn <= rtol * bn);
    while (!ok && it < maxit) {
        ++it;
        double rho = dot(n, rh, r);
        if (rho == 0.0) break;
        double beta = (rho / rho_old) * (alpha / omega);
        for (int i = 0; i < n; ++i) pv[i] = r[i] + beta * (pv[i] - omega * v[i]);
        M(mctx, pv, ph);
        csr_matvec(n, rowptr, col, val, ph, v);
        double rv = dot(n, rh, v);
        if (rv == 0.0) break;
        alpha = rho / rv;
        for (int i = 0; i < n; ++i) s[i] = r[i] - alpha * v[i];
        if (sqrt(dot(n, s, s)) <= rtol * bn) {
            for (int i = 0; i < n; ++i) x[i] += alpha * ph[i];
            ok = 1;
            break;
        }
        M(mctx, s, sh);
        csr_matvec(n, rowptr, col, val, sh, t);
        double tt = dot(n, t, t);
        omega = (tt > 0.0) ? dot(n, t, s) / tt : 0.0;
        for (int i = 0; i < n; ++i) {
            x[i] += alpha * ph[i] + omega * sh[i];
            r[i] = s[i] - omega * t[i];
        }
        rho_old = rho;
        rn = sqrt(dot(n, r, r));
        if (rn <= rtol * bn) ok = 1;
        if (omega == 0.0) break;
    }
    /* report the true residual */
    csr_matvec(n, rowptr, col, val, x, r);
    for (int i = 0; i < n; ++i) r[i] = b[i] - r[i];
    double tr = sqrt(dot(n, r, r)) / bn;
    if (iters) *iters = it;
    if (relres) *relres = tr;
    free(r); free(rh); free(pv); free(v); free(s);
    free(t); free(ph); free(sh);
    return (tr <= 10.0 * rtol) ? 0 : 1;
}

int orc_linear_solve(int n, const int* rowptr, const int* col,
                     const double* val, const double* b, double* x,
                     const orc_newton_opts* o, int* iters)
{
    if (n <= o->dense_max) {
        double* A = (double*)calloc((size_t)n * n, sizeof(double));
        for (int r = 0; r < n; ++r)
            for (int q = rowptr[r]; q < rowptr[r + 1]; ++q)
                A[(size_t)r * n + col[q]] += val[q];
        memcpy(x, b, sizeof(double) * (size_t)n);
        int rc = orc_dense_solve(n, A, x);
        free(A);
        if (iters) *iters = 0;
        return rc;
    }
    for (int i = 0; i < n; ++i) x[i] = 0.0;
    double rr;
    return orc_bicgstab_ilu0(n, rowptr, col, val, b, x, o->lin_rtol,
                             o->lin_maxit, iters, &rr);
}

/* ------------------------------------------------------------------------ */
/* geometric multigrid V-cycle preconditioner (Section 5.1)                 */
/* ------------------------------------------------------------------------ */
/* Levels: the grid halved in every direction while that keeps the top
 * square node-aligned; the matrix of every level is the Jacobian of the
 * discretised system on that grid (Section 5.1), at the injected state and
 * with cell-averaged phi and K.  Each level matrix is taken on the interior
 * unknowns: Dirichlet rows and columns are replaced by the identity and the
 * Dirichlet components of every multigrid vector are kept at zero.
 * Smoothers: damped 2x2-block Jacobi, damped block Jacobi over vertical
 * grid lines, or the multicolour block ILU_beta(0) (the paper's ILU_beta
 * smoother is not specified further); transfers: trilinear interpolation
 * and its transpose; coarsest level: dense LU. */

#define ORC_MAXLEV 16

typedef struct {
    int nlev;
    orc_problem P[ORC_MAXLEV];
    int n[ORC_MAXLEV];
    int *rp[ORC_MAXLEV], *ci[ORC_MAXLEV];
    double* A[ORC_MAXLEV];
    double* Dinv[ORC_MAXLEV];     /* [N][4]: inverse of the 2x2 diagonal block */
    unsigned char* dm[ORC_MAXLEV];/* [2N]: 1 on Dirichlet unknowns            */
    double *b[ORC_MAXLEV], *x[ORC_MAXLEV], *r[ORC_MAXLEV];
    double* LU;
    int* piv;
    int nu1, nu2;
    double omega;
    int line;                     /* vertical-line smoother (else point)      */
    int ilu;                      /* multicolour block ILU_beta(0) smoother   */
    int ilu_trans;                /* its factors are the untransposed level
                                     matrix's: sweeps apply (L U)^{-T}        */
    double* F[ORC_MAXLEV];        /* [N][27][4] ILU factors                   */
    double* Lb[ORC_MAXLEV];       /* [N][4] line blocks A(n, n-below)         */
    double* Db[ORC_MAXLEV];       /* [N][4] diagonal blocks A(n, n)           */
    double* Ub[ORC_MAXLEV];       /* [N][4] line blocks A(n, n-above)         */
} orc_mg;

static int mg_can_coarsen(const orc_problem* P)
{
    if (P->nx % 2 || P->ny % 2 || P->nz % 2) return 0;
    if ((P->bc_mode == 0 || P->bc_mode == 1) &&
        (((P->nx / 2) % 4) || ((P->ny / 2) % 4)))
        return 0;
    return 1;
}

static void mg_free(orc_mg* mg)
{
    for (int l = 0; l < mg->nlev; ++l) {
        free(mg->rp[l]); free(mg->ci[l]); free(mg->A[l]); free(mg->Dinv[l]);
        free(mg->dm[l]); free(mg->b[l]); free(mg->x[l]); free(mg->r[l]);
        free(mg->Lb[l]); free(mg->Db[l]); free(mg->Ub[l]); free(mg->F[l]);
    }
    free(mg->LU);
    free(mg->piv);
}

static double csr_get(const int* rp, const int* ci, const double* A, int r,
                      int c)
{
    for (int q = rp[r]; q < rp[r + 1]; ++q)
        if (ci[q] == c) return A[q];
    return 0.0;
}

/* the 2x2 block of rows (2r, 2r+1) and columns (2q, 2q+1), row-major */
static void csr_block(const int* rp, const int* ci, const double* A, int r, int q,
                      double* B)
{
    B[0] = csr_get(rp, ci, A, 2 * r, 2 * q);
    B[1] = csr_get(rp, ci, A, 2 * r, 2 * q + 1);
    B[2] = csr_get(rp, ci, A, 2 * r + 1, 2 * q);
    B[3] = csr_get(rp, ci, A, 2 * r + 1, 2 * q + 1);
}

static int mg_setup(orc_mg* mg, const orc_problem* P0, const double* phi0,
                    const double* K0, const double* p0, const double* c0,
                    double dt, int transpose, int smoother, double beta)
{
    int line = smoother == 1;
    memset(mg, 0, sizeof(*mg));
    /* point smoother, damping 0.5: at dt = 1/12 yr the pressure/salt
     * coupling next to the salt source makes block Jacobi with damping 0.7
     * diverge on some permeability fields.  Line smoother, damping 0.7: the
     * vertical coupling (gravity, the salt front) is solved exactly per
     * line, which keeps the V-cycle's contraction nearly independent of the
     * grid size where point Jacobi slows down. */
    mg->nu1 = 1;
    mg->nu2 = 1;
    mg->line = line;
    mg->ilu = smoother == 2;
    mg->ilu_trans = mg->ilu && transpose;
    /* ILU sweeps are undamped */
    mg->omega = mg->ilu ? 1.0 : (line ? 0.7 : 0.5);
    orc_problem P = *P0;
    double *phi = (double*)phi0, *K = (double*)K0, *p = (double*)p0,
           *c = (double*)c0;
    int owned = 0;
    int l = 0;
    for (;; ++l) {
        mg->P[l] = P;
        int N = orc_num_nodes(&P), n2 = 2 * N;
        mg->n[l] = n2;
        int nnz = orc_jac_nnz(&P);
        int* rp = malloc(sizeof(int) * ((size_t)n2 + 1));
        int* ci = malloc(sizeof(int) * (size_t)nnz);
        double* A = malloc(sizeof(double) * (size_t)nnz);
        orc_jac_pattern(&P, rp, ci);
        orc_jacobian(&P, phi, K, p, c, dt, rp, ci, A);
        unsigned char* pm = malloc((size_t)N);
        unsigned char* cm = malloc((size_t)N);
        orc_dirichlet(&P, pm, cm, NULL);
        unsigned char* dm = malloc((size_t)n2);
        for (int n = 0; n < N; ++n) {
            dm[2 * n] = pm[n];
            dm[2 * n + 1] = cm[n];
        }
        free(pm);
        free(cm);
        for (int r = 0; r < n2; ++r)
            for (int q = rp[r]; q < rp[r + 1]; ++q) {
                if (dm[r]) A[q] = (ci[q] == r) ? 1.0 : 0.0;
                else if (dm[ci[q]]) A[q] = 0.0;
            }
        if (mg->ilu) {
            /* the factors of the untransposed level matrix: the transposed
             * solve's sweeps use their transpose */
            double* B = (double*)malloc(sizeof(double) * 108 * (size_t)N);
            mg->F[l] = (double*)malloc(sizeof(double) * 108 * (size_t)N);
            orc_csr_to_blocks(&P, rp, ci, A, B);
            int bad = orc_mcilu_factor(&P, B, beta, mg->F[l]);
            free(B);
            if (bad) {
                mg->rp[l] = rp; mg->ci[l] = ci; mg->A[l] = A; mg->dm[l] = dm;
                mg->nlev = l + 1;
                if (owned) { free(phi); free(K); free(p); free(c); }
                return 1;
            }
        }
        if (transpose) {
            int* trp = malloc(sizeof(int) * ((size_t)n2 + 1));
            int* tci = malloc(sizeof(int) * (size_t)nnz);
            double* tA = malloc(sizeof(double) * (size_t)nnz);
            orc_csr_transpose(n2, rp, ci, A, trp, tci, tA);
            free(rp); free(ci); free(A);
            rp = trp; ci = tci; A = tA;
        }
        double* Dinv = malloc(sizeof(double) * 4 * (size_t)N);
        for (int n = 0; n < N; ++n) {
            double a = csr_get(rp, ci, A, 2 * n, 2 * n);
            double b = csr_get(rp, ci, A, 2 * n, 2 * n + 1);
            double cc = csr_get(rp, ci, A, 2 * n + 1, 2 * n);
            double d = csr_get(rp, ci, A, 2 * n + 1, 2 * n + 1);
            double det = a * d - b * cc;
            Dinv[4 * n + 0] = d / det;
            Dinv[4 * n + 1] = -b / det;
            Dinv[4 * n + 2] = -cc / det;
            Dinv[4 * n + 3] = a / det;
        }
        if (line) {
            double* Lb = calloc(4 * (size_t)N, sizeof(double));
            double* Db = calloc(4 * (size_t)N, sizeof(double));
            double* Ub = calloc(4 * (size_t)N, sizeof(double));
            int sz = (P.nx + 1) * (P.ny + 1);
            for (int n = 0; n < N; ++n) {
                int k = n / sz;
                csr_block(rp, ci, A, n, n, Db + 4 * n);
                if (k > 0) csr_block(rp, ci, A, n, n - sz, Lb + 4 * n);
                if (k < P.nz) csr_block(rp, ci, A, n, n + sz, Ub + 4 * n);
            }
            mg->Lb[l] = Lb; mg->Db[l] = Db; mg->Ub[l] = Ub;
        }
        mg->rp[l] = rp; mg->ci[l] = ci; mg->A[l] = A; mg->Dinv[l] = Dinv;
        mg->dm[l] = dm;
        mg->b[l] = calloc((size_t)n2, sizeof(double));
        mg->x[l] = calloc((size_t)n2, sizeof(double));
        mg->r[l] = calloc((size_t)n2, sizeof(double));
        if (!mg_can_coarsen(&P) || l == ORC_MAXLEV - 1) break;
        /* next level: injected state, arithmetic means of phi and K */
        orc_problem Pc = P;
        Pc.nx /= 2; Pc.ny /= 2; Pc.nz /= 2;
        int Nc = orc_num_nodes(&Pc), Cc = orc_num_cells(&Pc);
        double* phic = malloc(sizeof(double) * (size_t)Cc);
        double* Kc = malloc(sizeof(double) * (size_t)Cc);
        double* pc = malloc(sizeof(double) * (size_t)Nc);
        double* cc = malloc(sizeof(double) * (size_t)Nc);
        for (int k = 0; k < Pc.nz; ++k)
            for (int j = 0; j < Pc.ny; ++j)
                for (int i = 0; i < Pc.nx; ++i) {
                    double sp = 0.0, sk = 0.0;
                    for (int q = 0; q < 8; ++q) {
                        int f = (2 * i + (q & 1)) +
                                P.nx * ((2 * j + ((q >> 1) & 1)) +
                                        P.ny * (2 * k + (q >> 2)));
                        sp += phi[f];
                        sk += K[f];
                    }
                    phic[i + Pc.nx * (j + Pc.ny * k)] = sp / 8.0;
                    Kc[i + Pc.nx * (j + Pc.ny * k)] = sk / 8.0;
                }
        for (int k = 0; k <= Pc.nz; ++k)
            for (int j = 0; j <= Pc.ny; ++j)
                for (int i = 0; i <= Pc.nx; ++i) {
                    int f = node_id(&P, 2 * i, 2 * j, 2 * k);
                    pc[node_id(&Pc, i, j, k)] = p[f];
                    cc[node_id(&Pc, i, j, k)] = c[f];
                }
        if (owned) { free(phi); free(K); free(p); free(c); }
        phi = phic; K = Kc; p = pc; c = cc;
        owned = 1;
        P = Pc;
    }
    if (owned) { free(phi); free(K); free(p); free(c); }
    mg->nlev = l + 1;
    /* dense LU (partial pivoting) of the coarsest level */
    int L = mg->nlev - 1, n = mg->n[L];
    if (n > 4000) return 1;
    mg->LU = calloc((size_t)n * n, sizeof(double));
    mg->piv = malloc(sizeof(int) * (size_t)n);
    for (int r = 0; r < n; ++r)
        for (int q = mg->rp[L][r]; q < mg->rp[L][r + 1]; ++q)
            mg->LU[(size_t)r * n + mg->ci[L][q]] += mg->A[L][q];
    double* M = mg->LU;
    for (int k = 0; k < n; ++k) {
        int pv = k;
        for (int r = k + 1; r < n; ++r)
            if (fabs(M[(size_t)r * n + k]) > fabs(M[(size_t)pv * n + k])) pv = r;
        mg->piv[k] = pv;
        if (M[(size_t)pv * n + k] == 0.0) return 1;
        if (pv != k)
            for (int q = 0; q < n; ++q) {
                double t = M[(size_t)k * n + q];
                M[(size_t)k * n + q] = M[(size_t)pv * n + q];
                M[(size_t)pv * n + q] = t;
            }
        for (int r = k + 1; r < n; ++r) {
            double f = M[(size_t)r * n + k] / M[(size_t)k * n + k];
            M[(size_t)r * n + k] = f;
            for (int q = k + 1; q < n; ++q) M[(size_t)r * n + q] -= f * M[(size_t)k * n + q];
        }
    }
    return 0;
}

static void mg_coarse_solve(const orc_mg* mg, double* x)
{
    int n = mg->n[mg->nlev - 1];
    const double* M = mg->LU;
    for (int k = 0; k < n; ++k) {
        int pv = mg->piv[k];
        if (pv != k) { double t = x[k]; x[k] = x[pv]; x[pv] = t; }
        for (int r = k + 1; r < n; ++r) x[r] -= M[(size_t)r * n + k] * x[k];
    }
    for (int r = n - 1; r >= 0; --r) {
        double s = x[r];
        for (int q = r + 1; q < n; ++q) s -= M[(size_t)r * n + q] * x[q];
        x[r] = s / M[(size_t)r * n + r];
    }
}

static void mg_zero_dirichlet(const orc_mg* mg, int l, double* v)
{
    for (int i = 0; i < mg->n[l]; ++i)
        if (mg->dm[l][i]) v[i] = 0.0;
}

static void inv2x2(const double* M, double* Mi)
{
    double det = M[0] * M[3] - M[1] * M[2];
    Mi[0] = M[3] / det;
    Mi[1] = -M[1] / det;
    Mi[2] = -M[2] / det;
    Mi[3] = M[0] / det;
}

/* one damped line sweep: x += omega T^{-1} (b - A x), T the block-tridiagonal
 * part of A along each vertical grid line (i, j fixed), solved by block
 * Gaussian elimination (Thomas algorithm with 2x2 blocks) */
static void mg_smooth_line(const orc_mg* mg, int l, const double* b, double* x,
                           double* tmp)
{
    const orc_problem* P = &mg->P[l];
    int n = mg->n[l], nz = P->nz, sz = (P->nx + 1) * (P->ny + 1);
    csr_matvec(n, mg->rp[l], mg->ci[l], mg->A[l], x, tmp);
    double* C = malloc(sizeof(double) * 4 * (size_t)(nz + 1));
    double* g = malloc(sizeof(double) * 2 * (size_t)(nz + 1));
    for (int col = 0; col < sz; ++col) {
        for (int k = 0; k <= nz; ++k) {        /* forward elimination */
            int node = col + k * sz;
            double M[4], r[2], Mi[4];
            const double* D = mg->Db[l] + 4 * node;
            M[0] = D[0]; M[1] = D[1]; M[2] = D[2]; M[3] = D[3];
            r[0] = b[2 * node] - tmp[2 * node];
            r[1] = b[2 * node + 1] - tmp[2 * node + 1];
            if (k > 0) {                       /* M -= L C_{k-1}, r -= L g_{k-1} */
                const double* L = mg->Lb[l] + 4 * node;
                const double* Cp = C + 4 * (k - 1);
                const double* gp = g + 2 * (k - 1);
                M[0] -= L[0] * Cp[0] + L[1] * Cp[2];
                M[1] -= L[0] * Cp[1] + L[1] * Cp[3];
                M[2] -= L[2] * Cp[0] + L[3] * Cp[2];
                M[3] -= L[2] * Cp[1] + L[3] * Cp[3];
                r[0] -= L[0] * gp[0] + L[1] * gp[1];
                r[1] -= L[2] * gp[0] + L[3] * gp[1];
            }
            inv2x2(M, Mi);
            if (k < nz) {                      /* C_k = M^{-1} U_k */
                const double* U = mg->Ub[l] + 4 * node;
                C[4 * k + 0] = Mi[0] * U[0] + Mi[1] * U[2];
                C[4 * k + 1] = Mi[0] * U[1] + Mi[1] * U[3];
                C[4 * k + 2] = Mi[2] * U[0] + Mi[3] * U[2];
                C[4 * k + 3] = Mi[2] * U[1] + Mi[3] * U[3];
            }
            g[2 * k + 0] = Mi[0] * r[0] + Mi[1] * r[1];
            g[2 * k + 1] = Mi[2] * r[0] + Mi[3] * r[1];
        }
        for (int k = nz - 1; k >= 0; --k) {    /* back substitution */
            g[2 * k + 0] -= C[4 * k + 0] * g[2 * k + 2] + C[4 * k + 1] * g[2 * k + 3];
            g[2 * k + 1] -= C[4 * k + 2] * g[2 * k + 2] + C[4 * k + 3] * g[2 * k + 3];
        }
        for (int k = 0; k <= nz; ++k) {
            int node = col + k * sz;
            x[2 * node] += mg->omega * g[2 * k];
            x[2 * node + 1] += mg->omega * g[2 * k + 1];
        }
    }
    free(C);
    free(g);
    mg_zero_dirichlet(mg, l, x);
}

/* ------------------------------------------------------------------------ */
/* Multicolour block ILU_beta(0) (Section 5.1)                              */
/* ------------------------------------------------------------------------ */
/* The paper's multigrid smoother is ILU_beta, not specified further.
 * Reading: the incomplete LU factorisation with 2x2 blocks for scalars,
 * restricted to the block pattern of the level matrix (the 27-point
 * stencil), in the multicolour order of the nodes: colour = (i&1) + 2(j&1)
 * + 4(k&1), colours ascending, node index order within a colour.  Two nodes
 * of one colour never share a cell, so each colour class is an independent
 * set of the stencil.  The factorisation is Gaussian elimination in its IKJ
 * form with every update of an entry outside the pattern dropped (Saad,
 * Iterative Methods for Sparse Linear Systems, 2nd ed., Alg. 10.4); beta
 * times the dropped block is subtracted from the row's diagonal block
 * instead (beta = 0: block ILU(0); beta = 1: block modified ILU, whose L U
 * keeps every block row sum of A). */

static void node_ijk(const orc_problem* P, int n, int* i, int* j, int* k)
{
    int sx = P->nx + 1, sy = P->ny + 1;
    *i = n % sx;
    *j = (n / sx) % sy;
    *k = n / (sx * sy);
}

void orc_mc_rank(const orc_problem* P, int* rank)
{
    int N = orc_num_nodes(P), q = 0;
    for (int colour = 0; colour < 8; ++colour)
        for (int n = 0; n < N; ++n) {
            int i, j, k;
            node_ijk(P, n, &i, &j, &k);
            if (((i & 1) | ((j & 1) << 1) | ((k & 1) << 2)) == colour) rank[n] = q++;
        }
}

/* the neighbour of node n in slot s, or -1 outside the grid */
static int slot_node(const orc_problem* P, int n, int s)
{
    int i, j, k;
    node_ijk(P, n, &i, &j, &k);
    i += s % 3 - 1;
    j += (s / 3) % 3 - 1;
    k += s / 9 - 1;
    if (i < 0 || i > P->nx || j < 0 || j > P->ny || k < 0 || k > P->nz) return -1;
    return node_id(P, i, j, k);
}

/* the slot of node m in the row of node n, or -1 when they are not
 * neighbours */
static int node_slot(const orc_problem* P, int n, int m)
{
    int i, j, k, a, b, c;
    node_ijk(P, n, &i, &j, &k);
    node_ijk(P, m, &a, &b, &c);
    int dx = a - i, dy = b - j, dz = c - k;
    if (dx < -1 || dx > 1 || dy < -1 || dy > 1 || dz < -1 || dz > 1) return -1;
    return (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1);
}

void orc_csr_to_blocks(const orc_problem* P, const int* rowptr, const int* col,
                       const double* val, double* B)
{
    int N = orc_num_nodes(P);
    memset(B, 0, sizeof(double) * 108 * (size_t)N);
    for (int n = 0; n < N; ++n)
        for (int v = 0; v < 2; ++v)
            for (int q = rowptr[2 * n + v]; q < rowptr[2 * n + v + 1]; ++q) {
                int m = col[q] / 2, w = col[q] % 2;
                int s = node_slot(P, n, m);
                if (s < 0) abort();  /* not the 27-point block pattern */
                B[(size_t)n * 108 + 4 * s + 2 * v + w] += val[q];
            }
}

static void mul2x2(const double* a, const double* b, double* c)
{
    c[0] = a[0] * b[0] + a[1] * b[2];
    c[1] = a[0] * b[1] + a[1] * b[3];
    c[2] = a[2] * b[0] + a[3] * b[2];
    c[3] = a[2] * b[1] + a[3] * b[3];
}

int orc_mcilu_factor(const orc_problem* P, const double* A, double beta, double* F)
{
    int N = orc_num_nodes(P);
    int* rank = (int*)malloc(sizeof(int) * (size_t)N);
    int* order = (int*)malloc(sizeof(int) * (size_t)N);
    orc_mc_rank(P, rank);
    for (int n = 0; n < N; ++n) order[rank[n]] = n;
    memcpy(F, A, sizeof(double) * 108 * (size_t)N);
    int singular = 0;
    for (int q = 0; q < N; ++q) {
        int i = order[q];
        double* Fi = F + (size_t)i * 108;
        /* the slots of the row's earlier neighbours, by ascending rank */
        int ks[27], nk = 0;
        for (int s = 0; s < 27; ++s) {
            int k = slot_node(P, i, s);
            if (k < 0 || rank[k] >= rank[i]) continue;
            int t = nk++;
            while (t > 0 && rank[slot_node(P, i, ks[t - 1])] > rank[k]) {
                ks[t] = ks[t - 1];
                --t;
            }
            ks[t] = s;
        }
        for (int a = 0; a < nk; ++a) {
            int k = slot_node(P, i, ks[a]);
            const double* Fk = F + (size_t)k * 108;
            double Ui[4], l[4];
            inv2x2(Fk + 4 * 13, Ui);
            mul2x2(Fi + 4 * ks[a], Ui, l);            /* L_ik = A_ik U_kk^{-1} */
            memcpy(Fi + 4 * ks[a], l, sizeof l);
            for (int e = 0; e < 27; ++e) {            /* row k's U part */
                int j = slot_node(P, k, e);
                if (j < 0 || rank[j] <= rank[k]) continue;
                double lu[4];
                mul2x2(l, Fk + 4 * e, lu);
                int t = node_slot(P, i, j);
                for (int r = 0; r < 4; ++r) {
                    if (t >= 0) Fi[4 * t + r] -= lu[r];
                    else Fi[4 * 13 + r] -= beta * lu[r];
                }
            }
        }
        const double* D = Fi + 4 * 13;
        if (D[0] * D[3] - D[1] * D[2] == 0.0) singular = 1;
    }
    free(rank);
    free(order);
    return singular;
}

void orc_mcilu_solve(const orc_problem* P, const double* F, int transpose,
                     const double* r, double* z)
{
    int N = orc_num_nodes(P);
    int* rank = (int*)malloc(sizeof(int) * (size_t)N);
    int* order = (int*)malloc(sizeof(int) * (size_t)N);
    orc_mc_rank(P, rank);
    for (int n = 0; n < N; ++n) order[rank[n]] = n;
    /* z holds y of the first sweep, then the result */
    if (!transpose) {
        for (int q = 0; q < N; ++q) {                 /* L y = r */
            int i = order[q];
            double y0 = r[2 * i], y1 = r[2 * i + 1];
            for (int s = 0; s < 27; ++s) {
                int k = slot_node(P, i, s);
                if (k < 0 || rank[k] >= rank[i]) continue;
                const double* Lb = F + (size_t)i * 108 + 4 * s;
                y0 -= Lb[0] * z[2 * k] + Lb[1] * z[2 * k + 1];
                y1 -= Lb[2] * z[2 * k] + Lb[3] * z[2 * k + 1];
            }
            z[2 * i] = y0;
            z[2 * i + 1] = y1;
        }
        for (int q = N - 1; q >= 0; --q) {            /* U z = y */
            int i = order[q];
            double t0 = z[2 * i], t1 = z[2 * i + 1], Di[4];
            for (int s = 0; s < 27; ++s) {
                int j = slot_node(P, i, s);
                if (j < 0 || rank[j] <= rank[i]) continue;
                const double* Ub = F + (size_t)i * 108 + 4 * s;
                t0 -= Ub[0] * z[2 * j] + Ub[1] * z[2 * j + 1];
                t1 -= Ub[2] * z[2 * j] + Ub[3] * z[2 * j + 1];
            }
            inv2x2(F + (size_t)i * 108 + 4 * 13, Di);
            z[2 * i] = Di[0] * t0 + Di[1] * t1;
            z[2 * i + 1] = Di[2] * t0 + Di[3] * t1;
        }
    } else {
        /* (L U)^T = U^T L^T; U^T is lower block triangular in the order, with
         * the transposed pivots on its diagonal, L^T upper with unit blocks */
        for (int q = 0; q < N; ++q) {                 /* U^T y = r */
            int i = order[q];
            double t0 = r[2 * i], t1 = r[2 * i + 1], Di[4];
            for (int s = 0; s < 27; ++s) {
                int j = slot_node(P, i, s);
                if (j < 0 || rank[j] >= rank[i]) continue;
                const double* Ub = F + (size_t)j * 108 + 4 * node_slot(P, j, i);
                t0 -= Ub[0] * z[2 * j] + Ub[2] * z[2 * j + 1];
                t1 -= Ub[1] * z[2 * j] + Ub[3] * z[2 * j + 1];
            }
            inv2x2(F + (size_t)i * 108 + 4 * 13, Di);
            z[2 * i] = Di[0] * t0 + Di[2] * t1;
            z[2 * i + 1] = Di[1] * t0 + Di[3] * t1;
        }
        for (int q = N - 1; q >= 0; --q) {            /* L^T z = y */
            int i = order[q];
            double t0 = z[2 * i], t1 = z[2 * i + 1];
            for (int s = 0; s < 27; ++s) {
                int j = slot_node(P, i, s);
                if (j < 0 || rank[j] <= rank[i]) continue;
                const double* Lb = F + (size_t)j * 108 + 4 * node_slot(P, j, i);
                t0 -= Lb[0] * z[2 * j] + Lb[2] * z[2 * j + 1];
                t1 -= Lb[1] * z[2 * j] + Lb[3] * z[2 * j + 1];
            }
            z[2 * i] = t0;
            z[2 * i + 1] = t1;
        }
    }
    free(rank);
    free(order);
}

/* one ILU sweep: x += omega (L U)^{-1} (b - A x), or (L U)^{-T} for the
 * transposed level matrix (the factors of the untransposed one) */
static void mg_smooth_ilu(const orc_mg* mg, int l, const double* b, double* x,
                          double* tmp)
{
    int n = mg->n[l];
    csr_matvec(n, mg->rp[l], mg->ci[l], mg->A[l], x, tmp);
    double* r = (double*)calloc((size_t)n, sizeof(double));
    double* z = (double*)calloc((size_t)n, sizeof(double));
    for (int i = 0; i < n; ++i) r[i] = mg->dm[l][i] ? 0.0 : b[i] - tmp[i];
    orc_mcilu_solve(&mg->P[l], mg->F[l], mg->ilu_trans, r, z);
    for (int i = 0; i < n; ++i) x[i] += mg->omega * z[i];
    free(r);
    free(z);
    mg_zero_dirichlet(mg, l, x);
}

/* one damped block-Jacobi sweep: x += omega D^{-1} (b - A x) */
static void mg_smooth(const orc_mg* mg, int l, const double* b, double* x,
                      double* tmp)
{
    int n = mg->n[l];
    if (mg->line) {
        mg_smooth_line(mg, l, b, x, tmp);
        return;
    }
    if (mg->ilu) {
        mg_smooth_ilu(mg, l, b, x, tmp);
        return;
    }
    csr_matvec(n, mg->rp[l], mg->ci[l], mg->A[l], x, tmp);
    for (int node = 0; node < n / 2; ++node) {
        double rp = b[2 * node] - tmp[2 * node];
        double rc = b[2 * node + 1] - tmp[2 * node + 1];
        const double* D = mg->Dinv[l] + 4 * node;
        x[2 * node] += mg->omega * (D[0] * rp + D[1] * rc);
        x[2 * node + 1] += mg->omega * (D[2] * rp + D[3] * rc);
    }
    mg_zero_dirichlet(mg, l, x);
}

/* Trilinear interpolation from level l+1 to level l, written as a scatter
 * of every coarse value to the fine nodes within one fine cell of it, with
 * weight prod_d (1 - |offset_d|/2); restriction is its transpose. */
static void mg_transfer(const orc_mg* mg, int l, double* fine, double* coarse,
                        int restrict_)
{
    const orc_problem* Pf = &mg->P[l];
    const orc_problem* Pc = &mg->P[l + 1];
    if (restrict_)
        for (int q = 0; q < mg->n[l + 1]; ++q) coarse[q] = 0.0;
    for (int K = 0; K <= Pc->nz; ++K)
        for (int J = 0; J <= Pc->ny; ++J)
            for (int I = 0; I <= Pc->nx; ++I) {
                int nc = node_id(Pc, I, J, K);
                for (int c = -1; c <= 1; ++c)
                    for (int b = -1; b <= 1; ++b)
                        for (int a = -1; a <= 1; ++a) {
                            int i = 2 * I + a, j = 2 * J + b, k = 2 * K + c;
                            if (i < 0 || i > Pf->nx || j < 0 || j > Pf->ny || k < 0 ||
                                k > Pf->nz)
                                continue;
                            double w = (a ? 0.5 : 1.0) * (b ? 0.5 : 1.0) * (c ? 0.5 : 1.0);
                            int nf = node_id(Pf, i, j, k);
                            for (int v = 0; v < 2; ++v) {
                                if (restrict_) coarse[2 * nc + v] += w * fine[2 * nf + v];
                                else fine[2 * nf + v] += w * coarse[2 * nc + v];
                            }
                        }
            }
}

static void mg_vcycle(const orc_mg* mg, int l, const double* b, double* x)
{
    int n = mg->n[l];
    if (l == mg->nlev - 1) {
        memcpy(x, b, sizeof(double) * (size_t)n);
        mg_coarse_solve(mg, x);
        mg_zero_dirichlet(mg, l, x);
        return;
    }
    double* tmp = mg->r[l];
    for (int i = 0; i < n; ++i) x[i] = 0.0;
    for (int s = 0; s < mg->nu1; ++s) mg_smooth(mg, l, b, x, tmp);
    csr_matvec(n, mg->rp[l], mg->ci[l], mg->A[l], x, tmp);
    for (int i = 0; i < n; ++i) tmp[i] = b[i] - tmp[i];
    mg_zero_dirichlet(mg, l, tmp);
    mg_transfer(mg, l, tmp, mg->b[l + 1], 1);
    mg_zero_dirichlet(mg, l + 1, mg->b[l + 1]);
    mg_vcycle(mg, l + 1, mg->b[l + 1], mg->x[l + 1]);
    mg_transfer(mg, l, x, mg->x[l + 1], 0);
    mg_zero_dirichlet(mg, l, x);
    for (int s = 0; s < mg->nu2; ++s) mg_smooth(mg, l, b, x, tmp);
}

/* z = M r for the full Jacobian: the V-cycle on the interior unknowns and
 * the identity on the Dirichlet unknowns (whose rows are identity rows). */
static void mg_precond(void* vctx, const double* r, double* z)
{
    orc_mg* mg = (orc_mg*)vctx;
    int n = mg->n[0];
    double* b = mg->b[0];
    memcpy(b, r, sizeof(double) * (size_t)n);
    mg_zero_dirichlet(mg, 0, b);
    mg_vcycle(mg, 0, b, z);
    for (int i = 0; i < n; ++i)
        if (mg->dm[0][i]) z[i] = r[i];
}

int orc_smoother_apply(const orc_problem* P, const double* phi, const double* K,
                       const double* p, const double* c, double dt, int kind,
                       double beta, int transpose, const double* r, double* z)
{
    orc_mg mg;
    int rc = mg_setup(&mg, P, phi, K, p, c, dt, transpose, kind, beta);
    if (rc == 0) {
        for (int i = 0; i < mg.n[0]; ++i) z[i] = 0.0;
        mg.omega = 1.0;   /* one undamped sweep from 0: z = P^{-1} r */
        mg_smooth(&mg, 0, r, z, mg.r[0]);
    }
    mg_free(&mg);
    return rc;
}

/* Solve J x = b (or J^T x = b) at state (p, c); (rowptr, col, val) hold the
 * full J (or J^T).  Dense LU for small systems, else BiCGStab + V-cycle. */
static int solve_at_state(const orc_problem* P, const double* phi,
                          const double* K, const double* p, const double* c,
                          double dt, int transpose, const int* rowptr,
                          const int* col, const double* val, const double* b,
                          double* x, const orc_newton_opts* o, int* iters)
{
    int n = 2 * orc_num_nodes(P);
    if (n <= o->dense_max) return orc_linear_solve(n, rowptr, col, val, b, x, o, iters);
    orc_mg mg;
    int rc = mg_setup(&mg, P, phi, K, p, c, dt, transpose, o->smoother, o->ilu_beta);
    if (rc == 0) {
        for (int i = 0; i < n; ++i) x[i] = 0.0;
        double rr;
        rc = bicgstab(n, rowptr, col, val, b, x, o->lin_rtol, o->lin_maxit,
                      mg_precond, &mg, iters, &rr);
    }
    mg_free(&mg);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Newton with line search (Section 2.3, Section 5.1)                       */
/* ------------------------------------------------------------------------ */

static double norm2_pair(int N, const double* a, const double* b)
{
    double s = 0.0;
    for (int n = 0; n < N; ++n) s += a[n] * a[n] + b[n] * b[n];
    return sqrt(s);
}

int orc_newton_step(const orc_problem* P, const double* phi, const double* K,
                    double* p, double* c, double dt,
                    const orc_newton_opts* o, orc_step_info* info)
{
    int N = orc_num_nodes(P);
    int n2 = 2 * N;
    size_t sz = sizeof(double) * (size_t)N;
    double *p_old = malloc(sz), *c_old = malloc(sz), *Rp = malloc(sz),
           *Rc = malloc(sz), *pt = malloc(sz), *ct = malloc(sz),
           *Rpt = malloc(sz), *Rct = malloc(sz);
    double* rhs = malloc(2 * sz);
    double* du = malloc(2 * sz);
    unsigned char* pm = malloc((size_t)N);
    unsigned char* cm = malloc((size_t)N);
    double* cv = malloc(sz);
    orc_dirichlet(P, pm, cm, cv);
    memcpy(p_old, p, sz);
    memcpy(c_old, c, sz);
    /* the new state starts from the old one with Dirichlet data imposed */
    for (int n = 0; n < N; ++n) {
        if (pm[n]) p[n] = 0.0;
        if (cm[n]) c[n] = cv[n];
    }
    int nnz = orc_jac_nnz(P);
    int* rowptr = malloc(sizeof(int) * ((size_t)n2 + 1));
    int* col = malloc(sizeof(int) * (size_t)nnz);
    double* val = malloc(sizeof(double) * (size_t)nnz);
    orc_jac_pattern(P, rowptr, col);

    orc_residual(P, phi, K, p, c, p_old, c_old, dt, 1, Rp, Rc);
    double rn = norm2_pair(N, Rp, Rc);
    orc_step_info inf = {1, 0, 0, 0, rn, rn};
    /* below this level ||R|| is rounding noise: 2 eps times the norm of the
     * per-row sums of the magnitudes of the summed terms */
    double rfloor = 2.0 * 2.220446049250313e-16 *
                    orc_residual_magnitude(P, phi, K, p, c, c_old, dt);
    if (rn <= rfloor) inf.status = 0;
    for (int it = 1; it <= o->maxit && rn > rfloor; ++it) {
        orc_jacobian(P, phi, K, p, c, dt, rowptr, col, val);
        for (int n = 0; n < N; ++n) {
            rhs[2 * n] = -Rp[n];
            rhs[2 * n + 1] = -Rc[n];
        }
        int li = 0;
        if (solve_at_state(P, phi, K, p, c, dt, 0, rowptr, col, val, rhs, du, o, &li) != 0) {
            /* keep going: Newton only needs a descent direction */
            inf.status = 2;
        }
        inf.lin_iters += li;
        double lambda = 1.0, rt = 0.0, rfloor_t = 0.0;
        for (int ls = 0; ls <= o->ls_max; ++ls) {
            for (int n = 0; n < N; ++n) {
                pt[n] = p[n] + lambda * du[2 * n];
                ct[n] = c[n] + lambda * du[2 * n + 1];
            }
            orc_residual(P, phi, K, pt, ct, p_old, c_old, dt, 1, Rpt, Rct);
            rt = norm2_pair(N, Rpt, Rct);
            rfloor_t = 2.0 * 2.220446049250313e-16 *
                       orc_residual_magnitude(P, phi, K, pt, ct, c_old, dt);
            if (rt < (1.0 - 1e-4 * lambda) * rn || rt <= rfloor_t || ls == o->ls_max) break;
            lambda *= 0.5;
            inf.ls_cuts++;
        }
        double dpmax = 0.0, dcmax = 0.0;
        for (int n = 0; n < N; ++n) {
            double a = fabs(pt[n] - p[n]), b = fabs(ct[n] - c[n]);
            if (a > dpmax) dpmax = a;
            if (b > dcmax) dcmax = b;
        }
        memcpy(p, pt, sz);
        memcpy(c, ct, sz);
        memcpy(Rp, Rpt, sz);
        memcpy(Rc, Rct, sz);
        rn = rt;
        rfloor = rfloor_t;
        inf.newton_iters = it;
        if ((lambda == 1.0 && dcmax <= o->tol_c && dpmax <= o->tol_p) || rn <= rfloor) {
            inf.status = 0; /* a failed inner solve does not matter once R is solved */
            break;
        }
    }
    inf.res = rn;
    if (info) *info = inf;
    free(p_old); free(c_old); free(Rp); free(Rc); free(pt); free(ct);
    free(Rpt); free(Rct); free(rhs); free(du); free(pm); free(cm); free(cv);
    free(rowptr); free(col); free(val);
    return inf.status;
}

/* ------------------------------------------------------------------------ */
/* statistics (Section 3: eqs. pdestat, numer_var; exceedance estimate)     */
/* ------------------------------------------------------------------------ */

void orc_moments(int S, int N, const double* c, const double* w,
                 double threshold, double* mean, double* var, double* pexc)
{
    for (int n = 0; n < N; ++n) {
        double m = 0.0;
        for (int s = 0; s < S; ++s)
            m += (w ? w[s] : 1.0 / S) * c[(size_t)s * N + n];
        double v = 0.0, pe = 0.0;
        for (int s = 0; s < S; ++s) {
            double ws = w ? w[s] : 1.0 / S;
            double dv = m - c[(size_t)s * N + n];
            v += ws * dv * dv;
            if (c[(size_t)s * N + n] > threshold) pe += ws;
        }
        mean[n] = m;
        var[n] = v;
        pexc[n] = pe;
    }
}

/* ------------------------------------------------------------------------ */
/* porosity / permeability realisations (Section 2.2)                       */
/* ------------------------------------------------------------------------ */

static double kozeny_carman(double phi, double K_mean)
{
    double ref = (0.1 * 0.1 * 0.1) / (0.9 * 0.9);
    return K_mean * (phi * phi * phi / ((1.0 - phi) * (1.0 - phi))) / ref;
}

void orc_fields_sobol(const orc_problem* P, const double* xi, double K_mean,
                      double* phi, double* K)
{
    const double pi = 3.14159265358979323846;
    double hx = P->Lx / P->nx, hy = P->Ly / P->ny, hz = P->Lz / P->nz;
    for (int k = 0; k < P->nz; ++k)
        for (int j = 0; j < P->ny; ++j)
            for (int i = 0; i < P->nx; ++i) {
                int e = i + P->nx * (j + P->ny * k);
                double x = (i + 0.5) * hx, y = (j + 0.5) * hy,
                       z = (k + 0.5) * hz;
                double f = xi[0] * cos(pi * x / P->Lx) +
                           xi[1] * cos(pi * y / P->Ly) +
                           xi[2] * sin(2.0 * pi * z / P->Lz);
                phi[e] = 0.1 * (1.0 + 0.3 * f / 3.0);
                K[e] = kozeny_carman(phi[e], K_mean);
            }
}

void orc_fields_lognormal(const orc_problem* P, const double* Z,
                          double K_mean, double* phi, double* K)
{
    int C = orc_num_cells(P);
    for (int e = 0; e < C; ++e) {
        double v = 0.1 * exp(0.2 * Z[e]);
        if (v < 0.05) v = 0.05;
        if (v > 0.2) v = 0.2;
        phi[e] = v;
        K[e] = kozeny_carman(v, K_mean);
    }
}

void orc_fields_paper3rv(const orc_problem* P, const double* xi,
                         double K_mean, double* phi, double* K)
{
    const double pi = 3.14159265358979323846;
    double hx = P->Lx / P->nx, hy = P->Ly / P->ny, hz = P->Lz / P->nz;
    for (int k = 0; k < P->nz; ++k)
        for (int j = 0; j < P->ny; ++j)
            for (int i = 0; i < P->nx; ++i) {
                int e = i + P->nx * (j + P->ny * k);
                double sx = sin(pi * (i + 0.5) * hx / P->Lx);
                double sy = sin(pi * (j + 0.5) * hy / P->Ly);
                double sz = sin(pi * (k + 0.5) * hz / P->Lz);
                phi[e] = 0.1 + 0.01 * (xi[0] * sx + xi[1] * sy + xi[2] * sz +
                                       xi[0] * sx * sy + xi[1] * sx * sz);
                K[e] = kozeny_carman(phi[e], K_mean);
            }
}

/* ------------------------------------------------------------------------ */
/* plume functional and discrete adjoint                                    */
/* ------------------------------------------------------------------------ */

static int cell_is_low(const orc_problem* P, int k)
{
    return (k + 0.5) * (P->Lz / P->nz) < 0.5 * P->Lz;
}

double orc_objective(const orc_problem* P, const double* phi, const double* c)
{
    double vscv = (P->Lx / P->nx) * (P->Ly / P->ny) * (P->Lz / P->nz) / 8.0;
    double J = 0.0;
    for (int k = 0; k < P->nz; ++k) {
        if (!cell_is_low(P, k)) continue;
        for (int j = 0; j < P->ny; ++j)
            for (int i = 0; i < P->nx; ++i) {
                int e = i + P->nx * (j + P->ny * k);
                int nodes[8];
                cell_corners(P, i, j, k, nodes);
                for (int L = 0; L < 8; ++L) {
                    double cc = c[nodes[L]];
                    J += phi[e] * vscv * rho_of(P, cc) * cc;
                }
            }
    }
    return J;
}

/* Lagrangian L = J(u_N) - sum_n lambda_n^T R_n(u_n, u_{n-1}; theta).
 * Stationarity in u_N:  J_N^T lambda_N = dJ/du_N.
 * Stationarity in u_n:  J_n^T lambda_n = -(dR_{n+1}/du_n)^T lambda_{n+1}.
 * Gradient:             dJ/dtheta = dJ/dtheta|_direct
 *                                   - sum_n lambda_n^T dR_n/dtheta. */
int orc_adjoint_gradient(const orc_problem* P, const double* phi,
                         const double* K, const double* p0, const double* c0,
                         double dt, int n_steps, const orc_newton_opts* o,
                         double* J_out, double* dJ_dphi, double* dJ_dK)
{
    int N = orc_num_nodes(P), C = orc_num_cells(P), n2 = 2 * N;
    size_t sz = sizeof(double) * (size_t)N;
    double drho = P->rho1 - P->rho0;
    double vscv = (P->Lx / P->nx) * (P->Ly / P->ny) * (P->Lz / P->nz) / 8.0;
    double* ps = malloc(sz * (size_t)(n_steps + 1));
    double* cs = malloc(sz * (size_t)(n_steps + 1));
    memcpy(ps, p0, sz);
    memcpy(cs, c0, sz);
    int rc = 0;
    for (int n = 1; n <= n_steps; ++n) {
        memcpy(ps + (size_t)n * N, ps + (size_t)(n - 1) * N, sz);
        memcpy(cs + (size_t)n * N, cs + (size_t)(n - 1) * N, sz);
        orc_step_info inf;
        if (orc_newton_step(P, phi, K, ps + (size_t)n * N, cs + (size_t)n * N,
                            dt, o, &inf) != 0)
            rc = 1;
    }
    const double* cN = cs + (size_t)n_steps * N;
    *J_out = orc_objective(P, phi, cN);

    unsigned char* pm = malloc((size_t)N);
    unsigned char* cm = malloc((size_t)N);
    orc_dirichlet(P, pm, cm, NULL);
    int nnz = orc_jac_nnz(P);
    int* rowptr = malloc(sizeof(int) * ((size_t)n2 + 1));
    int* col = malloc(sizeof(int) * (size_t)nnz);
    double* val = malloc(sizeof(double) * (size_t)nnz);
    int* trowptr = malloc(sizeof(int) * ((size_t)n2 + 1));
    int* tcol = malloc(sizeof(int) * (size_t)nnz);
    double* tval = malloc(sizeof(double) * (size_t)nnz);
    orc_jac_pattern(P, rowptr, col);
    double* rhs = malloc(2 * sz);
    double* lam = malloc(2 * sz);

    /* direct part of dJ/dphi, and dJ/du_N */
    for (int e = 0; e < C; ++e) {
        dJ_dphi[e] = 0.0;
        dJ_dK[e] = 0.0;
    }
    memset(rhs, 0, 2 * sz);
    for (int k = 0; k < P->nz; ++k) {
        if (!cell_is_low(P, k)) continue;
        for (int j = 0; j < P->ny; ++j)
            for (int i = 0; i < P->nx; ++i) {
                int e = i + P->nx * (j + P->ny * k);
                int nodes[8];
                cell_corners(P, i, j, k, nodes);
                for (int L = 0; L < 8; ++L) {
                    double cc = cN[nodes[L]];
                    dJ_dphi[e] += vscv * rho_of(P, cc) * cc;
                    rhs[2 * nodes[L] + 1] +=
                        phi[e] * vscv * (rho_of(P, cc) + drho * cc);
                }
            }
    }

    scvf faces[12];
    int nf = 0;
    for (int d = 0; d < 3; ++d)
        for (int s = 0; s < 2; ++s)
            for (int t = 0; t < 2; ++t) make_scvf(P, d, s, t, &faces[nf++]);

    for (int n = n_steps; n >= 1; --n) {
        const double* pn = ps + (size_t)n * N;
        const double* cn = cs + (size_t)n * N;
        const double* co = cs + (size_t)(n - 1) * N;
        /* J_n^T lambda_n = rhs */
        orc_jacobian(P, phi, K, pn, cn, dt, rowptr, col, val);
        orc_csr_transpose(n2, rowptr, col, val, trowptr, tcol, tval);
        int li;
        if (solve_at_state(P, phi, K, pn, cn, dt, 1, trowptr, tcol, tval, rhs, lam, o, &li) != 0)
            rc = 1;
        /* gradient contributions -lambda_n^T dR_n/dtheta (non-Dirichlet
         * rows only: Dirichlet rows do not depend on theta) */
        for (int k = 0; k < P->nz; ++k)
            for (int j = 0; j < P->ny; ++j)
                for (int i = 0; i < P->nx; ++i) {
                    int e = i + P->nx * (j + P->ny * k);
                    int nodes[8];
                    cell_corners(P, i, j, k, nodes);
                    double pl[8], cl[8];
                    for (int L = 0; L < 8; ++L) {
                        pl[L] = pn[nodes[L]];
                        cl[L] = cn[nodes[L]];
                    }
                    double gphi = 0.0, gK = 0.0;
                    for (int L = 0; L < 8; ++L) {
                        int nd = nodes[L];
                        double rn = rho_of(P, cn[nd]), ro = rho_of(P, co[nd]);
                        if (!pm[nd]) gphi += lam[2 * nd] * vscv * (rn - ro) / dt;
                        if (!cm[nd])
                            gphi += lam[2 * nd + 1] * vscv *
                                    (rn * cn[nd] - ro * co[nd]) / dt;
                    }
                    for (int q = 0; q < 12; ++q) {
                        face_flux ff;
                        eval_face(P, &faces[q], phi[e], K[e], pl, cl, &ff);
                        int a = nodes[faces[q].La], b = nodes[faces[q].Lb];
                        double dF_dphi =
                            -ff.rho_ip * P->Dm * ff.gradc * faces[q].A;
                        double dm_dK = ff.m / K[e];
                        double dF_dK = ff.cup * dm_dK;
                        if (!cm[a]) gphi += lam[2 * a + 1] * dF_dphi;
                        if (!cm[b]) gphi -= lam[2 * b + 1] * dF_dphi;
                        if (!pm[a]) gK += lam[2 * a] * dm_dK;
                        if (!pm[b]) gK -= lam[2 * b] * dm_dK;
                        if (!cm[a]) gK += lam[2 * a + 1] * dF_dK;
                        if (!cm[b]) gK -= lam[2 * b + 1] * dF_dK;
                    }
                    dJ_dphi[e] -= gphi;
                    dJ_dK[e] -= gK;
                }
        /* rhs for step n-1: -(dR_n/du_{n-1})^T lambda_n; R_n depends on
         * u_{n-1} only through the old storage, -S(c_{n-1})/dt */
        if (n > 1) {
            memset(rhs, 0, 2 * sz);
            for (int k = 0; k < P->nz; ++k)
                for (int j = 0; j < P->ny; ++j)
                    for (int i = 0; i < P->nx; ++i) {
                        int e = i + P->nx * (j + P->ny * k);
                        int nodes[8];
                        cell_corners(P, i, j, k, nodes);
                        for (int L = 0; L < 8; ++L) {
                            int nd = nodes[L];
                            double dSp = phi[e] * vscv * drho / dt;
                            double dSc = phi[e] * vscv *
                                         (rho_of(P, co[nd]) + drho * co[nd]) /
                                         dt;
                            if (!pm[nd]) rhs[2 * nd + 1] += dSp * lam[2 * nd];
                            if (!cm[nd])
                                rhs[2 * nd + 1] += dSc * lam[2 * nd + 1];
                        }
                    }
        }
    }
    free(ps); free(cs); free(pm); free(cm); free(rowptr); free(col); free(val);
    free(trowptr); free(tcol); free(tval); free(rhs); free(lam);
    return rc;
}
