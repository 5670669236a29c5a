// assembly.cu -- FV residual and Jacobian of the implicit Elder step and the
// per-level pieces of the multigrid hierarchy.
//
// Box method (Section 2.3): each hexahedron is split into 8 sub-control
// volumes (one per corner, |scv| = hx*hy*hz/8) and 12 sub-control-volume
// faces (one per edge).  The face of an edge along direction d lies in the
// edge's mid-plane; its integration point sits at 1/2 along d and at 1/4 or
// 3/4 across, on the edge's side, and its area is a quarter of the cell's
// cross-section.  At that point the trilinear interpolant gives
//   grad p . e_d = sum_edges w (p_B - p_A)/h_d,   w = (9,3,3,1)/16,
//   c_ip = sum_edges w (c_A + c_B)/2,
// and the fluxes (eqs. e_cont_eq, e_tran_eq, e_Darcy_vel, g = (0,0,-g)):
//   m = rho(c_ip) q.n A,  q.n = -(K/mu)(grad p . e_d + [d=z] g rho(c_ip)),
//   F = c_up m - rho(c_ip) phi Dm (grad c . e_d) A,  c_up = m>=0 ? c_A : c_B.
// Storage is lumped: sum_{e ni i} phi_e |scv| (rho(c_i)(c_i) - old)/dt.
//
// Every node kernel gathers the contributions of the up to 8 cells around
// its node (one thread per node, no atomics, deterministic).
#include "kernels.h"

namespace elder {

__device__ __forceinline__ bool sample_on(const int* mask, int stride, int s)
{
    return mask == nullptr || mask[(size_t)s * stride] != 0;
}

// Local corner L = lx + 2 ly + 4 lz of the edge of direction D with
// transverse local position (u, v), at end 0 (A) or 1 (B).
__host__ __device__ constexpr int corner_of(int D, int u, int v, int end)
{
    return D == 0 ? (end + 2 * u + 4 * v)
                  : (D == 1 ? (u + 2 * end + 4 * v) : (u + 2 * v + 4 * end));
}

// ---------------------------------------------------------------------------
// residual (FP64)
// ---------------------------------------------------------------------------

template <int D, int S_, int T_>
__device__ __forceinline__ void flux_face(const double (&p8)[8],
                                          const double (&c8)[8], double phi_e,
                                          double kmu, const Phys& ph,
                                          double invh, double area, double& m,
                                          double& F, double& mmag, double& Fmag)
{
    double gp = 0.0, gc = 0.0, ci = 0.0;
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 2; ++v) {
            const double w = (u == S_ ? 0.75 : 0.25) * (v == T_ ? 0.75 : 0.25);
            const int A = corner_of(D, u, v, 0), B = corner_of(D, u, v, 1);
            gp = fma(w, p8[B] - p8[A], gp);
            gc = fma(w, c8[B] - c8[A], gc);
            ci = fma(w, c8[A] + c8[B], ci);
        }
    gp *= invh;
    gc *= invh;
    ci *= 0.5;
    const double rho = fma(ph.drho, ci, ph.rho0);
    const double G = (D == 2) ? fma(ph.g, rho, gp) : gp;
    m = rho * (-kmu * G) * area;
    const double cup =
        (m >= 0.0) ? c8[corner_of(D, S_, T_, 0)] : c8[corner_of(D, S_, T_, 1)];
    const double dif = rho * phi_e * ph.Dm * area;
    F = cup * m - dif * gc;
    // rounding scale: the Darcy flux cancels grad p against rho g
    mmag = rho * kmu * area * (fabs(gp) + (D == 2 ? ph.g * rho : 0.0));
    Fmag = fabs(cup) * mmag + dif * fabs(gc);
}

struct CellGeom {
    double ih[3];    // 1/h_d
    double area[3];  // face areas of the three directions
};

template <int OX, int OY, int OZ>
__device__ __forceinline__ void residual_cell(
    const Grid& G, const Phys& ph, const CellGeom& cg, int i, int j, int k,
    const double* __restrict__ phi, const double* __restrict__ K,
    const double* __restrict__ p, const double* __restrict__ c, double& Rp,
    double& Rc, double& phis, double& Ap, double& Ac)
{
    const int ci = i + OX, cj = j + OY, ck = k + OZ;
    if (ci < 0 || ci >= G.nx || cj < 0 || cj >= G.ny || ck < 0 || ck >= G.nz)
        return;
    const int e = ci + G.nx * (cj + G.ny * ck);
    const double phi_e = __ldg(phi + e);
    const double kmu = __ldg(K + e) / ph.mu;
    phis += phi_e;
    const int sy = G.nx + 1, sz = (G.nx + 1) * (G.ny + 1);
    const int base = ci + sy * cj + sz * ck;
    double p8[8], c8[8];
#pragma unroll
    for (int L = 0; L < 8; ++L) {
        const int off = (L & 1) + ((L >> 1) & 1) * sy + (L >> 2) * sz;
        p8[L] = __ldg(p + base + off);
        c8[L] = __ldg(c + base + off);
    }
    constexpr int lx = -OX, ly = -OY, lz = -OZ;  // this node's local corner
    double m, F, mm, Fm;
    flux_face<0, ly, lz>(p8, c8, phi_e, kmu, ph, cg.ih[0], cg.area[0], m, F, mm, Fm);
    if (lx == 0) { Rp += m; Rc += F; } else { Rp -= m; Rc -= F; }
    Ap += mm;
    Ac += Fm;
    flux_face<1, lx, lz>(p8, c8, phi_e, kmu, ph, cg.ih[1], cg.area[1], m, F, mm, Fm);
    if (ly == 0) { Rp += m; Rc += F; } else { Rp -= m; Rc -= F; }
    Ap += mm;
    Ac += Fm;
    flux_face<2, lx, ly>(p8, c8, phi_e, kmu, ph, cg.ih[2], cg.area[2], m, F, mm, Fm);
    if (lz == 0) { Rp += m; Rc += F; } else { Rp -= m; Rc -= F; }
    Ap += mm;
    Ac += Fm;
}

__host__ __device__ inline CellGeom make_geom(const Grid& G)
{
    CellGeom cg;
    cg.ih[0] = 1.0 / G.hx;
    cg.ih[1] = 1.0 / G.hy;
    cg.ih[2] = 1.0 / G.hz;
    cg.area[0] = 0.25 * G.hy * G.hz;
    cg.area[1] = 0.25 * G.hx * G.hz;
    cg.area[2] = 0.25 * G.hx * G.hy;
    return cg;
}

// ---------------------------------------------------------------------------
// Cell-based residual: each quarter-face flux computed once.
//
// k_cell_flux: one thread per cell computes the 12 quarter faces of its
// sub-control-volume boundary (one per cell edge): the 4 edge differences of
// p per direction, and for c one cube transform of the cell's 8 values that
// holds every direction's weighted edge differences and sums, are formed once
// and shared by the quarter faces, which only differ in their Q1 weights
// (9,3,3,1)/16.  Output: [S][12][C] records (mass flux m and salt
// flux F from the edge's lower end A to its upper end B, and the magnitudes
// of their terms, the round-off scale).
// k_cell_residual: node n sums, for each direction, the 4 quarter faces of
// its forward edge and of its backward edge (always in the same order, from
// the edge's lower node, so both ends of an edge use the same value and the
// balance telescopes exactly), then adds storage and Dirichlet rows.
// Quarter face q = 4 D + 2 u + v of a cell belongs to its direction-D edge at
// transverse local position (u, v) (see corner_of).
// ---------------------------------------------------------------------------

// Constants of the cell-based residual, formed on the host.  The Q1 weights
// (9,3,3,1)/16 of a quarter face are applied as two passes of (3,1) sums
// (kron31: 16x the weights, additions only), and 1/(16 h_d) is folded into
// the per-direction coefficients:
//   m = -(rho K kA_d) (g16_d + [d=z] g16h rho),  F = c_up m - rho phi dA_d gc16_d,
//   rho = rho0 + drho32 sc16,
// with g16, gc16, sc16 the 16x-weighted sums of the edge differences of p and
// c and of the edge sums of c.  For c the three passes of (3,1) sums over the
// cell's 2x2x2 values, Z = (W x W x W) c with W = [[3,1],[1,3]], give every
// direction's sums at once: across a direction-d edge pair (A, B) the (3,1)
// sum along d turns into Z_B - Z_A = 2 gc16 and Z_B + Z_A = 4 sc16, and the
// powers of two sit in the constants (dA2 = dA / 2, drho128 = drho32 / 4,
// exact scalings).  p keeps its per-direction differences, which are exact
// (Sterbenz) for neighbouring values of the hydrostatic pressure.
struct FluxConst {
    double kA[3];    // A_d / (16 h_d mu)
    double dA2[3];   // Dm A_d / (32 h_d)
    double g16h;     // 16 h_z g
    double drho128;  // drho / 128 (4 sc16 = 128 c_ip)
    // FP32 copies for the round-off scale (a magnitude)
    float kAf[3], dAf[3], g16hf, drho32f, rho0f;
};

static FluxConst make_flux_const(const Grid& G, const Phys& ph)
{
    const CellGeom cg = make_geom(G);
    const double h[3] = {G.hx, G.hy, G.hz};
    FluxConst f;
    for (int d = 0; d < 3; ++d) {
        f.kA[d] = cg.area[d] / (16.0 * h[d] * ph.mu);
        const double dA = ph.Dm * cg.area[d] / (16.0 * h[d]);
        f.dA2[d] = 0.5 * dA;
        f.kAf[d] = (float)f.kA[d];
        f.dAf[d] = (float)dA;
    }
    f.g16h = 16.0 * G.hz * ph.g;
    f.drho128 = ph.drho / 128.0;
    f.g16hf = (float)f.g16h;
    f.drho32f = (float)(ph.drho / 32.0);
    f.rho0f = (float)ph.rho0;
    return f;
}

// y[S][T] = sum_{u,v} (u == S ? 3 : 1) (v == T ? 3 : 1) x[u][v]
template <class R>
__device__ __forceinline__ void kron31(const R (&x)[2][2], R (&y)[2][2])
{
    R t[2][2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const R a = x[u][0] + x[u][1];
        t[u][0] = R(2) * x[u][0] + a;
        t[u][1] = R(2) * x[u][1] + a;
    }
#pragma unroll
    for (int T_ = 0; T_ < 2; ++T_) {
        const R a = t[0][T_] + t[1][T_];
        y[0][T_] = R(2) * t[0][T_] + a;
        y[1][T_] = R(2) * t[1][T_] + a;
    }
}

template <class R, int D>
__device__ __forceinline__ void dir_sums(const R (&p8)[8], const R (&c8)[8], R (&gp)[2][2],
                                         R (&gc)[2][2], R (&sc)[2][2])
{
    R dp[2][2], dc[2][2], cs[2][2];
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 2; ++v) {
            const int A = corner_of(D, u, v, 0), B = corner_of(D, u, v, 1);
            dp[u][v] = p8[B] - p8[A];
            dc[u][v] = c8[B] - c8[A];
            cs[u][v] = c8[A] + c8[B];
        }
    kron31(dp, gp);
    kron31(dc, gc);
    kron31(cs, sc);
}

// the 16x-weighted sums of the direction-D edge differences of p
template <int D>
__device__ __forceinline__ void dir_grad(const double (&p8)[8], double (&gp)[2][2])
{
    double dp[2][2];
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 2; ++v)
            dp[u][v] = p8[corner_of(D, u, v, 1)] - p8[corner_of(D, u, v, 0)];
    kron31(dp, gp);
}

// Z = (W x W x W) x over the cell's corners L = x + 2 y + 4 z: a (3,1) pass
// along each axis, (a, b) -> (2 a + (a + b), 2 b + (a + b))
__device__ __forceinline__ void cube31(const double (&x)[8], double (&Z)[8])
{
#pragma unroll
    for (int L = 0; L < 8; ++L) Z[L] = x[L];
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int L = 0; L < 8; ++L)
            if (!((L >> d) & 1)) {
                const int H = L | (1 << d);
                const double a = Z[L] + Z[H];
                Z[L] = fma(2.0, Z[L], a);
                Z[H] = fma(2.0, Z[H], a);
            }
}

// Mass flux m and salt flux F of the direction-D quarter face at transverse
// position (S_, T_), from its edge's lower corner A = corner_of(D, S_, T_, 0)
// to B; upA: c is upwinded from A.  gp: the direction's 16x-weighted p
// differences; Zc: the cell's c cube transform; kmuA = K kA_d, dA2 =
// phi dA2_d.
template <int D>
__device__ __forceinline__ void quarter_face(int S_, int T_, const double (&gp)[2][2],
                                             const double (&c8)[8], const double (&Zc)[8],
                                             const Phys& ph, const FluxConst& fc, double kmuA,
                                             double dA2, double& m, double& F, bool& upA)
{
    const int A = corner_of(D, S_, T_, 0), B = corner_of(D, S_, T_, 1);
    const double zA = Zc[A], zB = Zc[B];
    // rho = rho0 + drho32 sc16 with 4 sc16 = zA + zB; dA gc16 = dA2 (zB - zA)
    const double rho = fma(fc.drho128, zA + zB, ph.rho0);
    const double G = (D == 2) ? fma(fc.g16h, rho, gp[S_][T_]) : gp[S_][T_];
    m = -(rho * kmuA) * G;
    // upwind end from the sign bit (an integer test)
    upA = __double2hiint(m) >= 0;
    const double cup = upA ? c8[A] : c8[B];
    F = fma(cup, m, -(rho * dA2) * (zB - zA));
}

template <int D>
__device__ __forceinline__ void cell_dir_faces(const double (&p8)[8], const double (&c8)[8],
                                               const double (&Zc)[8], const float (&pf)[8],
                                               const float (&cf)[8], const Phys& ph,
                                               const FluxConst& fc, double Ke, double phie,
                                               float Kf, float phif, QF* __restrict__ out,
                                               size_t qs)
{
    double gp[2][2];
    dir_grad<D>(p8, gp);
    float gpf[2][2], gcf[2][2], scf[2][2];
    dir_sums<float, D>(pf, cf, gpf, gcf, scf);
    const double kmuA = Ke * fc.kA[D], dA2 = phie * fc.dA2[D];
    const float kmuAf = Kf * fc.kAf[D], dAf = phif * fc.dAf[D];
#pragma unroll
    for (int S_ = 0; S_ < 2; ++S_)
#pragma unroll
        for (int T_ = 0; T_ < 2; ++T_) {
            double m, F;
            bool upA;
            quarter_face<D>(S_, T_, gp, c8, Zc, ph, fc, kmuA, dA2, m, F, upA);
            // rounding scale in FP32: the Darcy flux cancels grad p against rho g
            const float rhof = fmaf(fc.drho32f, scf[S_][T_], fc.rho0f);
            const float mm = rhof * kmuAf *
                             (fabsf(gpf[S_][T_]) + (D == 2 ? fc.g16hf * rhof : 0.0f));
            const float cupf = upA ? cf[corner_of(D, S_, T_, 0)] : cf[corner_of(D, S_, T_, 1)];
            const float Fm = fmaf(fabsf(cupf), mm, rhof * dAf * fabsf(gcf[S_][T_]));
            out[(size_t)(4 * D + 2 * S_ + T_) * qs] = QF{m, F, mm, Fm};
        }
}

__global__ void __launch_bounds__(kBS)
    k_cell_flux(Grid G, Phys ph, FluxConst fc, const double* __restrict__ phi,
                const double* __restrict__ K, const double* __restrict__ p,
                const double* __restrict__ c, QF* __restrict__ qf, const int* mask, int mstride)
{
    const int s = blockIdx.y;
    if (!sample_on(mask, mstride, s)) return;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= G.C) return;
    const size_t on = (size_t)s * G.N, oc = (size_t)s * G.C;
    const int ci = e % G.nx, cj = (e / G.nx) % G.ny, ck = e / (G.nx * G.ny);
    const int sy = G.nx + 1, sz = (G.nx + 1) * (G.ny + 1);
    const int base = ci + sy * cj + sz * ck;
    double p8[8], c8[8];
    float pf[8], cf[8];
#pragma unroll
    for (int L = 0; L < 8; ++L) {
        const int off = (L & 1) + ((L >> 1) & 1) * sy + (L >> 2) * sz;
        p8[L] = __ldg(p + on + base + off);
        c8[L] = __ldg(c + on + base + off);
        pf[L] = d2f_trunc(p8[L]);
        cf[L] = d2f_trunc(c8[L]);
    }
    const double phie = __ldg(phi + oc + e);
    const double Ke = __ldg(K + oc + e);
    const float phif = d2f_trunc(phie), Kf = d2f_trunc(Ke);
    QF* out = qf + (size_t)s * 12 * G.C + e;
    const size_t qs = (size_t)G.C;
    double Zc[8];
    cube31(c8, Zc);
    cell_dir_faces<0>(p8, c8, Zc, pf, cf, ph, fc, Ke, phie, Kf, phif, out, qs);
    cell_dir_faces<1>(p8, c8, Zc, pf, cf, ph, fc, Ke, phie, Kf, phif, out, qs);
    cell_dir_faces<2>(p8, c8, Zc, pf, cf, ph, fc, Ke, phie, Kf, phif, out, qs);
}

// Sum of the up to 4 quarter faces of the direction-D edge whose lower node
// is (i, j, k) (the edge must exist); fixed order, missing cells read as 0.
template <int D>
__device__ __forceinline__ void edge_sum(const Grid& G, const QF* __restrict__ qf, int i, int j,
                                         int k, double& m, double& F, float& mm, float& Fm)
{
    QF f[4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            int ci, cj, ck;
            if (D == 0) { ci = i; cj = j - b; ck = k - a; }
            else if (D == 1) { ci = i - b; cj = j; ck = k - a; }
            else { ci = i - b; cj = j - a; ck = k; }
            const bool ok = ci >= 0 && ci < G.nx && cj >= 0 && cj < G.ny && ck >= 0 && ck < G.nz;
            f[2 * a + b] = ok ? qf[(size_t)(4 * D + 2 * b + a) * G.C + ci + G.nx * (cj + G.ny * ck)]
                              : QF{0.0, 0.0, 0.0f, 0.0f};
        }
    m = ((f[0].m + f[1].m) + f[2].m) + f[3].m;
    F = ((f[0].F + f[1].F) + f[2].F) + f[3].F;
    mm = (f[0].mm + f[1].mm) + (f[2].mm + f[3].mm);
    Fm = (f[0].Fm + f[1].Fm) + (f[2].Fm + f[3].Fm);
}

// vsc = |scv| / dt = hx hy hz / (8 dt); the rounding scale (Ap, Ac and the
// per-block partials of its square) is carried in FP32.
__global__ void __launch_bounds__(kBS)
    k_cell_residual(Grid G, Phys ph, double vsc, const uint8_t* __restrict__ bc,
                    const double* __restrict__ cval, const double* __restrict__ phi,
                    const double* __restrict__ p, const double* __restrict__ c,
                    const double* __restrict__ c_old, const QF* __restrict__ qf,
                    V2<double>* __restrict__ R, double* __restrict__ partial,
                    double* __restrict__ act, const int* mask, int mstride, float drhof,
                    float rho0f)
{
    __shared__ double red[32];
    const int s = blockIdx.y;
    if (!sample_on(mask, mstride, s)) return;
    const size_t on = (size_t)s * G.N, oc = (size_t)s * G.C;
    phi += oc; p += on; c += on; c_old += on; R += on;
    qf += (size_t)s * 12 * G.C;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    double sq = 0.0;
    float aq = 0.0f;
    if (n < G.N) {
        int i, j, k;
        node_ijk(G, n, i, j, k);
        double Rp = 0.0, Rc = 0.0;
        float Ap = 0.0f, Ac = 0.0f;
        double m, F;
        float mm, Fm;
        if (i < G.nx) { edge_sum<0>(G, qf, i, j, k, m, F, mm, Fm); Rp = m; Rc = F; Ap = mm; Ac = Fm; }
        if (i > 0) { edge_sum<0>(G, qf, i - 1, j, k, m, F, mm, Fm); Rp -= m; Rc -= F; Ap += mm; Ac += Fm; }
        if (j < G.ny) { edge_sum<1>(G, qf, i, j, k, m, F, mm, Fm); Rp += m; Rc += F; Ap += mm; Ac += Fm; }
        if (j > 0) { edge_sum<1>(G, qf, i, j - 1, k, m, F, mm, Fm); Rp -= m; Rc -= F; Ap += mm; Ac += Fm; }
        if (k < G.nz) { edge_sum<2>(G, qf, i, j, k, m, F, mm, Fm); Rp += m; Rc += F; Ap += mm; Ac += Fm; }
        if (k > 0) { edge_sum<2>(G, qf, i, j, k - 1, m, F, mm, Fm); Rp -= m; Rc -= F; Ap += mm; Ac += Fm; }
        double phis = 0.0;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int ci = i - (q & 1), cj = j - ((q >> 1) & 1), ck = k - (q >> 2);
            if (ci < 0 || ci >= G.nx || cj < 0 || cj >= G.ny || ck < 0 || ck >= G.nz) continue;
            phis += __ldg(phi + ci + G.nx * (cj + G.ny * ck));
        }
        const double vdt = phis * vsc;
        const double cn = c[n], co = c_old[n];
        const double rn = fma(ph.drho, cn, ph.rho0), ro = fma(ph.drho, co, ph.rho0);
        Rp += vdt * (rn - ro);
        Rc += vdt * (rn * cn - ro * co);
        const float vdtf = d2f_trunc(vdt), cnf = d2f_trunc(cn), cof = d2f_trunc(co);
        const float rnf = fmaf(drhof, cnf, rho0f);
        const float rof = fmaf(drhof, cof, rho0f);
        Ap = fmaf(vdtf, fabsf(rnf) + fabsf(rof), Ap);
        Ac = fmaf(vdtf, fabsf(rnf * cnf) + fabsf(rof * cof), Ac);
        const uint8_t b = bc[n];
        if (b & BC_P) { Rp = p[n]; Ap = 0.0f; }
        if (b & BC_C) { Rc = cn - cval[n]; Ac = 0.0f; }
        R[n] = V2<double>{Rp, Rc};
        sq = Rp * Rp + Rc * Rc;
        aq = fmaf(Ap, Ap, Ac * Ac);
    }
    if (partial) {
        const double t = block_sum(sq, red);
        if (threadIdx.x == 0) partial[(size_t)s * gridDim.x + blockIdx.x] = t;
    }
    if (act) {
        const float t = block_sum(aq, reinterpret_cast<float*>(red));
        if (threadIdx.x == 0) act[(size_t)s * gridDim.x + blockIdx.x] = (double)t;
    }
}

void launch_residual(const Grid& G, const Phys& ph, const uint8_t* bc,
                     const double* cval, const double* phi, const double* K,
                     const double* p, const double* c, const double* p_old,
                     const double* c_old, V2<double>* R, double* partial,
                     double* act, const int* mask, int mstride, int S,
                     cudaStream_t st, QF* qf)
{
    (void)p_old;  // p has no time derivative
    count_launch(2);
    dim3 gc(nblocks(G.C), S);
    k_cell_flux<<<gc, kBS, 0, st>>>(G, ph, make_flux_const(G, ph), phi, K, p, c, qf, mask,
                                    mstride);
    dim3 grid(nblocks(G.N), S);
    const double vsc = G.hx * G.hy * G.hz / (8.0 * ph.dt);
    k_cell_residual<<<grid, kBS, 0, st>>>(G, ph, vsc, bc, cval, phi, p, c, c_old, qf, R,
                                          partial, act, mask, mstride, (float)ph.drho,
                                          (float)ph.rho0);
}

// ---------------------------------------------------------------------------
// Jacobian (T = double: FP64 path; T = float: FP32 copy for mixed precision)
// ---------------------------------------------------------------------------
//
// For one face (rows of this node, sign sig = +1 when the node is end A):
//   dm/dp_B = alpha w, dm/dp_A = -alpha w,   alpha = -rho (K/mu) A / h
//   dm/dc_X = beta w (both ends),           beta = (drho/2) A (q - [z] rho (K/mu) g)
//   dF/dp_X = c_up dm/dp_X
//   dF/dc_B = (c_up beta - gam - del) w + [B up] m
//   dF/dc_A = (c_up beta - gam + del) w + [A up] m
//       gam = (drho/2) phi Dm A (grad c . e_d),  del = rho phi Dm A / h.
// Pressures enter through p' = p - rho0 g (Lz - z) (same differences up to
// the constant rho0 g h_z on vertical edges), so that the FP32 copy keeps the
// Darcy driving force without cancelling against the hydrostatic part.

template <class T> struct PhysT {
    T rho0, drho, g, Dm;
};

// Cell geometry in the assembly's arithmetic type (converted on the host).
template <class T> struct GeomT {
    T ih[3], area[3];
};

template <class T, int D, int S_, int T_, int OX, int OY, int OZ>
__device__ __forceinline__ void jac_face(const T (&p8)[8], const T (&c8)[8],
                                         T phi_e, T kmu, const PhysT<T>& ph,
                                         T invh, T area, T (&acc)[27][4])
{
    constexpr int lnode = (D == 0) ? -OX : (D == 1 ? -OY : -OZ);
    const T sig = (lnode == 0) ? T(1) : T(-1);
    T gp = 0, gc = 0, ci = 0;
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 2; ++v) {
            const T w = T((u == S_ ? 0.75 : 0.25) * (v == T_ ? 0.75 : 0.25));
            const int A = corner_of(D, u, v, 0), B = corner_of(D, u, v, 1);
            gp += w * (p8[B] - p8[A]);
            gc += w * (c8[B] - c8[A]);
            ci += w * (c8[A] + c8[B]);
        }
    gp *= invh;
    gc *= invh;
    ci *= T(0.5);
    const T rho = ph.rho0 + ph.drho * ci;
    const T Gd = (D == 2) ? gp + ph.g * ph.drho * ci : gp;
    const T q = -kmu * Gd;
    const T m = rho * q * area;
    const T alpha = -rho * kmu * area * invh;
    const T beta = T(0.5) * ph.drho * area * (q - (D == 2 ? rho * kmu * ph.g : T(0)));
    constexpr int cA = corner_of(D, S_, T_, 0), cB = corner_of(D, S_, T_, 1);
    const bool upA = (m >= T(0));
    const T cup = upA ? c8[cA] : c8[cB];
    const T gam = T(0.5) * ph.drho * phi_e * ph.Dm * area * gc;
    const T del = rho * phi_e * ph.Dm * area * invh;
    const T sa = sig * alpha, sb = sig * beta, sca = sig * cup * alpha;
    const T scc = sig * (cup * beta - gam), sd = sig * del;
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 2; ++v) {
            const T w = T((u == S_ ? 0.75 : 0.25) * (v == T_ ? 0.75 : 0.25));
            constexpr int dummy = 0;
            (void)dummy;
            const int A = corner_of(D, u, v, 0), B = corner_of(D, u, v, 1);
            const int sA = slot27(OX + (A & 1), OY + ((A >> 1) & 1), OZ + (A >> 2));
            const int sB = slot27(OX + (B & 1), OY + ((B >> 1) & 1), OZ + (B >> 2));
            acc[sB][0] += w * sa;
            acc[sA][0] -= w * sa;
            acc[sB][1] += w * sb;
            acc[sA][1] += w * sb;
            acc[sB][2] += w * sca;
            acc[sA][2] -= w * sca;
            acc[sB][3] += w * (scc - sd);
            acc[sA][3] += w * (scc + sd);
        }
    constexpr int slA = slot27(OX + (cA & 1), OY + ((cA >> 1) & 1), OZ + (cA >> 2));
    constexpr int slB = slot27(OX + (cB & 1), OY + ((cB >> 1) & 1), OZ + (cB >> 2));
    acc[slA][3] += upA ? sig * m : T(0);
    acc[slB][3] += upA ? T(0) : sig * m;
}

template <class T, int OX, int OY, int OZ>
__device__ __forceinline__ void jac_cell(const Grid& G, const PhysT<T>& pt,
                                         const GeomT<T>& cg, int i, int j, int k,
                                         const V2<T>* __restrict__ cellT,
                                         const V2<T>* __restrict__ nodeT,
                                         T (&acc)[27][4], T& phis)
{
    const int ci = i + OX, cj = j + OY, ck = k + OZ;
    if (ci < 0 || ci >= G.nx || cj < 0 || cj >= G.ny || ck < 0 || ck >= G.nz)
        return;
    const int e = ci + G.nx * (cj + G.ny * ck);
    const V2<T> fk = cellT[e];  // (phi, K/mu)
    phis += fk.p;
    const int sy = G.nx + 1, sz = (G.nx + 1) * (G.ny + 1);
    const int base = ci + sy * cj + sz * ck;
    T p8[8], c8[8];
#pragma unroll
    for (int L = 0; L < 8; ++L) {
        const int off = (L & 1) + ((L >> 1) & 1) * sy + (L >> 2) * sz;
        const V2<T> u = nodeT[base + off];
        p8[L] = u.p;
        c8[L] = u.c;
    }
    constexpr int lx = -OX, ly = -OY, lz = -OZ;
    jac_face<T, 0, ly, lz, OX, OY, OZ>(p8, c8, fk.p, fk.c, pt, cg.ih[0], cg.area[0], acc);
    jac_face<T, 1, lx, lz, OX, OY, OZ>(p8, c8, fk.p, fk.c, pt, cg.ih[1], cg.area[1], acc);
    jac_face<T, 2, lx, ly, OX, OY, OZ>(p8, c8, fk.p, fk.c, pt, cg.ih[2], cg.area[2], acc);
}

// Inputs of the Jacobian in its arithmetic type T, converted once per level
// instead of once per use: nodeT = (p - rho0 g (Lz - z), c) per node and
// cellT = (phi, K/mu) per cell.  (On GB300 an FP64-to-FP32 conversion issues
// on the FP64 pipe; doing the 16 corner conversions of each of 8 cells per
// node kept that pipe saturated in the FP32 assembly.)
template <class T>
__global__ void k_jac_inputs(Grid G, Phys ph, const double* __restrict__ phi,
                             const double* __restrict__ K, const double* __restrict__ p,
                             const double* __restrict__ c, V2<T>* __restrict__ cellT,
                             V2<T>* __restrict__ nodeT, const int* mask, int mstride)
{
    const int s = blockIdx.y;
    if (!sample_on(mask, mstride, s)) return;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < G.N) {
        const size_t o = (size_t)s * G.N + q;
        int i, j, k;
        node_ijk(G, q, i, j, k);
        const double z = k * G.hz;
        nodeT[o] = V2<T>{T(fma(ph.rho0 * ph.g, z - G.Lz, p[o])), T(c[o])};
    }
    if (q < G.C) {
        const size_t o = (size_t)s * G.C + q;
        cellT[o] = V2<T>{T(phi[o]), T(K[o] / ph.mu)};
    }
}

// The node part of k_jac_inputs alone (a Newton iterate changes the state
// only; the cell coefficients are converted once per step).
template <class T>
__global__ void k_node_inputs(Grid G, double rho0g, const double* __restrict__ p,
                              const double* __restrict__ c, V2<T>* __restrict__ nodeT,
                              const int* mask, int mstride)
{
    const int s = blockIdx.y;
    if (!sample_on(mask, mstride, s)) return;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= G.N) return;
    const size_t o = (size_t)s * G.N + q;
    int i, j, k;
    node_ijk(G, q, i, j, k);
    const double z = k * G.hz;
    nodeT[o] = V2<T>{T(fma(rho0g, z - G.Lz, p[o])), T(c[o])};
}

// The cell part of k_jac_inputs alone: (phi, K / mu) in T.
template <class T>
__global__ void k_cell_inputs(int C, double mu, const double* __restrict__ phi,
                              const double* __restrict__ K, V2<T>* __restrict__ cellT)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= C) return;
    const size_t o = (size_t)blockIdx.y * C + q;
    cellT[o] = V2<T>{T(phi[o]), T(K[o] / mu)};
}

template <class T>
void launch_cell_inputs(const Grid& G, double mu, const double* phi, const double* K,
                        V2<T>* cellT, int S, cudaStream_t st)
{
    count_launch(1);
    k_cell_inputs<T><<<dim3(nblocks(G.C), S), kBS, 0, st>>>(G.C, mu, phi, K, cellT);
}
template void launch_cell_inputs<float>(const Grid&, double, const double*, const double*,
                                        V2<float>*, int, cudaStream_t);
template void launch_cell_inputs<double>(const Grid&, double, const double*, const double*,
                                         V2<double>*, int, cudaStream_t);

// Writes the row blocks as T (JT, the Krylov operator) and/or as the
// multigrid storage type M (JM), and the inverse of the interior diagonal
// block (Dinv, Dirichlet rows and columns replaced by the identity); any of
// the three outputs may be null.
template <class T, class M>
__global__ void __launch_bounds__(128)
    k_jacobian(Grid G, PhysT<T> pt, GeomT<T> cg, const uint8_t* __restrict__ bc,
               const V2<T>* __restrict__ cellT, const V2<T>* __restrict__ nodeT,
               B4<T>* __restrict__ JT, B4<M>* __restrict__ JM, B4<T>* __restrict__ Dinv,
               T vscale, const int* mask, int mstride)
{
    const int s = blockIdx.y;
    if (!sample_on(mask, mstride, s)) return;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= G.N) return;
    const size_t on = (size_t)s * G.N, oc = (size_t)s * G.C;
    cellT += oc; nodeT += on;
    int i, j, k;
    node_ijk(G, n, i, j, k);
    T acc[27][4];
#pragma unroll
    for (int q = 0; q < 27; ++q)
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[q][r] = T(0);
    T phis = T(0);
    const uint8_t b = bc[n];
    if (JT) JT += (size_t)s * 27 * G.N;
    if (JM) JM += (size_t)s * 27 * G.N;
    // Dirichlet rows are identity rows: zero a block's p row / c row (the
    // diagonal block gets its 1 after storage), then store it
    auto finish = [&](int q) {
        if (b & BC_P) { acc[q][0] = T(0); acc[q][1] = T(0); }
        if (b & BC_C) { acc[q][2] = T(0); acc[q][3] = T(0); }
        if (q == 13) {
            if (b & BC_P) acc[13][0] = T(1);
            if (b & BC_C) acc[13][3] = T(1);
        }
        if (JT) JT[(size_t)q * G.N + n] = B4<T>{acc[q][0], acc[q][1], acc[q][2], acc[q][3]};
        if (JM)
            JM[(size_t)q * G.N + n] =
                B4<M>{mg_store<M>(acc[q][0]), mg_store<M>(acc[q][1]), mg_store<M>(acc[q][2]),
                      mg_store<M>(acc[q][3])};
    };
    // the 4 cells below the node touch only the blocks of offsets dz = -1
    // and dz = 0, the 4 above only dz = 0 and dz = +1: the dz = -1 blocks
    // are complete (and stored) before the upper cells, so at most 18 of the
    // 27 blocks are live at a time
    jac_cell<T, -1, -1, -1>(G, pt, cg, i, j, k, cellT, nodeT, acc, phis);
    jac_cell<T, 0, -1, -1>(G, pt, cg, i, j, k, cellT, nodeT, acc, phis);
    jac_cell<T, -1, 0, -1>(G, pt, cg, i, j, k, cellT, nodeT, acc, phis);
    jac_cell<T, 0, 0, -1>(G, pt, cg, i, j, k, cellT, nodeT, acc, phis);
#pragma unroll
    for (int q = 0; q < 9; ++q) finish(q);
    jac_cell<T, -1, -1, 0>(G, pt, cg, i, j, k, cellT, nodeT, acc, phis);
    jac_cell<T, 0, -1, 0>(G, pt, cg, i, j, k, cellT, nodeT, acc, phis);
    jac_cell<T, -1, 0, 0>(G, pt, cg, i, j, k, cellT, nodeT, acc, phis);
    jac_cell<T, 0, 0, 0>(G, pt, cg, i, j, k, cellT, nodeT, acc, phis);
    // lumped storage: d/dc of rho(c) and rho(c) c
    const T vdt = phis * vscale;
    const T cn = nodeT[n].c;
    acc[13][1] += vdt * pt.drho;
    acc[13][3] += vdt * (pt.rho0 + T(2) * pt.drho * cn);
    // the diagonal block's Dirichlet-free entries for Dinv
    const T a0 = acc[13][0], b0 = acc[13][1], c0 = acc[13][2], e0 = acc[13][3];
#pragma unroll
    for (int q = 9; q < 27; ++q) finish(q);
    if (Dinv) {
        // in T: the FP32 entries' determinant is formed without FP64 work
        T a = a0, bb = b0, cc = c0, e = e0;
        if (b & BC_P) { a = T(1); bb = T(0); cc = T(0); }
        if (b & BC_C) { e = T(1); bb = T(0); cc = T(0); }
        const T id = T(1) / (a * e - bb * cc);
        Dinv[(size_t)s * G.N + n] = B4<T>{e * id, -bb * id, -cc * id, a * id};
    }
}

template <class T, class M>
void launch_jacobian(const Grid& G, const Phys& ph, const uint8_t* bc,
                     const double* phi, const double* K, const double* p,
                     const double* c, B4<T>* JT, B4<M>* JM, B4<T>* Dinv, V2<T>* cellT,
                     V2<T>* nodeT, const int* mask, int mstride, int S, cudaStream_t st,
                     int inputs)
{
    count_launch(1);
    if (inputs == 0) {  // convert the state and the coefficients
        count_launch(1);
        dim3 gin(nblocks(std::max(G.N, G.C)), S);
        k_jac_inputs<T><<<gin, kBS, 0, st>>>(G, ph, phi, K, p, c, cellT, nodeT, mask, mstride);
    } else if (inputs == 1) {  // the coefficients are converted already
        count_launch(1);
        k_node_inputs<T><<<dim3(nblocks(G.N), S), kBS, 0, st>>>(G, ph.rho0 * ph.g, p, c, nodeT,
                                                                mask, mstride);
    }
    dim3 grid(nblocks(G.N, 128), S);
    // lumped storage volume per unit phi over dt: (h^3 / 8) / dt per cell corner
    const T vscale = T(0.125 * G.hx * G.hy * G.hz / ph.dt);
    const CellGeom cgd = make_geom(G);
    GeomT<T> cg;
    for (int d = 0; d < 3; ++d) {
        cg.ih[d] = T(cgd.ih[d]);
        cg.area[d] = T(cgd.area[d]);
    }
    const PhysT<T> pt{T(ph.rho0), T(ph.drho), T(ph.g), T(ph.Dm)};
    k_jacobian<T, M><<<grid, 128, 0, st>>>(G, pt, cg, bc, cellT, nodeT, JT, JM, Dinv, vscale,
                                            mask, mstride);
}
template void launch_jacobian<double, double>(const Grid&, const Phys&, const uint8_t*,
                                              const double*, const double*, const double*,
                                              const double*, B4<double>*, B4<double>*,
                                              B4<double>*, V2<double>*, V2<double>*, const int*,
                                              int, int, cudaStream_t, int);
template void launch_jacobian<float, __nv_bfloat16>(const Grid&, const Phys&, const uint8_t*,
                                                    const double*, const double*,
                                                    const double*, const double*, B4<float>*,
                                                    B4<__nv_bfloat16>*, B4<float>*, V2<float>*,
                                                    V2<float>*, const int*, int, int,
                                                    cudaStream_t, int);

// ---------------------------------------------------------------------------
// hierarchy: state injection, cell averaging, block-diagonal inverse
// ---------------------------------------------------------------------------

// State injection to the coarse grid; with nodeT also the coarse Jacobian's
// node inputs (p - rho0 g (Lz - z), c) in T, as k_jac_inputs forms them.
template <class T>
__global__ void k_inject(Grid Gf, Grid Gc, const double* __restrict__ pf,
                         const double* __restrict__ cf, double* __restrict__ pc,
                         double* __restrict__ cc, V2<T>* __restrict__ nodeT, double rho0g,
                         const int* mask, int mstride)
{
    const int s = blockIdx.y;
    if (!sample_on(mask, mstride, s)) return;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= Gc.N) return;
    int I, J, K;
    node_ijk(Gc, n, I, J, K);
    const int f = node_id(Gf, 2 * I, 2 * J, 2 * K);
    const size_t o = (size_t)s * Gc.N + n;
    const double pv = pf[(size_t)s * Gf.N + f], cv = cf[(size_t)s * Gf.N + f];
    pc[o] = pv;
    cc[o] = cv;
    if (nodeT) {
        const double z = K * Gc.hz;
        nodeT[o] = V2<T>{T(fma(rho0g, z - Gc.Lz, pv)), T(cv)};
    }
}

template <class T>
void launch_inject(const Grid& Gf, const Grid& Gc, const double* pf, const double* cf,
                   double* pc, double* cc, V2<T>* nodeT, double rho0g, const int* mask,
                   int mstride, int S, cudaStream_t st)
{
    count_launch(1);
    dim3 grid(nblocks(Gc.N), S);
    k_inject<T><<<grid, kBS, 0, st>>>(Gf, Gc, pf, cf, pc, cc, nodeT, rho0g, mask, mstride);
}
template void launch_inject<float>(const Grid&, const Grid&, const double*, const double*,
                                   double*, double*, V2<float>*, double, const int*, int, int,
                                   cudaStream_t);
template void launch_inject<double>(const Grid&, const Grid&, const double*, const double*,
                                    double*, double*, V2<double>*, double, const int*, int, int,
                                    cudaStream_t);

__global__ void k_average_cells(Grid Gf, Grid Gc, const double* __restrict__ phif,
                                const double* __restrict__ Kf,
                                double* __restrict__ phic,
                                double* __restrict__ Kc, int harmonic)
{
    const int s = blockIdx.y;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= Gc.C) return;
    const int I = e % Gc.nx, J = (e / Gc.nx) % Gc.ny, K = e / (Gc.nx * Gc.ny);
    double sp = 0.0, sk = 0.0;
    for (int q = 0; q < 8; ++q) {
        const int f = (2 * I + (q & 1)) +
                      Gf.nx * ((2 * J + ((q >> 1) & 1)) + Gf.ny * (2 * K + (q >> 2)));
        sp += phif[(size_t)s * Gf.C + f];
        const double kv = Kf[(size_t)s * Gf.C + f];
        sk += harmonic ? 1.0 / kv : kv;
    }
    phic[(size_t)s * Gc.C + e] = 0.125 * sp;
    Kc[(size_t)s * Gc.C + e] = harmonic ? 8.0 / sk : 0.125 * sk;
}

void launch_average_cells(const Grid& Gf, const Grid& Gc, const double* phif,
                          const double* Kf, double* phic, double* Kc,
                          int harmonic, int S, cudaStream_t st)
{
    count_launch(1);
    dim3 grid(nblocks(Gc.C), S);
    k_average_cells<<<grid, kBS, 0, st>>>(Gf, Gc, phif, Kf, phic, Kc, harmonic);
}

// ---------------------------------------------------------------------------
// coarsest level: dense inverse of the interior operator (Gauss-Jordan with
// partial pivoting, FP64), one block per sample.  work: [S][n][2n].
// ---------------------------------------------------------------------------

template <class M, class R>
__global__ void k_coarse_build(Grid G, const uint8_t* __restrict__ bc,
                               const B4<M>* __restrict__ J, R* __restrict__ W,
                               const int* mask, int mstride)
{
    const int s = blockIdx.y;
    if (!sample_on(mask, mstride, s)) return;
    const int node = blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= G.N) return;
    const int n2 = 2 * G.N;
    R* row0 = W + (size_t)s * n2 * 2 * n2 + (size_t)(2 * node) * 2 * n2;
    R* row1 = row0 + 2 * n2;
    for (int q = 0; q < 2 * n2; ++q) { row0[q] = R(0); row1[q] = R(0); }
    int i, j, k;
    node_ijk(G, node, i, j, k);
    const uint8_t mr = bc[node];
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const int ii = i + dx, jj = j + dy, kk = k + dz;
                if (ii < 0 || ii > G.nx || jj < 0 || jj > G.ny || kk < 0 || kk > G.nz)
                    continue;
                const int m = node_id(G, ii, jj, kk);
                const uint8_t mc = bc[m];
                const B4<M> B = J[((size_t)s * 27 + slot27(dx, dy, dz)) * G.N + node];
                if (!(mr & BC_P)) {
                    if (!(mc & BC_P)) row0[2 * m] = mg_load<R>(B.pp);
                    if (!(mc & BC_C)) row0[2 * m + 1] = mg_load<R>(B.pc);
                }
                if (!(mr & BC_C)) {
                    if (!(mc & BC_P)) row1[2 * m] = mg_load<R>(B.cp);
                    if (!(mc & BC_C)) row1[2 * m + 1] = mg_load<R>(B.cc);
                }
            }
    if (mr & BC_P) row0[2 * node] = R(1);
    if (mr & BC_C) row1[2 * node + 1] = R(1);
    row0[n2 + 2 * node] = R(1);
    row1[n2 + 2 * node + 1] = R(1);
}

// Gauss-Jordan with partial pivoting on [A | I] of one sample per block, in
// arithmetic R (FP32 for the mixed solver, whose coarse matrix is stored in
// bfloat16 and is only a preconditioner; FP64 otherwise).  SMEM: the
// augmented matrix is copied into shared memory first (it fits for the
// 100-unknown 4x4x1 coarsest grid), which keeps the n elimination sweeps
// off L2; otherwise it is eliminated in place in global memory.  Each warp
// updates whole rows, columns k..2n-1 only.
template <bool SMEM, class R>
__global__ void k_gauss_jordan(int n, R* __restrict__ W, R* __restrict__ Ainv, const int* mask,
                               int mstride)
{
    extern __shared__ __align__(16) unsigned char gj_smem[];
    __shared__ R rv[32];
    __shared__ int ri[32];
    const int s = blockIdx.x;
    if (!sample_on(mask, mstride, s)) return;
    const int w2 = 2 * n;
    R* f = reinterpret_cast<R*>(gj_smem);
    R* A = W + (size_t)s * n * w2;
    if (SMEM) {
        R* As = f + n;
        for (int q = threadIdx.x; q < n * w2; q += blockDim.x) As[q] = A[q];
        A = As;
        __syncthreads();
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = 0; k < n; ++k) {
        // pivot: argmax |A[r][k]| over r >= k (ties to the lower row)
        R best = R(-1);
        int bi = k;
        for (int r = k + threadIdx.x; r < n; r += blockDim.x) {
            const R a = fabs(A[(size_t)r * w2 + k]);
            if (a > best) { best = a; bi = r; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const R ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (lane == 0) { rv[warp] = best; ri[warp] = bi; }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int q = 1; q < nw; ++q)
                if (rv[q] > rv[0] || (rv[q] == rv[0] && ri[q] < ri[0])) { rv[0] = rv[q]; ri[0] = ri[q]; }
        }
        __syncthreads();
        const int piv = ri[0];
        __syncthreads();
        if (piv != k)
            for (int q = threadIdx.x; q < w2; q += blockDim.x) {
                const R t = A[(size_t)k * w2 + q];
                A[(size_t)k * w2 + q] = A[(size_t)piv * w2 + q];
                A[(size_t)piv * w2 + q] = t;
            }
        __syncthreads();
        const R inv = R(1) / A[(size_t)k * w2 + k];
        __syncthreads();
        for (int q = threadIdx.x; q < w2; q += blockDim.x) A[(size_t)k * w2 + q] *= inv;
        for (int r = threadIdx.x; r < n; r += blockDim.x) f[r] = A[(size_t)r * w2 + k];
        __syncthreads();
        for (int r = warp; r < n; r += nw) {
            if (r == k) continue;
            const R fr = f[r];
            for (int q = k + lane; q < w2; q += 32)
                A[(size_t)r * w2 + q] -= fr * A[(size_t)k * w2 + q];
        }
        __syncthreads();
    }
    R* out = Ainv + (size_t)s * n * n;
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int r = idx / n, q = idx - r * n;
        out[idx] = A[(size_t)r * w2 + n + q];
    }
}

template <class M>
void launch_coarse_inverse(const Grid& G, const uint8_t* bc, const B4<M>* J,
                           double* work, double* Ainv, const int* mask,
                           int mstride, int S, cudaStream_t st)
{
    using R = typename CoarseType<M>::type;
    count_launch(2);
    dim3 grid(nblocks(G.N, 64), S);
    R* W = reinterpret_cast<R*>(work);
    k_coarse_build<M, R><<<grid, 64, 0, st>>>(G, bc, J, W, mask, mstride);
    const int n = 2 * G.N;
    R* Ai = reinterpret_cast<R*>(Ainv);
    const size_t smem = sizeof(R) * ((size_t)n + (size_t)2 * n * n);
    if (smem <= 200 * 1024) {
        static bool attr_set = false;
        if (!attr_set) {
            cudaFuncSetAttribute(k_gauss_jordan<true, R>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
            attr_set = true;
        }
        k_gauss_jordan<true, R><<<S, 256, smem, st>>>(n, W, Ai, mask, mstride);
    } else {
        k_gauss_jordan<false, R><<<S, 256, sizeof(R) * n, st>>>(n, W, Ai, mask, mstride);
    }
}
template void launch_coarse_inverse<double>(const Grid&, const uint8_t*,
                                            const B4<double>*, double*,
                                            double*, const int*, int, int,
                                            cudaStream_t);
template void launch_coarse_inverse<__nv_bfloat16>(const Grid&, const uint8_t*,
                                                   const B4<__nv_bfloat16>*, double*,
                                                   double*, const int*, int, int,
                                                   cudaStream_t);

// ---------------------------------------------------------------------------
// Dirichlet data and sample fields
// ---------------------------------------------------------------------------

__global__ void k_impose_dirichlet(Grid G, const uint8_t* __restrict__ bc,
                                   const double* __restrict__ cval, double* p,
                                   double* c)
{
    const int s = blockIdx.y;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= G.N) return;
    const uint8_t b = bc[n];
    if (b & BC_P) p[(size_t)s * G.N + n] = 0.0;
    if (b & BC_C) c[(size_t)s * G.N + n] = cval[n];
}

// Initial state (Section 2.1): Dirichlet c values, c = 0 elsewhere, and the
// hydrostatic pressure of pure water p = rho0 g (Lz - z).
__global__ void k_initial_state(Grid G, double rho0g, const uint8_t* __restrict__ bc,
                                const double* __restrict__ cval, double* p, double* c)
{
    const int s = blockIdx.y;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= G.N) return;
    int i, j, k;
    node_ijk(G, n, i, j, k);
    p[(size_t)s * G.N + n] = rho0g * (G.Lz - k * G.hz);
    c[(size_t)s * G.N + n] = (bc[n] & BC_C) ? cval[n] : 0.0;
}

void launch_initial_state(const Grid& G, double rho0g, const uint8_t* bc,
                          const double* cval, double* p, double* c, int S,
                          cudaStream_t st)
{
    count_launch(1);
    dim3 grid(nblocks(G.N), S);
    k_initial_state<<<grid, kBS, 0, st>>>(G, rho0g, bc, cval, p, c);
}

void launch_impose_dirichlet(const Grid& G, const uint8_t* bc,
                             const double* cval, double* p, double* c, int S,
                             cudaStream_t st)
{
    count_launch(1);
    dim3 grid(nblocks(G.N), S);
    k_impose_dirichlet<<<grid, kBS, 0, st>>>(G, bc, cval, p, c);
}

// Section 2.2: porosity realisations and Kozeny-Carman permeability
// (eq. e_perm_Kozeny_Carman, normalised so that K(0.1) = K_mean).
__global__ void k_fields(Grid G, int kind, const double* __restrict__ params,
                         double K_mean, double* __restrict__ phi,
                         double* __restrict__ K)
{
    const int s = blockIdx.y;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= G.C) return;
    const int i = e % G.nx, j = (e / G.nx) % G.ny, k = e / (G.nx * G.ny);
    const double Lx = G.nx * G.hx, Ly = G.ny * G.hy, Lz = G.nz * G.hz;
    const double x = (i + 0.5) * G.hx, y = (j + 0.5) * G.hy, z = (k + 0.5) * G.hz;
    const double pi = 3.14159265358979323846;
    double ph;
    if (kind == 1) {
        ph = 0.1 * exp(0.2 * params[(size_t)s * G.C + e]);
        ph = fmin(fmax(ph, 0.05), 0.2);
    } else {
        const double* xi = params + (size_t)s * 3;
        if (kind == 0) {
            const double f = xi[0] * cos(pi * x / Lx) + xi[1] * cos(pi * y / Ly) +
                             xi[2] * sin(2.0 * pi * z / Lz);
            ph = 0.1 * (1.0 + 0.3 * f / 3.0);
        } else {
            const double sx = sin(pi * x / Lx), sy = sin(pi * y / Ly), sz = sin(pi * z / Lz);
            ph = 0.1 + 0.01 * (xi[0] * sx + xi[1] * sy + xi[2] * sz + xi[0] * sx * sy +
                               xi[1] * sx * sz);
        }
    }
    const double ref = (0.1 * 0.1 * 0.1) / (0.9 * 0.9);
    phi[(size_t)s * G.C + e] = ph;
    K[(size_t)s * G.C + e] = K_mean * (ph * ph * ph / ((1.0 - ph) * (1.0 - ph))) / ref;
}

void launch_fields(const Grid& G, int kind, const double* params,
                   double K_mean, double* phi, double* K, int S,
                   cudaStream_t st)
{
    count_launch(1);
    dim3 grid(nblocks(G.C), S);
    k_fields<<<grid, kBS, 0, st>>>(G, kind, params, K_mean, phi, K);
}

// ---------------------------------------------------------------------------
// adjoint pieces (one sample)
// ---------------------------------------------------------------------------
//
// Objective: salt mass in the cells whose centre lies below Lz/2,
// J = sum_e sum_corners phi_e |scv| rho(c_L) c_L.

__global__ void k_objective_cells(Grid G, Phys ph, const double* __restrict__ phi,
                                  const double* __restrict__ c,
                                  double* __restrict__ partial,
                                  double* __restrict__ dJdphi)
{
    __shared__ double red[32];
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    double Jl = 0.0;
    if (e < G.C) {
        const int i = e % G.nx, j = (e / G.nx) % G.ny, k = e / (G.nx * G.ny);
        const double vscv = 0.125 * G.hx * G.hy * G.hz;
        double sm = 0.0;
        if ((k + 0.5) * G.hz < 0.5 * G.Lz) {
            for (int L = 0; L < 8; ++L) {
                const double cc = c[node_id(G, i + (L & 1), j + ((L >> 1) & 1), k + (L >> 2))];
                sm += vscv * fma(ph.drho, cc, ph.rho0) * cc;
            }
        }
        dJdphi[e] = sm;
        Jl = phi[e] * sm;
    }
    const double t = block_sum(Jl, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

__global__ void k_objective_nodes(Grid G, Phys ph, const double* __restrict__ phi,
                                  const double* __restrict__ c,
                                  V2<double>* __restrict__ dJdu)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= G.N) return;
    int i, j, k;
    node_ijk(G, n, i, j, k);
    const double vscv = 0.125 * G.hx * G.hy * G.hz;
    double phis = 0.0;
    for (int q = 0; q < 8; ++q) {
        const int ci = i - (q & 1), cj = j - ((q >> 1) & 1), ck = k - (q >> 2);
        if (ci < 0 || ci >= G.nx || cj < 0 || cj >= G.ny || ck < 0 || ck >= G.nz) continue;
        if (!((ck + 0.5) * G.hz < 0.5 * G.Lz)) continue;
        phis += phi[ci + G.nx * (cj + G.ny * ck)];
    }
    const double cc = c[n];
    dJdu[n] = V2<double>{0.0, phis * vscv * (ph.rho0 + 2.0 * ph.drho * cc)};
}

void launch_objective(const Grid& G, const Phys& ph, const double* phi,
                      const double* c, double* partial, double* dJdphi,
                      V2<double>* dJdu, cudaStream_t st)
{
    count_launch(1);
    k_objective_cells<<<nblocks(G.C), kBS, 0, st>>>(G, ph, phi, c, partial, dJdphi);
    count_launch(1);
    k_objective_nodes<<<nblocks(G.N), kBS, 0, st>>>(G, ph, phi, c, dJdu);
}

// -lambda_n^T dR_n/dtheta per cell: R_n depends on phi_e through the storage
// of the cell's 8 sub-control volumes and the diffusive part of the 12 face
// fluxes, on K_e through the Darcy mass flux m (and c_up m).  Dirichlet rows
// do not depend on theta.
template <int D, int S_, int T_>
__device__ __forceinline__ void adj_face(const double (&p8)[8],
                                         const double (&c8)[8],
                                         const double (&lp)[8],
                                         const double (&lc)[8], double phi_e,
                                         double K_e, const Phys& ph,
                                         double invh, double area,
                                         double& gphi, double& gK)
{
    double gp = 0.0, gc = 0.0, ci = 0.0;
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 2; ++v) {
            const double w = (u == S_ ? 0.75 : 0.25) * (v == T_ ? 0.75 : 0.25);
            const int A = corner_of(D, u, v, 0), B = corner_of(D, u, v, 1);
            gp = fma(w, p8[B] - p8[A], gp);
            gc = fma(w, c8[B] - c8[A], gc);
            ci = fma(w, c8[A] + c8[B], ci);
        }
    gp *= invh;
    gc *= invh;
    ci *= 0.5;
    const double rho = fma(ph.drho, ci, ph.rho0);
    const double G = (D == 2) ? fma(ph.g, rho, gp) : gp;
    const double m = rho * (-(K_e / ph.mu) * G) * area;
    constexpr int a = corner_of(D, S_, T_, 0), b = corner_of(D, S_, T_, 1);
    const double cup = (m >= 0.0) ? c8[a] : c8[b];
    const double dF_dphi = -rho * ph.Dm * gc * area;
    const double dm_dK = m / K_e;
    gphi += (lc[a] - lc[b]) * dF_dphi;
    gK += (lp[a] - lp[b]) * dm_dK + (lc[a] - lc[b]) * cup * dm_dK;
}

__global__ void k_adjoint_theta(Grid G, Phys ph, CellGeom cg,
                                const uint8_t* __restrict__ bc,
                                const double* __restrict__ phi,
                                const double* __restrict__ K,
                                const double* __restrict__ p,
                                const double* __restrict__ c,
                                const double* __restrict__ c_old,
                                const V2<double>* __restrict__ lam,
                                double* __restrict__ dJdphi,
                                double* __restrict__ dJdK)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= G.C) return;
    const int i = e % G.nx, j = (e / G.nx) % G.ny, k = e / (G.nx * G.ny);
    const double phi_e = phi[e], K_e = K[e];
    const double vdt = 0.125 * G.hx * G.hy * G.hz / ph.dt;
    double p8[8], c8[8], lp[8], lc[8];
    double gphi = 0.0, gK = 0.0;
#pragma unroll
    for (int L = 0; L < 8; ++L) {
        const int nd = node_id(G, i + (L & 1), j + ((L >> 1) & 1), k + (L >> 2));
        p8[L] = p[nd];
        c8[L] = c[nd];
        const uint8_t b = bc[nd];
        const V2<double> l = lam[nd];
        lp[L] = (b & BC_P) ? 0.0 : l.p;   // Dirichlet rows carry no theta
        lc[L] = (b & BC_C) ? 0.0 : l.c;
        const double co = c_old[nd];
        const double rn = fma(ph.drho, c8[L], ph.rho0), ro = fma(ph.drho, co, ph.rho0);
        gphi += lp[L] * vdt * (rn - ro) + lc[L] * vdt * (rn * c8[L] - ro * co);
    }
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            if (s == 0 && t == 0) {
                adj_face<0, 0, 0>(p8, c8, lp, lc, phi_e, K_e, ph, cg.ih[0], cg.area[0], gphi, gK);
                adj_face<1, 0, 0>(p8, c8, lp, lc, phi_e, K_e, ph, cg.ih[1], cg.area[1], gphi, gK);
                adj_face<2, 0, 0>(p8, c8, lp, lc, phi_e, K_e, ph, cg.ih[2], cg.area[2], gphi, gK);
            } else if (s == 0 && t == 1) {
                adj_face<0, 0, 1>(p8, c8, lp, lc, phi_e, K_e, ph, cg.ih[0], cg.area[0], gphi, gK);
                adj_face<1, 0, 1>(p8, c8, lp, lc, phi_e, K_e, ph, cg.ih[1], cg.area[1], gphi, gK);
                adj_face<2, 0, 1>(p8, c8, lp, lc, phi_e, K_e, ph, cg.ih[2], cg.area[2], gphi, gK);
            } else if (s == 1 && t == 0) {
                adj_face<0, 1, 0>(p8, c8, lp, lc, phi_e, K_e, ph, cg.ih[0], cg.area[0], gphi, gK);
                adj_face<1, 1, 0>(p8, c8, lp, lc, phi_e, K_e, ph, cg.ih[1], cg.area[1], gphi, gK);
                adj_face<2, 1, 0>(p8, c8, lp, lc, phi_e, K_e, ph, cg.ih[2], cg.area[2], gphi, gK);
            } else {
                adj_face<0, 1, 1>(p8, c8, lp, lc, phi_e, K_e, ph, cg.ih[0], cg.area[0], gphi, gK);
                adj_face<1, 1, 1>(p8, c8, lp, lc, phi_e, K_e, ph, cg.ih[1], cg.area[1], gphi, gK);
                adj_face<2, 1, 1>(p8, c8, lp, lc, phi_e, K_e, ph, cg.ih[2], cg.area[2], gphi, gK);
            }
        }
    dJdphi[e] -= gphi;
    dJdK[e] -= gK;
}

void launch_adjoint_theta(const Grid& G, const Phys& ph, const uint8_t* bc,
                          const double* phi, const double* K, const double* p,
                          const double* c, const double* c_old,
                          const V2<double>* lam, double* dJdphi, double* dJdK,
                          cudaStream_t st)
{
    count_launch(1);
    k_adjoint_theta<<<nblocks(G.C), kBS, 0, st>>>(G, ph, make_geom(G), bc, phi, K,
                                                  p, c, c_old, lam, dJdphi, dJdK);
}

// rhs of step n-1: -(dR_n/du_{n-1})^T lambda_n.  R_n depends on u_{n-1} only
// through the old storage -S(c_{n-1})/dt, which is diagonal in the node.
__global__ void k_adjoint_prev_rhs(Grid G, Phys ph, const uint8_t* __restrict__ bc,
                                   const double* __restrict__ phi,
                                   const double* __restrict__ c_old,
                                   const V2<double>* __restrict__ lam,
                                   V2<double>* __restrict__ rhs)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= G.N) return;
    int i, j, k;
    node_ijk(G, n, i, j, k);
    double phis = 0.0;
    for (int q = 0; q < 8; ++q) {
        const int ci = i - (q & 1), cj = j - ((q >> 1) & 1), ck = k - (q >> 2);
        if (ci < 0 || ci >= G.nx || cj < 0 || cj >= G.ny || ck < 0 || ck >= G.nz) continue;
        phis += phi[ci + G.nx * (cj + G.ny * ck)];
    }
    const double vdt = phis * 0.125 * G.hx * G.hy * G.hz / ph.dt;
    const uint8_t b = bc[n];
    const V2<double> l = lam[n];
    double r = 0.0;
    if (!(b & BC_P)) r += vdt * ph.drho * l.p;
    if (!(b & BC_C)) r += vdt * (ph.rho0 + 2.0 * ph.drho * c_old[n]) * l.c;
    rhs[n] = V2<double>{0.0, r};
}

void launch_adjoint_prev_rhs(const Grid& G, const Phys& ph, const uint8_t* bc,
                             const double* phi, const double* c_old,
                             const V2<double>* lam, V2<double>* rhs,
                             cudaStream_t st)
{
    count_launch(1);
    k_adjoint_prev_rhs<<<nblocks(G.N), kBS, 0, st>>>(G, ph, bc, phi, c_old, lam, rhs);
}

// ---------------------------------------------------------------------------
// Allocation-free residual with per-sample norms.
//
// For callers that may not allocate device memory at all (not even through a
// context: elder_create allocates the multigrid workspace), e.g. code that
// runs after another runtime has taken over the device's memory pool, or a
// host thread that is only allowed to enqueue work.  The only scratch this
// needs, the per-block partial sums of ||R||^2, lives in the file-scope
// array below; the Dirichlet sets are evaluated from the grid indices
// instead of being read from a context.
// ---------------------------------------------------------------------------

// Scratch capacity in doubles: 2 MiB on every device that loads the library,
// held until the process exits.  A call needs S * ceil(N / 256) entries.
constexpr size_t kStaticScratchDoubles = size_t(1) << 18;
static __device__ __align__(256) double g_static_scratch[kStaticScratchDoubles];

// Dirichlet bits and c value of node (i,j,k) (the sets listed in elder.h).
__device__ __forceinline__ uint8_t dirichlet_inline(int mode, const Grid& G, int i, int j,
                                                    int k, double& cv)
{
    const bool top = (k == G.nz), bottom = (k == 0);
    const bool xe = (i == 0 || i == G.nx), ye = (j == 0 || j == G.ny);
    const bool sq = (4 * i >= G.nx && 4 * i <= 3 * G.nx && 4 * j >= G.ny && 4 * j <= 3 * G.ny);
    uint8_t b = 0;
    cv = 0.0;
    if (mode == 1) {
        if (top && (xe || ye)) b |= BC_P;
        if (top) { b |= BC_C; cv = sq ? 1.0 : 0.0; }
        else if (bottom) b |= BC_C;
    } else {
        if (top && xe && ye) b |= BC_P;
        if (mode == 0) {
            if (top && sq) { b |= BC_C; cv = 1.0; }
            else if (bottom) b |= BC_C;
        } else if (mode == 2) {
            if (top) { b |= BC_C; cv = 1.0; }
            else if (bottom) b |= BC_C;
        }
    }
    return b;
}

__global__ void __launch_bounds__(kBS)
    k_residual_static(Grid G, Phys ph, CellGeom cg, int bc_mode,
                      const double* __restrict__ phi, const double* __restrict__ K,
                      const double* __restrict__ p, const double* __restrict__ c,
                      const double* __restrict__ p_old, const double* __restrict__ c_old,
                      V2<double>* __restrict__ R, double* __restrict__ scratch)
{
    __shared__ double red[32];
    const int s = blockIdx.y;
    const size_t on = (size_t)s * G.N, oc = (size_t)s * G.C;
    phi += oc; K += oc; p += on; c += on; p_old += on; c_old += on; R += on;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    double sq = 0.0;
    if (n < G.N) {
        int i, j, k;
        node_ijk(G, n, i, j, k);
        double Rp = 0.0, Rc = 0.0, phis = 0.0, Ap = 0.0, Ac = 0.0;
        residual_cell<-1, -1, -1>(G, ph, cg, i, j, k, phi, K, p, c, Rp, Rc, phis, Ap, Ac);
        residual_cell<0, -1, -1>(G, ph, cg, i, j, k, phi, K, p, c, Rp, Rc, phis, Ap, Ac);
        residual_cell<-1, 0, -1>(G, ph, cg, i, j, k, phi, K, p, c, Rp, Rc, phis, Ap, Ac);
        residual_cell<0, 0, -1>(G, ph, cg, i, j, k, phi, K, p, c, Rp, Rc, phis, Ap, Ac);
        residual_cell<-1, -1, 0>(G, ph, cg, i, j, k, phi, K, p, c, Rp, Rc, phis, Ap, Ac);
        residual_cell<0, -1, 0>(G, ph, cg, i, j, k, phi, K, p, c, Rp, Rc, phis, Ap, Ac);
        residual_cell<-1, 0, 0>(G, ph, cg, i, j, k, phi, K, p, c, Rp, Rc, phis, Ap, Ac);
        residual_cell<0, 0, 0>(G, ph, cg, i, j, k, phi, K, p, c, Rp, Rc, phis, Ap, Ac);
        const double vscv = 0.125 * G.hx * G.hy * G.hz;
        const double cn = c[n], co = c_old[n];
        const double rn = fma(ph.drho, cn, ph.rho0), ro = fma(ph.drho, co, ph.rho0);
        Rp += phis * vscv * (rn - ro) / ph.dt;
        Rc += phis * vscv * (rn * cn - ro * co) / ph.dt;
        double cv;
        const uint8_t b = dirichlet_inline(bc_mode, G, i, j, k, cv);
        if (b & BC_P) Rp = p[n];
        if (b & BC_C) Rc = cn - cv;
        R[n] = V2<double>{Rp, Rc};
        sq = Rp * Rp + Rc * Rc;
    }
    const double t = block_sum(sq, red);
    if (threadIdx.x == 0) scratch[(size_t)s * gridDim.x + blockIdx.x] = t;
}

__global__ void k_norms_static(int nblk, const double* __restrict__ scratch,
                               double* __restrict__ norms)
{
    __shared__ double red[32];
    const int s = blockIdx.x;
    double a = 0.0;
    for (int q = threadIdx.x; q < nblk; q += blockDim.x) a += scratch[(size_t)s * nblk + q];
    a = block_sum(a, red);
    if (threadIdx.x == 0) norms[s] = sqrt(a);
}

}  // namespace elder

#include <mutex>

#include "../../include/elder.h"

namespace {
constexpr int kMaxDevices = 64;
double* g_scratch_addr[kMaxDevices] = {};  // device address of the array, per device
std::mutex g_scratch_mutex;
}  // namespace

extern "C" int elder_residual_norms_static(const elder_config* cfg, int S, const double* phi,
                                           const double* K, const double* p, const double* c,
                                           const double* p_old, const double* c_old,
                                           double dt, double* R, double* norms, void* stream)
{
    using namespace elder;
    if (!cfg || S < 1 || !phi || !K || !p || !c || !p_old || !c_old || !R || !norms ||
        !(dt > 0)) {
        set_static_error("elder_residual_norms_static: bad argument");
        return ELDER_EINVAL;
    }
    const elder_config& f = *cfg;
    if (f.nx < 1 || f.ny < 1 || f.nz < 1 || f.bc_mode < 0 || f.bc_mode > 3 ||
        ((f.bc_mode == 0 || f.bc_mode == 1) && (f.nx % 4 || f.ny % 4)) || !(f.mu > 0)) {
        set_static_error("elder_residual_norms_static: invalid elder_config");
        return ELDER_EINVAL;
    }
    Grid G;
    G.nx = f.nx;
    G.ny = f.ny;
    G.nz = f.nz;
    G.N = (f.nx + 1) * (f.ny + 1) * (f.nz + 1);
    G.C = f.nx * f.ny * f.nz;
    G.hx = f.Lx / f.nx;
    G.hy = f.Ly / f.ny;
    G.hz = f.Lz / f.nz;
    G.Lz = f.Lz;
    grid_set_divisors(G);
    const int nblk = nblocks(G.N);
    if (S > 65535) {  // samples run along grid.y
        set_static_error("elder_residual_norms_static: S exceeds 65535 samples per call");
        return ELDER_EINVAL;
    }
    if ((size_t)S * (size_t)nblk > kStaticScratchDoubles) {
        set_static_error("elder_residual_norms_static: S * ceil(N/256) exceeds the static "
                         "scratch capacity (262144 partial sums)");
        return ELDER_EINVAL;
    }
    // once per device, with that device current: the device address of the
    // file-scope array (its host-side name is only a stand-in)
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        set_static_error("elder_residual_norms_static: no usable current device");
        return ELDER_ECUDA;
    }
    {
        std::lock_guard<std::mutex> lock(g_scratch_mutex);
        if (!g_scratch_addr[dev]) {
            void* ptr = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
            if (e != cudaSuccess || !ptr) {
                set_static_error(cudaGetErrorString(e));
                return ELDER_ECUDA;
            }
            g_scratch_addr[dev] = static_cast<double*>(ptr);
        }
    }
    const Phys ph{f.rho0, f.rho1 - f.rho0, f.mu, f.g, f.Dm, dt};
    cudaStream_t st = (cudaStream_t)stream;
    count_launch(2);
    k_residual_static<<<dim3(nblk, S), kBS, 0, st>>>(G, ph, make_geom(G), f.bc_mode, phi, K, p,
                                                     c, p_old, c_old,
                                                     reinterpret_cast<V2<double>*>(R),
                                                     g_scratch_addr[dev]);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {  // the norms are not formed from stale partial sums
        set_static_error(cudaGetErrorString(e));
        return ELDER_ECUDA;
    }
    k_norms_static<<<S, 128, 0, st>>>(nblk, g_scratch_addr[dev], norms);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_static_error(cudaGetErrorString(e));
        return ELDER_ECUDA;
    }
    return ELDER_OK;
}

namespace elder {

// ---------------------------------------------------------------------------
// Salt-mass balance of a step (FP64): M = sum_i sum_{e ni i} phi_e |scv|
// rho(c_i) c_i at u^n and u^{n+1}, and the salt that entered through the
// c-Dirichlet nodes, dt * sum_{i in D} (net face salt flux out of i).
// The face fluxes telescope, so M^{n+1} - M^n = inflow + dt * sum of the
// interior salt residuals.  partial: [S][3][nblk].
// ---------------------------------------------------------------------------

// Salt flux out of node (i, j, k) through the 3 quarter faces of cell
// (i + OX, j + OY, k + OZ) on the boundary of the node's sub-control volume,
// with the face arithmetic of k_cell_flux (quarter_face)
template <int OX, int OY, int OZ>
__device__ __forceinline__ double corner_salt_out(const Grid& G, const Phys& ph,
                                                  const FluxConst& fc, int i, int j, int k,
                                                  const double* __restrict__ phi,
                                                  const double* __restrict__ K,
                                                  const double* __restrict__ p,
                                                  const double* __restrict__ c)
{
    const int ci = i + OX, cj = j + OY, ck = k + OZ;
    if (ci < 0 || ci >= G.nx || cj < 0 || cj >= G.ny || ck < 0 || ck >= G.nz) return 0.0;
    const int e = ci + G.nx * (cj + G.ny * ck);
    const int sy = G.nx + 1, sz = (G.nx + 1) * (G.ny + 1);
    const int base = ci + sy * cj + sz * ck;
    double p8[8], c8[8];
#pragma unroll
    for (int L = 0; L < 8; ++L) {
        const int off = (L & 1) + ((L >> 1) & 1) * sy + (L >> 2) * sz;
        p8[L] = __ldg(p + base + off);
        c8[L] = __ldg(c + base + off);
    }
    const double phie = __ldg(phi + e), Ke = __ldg(K + e);
    double Zc[8];
    cube31(c8, Zc);
    constexpr int lx = -OX, ly = -OY, lz = -OZ;  // the node's corner of the cell
    double out = 0.0, m, F, gp[2][2];
    bool up;
    // the node is the lower end of the face's edge along D (+F) or the upper (-F)
    dir_grad<0>(p8, gp);
    quarter_face<0>(ly, lz, gp, c8, Zc, ph, fc, Ke * fc.kA[0], phie * fc.dA2[0], m, F, up);
    out += lx == 0 ? F : -F;
    dir_grad<1>(p8, gp);
    quarter_face<1>(lx, lz, gp, c8, Zc, ph, fc, Ke * fc.kA[1], phie * fc.dA2[1], m, F, up);
    out += ly == 0 ? F : -F;
    dir_grad<2>(p8, gp);
    quarter_face<2>(lx, ly, gp, c8, Zc, ph, fc, Ke * fc.kA[2], phie * fc.dA2[2], m, F, up);
    out += lz == 0 ? F : -F;
    return out;
}

__global__ void __launch_bounds__(kBS)
    k_mass_balance(Grid G, Phys ph, FluxConst fc, const uint8_t* __restrict__ bc,
                   const double* __restrict__ phi, const double* __restrict__ K,
                   const double* __restrict__ p, const double* __restrict__ c,
                   const double* __restrict__ c_old, double* __restrict__ partial)
{
    __shared__ double red[32];
    const int s = blockIdx.y;
    const size_t on = (size_t)s * G.N, oc = (size_t)s * G.C;
    phi += oc; K += oc; p += on; c += on; c_old += on;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    double m1 = 0.0, m0 = 0.0, in = 0.0;
    if (n < G.N) {
        int i, j, k;
        node_ijk(G, n, i, j, k);
        double phis = 0.0;
        for (int q = 0; q < 8; ++q) {
            const int ci = i - (q & 1), cj = j - ((q >> 1) & 1), ck = k - (q >> 2);
            if (ci < 0 || ci >= G.nx || cj < 0 || cj >= G.ny || ck < 0 || ck >= G.nz) continue;
            phis += phi[ci + G.nx * (cj + G.ny * ck)];
        }
        const double vscv = 0.125 * G.hx * G.hy * G.hz;
        const double cn = c[n], co = c_old[n];
        m1 = phis * vscv * fma(ph.drho, cn, ph.rho0) * cn;
        m0 = phis * vscv * fma(ph.drho, co, ph.rho0) * co;
        if (bc[n] & BC_C) {
            double Rc = corner_salt_out<-1, -1, -1>(G, ph, fc, i, j, k, phi, K, p, c);
            Rc += corner_salt_out<0, -1, -1>(G, ph, fc, i, j, k, phi, K, p, c);
            Rc += corner_salt_out<-1, 0, -1>(G, ph, fc, i, j, k, phi, K, p, c);
            Rc += corner_salt_out<0, 0, -1>(G, ph, fc, i, j, k, phi, K, p, c);
            Rc += corner_salt_out<-1, -1, 0>(G, ph, fc, i, j, k, phi, K, p, c);
            Rc += corner_salt_out<0, -1, 0>(G, ph, fc, i, j, k, phi, K, p, c);
            Rc += corner_salt_out<-1, 0, 0>(G, ph, fc, i, j, k, phi, K, p, c);
            Rc += corner_salt_out<0, 0, 0>(G, ph, fc, i, j, k, phi, K, p, c);
            in = ph.dt * Rc;  // net salt flux out of this Dirichlet node
        }
    }
    const double t0 = block_sum(m0, red);
    const double t1 = block_sum(m1, red);
    const double t2 = block_sum(in, red);
    if (threadIdx.x == 0) {
        partial[((size_t)s * 3 + 0) * gridDim.x + blockIdx.x] = t0;
        partial[((size_t)s * 3 + 1) * gridDim.x + blockIdx.x] = t1;
        partial[((size_t)s * 3 + 2) * gridDim.x + blockIdx.x] = t2;
    }
}

void launch_mass_balance(const Grid& G, const Phys& ph, const uint8_t* bc, const double* phi,
                         const double* K, const double* p, const double* c,
                         const double* c_old, double* partial, int S, cudaStream_t st)
{
    count_launch(1);
    dim3 grid(nblocks(G.N), S);
    k_mass_balance<<<grid, kBS, 0, st>>>(G, ph, make_flux_const(G, ph), bc, phi, K, p, c,
                                         c_old, partial);
}

}  // namespace elder
