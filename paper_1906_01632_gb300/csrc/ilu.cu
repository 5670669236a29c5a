// ilu.cu -- multicolour block ILU_beta(0) smoother of the multigrid V-cycle
// (Section 5.1 names the smoother ILU_beta without defining it).
//
// Reading: the incomplete LU factorisation with 2x2 blocks, restricted to the
// 27-point block pattern of the level operator, in the multicolour node
// order: colour = (i&1) + 2(j&1) + 4(k&1), colours ascending.  Two nodes of
// one colour never share a cell, so every colour class is an independent set
// of the stencil: the rows of one colour are factored, and the triangular
// solves advance, in parallel, one launch per colour.  The factorisation is
// Gaussian elimination in IKJ form with every update of a block outside the
// pattern dropped; beta times the dropped block is subtracted from the row's
// diagonal block instead (beta = 0: block ILU(0); beta = 1: block modified
// ILU).  The operator is the interior one (Dirichlet rows and columns
// replaced by the identity), its diagonal block formed from the stored
// inverse Dinv exactly as the z-line factorisation forms it.
//
// Storage of the factors, per level and sample: F [27][N] in the multigrid
// storage type (slot q of row n the block of the neighbour at offset d, q =
// (dx+1) + 3(dy+1) + 9(dz+1): L where the neighbour's colour is smaller,
// U where it is larger) and Fd [N] in the solver type (the inverse of the
// pivot block U_nn).  The node axis of both is in colour-blocked order
// (IluLayout): a colour's rows are contiguous, so that the launch of one
// colour reads its factor rows at full coalescing.  The vectors keep the
// natural node order.
#include "kernels.h"

namespace elder {

namespace {

__device__ __forceinline__ bool on_(const int* mask, int stride, int s)
{
    return mask == nullptr || mask[(size_t)s * stride] != 0;
}

template <class T>
__device__ __forceinline__ B4<T> inv2_(const B4<T>& a)
{
    const T det = a.pp * a.cc - a.pc * a.cp;
    const T r = T(1) / det;
    return B4<T>{a.cc * r, -a.pc * r, -a.cp * r, a.pp * r};
}

template <class T>
__device__ __forceinline__ B4<T> mul2_(const B4<T>& a, const B4<T>& b)
{
    return B4<T>{fma(a.pp, b.pp, a.pc * b.cp), fma(a.pp, b.pc, a.pc * b.cc),
                 fma(a.cp, b.pp, a.cc * b.cp), fma(a.cp, b.pc, a.cc * b.cc)};
}

template <class T, class M>
__device__ __forceinline__ B4<T> load_blk(const B4<M>& q)
{
    return B4<T>{mg_load<T>(q.pp), mg_load<T>(q.pc), mg_load<T>(q.cp), mg_load<T>(q.cc)};
}

template <class T>
__device__ __forceinline__ B4<T> masked(B4<T> a, uint8_t row_bc, uint8_t col_bc)
{
    if (row_bc & BC_P) { a.pp = T(0); a.pc = T(0); }
    if (row_bc & BC_C) { a.cp = T(0); a.cc = T(0); }
    if (col_bc & BC_P) { a.pp = T(0); a.cp = T(0); }
    if (col_bc & BC_C) { a.pc = T(0); a.cc = T(0); }
    return a;
}

// axes along which the offset of slot q moves (bit 0 x, 1 y, 2 z): the
// neighbour's colour is the node's colour xor this
__host__ __device__ constexpr int slot_axes(int q)
{
    return ((q % 3) != 1 ? 1 : 0) | (((q / 3) % 3) != 1 ? 2 : 0) | ((q / 9) != 1 ? 4 : 0);
}

__device__ __forceinline__ bool inside(const Grid& G, int i, int j, int k)
{
    return i >= 0 && i <= G.nx && j >= 0 && j <= G.ny && k >= 0 && k <= G.nz;
}

// node (i, j, k) of thread t of colour c; false past the colour's last node
__device__ __forceinline__ bool colour_node(const Grid& G, const IluLayout& Lo, int c, int t,
                                            int& i, int& j, int& k)
{
    if (t >= Lo.off[c + 1] - Lo.off[c]) return false;
    const int cx = Lo.cnt_x[c & 1], cy = Lo.cnt_y[(c >> 1) & 1];
    const int ii = t % cx, r = t / cx;
    i = 2 * ii + (c & 1);
    j = 2 * (r % cy) + ((c >> 1) & 1);
    k = 2 * (r / cy) + ((c >> 2) & 1);
    return true;
}

// position of node (i, j, k) in the colour-blocked order
__device__ __forceinline__ int colour_pos(const IluLayout& Lo, int i, int j, int k)
{
    const int c = (i & 1) | ((j & 1) << 1) | ((k & 1) << 2);
    return Lo.off[c] + (i >> 1) + Lo.cnt_x[i & 1] * ((j >> 1) + Lo.cnt_y[j & 1] * (k >> 1));
}

// Factors of the rows of colour C.  Each thread eliminates its row in a
// register copy w: for the earlier colours cc = 0..C-1 in ascending order
// (the IKJ order: within one colour the neighbours do not interact), each
// neighbour k of colour cc turns w_k into L_ik = w_k U_kk^{-1} and subtracts
// L_ik U_kj from w_j for every neighbour j of k of a larger colour than
// cc (j in the row's pattern), or beta L_ik U_kj from the diagonal block
// (j outside it).  Rows of earlier colours are final: they were factored by
// earlier launches.
template <class T, class M, int C>
__global__ void __launch_bounds__(128)
    k_ilu_factor(Grid G, IluLayout Lo, const B4<M>* __restrict__ J,
                 const B4<T>* __restrict__ Dinv, const uint8_t* __restrict__ bc,
                 B4<M>* __restrict__ F, B4<T>* __restrict__ Fd, T beta, const int* mask,
                 int mstride)
{
    const int s = blockIdx.y;
    if (!on_(mask, mstride, s)) return;
    int i, j, k;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (!colour_node(G, Lo, C, t, i, j, k)) return;
    const int sy = G.nx + 1, sz = (G.nx + 1) * (G.ny + 1);
    const int n = i + sy * j + sz * k;
    const size_t on = (size_t)s * G.N;
    const B4<M>* Js = J + (size_t)s * 27 * G.N;
    B4<M>* Fs = F + (size_t)s * 27 * G.N;
    B4<T>* Fds = Fd + on;
    const uint8_t bn = bc[n];
    B4<T> w[27];
#pragma unroll
    for (int q = 0; q < 27; ++q) {
        const int dx = q % 3 - 1, dy = (q / 3) % 3 - 1, dz = q / 9 - 1;
        if (q == 13) {
            w[q] = inv2_(Dinv[on + n]);
        } else if (inside(G, i + dx, j + dy, k + dz)) {
            const int m = n + dx + dy * sy + dz * sz;
            w[q] = masked(load_blk<T, M>(Js[(size_t)q * G.N + n]), bn, bc[m]);
        } else {
            w[q] = B4<T>{T(0), T(0), T(0), T(0)};
        }
    }
    const int pn = Lo.off[C] + t;
    // Every load is issued unconditionally, so that the compiler can start
    // them ahead of the dependent arithmetic: a neighbour outside the grid
    // reads the row's own (not yet written) slots, and its terms are
    // selected away, never multiplied by 0 (the slots may hold any bits).
#pragma unroll
    for (int cc = 0; cc < C; ++cc) {
#pragma unroll
        for (int d = 0; d < 27; ++d) {
            if (d == 13 || slot_axes(d) != (C ^ cc)) continue;
            const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
            const bool okk = inside(G, i + dx, j + dy, k + dz);
            const int pk = okk ? colour_pos(Lo, i + dx, j + dy, k + dz) : pn;
            const B4<T> dk = Fds[pk];
            const B4<T> l = okk ? mul2_(w[d], dk) : B4<T>{T(0), T(0), T(0), T(0)};
            w[d] = l;
#pragma unroll
            for (int e = 0; e < 27; ++e) {
                if (e == 13 || (cc ^ slot_axes(e)) <= cc) continue;  // U part of row k
                const int ex = e % 3 - 1, ey = (e / 3) % 3 - 1, ez = e / 9 - 1;
                const int fx = dx + ex, fy = dy + ey, fz = dz + ez;
                const bool inpat = fx >= -1 && fx <= 1 && fy >= -1 && fy <= 1 &&
                                   fz >= -1 && fz <= 1;
                if (inpat) {
                    const bool ok = okk && inside(G, i + fx, j + fy, k + fz);
                    const B4<T> lu = mul2_(l, load_blk<T, M>(Fs[(size_t)e * G.N + pk]));
                    const int f = (fx + 1) + 3 * (fy + 1) + 9 * (fz + 1);
                    w[f].pp = ok ? w[f].pp - lu.pp : w[f].pp;
                    w[f].pc = ok ? w[f].pc - lu.pc : w[f].pc;
                    w[f].cp = ok ? w[f].cp - lu.cp : w[f].cp;
                    w[f].cc = ok ? w[f].cc - lu.cc : w[f].cc;
                } else if (beta != T(0) && okk && inside(G, i + fx, j + fy, k + fz)) {
                    // fill outside the pattern: beta times it onto the pivot
                    const B4<T> lu = mul2_(l, load_blk<T, M>(Fs[(size_t)e * G.N + pk]));
                    w[13].pp = fma(-beta, lu.pp, w[13].pp);
                    w[13].pc = fma(-beta, lu.pc, w[13].pc);
                    w[13].cp = fma(-beta, lu.cp, w[13].cp);
                    w[13].cc = fma(-beta, lu.cc, w[13].cc);
                }
            }
        }
    }
#pragma unroll
    for (int q = 0; q < 27; ++q) {
        if (q == 13) continue;
        Fs[(size_t)q * G.N + pn] =
            B4<M>{mg_store<M>(w[q].pp), mg_store<M>(w[q].pc), mg_store<M>(w[q].cp),
                  mg_store<M>(w[q].cc)};
    }
    Fds[pn] = inv2_(w[13]);
}

// One colour C of a triangular solve with the factors (the vector t holds the
// first solve's result for the processed rows, the second's after it):
//  PASS 0 (colours ascending): non-transposed L y = r, y_i = r_i - sum_lower
//    L_ik y_k; transposed U^T y = r, y_i = U_ii^{-T} (r_i - sum_lower U_ki^T
//    y_k).  r is read from src (b for a sweep from x = 0, else the masked
//    residual, in place in t).
//  PASS 1 (colours descending): non-transposed U z = y, z_i = U_ii^{-1} (y_i
//    - sum_upper U_ij z_j); transposed L^T z = y, z_i = y_i - sum_upper
//    L_ji^T z_j; then x_out = x + omega z (MODE 2) or omega z (MODE 1).
// "lower" / "upper": neighbours of smaller / larger colour, fixed at compile
// time by C.  The loads are unconditional (a neighbour outside the grid reads
// the node's own entries, and its term is selected away).
template <class T, class M, bool TRANS, int PASS, int MODE, int C>
__global__ void __launch_bounds__(kBS)
    k_ilu_pass(Grid G, IluLayout Lo, const B4<M>* __restrict__ F,
               const B4<T>* __restrict__ Fd, const uint8_t* __restrict__ bc, const V2<T>* src,
               V2<T>* tv, const V2<T>* x, V2<T>* xo, T omega, const int* mask, int mstride)
{
    const int s = blockIdx.y;
    if (!on_(mask, mstride, s)) return;
    int i, j, k;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (!colour_node(G, Lo, C, t, i, j, k)) return;
    const int sy = G.nx + 1, sz = (G.nx + 1) * (G.ny + 1);
    const int n = i + sy * j + sz * k;
    const size_t on = (size_t)s * G.N;
    const B4<M>* Fs = F + (size_t)s * 27 * G.N;
    const int pn = Lo.off[C] + t;
    const uint8_t bn = bc[n];
    T ap, ac;
    if (PASS == 0) {
        const V2<T> r = src[on + n];
        ap = (bn & BC_P) ? T(0) : r.p;
        ac = (bn & BC_C) ? T(0) : r.c;
    } else {
        const V2<T> y = tv[on + n];
        ap = y.p;
        ac = y.c;
    }
#pragma unroll
    for (int d = 0; d < 27; ++d) {
        if (d == 13) continue;
        const int cd = C ^ slot_axes(d);
        if (PASS == 0 ? cd > C : cd < C) continue;
        const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
        const bool ok = inside(G, i + dx, j + dy, k + dz);
        const V2<T> v = tv[on + (ok ? n + dx + dy * sy + dz * sz : n)];
        T np, nc;
        if (!TRANS) {
            const B4<T> b = load_blk<T, M>(Fs[(size_t)d * G.N + pn]);
            np = fma(-b.pp, v.p, fma(-b.pc, v.c, ap));
            nc = fma(-b.cp, v.p, fma(-b.cc, v.c, ac));
        } else {
            // row m's block of offset -d, transposed
            const int pm = ok ? colour_pos(Lo, i + dx, j + dy, k + dz) : pn;
            const B4<T> b = load_blk<T, M>(Fs[(size_t)(26 - d) * G.N + pm]);
            np = fma(-b.pp, v.p, fma(-b.cp, v.c, ap));
            nc = fma(-b.pc, v.p, fma(-b.cc, v.c, ac));
        }
        ap = ok ? np : ap;
        ac = ok ? nc : ac;
    }
    const bool pivot = (PASS == 0) == TRANS;
    if (pivot) {
        const B4<T> D = Fd[on + pn];
        const T zp = !TRANS ? fma(D.pp, ap, D.pc * ac) : fma(D.pp, ap, D.cp * ac);
        const T zc = !TRANS ? fma(D.cp, ap, D.cc * ac) : fma(D.pc, ap, D.cc * ac);
        ap = zp;
        ac = zc;
    }
    tv[on + n] = V2<T>{ap, ac};
    if (PASS == 1) {
        V2<T> xn{T(0), T(0)};
        if (MODE == 2) xn = x[on + n];
        T op = fma(omega, ap, xn.p), oc = fma(omega, ac, xn.c);
        if (bn & BC_P) op = T(0);
        if (bn & BC_C) oc = T(0);
        xo[on + n] = V2<T>{op, oc};
    }
}

}  // namespace

IluLayout ilu_layout(const Grid& G)
{
    IluLayout Lo{};
    Lo.cnt_x[0] = G.nx / 2 + 1;
    Lo.cnt_x[1] = (G.nx + 1) / 2;
    Lo.cnt_y[0] = G.ny / 2 + 1;
    Lo.cnt_y[1] = (G.ny + 1) / 2;
    const int cz[2] = {G.nz / 2 + 1, (G.nz + 1) / 2};
    Lo.off[0] = 0;
    for (int c = 0; c < 8; ++c)
        Lo.off[c + 1] = Lo.off[c] + Lo.cnt_x[c & 1] * Lo.cnt_y[(c >> 1) & 1] * cz[(c >> 2) & 1];
    return Lo;
}

template <class T, class M>
void launch_ilu_factor(const Grid& G, const B4<M>* J, const B4<T>* Dinv, const uint8_t* bc,
                       B4<M>* F, B4<T>* Fd, double beta, const int* mask, int mstride, int S,
                       cudaStream_t st)
{
    const IluLayout Lo = ilu_layout(G);
    for (int c = 0; c < 8; ++c) {
        count_launch(1);
        dim3 grid(nblocks(Lo.off[c + 1] - Lo.off[c], 128), S);
#define ELDER_ILUF(CC)                                                                  \
    case CC:                                                                            \
        k_ilu_factor<T, M, CC><<<grid, 128, 0, st>>>(G, Lo, J, Dinv, bc, F, Fd, T(beta), \
                                                     mask, mstride);                    \
        break;
        switch (c) {
            ELDER_ILUF(0) ELDER_ILUF(1) ELDER_ILUF(2) ELDER_ILUF(3)
            ELDER_ILUF(4) ELDER_ILUF(5) ELDER_ILUF(6) ELDER_ILUF(7)
        }
#undef ELDER_ILUF
    }
}

template <class T, class M>
void launch_ilu_apply(const Grid& G, const B4<M>* F, const B4<T>* Fd, const uint8_t* bc,
                      const V2<T>* r, V2<T>* t, const V2<T>* x, V2<T>* xo, double omega,
                      int trans, int mode, const int* mask, int mstride, int S, cudaStream_t st,
                      int bs)
{
    const IluLayout Lo = ilu_layout(G);
    const T w = T(omega);
    for (int q = 0; q < 16; ++q) {
        const int pass = q < 8 ? 0 : 1;
        const int c = pass == 0 ? q : 15 - q;
        count_launch(1);
        dim3 grid(nblocks(Lo.off[c + 1] - Lo.off[c], bs), S);
        const V2<T>* src = pass == 0 ? r : nullptr;
#define ELDER_ILUP(TR, PA, MO, CC)                                                            \
    case CC:                                                                                  \
        k_ilu_pass<T, M, TR, PA, MO, CC><<<grid, bs, 0, st>>>(G, Lo, F, Fd, bc, src, t, x, xo, w, \
                                                              mask, mstride);                 \
        break;
#define ELDER_ILUP_C(TR, PA, MO)                                                              \
    switch (c) {                                                                              \
        ELDER_ILUP(TR, PA, MO, 0) ELDER_ILUP(TR, PA, MO, 1) ELDER_ILUP(TR, PA, MO, 2)         \
        ELDER_ILUP(TR, PA, MO, 3) ELDER_ILUP(TR, PA, MO, 4) ELDER_ILUP(TR, PA, MO, 5)         \
        ELDER_ILUP(TR, PA, MO, 6) ELDER_ILUP(TR, PA, MO, 7)                                   \
    }
        if (pass == 0) {
            if (trans) { ELDER_ILUP_C(true, 0, 1) }
            else { ELDER_ILUP_C(false, 0, 1) }
        } else if (mode == 1) {
            if (trans) { ELDER_ILUP_C(true, 1, 1) }
            else { ELDER_ILUP_C(false, 1, 1) }
        } else {
            if (trans) { ELDER_ILUP_C(true, 1, 2) }
            else { ELDER_ILUP_C(false, 1, 2) }
        }
#undef ELDER_ILUP_C
#undef ELDER_ILUP
    }
}

#define ELDER_INST_ILU(T)                                                                  \
    template void launch_ilu_factor<T, MgType<T>::type>(                                   \
        const Grid&, const B4<MgType<T>::type>*, const B4<T>*, const uint8_t*,             \
        B4<MgType<T>::type>*, B4<T>*, double, const int*, int, int, cudaStream_t);         \
    template void launch_ilu_apply<T, MgType<T>::type>(                                    \
        const Grid&, const B4<MgType<T>::type>*, const B4<T>*, const uint8_t*,             \
        const V2<T>*, V2<T>*, const V2<T>*, V2<T>*, double, int, int, const int*, int, int, \
        cudaStream_t, int);
ELDER_INST_ILU(double)
ELDER_INST_ILU(float)
#undef ELDER_INST_ILU

}  // namespace elder
