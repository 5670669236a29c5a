// linalg.cu -- batched linear algebra of the Newton/BiCGStab/multigrid solve
// (Section 2.3 and Section 5.1): 27-point 2x2-block stencil products,
// damped block-Jacobi smoothing, full-weighting restriction / trilinear
// prolongation on the vertex-centred 2:1 hierarchy, the dense coarse solve,
// the BiCGStab vector updates (van der Vorst; Templates, Sec. 2.3.8) with
// FP64 inner products, and the Newton line-search bookkeeping.
//
// Every node kernel runs one thread per node with grid.y = sample and skips
// samples whose mask flag is 0 (converged or failed samples).  Reductions are
// two-stage and deterministic: per-block partials [S][2][nblk], then one
// block per sample sums them in a fixed order.
//
// Solver vectors hold the unknowns of the interior system: Dirichlet
// components are kept at 0 by masking every kernel's output.
#include <type_traits>
#include <cuda_pipeline.h>

#include "kernels.h"

namespace elder {

__device__ __forceinline__ bool on(const int* mask, int stride, int s)
{
    return mask == nullptr || mask[(size_t)s * stride] != 0;
}

static_assert(sizeof(KScal) % sizeof(int) == 0, "KScal layout");
static_assert(sizeof(NScal) % sizeof(int) == 0, "NScal layout");

// One neighbour term of the 27-point product.  The loads are unconditional
// (a missing neighbour reads node n itself and its term is selected to 0),
// so a thread issues all 54 loads of its row before the first use: the
// stencil kernels are memory-latency bound and need that parallelism.
template <class T, bool TRANS, class M>
__device__ __forceinline__ void stencil_term(const Grid& G, const B4<M>* __restrict__ J,
                                             const V2<T>* __restrict__ x, int n, int m,
                                             int slot, int tslot, bool ok, T& yp, T& yc,
                                             B4<M>* raw = nullptr)
{
    const int mm = ok ? m : n;
    const V2<T> xv = x[mm];
    const B4<M> b = !TRANS ? J[(size_t)slot * G.N + n] : J[(size_t)tslot * G.N + mm];
    if (raw) *raw = b;
    const T pp = ok ? mg_load<T>(b.pp) : T(0), pc = ok ? mg_load<T>(b.pc) : T(0);
    const T cp = ok ? mg_load<T>(b.cp) : T(0), cc = ok ? mg_load<T>(b.cc) : T(0);
    // explicit fused multiply-adds: every instantiation (one or two samples
    // per CTA) rounds the same way
    if (!TRANS) {
        yp = fma(pp, xv.p, fma(pc, xv.c, yp));
        yc = fma(cp, xv.p, fma(cc, xv.c, yc));
    } else {
        yp = fma(pp, xv.p, fma(cp, xv.c, yp));
        yc = fma(pc, xv.p, fma(cc, xv.c, yc));
    }
}

// y_n = sum over the 27 neighbours of the 2x2 block times x (or the
// transposed product, reading row m's block of offset -d).
template <class T, bool TRANS, class M>
__device__ __forceinline__ void stencil_apply(const Grid& G,
                                              const B4<M>* __restrict__ J,
                                              const V2<T>* __restrict__ x,
                                              int n, int i, int j, int k,
                                              T& yp, T& yc)
{
    const int sy = G.nx + 1, sz = (G.nx + 1) * (G.ny + 1);
    yp = T(0);
    yc = T(0);
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                const bool ok = (dx < 0 ? i > 0 : (dx > 0 ? i < G.nx : true)) &&
                                (dy < 0 ? j > 0 : (dy > 0 ? j < G.ny : true)) &&
                                (dz < 0 ? k > 0 : (dz > 0 ? k < G.nz : true));
                stencil_term<T, TRANS, M>(G, J, x, n, n + dx + dy * sy + dz * sz,
                                          slot27(dx, dy, dz), slot27(-dx, -dy, -dz), ok, yp, yc);
            }
}

// ---------------------------------------------------------------------------
// SpMV with fused inner products
// ---------------------------------------------------------------------------

template <class T, bool TRANS, int MODE>
__global__ void __launch_bounds__(kMaxBS)
    k_spmv(Grid G, const B4<T>* __restrict__ J, const uint8_t* __restrict__ bc,
           const V2<T>* __restrict__ x, V2<T>* __restrict__ y,
           const V2<T>* __restrict__ a, double* __restrict__ partial,
           const int* mask, int mstride)
{
    const int s = blockIdx.y;
    if (!on(mask, mstride, s)) return;
    const size_t on_ = (size_t)s * G.N;
    J += (size_t)s * 27 * G.N;
    x += on_;
    y += on_;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    double d0 = 0.0, d1 = 0.0;
    if (n < G.N) {
        int i, j, k;
        node_ijk(G, n, i, j, k);
        T yp, yc;
        stencil_apply<T, TRANS, T>(G, J, x, n, i, j, k, yp, yc);
        if (MODE != 3) {
            const uint8_t b = bc[n];
            if (b & BC_P) yp = T(0);
            if (b & BC_C) yc = T(0);
        }
        y[n] = V2<T>{yp, yc};
        if (MODE == 1 || MODE == 2) {
            const V2<T> av = a[on_ + n];
            d0 = dot2(av.p, av.c, yp, yc);
        }
        if (MODE == 2) d1 = dot2(yp, yc, yp, yc);
    }
    // One partial per warp of 32 nodes, so the sums do not depend on the
    // (tuned) block size: the inner products are bitwise reproducible.
    if (MODE == 1 || MODE == 2) {
        const int W = (G.N + 31) >> 5;
        const int wg = n >> 5;
        const double t0 = warp_sum(d0);
        const double t1 = (MODE == 2) ? warp_sum(d1) : 0.0;
        if ((threadIdx.x & 31) == 0 && wg < W) {
            partial[((size_t)s * 2 + 0) * W + wg] = t0;
            if (MODE == 2) partial[((size_t)s * 2 + 1) * W + wg] = t1;
        }
    }
}

template <class T>
void launch_spmv(const Grid& G, const B4<T>* J, const uint8_t* bc,
                 const V2<T>* x, V2<T>* y, int trans, int mode,
                 const V2<T>* a, double* partial, const int* mask,
                 int mstride, int S, cudaStream_t st, int bs)
{
    count_launch(1);
    dim3 grid(nblocks(G.N, bs), S);
#define ELDER_SPMV(TR, MO) \
    k_spmv<T, TR, MO><<<grid, bs, 0, st>>>(G, J, bc, x, y, a, partial, mask, mstride)
    if (!trans) {
        if (mode == 0) ELDER_SPMV(false, 0);
        else if (mode == 1) ELDER_SPMV(false, 1);
        else if (mode == 2) ELDER_SPMV(false, 2);
        else ELDER_SPMV(false, 3);
    } else {
        if (mode == 0) ELDER_SPMV(true, 0);
        else if (mode == 1) ELDER_SPMV(true, 1);
        else if (mode == 2) ELDER_SPMV(true, 2);
        else ELDER_SPMV(true, 3);
    }
#undef ELDER_SPMV
}

// ---------------------------------------------------------------------------
// multigrid: damped block-Jacobi smoother, residual, transfers, coarse solve
// ---------------------------------------------------------------------------

template <class T, class M, bool TRANS, bool ZEROX>
__global__ void __launch_bounds__(kMaxBS)
    k_smooth(Grid G, const B4<M>* __restrict__ J, const B4<T>* __restrict__ Dinv,
             const uint8_t* __restrict__ bc, const V2<T>* __restrict__ b,
             const V2<T>* __restrict__ x, V2<T>* __restrict__ xo, T omega,
             const int* mask, int mstride)
{
    const int s = blockIdx.y;
    if (!on(mask, mstride, s)) return;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= G.N) return;
    const size_t on_ = (size_t)s * G.N;
    const V2<T> bv = b[on_ + n];
    T rp = bv.p, rc = bv.c;
    V2<T> xn{T(0), T(0)};
    if (!ZEROX) {
        int i, j, k;
        node_ijk(G, n, i, j, k);
        T yp, yc;
        stencil_apply<T, TRANS, M>(G, J + (size_t)s * 27 * G.N, x + on_, n, i, j, k, yp, yc);
        rp -= yp;
        rc -= yc;
        xn = x[on_ + n];
    }
    const B4<T> d = Dinv[on_ + n];
    T zp, zc;
    if (!TRANS) { zp = d.pp * rp + d.pc * rc; zc = d.cp * rp + d.cc * rc; }
    else { zp = d.pp * rp + d.cp * rc; zc = d.pc * rp + d.cc * rc; }
    T op = xn.p + omega * zp, oc = xn.c + omega * zc;
    const uint8_t m = bc[n];
    if (m & BC_P) op = T(0);
    if (m & BC_C) oc = T(0);
    xo[on_ + n] = V2<T>{op, oc};
}

template <class T, class M>
void launch_smooth(const Grid& G, const B4<M>* J, const B4<T>* Dinv,
                   const uint8_t* bc, const V2<T>* b, const V2<T>* x,
                   V2<T>* xo, double omega, int trans, const int* mask,
                   int mstride, int S, cudaStream_t st, int bs)
{
    count_launch(1);
    dim3 grid(nblocks(G.N, bs), S);
    const T w = T(omega);
    if (x == nullptr) {
        if (trans) k_smooth<T, M, true, true><<<grid, bs, 0, st>>>(G, J, Dinv, bc, b, x, xo, w, mask, mstride);
        else k_smooth<T, M, false, true><<<grid, bs, 0, st>>>(G, J, Dinv, bc, b, x, xo, w, mask, mstride);
    } else {
        if (trans) k_smooth<T, M, true, false><<<grid, bs, 0, st>>>(G, J, Dinv, bc, b, x, xo, w, mask, mstride);
        else k_smooth<T, M, false, false><<<grid, bs, 0, st>>>(G, J, Dinv, bc, b, x, xo, w, mask, mstride);
    }
}

// ---------------------------------------------------------------------------
// z-line block Jacobi: x_out = x + omega L^{-1} (b - A x), L the block
// tridiagonal part of A along each vertical grid line (2x2 blocks of the
// offsets (0,0,-1), (0,0,0), (0,0,+1)).  One thread solves one line by the
// block Thomas algorithm.  It keeps the node-local pressure/salt coupling and
// the vertical (gravity) coupling implicit: next to a steep salt front on a
// rough permeability field the 2x2 diagonal blocks become nearly singular and
// point block Jacobi diverges locally, while the line solve stays stable.
// The diagonal block is recovered from Dinv (the inverse of the interior-
// masked block, kept in T precision); the off-diagonal line blocks come from
// the stored matrix, masked to the interior operator.
// ---------------------------------------------------------------------------

template <class T>
__device__ __forceinline__ B4<T> inv2(const B4<T>& a)
{
    const T det = a.pp * a.cc - a.pc * a.cp;
    const T r = T(1) / det;
    return B4<T>{a.cc * r, -a.pc * r, -a.cp * r, a.pp * r};
}

template <class T>
__device__ __forceinline__ B4<T> mul2(const B4<T>& a, const B4<T>& b)
{
    return B4<T>{a.pp * b.pp + a.pc * b.cp, a.pp * b.pc + a.pc * b.cc,
                 a.cp * b.pp + a.cc * b.cp, a.cp * b.pc + a.cc * b.cc};
}

// Raw (unmasked) line block of row n for the vertical offset dz = -1 or +1:
// the block of slot (0,0,dz) at row n, or for the transposed operator the
// block of slot (0,0,-dz) at row n + dz*sz read transposed.
template <class T, class M, bool TRANS>
__device__ __forceinline__ B4<T> raw_line_block(const B4<M>& q)
{
    if (!TRANS) return B4<T>{mg_load<T>(q.pp), mg_load<T>(q.pc), mg_load<T>(q.cp), mg_load<T>(q.cc)};
    return B4<T>{mg_load<T>(q.pp), mg_load<T>(q.cp), mg_load<T>(q.pc), mg_load<T>(q.cc)};
}

template <class T>
__device__ __forceinline__ B4<T> mask_block(B4<T> a, uint8_t row_bc, uint8_t col_bc)
{
    if (row_bc & BC_P) { a.pp = T(0); a.pc = T(0); }
    if (row_bc & BC_C) { a.cp = T(0); a.cc = T(0); }
    if (col_bc & BC_P) { a.pp = T(0); a.cp = T(0); }
    if (col_bc & BC_C) { a.pc = T(0); a.cc = T(0); }
    return a;
}

// Depth of the per-thread ring of line inputs in shared memory.
constexpr int kZlRing = 4;

// Asynchronous copy of one element (8, 16 or 32 bytes, naturally aligned)
// from global to shared memory.
template <class X>
__device__ __forceinline__ void async_copy(X* dst, const X* src)
{
    static_assert(sizeof(X) % 8 == 0 && sizeof(X) <= 32, "element size");
    constexpr int step = (sizeof(X) % 16 == 0) ? 16 : 8;
#pragma unroll
    for (int o = 0; o < (int)sizeof(X); o += step)
        __pipeline_memcpy_async(reinterpret_cast<char*>(dst) + o,
                                reinterpret_cast<const char*>(src) + o, step);
}

// The Thomas factors C_k = M_k^{-1} U_k and g_k of the forward sweep live in
// shared memory, [k][thread], for the backward sweep; the forward recursion
// carries C_{k-1} and g_{k-1} in registers.  The inputs of node k (rhs,
// inverse diagonal block, the two vertical line blocks) reach a per-thread
// ring of kZlRing slots in shared memory by asynchronous copies issued
// kZlRing nodes ahead: each thread walks its line serially, and the ring
// keeps several nodes' loads in flight per thread.
// MODE 1: x = 0, x_out = omega L^{-1} b;
// MODE 2: b holds the residual b - A x (masked), x_out = x + omega L^{-1} b.
// A sweep from a nonzero x is the multigrid residual kernel (all nodes in
// parallel, at stream rate) followed by MODE 2: folding the 27-point
// residual into the line kernel runs at a third of the bandwidth, because
// each thread walks its line serially and few warps fit an SM.
template <class T, class M, bool TRANS, int MODE>
__global__ void __launch_bounds__(kLineBS)
    k_smooth_zline(Grid G, const B4<M>* __restrict__ J, const B4<T>* __restrict__ Dinv,
                   const uint8_t* __restrict__ bc, const V2<T>* __restrict__ b,
                   const V2<T>* __restrict__ x, V2<T>* __restrict__ xo, T omega,
                   const int* mask, int mstride)
{
    extern __shared__ __align__(16) unsigned char zl_smem[];
    const int s = blockIdx.y;
    if (!on(mask, mstride, s)) return;
    const int bsz = blockDim.x, tx = threadIdx.x;
    B4<T>* Cs = reinterpret_cast<B4<T>*>(zl_smem);                  // [nz][bsz]
    V2<T>* gs = reinterpret_cast<V2<T>*>(Cs + (size_t)G.nz * bsz);   // [nz+1][bsz]
    B4<T>* Rdi = reinterpret_cast<B4<T>*>(gs + (size_t)(G.nz + 1) * bsz);  // [ring][bsz]
    V2<T>* Rb = reinterpret_cast<V2<T>*>(Rdi + (size_t)kZlRing * bsz);
    B4<M>* RL = reinterpret_cast<B4<M>*>(Rb + (size_t)kZlRing * bsz);
    B4<M>* RU = RL + (size_t)kZlRing * bsz;
    const int sz = (G.nx + 1) * (G.ny + 1);
    const int col = blockIdx.x * bsz + tx;
    if (col >= sz) return;
    const size_t on_ = (size_t)s * G.N;
    const B4<M>* Js = J + (size_t)s * 27 * G.N;
    const V2<T>* xs = (MODE == 1) ? nullptr : x + on_;
    // copies of node k into ring slot k % kZlRing (one commit group per node,
    // empty past the end of the line)
    auto issue = [&](int k) {
        if (k <= G.nz) {
            const int n = col + k * sz;
            const int q = (k % kZlRing) * bsz + tx;
            async_copy(Rb + q, b + on_ + n);
            async_copy(Rdi + q, Dinv + on_ + n);
            if (k > 0)
                async_copy(RL + q, !TRANS ? Js + (size_t)slot27(0, 0, -1) * G.N + n
                                          : Js + (size_t)slot27(0, 0, 1) * G.N + n - sz);
            if (k < G.nz)
                async_copy(RU + q, !TRANS ? Js + (size_t)slot27(0, 0, 1) * G.N + n
                                          : Js + (size_t)slot27(0, 0, -1) * G.N + n + sz);
        }
        __pipeline_commit();
    };
#pragma unroll
    for (int k = 0; k < kZlRing; ++k) issue(k);
    B4<T> Cp{T(0), T(0), T(0), T(0)};
    V2<T> gp{T(0), T(0)};
    uint8_t bc_prev = 0;
    uint8_t mk = bc[col];
    uint8_t bnext = (G.nz >= 1) ? bc[col + sz] : uint8_t(0);
    for (int k = 0; k <= G.nz; ++k) {
        const uint8_t bc_next = bnext;
        bnext = (k + 2 <= G.nz) ? bc[col + (k + 2) * sz] : uint8_t(0);
        // node k's group is complete once at most kZlRing - 1 newer ones pend
        __pipeline_wait_prior(kZlRing - 1);
        const int q = (k % kZlRing) * bsz + tx;
        const V2<T> bv = Rb[q];
        B4<T> di = Rdi[q];
        B4<M> qL{}, qU{};
        if (k > 0) qL = RL[q];
        if (k < G.nz) qU = RU[q];
        T rp = bv.p, rc = bv.c;
        if (mk & BC_P) rp = T(0);
        if (mk & BC_C) rc = T(0);
        if (TRANS) di = B4<T>{di.pp, di.cp, di.pc, di.cc};
        B4<T> Mk = inv2(di);
        if (k > 0) {
            const B4<T> L = mask_block(raw_line_block<T, M, TRANS>(qL), mk, bc_prev);
            const B4<T> LC = mul2(L, Cp);
            Mk.pp -= LC.pp; Mk.pc -= LC.pc; Mk.cp -= LC.cp; Mk.cc -= LC.cc;
            rp -= L.pp * gp.p + L.pc * gp.c;
            rc -= L.cp * gp.p + L.cc * gp.c;
        }
        const B4<T> Mi = inv2(Mk);
        if (k < G.nz) {
            const B4<T> U = mask_block(raw_line_block<T, M, TRANS>(qU), mk, bc_next);
            Cp = mul2(Mi, U);
            Cs[(size_t)k * bsz + tx] = Cp;
        }
        gp = V2<T>{Mi.pp * rp + Mi.pc * rc, Mi.cp * rp + Mi.cc * rc};
        gs[(size_t)k * bsz + tx] = gp;
        bc_prev = mk;
        mk = bc_next;
        // every value of slot q is in registers and used above: refill it
        issue(k + kZlRing);
    }
    __pipeline_wait_prior(0);
    V2<T> d = gp;
    for (int k = G.nz;; --k) {
        const int n = col + k * sz;
        if (k < G.nz) {
            const B4<T> C = Cs[(size_t)k * bsz + tx];
            const V2<T> g = gs[(size_t)k * bsz + tx];
            d = V2<T>{g.p - (C.pp * d.p + C.pc * d.c), g.c - (C.cp * d.p + C.cc * d.c)};
        }
        V2<T> xn{T(0), T(0)};
        if (MODE != 1) xn = xs[n];
        T op = xn.p + omega * d.p, oc = xn.c + omega * d.c;
        const uint8_t m = bc[n];
        if (m & BC_P) op = T(0);
        if (m & BC_C) oc = T(0);
        xo[on_ + n] = V2<T>{op, oc};
        if (k == 0) break;
    }
}

// Threads per block of the z-line sweep: as many as fit the per-thread
// Thomas storage and input ring in 96 KiB of shared memory (at least one
// warp).
template <class T, class M>
inline int zline_block(const Grid& G, size_t* smem)
{
    const size_t per = (size_t)G.nz * sizeof(B4<T>) + (size_t)(G.nz + 1) * sizeof(V2<T>) +
                       (size_t)kZlRing * (sizeof(B4<T>) + sizeof(V2<T>) + 2 * sizeof(B4<M>));
    int bs = (int)std::min<size_t>(kLineBS, (96 * 1024 / per) / 32 * 32);
    if (bs < 32) bs = 32;
    *smem = per * bs;
    return bs;
}

template <class T, class M>
void launch_smooth_zline(const Grid& G, const B4<M>* J, const B4<T>* Dinv, const uint8_t* bc,
                         const V2<T>* b, const V2<T>* x, V2<T>* xo, double omega, int trans,
                         const int* mask, int mstride, int S, cudaStream_t st, int mode)
{
    if (G.nz + 1 > kMaxLine) return;  // callers check the line limit first
    count_launch(1);
    size_t smem = 0;
    const int bs = zline_block<T, M>(G, &smem);
    dim3 grid(nblocks((G.nx + 1) * (G.ny + 1), bs), S);
    const T w = T(omega);
#define ELDER_ZL(TR, MO)                                                                       \
    do {                                                                                       \
        static bool attr_set = false;                                                          \
        if (!attr_set) {                                                                       \
            cudaFuncSetAttribute(k_smooth_zline<T, M, TR, MO>,                                 \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);     \
            attr_set = true;                                                                   \
        }                                                                                      \
        k_smooth_zline<T, M, TR, MO><<<grid, bs, smem, st>>>(G, J, Dinv, bc, b, x, xo, w, mask, \
                                                             mstride);                         \
    } while (0)
    if (mode == 1) {
        if (trans) ELDER_ZL(true, 1);
        else ELDER_ZL(false, 1);
    } else {
        if (trans) ELDER_ZL(true, 2);
        else ELDER_ZL(false, 2);
    }
#undef ELDER_ZL
}

// Block-LU factors of the vertical lines of a level's operator, once per
// assembly: for node k of a line, with M_0 = D_0 and M_k = D_k - L_k C_{k-1},
// zMi = M_k^{-1} and zC = C_k = M_k^{-1} U_k (D the diagonal block, formed
// as the inverse of the stored inverse Dinv exactly as the line sweep of
// k_smooth_zline does; L, U the masked vertical line blocks).  Each line
// sweep then only substitutes: the forward elimination and the inversions
// leave the per-sweep work.
template <class T, class M>
__global__ void __launch_bounds__(kBS)
    k_zline_factor(Grid G, const B4<M>* __restrict__ J, const B4<T>* __restrict__ Dinv,
                   const uint8_t* __restrict__ bc, B4<T>* __restrict__ zMi,
                   B4<T>* __restrict__ zC, const int* mask, int mstride)
{
    const int s = blockIdx.y;
    if (!on(mask, mstride, s)) return;
    const int sz = (G.nx + 1) * (G.ny + 1);
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= sz) return;
    const size_t on_ = (size_t)s * G.N;
    const B4<M>* Js = J + (size_t)s * 27 * G.N;
    const B4<M>* Jl = Js + (size_t)slot27(0, 0, -1) * G.N;
    const B4<M>* Ju = Js + (size_t)slot27(0, 0, 1) * G.N;
    B4<T> Cp{T(0), T(0), T(0), T(0)};
    uint8_t bc_prev = 0;
    for (int k = 0; k <= G.nz; ++k) {
        const int n = col + k * sz;
        const uint8_t mk = bc[n];
        B4<T> Mk = inv2(Dinv[on_ + n]);
        if (k > 0) {
            const B4<T> L = mask_block(raw_line_block<T, M, false>(Jl[n]), mk, bc_prev);
            const B4<T> LC = mul2(L, Cp);
            Mk.pp -= LC.pp; Mk.pc -= LC.pc; Mk.cp -= LC.cp; Mk.cc -= LC.cc;
        }
        const B4<T> Mi = inv2(Mk);
        zMi[on_ + n] = Mi;
        if (k < G.nz) {
            const uint8_t bn = bc[n + sz];
            const B4<T> U = mask_block(raw_line_block<T, M, false>(Ju[n]), mk, bn);
            Cp = mul2(Mi, U);
            zC[on_ + n] = Cp;
        }
        bc_prev = mk;
    }
}

template <class T, class M>
void launch_zline_factor(const Grid& G, const B4<M>* J, const B4<T>* Dinv, const uint8_t* bc,
                         B4<T>* zMi, B4<T>* zC, const int* mask, int mstride, int S,
                         cudaStream_t st)
{
    count_launch(1);
    dim3 grid(nblocks((G.nx + 1) * (G.ny + 1)), S);
    k_zline_factor<T, M><<<grid, kBS, 0, st>>>(G, J, Dinv, bc, zMi, zC, mask, mstride);
}

// One damped z-line sweep with the factors of k_zline_factor (the
// non-transposed operator): forward substitution g_k = zMi_k (r_k - L_k
// g_{k-1}), g kept in x_out, then back substitution d_k = g_k - zC_k d_{k+1}
// and x_out = x + omega d (x = 0 in MODE 1; in MODE 2 r is the masked
// residual b - A x).  One thread per line of SPC samples: the SPC
// recursions are independent, so their steps overlap (the autotuner picks
// SPC with the block size); the loads of a node do not depend on the
// recursion, so unrolled iterations keep several nodes in flight.  An
// inactive sample's line is read as sample s0's and not written.
template <class T, class M, int MODE, int SPC>
__global__ void __launch_bounds__(kBS)
    k_zline_apply(Grid G, const B4<M>* __restrict__ J, const B4<T>* __restrict__ zMi,
                  const B4<T>* __restrict__ zC, const uint8_t* __restrict__ bc,
                  const V2<T>* __restrict__ r, const V2<T>* __restrict__ x, V2<T>* xo, T omega,
                  const int* mask, int mstride, int S)
{
    const int s0 = blockIdx.y * SPC;
    bool act[SPC];
    bool any = false;
#pragma unroll
    for (int q = 0; q < SPC; ++q) {
        act[q] = s0 + q < S && on(mask, mstride, s0 + q);
        any = any || act[q];
    }
    if (!any) return;
    const int sz = (G.nx + 1) * (G.ny + 1);
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= sz) return;
    size_t on_[SPC];
#pragma unroll
    for (int q = 0; q < SPC; ++q) on_[q] = (size_t)(act[q] ? s0 + q : s0) * G.N;
    const size_t jl = (size_t)slot27(0, 0, -1) * G.N;
    V2<T> gp[SPC];
#pragma unroll
    for (int q = 0; q < SPC; ++q) gp[q] = V2<T>{T(0), T(0)};
    uint8_t bc_prev = 0;
#pragma unroll 4
    for (int k = 0; k <= G.nz; ++k) {
        const int n = col + k * sz;
        const uint8_t mk = bc[n];
#pragma unroll
        for (int q = 0; q < SPC; ++q) {
            const V2<T> bv = r[on_[q] + n];
            const B4<M> qL = J[on_[q] * 27 + jl + (k > 0 ? n : col)];
            const B4<T> Mi = zMi[on_[q] + n];
            T rp = (mk & BC_P) ? T(0) : bv.p;
            T rc = (mk & BC_C) ? T(0) : bv.c;
            if (k > 0) {
                const B4<T> L = mask_block(raw_line_block<T, M, false>(qL), mk, bc_prev);
                rp = fma(-L.pp, gp[q].p, fma(-L.pc, gp[q].c, rp));
                rc = fma(-L.cp, gp[q].p, fma(-L.cc, gp[q].c, rc));
            }
            gp[q] = V2<T>{fma(Mi.pp, rp, Mi.pc * rc), fma(Mi.cp, rp, Mi.cc * rc)};
            if (act[q]) xo[on_[q] + n] = gp[q];
        }
        bc_prev = mk;
    }
    V2<T> d[SPC];
#pragma unroll
    for (int q = 0; q < SPC; ++q) d[q] = gp[q];
#pragma unroll 4
    for (int k = G.nz; k >= 0; --k) {
        const int n = col + k * sz;
        const uint8_t m = bc[n];
#pragma unroll
        for (int q = 0; q < SPC; ++q) {
            if (!act[q]) continue;
            if (k < G.nz) {
                const B4<T> C = zC[on_[q] + n];
                const V2<T> g = xo[on_[q] + n];
                d[q] = V2<T>{fma(-C.pp, d[q].p, fma(-C.pc, d[q].c, g.p)),
                             fma(-C.cp, d[q].p, fma(-C.cc, d[q].c, g.c))};
            }
            V2<T> xn{T(0), T(0)};
            if (MODE != 1) xn = x[on_[q] + n];
            T op = fma(omega, d[q].p, xn.p), oc = fma(omega, d[q].c, xn.c);
            if (m & BC_P) op = T(0);
            if (m & BC_C) oc = T(0);
            xo[on_[q] + n] = V2<T>{op, oc};
        }
    }
}

template <class T, class M>
void launch_zline_apply(const Grid& G, const B4<M>* J, const B4<T>* zMi, const B4<T>* zC,
                        const uint8_t* bc, const V2<T>* r, const V2<T>* x, V2<T>* xo,
                        double omega, const int* mask, int mstride, int S, cudaStream_t st,
                        int mode, int bs, int spc)
{
    count_launch(1);
    dim3 grid(nblocks((G.nx + 1) * (G.ny + 1), bs), (S + spc - 1) / spc);
#define ELDER_ZLA(MO, SP)                                                                      \
    k_zline_apply<T, M, MO, SP><<<grid, bs, 0, st>>>(G, J, zMi, zC, bc, r, x, xo, T(omega),   \
                                                     mask, mstride, S)
    if (mode == 1) {
        if (spc == 2) ELDER_ZLA(1, 2);
        else ELDER_ZLA(1, 1);
    } else {
        if (spc == 2) ELDER_ZLA(2, 2);
        else ELDER_ZLA(2, 1);
    }
#undef ELDER_ZLA
}

// SPC samples per CTA: a thread forms the residual of its node in SPC
// samples, whose loads are independent (more loads in flight per thread at
// the price of registers); the autotuner picks SPC with the block size.  The
// loads of an inactive sample read sample s0's rows and its result is not
// stored.  At SPC = 1, at most 32 registers: every warp slot of an SM can
// then hold a warp, which this latency-bound stencil needs (at 34 a quarter
// stayed empty).
template <class T, class M, bool TRANS, int SPC>
__global__ void __launch_bounds__(kMaxBS, (2048 / kMaxBS) / SPC)
    k_mg_residual(Grid G, const B4<M>* __restrict__ J, const uint8_t* __restrict__ bc,
                  const V2<T>* __restrict__ b, const V2<T>* __restrict__ x,
                  V2<T>* __restrict__ r, const int* mask, int mstride, int S)
{
    const int s0 = blockIdx.y * SPC;
    bool act[SPC];
    bool any = false;
#pragma unroll
    for (int q = 0; q < SPC; ++q) {
        act[q] = s0 + q < S && on(mask, mstride, s0 + q);
        any = any || act[q];
    }
    if (!any) return;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= G.N) return;
    int i, j, k;
    node_ijk(G, n, i, j, k);
    T yp[SPC], yc[SPC];
#pragma unroll
    for (int q = 0; q < SPC; ++q) {
        const size_t s = act[q] ? s0 + q : s0;
        stencil_apply<T, TRANS, M>(G, J + s * 27 * G.N, x + s * G.N, n, i, j, k, yp[q], yc[q]);
    }
    const uint8_t m = bc[n];
#pragma unroll
    for (int q = 0; q < SPC; ++q) {
        if (!act[q]) continue;
        const size_t on_ = (size_t)(s0 + q) * G.N;
        const V2<T> bv = b[on_ + n];
        T rp = bv.p - yp[q], rc = bv.c - yc[q];
        if (m & BC_P) rp = T(0);
        if (m & BC_C) rc = T(0);
        r[on_ + n] = V2<T>{rp, rc};
    }
}

template <class T, class M>
void launch_mg_residual(const Grid& G, const B4<M>* J, const uint8_t* bc,
                        const V2<T>* b, const V2<T>* x, V2<T>* r, int trans,
                        const int* mask, int mstride, int S, cudaStream_t st, int bs, int spc)
{
    count_launch(1);
    dim3 grid(nblocks(G.N, bs), (S + spc - 1) / spc);
#define ELDER_MGR(TR, SP) \
    k_mg_residual<T, M, TR, SP><<<grid, bs, 0, st>>>(G, J, bc, b, x, r, mask, mstride, S)
    if (spc == 2) {
        if (trans) ELDER_MGR(true, 2);
        else ELDER_MGR(false, 2);
    } else {
        if (trans) ELDER_MGR(true, 1);
        else ELDER_MGR(false, 1);
    }
#undef ELDER_MGR
}

// Full weighting = transpose of trilinear interpolation on the vertex-centred
// 2:1 hierarchy (coarse node (I,J,K) is fine node (2I,2J,2K)).
template <class T>
__global__ void __launch_bounds__(kBS)
    k_restrict(Grid Gf, Grid Gc, const uint8_t* __restrict__ bcc,
               const V2<T>* __restrict__ rf, V2<T>* __restrict__ bco,
               const int* mask, int mstride)
{
    const int s = blockIdx.y;
    if (!on(mask, mstride, s)) return;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= Gc.N) return;
    int I, J, K;
    node_ijk_fast(Gc, n, I, J, K);
    rf += (size_t)s * Gf.N;
    T sp = T(0), sc = T(0);
#pragma unroll
    for (int c = -1; c <= 1; ++c)
#pragma unroll
        for (int b = -1; b <= 1; ++b)
#pragma unroll
            for (int a = -1; a <= 1; ++a) {
                const int fi = 2 * I + a, fj = 2 * J + b, fk = 2 * K + c;
                if (fi < 0 || fi > Gf.nx || fj < 0 || fj > Gf.ny || fk < 0 || fk > Gf.nz)
                    continue;
                const T w = T((a == 0 ? 1.0 : 0.5) * (b == 0 ? 1.0 : 0.5) * (c == 0 ? 1.0 : 0.5));
                const V2<T> v = rf[node_id(Gf, fi, fj, fk)];
                sp += w * v.p;
                sc += w * v.c;
            }
    const uint8_t m = bcc[n];
    if (m & BC_P) sp = T(0);
    if (m & BC_C) sc = T(0);
    bco[(size_t)s * Gc.N + n] = V2<T>{sp, sc};
}

template <class T>
void launch_restrict(const Grid& Gf, const Grid& Gc, const uint8_t* bcc,
                     const V2<T>* rf, V2<T>* bco, const int* mask, int mstride,
                     int S, cudaStream_t st)
{
    count_launch(1);
    dim3 grid(nblocks(Gc.N), S);
    k_restrict<T><<<grid, kBS, 0, st>>>(Gf, Gc, bcc, rf, bco, mask, mstride);
}

template <class T>
__global__ void __launch_bounds__(kBS)
    k_prolong_add(Grid Gf, Grid Gc, const uint8_t* __restrict__ bcf,
                  const V2<T>* __restrict__ xc, V2<T>* __restrict__ xf,
                  const int* mask, int mstride)
{
    const int s = blockIdx.y;
    if (!on(mask, mstride, s)) return;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= Gf.N) return;
    int i, j, k;
    node_ijk_fast(Gf, n, i, j, k);
    xc += (size_t)s * Gc.N;
    // trilinear interpolation as three nested averages of the 8 coarse
    // parents; for an even fine index both parents are the same node, whose
    // average is exact, so no branch depends on the parity
    const int sxc = Gc.nx + 1, szc = (Gc.nx + 1) * (Gc.ny + 1);
    const int c0 = (i >> 1) + sxc * (j >> 1) + szc * (k >> 1);
    const int di = i & 1, dj = (j & 1) * sxc, dk = (k & 1) * szc;
    V2<T> v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q)
        v[q] = xc[c0 + ((q & 1) ? di : 0) + ((q & 2) ? dj : 0) + ((q & 4) ? dk : 0)];
    const T h = T(0.5);
    T ap[4], ac[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        ap[q] = h * (v[2 * q].p + v[2 * q + 1].p);
        ac[q] = h * (v[2 * q].c + v[2 * q + 1].c);
    }
    const T bp0 = h * (ap[0] + ap[1]), bp1 = h * (ap[2] + ap[3]);
    const T bc0 = h * (ac[0] + ac[1]), bc1 = h * (ac[2] + ac[3]);
    const T sp = h * (bp0 + bp1), sc = h * (bc0 + bc1);
    const uint8_t m = bcf[n];
    V2<T> o = xf[(size_t)s * Gf.N + n];
    o.p = (m & BC_P) ? T(0) : o.p + sp;
    o.c = (m & BC_C) ? T(0) : o.c + sc;
    xf[(size_t)s * Gf.N + n] = o;
}

template <class T>
void launch_prolong_add(const Grid& Gf, const Grid& Gc, const uint8_t* bcf,
                        const V2<T>* xc, V2<T>* xf, const int* mask,
                        int mstride, int S, cudaStream_t st)
{
    count_launch(1);
    dim3 grid(nblocks(Gf.N), S);
    k_prolong_add<T><<<grid, kBS, 0, st>>>(Gf, Gc, bcf, xc, xf, mask, mstride);
}

// x = A_c^{-1} b on the coarsest grid (FP64 inverse), one block per sample.
template <class T>
__global__ void k_coarse_apply(int n, const T* __restrict__ Ainv,
                               const V2<T>* __restrict__ b, V2<T>* __restrict__ x,
                               int trans, const int* mask, int mstride)
{
    extern __shared__ __align__(16) unsigned char ca_smem[];
    T* bs = reinterpret_cast<T*>(ca_smem);
    const int s = blockIdx.x;
    if (!on(mask, mstride, s)) return;
    const T* bb = reinterpret_cast<const T*>(b + (size_t)s * (n / 2));
    for (int q = threadIdx.x; q < n; q += blockDim.x) bs[q] = bb[q];
    __syncthreads();
    const T* A = Ainv + (size_t)s * n * n;
    T* xx = reinterpret_cast<T*>(x + (size_t)s * (n / 2));
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
        T acc = T(0);
        if (!trans)
            for (int q = 0; q < n; ++q) acc = fma(A[(size_t)r * n + q], bs[q], acc);
        else
            for (int q = 0; q < n; ++q) acc = fma(A[(size_t)q * n + r], bs[q], acc);
        xx[r] = acc;
    }
}

template <class T>
void launch_coarse_apply(const Grid& G, const double* Ainv, const V2<T>* b,
                         V2<T>* x, int trans, const int* mask, int mstride,
                         int S, cudaStream_t st)
{
    count_launch(1);
    const int n = 2 * G.N;
    // the inverse is stored in the solver's arithmetic (CoarseType of its
    // multigrid storage type: FP32 for the mixed solver, FP64 otherwise)
    k_coarse_apply<T><<<S, 128, sizeof(T) * n, st>>>(n, reinterpret_cast<const T*>(Ainv), b, x,
                                                     trans, mask, mstride);
}

// ---------------------------------------------------------------------------
// BiCGStab vector updates and per-sample scalars
// ---------------------------------------------------------------------------

template <class T>
__global__ void __launch_bounds__(kBS)
    k_bicg_init(Grid G, const uint8_t* __restrict__ bc, const V2<T>* __restrict__ b,
                V2<T>* x, V2<T>* r, V2<T>* rh, V2<T>* p, V2<T>* v,
                double* __restrict__ partial, const KScal* ks)
{
    __shared__ double red[32];
    const int s = blockIdx.y;
    if (!ks[s].active) return;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    double d = 0.0;
    if (n < G.N) {
        const size_t q = (size_t)s * G.N + n;
        V2<T> bv = b[q];
        const uint8_t m = bc[n];
        if (m & BC_P) bv.p = T(0);
        if (m & BC_C) bv.c = T(0);
        const V2<T> z{T(0), T(0)};
        x[q] = z;
        p[q] = z;
        v[q] = z;
        r[q] = bv;
        rh[q] = bv;
        d = dot2(bv.p, bv.c, bv.p, bv.c);
    }
    const double t = block_sum(d, red);
    if (threadIdx.x == 0) partial[((size_t)s * 2) * gridDim.x + blockIdx.x] = t;
}

template <class T>
void launch_bicg_init(const Grid& G, const uint8_t* bc, const V2<T>* b,
                      V2<T>* x, V2<T>* r, V2<T>* rh, V2<T>* p, V2<T>* v,
                      double* partial, KScal* ks, int S, cudaStream_t st)
{
    count_launch(1);
    dim3 grid(nblocks(G.N), S);
    k_bicg_init<T><<<grid, kBS, 0, st>>>(G, bc, b, x, r, rh, p, v, partial, ks);
}

template <class T>
__global__ void __launch_bounds__(kBS)
    k_bicg_p(int N, const V2<T>* __restrict__ r, const V2<T>* __restrict__ v,
             V2<T>* __restrict__ p, const KScal* ks)
{
    const int s = blockIdx.y;
    const KScal k = ks[s];
    if (!k.active) return;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const T b = ks_beta<T>(k), w = ks_omega<T>(k);
    const size_t q = (size_t)s * N + n;
    const V2<T> rv = r[q], vv = v[q];
    V2<T> pv = p[q];
    pv.p = rv.p + b * (pv.p - w * vv.p);
    pv.c = rv.c + b * (pv.c - w * vv.c);
    p[q] = pv;
}

template <class T>
void launch_bicg_p(const Grid& G, const V2<T>* r, const V2<T>* v, V2<T>* p,
                   const KScal* ks, int S, cudaStream_t st)
{
    count_launch(1);
    dim3 grid(nblocks(G.N), S);
    k_bicg_p<T><<<grid, kBS, 0, st>>>(G.N, r, v, p, ks);
}

template <class T>
__global__ void __launch_bounds__(kBS)
    k_bicg_s(int N, const V2<T>* __restrict__ r, const V2<T>* __restrict__ v,
             V2<T>* __restrict__ sv, const KScal* ks)
{
    const int s = blockIdx.y;
    const KScal k = ks[s];
    if (!k.active) return;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const T a = ks_alpha<T>(k);
    const size_t q = (size_t)s * N + n;
    const V2<T> rv = r[q], vv = v[q];
    sv[q] = V2<T>{rv.p - a * vv.p, rv.c - a * vv.c};
}

template <class T>
void launch_bicg_s(const Grid& G, const V2<T>* r, const V2<T>* v, V2<T>* s,
                   double* partial, const KScal* ks, int S, cudaStream_t st)
{
    count_launch(1);
    (void)partial;
    dim3 grid(nblocks(G.N), S);
    k_bicg_s<T><<<grid, kBS, 0, st>>>(G.N, r, v, s, ks);
}

// Each thread updates kXrNodes consecutive-stride nodes and sums its own
// terms of the two inner products before the FP64 block reduction (for the
// FP32 solver the per-thread sum is FP32, see dot2).
constexpr int kXrNodes = 4;

template <class T>
__global__ void __launch_bounds__(kBS)
    k_bicg_xr(int N, const V2<T>* __restrict__ ph, const V2<T>* __restrict__ sh,
              const V2<T>* __restrict__ sv, const V2<T>* __restrict__ t,
              const V2<T>* __restrict__ rh, V2<T>* __restrict__ x,
              V2<T>* __restrict__ r, double* __restrict__ partial,
              const KScal* ks)
{
    __shared__ double red[32];
    const int s = blockIdx.y;
    const KScal k = ks[s];
    if (!k.active) return;
    const T a = ks_alpha<T>(k), w = ks_omega<T>(k);
    T l0 = T(0), l1 = T(0);
    const int stride = gridDim.x * blockDim.x;
#pragma unroll
    for (int u = 0; u < kXrNodes; ++u) {
        const int n = blockIdx.x * blockDim.x + threadIdx.x + u * stride;
        if (n < N) {
            const size_t q = (size_t)s * N + n;
            const V2<T> pv = ph[q], shv = sh[q], svv = sv[q], tv = t[q], rhv = rh[q];
            V2<T> xv = x[q];
            xv.p += a * pv.p + w * shv.p;
            xv.c += a * pv.c + w * shv.c;
            x[q] = xv;
            const V2<T> rv{svv.p - w * tv.p, svv.c - w * tv.c};
            r[q] = rv;
            l0 += rv.p * rv.p + rv.c * rv.c;
            l1 += rhv.p * rv.p + rhv.c * rv.c;
        }
    }
    const double t0 = block_sum((double)l0, red);
    const double t1 = block_sum((double)l1, red);
    if (threadIdx.x == 0) {
        partial[((size_t)s * 2 + 0) * gridDim.x + blockIdx.x] = t0;
        partial[((size_t)s * 2 + 1) * gridDim.x + blockIdx.x] = t1;
    }
}

template <class T>
void launch_bicg_xr(const Grid& G, const V2<T>* ph, const V2<T>* sh,
                    const V2<T>* s, const V2<T>* t, const V2<T>* rh, V2<T>* x,
                    V2<T>* r, double* partial, const KScal* ks, int S,
                    cudaStream_t st)
{
    count_launch(1);
    dim3 grid(bicg_xr_blocks(G.N), S);
    k_bicg_xr<T><<<grid, kBS, 0, st>>>(G.N, ph, sh, s, t, rh, x, r, partial, ks);
}

// One block per sample: fixed-order sums of the partials and the BiCGStab
// scalar recurrences.
__global__ void k_bicg_finalize(int stage, const double* __restrict__ partial,
                                int nblk, KScal* ks, double rtol, int maxit)
{
    __shared__ double red[32];
    const int s = blockIdx.x;
    KScal k = ks[s];
    if (!k.active) return;
    double a0 = 0.0, a1 = 0.0;
    for (int q = threadIdx.x; q < nblk; q += blockDim.x) {
        a0 += partial[((size_t)s * 2 + 0) * nblk + q];
        a1 += partial[((size_t)s * 2 + 1) * nblk + q];
    }
    a0 = block_sum(a0, red);
    a1 = block_sum(a1, red);
    if (threadIdx.x != 0) return;
    if (stage == 0) {  // after init: ||b||^2 = (rh, r)
        k.bn2 = a0;
        k.rn2 = a0;
        k.rho = a0;
        k.rho_old = 1.0;
        k.alpha = 1.0;
        k.omega = 1.0;
        k.iters = 0;
        k.status = 0;
        k.best_rn2 = a0;
        k.improved = 0;
        k.beta = 0.0;  // p = v = 0: the first update sets p = r
        k.alpha_f = 1.0f;
        k.omega_f = 1.0f;
        k.beta_f = 0.0f;
        if (!(a0 > 0.0)) {
            k.active = 0;
            if (!isfinite(a0)) k.status = ELDER_SAMPLE_NONFINITE_;
        }
    } else if (stage == 1) {  // alpha = rho / (rh, v)
        if (a0 == 0.0 || !isfinite(a0)) {
            k.active = 0;
            k.status = ELDER_SAMPLE_BREAKDOWN_;
        } else {
            k.alpha = k.rho / a0;
            k.alpha_f = (float)k.alpha;
        }
    } else if (stage == 2) {  // omega = (t, s) / (t, t)
        k.omega = (a1 > 0.0) ? a0 / a1 : 0.0;
        k.omega_f = (float)k.omega;
    } else {  // end of iteration: ||r||^2 and the next rho = (rh, r)
        k.rn2 = a0;
        k.rho_old = k.rho;
        k.rho = a1;
        k.iters += 1;
        k.improved = a0 < k.best_rn2;
        if (k.improved) k.best_rn2 = a0;
        k.beta = (k.omega != 0.0 && k.rho_old != 0.0) ? (k.rho / k.rho_old) * (k.alpha / k.omega)
                                                      : 0.0;
        k.beta_f = (float)k.beta;
        if (!isfinite(a0)) {
            k.active = 0;
            k.status = ELDER_SAMPLE_NONFINITE_;
        } else if (a0 <= rtol * rtol * k.bn2) {
            k.active = 0;
        } else if (k.iters >= maxit) {
            k.active = 0;
            k.status = ELDER_SAMPLE_KRYLOV_MAXIT_;
        } else if (k.rho == 0.0 || k.omega == 0.0) {
            k.active = 0;
            k.status = ELDER_SAMPLE_BREAKDOWN_;
        }
    }
    ks[s] = k;
}

void launch_bicg_finalize(int stage, const double* partial, int nblk,
                          KScal* ks, double rtol, int maxit, int S,
                          cudaStream_t st)
{
    count_launch(1);
    k_bicg_finalize<<<S, 128, 0, st>>>(stage, partial, nblk, ks, rtol, maxit);
}

template <class T>
__global__ void k_bicg_keep(int N, V2<T>* __restrict__ x, V2<T>* __restrict__ xbest,
                            const KScal* ks, int keep)
{
    const int s = blockIdx.y;
    const KScal& k = ks[s];
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const size_t q = (size_t)s * N + n;
    if (keep == 1) {
        if (k.improved) xbest[q] = x[q];
    } else if (k.status != 0 || k.active) {
        x[q] = xbest[q];
    }
}

template <class T>
void launch_bicg_keep(const Grid& G, V2<T>* x, V2<T>* xbest, const KScal* ks, int keep, int S,
                      cudaStream_t st)
{
    count_launch(1);
    dim3 grid(nblocks(G.N), S);
    k_bicg_keep<T><<<grid, kBS, 0, st>>>(G.N, x, xbest, ks, keep);
}

// ---------------------------------------------------------------------------
// Newton with line search
// ---------------------------------------------------------------------------

// which = 0: ||R(u)||, res0 and the round-off floor of ||R|| (2 eps times the
// norm of the per-row sums of the magnitudes of the summed terms);
// which = 1: ||R(u_trial)|| and the floor at the trial state
__global__ void k_norm_finalize(const double* __restrict__ partial,
                                const double* __restrict__ act, int nblk, NScal* ns,
                                int which)
{
    __shared__ double red[32];
    const int s = blockIdx.x;
    if (which == 1 && !ns[s].ls_active) return;
    if (which == 0 && !ns[s].active) return;
    double a = 0.0, b = 0.0;
    for (int q = threadIdx.x; q < nblk; q += blockDim.x) {
        a += partial[(size_t)s * nblk + q];
        if (act) b += act[(size_t)s * nblk + q];
    }
    a = block_sum(a, red);
    b = block_sum(b, red);
    if (threadIdx.x != 0) return;
    const double r = sqrt(a);
    if (which == 0) {
        ns[s].rn = r;
        ns[s].res0 = r;
        ns[s].rfloor = 2.0 * 2.220446049250313e-16 * sqrt(b);
        if (!isfinite(r)) {
            ns[s].active = 0;
            ns[s].ls_active = 0;
            ns[s].status = ELDER_SAMPLE_NONFINITE_;
        } else if (r <= ns[s].rfloor) {  // already a solution to round-off
            ns[s].active = 0;
            ns[s].ls_active = 0;
            ns[s].status = 0;
        }
    } else {
        ns[s].rt = r;
        ns[s].rfloor_t = 2.0 * 2.220446049250313e-16 * sqrt(b);
    }
}

void launch_norm_finalize(const double* partial, const double* act, int nblk, NScal* ns,
                          int which, int S, cudaStream_t st)
{
    count_launch(1);
    k_norm_finalize<<<S, 128, 0, st>>>(partial, act, nblk, ns, which);
}

template <class T>
__global__ void __launch_bounds__(kBS)
    k_newton_rhs(int N, const V2<double>* __restrict__ R, V2<T>* __restrict__ b,
                 const NScal* ns)
{
    const int s = blockIdx.y;
    if (!ns[s].active) return;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const size_t q = (size_t)s * N + n;
    const V2<double> r = R[q];
    b[q] = V2<T>{T(-r.p), T(-r.c)};
}

template <class T>
void launch_newton_rhs(const Grid& G, const V2<double>* R, V2<T>* b,
                       const NScal* ns, int S, cudaStream_t st)
{
    count_launch(1);
    dim3 grid(nblocks(G.N), S);
    k_newton_rhs<T><<<grid, kBS, 0, st>>>(G.N, R, b, ns);
}

template <class T>
__global__ void __launch_bounds__(kBS)
    k_newton_trial(int N, const double* __restrict__ p, const double* __restrict__ c,
                   const V2<T>* __restrict__ dx, double* __restrict__ pt,
                   double* __restrict__ ct, double* __restrict__ partial,
                   const NScal* ns)
{
    __shared__ double red[32];
    const int s = blockIdx.y;
    if (!ns[s].ls_active) return;
    const double lam = ns[s].lambda;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if constexpr (std::is_same<T, float>::value) {
        // FP32 correction: lambda is a power of two (1 halved by the line
        // search), so lambda d is exact in FP32 (above 2^-126 in magnitude;
        // below, it rounds to FP32's subnormals, far under the rounding of p
        // and c) and its widening exact; the maxima of the magnitudes are
        // integer maxima of their bit patterns.  Neither touches the FP64
        // pipe, and the values equal the FP64 form's, lambda (double) d.
        const float lamf = d2f_trunc(lam);
        unsigned up = 0u, uc = 0u;
        if (n < N) {
            const size_t q = (size_t)s * N + n;
            const V2<T> d = dx[q];
            const float dpf = lamf * d.p, dcf = lamf * d.c;
            pt[q] = p[q] + f2d_exact(dpf);
            ct[q] = c[q] + f2d_exact(dcf);
            // a non-finite correction must never meet the Newton stop: NaN
            // enters the maxima as +inf
            up = mag_bits(dpf);
            uc = mag_bits(dcf);
        }
        unsigned* ured = reinterpret_cast<unsigned*>(red);
        const unsigned t0 = block_max(up, ured);
        const unsigned t1 = block_max(uc, ured);
        if (threadIdx.x == 0) {
            partial[((size_t)s * 2 + 0) * gridDim.x + blockIdx.x] = f2d_exact(__uint_as_float(t0));
            partial[((size_t)s * 2 + 1) * gridDim.x + blockIdx.x] = f2d_exact(__uint_as_float(t1));
        }
        return;
    }
    double mp = 0.0, mc = 0.0;
    if (n < N) {
        const size_t q = (size_t)s * N + n;
        const V2<T> d = dx[q];
        const double dp = lam * (double)d.p, dc = lam * (double)d.c;
        pt[q] = p[q] + dp;
        ct[q] = c[q] + dc;
        // a non-finite correction must never meet the Newton stop: block_max
        // (fmax) would drop a NaN, so it enters the maxima as +inf
        mp = isfinite(dp) ? fabs(dp) : INFINITY;
        mc = isfinite(dc) ? fabs(dc) : INFINITY;
    }
    const double t0 = block_max(mp, red);
    const double t1 = block_max(mc, red);
    if (threadIdx.x == 0) {
        partial[((size_t)s * 2 + 0) * gridDim.x + blockIdx.x] = t0;
        partial[((size_t)s * 2 + 1) * gridDim.x + blockIdx.x] = t1;
    }
}

template <class T>
void launch_newton_trial(const Grid& G, const double* p, const double* c,
                         const V2<T>* dx, double* pt, double* ct,
                         double* partial, const NScal* ns, int S,
                         cudaStream_t st)
{
    count_launch(1);
    dim3 grid(nblocks(G.N), S);
    k_newton_trial<T><<<grid, kBS, 0, st>>>(G.N, p, c, dx, pt, ct, partial, ns);
}

// Armijo-type acceptance ||R(u + lambda d)|| < (1 - 1e-4 lambda) ||R(u)||;
// after ls_max halvings the last trial is taken.
__global__ void k_newton_ls_finalize(const double* __restrict__ pmax, int nblk,
                                     NScal* ns, int ls_max)
{
    __shared__ double red[32];
    const int s = blockIdx.x;
    if (!ns[s].ls_active) return;
    double a0 = 0.0, a1 = 0.0;
    for (int q = threadIdx.x; q < nblk; q += blockDim.x) {
        a0 = fmax(a0, pmax[((size_t)s * 2 + 0) * nblk + q]);
        a1 = fmax(a1, pmax[((size_t)s * 2 + 1) * nblk + q]);
    }
    a0 = block_max(a0, red);
    a1 = block_max(a1, red);
    if (threadIdx.x != 0) return;
    NScal k = ns[s];
    k.dmax_p = a0;
    k.dmax_c = a1;
    const bool finite = isfinite(k.rt);
    // a trial at the round-off floor of ||R|| is accepted as it is: below
    // that level the decrease test compares rounding noise
    if (finite && (k.rt < (1.0 - 1e-4 * k.lambda) * k.rn || k.rt <= k.rfloor_t)) {
        k.ls_active = 0;
        k.accepted = 1;
    } else if (k.ls_count >= ls_max) {  // no step length decreased ||R||
        k.ls_active = 0;
        k.active = 0;
        k.status = ELDER_SAMPLE_LINESEARCH_;
    } else {
        k.lambda *= 0.5;
        k.ls_count += 1;
        k.ls_cuts += 1;
    }
    ns[s] = k;
}

void launch_newton_ls_finalize(const double* partial_res,
                               const double* partial_max, int nblk,
                               NScal* ns, int ls_max, int S, cudaStream_t st)
{
    count_launch(1);
    (void)partial_res;
    k_newton_ls_finalize<<<S, 128, 0, st>>>(partial_max, nblk, ns, ls_max);
}

__global__ void __launch_bounds__(kBS)
    k_newton_accept(int N, double* __restrict__ p, double* __restrict__ c,
                    const double* __restrict__ pt, const double* __restrict__ ct,
                    V2<double>* __restrict__ R, const V2<double>* __restrict__ Rt,
                    const NScal* ns)
{
    const int s = blockIdx.y;
    if (!ns[s].accepted) return;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const size_t q = (size_t)s * N + n;
    p[q] = pt[q];
    c[q] = ct[q];
    if (!ns[s].skip_res) R[q] = Rt[q];  // else R stays that of the last evaluated iterate
}

void launch_newton_accept(const Grid& G, double* p, double* c,
                          const double* pt, const double* ct, V2<double>* R,
                          const V2<double>* Rt, const NScal* ns, int S,
                          cudaStream_t st)
{
    count_launch(1);
    dim3 grid(nblocks(G.N), S);
    k_newton_accept<<<grid, kBS, 0, st>>>(G.N, p, c, pt, ct, R, Rt, ns);
}

// With inexact linear solves Newton converges linearly: from two
// consecutive full steps the contraction is theta = |d_k| / |d_{k-1}| and
// the remaining error about theta / (1 - theta) |d_k|.  A full step stops
// the iteration when that estimate, or the last correction itself, is
// within tolerance.
__device__ __forceinline__ bool newton_small(const NScal& k, double tol_p, double tol_c,
                                             int estimate)
{
    if (k.lambda != 1.0) return false;
    if (k.dmax_c <= tol_c && k.dmax_p <= tol_p) return true;
    if (estimate && k.full_prev && k.dprev_c > 0.0 && k.dprev_p > 0.0) {
        const double th = fmax(k.dmax_c / k.dprev_c, k.dmax_p / k.dprev_p);
        if (th < 0.5) {
            const double f = th / (1.0 - th);
            return f * k.dmax_c <= tol_c && f * k.dmax_p <= tol_p;
        }
    }
    return false;
}

// Before the trial residual of a full step (lambda = 1): the sizes of the
// correction (per-block maxima of k_newton_trial) decide the stop already,
// and a sample that meets it is accepted without its trial residual (its
// Armijo test would only compare a converged iterate).
__global__ void k_newton_predict(const double* __restrict__ pmax, int nblk, NScal* ns,
                                 double tol_p, double tol_c, int estimate)
{
    __shared__ double red[32];
    const int s = blockIdx.x;
    if (!ns[s].ls_active || ns[s].lambda != 1.0) return;
    double a0 = 0.0, a1 = 0.0;
    for (int q = threadIdx.x; q < nblk; q += blockDim.x) {
        a0 = fmax(a0, pmax[((size_t)s * 2 + 0) * nblk + q]);
        a1 = fmax(a1, pmax[((size_t)s * 2 + 1) * nblk + q]);
    }
    a0 = block_max(a0, red);
    a1 = block_max(a1, red);
    if (threadIdx.x != 0) return;
    NScal k = ns[s];
    k.dmax_p = a0;
    k.dmax_c = a1;
    if (newton_small(k, tol_p, tol_c, estimate)) {
        k.ls_active = 0;
        k.accepted = 1;
        k.skip_res = 1;
        ns[s] = k;
    }
}

void launch_newton_predict(const double* partial_max, int nblk, NScal* ns, double tol_p,
                           double tol_c, int estimate, int S, cudaStream_t st)
{
    count_launch(1);
    k_newton_predict<<<S, 128, 0, st>>>(partial_max, nblk, ns, tol_p, tol_c, estimate);
}

__global__ void k_newton_check(NScal* ns, const KScal* ks, double tol_p,
                               double tol_c, int maxit, int estimate, int S)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    NScal k = ns[s];
    if (!k.active) return;
    k.kiters += ks[s].iters;
    if (k.accepted) {
        k.iters += 1;
        if (k.skip_res) {
            // accepted by k_newton_predict: its correction met the stop (rn
            // stays the norm of the last evaluated iterate)
            k.active = 0;
            k.status = 0;
        } else {
            k.rn = k.rt;
            k.rfloor = k.rfloor_t;
            // the correction-size stop (or R at its round-off floor)
            const bool small = newton_small(k, tol_p, tol_c, estimate);
            k.full_prev = (k.lambda == 1.0);
            k.dprev_c = k.dmax_c;
            k.dprev_p = k.dmax_p;
            if (small || k.rn <= k.rfloor) {
                k.active = 0;
                k.status = 0;
            } else if (k.iters >= maxit) {
                k.active = 0;
                k.status = ELDER_SAMPLE_NEWTON_MAXIT_;
            }
        }
    }
    k.skip_res = 0;
    k.accepted = 0;
    k.ls_count = 0;
    k.lambda = 1.0;
    k.ls_active = k.active;
    ns[s] = k;
}

void launch_newton_check(NScal* ns, const KScal* ks, double tol_p,
                         double tol_c, int maxit, int estimate, int S, cudaStream_t st)
{
    count_launch(1);
    k_newton_check<<<nblocks(S, 128), 128, 0, st>>>(ns, ks, tol_p, tol_c, maxit, estimate, S);
}

// Newton's starting point from the last states: order 1 the linear
// extrapolation 2 u^n - u^{n-1}, order 2 the quadratic 3 u^n - 3 u^{n-1} +
// u^{n-2}; the salt fraction clipped to [0, 1] (Dirichlet values are imposed
// afterwards).  h1, h2 hold u^{n-1}, u^{n-2}.
__global__ void k_extrapolate(int N, int order, const double* __restrict__ p_n,
                              const double* __restrict__ c_n, const double* __restrict__ p1,
                              const double* __restrict__ c1, const double* __restrict__ p2,
                              const double* __restrict__ c2, double* __restrict__ p,
                              double* __restrict__ c)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const size_t q = (size_t)blockIdx.y * N + n;
    double pe, ce;
    if (order == 2) {
        pe = 3.0 * (p_n[q] - p1[q]) + p2[q];
        ce = 3.0 * (c_n[q] - c1[q]) + c2[q];
    } else {
        pe = 2.0 * p_n[q] - p1[q];
        ce = 2.0 * c_n[q] - c1[q];
    }
    p[q] = pe;
    c[q] = fmin(1.0, fmax(0.0, ce));
}

void launch_extrapolate(const Grid& G, int order, const double* p_n, const double* c_n,
                        const double* p1, const double* c1, const double* p2, const double* c2,
                        double* p, double* c, int S, cudaStream_t st)
{
    count_launch(1);
    dim3 grid(nblocks(G.N), S);
    k_extrapolate<<<grid, kBS, 0, st>>>(G.N, order, p_n, c_n, p1, c1, p2, c2, p, c);
}

__global__ void k_newton_restore_failed(int N, double* __restrict__ p,
                                        double* __restrict__ c,
                                        const double* __restrict__ p_old,
                                        const double* __restrict__ c_old,
                                        const NScal* ns)
{
    const int s = blockIdx.y;
    if (ns[s].status == 0) return;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const size_t q = (size_t)s * N + n;
    p[q] = p_old[q];
    c[q] = c_old[q];
}

void launch_newton_restore_failed(const Grid& G, double* p, double* c,
                                  const double* p_old, const double* c_old,
                                  const NScal* ns, int S, cudaStream_t st)
{
    count_launch(1);
    dim3 grid(nblocks(G.N), S);
    k_newton_restore_failed<<<grid, kBS, 0, st>>>(G.N, p, c, p_old, c_old, ns);
}

// ---------------------------------------------------------------------------
// sample statistics (Section 3: eqs. pdestat, numer_var; exceedance estimate)
// ---------------------------------------------------------------------------
//
// One pass over the S fields per node, shifted by the first sample's value
// for stability: with d_i = c_i - c_0, S1 = sum w d, S2 = sum w d^2,
// W = sum w: mean = c_0 W + S1 and sum w (mean - c)^2 =
// (mean - c_0)^2 W - 2 (mean - c_0) S1 + S2.
__global__ void __launch_bounds__(kBS)
    k_moments(int N, int S, const double* __restrict__ c,
              const double* __restrict__ w, double threshold,
              double* __restrict__ mean, double* __restrict__ var,
              double* __restrict__ pexc)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const double c0 = c[n];
    const double wu = 1.0 / S;
    double S1 = 0.0, S2 = 0.0, W = 0.0, P = 0.0;
    for (int s = 0; s < S; ++s) {
        const double ws = w ? __ldg(w + s) : wu;
        const double cv = __ldcs(c + (size_t)s * N + n);
        const double d = cv - c0;
        S1 = fma(ws, d, S1);
        S2 = fma(ws * d, d, S2);
        W += ws;
        if (cv > threshold) P += ws;
    }
    const double m = fma(c0, W, S1);
    const double dm = m - c0;
    mean[n] = m;
    var[n] = fmax(fma(dm * dm, W, fma(-2.0 * dm, S1, S2)), 0.0);
    pexc[n] = P;
}

void launch_moments(int N, int S, const double* c, const double* w,
                    double threshold, double* mean, double* var,
                    double* pexc, cudaStream_t st)
{
    count_launch(1);
    k_moments<<<nblocks(N), kBS, 0, st>>>(N, S, c, w, threshold, mean, var, pexc);
}

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------

__global__ void k_sum_partials(const double* __restrict__ partial, int nblk,
                               double* __restrict__ out)
{
    __shared__ double red[32];
    double a = 0.0;
    for (int q = threadIdx.x; q < nblk; q += blockDim.x) a += partial[(size_t)blockIdx.x * nblk + q];
    a = block_sum(a, red);
    if (threadIdx.x == 0) out[blockIdx.x] = a;
}

void launch_sum_partials(const double* partial, int nblk, double* out, int S,
                         cudaStream_t st)
{
    count_launch(1);
    k_sum_partials<<<S, 128, 0, st>>>(partial, nblk, out);
}

// which = 0: y = a x on Dirichlet components only, 0 elsewhere;
// which = 1: y += a x on Dirichlet components only;
// which = 2: y += a x on interior components only.
template <class T>
__global__ void k_axpy_mask(Grid G, const uint8_t* __restrict__ bc,
                            const V2<T>* __restrict__ x, V2<T>* __restrict__ y,
                            double a, int which)
{
    const int s = blockIdx.y;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= G.N) return;
    const size_t q = (size_t)s * G.N + n;
    const uint8_t m = bc[n];
    const V2<T> xv = x[q];
    V2<T> yv = (which == 0) ? V2<T>{T(0), T(0)} : y[q];
    const bool dp = (m & BC_P) != 0, dc = (m & BC_C) != 0;
    if (which <= 1) {
        if (dp) yv.p += T(a) * xv.p;
        if (dc) yv.c += T(a) * xv.c;
    } else {
        if (!dp) yv.p += T(a) * xv.p;
        if (!dc) yv.c += T(a) * xv.c;
    }
    y[q] = yv;
}

template <class T>
void launch_axpy_mask(const Grid& G, const uint8_t* bc, const V2<T>* x,
                      V2<T>* y, double a, int which, int S, cudaStream_t st)
{
    count_launch(1);
    dim3 grid(nblocks(G.N), S);
    k_axpy_mask<T><<<grid, kBS, 0, st>>>(G, bc, x, y, a, which);
}

template <class Ts, class Td>
__global__ void k_convert(const V2<Ts>* __restrict__ x, V2<Td>* __restrict__ y,
                          size_t n)
{
    const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const V2<Ts> v = x[q];
    y[q] = V2<Td>{Td(v.p), Td(v.c)};
}

template <class Ts, class Td>
void launch_convert(const V2<Ts>* x, V2<Td>* y, size_t n, cudaStream_t st)
{
    count_launch(1);
    k_convert<Ts, Td><<<(unsigned)((n + kBS - 1) / kBS), kBS, 0, st>>>(x, y, n);
}

// ---------------------------------------------------------------------------
// explicit instantiations
// ---------------------------------------------------------------------------
#define ELDER_INST(T)                                                                    \
    template void launch_spmv<T>(const Grid&, const B4<T>*, const uint8_t*,              \
                                 const V2<T>*, V2<T>*, int, int, const V2<T>*,           \
                                 double*, const int*, int, int, cudaStream_t, int);      \
    template void launch_smooth<T, MgType<T>::type>(                                     \
        const Grid&, const B4<MgType<T>::type>*, const B4<T>*, const uint8_t*,           \
        const V2<T>*, const V2<T>*, V2<T>*, double, int, const int*, int, int,           \
        cudaStream_t, int);                                                              \
    template void launch_mg_residual<T, MgType<T>::type>(                                \
        const Grid&, const B4<MgType<T>::type>*, const uint8_t*, const V2<T>*,           \
        const V2<T>*, V2<T>*, int, const int*, int, int, cudaStream_t, int, int);        \
    template void launch_restrict<T>(const Grid&, const Grid&, const uint8_t*,           \
                                     const V2<T>*, V2<T>*, const int*, int, int,         \
                                     cudaStream_t);                                      \
    template void launch_prolong_add<T>(const Grid&, const Grid&, const uint8_t*,        \
                                        const V2<T>*, V2<T>*, const int*, int, int,      \
                                        cudaStream_t);                                   \
    template void launch_coarse_apply<T>(const Grid&, const double*, const V2<T>*,       \
                                         V2<T>*, int, const int*, int, int,              \
                                         cudaStream_t);                                  \
    template void launch_bicg_init<T>(const Grid&, const uint8_t*, const V2<T>*, V2<T>*, \
                                      V2<T>*, V2<T>*, V2<T>*, V2<T>*, double*, KScal*,   \
                                      int, cudaStream_t);                                \
    template void launch_bicg_p<T>(const Grid&, const V2<T>*, const V2<T>*, V2<T>*,      \
                                   const KScal*, int, cudaStream_t);                     \
    template void launch_bicg_s<T>(const Grid&, const V2<T>*, const V2<T>*, V2<T>*,      \
                                   double*, const KScal*, int, cudaStream_t);            \
    template void launch_bicg_xr<T>(const Grid&, const V2<T>*, const V2<T>*,             \
                                    const V2<T>*, const V2<T>*, const V2<T>*, V2<T>*,    \
                                    V2<T>*, double*, const KScal*, int, cudaStream_t);   \
    template void launch_newton_rhs<T>(const Grid&, const V2<double>*, V2<T>*,           \
                                       const NScal*, int, cudaStream_t);                 \
    template void launch_newton_trial<T>(const Grid&, const double*, const double*,      \
                                         const V2<T>*, double*, double*, double*,        \
                                         const NScal*, int, cudaStream_t);               \
    template void launch_axpy_mask<T>(const Grid&, const uint8_t*, const V2<T>*, V2<T>*, \
                                      double, int, int, cudaStream_t);                   \
    template void launch_bicg_keep<T>(const Grid&, V2<T>*, V2<T>*, const KScal*, int,    \
                                      int, cudaStream_t);                                \
    template void launch_smooth_zline<T, typename MgType<T>::type>(                      \
        const Grid&, const B4<typename MgType<T>::type>*, const B4<T>*, const uint8_t*,  \
        const V2<T>*, const V2<T>*, V2<T>*, double, int, const int*, int, int,           \
        cudaStream_t, int);                                                              \
    template void launch_zline_factor<T, typename MgType<T>::type>(                      \
        const Grid&, const B4<typename MgType<T>::type>*, const B4<T>*, const uint8_t*,  \
        B4<T>*, B4<T>*, const int*, int, int, cudaStream_t);                             \
    template void launch_zline_apply<T, typename MgType<T>::type>(                       \
        const Grid&, const B4<typename MgType<T>::type>*, const B4<T>*, const B4<T>*,    \
        const uint8_t*, const V2<T>*, const V2<T>*, V2<T>*, double, const int*, int, int,\
        cudaStream_t, int, int, int);
ELDER_INST(double)
ELDER_INST(float)
#undef ELDER_INST
template void launch_convert<double, float>(const V2<double>*, V2<float>*, size_t, cudaStream_t);
template void launch_convert<float, double>(const V2<float>*, V2<double>*, size_t, cudaStream_t);
template void launch_convert<double, double>(const V2<double>*, V2<double>*, size_t, cudaStream_t);

}  // namespace elder
