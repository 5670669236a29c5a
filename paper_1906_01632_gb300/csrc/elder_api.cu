// elder_api.cu -- context, multigrid hierarchy, Newton / BiCGStab drivers and
// the C ABI declared in include/elder.h.
//
// One implicit Euler step (Sections 2.3 and 5.1) for a batch of S samples:
//   Newton on the FP64 residual, with a line search;
//   each Newton system J d = -R solved by BiCGStab, right-preconditioned by
//   one geometric-multigrid V-cycle whose level matrices are the Jacobians
//   re-assembled on each grid (injected state, cell-averaged phi and K);
//   damped 2x2-block-Jacobi smoothing, full weighting / trilinear transfers,
//   dense inverse on the coarsest grid.
// Batching: every kernel covers all samples (grid.y); converged or failed
// samples are masked out by per-sample flags that live on the device.  The
// host only polls those flags (a few bytes) between Newton and Krylov
// iterations.  With use_graphs the body of one BiCGStab iteration (two
// V-cycles, two stencil products, vector updates, scalar recurrences) is
// captured once per (S, transpose) and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/elder.h"
#include "kernels.h"

using namespace elder;

namespace {

thread_local std::string g_create_error = "no error";

constexpr int KSTRIDE = sizeof(KScal) / sizeof(int);
constexpr int NSTRIDE = sizeof(NScal) / sizeof(int);
constexpr int MAX_COARSE_UNKNOWNS = 1200;

struct Fail {
    int code;
    std::string msg;
};

#define CK(call)                                                              \
    do {                                                                      \
        cudaError_t e_ = (call);                                              \
        if (e_ != cudaSuccess)                                                \
            throw Fail{e_ == cudaErrorMemoryAllocation ? ELDER_ENOMEM          \
                                                       : ELDER_ECUDA,         \
                       std::string(#call) + ": " + cudaGetErrorString(e_)};   \
    } while (0)

#define CKL() CK(cudaGetLastError())

template <class X> X* dalloc(size_t n)
{
    void* p = nullptr;
    if (n == 0) n = 1;
    CK(cudaMalloc(&p, n * sizeof(X)));
    return static_cast<X*>(p);
}

struct DevFree {
    std::vector<void*> ptrs;
    void add(void* p) { ptrs.push_back(p); }
    ~DevFree()
    {
        for (void* p : ptrs) cudaFree(p);
    }
};

// Dirichlet sets (Section 2.1 and the caption of Fig. 1); see elder.h.
void dirichlet_host(const elder_config& cf, const Grid& G, std::vector<uint8_t>& bc,
                    std::vector<double>& cval)
{
    bc.assign(G.N, 0);
    cval.assign(G.N, 0.0);
    for (int k = 0; k <= G.nz; ++k)
        for (int j = 0; j <= G.ny; ++j)
            for (int i = 0; i <= G.nx; ++i) {
                const int n = node_id(G, i, j, k);
                const bool top = (k == G.nz), bottom = (k == 0);
                const bool xe = (i == 0 || i == G.nx), ye = (j == 0 || j == G.ny);
                const bool sq = (4 * i >= G.nx && 4 * i <= 3 * G.nx && 4 * j >= G.ny &&
                                 4 * j <= 3 * G.ny);
                uint8_t b = 0;
                double cv = 0.0;
                switch (cf.bc_mode) {
                case 0:
                    if (top && xe && ye) b |= BC_P;
                    if (top && sq) { b |= BC_C; cv = 1.0; }
                    else if (bottom) b |= BC_C;
                    break;
                case 1:
                    if (top && (xe || ye)) b |= BC_P;
                    if (top) { b |= BC_C; cv = sq ? 1.0 : 0.0; }
                    else if (bottom) b |= BC_C;
                    break;
                case 2:
                    if (top && xe && ye) b |= BC_P;
                    if (top) { b |= BC_C; cv = 1.0; }
                    else if (bottom) b |= BC_C;
                    break;
                default:
                    if (top && xe && ye) b |= BC_P;
                    break;
                }
                bc[n] = b;
                cval[n] = cv;
            }
}

Grid make_grid(int nx, int ny, int nz, double Lx, double Ly, double Lz)
{
    Grid G;
    G.nx = nx;
    G.ny = ny;
    G.nz = nz;
    G.N = (nx + 1) * (ny + 1) * (nz + 1);
    G.C = nx * ny * nz;
    G.hx = Lx / nx;
    G.hy = Ly / ny;
    G.hz = Lz / nz;
    G.Lz = Lz;
    grid_set_divisors(G);
    return G;
}

}  // namespace

// ---------------------------------------------------------------------------
// solver state for one precision
// ---------------------------------------------------------------------------

struct SolverBase {
    virtual ~SolverBase() {}
};

template <class T> struct Solver : SolverBase {
    int S = 0;
    using M = typename MgType<T>::type;
    B4<T>* J0 = nullptr;           // level-0 Krylov operator (T)
    std::vector<B4<M>*> Jm;        // multigrid matrices per level (M)
    std::vector<B4<T>*> Dinv;      // inverse interior diagonal blocks per level
    std::vector<B4<T>*> zMi, zC;   // block-LU factors of the vertical lines per level
    std::vector<B4<M>*> F;         // multicolour ILU factors per level (ILU smoother)
    std::vector<B4<T>*> Fd;        // their inverse pivot blocks
    std::vector<V2<T>*> mb, mx, mx2, mr;  // multigrid vectors per level
    V2<T> *x = nullptr, *r = nullptr, *rh = nullptr, *p = nullptr, *v = nullptr,
          *s = nullptr, *t = nullptr, *ph = nullptr, *sh = nullptr, *b = nullptr,
          *xbest = nullptr, *xd = nullptr;
    double *Ainv = nullptr, *work = nullptr;
    DevFree mem;
    std::map<std::pair<int, int>, cudaGraphExec_t> graphs;  // (S, trans)
    std::map<std::pair<int, int>, long long> graph_kernels;  // kernel nodes
    ~Solver()
    {
        for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
    }
};

// Per-class CUDA-event accounting (elder_profile).
struct ProfRec {
    cudaEvent_t a, b;
    int cls;
    double bytes, flops;
};

struct Prof {
    bool on = false;
    std::vector<cudaEvent_t> pool;
    std::vector<ProfRec> pending;
    long long launches[ELDER_K_CLASSES] = {};
    double ms[ELDER_K_CLASSES] = {}, bytes[ELDER_K_CLASSES] = {}, flops[ELDER_K_CLASSES] = {};
    ~Prof()
    {
        for (auto& r : pending) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
        for (auto e : pool) cudaEventDestroy(e);
    }
};

// Key of a captured step: everything the graph bakes in.
struct StepKey {
    int S, order, prec, newton_maxit, lin_maxit, ls_max, estimate, smoother, nu2;
    double lin_rtol, omega, dt;
    const void* ptr[6];  // phi, K, p, c, p_hist, c_hist
    bool operator==(const StepKey& o) const
    {
        return std::memcmp(this, &o, sizeof(StepKey)) == 0;
    }
};

// One captured implicit step: the prologue, a while node over the Newton
// iterations whose body holds while nodes over the Krylov iterations and
// over the line search, and the epilogue.  k_*: kernels per prologue,
// Newton body (outside the inner loops), Krylov body, line-search body and
// epilogue, for the launch count of a replay.
struct StepGraph {
    StepKey key;
    cudaGraphExec_t exec = nullptr;
    long long k_pro = 0, k_nb = 0, k_kb = 0, k_lb = 0, k_epi = 0;
};

struct elder_ctx {
    elder_config cfg;
    int device = 0;
    Prof prof;
    // sample counts behind the byte model of the profiled launches
    int n_active_newton = 0, n_active_ls = 0, n_active_k = 0;
    std::string err = "no error";
    std::vector<Grid> grids;
    std::vector<uint8_t*> bc;          // per level [N]
    double* cval = nullptr;            // level 0 [N]
    std::vector<double*> phi, K, pl, cl;  // levels >= 1: [S][C], [S][N]
    double *p_old = nullptr, *c_old = nullptr, *pt = nullptr, *ct = nullptr;
    V2<double> *R = nullptr, *Rt = nullptr, *tmp2 = nullptr;
    double* partial = nullptr;         // [S][2][nblk0]
    double* partial2 = nullptr;
    double* partial3 = nullptr;
    double* pk = nullptr;              // packed batch for the FP64 re-solve
    QF* qf = nullptr;                  // [S][12][C] quarter-face fluxes of the residual
    double* mass = nullptr;            // [S][3] salt-mass balance
    double* h_mass = nullptr;          // pinned
    NScal* ns = nullptr;
    KScal* ks = nullptr;
    NScal* h_ns = nullptr;             // pinned
    KScal* h_ks = nullptr;             // pinned
    double* h_scalar = nullptr;        // pinned
    DevFree mem;
    std::unique_ptr<Solver<double>> s64;
    std::unique_ptr<Solver<float>> s32;
    int nblk0 = 0;
    // threads per block of the autotuned kernel classes (indexed by ELDER_K_*)
    int bs[ELDER_K_CLASSES] = {kBS, kBS, kBS, kBS, kBS, 128};
    // samples per CTA of the multigrid residual and the z-line sweep
    int spc[ELDER_K_CLASSES] = {1, 1, 1, 1, 1, 1};
    // the (threads per block, samples per CTA) candidates' ms per launch of
    // the multigrid residual [0] and the z-line sweep [1]
    float tune2_ms[2][6] = {};
    int smoother_now = ELDER_SMOOTH_JACOBI;  // smoother of the solve in progress
    double omega_now = 0.5;                  // its damping
    int nu2_now = 1;                         // its post-smoothing sweeps
    // Jacobian inputs per level in the assembly's arithmetic type (room for
    // FP64 pairs): node (p - rho0 g (Lz - z), c) [S][N], cell (phi, K/mu) [S][C]
    std::vector<double*> jn, jc;
    bool tuned[2] = {false, false};    // per precision (FP64, FP32)
    float tune_ms[3][3] = {};          // [class smooth/spmv/mgres][bs 128/256/512]
    // device-controlled steps (use_graphs = 2): captured step graphs, most
    // recent last; loop counters [0..2] and bodies run per loop [3..5]
    std::vector<StepGraph> step_graphs;
    bool step_graph_ok = true;
    std::string step_graph_note;
    long long step_graph_replays = 0;
    int* loopc = nullptr;
    int* h_loopc = nullptr;            // pinned
    ~elder_ctx()
    {
        for (auto& g : step_graphs) cudaGraphExecDestroy(g.exec);
        if (h_loopc) cudaFreeHost(h_loopc);
        s64.reset();
        s32.reset();
        if (h_ns) cudaFreeHost(h_ns);
        if (h_ks) cudaFreeHost(h_ks);
        if (h_scalar) cudaFreeHost(h_scalar);
        if (h_mass) cudaFreeHost(h_mass);
    }
};

std::atomic<long long> g_launches{0};

namespace elder {
void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
void set_static_error(const char* msg) { g_create_error = msg; }
}  // namespace elder

namespace {

Phys make_phys(const elder_config& c, double dt)
{
    return Phys{c.rho0, c.rho1 - c.rho0, c.mu, c.g, c.Dm, dt};
}

// Algorithmic DRAM bytes and flops per node of one launch (every array the
// kernel must touch, read or written once; neighbour reuse of x is free).
// T = bytes of the solver type.  J row: 27 blocks of 4; vectors: 2 values.
// Damping of the configured smoother.
double configured_omega(const elder_config& cf)
{
    if (cf.smoother == ELDER_SMOOTH_ILU) return cf.omega_ilu;
    return cf.smoother == ELDER_SMOOTH_ZLINE ? cf.omega_line : cf.omega;
}

double model_bytes(int cls, int T, int Mz, const Grid& G, int line)
{
    // T: bytes of a vector / Dinv entry; Mz: bytes of a stored matrix entry
    // (for the Jacobian class: Mz of the multigrid copy, T of the Krylov copy
    // or 0 when the level has none).  line (SMOOTH0): 1 the z-line sweep that
    // factors as it goes, reading the two vertical line blocks of J besides
    // Dinv; 2 the sweep with the assembly's line factors (zMi, zC and the
    // lower line block); 3 the multicolour ILU sweep from x = 0 (both
    // triangular solves: the 26 factor blocks, the inverse pivot, b, the
    // scratch vector written, read and written again, x_out, bc twice).
    // line (JACOBIAN): bit 0 with the line factorisation, bit 1 with the ILU
    // factorisation (J, Dinv and bc read, the factors written).
    const double cells_per_node = (double)G.C / G.N;
    const int Td = T ? T : Mz;
    switch (cls) {
    case ELDER_K_SMOOTH: return 108 * Mz + (4 + 2 + 2 + 2) * T + 1;  // J, Dinv, b, x, xo, bc
    case ELDER_K_SMOOTH0:
        if (line == 3) return 104 * Mz + (4 + 2 + 2 + 2 + 2 + 2) * T + 2;
        if (line == 2) return (4 + 4 + 2 + 2) * T + 4 * Mz + 1;    // zMi, zC, b, xo, L, bc
        return (4 + 2 + 2) * T + 1 + (line ? 8 * Mz : 0);          // Dinv, b, xo, bc (+ L, U)
    case ELDER_K_SPMV: return 108 * Mz + (2 + 2 + 2) * T + 1;        // J, x, y, a, bc
    case ELDER_K_MGRES: return 108 * Mz + (2 + 2 + 2) * T + 1;       // J, x, b, r, bc
    case ELDER_K_RESIDUAL:  // p, c, c_old, R, cval, bc, phi, K
        return 3 * 8 + 16 + 8 + 1 + 16 * cells_per_node;
    case ELDER_K_JACOBIAN:  // J written (Krylov + multigrid copies), Dinv; p, c, bc, phi, K;
                            // line factors: Dinv, L, U, bc read, zMi, zC written
        return 108 * T + 108 * Mz + 4 * Td + 16 + 1 + 16 * cells_per_node +
               ((line & 1) ? 12 * Td + 8 * Mz + 1 : 0) +
               ((line & 2) ? 108 * Mz + 104 * Mz + 8 * Td + 1 : 0);
    }
    return 0.0;
}

double model_flops(int cls, const Grid& G)
{
    const double cells_per_node = (double)G.C / G.N;
    switch (cls) {
    case ELDER_K_SMOOTH: return 216 + 8 + 4 + 4;
    case ELDER_K_SMOOTH0: return 8 + 2;
    case ELDER_K_SPMV: return 216 + 8;
    case ELDER_K_MGRES: return 216 + 2;
    case ELDER_K_RESIDUAL:
        // FP64 flops (FMA = 2) of the quarter-face form.  Per cell: for p
        // and each direction 4 edge differences and one (3,1) weight pass of
        // 20 (72); for c the three (3,1) passes over the cell's 8 values
        // (60); per quarter face the sum and difference of the two weighted
        // c values and 8 (+2 on vertical edges) for rho, m, F (128); 6 for
        // the coefficients: 266.  Per node: 36 edge sums, 10 edge
        // accumulations, 8 porosity sums and 21 for storage and the squared
        // norm: 75.
        return 266 * cells_per_node + 75;
    case ELDER_K_JACOBIAN: return 24 * (54 + 66) + 10;
    }
    return 0.0;
}

int prof_begin(elder_ctx* ctx, cudaStream_t st)
{
    Prof& P = ctx->prof;
    if (!P.on) return -1;
    ProfRec r;
    for (cudaEvent_t* e : {&r.a, &r.b}) {
        if (!P.pool.empty()) {
            *e = P.pool.back();
            P.pool.pop_back();
        } else {
            CK(cudaEventCreate(e));
        }
    }
    CK(cudaEventRecord(r.a, st));
    r.cls = -1;
    P.pending.push_back(r);
    return (int)P.pending.size() - 1;
}

// variant: for SMOOTH0 -1 = by the smoother in use, 2 = the factored z-line
// sweep; for JACOBIAN 1 = with the line factorisation
void prof_end(elder_ctx* ctx, int idx, int cls, const Grid& G, int T, int Mz, int samples,
              cudaStream_t st, int variant = -1)
{
    if (idx < 0) return;
    ProfRec& r = ctx->prof.pending[idx];
    CK(cudaEventRecord(r.b, st));
    r.cls = cls;
    int line = ctx->smoother_now == ELDER_SMOOTH_ZLINE && G.nz + 1 <= kMaxLine ? 1 : 0;
    if (variant >= 0) line = variant;
    r.bytes = model_bytes(cls, T, Mz, G, line) * G.N * samples;
    r.flops = model_flops(cls, G) * G.N * samples;
}

// after a stream synchronisation: accumulate and recycle the events
void prof_drain(elder_ctx* ctx)
{
    Prof& P = ctx->prof;
    for (auto& r : P.pending) {
        float ms = 0.f;
        CK(cudaEventSynchronize(r.b));
        CK(cudaEventElapsedTime(&ms, r.a, r.b));
        if (r.cls >= 0) {
            P.launches[r.cls] += 1;
            P.ms[r.cls] += ms;
            P.bytes[r.cls] += r.bytes;
            P.flops[r.cls] += r.flops;
        }
        P.pool.push_back(r.a);
        P.pool.push_back(r.b);
    }
    P.pending.clear();
}

template <class T> std::unique_ptr<Solver<T>>& solver_slot(elder_ctx* ctx);
template <> std::unique_ptr<Solver<double>>& solver_slot<double>(elder_ctx* ctx)
{
    return ctx->s64;
}
template <> std::unique_ptr<Solver<float>>& solver_slot<float>(elder_ctx* ctx)
{
    return ctx->s32;
}

template <class T> void solver_alloc(elder_ctx* ctx, Solver<T>& sv, int cap);

// The solver of precision T with room for at least `cap` samples (its
// workspace is reallocated when a call needs more).
template <class T> Solver<T>& solver_reserve(elder_ctx* ctx, int cap)
{
    std::unique_ptr<Solver<T>>& up = solver_slot<T>(ctx);
    if (up && up->S >= cap) return *up;
    up.reset(new Solver<T>());
    solver_alloc<T>(ctx, *up, cap);
    return *up;
}

template <class T> void solver_alloc(elder_ctx* ctx, Solver<T>& sv, int cap)
{
    if (sv.S) return;
    // the coarsest level is solved by a dense inverse: bound its size
    if (2 * ctx->grids.back().N > MAX_COARSE_UNKNOWNS) {
        char buf[200];
        std::snprintf(buf, sizeof buf,
                      "coarsest grid %dx%dx%d has %d unknowns (> %d): the grid does not "
                      "coarsen far enough for the multigrid solver",
                      ctx->grids.back().nx, ctx->grids.back().ny, ctx->grids.back().nz,
                      2 * ctx->grids.back().N, MAX_COARSE_UNKNOWNS);
        throw Fail{ELDER_EINVAL, buf};
    }
    const int S = cap;
    const int L = (int)ctx->grids.size();
    for (int l = 0; l < L; ++l) {
        const Grid& G = ctx->grids[l];
        const size_t nN = (size_t)S * G.N;
        sv.Jm.push_back(dalloc<B4<typename Solver<T>::M>>(nN * 27));
        sv.mem.add(sv.Jm.back());
        if (l == 0) {
            if (std::is_same<T, typename Solver<T>::M>::value) {
                sv.J0 = reinterpret_cast<B4<T>*>(sv.Jm[0]);  // one array serves both
            } else {
                sv.J0 = dalloc<B4<T>>(nN * 27);
                sv.mem.add(sv.J0);
            }
        }
        sv.Dinv.push_back(dalloc<B4<T>>(nN));
        sv.mem.add(sv.Dinv.back());
        if (G.nz + 1 <= kMaxLine) {
            sv.zMi.push_back(dalloc<B4<T>>(nN));
            sv.mem.add(sv.zMi.back());
            sv.zC.push_back(dalloc<B4<T>>(nN));
            sv.mem.add(sv.zC.back());
        } else {
            sv.zMi.push_back(nullptr);
            sv.zC.push_back(nullptr);
        }
        // the ILU smoother's factors on every smoothed level (the coarsest
        // is solved by its dense inverse)
        if (ctx->cfg.smoother == ELDER_SMOOTH_ILU && l < L - 1) {
            sv.F.push_back(dalloc<B4<typename Solver<T>::M>>(nN * 27));
            sv.mem.add(sv.F.back());
            sv.Fd.push_back(dalloc<B4<T>>(nN));
            sv.mem.add(sv.Fd.back());
        } else {
            sv.F.push_back(nullptr);
            sv.Fd.push_back(nullptr);
        }
        for (auto* vec : {&sv.mb, &sv.mx, &sv.mx2, &sv.mr}) {
            vec->push_back(dalloc<V2<T>>(nN));
            sv.mem.add(vec->back());
        }
    }
    const size_t n0 = (size_t)S * ctx->grids[0].N;
    for (V2<T>** q : {&sv.x, &sv.r, &sv.rh, &sv.p, &sv.v, &sv.s, &sv.t, &sv.ph, &sv.sh, &sv.b,
                      &sv.xbest, &sv.xd}) {
        *q = dalloc<V2<T>>(n0);
        sv.mem.add(*q);
    }
    const int nc = 2 * ctx->grids.back().N;
    sv.Ainv = dalloc<double>((size_t)S * nc * nc);
    sv.mem.add(sv.Ainv);
    sv.work = dalloc<double>((size_t)S * nc * 2 * nc);
    sv.mem.add(sv.work);
    sv.S = S;
}

// Re-discretised Jacobians on every level (Section 5.1): level 0 at the
// current iterate, coarser levels at the injected state with the averaged
// coefficients; then the block-diagonal inverses and the coarse inverse.
template <class T>
void assemble(elder_ctx* ctx, Solver<T>& sv, int S, const double* phi0,
              const double* K0, const double* p0, const double* c0,
              const Phys& ph, const int* mask, int mstride, int n_active,
              cudaStream_t st)
{
    const int L = (int)ctx->grids.size();
    for (int l = 0; l < L; ++l) {
        const Grid& G = ctx->grids[l];
        const double* phi = l == 0 ? phi0 : ctx->phi[l];
        const double* K = l == 0 ? K0 : ctx->K[l];
        const double* p = l == 0 ? p0 : ctx->pl[l];
        const double* c = l == 0 ? c0 : ctx->cl[l];
        V2<T>* nodeT = reinterpret_cast<V2<T>*>(ctx->jn[l]);
        V2<T>* cellT = reinterpret_cast<V2<T>*>(ctx->jc[l]);
        if (l > 0) {
            const double* pf = l == 1 ? p0 : ctx->pl[l - 1];
            const double* cf = l == 1 ? c0 : ctx->cl[l - 1];
            launch_inject<T>(ctx->grids[l - 1], G, pf, cf, ctx->pl[l], ctx->cl[l], nodeT,
                             ph.rho0 * ph.g, mask, mstride, S, st);
        }
        const int pi = prof_begin(ctx, st);
        using M = typename Solver<T>::M;
        B4<T>* JT = (l == 0 && !std::is_same<T, M>::value) ? sv.J0 : nullptr;
        // the cell inputs of every level were converted once for the step
        // (average_coefficients); the coarse node inputs came with the
        // injection, the finest level's are converted here
        launch_jacobian<T, M>(G, ph, ctx->bc[l], phi, K, p, c, JT, sv.Jm[l], sv.Dinv[l], cellT,
                              nodeT, mask, mstride, S, st, l == 0 ? 1 : 2);
        // the vertical lines' block-LU factors for the z-line sweeps
        if (sv.zMi[l])
            launch_zline_factor<T, M>(G, sv.Jm[l], sv.Dinv[l], ctx->bc[l], sv.zMi[l], sv.zC[l],
                                      mask, mstride, S, st);
        // the multicolour ILU factors for the ILU sweeps
        if (sv.F[l])
            launch_ilu_factor<T, M>(G, sv.Jm[l], sv.Dinv[l], ctx->bc[l], sv.F[l], sv.Fd[l],
                                    ctx->cfg.ilu_beta, mask, mstride, S, st);
        prof_end(ctx, pi, ELDER_K_JACOBIAN, G, JT ? (int)sizeof(T) : 0, (int)sizeof(M), n_active,
                 st, (sv.zMi[l] ? 1 : 0) | (sv.F[l] ? 2 : 0));
    }
    launch_coarse_inverse<typename Solver<T>::M>(ctx->grids.back(), ctx->bc.back(), sv.Jm.back(),
                                                 sv.work,
                             sv.Ainv, mask, mstride, S, st);
    CKL();
}

// Coefficients of the coarse grids (cell averages) and the cell inputs of
// every level's Jacobian in the assembly type T, once per step.
template <class T>
void average_coefficients(elder_ctx* ctx, int S, const double* phi0,
                          const double* K0, cudaStream_t st)
{
    for (size_t l = 1; l < ctx->grids.size(); ++l) {
        const double* pf = l == 1 ? phi0 : ctx->phi[l - 1];
        const double* kf = l == 1 ? K0 : ctx->K[l - 1];
        launch_average_cells(ctx->grids[l - 1], ctx->grids[l], pf, kf, ctx->phi[l],
                             ctx->K[l], ctx->cfg.coarse_K_harmonic, S, st);
    }
    for (size_t l = 0; l < ctx->grids.size(); ++l)
        launch_cell_inputs<T>(ctx->grids[l], ctx->cfg.mu, l == 0 ? phi0 : ctx->phi[l],
                              l == 0 ? K0 : ctx->K[l], reinterpret_cast<V2<T>*>(ctx->jc[l]),
                              S, st);
    CKL();
}

// One V-cycle: out = M b on level l (masked by the Krylov flags).
template <class T>
void vcycle(elder_ctx* ctx, Solver<T>& sv, int l, const V2<T>* b, V2<T>* out,
            int trans, int S, cudaStream_t st)
{
    const int L = (int)ctx->grids.size();
    const Grid& G = ctx->grids[l];
    const int* mask = &ctx->ks[0].active;
    if (l == L - 1) {
        launch_coarse_apply<T>(G, sv.Ainv, b, out, trans, mask, KSTRIDE, S, st);
        return;
    }
    const elder_config& cf = ctx->cfg;
    const int nu1 = std::max(1, cf.nu1), nu2 = std::max(0, ctx->nu2_now);
    const int sweeps = nu1 + nu2;
    V2<T>* bufA = out;
    V2<T>* bufB = sv.mx2[l];
    // choose the first buffer so that the last sweep lands in `out`
    V2<T>* cur = ((sweeps - 1) % 2 == 0) ? bufA : bufB;
    V2<T>* oth = (cur == bufA) ? bufB : bufA;
    using M = typename Solver<T>::M;
    const int na = ctx->n_active_k;
    const int bs_sm = ctx->bs[ELDER_K_SMOOTH], bs_mr = ctx->bs[ELDER_K_MGRES];
    const int bs_zl = ctx->bs[ELDER_K_SMOOTH0], spc_zl = ctx->spc[ELDER_K_SMOOTH0];
    // (the transposed residual keeps one sample per CTA: two spill registers)
    const int spc_mr = trans ? 1 : ctx->spc[ELDER_K_MGRES];
    const bool line = ctx->smoother_now == ELDER_SMOOTH_ZLINE && G.nz + 1 <= kMaxLine;
    // the non-transposed z-line sweep substitutes with the line factors of
    // the assembly; the transposed one (adjoint solves) factors as it goes
    const bool fact = line && !trans && sv.zMi[l];
    // the ILU sweeps keep their triangular solves in the level's residual
    // vector (free until the restriction's residual is formed)
    const bool ilu = ctx->smoother_now == ELDER_SMOOTH_ILU && sv.F[l];
    auto sweep = [&](const V2<T>* xin, V2<T>* xout) {
        if (ilu && xin == nullptr) {
            launch_ilu_apply<T, M>(G, sv.F[l], sv.Fd[l], ctx->bc[l], b, sv.mr[l], nullptr, xout,
                                   ctx->omega_now, trans, 1, mask, KSTRIDE, S, st);
        } else if (ilu) {
            launch_mg_residual<T, M>(G, sv.Jm[l], ctx->bc[l], b, xin, sv.mr[l], trans, mask,
                                     KSTRIDE, S, st, bs_mr, spc_mr);
            launch_ilu_apply<T, M>(G, sv.F[l], sv.Fd[l], ctx->bc[l], sv.mr[l], sv.mr[l], xin,
                                   xout, ctx->omega_now, trans, 2, mask, KSTRIDE, S, st);
        } else if (fact && xin == nullptr) {
            launch_zline_apply<T, M>(G, sv.Jm[l], sv.zMi[l], sv.zC[l], ctx->bc[l], b, nullptr,
                                     xout, ctx->omega_now, mask, KSTRIDE, S, st, 1, bs_zl, spc_zl);
        } else if (fact) {
            launch_mg_residual<T, M>(G, sv.Jm[l], ctx->bc[l], b, xin, sv.mr[l], trans, mask,
                                     KSTRIDE, S, st, bs_mr, spc_mr);
            launch_zline_apply<T, M>(G, sv.Jm[l], sv.zMi[l], sv.zC[l], ctx->bc[l], sv.mr[l], xin,
                                     xout, ctx->omega_now, mask, KSTRIDE, S, st, 2, bs_zl, spc_zl);
        } else if (line && xin == nullptr) {
            launch_smooth_zline<T, M>(G, sv.Jm[l], sv.Dinv[l], ctx->bc[l], b, xin, xout,
                                      ctx->omega_now, trans, mask, KSTRIDE, S, st, 1);
        } else if (line) {
            // residual at full stream rate into the level's residual vector
            // (free once the restriction has been made), then the line solves
            launch_mg_residual<T, M>(G, sv.Jm[l], ctx->bc[l], b, xin, sv.mr[l], trans, mask,
                                     KSTRIDE, S, st, bs_mr);
            launch_smooth_zline<T, M>(G, sv.Jm[l], sv.Dinv[l], ctx->bc[l], sv.mr[l], xin, xout,
                                      ctx->omega_now, trans, mask, KSTRIDE, S, st, 2);
        } else
            launch_smooth<T, M>(G, sv.Jm[l], sv.Dinv[l], ctx->bc[l], b, xin, xout, ctx->omega_now,
                                trans, mask, KSTRIDE, S, st, bs_sm);
    };
    int pi = prof_begin(ctx, st);
    sweep(nullptr, cur);
    prof_end(ctx, pi, ELDER_K_SMOOTH0, G, sizeof(T), sizeof(M), na, st,
             ilu ? 3 : (fact ? 2 : -1));
    for (int q = 1; q < nu1; ++q) {
        pi = prof_begin(ctx, st);
        sweep(cur, oth);
        prof_end(ctx, pi, ELDER_K_SMOOTH, G, sizeof(T), sizeof(M), na, st);
        std::swap(cur, oth);
    }
    pi = prof_begin(ctx, st);
    launch_mg_residual<T, M>(G, sv.Jm[l], ctx->bc[l], b, cur, sv.mr[l], trans, mask, KSTRIDE, S,
                             st, bs_mr, spc_mr);
    prof_end(ctx, pi, ELDER_K_MGRES, G, sizeof(T), sizeof(M), na, st);
    launch_restrict<T>(G, ctx->grids[l + 1], ctx->bc[l + 1], sv.mr[l], sv.mb[l + 1], mask,
                       KSTRIDE, S, st);
    vcycle<T>(ctx, sv, l + 1, sv.mb[l + 1], sv.mx[l + 1], trans, S, st);
    launch_prolong_add<T>(G, ctx->grids[l + 1], ctx->bc[l], sv.mx[l + 1], cur, mask, KSTRIDE,
                          S, st);
    for (int q = 0; q < nu2; ++q) {
        pi = prof_begin(ctx, st);
        sweep(cur, oth);
        prof_end(ctx, pi, ELDER_K_SMOOTH, G, sizeof(T), sizeof(M), na, st);
        std::swap(cur, oth);
    }
    if (cur != out) CK(cudaMemcpyAsync(out, cur, sizeof(V2<T>) * (size_t)S * G.N,
                                       cudaMemcpyDeviceToDevice, st));
}

// Autotuner: threads per block of the three J-streaming kernel classes,
// chosen once per context and precision by timing every candidate (CUDA
// events, 3 launches after a warm-up) on the first assembled level-0
// operator of a step with all S samples active.
template <class T>
void autotune(elder_ctx* ctx, Solver<T>& sv, int S, cudaStream_t st)
{
    const int idx = std::is_same<T, float>::value ? 1 : 0;
    if (ctx->tuned[idx] || !ctx->cfg.autotune) return;
    if (ctx->cfg.autotune == 2) {  // fixed: two samples per CTA, default blocks
        ctx->spc[ELDER_K_MGRES] = ctx->spc[ELDER_K_SMOOTH0] = 2;
        ctx->tuned[idx] = true;
        return;
    }
    using M = typename Solver<T>::M;
    const Grid& G = ctx->grids[0];
    const size_t nv = (size_t)S * G.N;
    CK(cudaMemsetAsync(sv.mb[0], 0, sizeof(V2<T>) * nv, st));
    CK(cudaMemsetAsync(sv.mx[0], 0, sizeof(V2<T>) * nv, st));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const int cand[3] = {kMinBS, kBS, kMaxBS};
    const int cls[3] = {ELDER_K_SMOOTH, ELDER_K_SPMV, ELDER_K_MGRES};
    for (int c = 0; c < 3; ++c) {
        float best = 1e30f;
        for (int q = 0; q < 3; ++q) {
            auto run = [&]() {
                if (c == 0)
                    launch_smooth<T, M>(G, sv.Jm[0], sv.Dinv[0], ctx->bc[0], sv.mb[0], sv.mx[0],
                                        sv.mx2[0], ctx->cfg.omega, 0, nullptr, 0, S, st, cand[q]);
                else if (c == 1)
                    launch_spmv<T>(G, sv.J0, ctx->bc[0], sv.mx[0], sv.mx2[0], 0, 0, nullptr,
                                   nullptr, nullptr, 0, S, st, cand[q]);
                else
                    launch_mg_residual<T, M>(G, sv.Jm[0], ctx->bc[0], sv.mb[0], sv.mx[0],
                                             sv.mx2[0], 0, nullptr, 0, S, st, cand[q]);
            };
            run();
            CK(cudaEventRecord(e0, st));
            for (int r = 0; r < 3; ++r) run();
            CK(cudaEventRecord(e1, st));
            CK(cudaEventSynchronize(e1));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            ctx->tune_ms[c][q] = ms / 3.f;
            if (ms < best) {
                best = ms;
                ctx->bs[cls[c]] = cand[q];
            }
        }
    }
    // (threads per block, samples per CTA) of the multigrid residual and of
    // the factored z-line sweep from x = 0 (the default V(1,0) cycle's only
    // sweep); two samples per CTA give a thread two independent stencil rows
    // or line recursions
    if (sv.zMi[0] && G.nz + 1 <= kMaxLine) {
        const int bsm[3] = {kMinBS, kBS, kMaxBS}, bsz[3] = {64, 128, 256};
        for (int c = 0; c < 2; ++c) {
            float best = 1e30f;
            for (int q = 0; q < 6; ++q) {
                const int bsq = c == 0 ? bsm[q % 3] : bsz[q % 3], spq = 1 + q / 3;
                auto run = [&]() {
                    if (c == 0)
                        launch_mg_residual<T, M>(G, sv.Jm[0], ctx->bc[0], sv.mb[0], sv.mx[0],
                                                 sv.mx2[0], 0, nullptr, 0, S, st, bsq, spq);
                    else
                        launch_zline_apply<T, M>(G, sv.Jm[0], sv.zMi[0], sv.zC[0], ctx->bc[0],
                                                 sv.mb[0], nullptr, sv.mx2[0], 1.0, nullptr, 0, S,
                                                 st, 1, bsq, spq);
                };
                run();
                CK(cudaEventRecord(e0, st));
                for (int r = 0; r < 3; ++r) run();
                CK(cudaEventRecord(e1, st));
                CK(cudaEventSynchronize(e1));
                float ms = 0.f;
                CK(cudaEventElapsedTime(&ms, e0, e1));
                ctx->tune2_ms[c][q] = ms / 3.f;
                if (ms < best) {
                    best = ms;
                    const int cl = c == 0 ? ELDER_K_MGRES : ELDER_K_SMOOTH0;
                    ctx->bs[cl] = bsq;
                    ctx->spc[cl] = spq;
                }
            }
        }
    }
    CK(cudaEventDestroy(e0));
    CK(cudaEventDestroy(e1));
    CKL();
    ctx->tuned[idx] = true;
}

template <class T>
void bicg_iteration(elder_ctx* ctx, Solver<T>& sv, int trans, double rtol, int maxit,
                    int S, cudaStream_t st)
{
    const Grid& G = ctx->grids[0];
    const int bs_mv = ctx->bs[ELDER_K_SPMV];
    const int nb_mv = nblocks(G.N, 32);  // per-warp partials of the stencil products
    KScal* ks = ctx->ks;
    const int* mask = &ks[0].active;
    launch_bicg_p<T>(G, sv.r, sv.v, sv.p, ks, S, st);
    vcycle<T>(ctx, sv, 0, sv.p, sv.ph, trans, S, st);
    int pi = prof_begin(ctx, st);
    launch_spmv<T>(G, sv.J0, ctx->bc[0], sv.ph, sv.v, trans, 1, sv.rh, ctx->partial, mask,
                   KSTRIDE, S, st, bs_mv);
    prof_end(ctx, pi, ELDER_K_SPMV, G, sizeof(T), sizeof(T), ctx->n_active_k, st);
    launch_bicg_finalize(1, ctx->partial, nb_mv, ks, rtol, maxit, S, st);
    launch_bicg_s<T>(G, sv.r, sv.v, sv.s, nullptr, ks, S, st);
    vcycle<T>(ctx, sv, 0, sv.s, sv.sh, trans, S, st);
    pi = prof_begin(ctx, st);
    launch_spmv<T>(G, sv.J0, ctx->bc[0], sv.sh, sv.t, trans, 2, sv.s, ctx->partial, mask,
                   KSTRIDE, S, st, bs_mv);
    prof_end(ctx, pi, ELDER_K_SPMV, G, sizeof(T), sizeof(T), ctx->n_active_k, st);
    launch_bicg_finalize(2, ctx->partial, nb_mv, ks, rtol, maxit, S, st);
    launch_bicg_xr<T>(G, sv.ph, sv.sh, sv.s, sv.t, sv.rh, sv.x, sv.r, ctx->partial, ks, S, st);
    launch_bicg_finalize(3, ctx->partial, bicg_xr_blocks(G.N), ks, rtol, maxit, S, st);
}

__global__ void k_arm_krylov(KScal* ks, const NScal* ns, int S)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    ks[s].active = ns ? ns[s].active : 1;
    ks[s].iters = 0;
    ks[s].status = 0;
}

bool any_krylov_active(elder_ctx* ctx, int S, cudaStream_t st)
{
    CK(cudaMemcpyAsync(ctx->h_ks, ctx->ks, sizeof(KScal) * S, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    prof_drain(ctx);
    int n = 0;
    for (int s = 0; s < S; ++s) n += ctx->h_ks[s].active ? 1 : 0;
    ctx->n_active_k = n;
    return n > 0;
}

// Solve A x = b (or A^T x = b) on the interior system for the samples whose
// Newton flag is set (all samples when ns == nullptr).  b and the result
// live in sv.b and sv.x.  With keep_best, a sample that stops without
// reaching rtol returns its iterate of smallest residual instead of the last.
template <class T>
void bicgstab(elder_ctx* ctx, Solver<T>& sv, int trans, double rtol, int maxit,
              const NScal* ns, int S, cudaStream_t st, int keep_best = 0)
{
    const Grid& G = ctx->grids[0];
    k_arm_krylov<<<nblocks(S, 128), 128, 0, st>>>(ctx->ks, ns, S);
    count_launch(1);
    ctx->n_active_k = ns ? ctx->n_active_newton : S;
    launch_bicg_init<T>(G, ctx->bc[0], sv.b, sv.x, sv.r, sv.rh, sv.p, sv.v, ctx->partial,
                        ctx->ks, S, st);
    launch_bicg_finalize(0, ctx->partial, ctx->nblk0, ctx->ks, rtol, maxit, S, st);
    if (keep_best)
        CK(cudaMemsetAsync(sv.xbest, 0, sizeof(V2<T>) * S * G.N, st));
    CKL();
    // The captured finalize kernels bake in rtol and maxit; graphs are keyed
    // on (S, trans) only, so they serve the configured values only, and are
    // bypassed while per-launch events are recorded.
    const bool use_exec = ctx->cfg.use_graphs != 0 && !ctx->prof.on &&
                          rtol == ctx->cfg.lin_rtol && maxit == ctx->cfg.lin_maxit &&
                          ctx->smoother_now == ctx->cfg.smoother &&
                          ctx->omega_now == configured_omega(ctx->cfg) &&
                          ctx->nu2_now == ctx->cfg.nu2;
    cudaGraphExec_t exec = nullptr;
    long long per_replay = 0;
    if (use_exec) {
        auto key = std::make_pair(S, trans);
        auto it = sv.graphs.find(key);
        if (it == sv.graphs.end()) {
            cudaStream_t cs;
            CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
            cudaGraph_t g;
            const long long before = g_launches.load();
            CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
            bicg_iteration<T>(ctx, sv, trans, rtol, maxit, S, cs);
            CK(cudaStreamEndCapture(cs, &g));
            per_replay = g_launches.load() - before;
            g_launches.fetch_sub(per_replay);  // captured, not launched
            CK(cudaGraphInstantiate(&exec, g, 0));
            CK(cudaGraphDestroy(g));
            CK(cudaStreamDestroy(cs));
            sv.graphs[key] = exec;
            sv.graph_kernels[key] = per_replay;
        } else {
            exec = it->second;
            per_replay = sv.graph_kernels[key];
        }
    }
    const int poll = ctx->prof.on ? 1 : 2;
    for (int it = 0; it < maxit; ++it) {
        if (it % poll == 0 && !any_krylov_active(ctx, S, st)) break;
        if (use_exec) {
            CK(cudaGraphLaunch(exec, st));
            count_launch((int)per_replay);
        } else {
            bicg_iteration<T>(ctx, sv, trans, rtol, maxit, S, st);
        }
        if (keep_best) launch_bicg_keep<T>(G, sv.x, sv.xbest, ctx->ks, 1, S, st);
        CKL();
    }
    if (keep_best) launch_bicg_keep<T>(G, sv.x, sv.xbest, ctx->ks, 2, S, st);
}

// Solver settings of one Newton solve (Section 2.3 and Section 5.1).
struct NewtonSettings {
    double lin_rtol;
    int lin_maxit, ls_max, newton_maxit, estimate, keep_best, smoother;
    double omega;
    int nu2;  // post-smoothing sweeps of the V-cycle
};

NewtonSettings configured_settings(const elder_config& cf)
{
    return NewtonSettings{cf.lin_rtol, cf.lin_maxit, cf.ls_max, cf.newton_maxit,
                          cf.newton_estimate, 0, cf.smoother, configured_omega(cf), cf.nu2};
}

// Damping of the robust re-solve's z-line smoother: on the steepest first
// steps of rough fields 0.5 converges where larger values need more
// iterations or stall.
constexpr double kRobustOmega = 0.5;

// Settings of the last re-solve of a failed sample: the z-line smoother, a
// tighter and longer Krylov solve that returns its best iterate, more step
// halvings and Newton iterations, and only the plain correction-size stop.
// Steep initial fronts on rough permeability fields make the point smoother
// diverge locally and the Krylov solve stall.
NewtonSettings robust_settings(const elder_config& cf)
{
    NewtonSettings r = configured_settings(cf);
    r.smoother = ELDER_SMOOTH_ZLINE;
    r.omega = kRobustOmega;
    r.nu2 = std::max(cf.nu2, 1);
    r.lin_rtol = std::min(cf.lin_rtol, 1e-6);
    r.lin_maxit = std::max(20 * cf.lin_maxit, 2000);
    r.ls_max = std::max(cf.ls_max, 16);
    r.newton_maxit = std::max(2 * cf.newton_maxit, 50);
    r.estimate = 0;
    r.keep_best = 1;
    return r;
}

// Sample 0's Krylov solve ended by reaching its tolerance.
bool krylov_converged(elder_ctx* ctx, cudaStream_t st)
{
    CK(cudaMemcpyAsync(ctx->h_ks, ctx->ks, sizeof(KScal), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return ctx->h_ks[0].status == 0 && !ctx->h_ks[0].active;
}

int finish_step(elder_ctx* ctx, int S, int32_t* status, elder_stats* stats);

// ---------------------------------------------------------------------------
// Device-controlled step (use_graphs = 2): the whole implicit step is one
// captured CUDA graph.  Its Newton iterations, the BiCGStab iterations of
// each Newton system and the line search are while nodes whose conditions
// kernels set on the device from the per-sample flags (any sample still
// iterating, and an iteration cap); the host launches the graph and reads
// the per-sample results once.
// ---------------------------------------------------------------------------

// Condition of a while node: some sample's flag (flags[s * stride]) is set
// and fewer than `limit` bodies have run.  first = 1 (before the loop) resets
// the loop's counter; otherwise one more body has run, which is also added
// to the step's running total for that loop (the launch count of a replay).
__global__ void k_loop_cond(cudaGraphConditionalHandle h, const int* __restrict__ flags,
                            int stride, int S, int* counter, int* total, int limit, int first)
{
    int any = 0;
    for (int s = threadIdx.x; s < S; s += blockDim.x) any |= flags[(size_t)s * stride];
    any = __syncthreads_or(any);
    if (threadIdx.x != 0) return;
    const int c = first ? 0 : *counter + 1;
    *counter = c;
    if (!first) *total += 1;
    cudaGraphSetConditional(h, (any && c < limit) ? 1u : 0u);
}

void launch_loop_cond(cudaGraphConditionalHandle h, const int* flags, int stride, int S,
                      int* counter, int* total, int limit, int first, cudaStream_t st)
{
    count_launch(1);
    k_loop_cond<<<1, 256, 0, st>>>(h, flags, stride, S, counter, total, limit, first);
}

// Newton scalars at the start of a step: every sample iterating, full step.
__global__ void k_newton_init(NScal* ns, int S)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    NScal z{};
    z.active = 1;
    z.ls_active = 1;
    z.lambda = 1.0;
    ns[s] = z;
}

// A sample still iterating after the Newton loop's cap has run out of
// Newton iterations.
__global__ void k_newton_cap(NScal* ns, int S)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S || !ns[s].active) return;
    ns[s].active = 0;
    ns[s].status = ELDER_SAMPLE_NEWTON_MAXIT;
}

// Appends a while node after the current dependencies of the capture on
// `cs` (handle created on the capturing graph), makes it the capture's only
// dependency and returns its body graph.
cudaGraph_t append_while(cudaStream_t cs, cudaGraphConditionalHandle h)
{
    cudaStreamCaptureStatus stt;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* ed = nullptr;
    size_t nd = 0;
    CK(cudaStreamGetCaptureInfo(cs, &stt, nullptr, &g, &deps, &ed, &nd));
    // zeroed storage: the struct's union has no default constructor
    alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
    std::memset(raw, 0, sizeof raw);
    cudaGraphNodeParams& prm = *reinterpret_cast<cudaGraphNodeParams*>(raw);
    prm.type = cudaGraphNodeTypeConditional;
    prm.conditional.handle = h;
    prm.conditional.type = cudaGraphCondTypeWhile;
    prm.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, g, deps, ed, nd, &prm));
    CK(cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1,
                                           cudaStreamSetCaptureDependencies));
    return prm.conditional.phGraph_out[0];
}

// Captures the step (the same launches, in the same order, as the
// host-driven loop of step_impl) into out.exec.  Returns false, with the
// reason in ctx->step_graph_note, when the capture fails; the caller then
// runs the host-driven loop.
template <class T>
bool build_step_graph(elder_ctx* ctx, Solver<T>& sv, int S, const double* phi, const double* K,
                      double* p, double* c, double dt, const NewtonSettings& set, int order,
                      double* p_hist, double* c_hist, StepGraph& out)
{
    const elder_config& cf = ctx->cfg;
    const Grid& G = ctx->grids[0];
    const Phys ph = make_phys(cf, dt);
    const size_t nN = (size_t)S * G.N;
    const int nb = ctx->nblk0;
    NScal* ns = ctx->ns;
    KScal* ks = ctx->ks;
    const int* nmask = &ns[0].active;
    const int* lsmask = &ns[0].ls_active;
    const int* kmask = &ks[0].active;
    int* cnt = ctx->loopc;      // loop counters: Newton, Krylov, line search
    int* tot = ctx->loopc + 3;  // bodies run in this step, per loop
    const auto mode = cudaStreamCaptureModeThreadLocal;
    cudaStream_t cs = nullptr, cb1 = nullptr, cb2 = nullptr;
    cudaGraph_t g = nullptr;
    const long long launches0 = g_launches.load();
    try {
        CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        CK(cudaStreamCreateWithFlags(&cb1, cudaStreamNonBlocking));
        CK(cudaStreamCreateWithFlags(&cb2, cudaStreamNonBlocking));
        CK(cudaGraphCreate(&g, 0));
        cudaGraphConditionalHandle hN, hK, hL;
        CK(cudaGraphConditionalHandleCreate(&hN, g, 0, 0));
        // ---- prologue ----
        CK(cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, mode));
        long long k0 = g_launches.load();
        CK(cudaMemsetAsync(tot, 0, 3 * sizeof(int), cs));
        CK(cudaMemcpyAsync(ctx->p_old, p, sizeof(double) * nN, cudaMemcpyDeviceToDevice, cs));
        CK(cudaMemcpyAsync(ctx->c_old, c, sizeof(double) * nN, cudaMemcpyDeviceToDevice, cs));
        if (p_hist) {
            launch_extrapolate(G, order, ctx->p_old, ctx->c_old, p_hist, c_hist,
                               order == 2 ? p_hist + nN : nullptr,
                               order == 2 ? c_hist + nN : nullptr, p, c, S, cs);
            if (order == 2) {
                CK(cudaMemcpyAsync(p_hist + nN, p_hist, sizeof(double) * nN,
                                   cudaMemcpyDeviceToDevice, cs));
                CK(cudaMemcpyAsync(c_hist + nN, c_hist, sizeof(double) * nN,
                                   cudaMemcpyDeviceToDevice, cs));
            }
            CK(cudaMemcpyAsync(p_hist, ctx->p_old, sizeof(double) * nN, cudaMemcpyDeviceToDevice,
                               cs));
            CK(cudaMemcpyAsync(c_hist, ctx->c_old, sizeof(double) * nN, cudaMemcpyDeviceToDevice,
                               cs));
        }
        launch_impose_dirichlet(G, ctx->bc[0], ctx->cval, p, c, S, cs);
        average_coefficients<T>(ctx, S, phi, K, cs);
        k_newton_init<<<nblocks(S, 128), 128, 0, cs>>>(ns, S);
        count_launch(1);
        launch_residual(G, ph, ctx->bc[0], ctx->cval, phi, K, p, c, ctx->p_old, ctx->c_old,
                        ctx->R, ctx->partial, ctx->partial2, nullptr, 0, S, cs, ctx->qf);
        launch_norm_finalize(ctx->partial, ctx->partial2, nb, ns, 0, S, cs);
        launch_loop_cond(hN, nmask, NSTRIDE, S, cnt + 0, tot + 0, set.newton_maxit, 1, cs);
        CKL();
        out.k_pro = g_launches.load() - k0;
        // ---- Newton iteration ----
        cudaGraph_t bN = append_while(cs, hN);
        CK(cudaGraphConditionalHandleCreate(&hK, bN, 0, 0));
        CK(cudaGraphConditionalHandleCreate(&hL, bN, 0, 0));
        CK(cudaStreamBeginCaptureToGraph(cb1, bN, nullptr, nullptr, 0, mode));
        k0 = g_launches.load();
        assemble<T>(ctx, sv, S, phi, K, p, c, ph, nmask, NSTRIDE, S, cb1);
        launch_newton_rhs<T>(G, ctx->R, sv.b, ns, S, cb1);
        ctx->smoother_now = set.smoother;
        ctx->omega_now = set.omega;
        ctx->nu2_now = set.nu2;
        k_arm_krylov<<<nblocks(S, 128), 128, 0, cb1>>>(ks, ns, S);
        count_launch(1);
        launch_bicg_init<T>(G, ctx->bc[0], sv.b, sv.x, sv.r, sv.rh, sv.p, sv.v, ctx->partial, ks,
                            S, cb1);
        launch_bicg_finalize(0, ctx->partial, nb, ks, set.lin_rtol, set.lin_maxit, S, cb1);
        launch_loop_cond(hK, kmask, KSTRIDE, S, cnt + 1, tot + 1, set.lin_maxit, 1, cb1);
        // BiCGStab iterations
        cudaGraph_t bK = append_while(cb1, hK);
        CK(cudaStreamBeginCaptureToGraph(cb2, bK, nullptr, nullptr, 0, mode));
        long long k1 = g_launches.load();
        bicg_iteration<T>(ctx, sv, 0, set.lin_rtol, set.lin_maxit, S, cb2);
        launch_loop_cond(hK, kmask, KSTRIDE, S, cnt + 1, tot + 1, set.lin_maxit, 0, cb2);
        CKL();
        out.k_kb = g_launches.load() - k1;
        CK(cudaStreamEndCapture(cb2, &bK));
        ctx->smoother_now = cf.smoother;
        ctx->omega_now = configured_omega(cf);
        ctx->nu2_now = cf.nu2;
        // line search: the full step, the stop test on its correction, then
        // trial residuals and halvings while any sample's search runs
        launch_newton_trial<T>(G, p, c, sv.x, ctx->pt, ctx->ct, ctx->partial2, ns, S, cb1);
        launch_newton_predict(ctx->partial2, nb, ns, cf.newton_tol_p, cf.newton_tol_c,
                              set.estimate, S, cb1);
        launch_loop_cond(hL, lsmask, NSTRIDE, S, cnt + 2, tot + 2, set.ls_max + 1, 1, cb1);
        cudaGraph_t bL = append_while(cb1, hL);
        CK(cudaStreamBeginCaptureToGraph(cb2, bL, nullptr, nullptr, 0, mode));
        k1 = g_launches.load();
        launch_residual(G, ph, ctx->bc[0], ctx->cval, phi, K, ctx->pt, ctx->ct, ctx->p_old,
                        ctx->c_old, ctx->Rt, ctx->partial, ctx->partial3, lsmask, NSTRIDE, S, cb2,
                        ctx->qf);
        launch_norm_finalize(ctx->partial, ctx->partial3, nb, ns, 1, S, cb2);
        launch_newton_ls_finalize(nullptr, ctx->partial2, nb, ns, set.ls_max, S, cb2);
        launch_newton_trial<T>(G, p, c, sv.x, ctx->pt, ctx->ct, ctx->partial2, ns, S, cb2);
        launch_loop_cond(hL, lsmask, NSTRIDE, S, cnt + 2, tot + 2, set.ls_max + 1, 0, cb2);
        CKL();
        out.k_lb = g_launches.load() - k1;
        CK(cudaStreamEndCapture(cb2, &bL));
        launch_newton_accept(G, p, c, ctx->pt, ctx->ct, ctx->R, ctx->Rt, ns, S, cb1);
        launch_newton_check(ns, ks, cf.newton_tol_p, cf.newton_tol_c, set.newton_maxit,
                            set.estimate, S, cb1);
        launch_loop_cond(hN, nmask, NSTRIDE, S, cnt + 0, tot + 0, set.newton_maxit, 0, cb1);
        CKL();
        out.k_nb = g_launches.load() - k0 - out.k_kb - out.k_lb;
        CK(cudaStreamEndCapture(cb1, &bN));
        // ---- epilogue ----
        k0 = g_launches.load();
        k_newton_cap<<<nblocks(S, 128), 128, 0, cs>>>(ns, S);
        count_launch(1);
        launch_newton_restore_failed(G, p, c, ctx->p_old, ctx->c_old, ns, S, cs);
        launch_mass_balance(G, ph, ctx->bc[0], phi, K, p, c, ctx->c_old, ctx->partial3, S, cs);
        launch_sum_partials(ctx->partial3, nb, ctx->mass, 3 * S, cs);
        CKL();
        out.k_epi = g_launches.load() - k0;
        CK(cudaStreamEndCapture(cs, &g));
        CK(cudaGraphInstantiate(&out.exec, g, 0));
        CK(cudaGraphDestroy(g));
        g = nullptr;
        for (cudaStream_t q : {cs, cb1, cb2}) cudaStreamDestroy(q);
        g_launches.store(launches0);  // captured, not launched
        return true;
    } catch (const Fail& f) {
        ctx->step_graph_note = f.msg;
        for (cudaStream_t q : {cb2, cb1, cs}) {
            if (!q) continue;
            cudaStreamCaptureStatus cst;
            if (cudaStreamIsCapturing(q, &cst) == cudaSuccess &&
                cst != cudaStreamCaptureStatusNone) {
                cudaGraph_t dropped = nullptr;
                cudaStreamEndCapture(q, &dropped);
                if (dropped && dropped != g) cudaGraphDestroy(dropped);
            }
        }
        if (g) cudaGraphDestroy(g);
        for (cudaStream_t q : {cs, cb1, cb2})
            if (q) cudaStreamDestroy(q);
        cudaGetLastError();
        ctx->smoother_now = cf.smoother;
        ctx->omega_now = configured_omega(cf);
        ctx->nu2_now = cf.nu2;
        g_launches.store(launches0);
        return false;
    }
}

// Replays (capturing on first use) the step graph of these arguments.
// Returns false when no graph could be built; the step has then not run.
template <class T>
bool step_graph(elder_ctx* ctx, Solver<T>& sv, int S, const double* phi, const double* K,
                double* p, double* c, double dt, cudaStream_t st, const NewtonSettings& set,
                int order, double* p_hist, double* c_hist)
{
    StepKey key;
    std::memset(&key, 0, sizeof key);
    key.S = S;
    key.order = p_hist ? order : 0;
    key.prec = (int)sizeof(T);
    key.newton_maxit = set.newton_maxit;
    key.lin_maxit = set.lin_maxit;
    key.ls_max = set.ls_max;
    key.estimate = set.estimate;
    key.smoother = set.smoother;
    key.nu2 = set.nu2;
    key.lin_rtol = set.lin_rtol;
    key.omega = set.omega;
    key.dt = dt;
    const void* ptrs[6] = {phi, K, p, c, p_hist, c_hist};
    for (int q = 0; q < 6; ++q) key.ptr[q] = ptrs[q];
    auto& cache = ctx->step_graphs;
    StepGraph sg;
    auto it = std::find_if(cache.begin(), cache.end(),
                           [&](const StepGraph& x) { return x.key == key; });
    if (it != cache.end()) {
        sg = *it;
        cache.erase(it);
    } else {
        sg.key = key;
        if (!build_step_graph<T>(ctx, sv, S, phi, K, p, c, dt, set, order, p_hist, c_hist, sg)) {
            ctx->step_graph_ok = false;
            return false;
        }
        if (cache.size() >= 4) {  // keep the four most recent argument sets
            cudaGraphExecDestroy(cache.front().exec);
            cache.erase(cache.begin());
        }
    }
    cache.push_back(sg);  // most recent last
    CK(cudaGraphLaunch(sg.exec, st));
    ctx->step_graph_replays += 1;
    CK(cudaMemcpyAsync(ctx->h_ns, ctx->ns, sizeof(NScal) * S, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(ctx->h_mass, ctx->mass, sizeof(double) * 3 * S, cudaMemcpyDeviceToHost,
                       st));
    CK(cudaMemcpyAsync(ctx->h_loopc, ctx->loopc, sizeof(int) * 8, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    count_launch((int)(sg.k_pro + sg.k_epi + ctx->h_loopc[3] * sg.k_nb +
                       ctx->h_loopc[4] * sg.k_kb + ctx->h_loopc[5] * sg.k_lb));
    return true;
}

template <class T>
int step_impl(elder_ctx* ctx, int S, const double* phi, const double* K, double* p,
              double* c, double dt, int32_t* status, elder_stats* stats, cudaStream_t st,
              const NewtonSettings& set, int order = 0, double* p_hist = nullptr,
              double* c_hist = nullptr, bool allow_graph = false)
{
    Solver<T>& sv = solver_reserve<T>(ctx, S);
    // the device-controlled step once the context is tuned, for the
    // configured (not the robust) settings and outside profiling
    const int tidx = std::is_same<T, float>::value ? 1 : 0;
    if (allow_graph && ctx->cfg.use_graphs == 2 && ctx->step_graph_ok && !ctx->prof.on &&
        !set.keep_best && (ctx->tuned[tidx] || !ctx->cfg.autotune) &&
        step_graph<T>(ctx, sv, S, phi, K, p, c, dt, st, set, order, p_hist, c_hist))
        return finish_step(ctx, S, status, stats);
    const elder_config& cf = ctx->cfg;
    const Grid& G = ctx->grids[0];
    const Phys ph = make_phys(cf, dt);
    const size_t nN = (size_t)S * G.N;
    const int nb = ctx->nblk0;
    NScal* ns = ctx->ns;
    const int* nmask = &ns[0].active;
    const int* lsmask = &ns[0].ls_active;

    CK(cudaMemcpyAsync(ctx->p_old, p, sizeof(double) * nN, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(ctx->c_old, c, sizeof(double) * nN, cudaMemcpyDeviceToDevice, st));
    if (p_hist) {
        // Newton starts from the extrapolation of u^n and the order history
        // levels (u^{n-1}[, u^{n-2}]); the history shifts by one level and
        // its first level receives u^n for the next call
        launch_extrapolate(G, order, ctx->p_old, ctx->c_old, p_hist, c_hist,
                           order == 2 ? p_hist + nN : nullptr, order == 2 ? c_hist + nN : nullptr,
                           p, c, S, st);
        if (order == 2) {
            CK(cudaMemcpyAsync(p_hist + nN, p_hist, sizeof(double) * nN, cudaMemcpyDeviceToDevice,
                               st));
            CK(cudaMemcpyAsync(c_hist + nN, c_hist, sizeof(double) * nN, cudaMemcpyDeviceToDevice,
                               st));
        }
        CK(cudaMemcpyAsync(p_hist, ctx->p_old, sizeof(double) * nN, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(c_hist, ctx->c_old, sizeof(double) * nN, cudaMemcpyDeviceToDevice, st));
    }
    launch_impose_dirichlet(G, ctx->bc[0], ctx->cval, p, c, S, st);
    average_coefficients<T>(ctx, S, phi, K, st);
    for (int s = 0; s < S; ++s) {
        NScal z;
        std::memset(&z, 0, sizeof(z));
        z.active = 1;
        z.ls_active = 1;
        z.lambda = 1.0;
        ctx->h_ns[s] = z;
    }
    CK(cudaMemcpyAsync(ns, ctx->h_ns, sizeof(NScal) * S, cudaMemcpyHostToDevice, st));
    int pi = prof_begin(ctx, st);
    launch_residual(G, ph, ctx->bc[0], ctx->cval, phi, K, p, c, ctx->p_old, ctx->c_old, ctx->R,
                    ctx->partial, ctx->partial2, nullptr, 0, S, st, ctx->qf);
    prof_end(ctx, pi, ELDER_K_RESIDUAL, G, 8, 8, S, st);
    launch_norm_finalize(ctx->partial, ctx->partial2, nb, ns, 0, S, st);
    CKL();

    for (int it = 0; it < set.newton_maxit; ++it) {
        CK(cudaMemcpyAsync(ctx->h_ns, ns, sizeof(NScal) * S, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        prof_drain(ctx);
        int na = 0;
        for (int s = 0; s < S; ++s) na += ctx->h_ns[s].active ? 1 : 0;
        if (na == 0) break;
        ctx->n_active_newton = na;
        ctx->n_active_ls = na;
        assemble<T>(ctx, sv, S, phi, K, p, c, ph, nmask, NSTRIDE, na, st);
        if (it == 0) autotune<T>(ctx, sv, S, st);
        launch_newton_rhs<T>(G, ctx->R, sv.b, ns, S, st);
        ctx->smoother_now = set.smoother;
        ctx->omega_now = set.omega;
        ctx->nu2_now = set.nu2;
        bicgstab<T>(ctx, sv, 0, set.lin_rtol, set.lin_maxit, ns, S, st, set.keep_best);
        ctx->smoother_now = cf.smoother;
        ctx->omega_now = configured_omega(cf);
        ctx->nu2_now = cf.nu2;
        for (int ls = 0; ls <= set.ls_max; ++ls) {
            launch_newton_trial<T>(G, p, c, sv.x, ctx->pt, ctx->ct, ctx->partial2, ns, S, st);
            // full step: samples whose correction meets the stop need no
            // trial residual (they drop out of its mask)
            if (ls == 0) {
                launch_newton_predict(ctx->partial2, nb, ns, cf.newton_tol_p, cf.newton_tol_c,
                                      set.estimate, S, st);
                if (ctx->prof.on) {  // the residual's work counts only the samples left
                    CK(cudaMemcpyAsync(ctx->h_ns, ns, sizeof(NScal) * S, cudaMemcpyDeviceToHost,
                                       st));
                    CK(cudaStreamSynchronize(st));
                    int nls = 0;
                    for (int s = 0; s < S; ++s) nls += ctx->h_ns[s].ls_active ? 1 : 0;
                    ctx->n_active_ls = nls;
                }
            }
            pi = prof_begin(ctx, st);
            launch_residual(G, ph, ctx->bc[0], ctx->cval, phi, K, ctx->pt, ctx->ct, ctx->p_old,
                            ctx->c_old, ctx->Rt, ctx->partial, ctx->partial3, lsmask, NSTRIDE,
                            S, st, ctx->qf);
            prof_end(ctx, pi, ELDER_K_RESIDUAL, G, 8, 8, ctx->n_active_ls, st);
            launch_norm_finalize(ctx->partial, ctx->partial3, nb, ns, 1, S, st);
            launch_newton_ls_finalize(nullptr, ctx->partial2, nb, ns, set.ls_max, S, st);
            CKL();
            CK(cudaMemcpyAsync(ctx->h_ns, ns, sizeof(NScal) * S, cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            prof_drain(ctx);
            int nls = 0;
            for (int s = 0; s < S; ++s) nls += ctx->h_ns[s].ls_active ? 1 : 0;
            ctx->n_active_ls = nls;
            if (nls == 0) break;
        }
        launch_newton_accept(G, p, c, ctx->pt, ctx->ct, ctx->R, ctx->Rt, ns, S, st);
        launch_newton_check(ns, ctx->ks, cf.newton_tol_p, cf.newton_tol_c, set.newton_maxit,
                            set.estimate, S, st);
        CKL();
    }
    // samples still active here ran out of Newton iterations
    CK(cudaMemcpyAsync(ctx->h_ns, ns, sizeof(NScal) * S, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    bool changed = false;
    for (int s = 0; s < S; ++s)
        if (ctx->h_ns[s].active) {
            ctx->h_ns[s].active = 0;
            ctx->h_ns[s].status = ELDER_SAMPLE_NEWTON_MAXIT;
            changed = true;
        }
    if (changed)
        CK(cudaMemcpyAsync(ns, ctx->h_ns, sizeof(NScal) * S, cudaMemcpyHostToDevice, st));
    launch_newton_restore_failed(G, p, c, ctx->p_old, ctx->c_old, ns, S, st);
    launch_mass_balance(G, ph, ctx->bc[0], phi, K, p, c, ctx->c_old, ctx->partial3, S, st);
    launch_sum_partials(ctx->partial3, nb, ctx->mass, 3 * S, st);
    CK(cudaMemcpyAsync(ctx->h_mass, ctx->mass, sizeof(double) * 3 * S, cudaMemcpyDeviceToHost,
                       st));
    CKL();
    CK(cudaStreamSynchronize(st));
    prof_drain(ctx);
    return finish_step(ctx, S, status, stats);
}

// Per-sample status and statistics of a finished step from the host copies
// of the Newton scalars and the salt-mass balance.
int finish_step(elder_ctx* ctx, int S, int32_t* status, elder_stats* stats)
{
    int rc = ELDER_OK;
    for (int s = 0; s < S; ++s) {
        const NScal& k = ctx->h_ns[s];
        if (status) status[s] = k.status;
        if (stats) {
            stats[s].status = k.status;
            stats[s].newton_iters = k.iters;
            stats[s].krylov_iters = k.kiters;
            stats[s].ls_cuts = k.ls_cuts;
            stats[s].res0 = k.res0;
            stats[s].res = k.rn;
            stats[s].fp64_retry = 0;
            stats[s].pad = 0;
            stats[s].salt_mass0 = ctx->h_mass[3 * s + 0];
            stats[s].salt_mass = ctx->h_mass[3 * s + 1];
            stats[s].salt_inflow = ctx->h_mass[3 * s + 2];
        }
        if (k.status != 0) rc = ELDER_ENOTCONV;
    }
    return rc;
}

// Solves the step again from u^n, in FP64 with the settings `set`, for the
// samples listed in `idx` (packed into batches of at most 32 samples and 2^25
// node-samples).  Their
// entries of st1 and sts are replaced; the iteration counts accumulate and
// fp64_retry records `tier`.
void resolve_fp64(elder_ctx* ctx, const std::vector<int>& idx, const double* phi,
                  const double* K, double* p, double* c, double dt, const NewtonSettings& set,
                  int tier, std::vector<int32_t>& st1, std::vector<elder_stats>& sts,
                  cudaStream_t st)
{
    const Grid& G = ctx->grids[0];
    const size_t N = G.N, C = G.C;
    // at most 32 samples, and at most 2^25 node-samples per batch (the FP64
    // solver's workspace is ~1.3 KB per node: ~44 GB at that bound)
    const int chunk = std::max(
        1, std::min({32, ctx->cfg.max_samples, (int)((size_t(1) << 25) / N)}));
    if (!ctx->pk) {
        ctx->pk = dalloc<double>((size_t)chunk * (2 * N + 2 * C));
        ctx->mem.add(ctx->pk);
    }
    double* pk_p = ctx->pk;
    double* pk_c = pk_p + chunk * N;
    double* pk_phi = pk_c + chunk * N;
    double* pk_K = pk_phi + chunk * C;
    for (size_t b0 = 0; b0 < idx.size(); b0 += chunk) {
        const int F = (int)std::min<size_t>(chunk, idx.size() - b0);
        for (int q = 0; q < F; ++q) {
            const size_t s = idx[b0 + q];
            CK(cudaMemcpyAsync(pk_p + q * N, p + s * N, 8 * N, cudaMemcpyDeviceToDevice, st));
            CK(cudaMemcpyAsync(pk_c + q * N, c + s * N, 8 * N, cudaMemcpyDeviceToDevice, st));
            CK(cudaMemcpyAsync(pk_phi + q * C, phi + s * C, 8 * C, cudaMemcpyDeviceToDevice, st));
            CK(cudaMemcpyAsync(pk_K + q * C, K + s * C, 8 * C, cudaMemcpyDeviceToDevice, st));
        }
        std::vector<int32_t> st2(F);
        std::vector<elder_stats> s2(F);
        step_impl<double>(ctx, F, pk_phi, pk_K, pk_p, pk_c, dt, st2.data(), s2.data(), st, set);
        for (int q = 0; q < F; ++q) {
            const size_t s = idx[b0 + q];
            CK(cudaMemcpyAsync(p + s * N, pk_p + q * N, 8 * N, cudaMemcpyDeviceToDevice, st));
            CK(cudaMemcpyAsync(c + s * N, pk_c + q * N, 8 * N, cudaMemcpyDeviceToDevice, st));
            st1[s] = st2[q];
            s2[q].newton_iters += sts[s].newton_iters;
            s2[q].krylov_iters += sts[s].krylov_iters;
            s2[q].ls_cuts += sts[s].ls_cuts;
            s2[q].fp64_retry = tier;
            sts[s] = s2[q];
        }
    }
    CK(cudaStreamSynchronize(st));
}

// One implicit step of S samples.  ELDER_MIXED runs the FP32 multigrid and
// Krylov solver first and solves the samples whose Newton iteration fails
// again from u^n in FP64 (tier 1); samples that still fail (in either
// precision) get a last FP64 solve with robust settings (tier 2).
int step_tiers(elder_ctx* ctx, int S, const double* phi, const double* K, double* p,
               double* c, double dt, int32_t* status, elder_stats* stats, cudaStream_t st,
               int order = 0, double* p_hist = nullptr, double* c_hist = nullptr)
{
    std::vector<int32_t> st1(S);
    std::vector<elder_stats> sts(S);
    const NewtonSettings conf = configured_settings(ctx->cfg);
    const bool mixed = ctx->cfg.precision == ELDER_MIXED;
    // (re-solves of failed samples start again from u^n, which a failed
    // sample holds)
    if (mixed) {
        NewtonSettings mset = conf;
        if (ctx->cfg.mixed_newton_maxit > 0) mset.newton_maxit = ctx->cfg.mixed_newton_maxit;
        step_impl<float>(ctx, S, phi, K, p, c, dt, st1.data(), sts.data(), st, mset, order,
                         p_hist, c_hist, true);
    }
    else
        step_impl<double>(ctx, S, phi, K, p, c, dt, st1.data(), sts.data(), st, conf, order,
                          p_hist, c_hist, true);
    auto failed = [&]() {
        std::vector<int> f;
        for (int s = 0; s < S; ++s)
            if (st1[s] != 0) f.push_back(s);
        return f;
    };
    std::vector<int> f = failed();
    if (!f.empty() && mixed) {
        resolve_fp64(ctx, f, phi, K, p, c, dt, conf, 1, st1, sts, st);
        f = failed();
    }
    if (!f.empty())
        resolve_fp64(ctx, f, phi, K, p, c, dt, robust_settings(ctx->cfg), 2, st1, sts, st);
    int rc = ELDER_OK;
    for (int s = 0; s < S; ++s) {
        if (status) status[s] = st1[s];
        if (stats) stats[s] = sts[s];
        if (st1[s] != 0) rc = ELDER_ENOTCONV;
    }
    return rc;
}

template <class T>
int solve_impl(elder_ctx* ctx, int S, const double* phi, const double* K, const double* p,
               const double* c, double dt, int trans, const double* rhs, double* x,
               double rtol, int32_t* status, cudaStream_t st)
{
    Solver<T>& sv = solver_reserve<T>(ctx, S);
    const Grid& G = ctx->grids[0];
    const Phys ph = make_phys(ctx->cfg, dt);
    const size_t nN = (size_t)S * G.N;
    average_coefficients<T>(ctx, S, phi, K, st);
    assemble<T>(ctx, sv, S, phi, K, p, c, ph, nullptr, 0, S, st);
    const V2<double>* rhs2 = reinterpret_cast<const V2<double>*>(rhs);
    V2<double>* x2 = reinterpret_cast<V2<double>*>(x);
    // rhs in solver precision
    V2<T>* bT = sv.b;
    if (std::is_same<T, double>::value)
        CK(cudaMemcpyAsync(bT, rhs, sizeof(double) * 2 * nN, cudaMemcpyDeviceToDevice, st));
    else
        launch_convert<double, T>(rhs2, bT, nN, st);
    // Dirichlet rows of J are identity rows (R = u - u_D).
    // forward:   x_D = rhs_D, interior rhs_I - J_ID x_D
    // transpose: interior J_II^T y_I = rhs_I, then y_D = rhs_D - J_ID^T y_I
    // (x_D is kept in sv.xd: the multigrid vectors are overwritten by the solve)
    if (!trans) {
        launch_axpy_mask<T>(G, ctx->bc[0], bT, sv.xd, 1.0, 0, S, st);     // xd = b on D
        launch_spmv<T>(G, sv.J0, ctx->bc[0], sv.xd, sv.mx2[0], 0, 0, nullptr, nullptr,
                       nullptr, 0, S, st);                                 // J x_D (interior)
        launch_axpy_mask<T>(G, ctx->bc[0], sv.mx2[0], bT, -1.0, 2, S, st);
    }
    bicgstab<T>(ctx, sv, trans, rtol, ctx->cfg.lin_maxit, nullptr, S, st);
    if (!trans) {
        launch_axpy_mask<T>(G, ctx->bc[0], sv.xd, sv.x, 1.0, 1, S, st);
    } else {
        // (A^T y_I) on Dirichlet rows, unmasked
        launch_spmv<T>(G, sv.J0, ctx->bc[0], sv.x, sv.mx2[0], 1, 3, nullptr, nullptr,
                       nullptr, 0, S, st);
        // x_D = rhs_D - (A^T y_I)_D : rebuild rhs in mr then combine
        if (std::is_same<T, double>::value)
            CK(cudaMemcpyAsync(sv.mr[0], rhs, sizeof(double) * 2 * nN,
                               cudaMemcpyDeviceToDevice, st));
        else
            launch_convert<double, T>(rhs2, sv.mr[0], nN, st);
        launch_axpy_mask<T>(G, ctx->bc[0], sv.mx2[0], sv.mr[0], -1.0, 1, S, st);
        launch_axpy_mask<T>(G, ctx->bc[0], sv.mr[0], sv.x, 1.0, 1, S, st);
    }
    if (std::is_same<T, double>::value)
        CK(cudaMemcpyAsync(x, sv.x, sizeof(double) * 2 * nN, cudaMemcpyDeviceToDevice, st));
    else
        launch_convert<T, double>(sv.x, x2, nN, st);
    CKL();
    CK(cudaMemcpyAsync(ctx->h_ks, ctx->ks, sizeof(KScal) * S, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    int rc = ELDER_OK;
    for (int s = 0; s < S; ++s) {
        int stt = ctx->h_ks[s].status;
        if (stt == 0 && ctx->h_ks[s].active) stt = ELDER_SAMPLE_KRYLOV_MAXIT;
        if (status) status[s] = stt;
        if (stt != 0) rc = ELDER_ENOTCONV;
    }
    return rc;
}

// elder_smoother_apply in the multigrid precision of T's solver.
template <class T>
void smoother_apply_impl(elder_ctx* ctx, int S, const double* phi, const double* K,
                         const double* p, const double* c, double dt, int kind, int trans,
                         const double* r, double* z, cudaStream_t st)
{
    using M = typename Solver<T>::M;
    Solver<T>& sv = solver_reserve<T>(ctx, S);
    const Grid& G = ctx->grids[0];
    const size_t nN = (size_t)S * G.N;
    average_coefficients<T>(ctx, S, phi, K, st);
    assemble<T>(ctx, sv, S, phi, K, p, c, make_phys(ctx->cfg, dt), nullptr, 0, S, st);
    V2<T>* bT = sv.b;
    if (std::is_same<T, double>::value)
        CK(cudaMemcpyAsync(bT, r, sizeof(double) * 2 * nN, cudaMemcpyDeviceToDevice, st));
    else
        launch_convert<double, T>(reinterpret_cast<const V2<double>*>(r), bT, nN, st);
    DevFree tmp;
    if (kind == ELDER_SMOOTH_JACOBI) {
        launch_smooth<T, M>(G, sv.Jm[0], sv.Dinv[0], ctx->bc[0], bT, nullptr, sv.x, 1.0, trans,
                            nullptr, 0, S, st, kBS);
    } else if (kind == ELDER_SMOOTH_ZLINE) {
        if (!trans && sv.zMi[0])
            launch_zline_apply<T, M>(G, sv.Jm[0], sv.zMi[0], sv.zC[0], ctx->bc[0], bT, nullptr,
                                     sv.x, 1.0, nullptr, 0, S, st, 1);
        else
            launch_smooth_zline<T, M>(G, sv.Jm[0], sv.Dinv[0], ctx->bc[0], bT, nullptr, sv.x,
                                      1.0, trans, nullptr, 0, S, st, 1);
    } else {
        B4<M>* F = sv.F[0];
        B4<T>* Fd = sv.Fd[0];
        if (!F) {  // not configured: factors for this call
            F = dalloc<B4<M>>(nN * 27);
            tmp.add(F);
            Fd = dalloc<B4<T>>(nN);
            tmp.add(Fd);
            launch_ilu_factor<T, M>(G, sv.Jm[0], sv.Dinv[0], ctx->bc[0], F, Fd,
                                    ctx->cfg.ilu_beta, nullptr, 0, S, st);
        }
        launch_ilu_apply<T, M>(G, F, Fd, ctx->bc[0], bT, sv.mr[0], nullptr, sv.x, 1.0, trans, 1,
                               nullptr, 0, S, st);
    }
    if (std::is_same<T, double>::value)
        CK(cudaMemcpyAsync(z, sv.x, sizeof(double) * 2 * nN, cudaMemcpyDeviceToDevice, st));
    else
        launch_convert<T, double>(sv.x, reinterpret_cast<V2<double>*>(z), nN, st);
    CKL();
    CK(cudaStreamSynchronize(st));  // before the temporary factors are freed
}


int set_error(elder_ctx* ctx, const Fail& f)
{
    if (ctx) ctx->err = f.msg;
    else g_create_error = f.msg;
    return f.code;
}

}  // namespace

namespace {

// FMA-chain probe of the arithmetic peak: 8 independent chains per thread
// keep every FMA pipe busy; the sum is stored only if it equals a value it
// never takes, so that the chains are not optimised away.
template <class F>
__global__ void __launch_bounds__(256) k_fma_peak(const F* __restrict__ in, F* __restrict__ out,
                                                 int iters)
{
    const F b = in[1], c = in[2];
    F a[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) a[q] = in[0] + F(threadIdx.x + q);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int q = 0; q < 8; ++q) a[q] = fma(a[q], b, c);
    }
    F sum = F(0);
#pragma unroll
    for (int q = 0; q < 8; ++q) sum += a[q];
    if (sum == in[3]) out[blockIdx.x * blockDim.x + threadIdx.x] = sum;
}

template <class F> double fma_peak_gflops(int iters, cudaStream_t st)
{
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * 8, threads = 256;
    DevFree mem;
    F* buf = dalloc<F>(4 + (size_t)blocks * threads);
    mem.add(buf);
    const F h[4] = {F(1), F(0.999999), F(1e-7), F(-12345.0)};
    CK(cudaMemcpyAsync(buf, h, sizeof h, cudaMemcpyHostToDevice, st));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best = 1e30f;
    for (int r = 0; r < 4; ++r) {  // launch 0 warms up
        CK(cudaEventRecord(e0, st));
        k_fma_peak<F><<<blocks, threads, 0, st>>>(buf, buf + 4, iters);
        CK(cudaEventRecord(e1, st));
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        if (r > 0) best = std::min(best, ms);
    }
    count_launch(4);
    CK(cudaEventDestroy(e0));
    CK(cudaEventDestroy(e1));
    CKL();
    const double flops = 2.0 * 8.0 * (double)iters * blocks * threads;
    return flops / (best * 1e-3) / 1e9;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

extern "C" {

int elder_config_default(elder_config* cfg, int nx, int ny, int nz)
{
    if (!cfg) return ELDER_EINVAL;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->nx = nx;
    cfg->ny = ny;
    cfg->nz = nz;
    cfg->Lx = 600.0;
    cfg->Ly = 600.0;
    cfg->Lz = 150.0;
    cfg->rho0 = 1000.0;
    cfg->rho1 = 1200.0;
    cfg->mu = 1e-3;
    cfg->g = 9.81;
    cfg->Dm = 3.565e-6;
    cfg->bc_mode = 0;
    cfg->precision = ELDER_FP64;
    cfg->max_samples = 1;
    cfg->newton_maxit = 25;
    cfg->newton_tol_c = 1e-11;
    cfg->newton_tol_p = 1e-11 * 1000.0 * 9.81 * 150.0;
    cfg->ls_max = 6;
    cfg->lin_rtol = 1e-2;
    cfg->lin_maxit = 100;
    cfg->mg_levels = 0;
    cfg->nu1 = 1;
    cfg->nu2 = 0;
    cfg->omega = 0.5;
    cfg->omega_line = 0.95;
    cfg->coarse_K_harmonic = 0;
    cfg->use_graphs = 2;
    cfg->autotune = 1;
    cfg->newton_estimate = 1;
    cfg->smoother = ELDER_SMOOTH_ZLINE;
    cfg->mixed_newton_maxit = 0;
    cfg->ilu_beta = 0.0;
    cfg->omega_ilu = 1.0;
    return ELDER_OK;
}

const char* elder_last_error(const elder_ctx* ctx)
{
    return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

int elder_create(const elder_config* cfg, elder_ctx** out)
{
    if (!out) return ELDER_EINVAL;
    *out = nullptr;
    if (!cfg) {
        g_create_error = "cfg is NULL";
        return ELDER_EINVAL;
    }
    const elder_config& c = *cfg;
    if (c.nx < 1 || c.ny < 1 || c.nz < 1 || c.max_samples < 1 || !(c.Lx > 0) ||
        !(c.Ly > 0) || !(c.Lz > 0) || !(c.mu > 0) || c.bc_mode < 0 || c.bc_mode > 3 ||
        (c.precision != ELDER_FP64 && c.precision != ELDER_MIXED) || c.newton_maxit < 1 ||
        c.autotune < 0 || c.autotune > 2 ||
        c.lin_maxit < 1 || c.nu1 < 1 || c.nu2 < 0 || c.ls_max < 0 ||
        (c.smoother != ELDER_SMOOTH_JACOBI && c.smoother != ELDER_SMOOTH_ZLINE &&
         c.smoother != ELDER_SMOOTH_ILU) ||
        !(c.omega > 0) || !(c.omega_line > 0) || !(c.omega_ilu > 0) ||
        !std::isfinite(c.ilu_beta) || c.mixed_newton_maxit < 0 ||
        c.use_graphs < 0 || c.use_graphs > 2) {
        g_create_error = "invalid elder_config";
        return ELDER_EINVAL;
    }
    if (c.smoother == ELDER_SMOOTH_ZLINE && c.nz + 1 > kMaxLine) {
        g_create_error = "the z-line smoother needs nz <= 128";
        return ELDER_EINVAL;
    }
    if ((c.bc_mode == 0 || c.bc_mode == 1) && (c.nx % 4 || c.ny % 4)) {
        g_create_error = "bc_mode 0/1 need nx and ny divisible by 4 (square edges on nodes)";
        return ELDER_EINVAL;
    }
    std::unique_ptr<elder_ctx> ctx(new elder_ctx());
    ctx->cfg = c;
    ctx->smoother_now = c.smoother;
    ctx->omega_now = configured_omega(c);
    ctx->nu2_now = c.nu2;
    try {
        CK(cudaGetDevice(&ctx->device));
        // hierarchy: halve while all three counts are even (and the top square
        // stays node-aligned in modes 0/1)
        Grid G = make_grid(c.nx, c.ny, c.nz, c.Lx, c.Ly, c.Lz);
        ctx->grids.push_back(G);
        while (c.mg_levels == 0 || (int)ctx->grids.size() < c.mg_levels) {
            const Grid& Gf = ctx->grids.back();
            if (Gf.nx % 2 || Gf.ny % 2 || Gf.nz % 2) break;
            if ((c.bc_mode == 0 || c.bc_mode == 1) && ((Gf.nx / 2) % 4 || (Gf.ny / 2) % 4))
                break;
            ctx->grids.push_back(make_grid(Gf.nx / 2, Gf.ny / 2, Gf.nz / 2, c.Lx, c.Ly, c.Lz));
        }
        const int S = c.max_samples;
        const int L = (int)ctx->grids.size();
        ctx->phi.assign(L, nullptr);
        ctx->K.assign(L, nullptr);
        ctx->pl.assign(L, nullptr);
        ctx->cl.assign(L, nullptr);
        for (int l = 0; l < L; ++l) {
            const Grid& Gl = ctx->grids[l];
            std::vector<uint8_t> bc;
            std::vector<double> cv;
            dirichlet_host(c, Gl, bc, cv);
            uint8_t* dbc = dalloc<uint8_t>(Gl.N);
            ctx->mem.add(dbc);
            CK(cudaMemcpy(dbc, bc.data(), Gl.N, cudaMemcpyHostToDevice));
            ctx->bc.push_back(dbc);
            if (l == 0) {
                ctx->cval = dalloc<double>(Gl.N);
                ctx->mem.add(ctx->cval);
                CK(cudaMemcpy(ctx->cval, cv.data(), sizeof(double) * Gl.N,
                              cudaMemcpyHostToDevice));
            } else {
                ctx->phi[l] = dalloc<double>((size_t)S * Gl.C);
                ctx->K[l] = dalloc<double>((size_t)S * Gl.C);
                ctx->pl[l] = dalloc<double>((size_t)S * Gl.N);
                ctx->cl[l] = dalloc<double>((size_t)S * Gl.N);
                for (void* q : {(void*)ctx->phi[l], (void*)ctx->K[l], (void*)ctx->pl[l],
                                (void*)ctx->cl[l]})
                    ctx->mem.add(q);
            }
        }
        const size_t nN = (size_t)S * G.N;
        ctx->nblk0 = nblocks(G.N);
        for (double** q : {&ctx->p_old, &ctx->c_old, &ctx->pt, &ctx->ct}) {
            *q = dalloc<double>(nN);
            ctx->mem.add(*q);
        }
        for (V2<double>** q : {&ctx->R, &ctx->Rt, &ctx->tmp2}) {
            *q = dalloc<V2<double>>(nN);
            ctx->mem.add(*q);
        }
        // the stencil products write one partial per warp of 32 nodes
        ctx->partial = dalloc<double>((size_t)S * 2 * nblocks(G.N, 32));
        ctx->partial2 = dalloc<double>((size_t)S * 2 * ctx->nblk0);
        ctx->partial3 = dalloc<double>((size_t)S * 3 * ctx->nblk0);
        ctx->qf = dalloc<QF>((size_t)S * 12 * G.C);
        ctx->mem.add(ctx->qf);
        // Jacobian inputs in the solver's arithmetic type, reused level by level
        for (const Grid& Gl : ctx->grids) {
            ctx->jn.push_back(dalloc<double>((size_t)S * 2 * Gl.N));
            ctx->mem.add(ctx->jn.back());
            ctx->jc.push_back(dalloc<double>((size_t)S * 2 * Gl.C));
            ctx->mem.add(ctx->jc.back());
        }
        ctx->mass = dalloc<double>((size_t)3 * S);
        ctx->mem.add(ctx->mass);
        CK(cudaMallocHost((void**)&ctx->h_mass, sizeof(double) * 3 * S));
        ctx->mem.add(ctx->partial3);
        ctx->ns = dalloc<NScal>(S);
        ctx->ks = dalloc<KScal>(S);
        for (void* q : {(void*)ctx->partial, (void*)ctx->partial2, (void*)ctx->ns,
                        (void*)ctx->ks})
            ctx->mem.add(q);
        CK(cudaMemset(ctx->ks, 0, sizeof(KScal) * S));
        CK(cudaMemset(ctx->ns, 0, sizeof(NScal) * S));
        CK(cudaMallocHost((void**)&ctx->h_ns, sizeof(NScal) * S));
        CK(cudaMallocHost((void**)&ctx->h_ks, sizeof(KScal) * S));
        CK(cudaMallocHost((void**)&ctx->h_scalar, sizeof(double) * 64));
        ctx->loopc = dalloc<int>(8);
        ctx->mem.add(ctx->loopc);
        CK(cudaMemset(ctx->loopc, 0, 8 * sizeof(int)));
        CK(cudaMallocHost((void**)&ctx->h_loopc, sizeof(int) * 8));
        // solver workspace up front when the grid supports the solver (grids
        // that do not still serve the residual, Jacobian and moment calls)
        if (2 * ctx->grids.back().N <= MAX_COARSE_UNKNOWNS) {
            if (c.precision == ELDER_MIXED)
                solver_reserve<float>(ctx.get(), S);
            else
                solver_reserve<double>(ctx.get(), S);
        }
        CK(cudaDeviceSynchronize());
    } catch (const Fail& f) {
        g_create_error = f.msg;
        return f.code;
    }
    *out = ctx.release();
    return ELDER_OK;
}

int elder_destroy(elder_ctx* ctx)
{
    delete ctx;
    return ELDER_OK;
}

int elder_sizes(const elder_ctx* ctx, int64_t* N, int64_t* C, int* levels)
{
    if (!ctx) return ELDER_EINVAL;
    if (N) *N = ctx->grids[0].N;
    if (C) *C = ctx->grids[0].C;
    if (levels) *levels = (int)ctx->grids.size();
    return ELDER_OK;
}

static bool bad_S(elder_ctx* ctx, int S)
{
    if (S < 1 || S > ctx->cfg.max_samples) {
        ctx->err = "S out of range [1, max_samples]";
        return true;
    }
    return false;
}

int elder_fields(elder_ctx* ctx, int S, int kind, const double* params, double K_mean,
                 double* phi, double* K, void* stream)
{
    if (!ctx) return ELDER_EINVAL;
    if (S < 1 || kind < 0 || kind > 2 || !params || !phi || !K) {
        ctx->err = "elder_fields: bad argument";
        return ELDER_EINVAL;
    }
    try {
        launch_fields(ctx->grids[0], kind, params, K_mean, phi, K, S, (cudaStream_t)stream);
        CKL();
    } catch (const Fail& f) {
        return set_error(ctx, f);
    }
    return ELDER_OK;
}

int elder_residual(elder_ctx* ctx, int S, const double* phi, const double* K,
                   const double* p, const double* c, const double* p_old,
                   const double* c_old, double dt, double* R, void* stream)
{
    if (!ctx) return ELDER_EINVAL;
    if (bad_S(ctx, S)) return ELDER_EINVAL;
    if (!phi || !K || !p || !c || !p_old || !c_old || !R || !(dt > 0)) {
        ctx->err = "elder_residual: bad argument";
        return ELDER_EINVAL;
    }
    try {
        launch_residual(ctx->grids[0], make_phys(ctx->cfg, dt), ctx->bc[0], ctx->cval, phi, K,
                        p, c, p_old, c_old, reinterpret_cast<V2<double>*>(R), nullptr, nullptr,
                        nullptr, 0, S, (cudaStream_t)stream, ctx->qf);
        CKL();
    } catch (const Fail& f) {
        return set_error(ctx, f);
    }
    return ELDER_OK;
}

int elder_jacobian(elder_ctx* ctx, int S, const double* phi, const double* K,
                   const double* p, const double* c, double dt, double* J, void* stream)
{
    if (!ctx) return ELDER_EINVAL;
    if (bad_S(ctx, S)) return ELDER_EINVAL;
    if (!phi || !K || !p || !c || !J || !(dt > 0)) {
        ctx->err = "elder_jacobian: bad argument";
        return ELDER_EINVAL;
    }
    try {
        V2<double>* nodeT = reinterpret_cast<V2<double>*>(ctx->jn[0]);
        V2<double>* cellT = reinterpret_cast<V2<double>*>(ctx->jc[0]);
        launch_jacobian<double, double>(ctx->grids[0], make_phys(ctx->cfg, dt), ctx->bc[0], phi,
                                        K, p, c, reinterpret_cast<B4<double>*>(J), nullptr,
                                        nullptr, cellT, nodeT, nullptr, 0, S,
                                        (cudaStream_t)stream);
        CKL();
    } catch (const Fail& f) {
        return set_error(ctx, f);
    }
    return ELDER_OK;
}

int elder_step(elder_ctx* ctx, int S, const double* phi, const double* K, double* p,
               double* c, double dt, int32_t* status, elder_stats* stats, void* stream)
{
    if (!ctx) return ELDER_EINVAL;
    if (bad_S(ctx, S)) return ELDER_EINVAL;
    if (!phi || !K || !p || !c || !(dt > 0)) {
        ctx->err = "elder_step: bad argument";
        return ELDER_EINVAL;
    }
    try {
        return step_tiers(ctx, S, phi, K, p, c, dt, status, stats, (cudaStream_t)stream);
    } catch (const Fail& f) {
        return set_error(ctx, f);
    }
}

int elder_step_extrapolated(elder_ctx* ctx, int S, const double* phi, const double* K,
                            double* p_prev, double* c_prev, double* p, double* c, double dt,
                            int32_t* status, elder_stats* stats, void* stream)
{
    if (!ctx) return ELDER_EINVAL;
    if (bad_S(ctx, S)) return ELDER_EINVAL;
    if (!phi || !K || !p || !c || !p_prev || !c_prev || !(dt > 0)) {
        ctx->err = "elder_step_extrapolated: bad argument";
        return ELDER_EINVAL;
    }
    try {
        return step_tiers(ctx, S, phi, K, p, c, dt, status, stats, (cudaStream_t)stream, 1, p_prev,
                          c_prev);
    } catch (const Fail& f) {
        return set_error(ctx, f);
    }
}

int elder_step_predicted(elder_ctx* ctx, int S, const double* phi, const double* K, int order,
                         double* p_hist, double* c_hist, double* p, double* c, double dt,
                         int32_t* status, elder_stats* stats, void* stream)
{
    if (!ctx) return ELDER_EINVAL;
    if (bad_S(ctx, S)) return ELDER_EINVAL;
    if (!phi || !K || !p || !c || !p_hist || !c_hist || !(dt > 0) || order < 1 || order > 2) {
        ctx->err = "elder_step_predicted: bad argument";
        return ELDER_EINVAL;
    }
    try {
        return step_tiers(ctx, S, phi, K, p, c, dt, status, stats, (cudaStream_t)stream, order,
                          p_hist, c_hist);
    } catch (const Fail& f) {
        return set_error(ctx, f);
    }
}

int elder_solve(elder_ctx* ctx, int S, const double* phi, const double* K, const double* p,
                const double* c, double dt, int transpose, const double* rhs, double* x,
                double rtol, int32_t* status, void* stream)
{
    if (!ctx) return ELDER_EINVAL;
    if (bad_S(ctx, S)) return ELDER_EINVAL;
    if (!phi || !K || !p || !c || !rhs || !x || !(dt > 0) || !(rtol > 0)) {
        ctx->err = "elder_solve: bad argument";
        return ELDER_EINVAL;
    }
    try {
        if (ctx->cfg.precision == ELDER_MIXED && rtol >= 1e-6)
            return solve_impl<float>(ctx, S, phi, K, p, c, dt, transpose, rhs, x, rtol, status,
                                     (cudaStream_t)stream);
        return solve_impl<double>(ctx, S, phi, K, p, c, dt, transpose, rhs, x, rtol, status,
                                  (cudaStream_t)stream);
    } catch (const Fail& f) {
        return set_error(ctx, f);
    }
}

int elder_smoother_apply(elder_ctx* ctx, int S, const double* phi, const double* K,
                         const double* p, const double* c, double dt, int kind, int transpose,
                         const double* r, double* z, void* stream)
{
    if (!ctx) return ELDER_EINVAL;
    if (bad_S(ctx, S)) return ELDER_EINVAL;
    if (!phi || !K || !p || !c || !r || !z || !(dt > 0) || kind < ELDER_SMOOTH_JACOBI ||
        kind > ELDER_SMOOTH_ILU || (transpose != 0 && transpose != 1)) {
        ctx->err = "elder_smoother_apply: bad argument";
        return ELDER_EINVAL;
    }
    if (kind == ELDER_SMOOTH_ZLINE && ctx->grids[0].nz + 1 > kMaxLine) {
        ctx->err = "elder_smoother_apply: the z-line smoother needs nz <= 128";
        return ELDER_EINVAL;
    }
    try {
        if (ctx->cfg.precision == ELDER_MIXED)
            smoother_apply_impl<float>(ctx, S, phi, K, p, c, dt, kind, transpose, r, z,
                                       (cudaStream_t)stream);
        else
            smoother_apply_impl<double>(ctx, S, phi, K, p, c, dt, kind, transpose, r, z,
                                        (cudaStream_t)stream);
    } catch (const Fail& f) {
        return set_error(ctx, f);
    }
    return ELDER_OK;
}

int elder_initial_state(elder_ctx* ctx, int S, double* p, double* c, void* stream)
{
    if (!ctx) return ELDER_EINVAL;
    if (S < 1 || !p || !c) {
        ctx->err = "elder_initial_state: bad argument";
        return ELDER_EINVAL;
    }
    try {
        launch_initial_state(ctx->grids[0], ctx->cfg.rho0 * ctx->cfg.g, ctx->bc[0], ctx->cval,
                             p, c, S, (cudaStream_t)stream);
        CKL();
    } catch (const Fail& f) {
        return set_error(ctx, f);
    }
    return ELDER_OK;
}

int elder_profile(elder_ctx* ctx, int on)
{
    if (!ctx) return ELDER_EINVAL;
    try {
        CK(cudaDeviceSynchronize());
        prof_drain(ctx);
    } catch (const Fail& f) {
        return set_error(ctx, f);
    }
    Prof& P = ctx->prof;
    if (on) {
        for (int k = 0; k < ELDER_K_CLASSES; ++k) {
            P.launches[k] = 0;
            P.ms[k] = P.bytes[k] = P.flops[k] = 0.0;
        }
    }
    P.on = on != 0;
    return ELDER_OK;
}

int elder_profile_read(const elder_ctx* ctx, int kernel_class, int64_t* launches, double* ms,
                       double* bytes, double* flops)
{
    if (!ctx || kernel_class < 0 || kernel_class >= ELDER_K_CLASSES) return ELDER_EINVAL;
    const Prof& P = ctx->prof;
    if (launches) *launches = P.launches[kernel_class];
    if (ms) *ms = P.ms[kernel_class];
    if (bytes) *bytes = P.bytes[kernel_class];
    if (flops) *flops = P.flops[kernel_class];
    return ELDER_OK;
}

int elder_autotune_result(const elder_ctx* ctx, int* bs_smooth, int* bs_spmv, int* bs_mgres,
                          float* ms)
{
    if (!ctx) return ELDER_EINVAL;
    if (bs_smooth) *bs_smooth = ctx->bs[ELDER_K_SMOOTH];
    if (bs_spmv) *bs_spmv = ctx->bs[ELDER_K_SPMV];
    if (bs_mgres) *bs_mgres = ctx->bs[ELDER_K_MGRES];
    if (ms)
        for (int c = 0; c < 3; ++c)
            for (int q = 0; q < 3; ++q) ms[3 * c + q] = ctx->tune_ms[c][q];
    return ELDER_OK;
}

int elder_measure_peak(int kind, double* gflops, void* stream)
{
    if (!gflops || kind < 0 || kind > 1) {
        g_create_error = "elder_measure_peak: bad argument";
        return ELDER_EINVAL;
    }
    try {
        *gflops = kind == 0 ? fma_peak_gflops<double>(4000, (cudaStream_t)stream)
                            : fma_peak_gflops<float>(200000, (cudaStream_t)stream);
    } catch (const Fail& f) {
        g_create_error = f.msg;
        return f.code;
    }
    return ELDER_OK;
}

int elder_autotune_choice(const elder_ctx* ctx, int kernel_class, int* threads_per_block,
                          int* samples_per_cta, float* ms)
{
    if (!ctx || kernel_class < 0 || kernel_class >= ELDER_K_CLASSES) return ELDER_EINVAL;
    if (threads_per_block) *threads_per_block = ctx->bs[kernel_class];
    if (samples_per_cta) *samples_per_cta = ctx->spc[kernel_class];
    if (ms) {
        const int row = kernel_class == ELDER_K_MGRES ? 0 : kernel_class == ELDER_K_SMOOTH0 ? 1 : -1;
        for (int q = 0; q < 6; ++q) ms[q] = row >= 0 ? ctx->tune2_ms[row][q] : 0.f;
    }
    return ELDER_OK;
}

int elder_graph_status(const elder_ctx* ctx, int* cached, int64_t* replays, const char** note)
{
    if (!ctx) return ELDER_EINVAL;
    if (cached) *cached = (int)ctx->step_graphs.size();
    if (replays) *replays = ctx->step_graph_replays;
    if (note) *note = ctx->step_graph_note.c_str();
    return ELDER_OK;
}

int elder_launch_count(int64_t* launches)
{
    if (!launches) return ELDER_EINVAL;
    *launches = g_launches.load();
    return ELDER_OK;
}

int elder_moments(elder_ctx* ctx, int S, const double* c, const double* w, double threshold,
                  double* mean, double* var, double* p_exceed, void* stream)
{
    if (!ctx) return ELDER_EINVAL;
    if (S < 1 || !c || !mean || !var || !p_exceed) {
        ctx->err = "elder_moments: bad argument";
        return ELDER_EINVAL;
    }
    try {
        launch_moments(ctx->grids[0].N, S, c, w, threshold, mean, var, p_exceed,
                       (cudaStream_t)stream);
        CKL();
    } catch (const Fail& f) {
        return set_error(ctx, f);
    }
    return ELDER_OK;
}

int elder_grad(elder_ctx* ctx, int n_steps, const double* phi, const double* K,
               const double* p0, const double* c0, double dt, int ckpt_every, double* J_out,
               double* dJ_dphi, double* dJ_dK, void* stream)
{
    if (!ctx) return ELDER_EINVAL;
    if (n_steps < 1 || ckpt_every < 1 || !phi || !K || !p0 || !c0 || !J_out || !dJ_dphi ||
        !dJ_dK || !(dt > 0)) {
        ctx->err = "elder_grad: bad argument";
        return ELDER_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const Grid& G = ctx->grids[0];
    const Phys ph = make_phys(ctx->cfg, dt);
    const size_t N = G.N;
    try {
        Solver<double>& sv = solver_reserve<double>(ctx, 1);
        DevFree local;
        const int nck = (n_steps + ckpt_every - 1) / ckpt_every + 1;
        double* ck = dalloc<double>(2 * N * nck);  // checkpoints (p, c) every k steps
        local.add(ck);
        double* seg = dalloc<double>(2 * N * (ckpt_every + 1));  // recomputed segment
        local.add(seg);
        V2<double>* rhs = dalloc<V2<double>>(N);
        local.add(rhs);
        double* pj = dalloc<double>(ctx->nblk0 + nblocks(G.C) + 1);
        local.add(pj);
        double* dsum = pj + ctx->nblk0 + nblocks(G.C);
        double* cur = dalloc<double>(2 * N);
        local.add(cur);
        int32_t stat = 0;
        auto fwd_step = [&](double* pc) -> int {
            return step_tiers(ctx, 1, phi, K, pc, pc + N, dt, &stat, nullptr, st);
        };
        // forward sweep with checkpoints
        CK(cudaMemcpyAsync(cur, p0, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(cur + N, c0, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(ck, cur, sizeof(double) * 2 * N, cudaMemcpyDeviceToDevice, st));
        int rc_all = ELDER_OK;
        for (int n = 1; n <= n_steps; ++n) {
            if (fwd_step(cur) != ELDER_OK) {
                rc_all = ELDER_ENOTCONV;
                ctx->err = "elder_grad: forward step " + std::to_string(n) +
                           " failed with sample status " + std::to_string(stat);
            }
            if (n % ckpt_every == 0)
                CK(cudaMemcpyAsync(ck + 2 * N * (n / ckpt_every), cur, sizeof(double) * 2 * N,
                                   cudaMemcpyDeviceToDevice, st));
        }
        // objective, dJ/dphi (direct part) and dJ/du_N
        CK(cudaMemsetAsync(dJ_dK, 0, sizeof(double) * G.C, st));
        launch_objective(G, ph, phi, cur + N, pj, dJ_dphi, rhs, st);
        launch_sum_partials(pj, nblocks(G.C), dsum, 1, st);
        CKL();
        CK(cudaMemcpyAsync(ctx->h_scalar, dsum, sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        *J_out = ctx->h_scalar[0];
        // reverse sweep, segment by segment
        const int last_seg = (n_steps - 1) / ckpt_every;
        for (int sg = last_seg; sg >= 0; --sg) {
            const int k0 = sg * ckpt_every;
            const int k1 = std::min(n_steps, k0 + ckpt_every);
            CK(cudaMemcpyAsync(seg, ck + 2 * N * sg, sizeof(double) * 2 * N,
                               cudaMemcpyDeviceToDevice, st));
            for (int n = k0 + 1; n <= k1; ++n) {
                double* dst = seg + 2 * N * (n - k0);
                CK(cudaMemcpyAsync(dst, seg + 2 * N * (n - k0 - 1), sizeof(double) * 2 * N,
                                   cudaMemcpyDeviceToDevice, st));
                if (fwd_step(dst) != ELDER_OK) {
                    rc_all = ELDER_ENOTCONV;
                    ctx->err = "elder_grad: recomputed step " + std::to_string(n) +
                               " failed with sample status " + std::to_string(stat);
                }
            }
            for (int n = k1; n >= k0 + 1; --n) {
                const double* un = seg + 2 * N * (n - k0);
                const double* uo = seg + 2 * N * (n - k0 - 1);
                // J_n^T lambda_n = rhs (interior part; the Dirichlet rows of R_n
                // neither depend on theta nor on u_{n-1}, so lambda_D is not needed)
                average_coefficients<double>(ctx, 1, phi, K, st);
                assemble<double>(ctx, sv, 1, phi, K, un, un + N, ph, nullptr, 0, 1, st);
                CK(cudaMemcpyAsync(sv.b, rhs, sizeof(double) * 2 * N, cudaMemcpyDeviceToDevice,
                                   st));
                bicgstab<double>(ctx, sv, 1, 1e-12, std::max(ctx->cfg.lin_maxit, 400), nullptr,
                                 1, st);
                if (!krylov_converged(ctx, st)) {
                    // the transposed system of a step on a steep front: again
                    // with the z-line smoother and a longer solve
                    ctx->smoother_now = ELDER_SMOOTH_ZLINE;
                    ctx->omega_now = kRobustOmega;
                    ctx->nu2_now = std::max(ctx->cfg.nu2, 1);
                    bicgstab<double>(ctx, sv, 1, 1e-12, std::max(20 * ctx->cfg.lin_maxit, 4000),
                                     nullptr, 1, st, 1);
                    ctx->smoother_now = ctx->cfg.smoother;
                    ctx->omega_now = configured_omega(ctx->cfg);
                    ctx->nu2_now = ctx->cfg.nu2;
                    if (!krylov_converged(ctx, st)) {
                        rc_all = ELDER_ENOTCONV;
                        ctx->err = "elder_grad: adjoint solve of step " + std::to_string(n) +
                                   " did not reach its tolerance";
                    }
                }
                launch_adjoint_theta(G, ph, ctx->bc[0], phi, K, un, un + N, uo + N, sv.x,
                                     dJ_dphi, dJ_dK, st);
                if (n > 1)
                    launch_adjoint_prev_rhs(G, ph, ctx->bc[0], phi, uo + N, sv.x, rhs, st);
                CKL();
            }
        }
        CK(cudaStreamSynchronize(st));
        return rc_all;
    } catch (const Fail& f) {
        return set_error(ctx, f);
    }
}

}  // extern "C"
