// gpc.cu -- generalised polynomial chaos surrogate (Section 3: eqs.
// PCEdecom2, PCEcoef, PCEcoef2, var, PCEpoint and the exceedance estimate;
// Appendix A: Legendre polynomials).
//
// The expansion is built from the batched Elder step run at the points of a
// tensor Gauss-Legendre rule: one field u(x, theta_i) per point.  Two
// kernels do the work:
//   k_gpc_project  coefficients u_beta(x) for every node (FP64; the block
//                  first tabulates 0.5^M w_i P_beta(theta_i) / Q_beta in
//                  shared memory, then each thread streams its node's values
//                  and keeps one FP64 accumulator per basis function);
//   k_gpc_exceed   the surrogate at N_s sample points per node and the count
//                  above a threshold (FP32: coefficients in registers, FP32
//                  basis values of a chunk of samples broadcast from shared
//                  memory, samples split across blocks with integer atomics).
#include <cstdint>
#include <cstring>
#include <vector>
#include <algorithm>
#include <cmath>

#include "elder.h"
#include "kernels.h"

namespace elder {
namespace {

constexpr int kGpcMaxM = 8;      // stochastic dimensions
constexpr int kGpcMaxDeg = 16;   // largest degree in one variable
constexpr int kGpcBS = 128;      // threads per block
constexpr int kGpcChunk = 128;   // samples per shared-memory chunk (even)

// P_0..P_n at x by (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1} (Appendix A).
__host__ __device__ inline void legendre_all(int n, double x, double* P)
{
    P[0] = 1.0;
    if (n >= 1) P[1] = x;
    for (int k = 1; k < n; ++k) P[k + 1] = ((2 * k + 1) * x * P[k] - k * P[k - 1]) / (k + 1);
}

// FP32 recurrence for the surrogate evaluation (its sums are FP32 anyway;
// on GB300 FP64 runs at 1/64 of the FP32 rate).
__device__ inline void legendre_all_f(int n, float x, float* P)
{
    P[0] = 1.0f;
    if (n >= 1) P[1] = x;
    for (int k = 1; k < n; ++k) P[k + 1] = ((2 * k + 1) * x * P[k] - k * P[k - 1]) / (k + 1);
}

// coef[t][n] = sum_i Bq[t][i] u[i][n] with Bq = 0.5^M w_i P_t(theta_i) / Q_t
// (eq. PCEcoef); TP >= T accumulators per thread.
template <int TP>
__global__ void __launch_bounds__(kGpcBS)
    k_gpc_project(int M, int T, const int32_t* __restrict__ beta, int Nq,
                  const double* __restrict__ theta, const double* __restrict__ w, int N,
                  const double* __restrict__ u, double* __restrict__ coef,
                  double* __restrict__ mean, double* __restrict__ var, int maxdeg)
{
    extern __shared__ double sh[];
    double* Bq = sh;               // [T][Nq]
    double* Qt = sh + T * Nq;      // [T]
    for (int q = threadIdx.x; q < T * Nq; q += blockDim.x) {
        const int t = q / Nq, i = q % Nq;
        double P1[kGpcMaxM * (kGpcMaxDeg + 1)];
        double v = 1.0, Q = 1.0;
        for (int j = 0; j < M; ++j) {
            const int b = min(max((int)beta[t * M + j], 0), maxdeg);
            legendre_all(b, theta[(size_t)i * M + j], P1 + j * (kGpcMaxDeg + 1));
            v *= P1[j * (kGpcMaxDeg + 1) + b];
            Q *= 1.0 / (2.0 * b + 1.0);
        }
        Bq[q] = ldexp(w[i] * v / Q, -M);
        if (i == 0) Qt[t] = Q;
    }
    __syncthreads();
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    double acc[TP];
#pragma unroll
    for (int t = 0; t < TP; ++t) acc[t] = 0.0;
    for (int i = 0; i < Nq; ++i) {
        const double ui = u[(size_t)i * N + n];
#pragma unroll
        for (int t = 0; t < TP; ++t)
            if (t < T) acc[t] = fma(Bq[t * Nq + i], ui, acc[t]);
    }
    double vs = 0.0;
#pragma unroll
    for (int t = 0; t < TP; ++t) {
        if (t < T) {
            coef[(size_t)t * N + n] = acc[t];
            if (t > 0) vs += Qt[t] * acc[t] * acc[t];
        }
    }
    if (mean) mean[n] = acc[0];
    if (var) var[n] = vs;
}

// Surrogate at Ns points for the listed nodes; counts of values above the
// threshold accumulate in cnt (64-bit, one per listed node).
//
// Per chunk of kGpcChunk samples the block first tabulates, with all its
// threads, the FP32 Legendre values P_k(theta_m) of every sample (Ps) and
// then the basis values P_beta(theta) = prod_m P_{beta_m}(theta_m) (Bs, the
// product over m in order).  Each thread keeps the FP32 coefficients of NPT
// listed nodes (k0 + r blockDim.x) in registers, so every basis value read
// from shared memory feeds NPT FMA chains; SPT samples are evaluated at a
// time.  Each sum runs over t in order.
// Dynamic shared memory: Bs [kGpcChunk][TP] floats, Ps [kGpcChunk][M][maxdeg+1]
// floats, the clamped multi-indices [T][M] ints.
template <int TP, int NPT, int SPT>
__global__ void __launch_bounds__(kGpcBS)
    k_gpc_exceed(int M, int T, const int32_t* __restrict__ beta, int N,
                 const double* __restrict__ coef, int n_pts, const int32_t* __restrict__ nodes,
                 int Ns, const double* __restrict__ theta, float thr, int maxdeg,
                 unsigned long long* __restrict__ cnt)
{
    extern __shared__ __align__(16) unsigned char gx_smem[];
    float* Bs = reinterpret_cast<float*>(gx_smem);          // [kGpcChunk][TP]
    const int D1 = maxdeg + 1;
    float* Ps = Bs + kGpcChunk * TP;                         // [kGpcChunk][M][D1]
    int* bs = reinterpret_cast<int*>(Ps + kGpcChunk * M * D1);  // [T][M]
    // multi-index entries outside [0, maxdeg] are clamped: a caller error
    // gives wrong values, never an out-of-range read
    for (int e = threadIdx.x; e < T * M; e += blockDim.x)
        bs[e] = min(max((int)beta[e], 0), maxdeg);
    int kk[NPT];
    bool live[NPT];
    float cv[NPT][TP];
#pragma unroll
    for (int r = 0; r < NPT; ++r) {
        kk[r] = blockIdx.x * NPT * blockDim.x + r * blockDim.x + threadIdx.x;
        live[r] = kk[r] < n_pts;
        const int n = live[r] ? (nodes ? nodes[kk[r]] : kk[r]) : 0;
#pragma unroll
        for (int t = 0; t < TP; ++t)
            cv[r][t] = (live[r] && t < T) ? (float)coef[(size_t)t * N + n] : 0.f;
    }
    // this block's slice of the samples
    const int per = (Ns + gridDim.y - 1) / gridDim.y;
    const int s0 = blockIdx.y * per;
    const int s1 = min(Ns, s0 + per);
    unsigned int count[NPT];
#pragma unroll
    for (int r = 0; r < NPT; ++r) count[r] = 0;
    for (int cs = s0; cs < s1; cs += kGpcChunk) {
        const int nc = min(kGpcChunk, s1 - cs);
        __syncthreads();
        for (int e = threadIdx.x; e < nc * M; e += blockDim.x) {
            const int j = e / M, m = e - j * M;
            legendre_all_f(maxdeg, (float)theta[(size_t)(cs + j) * M + m], Ps + e * D1);
        }
        __syncthreads();
        // rows at or past nc (the tail of the last chunk) are zero
        for (int e = threadIdx.x; e < kGpcChunk * TP; e += blockDim.x) {
            const int j = e / TP, t = e - j * TP;
            float v = 0.f;
            if (j < nc && t < T) {
                v = 1.f;
                for (int m = 0; m < M; ++m) v *= Ps[(j * M + m) * D1 + bs[t * M + m]];
            }
            Bs[e] = v;
        }
        __syncthreads();
        // SPT samples at a time (kGpcChunk is a multiple of SPT): SPT NPT
        // independent FMA chains; the last group may run into zero rows
        // past nc, which are not counted
        for (int j = 0; j < nc; j += SPT) {
            float a[SPT][NPT];
#pragma unroll
            for (int q = 0; q < SPT; ++q)
#pragma unroll
                for (int r = 0; r < NPT; ++r) a[q][r] = 0.f;
#pragma unroll
            for (int t = 0; t < TP; t += 4) {
#pragma unroll
                for (int q = 0; q < SPT; ++q) {
                    const float4 b = *reinterpret_cast<const float4*>(Bs + (j + q) * TP + t);
#pragma unroll
                    for (int r = 0; r < NPT; ++r) {
                        a[q][r] = fmaf(cv[r][t], b.x, a[q][r]);
                        a[q][r] = fmaf(cv[r][t + 1], b.y, a[q][r]);
                        a[q][r] = fmaf(cv[r][t + 2], b.z, a[q][r]);
                        a[q][r] = fmaf(cv[r][t + 3], b.w, a[q][r]);
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < SPT; ++q) {
                const bool vq = j + q < nc;
#pragma unroll
                for (int r = 0; r < NPT; ++r) count[r] += (vq && a[q][r] > thr) ? 1u : 0u;
            }
        }
    }
#pragma unroll
    for (int r = 0; r < NPT; ++r)
        if (live[r] && count[r]) atomicAdd(cnt + kk[r], (unsigned long long)count[r]);
}

// ---------------------------------------------------------------------------
// Tensor-core evaluation of the surrogate count (sm_103a tcgen05).
//
// The surrogate values of a tile of 128 listed nodes at a chunk of 128
// samples form the product U = C B of the node tile's coefficients C
// (128 x T) and the chunk's basis values B (T x 128): a dense contraction,
// run as a TF32 matrix product on the tensor cores with FP32 accumulators in
// tensor memory.  Each FP32 factor x is split as x = x_hi + x_lo with x_hi
// exactly representable in TF32 (the low 13 mantissa bits cleared), and the
// three products C_hi B_hi + C_hi B_lo + C_lo B_hi are one product over the
// stacked inner dimension K' = 3 TP (padded to a multiple of 8):
//   A' = [C_hi | C_hi | C_lo] (128 x K'),  B' = [B_hi ; B_lo ; B_hi] (K' x 128).
// The dropped C_lo B_lo and the TF32 rounding of the lo parts leave at most
// 3 2^-20 |c| |P| per term; with the FP32 accumulation of the K'/8 partial
// products the error stays below the FP32 path's bound 16 T 2^-24 sum |c|.
//
// One CTA: one node tile (A' in shared memory, loaded once) and a slice of
// the samples in chunks of 128.  Warps 0-3 count (each thread owns one node
// row of the accumulator and compares its 128 columns with the threshold
// after a tcgen05.ld), warps 4-7 write each chunk's B' into one of two
// shared-memory buffers, warp 8 issues the MMAs (one thread) into one of two
// TMEM accumulators.  mbarriers hand the buffers over; every wait gives up
// after a bounded number of polls, sets the error flag and lets the kernel
// finish.
//
// Shared-memory operands use the no-swizzle K-major layout of 8-row x 16-byte
// core matrices: element (row, k) at ((row / 8) * (K' / 4) + k / 4) * 128 +
// (row % 8) * 16 + (k % 4) * 4 bytes; the stride between core matrices along
// K is 128 B, along the rows K' / 4 * 128 B.
// ---------------------------------------------------------------------------

constexpr int kTcRows = 128;      // node rows per tile (MMA M)
constexpr int kTcCols = 128;      // samples per chunk (MMA N)
constexpr int kTcKp = 112;        // stacked inner dimension K' (3 x 36 + pad)
constexpr int kTcTP = 36;         // terms per part (T <= 36)
constexpr int kTcMaxM = 4;        // stochastic dimensions of the tensor-core path
constexpr int kTcMaxDeg = 8;      // largest degree of the tensor-core path
constexpr int kTcTileBytes = kTcRows * kTcKp * 4;  // 57344
constexpr unsigned kTcPolls = 1u << 26;            // bound of every mbarrier wait

__device__ __forceinline__ unsigned smem_u32(const void* p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned bar)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(bar)
                 : "memory");
}

// Polls the barrier's phase of the given parity; false when it gave up (the
// error flag is then set) or another thread already gave up.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, int* err,
                                          volatile int* abort_flag)
{
    for (unsigned it = 0; it < kTcPolls; ++it) {
        unsigned done = 0;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 1023u) == 1023u && *abort_flag) return false;
    }
    *abort_flag = 1;
    atomicExch(err, 1);
    return false;
}

__device__ __forceinline__ void fence_async_shared()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after()
{
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before()
{
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor, no swizzle: start, leading-dimension
// (K-direction core-matrix stride) and stride-dimension (row-group stride)
// byte offsets, each in 16-byte units, and the descriptor version bits.
__device__ __forceinline__ uint64_t tc_desc(unsigned addr, unsigned lbo, unsigned sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor: D FP32, A and B TF32, both K-major, N = 128,
// M = 128.
constexpr uint32_t kTcIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTcCols >> 3) << 17) |
                              ((uint32_t)(kTcRows >> 4) << 24);

__device__ __forceinline__ void tc_mma(unsigned d_tmem, uint64_t a, uint64_t b, unsigned acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(kTcIdesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void tc_commit(unsigned bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// 32 consecutive accumulator columns of this warp's 32 lanes, one row per
// thread.
__device__ __forceinline__ void tc_ld32(unsigned taddr, float* v)
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
        "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
        "%30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
#pragma unroll
    for (int q = 0; q < 32; ++q) v[q] = __uint_as_float(r[q]);
}

__device__ __forceinline__ void tc_wait_ld()
{
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// x = hi + lo with hi exactly representable in TF32 (10 mantissa bits)
__device__ __forceinline__ void tf32_split(float x, float& hi, float& lo)
{
    hi = __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
    lo = x - hi;
}

// byte offset of element (row, k) in the no-swizzle K-major operand layout
__device__ __forceinline__ int tc_off(int row, int k)
{
    return ((row >> 3) * (kTcKp / 4) + (k >> 2)) * 128 + (row & 7) * 16 + (k & 3) * 4;
}

__device__ __forceinline__ void tc_mma_ta(unsigned d_tmem, unsigned a_tmem, uint64_t b, unsigned acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b), "r"(kTcIdesc), "r"(acc)
        : "memory");
}

// 16 consecutive columns of this warp's 32 lanes from registers, one row per
// thread.
__device__ __forceinline__ void tc_st16(unsigned taddr, const float* v)
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15, %16};" ::"r"(taddr),
        "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
        "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
        "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
        "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
        "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
        "r"(__float_as_uint(v[15]))
        : "memory");
}

// Two node tiles per CTA: their A' operands live in tensor memory (written
// once by the counting warps), so every basis chunk the producers build
// feeds two products.  Tensor memory: accumulators of tiles 0 and 1 at
// columns 0 and 128, A' of tiles 0 and 1 at columns 256 and 384 (112 used).
constexpr int kTcTiles = 2;

constexpr int kTcCountWarps = 4;   // one per TMEM lane quarter
// Degree of variable m in term t of the total-degree-4 basis in 3 variables,
// in the order elder_gpc_indices gives it (total degree ascending, then the
// degree vector lexicographically ascending); -1 past its 35 terms.
__host__ __device__ constexpr int canon_deg(int t, int m)
{
    int q = 0;
    for (int s = 0; s <= 4; ++s)
        for (int a = 0; a <= s; ++a)
            for (int b = 0; b <= s - a; ++b) {
                if (q == t) return m == 0 ? a : (m == 1 ? b : s - a - b);
                ++q;
            }
    return -1;
}
constexpr int kCanonT = 35;

// One step of the Legendre recurrence, (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1},
// with the ratios as constants (the same arithmetic in both basis builders).
__device__ __forceinline__ float leg_next(int k, float x, float p0, float pm1)
{
    return fmaf((float(2 * k + 1) / float(k + 1)) * x, p0, -(float(k) / float(k + 1)) * pm1);
}

constexpr int kTcSplit = 3;        // basis builders per sample (12 of the 36 terms each)
constexpr int kTcProdWarps = 4 * kTcSplit;
constexpr int kTcPartTerms = kTcTP / kTcSplit;  // terms per basis builder
static_assert(kTcTP % (4 * kTcSplit) == 0, "whole 4-term groups per basis builder");
constexpr int kTcThreads = 32 * (kTcCountWarps + kTcProdWarps + 1);

// The basis builder's terms for the total-degree-4 basis in 3 variables in
// canonical order: part PART holds terms 12 PART .. 12 PART + 11, whose
// degrees are compile-time constants, so that each basis value is a product
// of the sample's Legendre values in registers, P[m][k] = P_k(theta_m),
// formed in the same order as the general builder, (P_a P_b) P_c.
template <int PART>
__device__ __forceinline__ void canon_build(const float (&P)[3][5], bool ok, unsigned char* Bs,
                                            int col)
{
#pragma unroll
    for (int g = 0; g < kTcPartTerms; g += 4) {
        const int t0 = PART * kTcPartTerms + g;
        float4 hi4, lo4;
        float* hp = &hi4.x;
        float* lp = &lo4.x;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int t = t0 + r;
            float v = 0.f;
            if (t < kCanonT && ok)
                v = (P[0][canon_deg(t, 0)] * P[1][canon_deg(t, 1)]) * P[2][canon_deg(t, 2)];
            tf32_split(v, hp[r], lp[r]);
        }
        *reinterpret_cast<float4*>(Bs + tc_off(col, t0)) = hi4;
        *reinterpret_cast<float4*>(Bs + tc_off(col, kTcTP + t0)) = lo4;
        *reinterpret_cast<float4*>(Bs + tc_off(col, 2 * kTcTP + t0)) = hi4;
    }
}

__global__ void __launch_bounds__(kTcThreads, 1)
    k_gpc_exceed_tc(int M, int T, const int32_t* __restrict__ beta, int maxdeg, int N,
                    const double* __restrict__ coef, int n_pts, const int32_t* __restrict__ nodes,
                    int Ns, const double* __restrict__ theta, float thr,
                    unsigned long long* __restrict__ cnt, int* err)
{
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    unsigned char* Bs0 = tc_smem;                          // B' chunk buffers
    unsigned long long* bars =
        reinterpret_cast<unsigned long long*>(tc_smem + 2 * kTcTileBytes);  // 8 barriers
    unsigned* tmem_slot = reinterpret_cast<unsigned*>(bars + 8);
    // per term and dimension, the offset of P_{beta_tm}(theta_m) in ptab
    int* boff = reinterpret_cast<int*>(tmem_slot + 4);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(boff + kTcTP * kTcMaxM);
    // Legendre values of a chunk, [m][k][sample]
    float* ptab = reinterpret_cast<float*>(tc_smem + 2 * kTcTileBytes + 1024);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tile0 = blockIdx.x * kTcTiles * kTcRows;
    // this CTA's slice of the samples, whole chunks
    const int nchunk_all = (Ns + kTcCols - 1) / kTcCols;
    const int per = (nchunk_all + gridDim.y - 1) / gridDim.y;
    const int c0 = blockIdx.y * per;
    const int nchunk = max(0, min(nchunk_all, c0 + per) - c0);
    // full[b], empty[b]: B' buffer b written / read by the MMAs;
    // tfull[q], tempty[q]: accumulator of tile q written by the MMAs / read out
    const unsigned full0 = smem_u32(bars + 0), empty0 = smem_u32(bars + 2);
    const unsigned tfull0 = smem_u32(bars + 4), tempty0 = smem_u32(bars + 6);
    if (threadIdx.x == 0) {
        for (int b = 0; b < 2; ++b) {
            mbar_init(full0 + 8 * b, 32 * kTcProdWarps);
            mbar_init(empty0 + 8 * b, 1);
            mbar_init(tfull0 + 8 * b, 1);
            mbar_init(tempty0 + 8 * b, 32 * kTcCountWarps);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int e = threadIdx.x; e < T * M; e += blockDim.x) {
        const int m = e % M;
        boff[e] = (m * (kTcMaxDeg + 1) + min(max((int)beta[e], 0), maxdeg)) * kTcSplit * kTcCols;
    }
    // the inner-dimension padding of both B' buffers stays zero
    for (int e = threadIdx.x; e < 2 * kTcCols; e += blockDim.x) {
        unsigned char* Bs = Bs0 + (e / kTcCols) * kTcTileBytes;
        *reinterpret_cast<float4*>(Bs + tc_off(e % kTcCols, 3 * kTcTP)) =
            make_float4(0.f, 0.f, 0.f, 0.f);
    }
    fence_async_shared();
    if (warp == 0) {  // all 512 columns: 2 accumulators, 2 A' operands
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                         smem_u32(tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = *tmem_slot;
    if (warp < 4) {
        // A' = [C_hi | C_hi | C_lo] of both tiles into tensor memory: thread
        // <-> row 32 warp + lane, rows past n_pts and terms past T zero
        const int row = 32 * warp + lane;
        for (int q = 0; q < kTcTiles; ++q) {
            const int kk = tile0 + q * kTcRows + row;
            const int n = kk < n_pts ? (nodes ? nodes[kk] : kk) : -1;
            const unsigned ta = tmem + ((unsigned)(32 * warp) << 16) + 256u + 128u * q;
#pragma unroll 1
            for (int k0 = 0; k0 < kTcKp; k0 += 16) {
                float v[16];
#pragma unroll
                for (int r = 0; r < 16; ++r) {
                    const int k = k0 + r, part = k / kTcTP, t = k - part * kTcTP;
                    float x = 0.f;
                    if (part < 3 && t < T && n >= 0) {
                        float hi, lo;
                        tf32_split((float)coef[(size_t)t * N + n], hi, lo);
                        x = part < 2 ? hi : lo;
                    }
                    v[r] = x;
                }
                tc_st16(ta + k0, v);
            }
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp < kTcCountWarps) {
        // ---- counting: thread <-> node row 32 (warp % 4) + lane of each
        // tile, columns [64 h, 64 h + 64) with h = warp / 4 ----
        unsigned count[kTcTiles] = {0u, 0u};
        const int quarter = warp & 3;
        const int row = 32 * quarter + lane;
        for (int i = 0; i < nchunk; ++i) {
            const int valid = min(kTcCols, Ns - (c0 + i) * kTcCols);
            bool stop = false;
            for (int q = 0; q < kTcTiles && !stop; ++q) {
                if (!mbar_wait(tfull0 + 8 * q, i & 1, err, abort_flag)) {
                    stop = true;
                    break;
                }
                tc_fence_after();
                const unsigned ta =
                    tmem + ((unsigned)(32 * quarter) << 16) + (unsigned)(q * kTcCols);
                unsigned c = 0;
#pragma unroll
                for (int h = 0; h < kTcCols; h += 64) {
                    float v0[32], v1[32];
                    tc_ld32(ta + h, v0);
                    tc_ld32(ta + h + 32, v1);
                    tc_wait_ld();
                    if (valid == kTcCols) {
                        // four independent partial counts: no serial chain of
                        // dependent adds
                        unsigned cq[4] = {0u, 0u, 0u, 0u};
#pragma unroll
                        for (int r = 0; r < 32; ++r)
                            cq[r & 3] += (unsigned)(v0[r] > thr) + (unsigned)(v1[r] > thr);
                        c += (cq[0] + cq[1]) + (cq[2] + cq[3]);
                    } else {  // the last, ragged chunk
#pragma unroll
                        for (int r = 0; r < 32; ++r) {
                            c += (h + r < valid && v0[r] > thr) ? 1u : 0u;
                            c += (h + 32 + r < valid && v1[r] > thr) ? 1u : 0u;
                        }
                    }
                }
                count[q] += c;
                tc_fence_before();
                mbar_arrive(tempty0 + 8 * q);
            }
            if (stop) break;
        }
        for (int q = 0; q < kTcTiles; ++q) {
            const int kk = tile0 + q * kTcRows + row;
            if (kk < n_pts && count[q]) atomicAdd(cnt + kk, (unsigned long long)count[q]);
        }
    } else if (warp < kTcCountWarps + kTcProdWarps) {
        // ---- B' chunks: kTcSplit threads per sample column, 12 terms each ----
        // Each thread forms its sample's Legendre values in its own column of
        // ptab, [(m * 9 + k) * kTcSplit * 128 + p] (consecutive threads,
        // consecutive words), then per group of 4 terms the basis products,
        // split and stored as one 16-byte row segment of a core matrix in
        // each of the three parts
        const int pt = threadIdx.x - 32 * kTcCountWarps;
        const int col = pt & (kTcCols - 1), part = pt / kTcCols;
        const int tbeg = part * kTcPartTerms;
        int bo[kTcPartTerms][kTcMaxM];
#pragma unroll
        for (int r = 0; r < kTcPartTerms; ++r)
#pragma unroll
            for (int m = 0; m < kTcMaxM; ++m)
                bo[r][m] = (tbeg + r < T && m < M) ? boff[(tbeg + r) * M + m] : 0;
        // the total-degree-4 basis in 3 variables in canonical order takes
        // the register builder (canon_build); any other basis the table
        bool canon = M == 3 && T == kCanonT && maxdeg == 4;
        for (int e = 0; canon && e < kCanonT * 3; ++e)
            canon = beta[e] == canon_deg(e / 3, e % 3);
        // the next chunk's sample coordinates are loaded one chunk ahead and
        // held in FP64 until that chunk: the FP32 conversion is their first
        // use, so the load's latency hides behind a chunk of work
        double xn[kTcMaxM];
        auto load_theta = [&](int i) {
            const int j = (c0 + i) * kTcCols + col;
#pragma unroll
            for (int m = 0; m < kTcMaxM; ++m)
                xn[m] = (i < nchunk && j < Ns && m < M) ? theta[(size_t)j * M + m] : 0.0;
        };
        load_theta(0);
        for (int i = 0; i < nchunk; ++i) {
            const int b = i & 1;
            unsigned char* Bs = Bs0 + b * kTcTileBytes;
            float xc[kTcMaxM];
#pragma unroll
            for (int m = 0; m < kTcMaxM; ++m) xc[m] = (float)xn[m];
            load_theta(i + 1);
            if (i >= 2 && !mbar_wait(empty0 + 8 * b, ((i >> 1) - 1) & 1, err, abort_flag)) break;
            const int j = (c0 + i) * kTcCols + col;
            const bool ok = j < Ns;
            if (canon) {
                float P[3][5];
#pragma unroll
                for (int m = 0; m < 3; ++m) {
                    const float x = xc[m];
                    float pm1 = 1.f, p0 = x;
                    P[m][0] = 1.f;
                    P[m][1] = x;
#pragma unroll
                    for (int k = 1; k < 4; ++k) {
                        const float p1 = leg_next(k, x, p0, pm1);
                        P[m][k + 1] = p1;
                        pm1 = p0;
                        p0 = p1;
                    }
                }
                if (part == 0) canon_build<0>(P, ok, Bs, col);
                else if (part == 1) canon_build<1>(P, ok, Bs, col);
                else canon_build<2>(P, ok, Bs, col);
                fence_async_shared();
                mbar_arrive(full0 + 8 * b);
                continue;
            }
#pragma unroll
            for (int m = 0; m < kTcMaxM; ++m) {
                if (m < M) {
                    const float x = xc[m];
                    float pm1 = 1.f, p0 = x;
                    ptab[(m * (kTcMaxDeg + 1)) * kTcSplit * kTcCols + pt] = 1.f;
                    if (maxdeg >= 1) ptab[(m * (kTcMaxDeg + 1) + 1) * kTcSplit * kTcCols + pt] = x;
                    // (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1} with the ratios
                    // folded into constants
#pragma unroll
                    for (int k = 1; k < kTcMaxDeg; ++k) {
                        if (k < maxdeg) {
                            const float p1 = leg_next(k, x, p0, pm1);
                            ptab[(m * (kTcMaxDeg + 1) + k + 1) * kTcSplit * kTcCols + pt] = p1;
                            pm1 = p0;
                            p0 = p1;
                        }
                    }
                }
            }
            // (each thread reads back only its own column; the table
            // offsets of its terms sit in registers, bo)
#pragma unroll
            for (int g = 0; g < kTcPartTerms; g += 4) {
                const int t0 = tbeg + g;
                float4 hi4, lo4;
                float* hp = &hi4.x;
                float* lp = &lo4.x;
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int t = t0 + r;
                    float v = 0.f;
                    if (ok && t < T) {
                        v = 1.f;
#pragma unroll
                        for (int m = 0; m < kTcMaxM; ++m)
                            if (m < M) v *= ptab[bo[g + r][m] + pt];
                    }
                    tf32_split(v, hp[r], lp[r]);
                }
                *reinterpret_cast<float4*>(Bs + tc_off(col, t0)) = hi4;
                *reinterpret_cast<float4*>(Bs + tc_off(col, kTcTP + t0)) = lo4;
                *reinterpret_cast<float4*>(Bs + tc_off(col, 2 * kTcTP + t0)) = hi4;
            }
            fence_async_shared();
            mbar_arrive(full0 + 8 * b);
        }
    } else if (lane == 0) {
        // ---- MMA issue: both tiles against each chunk ----
        constexpr unsigned kLbo = 128, kSbo = (kTcKp / 4) * 128;
        for (int i = 0; i < nchunk; ++i) {
            const int b = i & 1;
            if (!mbar_wait(full0 + 8 * b, (i >> 1) & 1, err, abort_flag)) break;
            const unsigned b_base = smem_u32(Bs0 + b * kTcTileBytes);
            bool stop = false;
            for (int q = 0; q < kTcTiles; ++q) {
                if (i >= 1 && !mbar_wait(tempty0 + 8 * q, (i - 1) & 1, err, abort_flag)) {
                    stop = true;
                    break;
                }
                tc_fence_after();
                const unsigned d = tmem + (unsigned)(q * kTcCols);
                const unsigned a = tmem + 256u + 128u * q;
#pragma unroll
                for (int ks = 0; ks < kTcKp / 8; ++ks)
                    tc_mma_ta(d, a + 8 * ks, tc_desc(b_base + ks * 256, kLbo, kSbo), ks > 0 ? 1u : 0u);
                tc_commit(tfull0 + 8 * q);
            }
            if (stop) break;
            tc_commit(empty0 + 8 * b);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
    }
}

// Set by a tensor-core count whose bounded wait gave up (one flag per
// device, cleared by each call before its kernel).
__device__ int g_gpc_tc_err;

__global__ void k_gpc_counts_to_fraction(int n_pts, int Ns, double* p, const int* err)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_pts) return;
    unsigned long long c;
    memcpy(&c, p + k, sizeof(c));
    p[k] = (err && *err) ? __longlong_as_double(0x7FF8000000000000ll) : (double)c / (double)Ns;
}

int round_tp(int T) { return T <= 8 ? 8 : T <= 16 ? 16 : T <= 24 ? 24 : T <= 32 ? 32 : T <= 40 ? 40 : T <= 48 ? 48 : T <= 56 ? 56 : 64; }

}  // namespace
}  // namespace elder

using namespace elder;

extern "C" {

int elder_gauss_legendre(int q, double* x, double* w)
{
    if (q < 1 || q > 64 || !x || !w) {
        set_static_error("elder_gauss_legendre: q must be in [1, 64] and x, w non-NULL");
        return ELDER_EINVAL;
    }
    // Newton iteration on P_q from x0 = cos(pi (i + 3/4) / (q + 1/2)), with
    // P_q' = q (x P_q - P_{q-1}) / (x^2 - 1) and w = 2 / ((1 - x^2) P_q'^2).
    std::vector<double> P(q + 1);
    for (int i = 0; i < q; ++i) {
        double z = std::cos(3.14159265358979323846 * (i + 0.75) / (q + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            legendre_all(q, z, P.data());
            dp = q * (z * P[q] - P[q - 1]) / (z * z - 1.0);
            const double dz = P[q] / dp;
            z -= dz;
            if (std::fabs(dz) <= 1e-16 * std::max(1.0, std::fabs(z))) break;
        }
        legendre_all(q, z, P.data());
        dp = q * (z * P[q] - P[q - 1]) / (z * z - 1.0);
        x[q - 1 - i] = z;  // ascending order
        w[q - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
    if (q == 1) {
        x[0] = 0.0;
        w[0] = 2.0;
    }
    return ELDER_OK;
}

int elder_gpc_indices(int M, int p, int rule, int* n_terms, int32_t* beta, int capacity)
{
    if (M < 1 || M > kGpcMaxM || p < 0 || p > kGpcMaxDeg || rule < 0 || rule > 2 || !n_terms) {
        set_static_error("elder_gpc_indices: bad argument");
        return ELDER_EINVAL;
    }
    std::vector<std::vector<int32_t>> out;
    std::vector<int32_t> b(M, 0);
    while (true) {
        long long sum = 0, prod = 1;
        for (int j = 0; j < M; ++j) {
            sum += b[j];
            prod *= b[j] + 1;
        }
        const bool ok = rule == 0 ? sum <= p : rule == 1 ? true : prod <= p + 1;
        if (ok) out.push_back(b);
        int j = M - 1;  // odometer over {0..p}^M, last variable fastest
        while (j >= 0 && b[j] == p) b[j--] = 0;
        if (j < 0) break;
        ++b[j];
    }
    std::stable_sort(out.begin(), out.end(), [](const std::vector<int32_t>& a,
                                                const std::vector<int32_t>& c) {
        int sa = 0, sc = 0;
        for (size_t j = 0; j < a.size(); ++j) {
            sa += a[j];
            sc += c[j];
        }
        if (sa != sc) return sa < sc;
        return a < c;
    });
    *n_terms = (int)out.size();
    if (!beta) return ELDER_OK;
    if (capacity < (int)out.size()) {
        set_static_error("elder_gpc_indices: capacity below the number of terms");
        return ELDER_EINVAL;
    }
    for (size_t t = 0; t < out.size(); ++t)
        std::memcpy(beta + t * M, out[t].data(), sizeof(int32_t) * M);
    return ELDER_OK;
}

int elder_gpc_project(int M, int T, const int32_t* beta, int maxdeg, int Nq, const double* theta,
                      const double* w, int N, const double* u, double* coef, double* mean,
                      double* var, void* stream)
{
    if (M < 1 || M > kGpcMaxM || T < 1 || T > 64 || maxdeg < 0 || maxdeg > kGpcMaxDeg ||
        Nq < 1 || N < 1 || !beta || !theta || !w || !u || !coef) {
        set_static_error("elder_gpc_project: bad argument");
        return ELDER_EINVAL;
    }
    const size_t smem = sizeof(double) * ((size_t)T * Nq + T);
    if (smem > 200 * 1024) {
        set_static_error("elder_gpc_project: T * Nq too large for one block's table");
        return ELDER_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int grid = (N + kGpcBS - 1) / kGpcBS;
    const int TP = round_tp(T);
    cudaError_t e = cudaSuccess;
#define ELDER_GPC_PROJ(TPV)                                                                     \
    do {                                                                                        \
        e = cudaFuncSetAttribute(k_gpc_project<TPV>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                 (int)smem);                                                   \
        if (e == cudaSuccess)                                                                   \
            k_gpc_project<TPV><<<grid, kGpcBS, smem, st>>>(M, T, beta, Nq, theta, w, N, u, coef, \
                                                           mean, var, maxdeg);                  \
    } while (0)
    switch (TP) {
        case 8: ELDER_GPC_PROJ(8); break;
        case 16: ELDER_GPC_PROJ(16); break;
        case 24: ELDER_GPC_PROJ(24); break;
        case 32: ELDER_GPC_PROJ(32); break;
        case 40: ELDER_GPC_PROJ(40); break;
        case 48: ELDER_GPC_PROJ(48); break;
        case 56: ELDER_GPC_PROJ(56); break;
        default: ELDER_GPC_PROJ(64); break;
    }
#undef ELDER_GPC_PROJ
    count_launch(1);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_static_error(cudaGetErrorString(e));
        return ELDER_ECUDA;
    }
    return ELDER_OK;
}

int elder_gpc_exceed_engine(int engine, int M, int T, const int32_t* beta, int maxdeg, int N,
                            const double* coef, int n_pts, const int32_t* nodes, int Ns,
                            const double* theta, double threshold, double* p_exceed,
                            void* stream)
{
    if (M < 1 || M > kGpcMaxM || T < 1 || T > 64 || maxdeg < 0 || maxdeg > kGpcMaxDeg ||
        N < 1 || n_pts < 1 || (!nodes && n_pts > N) || Ns < 1 || !beta || !coef || !theta ||
        !p_exceed || engine < 0 || engine > 2) {
        set_static_error("elder_gpc_exceed: bad argument");
        return ELDER_EINVAL;
    }
    const bool tc_ok = M <= kTcMaxM && maxdeg <= kTcMaxDeg && T <= kTcTP;
    if (engine == 2 && !tc_ok) {
        set_static_error("elder_gpc_exceed: the tensor-core count needs M <= 4, maxdeg <= 8, "
                         "T <= 36");
        return ELDER_EINVAL;
    }
    const bool use_tc = engine == 2 || (engine == 0 && tc_ok);
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long* cnt = reinterpret_cast<unsigned long long*>(p_exceed);
    cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * n_pts, st);
    if (e != cudaSuccess) {
        set_static_error(cudaGetErrorString(e));
        return ELDER_ECUDA;
    }
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const float thr = (float)threshold;
    int* err = nullptr;
    if (use_tc) {
        void* ep = nullptr;
        e = cudaGetSymbolAddress(&ep, g_gpc_tc_err);
        if (e == cudaSuccess) e = cudaMemsetAsync(ep, 0, sizeof(int), st);
        if (e != cudaSuccess) {
            set_static_error(cudaGetErrorString(e));
            return ELDER_ECUDA;
        }
        err = static_cast<int*>(ep);
        const int gx = (n_pts + kTcTiles * kTcRows - 1) / (kTcTiles * kTcRows);
        const int nchunk = (Ns + kTcCols - 1) / kTcCols;
        // one CTA fits an SM: split the chunks into gy slices so that the
        // waves of gx * gy CTAs times the chunks per slice is least (the last
        // wave otherwise runs part-empty), with at least 16 chunks per slice
        // so that each CTA's set-up (TMEM, coefficients) stays amortised
        // (the fewest slices within 0.5 % of the least cost)
        const int gy_max = std::min(65535, std::max(1, nchunk / 16));
        auto slice_cost = [&](int g) {
            return (((long long)gx * g + sms - 1) / sms) * ((nchunk + g - 1) / g);
        };
        long long best = slice_cost(1);
        for (int g = 2; g <= gy_max; ++g) best = std::min(best, slice_cost(g));
        int gy = 1;
        while (gy < gy_max && slice_cost(gy) * 200 > best * 201) ++gy;
        // operands, then 1 KiB of barriers, TMEM slot, indices and flag,
        // then the Legendre table [4][9][kTcSplit * 128]
        const size_t smem = 2 * (size_t)kTcTileBytes + 1024 +
                            sizeof(float) * kTcMaxM * (kTcMaxDeg + 1) * kTcSplit * kTcCols;
        e = cudaFuncSetAttribute(k_gpc_exceed_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e == cudaSuccess) {
            k_gpc_exceed_tc<<<dim3(gx, gy), kTcThreads, smem, st>>>(M, T, beta, maxdeg, N, coef, n_pts,
                                                             nodes, Ns, theta, thr, cnt, err);
            count_launch(1);
        }
    } else {
        const int TP = (T + 3) / 4 * 4;       // terms padded to a multiple of 4
        const int NPT = TP <= 36 ? 4 : 2;     // listed nodes per thread
        const int gx = (n_pts + NPT * kGpcBS - 1) / (NPT * kGpcBS);
        // enough sample slices to give every SM several blocks, at least one
        // chunk per slice
        int gy = std::max(1, (8 * sms + gx - 1) / gx);
        gy = std::min(gy, std::max(1, (Ns + kGpcChunk - 1) / kGpcChunk));
        gy = std::min(gy, 65535);
        dim3 grid(gx, gy);
        const size_t smem = sizeof(float) * ((size_t)kGpcChunk * TP + (size_t)kGpcChunk * M * (maxdeg + 1)) +
                            sizeof(int) * (size_t)T * M;
#define ELDER_GPC_EXC(TPV, NPTV)                                                                   \
    do {                                                                                           \
        cudaFuncSetAttribute(k_gpc_exceed<TPV, NPTV, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             (int)smem);                                                           \
        k_gpc_exceed<TPV, NPTV, 4><<<grid, kGpcBS, smem, st>>>(M, T, beta, N, coef, n_pts, nodes, Ns, \
                                                            theta, thr, maxdeg, cnt);              \
    } while (0)
        switch (TP) {
            case 4: ELDER_GPC_EXC(4, 4); break;
            case 8: ELDER_GPC_EXC(8, 4); break;
            case 12: ELDER_GPC_EXC(12, 4); break;
            case 16: ELDER_GPC_EXC(16, 4); break;
            case 20: ELDER_GPC_EXC(20, 4); break;
            case 24: ELDER_GPC_EXC(24, 4); break;
            case 28: ELDER_GPC_EXC(28, 4); break;
            case 32: ELDER_GPC_EXC(32, 4); break;
            case 36: ELDER_GPC_EXC(36, 4); break;
            case 40: ELDER_GPC_EXC(40, 2); break;
            case 44: ELDER_GPC_EXC(44, 2); break;
            case 48: ELDER_GPC_EXC(48, 2); break;
            case 52: ELDER_GPC_EXC(52, 2); break;
            case 56: ELDER_GPC_EXC(56, 2); break;
            case 60: ELDER_GPC_EXC(60, 2); break;
            default: ELDER_GPC_EXC(64, 2); break;
        }
#undef ELDER_GPC_EXC
        count_launch(1);
    }
    k_gpc_counts_to_fraction<<<(n_pts + 255) / 256, 256, 0, st>>>(n_pts, Ns, p_exceed, err);
    count_launch(1);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_static_error(cudaGetErrorString(e));
        return ELDER_ECUDA;
    }
    return ELDER_OK;
}

int elder_gpc_exceed(int M, int T, const int32_t* beta, int maxdeg, int N, const double* coef,
                     int n_pts, const int32_t* nodes, int Ns, const double* theta,
                     double threshold, double* p_exceed, void* stream)
{
    return elder_gpc_exceed_engine(0, M, T, beta, maxdeg, N, coef, n_pts, nodes, Ns, theta,
                                   threshold, p_exceed, stream);
}

}  // extern "C"
