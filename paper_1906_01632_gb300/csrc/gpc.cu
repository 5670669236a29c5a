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

__global__ void k_gpc_counts_to_fraction(int n_pts, int Ns, double* p)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_pts) return;
    unsigned long long c;
    memcpy(&c, p + k, sizeof(c));
    p[k] = (double)c / (double)Ns;
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

int elder_gpc_exceed(int M, int T, const int32_t* beta, int maxdeg, int N, const double* coef,
                     int n_pts, const int32_t* nodes, int Ns, const double* theta,
                     double threshold, double* p_exceed, void* stream)
{
    if (M < 1 || M > kGpcMaxM || T < 1 || T > 64 || maxdeg < 0 || maxdeg > kGpcMaxDeg ||
        N < 1 || n_pts < 1 || (!nodes && n_pts > N) || Ns < 1 || !beta || !coef || !theta ||
        !p_exceed) {
        set_static_error("elder_gpc_exceed: bad argument");
        return ELDER_EINVAL;
    }
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
    const int TP = (T + 3) / 4 * 4;       // terms padded to a multiple of 4
    const int NPT = TP <= 36 ? 4 : 2;     // listed nodes per thread
    const int gx = (n_pts + NPT * kGpcBS - 1) / (NPT * kGpcBS);
    // enough sample slices to give every SM several blocks, at least one
    // chunk per slice
    int gy = std::max(1, (8 * sms + gx - 1) / gx);
    gy = std::min(gy, std::max(1, (Ns + kGpcChunk - 1) / kGpcChunk));
    gy = std::min(gy, 65535);
    dim3 grid(gx, gy);
    const float thr = (float)threshold;
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
    k_gpc_counts_to_fraction<<<(n_pts + 255) / 256, 256, 0, st>>>(n_pts, Ns, p_exceed);
    count_launch(2);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_static_error(cudaGetErrorString(e));
        return ELDER_ECUDA;
    }
    return ELDER_OK;
}

}  // extern "C"
