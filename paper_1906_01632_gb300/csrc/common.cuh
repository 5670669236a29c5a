// common.cuh -- device-side definitions shared by the Elder step kernels.
//
// Grid, physical constants, Dirichlet bits and small vector types.  The
// discretisation is the vertex-centred box method of Section 2.3 on a
// structured hexahedral box; node n = i + (nx+1)*(j + (ny+1)*k), cell
// e = i + nx*(j + ny*k).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "bits.cuh"

namespace elder {

// Division of a 32-bit unsigned dividend by a fixed divisor d through a
// multiply-high and two shifts (Granlund and Montgomery, "Division by
// invariant integers using multiplication", PLDI 1994, Figure 4.1): with
// l = ceil(log2 d) and m = floor(2^32 (2^l - d) / d) + 1, the quotient is
// (t + ((n - t) >> min(l, 1))) >> max(l - 1, 0), t = mulhi(m, n), exact for
// every n < 2^32.
struct FastDiv {
    unsigned m;
    int s1, s2;
};

inline FastDiv make_fastdiv(unsigned d)
{
    int l = 0;
    while ((1ull << l) < d) ++l;
    const unsigned long long m = ((1ull << 32) * ((1ull << l) - d)) / d + 1;
    return FastDiv{(unsigned)m, l < 1 ? l : 1, l > 1 ? l - 1 : 0};
}

struct Grid {
    int nx, ny, nz;   // cells per direction
    int N, C;         // nodes, cells
    double hx, hy, hz;
    double Lz;
    FastDiv d_row, d_plane;  // division by nx+1 and by (nx+1)(ny+1)
};

inline void grid_set_divisors(Grid& G)
{
    G.d_row = make_fastdiv((unsigned)(G.nx + 1));
    G.d_plane = make_fastdiv((unsigned)((G.nx + 1) * (G.ny + 1)));
}

// Constants of Table 1 / eq. e_lin_density and the time step.
struct Phys {
    double rho0, drho;   // rho(c) = rho0 + drho * c
    double mu, g, Dm;    // viscosity, gravity (along -z), molecular diffusion
    double dt;           // time step [s]
};

// Per-sample status codes (values of the C ABI's ELDER_SAMPLE_*).
constexpr int ELDER_SAMPLE_NEWTON_MAXIT_ = 1;
constexpr int ELDER_SAMPLE_KRYLOV_MAXIT_ = 2;
constexpr int ELDER_SAMPLE_BREAKDOWN_ = 3;
constexpr int ELDER_SAMPLE_NONFINITE_ = 4;
constexpr int ELDER_SAMPLE_LINESEARCH_ = 5;

// Dirichlet bits per node (the same on every sample).
enum : uint8_t { BC_P = 1, BC_C = 2 };

// Column slot of the neighbour at offset (dx,dy,dz) in a 27-point row.
__host__ __device__ constexpr int slot27(int dx, int dy, int dz)
{
    return (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1);
}

template <class T> struct alignas(2 * sizeof(T)) V2 { T p, c; };
// 2x2 Jacobian block: rows (p-eq, c-eq) x cols (p, c).
template <class T> struct alignas(4 * sizeof(T)) B4 { T pp, pc, cp, cc; };

// Storage type of the multigrid matrices for solver precision T: the FP32
// solver keeps them in bfloat16 (the V-cycle is only a preconditioner; the
// Krylov operator keeps its FP32 copy), the FP64 solver in double.
template <class T> struct MgType { using type = T; };
template <> struct MgType<float> { using type = __nv_bfloat16; };

// Arithmetic of the dense coarsest-grid inverse: FP32 under bfloat16
// multigrid matrices (mixed solver), FP64 otherwise.
template <class M> struct CoarseType { using type = double; };
template <> struct CoarseType<__nv_bfloat16> { using type = float; };

template <class T> __device__ __forceinline__ T mg_load(__nv_bfloat16 v)
{
    return T(__bfloat162float(v));
}
template <class T> __device__ __forceinline__ T mg_load(float v) { return T(v); }
template <class T> __device__ __forceinline__ T mg_load(double v) { return T(v); }
template <class M> __device__ __forceinline__ M mg_store(double v) { return M(v); }
template <> __device__ __forceinline__ __nv_bfloat16 mg_store<__nv_bfloat16>(double v)
{
    return __float2bfloat16_rn(float(v));
}

__host__ __device__ inline int node_id(const Grid& G, int i, int j, int k)
{
    return i + (G.nx + 1) * (j + (G.ny + 1) * k);
}

__device__ __forceinline__ unsigned fastdiv(unsigned n, const FastDiv& f)
{
    const unsigned t = __umulhi(f.m, n);
    return (t + ((n - t) >> f.s1)) >> f.s2;
}

// node_ijk by the grid's multiply-high divisors (for the instruction-bound
// transfer kernels)
__device__ __forceinline__ void node_ijk_fast(const Grid& G, int n, int& i, int& j, int& k)
{
    const int nx1 = G.nx + 1;
    k = (int)fastdiv((unsigned)n, G.d_plane);
    const int r = n - k * nx1 * (G.ny + 1);
    j = (int)fastdiv((unsigned)r, G.d_row);
    i = r - j * nx1;
}

__device__ __forceinline__ void node_ijk(const Grid& G, int n, int& i, int& j,
                                         int& k)
{
    int nx1 = G.nx + 1, ny1 = G.ny + 1;
    k = n / (nx1 * ny1);
    int r = n - k * nx1 * ny1;
    j = r / nx1;
    i = r - j * nx1;
}

__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum of one value per thread (blockDim.x a multiple of 32,
// at most 1024); every thread receives the result.
__device__ __forceinline__ float block_sum(float v, float* smem32)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) smem32[w] = v;
    __syncthreads();
    int nw = blockDim.x >> 5;
    float t = (threadIdx.x < nw) ? smem32[threadIdx.x] : 0.0f;
    if (w == 0)
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) smem32[0] = t;
    __syncthreads();
    float r = smem32[0];
    __syncthreads();
    return r;
}

__device__ __forceinline__ double block_sum(double v, double* smem32)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) smem32[w] = v;
    __syncthreads();
    int nw = blockDim.x >> 5;
    double t = (threadIdx.x < nw) ? smem32[threadIdx.x] : 0.0;
    if (w == 0)
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) smem32[0] = t;
    __syncthreads();
    double r = smem32[0];
    __syncthreads();
    return r;
}

// Block-wide maximum of unsigned values (integer pipe)
__device__ __forceinline__ unsigned block_max(unsigned v, unsigned* smem32)
{
    v = __reduce_max_sync(0xffffffffu, v);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) smem32[w] = v;
    __syncthreads();
    int nw = blockDim.x >> 5;
    unsigned t = (threadIdx.x < nw) ? smem32[threadIdx.x] : 0u;
    if (w == 0) t = __reduce_max_sync(0xffffffffu, t);
    if (threadIdx.x == 0) smem32[0] = t;
    __syncthreads();
    unsigned r = smem32[0];
    __syncthreads();
    return r;
}

__device__ __forceinline__ double block_max(double v, double* smem32)
{
    for (int o = 16; o > 0; o >>= 1)
        v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) smem32[w] = v;
    __syncthreads();
    int nw = blockDim.x >> 5;
    double t = (threadIdx.x < nw) ? smem32[threadIdx.x] : 0.0;
    if (w == 0)
        for (int o = 16; o > 0; o >>= 1)
            t = fmax(t, __shfl_xor_sync(0xffffffffu, t, o));
    if (threadIdx.x == 0) smem32[0] = t;
    __syncthreads();
    double r = smem32[0];
    __syncthreads();
    return r;
}

}  // namespace elder
