// common.cuh -- device helpers shared by the batched QR / Jacobi / randomized SVD kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/bsvd.h"

namespace bsvd {

// unit roundoff of each element type
template <typename T> struct Unit;
template <> struct Unit<float> { static constexpr double value = 5.9604644775390625e-08; };   // 2^-24
template <> struct Unit<double> { static constexpr double value = 1.1102230246251565e-16; };  // 2^-53

__device__ __forceinline__ float dsqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double dsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float drsqrt(float x) { return __frsqrt_rn(x); }
__device__ __forceinline__ double drsqrt(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ float rcp_rn(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp_rn(double x) { return __drcp_rn(x); }
__device__ __forceinline__ float dabs(float x) { return fabsf(x); }
__device__ __forceinline__ double dabs(double x) { return fabs(x); }

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// sum over aligned groups of G consecutive lanes (G a power of two <= 32)
template <int G, typename T>
__device__ __forceinline__ T group_sum(T v)
{
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Round-robin ("circle") ordering of Section 5: np (even) column positions, np - 1 steps of
// np / 2 disjoint pairs; position np - 1 stays fixed while the others rotate by one each step.
// Returns the pair (p < q) handled by slot k in step `step`.  (Host-callable for tests.)
__host__ __device__ __forceinline__ void round_robin_pair(int np, int step, int k, int& p, int& q)
{
    int a, b;
    if (k == 0) {
        a = np - 1;
        b = step;
    } else {
        const int r = np - 1;
        a = step + k;
        if (a >= r) a -= r;
        b = step - k;
        if (b < 0) b += r;
    }
    p = a < b ? a : b;
    q = a < b ? b : a;
}

// rot(G) of Algorithm 2 in precision P: returns true and (c, s) when the pair must be rotated.
template <typename P>
__device__ __forceinline__ bool jacobi_rotation(P alpha, P beta, P gamma, P tol, P& c, P& s)
{
    if (!(alpha > P(0)) || !(beta > P(0))) return false;
    if (dabs(gamma) <= tol * dsqrt(alpha) * dsqrt(beta)) return false;
    const P zeta = (beta - alpha) / (P(2) * gamma);
    const P big = sizeof(P) == 4 ? P(1e18) : P(1e150);
    P t;
    if (dabs(zeta) > big)
        t = P(0.5) / zeta;
    else
        t = (zeta >= P(0) ? P(1) : P(-1)) / (dabs(zeta) + dsqrt(P(1) + zeta * zeta));
    c = drsqrt(P(1) + t * t);
    s = c * t;
    return true;
}

// Rotation test |gamma| > tol sqrt(alpha beta) for alpha, beta > 0.  Only the comparison matters, so
// FP32 uses the hardware reciprocal square root (x * rsqrt(x) = sqrt(x) to ~2 ulp) and FP64
// compares squares (no square root; exact up to one rounding, range ample for FP64 data).
__device__ __forceinline__ bool off_diagonal_large(float alpha, float beta, float gamma, float tol)
{
    return fabsf(gamma) > tol * (alpha * rsqrtf(alpha)) * (beta * rsqrtf(beta));
}
__device__ __forceinline__ bool off_diagonal_large(double alpha, double beta, double gamma, double tol)
{
    return gamma * gamma > (tol * tol) * alpha * beta;
}

// 2^-floor(log2 x) for x > 0, read off the exponent bits (exact; clamped at the range ends).
__device__ __forceinline__ float pow2_scale(float x)
{
    int e = (__float_as_int(x) >> 23) & 0xff;
    e = e < 1 ? 1 : (e > 253 ? 253 : e);
    return __int_as_float((254 - e) << 23);
}
__device__ __forceinline__ double pow2_scale(double x)
{
    long long e = (__double_as_longlong(x) >> 52) & 0x7ff;
    e = e < 1 ? 1 : (e > 2045 ? 2045 : e);
    return __longlong_as_double((2046 - e) << 52);
}

// Smaller root t of t^2 + 2 zeta t - 1 = 0, zeta = (beta - alpha) / (2 gamma), written as
// t = 2 gamma sign(beta - alpha) / (|beta - alpha| + sqrt((beta - alpha)^2 + 4 gamma^2))
// (one division, one square root).  t is invariant under scaling (beta - alpha, gamma) together,
// so both are first scaled by a power of two to [1, 2): the squares can then neither overflow nor
// underflow, which matters when alpha, beta, gamma are themselves squares of small numbers.
template <typename P>
__device__ __forceinline__ P jacobi_t(P alpha, P beta, P gamma)
{
    const P d = beta - alpha, g2 = P(2) * gamma;
    const P ad = dabs(d), ag = dabs(g2);
    const P sc = pow2_scale(ad > ag ? ad : ag);
    const P dn = ad * sc, gn = g2 * sc;
    const P t = gn / (dn + dsqrt(dn * dn + gn * gn));
    return d >= P(0) ? t : -t;
}

// Grid for a persistent launch: as many CTAs as can be resident at once (SM count x occupancy),
// never more than the work items.
template <typename K>
inline int persistent_grid(K kernel, int threads, size_t smem, long long work)
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem);
    if (sms < 1) sms = 1;
    if (per < 1) per = 1;
    const long long g = (long long)sms * per;
    const long long n = work < g ? work : g;
    return (int)(n > 0 ? n : 1);
}

// Dynamic work queue for persistent kernels: the CTA claims its next position with one atomic on
// a counter zeroed (by a memset in stream order) before the launch.  Called by all threads; the
// first barrier also separates the previous item's shared-memory use from the next one's.
__device__ __forceinline__ long long next_work(unsigned long long* counter)
{
    __shared__ long long s_item;
    __syncthreads();
    if (threadIdx.x == 0) s_item = (long long)atomicAdd(counter, 1ull);
    __syncthreads();
    return s_item;
}

// The items a batched kernel visits.  Without a list (idx == null) the grid has one CTA per item
// and the hardware scheduler balances items of uneven cost.  With a list -- item indices in device
// memory whose length is known only on the device, e.g. the matrices still active in a later
// round of a captured CUDA graph -- the grid is persistent and its CTAs claim list positions from
// `claim`, so an item left out of the list costs nothing.
struct ItemList {
    const int* idx;             // item indices (device), or null: every item of the batch
    const int* count;           // number of entries of idx (device)
    unsigned long long* claim;  // claim counter (device); the launcher zeroes it
};

inline ItemList all_items() { return ItemList{nullptr, nullptr, nullptr}; }

__device__ __forceinline__ int list_item(const ItemList& wl)
{
    const long long i = next_work(wl.claim);
    return i < (long long)*wl.count ? wl.idx[i] : -1;
}

// first item of this CTA, or -1; every thread of the CTA must call it
__device__ __forceinline__ int item_first(const ItemList& wl, int batch)
{
    if (wl.idx == nullptr) return (int)blockIdx.x < batch ? (int)blockIdx.x : -1;
    return list_item(wl);
}

// next item after b, or -1; every thread of the CTA must call it
__device__ __forceinline__ int item_next(const ItemList& wl, int batch, int b)
{
    if (wl.idx == nullptr) {
        __syncthreads();  // the shared memory of item b is reused by the next one
        const long long nb = (long long)b + gridDim.x;
        return nb < batch ? (int)nb : -1;
    }
    return list_item(wl);
}

// Grid of a launch over `batch` items (or over a list of at most `batch` entries, whose claim
// counter is zeroed here in stream order); 0 on a CUDA error.
template <typename K>
inline int item_grid(K kernel, int threads, size_t smem, const ItemList& wl, int batch, cudaStream_t st)
{
    if (wl.idx == nullptr) return batch < 1 ? 1 : (batch < (1 << 30) ? batch : (1 << 30));
    if (cudaMemsetAsync(wl.claim, 0, sizeof(unsigned long long), st) != cudaSuccess) return 0;
    return persistent_grid(kernel, threads, smem, batch);
}

inline int ceil_div(int a, int b) { return (a + b - 1) / b; }

}  // namespace bsvd
