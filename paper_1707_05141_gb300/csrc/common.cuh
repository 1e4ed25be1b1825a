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
// Returns the pair (p < q) handled by slot k in step `step`.
__device__ __forceinline__ void round_robin_pair(int np, int step, int k, int& p, int& q)
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

inline int ceil_div(int a, int b) { return (a + b - 1) / b; }

}  // namespace bsvd
