// house.cuh -- Householder QR of one matrix held in shared memory by the threads of a CTA
// (Algorithm 1, Section 2.1; the per-matrix factorisation of Section 3.1's batched kernel).
#pragma once

#include "common.cuh"

namespace bsvd {

// The reflector of column i, formed by one warp: v = house(S(i:m, i)) (norm by a warp shuffle
// reduction), stored normalised so that the reflector is I - 2 v v^T in S(i:m, i), and
// R(i, i) = -sign(x_0) ||x|| in diag[i].  A zero column gives v = 0 (identity reflector), R(i, i) = 0.
template <typename T>
__device__ __forceinline__ void house_reflector(T* col, int i, int m, T* diag, int lane)
{
    const T x0 = col[i];  // read by every lane before the shuffles below
    T ss = T(0);
    for (int r = i + lane; r < m; r += 32) ss += col[r] * col[r];
    ss = warp_sum(ss);
    const T alpha = dsqrt(ss);
    if (alpha > T(0)) {
        const T sg = x0 >= T(0) ? T(1) : T(-1);
        // ||x + sign(x0) alpha e1||^2 = 2 alpha (alpha + |x0|)
        const T inv = drsqrt(T(2) * alpha * (alpha + dabs(x0)));
        for (int r = i + lane; r < m; r += 32) col[r] = (r == i ? x0 + sg * alpha : col[r]) * inv;
        if (lane == 0) diag[i] = -sg * alpha;
    } else if (lane == 0) {
        diag[i] = T(0);  // zero column: v = 0 (already zero), identity reflector
    }
}

// Factor the m x n (m >= n) column-major matrix S (leading dimension ld) in place with all
// blockDim.x threads (whole warps): reflector i (house_reflector) is applied to the trailing
// columns, one column per warp (M^T v as a warp reduction, then the rank-1 update).  Look-ahead:
// the warp that owns column i + 1 updates it first and forms reflector i + 1 at once, while the
// other warps are still applying reflector i to their columns, so each column costs one barrier.
// On return the strict upper triangle of S holds R above its diagonal.  Callers synchronise
// before and after.
template <typename T>
__device__ __forceinline__ void house_factor_smem(T* S, int ld, T* diag, int m, int n)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    if (n > 0 && warp == 0) house_reflector(S, 0, m, diag, lane);
    __syncthreads();
    for (int i = 0; i < n; ++i) {
        const T* col = S + (size_t)i * ld;
        // this warp's first column right of i: columns j with j % nwarps == warp
        const int first = i + 1 + ((warp - (i + 1) % nwarps) + nwarps) % nwarps;
        for (int j = first; j < n; j += nwarps) {
            T* cj = S + (size_t)j * ld;
            T w = T(0);
            for (int r = i + lane; r < m; r += 32) w += col[r] * cj[r];
            w = T(2) * warp_sum(w);
            for (int r = i + lane; r < m; r += 32) cj[r] -= w * col[r];
            if (j == i + 1) {
                __syncwarp();
                house_reflector(cj, j, m, diag, lane);
            }
        }
        __syncthreads();
    }
}

// The same factorisation for m <= 32 RPL: each warp keeps reflector i's rows (i + lane + 32 t) in
// registers for the whole step and each of its trailing columns in registers between the product and
// the update, so an element costs one shared load, one shared store and two FMAs (the loop above
// reads the reflector twice and the column twice).
template <typename T, int RPL>
__device__ __forceinline__ void house_factor_smem_rows(T* S, int ld, T* diag, int m, int n)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    if (n > 0 && warp == 0) house_reflector(S, 0, m, diag, lane);
    __syncthreads();
    for (int i = 0; i < n; ++i) {
        const T* col = S + (size_t)i * ld;
        T v[RPL];
#pragma unroll
        for (int t = 0; t < RPL; ++t) {
            const int r = i + lane + 32 * t;
            v[t] = r < m ? col[r] : T(0);
        }
        const int first = i + 1 + ((warp - (i + 1) % nwarps) + nwarps) % nwarps;
        // two of the warp's columns at a time: their reductions are independent, so their shuffle
        // latencies overlap (the second is a column past n when the warp has an odd count left)
        for (int j = first; j < n; j += 2 * nwarps) {
            const int j2 = j + nwarps;
            const bool two = j2 < n;
            T* cj = S + (size_t)j * ld;
            T* cj2 = S + (size_t)(two ? j2 : j) * ld;
            T x[RPL], y[RPL];
            T w0 = T(0), w1 = T(0);
#pragma unroll
            for (int t = 0; t < RPL; ++t) {
                const int r = i + lane + 32 * t;
                x[t] = r < m ? cj[r] : T(0);
                y[t] = r < m && two ? cj2[r] : T(0);
                w0 = fma(v[t], x[t], w0);
                w1 = fma(v[t], y[t], w1);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                w0 += __shfl_xor_sync(0xffffffffu, w0, o);
                w1 += __shfl_xor_sync(0xffffffffu, w1, o);
            }
            w0 *= T(2);
            w1 *= T(2);
#pragma unroll
            for (int t = 0; t < RPL; ++t) {
                const int r = i + lane + 32 * t;
                if (r < m) {
                    cj[r] = fma(-w0, v[t], x[t]);
                    if (two) cj2[r] = fma(-w1, v[t], y[t]);
                }
            }
            if (j == i + 1) {
                __syncwarp();
                house_reflector(cj, j, m, diag, lane);
            }
        }
        __syncthreads();
    }
}

}  // namespace bsvd
