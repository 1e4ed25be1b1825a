// house.cuh -- Householder QR of one matrix held in shared memory by the threads of a CTA
// (Algorithm 1, Section 2.1; the per-matrix factorisation of Section 3.1's batched kernel).
#pragma once

#include "common.cuh"

namespace bsvd {

// Factor the m x n (m >= n) column-major matrix S (leading dimension ld) in place with all
// blockDim.x threads (whole warps): for each column i a single warp forms the reflector
// v = house(S(i:m, i)) (norm by a warp shuffle reduction), stores it, normalised so that the
// reflector is I - 2 v v^T, in S(i:m, i) and R(i, i) = -sign(x_0) ||x|| in diag[i]; then every warp
// applies it to the trailing columns, one column per warp (M^T v as a warp reduction, then the
// rank-1 update).  On return the strict upper triangle of S holds R above its diagonal.  A zero
// column gives v = 0 (identity reflector) and R(i, i) = 0.  Callers synchronise before and after.
template <typename T>
__device__ __forceinline__ void house_factor_smem(T* S, int ld, T* diag, int m, int n)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int i = 0; i < n; ++i) {
        T* col = S + (size_t)i * ld;
        if (warp == 0) {
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
        __syncthreads();
        for (int j = i + 1 + warp; j < n; j += nwarps) {
            T* cj = S + (size_t)j * ld;
            T w = T(0);
            for (int r = i + lane; r < m; r += 32) w += col[r] * cj[r];
            w = T(2) * warp_sum(w);
            for (int r = i + lane; r < m; r += 32) cj[r] -= w * col[r];
        }
        __syncthreads();
    }
}

}  // namespace bsvd
