// philox.cuh -- counter-based Gaussian sampling for the randomized SVD (Omega = Rand(n, k+p), §7).
//
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as easy as 1, 2, 3",
// SC 2011): ten rounds, each two 32x32->64-bit multiplies by 0xD2511F53 and 0xCD9E8D57 whose
// high halves are xored with the other words and the key; the key is bumped by the Weyl
// constants 0x9E3779B9, 0xBB67AE85 between rounds.  Normals by Box & Muller (1958).
//
// Entry (row r, column c) of Gaussian stream `tag` of matrix `index` under `seed`: counter
// (r / 4, c, index, tag), key (seed low, seed high); words (w0, w1) give rows 4g and 4g+1,
// (w2, w3) rows 4g+2 and 4g+3, with u = (w + 1/2) 2^-32 and z = sqrt(-2 ln u_a) (cos, sin)(2 pi u_b).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace bsvd {

__device__ __forceinline__ uint4 philox4x32_10(uint4 x, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * x.x, hi0 = __umulhi(0xD2511F53u, x.x);
        const uint32_t lo1 = 0xCD9E8D57u * x.z, hi1 = __umulhi(0xCD9E8D57u, x.z);
        x = make_uint4(hi1 ^ x.y ^ k0, lo1, hi0 ^ x.w ^ k1, lo0);
    }
    return x;
}

// the four normals of rows 4g .. 4g+3 of column c
__device__ __forceinline__ float4 gauss4(unsigned long long seed, uint32_t index, uint32_t tag, uint32_t g, uint32_t c)
{
    const uint4 w = philox4x32_10(make_uint4(g, c, index, tag), (uint32_t)seed, (uint32_t)(seed >> 32));
    const float s32 = 2.3283064365386963e-10f;  // 2^-32
    const float ua = ((float)w.x + 0.5f) * s32, ub = ((float)w.y + 0.5f) * s32;
    const float uc = ((float)w.z + 0.5f) * s32, ud = ((float)w.w + 0.5f) * s32;
    const float r0 = sqrtf(-2.0f * logf(ua)), r1 = sqrtf(-2.0f * logf(uc));
    float s0, c0, s1, c1;
    sincospif(2.0f * ub, &s0, &c0);
    sincospif(2.0f * ud, &s1, &c1);
    return make_float4(r0 * c0, r0 * s0, r1 * c1, r1 * s1);
}

// four FP64 normals
struct Gauss4d {
    double x, y, z, w;
};

// the same four normals in FP64 (the FP64 randomized SVD): uniforms exact in double, double log
// and sin / cos
__device__ __forceinline__ Gauss4d gauss4d(unsigned long long seed, uint32_t index, uint32_t tag, uint32_t g,
                                           uint32_t c)
{
    const uint4 w = philox4x32_10(make_uint4(g, c, index, tag), (uint32_t)seed, (uint32_t)(seed >> 32));
    const double s32 = 2.3283064365386963e-10;  // 2^-32
    const double ua = ((double)w.x + 0.5) * s32, ub = ((double)w.y + 0.5) * s32;
    const double uc = ((double)w.z + 0.5) * s32, ud = ((double)w.w + 0.5) * s32;
    const double r0 = sqrt(-2.0 * log(ua)), r1 = sqrt(-2.0 * log(uc));
    double s0, c0, s1, c1;
    sincospi(2.0 * ub, &s0, &c0);
    sincospi(2.0 * ud, &s1, &c1);
    return Gauss4d{r0 * c0, r0 * s0, r1 * c1, r1 * s1};
}

__device__ __forceinline__ float gauss1(unsigned long long seed, uint32_t index, uint32_t tag, uint32_t r, uint32_t c)
{
    const float4 z = gauss4(seed, index, tag, r >> 2, c);
    const int s = r & 3;
    return s == 0 ? z.x : (s == 1 ? z.y : (s == 2 ? z.z : z.w));
}

}  // namespace bsvd
