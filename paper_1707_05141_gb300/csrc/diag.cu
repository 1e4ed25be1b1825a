// diag.cu -- diagnostics outside the method: direct access to the sampling generator (so that tests
// can compare it word for word with an independent implementation) and an FMA throughput probe
// (so that the benchmark measures the FP32 / FP64 pipe peaks its ALU rooflines divide by).
#include <cuda_runtime.h>

#include "common.cuh"
#include "philox.cuh"

namespace bsvd {

__global__ void philox_gauss_kernel(int count, const unsigned* ctr, unsigned long long seed, unsigned* words,
                                    float* gauss, double* gauss64)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
    if (words) {
        const uint4 w = philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
        words[4 * i] = w.x;
        words[4 * i + 1] = w.y;
        words[4 * i + 2] = w.z;
        words[4 * i + 3] = w.w;
    }
    // counter (g, c, index, tag) of the sampling streams: g = rows / 4, c = column
    if (gauss) {
        const float4 z = gauss4(seed, c.z, c.w, c.x, c.y);
        gauss[4 * i] = z.x;
        gauss[4 * i + 1] = z.y;
        gauss[4 * i + 2] = z.z;
        gauss[4 * i + 3] = z.w;
    }
    if (gauss64) {
        const Gauss4d z = gauss4d(seed, c.z, c.w, c.x, c.y);
        gauss64[4 * i] = z.x;
        gauss64[4 * i + 1] = z.y;
        gauss64[4 * i + 2] = z.z;
        gauss64[4 * i + 3] = z.w;
    }
}

// 16 independent FMA chains per thread (enough to hide the pipe latency at any occupancy the grid
// gives); the chains are summed and stored so that nothing is dead code
template <typename T>
__global__ void __launch_bounds__(256) fma_probe_kernel(int iters, T x, T y, T* out)
{
    T a[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) a[c] = T(threadIdx.x + c);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < 16; ++c) a[c] = fma(a[c], x, y);
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < 16; ++c) s += a[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace bsvd

using namespace bsvd;

extern "C" {

int bsvd_philox_gauss(int count, const unsigned* d_ctr, unsigned long long seed, unsigned* d_words, float* d_gauss,
                      double* d_gauss64, void* stream)
{
    if (count < 0) return -1;
    if (count == 0) return BSVD_SUCCESS;
    if (!d_ctr) return -2;
    cudaStream_t st = (cudaStream_t)stream;
    philox_gauss_kernel<<<(count + 127) / 128, 128, 0, st>>>(count, d_ctr, seed, d_words, d_gauss, d_gauss64);
    return cudaGetLastError() == cudaSuccess ? BSVD_SUCCESS : BSVD_ERR_CUDA;
}

long long bsvd_fma_probe(int dtype, int blocks, int iters, void* d_out, void* stream)
{
    if (dtype != BSVD_F32 && dtype != BSVD_F64) return -1;
    if (blocks < 1) return -2;
    if (iters < 1) return -3;
    if (!d_out) return -4;
    cudaStream_t st = (cudaStream_t)stream;
    if (dtype == BSVD_F32)
        fma_probe_kernel<float><<<blocks, 256, 0, st>>>(iters, 0.999999f, 1e-7f, (float*)d_out);
    else
        fma_probe_kernel<double><<<blocks, 256, 0, st>>>(iters, 0.999999999, 1e-12, (double*)d_out);
    if (cudaGetLastError() != cudaSuccess) return BSVD_ERR_CUDA;
    return 2LL * 16 * 256 * (long long)blocks * iters;  // flops
}

}  // extern "C"
