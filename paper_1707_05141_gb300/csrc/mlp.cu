// mlp.cu -- learned rank predictor for the randomized SVD: sketch features, a 16 -> 64 -> 64 -> 1
// multilayer perceptron (forward, gradient, Adam step).  The paper has no learned part; the
// network only chooses the first sample count of the adaptive range finder, whose posterior
// estimate still decides (and corrects) every result.
//
// Features (16 per block, from one pass over A plus one pass over A^T for 8 Gaussian probes G,
// Philox stream 2):
//   f0, f1    m / 256, n / 256
//   f2        log10 ||A||_F
//   f3..f6    log10 of (max, min, mean, rms-deviation) of column norms / ||A||_F
//   f7, f8    log10 mean(y), std(y) / mean(y)   with y_j = ||A g_j||^2 / ||A||_F^2
//   f9..f11   log10 (mean, max, min) of w_j = ||A^T A g_j||^2 / (||A g_j||^2 ||A||_F^2)
//   f12, f13  log10 (max, min) of y_j
//   f14       log10 of the stable-rank estimate ||A||_F^2 / max_j(||A^T A g_j|| / ||A g_j||)^2
//   f15       fraction of ||A||_F^2 in the largest eighth of the column norms
// Network: h1 = relu(W1 f + b1), h2 = relu(W2 h1 + b2), y = w3 . h2 + b3, target log(rank + 1).
// Parameter vector: W1 (64 x 16 row-major), b1 (64), W2 (64 x 64), b2 (64), w3 (64), b3 (1).
#include <cuda_runtime.h>

#include "common.cuh"
#include "philox.cuh"

namespace bsvd {

constexpr int kF = 16, kH = 64;
constexpr int oW1 = 0, oB1 = oW1 + kH * kF, oW2 = oB1 + kH, oB2 = oW2 + kH * kH, oW3 = oB2 + kH, oB3 = oW3 + kH;
constexpr int kParams = oB3 + 1;  // 5313
constexpr int kProbesF = 8;

__device__ __forceinline__ float safe_log10(double x) { return (float)log10(x > 1e-300 ? x : 1e-300); }

// one CTA per block
__global__ void __launch_bounds__(256) sketch_features_kernel(int batch, const float* const* A, const int* M,
                                                              const int* N, const int* LDA, unsigned long long seed,
                                                              float* feat)
{
    __shared__ float cn[256];           // column norms squared
    __shared__ float ys[256][kProbesF]; // Y = A G (m x 8)
    __shared__ double yy[kProbesF], ww[kProbesF];
    const int b = blockIdx.x;
    float* f = feat + (size_t)b * kF;
    const int m = M[b], n = N[b], lda = LDA[b];
    if (m <= 0 || n <= 0 || m > 256 || n > 256 || lda < m) {
        for (int i = threadIdx.x; i < kF; i += blockDim.x) f[i] = 0.f;
        return;
    }
    const float* a = A[b];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // column norms (one warp per column)
    for (int j = warp; j < n; j += 8) {
        float s = 0.f;
        for (int i = lane; i < m; i += 32) s = fmaf(a[(size_t)j * lda + i], a[(size_t)j * lda + i], s);
        s = warp_sum(s);
        if (lane == 0) cn[j] = s;
    }
    // G (n x 8) once per block, four rows per Philox call
    __shared__ float gs[256][kProbesF];
    for (int e = threadIdx.x; e < ((n + 3) / 4) * kProbesF; e += blockDim.x) {
        const int g = e / kProbesF, p = e % kProbesF;
        const float4 z = gauss4(seed, (uint32_t)b, 2u, (uint32_t)g, (uint32_t)p);
        gs[4 * g][p] = z.x;
        if (4 * g + 1 < n) gs[4 * g + 1][p] = z.y;
        if (4 * g + 2 < n) gs[4 * g + 2][p] = z.z;
        if (4 * g + 3 < n) gs[4 * g + 3][p] = z.w;
    }
    __syncthreads();
    // Y = A G, thread per row
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        float acc[kProbesF] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int j = 0; j < n; ++j) {
            const float x = a[(size_t)j * lda + i];
#pragma unroll
            for (int p = 0; p < kProbesF; ++p) acc[p] = fmaf(x, gs[j][p], acc[p]);
        }
#pragma unroll
        for (int p = 0; p < kProbesF; ++p) ys[i][p] = acc[p];
    }
    __syncthreads();
    // ||Y_p||^2 and ||A^T Y_p||^2
    if (threadIdx.x < kProbesF) {
        double s = 0.0;
        for (int i = 0; i < m; ++i) s += (double)ys[i][threadIdx.x] * ys[i][threadIdx.x];
        yy[threadIdx.x] = s;
    }
    double wacc[kProbesF] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        float z[kProbesF] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int i = 0; i < m; ++i) {
            const float x = a[(size_t)j * lda + i];
#pragma unroll
            for (int p = 0; p < kProbesF; ++p) z[p] = fmaf(x, ys[i][p], z[p]);
        }
#pragma unroll
        for (int p = 0; p < kProbesF; ++p) wacc[p] += (double)z[p] * z[p];
    }
    __shared__ double wpart[8][kProbesF];
#pragma unroll
    for (int p = 0; p < kProbesF; ++p) {
        double v = wacc[p];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) wpart[warp][p] = v;
    }
    __syncthreads();
    if (threadIdx.x < kProbesF) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += wpart[w][threadIdx.x];
        ww[threadIdx.x] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double fro2 = 0.0, cmax = 0.0, cmin = 1e300, lsum = 0.0, lsq = 0.0;
        for (int j = 0; j < n; ++j) {
            const double c = cn[j];
            fro2 += c;
        }
        const double fro = sqrt(fro2);
        for (int j = 0; j < n; ++j) {
            const double r = sqrt((double)cn[j]) / (fro > 0 ? fro : 1.0);
            cmax = r > cmax ? r : cmax;
            cmin = r < cmin ? r : cmin;
            const double l = log10(r > 1e-300 ? r : 1e-300);
            lsum += l;
            lsq += l * l;
        }
        const double lmean = lsum / n;
        // energy in the largest eighth of the columns (partial selection by repeated max)
        int top = n / 8 > 0 ? n / 8 : 1;
        double etop = 0.0;
        {
            float tmp[256];
            for (int j = 0; j < n; ++j) tmp[j] = cn[j];
            for (int t = 0; t < top; ++t) {
                int bi = 0;
                for (int j = 1; j < n; ++j) bi = tmp[j] > tmp[bi] ? j : bi;
                etop += tmp[bi];
                tmp[bi] = -1.f;
            }
        }
        double ymean = 0.0, ymax = 0.0, ymin = 1e300, wmean = 0.0, wmax = 0.0, wmin = 1e300, rmax = 0.0;
        for (int p = 0; p < kProbesF; ++p) {
            const double y = yy[p] / (fro2 > 0 ? fro2 : 1.0);
            const double w = yy[p] > 0 ? ww[p] / (yy[p] * (fro2 > 0 ? fro2 : 1.0)) : 0.0;
            ymean += y / kProbesF;
            ymax = y > ymax ? y : ymax;
            ymin = y < ymin ? y : ymin;
            wmean += w / kProbesF;
            wmax = w > wmax ? w : wmax;
            wmin = w < wmin ? w : wmin;
            const double r = yy[p] > 0 ? sqrt(ww[p] / yy[p]) : 0.0;
            rmax = r > rmax ? r : rmax;
        }
        double ysd = 0.0;
        for (int p = 0; p < kProbesF; ++p) {
            const double y = yy[p] / (fro2 > 0 ? fro2 : 1.0) - ymean;
            ysd += y * y / kProbesF;
        }
        f[0] = m / 256.f;
        f[1] = n / 256.f;
        f[2] = safe_log10(fro);
        f[3] = safe_log10(cmax);
        f[4] = safe_log10(cmin);
        f[5] = (float)lmean;
        f[6] = (float)sqrt(fmax(lsq / n - lmean * lmean, 0.0));
        f[7] = safe_log10(ymean);
        f[8] = (float)(ymean > 0 ? sqrt(ysd) / ymean : 0.0);
        f[9] = safe_log10(wmean);
        f[10] = safe_log10(wmax);
        f[11] = safe_log10(wmin);
        f[12] = safe_log10(ymax);
        f[13] = safe_log10(ymin);
        f[14] = safe_log10(rmax > 0 ? fro2 / (rmax * rmax) : 1.0);
        f[15] = (float)(fro2 > 0 ? etop / fro2 : 0.0);
    }
}

// forward: one thread per sample; weights in shared memory
__device__ __forceinline__ float mlp_eval(const float* P, const float* x, float* h1, float* h2)
{
    for (int o = 0; o < kH; ++o) {
        float s = P[oB1 + o];
#pragma unroll
        for (int i = 0; i < kF; ++i) s = fmaf(P[oW1 + o * kF + i], x[i], s);
        h1[o] = s > 0.f ? s : 0.f;
    }
    for (int o = 0; o < kH; ++o) {
        float s = P[oB2 + o];
        for (int i = 0; i < kH; ++i) s = fmaf(P[oW2 + o * kH + i], h1[i], s);
        h2[o] = s > 0.f ? s : 0.f;
    }
    float y = P[oB3];
    for (int i = 0; i < kH; ++i) y = fmaf(P[oW3 + i], h2[i], y);
    return y;
}

__global__ void __launch_bounds__(128) mlp_forward_kernel(int batch, const float* feat, const float* params, float* out,
                                                          int* hint, float margin, const int* M, const int* N)
{
    __shared__ float P[kParams];
    for (int i = threadIdx.x; i < kParams; i += blockDim.x) P[i] = params[i];
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= batch) return;
    float x[kF], h1[kH], h2[kH];
#pragma unroll
    for (int i = 0; i < kF; ++i) x[i] = feat[(size_t)s * kF + i];
    const float y = mlp_eval(P, x, h1, h2);
    if (out) out[s] = y;
    if (hint) {
        // predicted rank exp(y) - 1, plus a margin, at least 1, at most min(m, n)
        float r = expf(fminf(y, 8.f)) - 1.f + margin;
        r = r > 1.f ? (r < 65536.f ? r : 65536.f) : 1.f;  // also maps a NaN margin to 1: the int below is defined
        int h = (int)ceilf(r);
        if (M && N) {
            const int k = M[s] < N[s] ? M[s] : N[s];
            h = h < k ? h : k;
        }
        hint[s] = h;
    }
}

// gradient of L = (1 / 2B) sum_s (y_s - t_s)^2; grad must be zeroed by the caller's launch
// sequence (mlp_zero_kernel); loss accumulated in *loss
__global__ void __launch_bounds__(128) mlp_grad_kernel(int batch, const float* feat, const float* target,
                                                       const float* params, float* grad, float* loss)
{
    __shared__ float P[kParams];
    __shared__ float G[kParams];
    for (int i = threadIdx.x; i < kParams; i += blockDim.x) {
        P[i] = params[i];
        G[i] = 0.f;
    }
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < batch) {
        float x[kF], h1[kH], h2[kH];
#pragma unroll
        for (int i = 0; i < kF; ++i) x[i] = feat[(size_t)s * kF + i];
        const float y = mlp_eval(P, x, h1, h2);
        const float r = y - target[s];
        atomicAdd(loss, 0.5f * r * r / batch);
        const float dy = r / batch;
        atomicAdd(&G[oB3], dy);
        float d2[kH];
        for (int i = 0; i < kH; ++i) {
            atomicAdd(&G[oW3 + i], dy * h2[i]);
            d2[i] = h2[i] > 0.f ? dy * P[oW3 + i] : 0.f;
        }
        float d1[kH];
        for (int i = 0; i < kH; ++i) d1[i] = 0.f;
        for (int o = 0; o < kH; ++o) {
            if (d2[o] == 0.f) continue;
            atomicAdd(&G[oB2 + o], d2[o]);
            for (int i = 0; i < kH; ++i) {
                atomicAdd(&G[oW2 + o * kH + i], d2[o] * h1[i]);
                d1[i] = fmaf(P[oW2 + o * kH + i], d2[o], d1[i]);
            }
        }
        for (int o = 0; o < kH; ++o) {
            const float d = h1[o] > 0.f ? d1[o] : 0.f;
            if (d == 0.f) continue;
            atomicAdd(&G[oB1 + o], d);
#pragma unroll
            for (int i = 0; i < kF; ++i) atomicAdd(&G[oW1 + o * kF + i], d * x[i]);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kParams; i += blockDim.x)
        if (G[i] != 0.f) atomicAdd(&grad[i], G[i]);
}

__global__ void mlp_zero_kernel(float* grad, float* loss)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kParams; i += gridDim.x * blockDim.x) grad[i] = 0.f;
    if (blockIdx.x == 0 && threadIdx.x == 0 && loss) *loss = 0.f;
}

__global__ void mlp_adam_kernel(int nparams, float* params, const float* grad, float* mom, float* vel, int step,
                                float lr, float b1, float b2, float eps)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nparams) return;
    const float g = grad[i];
    const float m = b1 * mom[i] + (1.f - b1) * g;
    const float v = b2 * vel[i] + (1.f - b2) * g * g;
    mom[i] = m;
    vel[i] = v;
    const float mh = m / (1.f - powf(b1, (float)step));
    const float vh = v / (1.f - powf(b2, (float)step));
    params[i] -= lr * mh / (sqrtf(vh) + eps);
}

}  // namespace bsvd

using namespace bsvd;

extern "C" {

int bsvd_sketch_features(int batch, int max_m, int max_n, void* const* dA, const int* d_m, const int* d_n,
                         const int* d_lda, unsigned long long seed, float* d_features, void* stream)
{
    if (batch < 0) return -1;
    if (max_m < 0 || max_m > 256) return -2;
    if (max_n < 0 || max_n > 256) return -3;
    if (batch == 0) return BSVD_SUCCESS;
    if (!dA) return -4;
    if (!d_m) return -5;
    if (!d_n) return -6;
    if (!d_lda) return -7;
    if (!d_features) return -9;
    sketch_features_kernel<<<batch, 256, 0, (cudaStream_t)stream>>>(batch, (const float* const*)dA, d_m, d_n, d_lda,
                                                                     seed, d_features);
    return cudaGetLastError() == cudaSuccess ? BSVD_SUCCESS : BSVD_ERR_CUDA;
}

int bsvd_mlp_forward(int batch, const float* d_features, const float* d_params, float* d_out, int* d_rank_hint,
                     float margin, const int* d_m, const int* d_n, void* stream)
{
    if (batch < 0) return -1;
    if (batch == 0) return BSVD_SUCCESS;
    if (!d_features) return -2;
    if (!d_params) return -3;
    if (!d_out && !d_rank_hint) return -4;
    mlp_forward_kernel<<<(batch + 127) / 128, 128, 0, (cudaStream_t)stream>>>(batch, d_features, d_params, d_out,
                                                                              d_rank_hint, margin, d_m, d_n);
    return cudaGetLastError() == cudaSuccess ? BSVD_SUCCESS : BSVD_ERR_CUDA;
}

int bsvd_mlp_grad(int batch, const float* d_features, const float* d_target, const float* d_params, float* d_grad,
                  float* d_loss, void* stream)
{
    if (batch < 0) return -1;
    if (!d_features) return -2;
    if (!d_target) return -3;
    if (!d_params) return -4;
    if (!d_grad) return -5;
    if (!d_loss) return -6;
    cudaStream_t st = (cudaStream_t)stream;
    mlp_zero_kernel<<<8, 256, 0, st>>>(d_grad, d_loss);
    if (batch > 0)
        mlp_grad_kernel<<<(batch + 127) / 128, 128, 0, st>>>(batch, d_features, d_target, d_params, d_grad, d_loss);
    return cudaGetLastError() == cudaSuccess ? BSVD_SUCCESS : BSVD_ERR_CUDA;
}

int bsvd_mlp_adam(int nparams, float* d_params, const float* d_grad, float* d_m, float* d_v, int step, float lr,
                  float beta1, float beta2, float eps, void* stream)
{
    if (nparams != kParams) return -1;
    if (!d_params) return -2;
    if (!d_grad) return -3;
    if (!d_m) return -4;
    if (!d_v) return -5;
    if (step < 1) return -6;
    mlp_adam_kernel<<<(nparams + 255) / 256, 256, 0, (cudaStream_t)stream>>>(nparams, d_params, d_grad, d_m, d_v, step,
                                                                             lr, beta1, beta2, eps);
    return cudaGetLastError() == cudaSuccess ? BSVD_SUCCESS : BSVD_ERR_CUDA;
}

int bsvd_mlp_param_count(void) { return kParams; }

}  // extern "C"
