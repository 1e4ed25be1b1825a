// rsvd_tc.cu -- the randomized SVD's sampling product Y = A [Omega | W] on the tensor cores
// (Algorithm 4, step 1; FP32 data).
//
// One CTA of 128 threads per block (persistent over the list of sampling blocks, two CTAs per SM).
// Y's Omega columns are a tcgen05.mma product of kind::tf32 with the accumulator in tensor memory:
// A (m x n, m <= 256, up to two 128-row M tiles) and Omega (n x l, l <= 128, N padded to a multiple
// of 16) are staged in 32-row chunks of K = n in the canonical K-major layout without swizzle
// (two stages, the next chunk loaded while the tensor core multiplies the current one), with Omega
// generated straight into shared memory from the Philox stream (the bits the FP32 sampling draws).
// The tensor core reads the FP32 operands as TF32 (10-bit mantissa) and accumulates in FP32: the
// sample only has to span the dominant subspace, which the power step that follows refines with
// FP32 products.  The 8 probe columns of the posterior estimate must stay FP32-accurate: they are
// summed on the FP32 pipes from the same staged A chunks, so A is read from memory once.
// Every wait is bounded; a wait that gives up raises a flag the finish kernel turns into
// BSVD_INFO_DEVICE_TIMEOUT, and the CTA drains its own MMAs (bounded again) before freeing TMEM.
#include <cuda_runtime.h>

#include "common.cuh"
#include "launch.cuh"
#include "philox.cuh"
#include "tcgen05.cuh"

namespace bsvd {

namespace {

constexpr int kKc = 32;                                     // K (rows of A^T / Omega) per chunk
constexpr int kProbeCols = 8;
constexpr uint32_t kLbo = 128;                              // K-adjacent core matrices
constexpr uint32_t kSbo = (kKc / 4) * 128;                  // 1024 B between 8-row groups
constexpr uint32_t kATile = 128u * kKc * 4u;                // 16 KB: one 128-row M tile x 32 K
constexpr uint32_t kStageA = 2 * kATile;                    // two M tiles
constexpr uint32_t kStageB = 128u * kKc * 4u;               // up to 128 Omega columns x 32 K
constexpr uint32_t kStage = kStageA + kStageB;              // 48 KB
constexpr int kStages = 2;
constexpr uint32_t kTmemCols = 256;                         // two M tiles x up to 128 columns
constexpr size_t kSmem = kStages * kStage + 1024 + 64;      // + alignment slack

__device__ __forceinline__ unsigned char* align1k(unsigned char* p)
{
    return reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(p) + 1023) & ~(uintptr_t)1023);
}

// sample of one block: Y(:, 0:l) = A Omega on the tensor cores, Y(:, l:l+8) = A W on the FP32 pipes
__device__ __forceinline__ void sample_item(int b, float* const* A, const int* LDA, float* const* Y, const int* M,
                                            const int* N, const int* L, unsigned long long seed,
                                            unsigned char* sm, uint32_t tmem, uint64_t* bars, uint32_t& phase,
                                            uint32_t& used, float (*wsm)[kProbeCols], int* timeouts)
{
    const int m = M[b], n = N[b], l = L[b];
    if (m <= 0 || n <= 0 || l <= 0) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float* a = A[b];
    const int lda = LDA[b];
    const int mt = (m + 127) >> 7;                     // M tiles (1 or 2)
    const int npad = (l + 15) & ~15;                   // N of the MMA: 16 .. 128
    const int nch = (n + kKc - 1) / kKc;
    const uint32_t idesc = tc::idesc_tf32(128, npad);
    // probe accumulators: rows tid and tid + 128
    float pr[2][kProbeCols];
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int j = 0; j < kProbeCols; ++j) pr[h][j] = 0.f;
    bool ok = true;
    for (int c = 0; c < nch; ++c) {
        const int s = c % kStages;
        unsigned char* stA = sm + s * kStage;
        unsigned char* stB = stA + kStageA;
        const int k0 = c * kKc;
        if (c >= kStages) {  // the MMAs of chunk c - 2 read this stage
            if (ok) ok = tc::mbar_wait(&bars[s], (phase >> s) & 1u);
            phase ^= 1u << s;
        }
        // A chunk: rows 0 .. 128 mt - 1, K = k0 .. k0 + 31; thread row = lane + 32 w', 4-column
        // group g; the warp's 32 loads of one column are consecutive rows (coalesced)
        for (int u = tid; u < mt * 128 * (kKc / 4); u += 128) {
            const int g = u / (mt * 128), row = u - g * (mt * 128);
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (row < m) {
                const int k = k0 + 4 * g;
                const float* src = a + (size_t)k * lda + row;
                if (k + 0 < n) v.x = src[0];
                if (k + 1 < n) v.y = src[(size_t)lda];
                if (k + 2 < n) v.z = src[2 * (size_t)lda];
                if (k + 3 < n) v.w = src[3 * (size_t)lda];
            }
            const int t = row >> 7, r = row & 127;
            *reinterpret_cast<float4*>(stA + t * kATile + tc::kmajor_offset(r, 4 * g, kLbo, kSbo)) = v;
        }
        // Omega chunk: row c' of B = column c' of Omega, K = k0 .. k0 + 31, from Philox (counter
        // (k / 4, c', b, 0): the four K values of one call are one 16-byte unit of the layout)
        for (int u = tid; u < npad * (kKc / 4); u += 128) {
            const int g = u / npad, col = u - g * npad;
            const int k = k0 + 4 * g;
            float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
            if (col < l && k < n) {
                z = gauss4(seed, (uint32_t)b, 0u, (uint32_t)(k >> 2), (uint32_t)col);
                if (k + 1 >= n) z.y = 0.f;
                if (k + 2 >= n) z.z = 0.f;
                if (k + 3 >= n) z.w = 0.f;
            }
            *reinterpret_cast<float4*>(stB + tc::kmajor_offset(col, 4 * g, kLbo, kSbo)) = z;
        }
        // probe rows of this chunk (stream 1), FP32
        for (int u = tid; u < (kKc / 4) * kProbeCols; u += 128) {
            const int g = u / kProbeCols, j = u - g * kProbeCols;
            const int k = k0 + 4 * g;
            float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
            if (k < n) z = gauss4(seed, (uint32_t)b, 1u, (uint32_t)(k >> 2), (uint32_t)j);
            wsm[4 * g + 0][j] = k + 0 < n ? z.x : 0.f;
            wsm[4 * g + 1][j] = k + 1 < n ? z.y : 0.f;
            wsm[4 * g + 2][j] = k + 2 < n ? z.z : 0.f;
            wsm[4 * g + 3][j] = k + 3 < n ? z.w : 0.f;
        }
        tc::fence_smem_to_async();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            const uint32_t bA = tc::smem_u32(stA), bB = tc::smem_u32(stB);
            for (int t = 0; t < mt; ++t) {
#pragma unroll
                for (int kk = 0; kk < kKc / 8; ++kk) {
                    const uint64_t da = tc::desc_kmajor(bA + t * kATile + kk * 2 * kLbo, kLbo, kSbo);
                    const uint64_t db = tc::desc_kmajor(bB + kk * 2 * kLbo, kLbo, kSbo);
                    tc::mma_tf32(tmem + (uint32_t)(t * 128), da, db, idesc, (c > 0 || kk > 0) ? 1u : 0u);
                }
            }
            tc::mma_commit(&bars[s]);
        }
        used |= 1u << s;
        // probes from the staged chunk (the tensor core only reads it)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int row = tid + 128 * h;
            if (row < mt * 128) {
                const int t = row >> 7, r = row & 127;
#pragma unroll
                for (int g = 0; g < kKc / 4; ++g) {
                    const float4 x = *reinterpret_cast<const float4*>(stA + t * kATile +
                                                                      tc::kmajor_offset(r, 4 * g, kLbo, kSbo));
#pragma unroll
                    for (int j = 0; j < kProbeCols; ++j) {
                        float acc = pr[h][j];
                        acc = fmaf(x.x, wsm[4 * g + 0][j], acc);
                        acc = fmaf(x.y, wsm[4 * g + 1][j], acc);
                        acc = fmaf(x.z, wsm[4 * g + 2][j], acc);
                        acc = fmaf(x.w, wsm[4 * g + 3][j], acc);
                        pr[h][j] = acc;
                    }
                }
            }
        }
        __syncthreads();  // wsm is rewritten by the next chunk
    }
    // drain: the last (up to two) chunks' commits
    for (int c = nch > kStages ? nch - kStages : 0; c < nch; ++c) {
        const int s = c % kStages;
        if (ok) ok = tc::mbar_wait(&bars[s], (phase >> s) & 1u);
        phase ^= 1u << s;
    }
    tc::fence_after_sync();
    if (!ok && tid == 0) atomicAdd(timeouts, 1);
    // epilogue: warp w reads TMEM lanes 32 w .. 32 w + 31 (rows), 32 columns at a time
    float* y = Y[b];
    for (int t = 0; t < mt; ++t) {
        const int row = t * 128 + warp * 32 + lane;
        for (int c0 = 0; c0 < npad; c0 += 32) {
            float v[32];
            tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(t * 128 + c0), v);
            if (row < m) {
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (c0 + j < l) y[(size_t)(c0 + j) * m + row] = v[j];
            }
        }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int row = tid + 128 * h;
        if (row < m) {
#pragma unroll
            for (int j = 0; j < kProbeCols; ++j) y[(size_t)(l + j) * m + row] = pr[h][j];
        }
    }
    tc::fence_before_sync();
}

__global__ void __launch_bounds__(128) rs_sample_tc_kernel(ItemList wl, float* const* A, const int* LDA, float* const* Y,
                                                           const int* M, const int* N, const int* L,
                                                           unsigned long long seed, int* timeouts)
{
    extern __shared__ __align__(16) unsigned char raw[];
    __shared__ uint64_t bars[kStages];
    __shared__ uint32_t tmem_slot;
    __shared__ float wsm[kKc][kProbeCols];
    __shared__ int s_skip;
    unsigned char* sm = align1k(raw);
    if (threadIdx.x < 32) {
        tc::tmem_alloc(&tmem_slot, kTmemCols);
        tc::tmem_relinquish();
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) tc::mbar_init(&bars[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    uint32_t phase = 0, used = 0;
    for (int b = list_item(wl); b >= 0; b = list_item(wl)) {
        // after any wait of the call gave up, the remaining blocks are skipped (results invalid);
        // thread 0 decides for the whole CTA (list_item's barrier orders the next write of s_skip)
        if (threadIdx.x == 0) s_skip = *reinterpret_cast<volatile int*>(timeouts);
        __syncthreads();
        if (s_skip == 0) sample_item(b, A, LDA, Y, M, N, L, seed, sm, tmem, bars, phase, used, wsm, timeouts);
    }
    // a CTA whose wait gave up may still have MMAs in flight: wait (bounded) for the last commit of
    // every stage it used before the tensor memory is released
    __syncthreads();
    if (threadIdx.x == 0) s_skip = *reinterpret_cast<volatile int*>(timeouts);
    __syncthreads();
    if (s_skip != 0) {
        for (int s = 0; s < kStages; ++s)
            if ((used >> s) & 1u) tc::mbar_wait(&bars[s], ((phase >> s) & 1u) ^ 1u);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (threadIdx.x < 32) tc::tmem_dealloc(tmem, kTmemCols);
}

}  // namespace

int launch_rs_sample_tc(int batch, ItemList wl, float* const* A, const int* LDA, float* const* Y, const int* M,
                        const int* N, const int* L, unsigned long long seed, int* timeouts, cudaStream_t st)
{
    if (cudaFuncSetAttribute(rs_sample_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem) !=
        cudaSuccess)
        return BSVD_ERR_CUDA;
    if (wl.idx == nullptr) return BSVD_ERR_UNSUPPORTED;  // always driven by the sampling list
    if (cudaMemsetAsync(wl.claim, 0, sizeof(unsigned long long), st) != cudaSuccess) return BSVD_ERR_CUDA;
    // two CTAs per SM: 2 x 256 TMEM columns and 2 x 97 KB of shared memory; the occupancy query
    // reports one for a kernel that allocates tensor memory, so the grid is set from these limits
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = batch < 2 * sms ? (batch > 0 ? batch : 1) : 2 * sms;
    rs_sample_tc_kernel<<<grid, 128, kSmem, st>>>(wl, A, LDA, Y, M, N, L, seed, timeouts);
    return cudaGetLastError() == cudaSuccess ? BSVD_SUCCESS : BSVD_ERR_CUDA;
}

}  // namespace bsvd
