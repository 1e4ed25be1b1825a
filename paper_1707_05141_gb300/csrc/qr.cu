// qr.cu -- batched Householder QR (Algorithm 1, Section 2.1; batched kernel of Section 3.1).
//
// One CTA per matrix.  The m x n matrix is staged once in shared memory with coalesced column
// loads and factored there: for each column a single warp forms the reflector (norm by a warp
// shuffle reduction, as in Section 3.1), then all warps apply it to the trailing columns, one
// warp per column: the transpose-matrix-vector product M^T v is a warp reduction per column
// followed by the rank-1 update.  R is written straight from shared memory; Q is formed in the
// same buffer by backward accumulation of the reflectors (Q = H_0 H_1 ... H_{n-1} [I; 0]), each
// reflector consumed in place as its column of Q is produced, so shared memory holds one m x n
// matrix plus n diagonal entries.  Nothing goes to global memory but the outputs.
#include <cuda_runtime.h>

#include "common.cuh"
#include "house.cuh"
#include "launch.cuh"

namespace bsvd {

// QROWS: rows per lane of the register-resident Q formation (m <= 32 QROWS; taller matrices
// accumulate Q backwards in shared memory)
template <typename T, int QROWS>
__global__ void qr_kernel(int batch, int max_m, int max_n, T* const* A, const int* M, const int* N,
                          const int* LDA, T* const* Q, const int* LDQ, T* const* R, const int* LDR,
                          int* info, ItemList wl, int r_trans, const int* a_trans)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* S = reinterpret_cast<T*>(smem_raw);
    const int ld = max_m | 1;  // odd: the transposed load's stores spread over the banks
    T* diag = S + (size_t)ld * max_n;

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int nwarps = blockDim.x >> 5;

    for (int b = item_first(wl, batch); b >= 0; b = item_next(wl, batch, b)) {
        const int m = M[b], n = N[b], lda = LDA[b];
        const bool at = a_trans && a_trans[b];  // factor A^T: the stored matrix is n x m, ld lda
        const int ldq = Q ? LDQ[b] : m, ldr = R ? LDR[b] : n;
        const bool bad = m < 0 || n < 0 || m < n || m > max_m || n > max_n || lda < ((at ? n : m) > 1 ? (at ? n : m) : 1) ||
                         (Q && ldq < (m > 1 ? m : 1)) || (R && ldr < (n > 1 ? n : 1));
        if (bad) {
            if (tid == 0) info[b] = BSVD_INFO_BAD_SHAPE;
            continue;
        }
        if (tid == 0) info[b] = 0;
        if (n == 0) continue;
        const T* a = A[b];
        int nonfinite = 0;  // a NaN or an infinity in A (the factorisation would take a NaN norm for 0)
        if (!at) {
            for (int j = warp; j < n; j += nwarps)
                for (int i = lane; i < m; i += 32) {
                    const T x = a[(size_t)j * lda + i];
                    nonfinite |= !isfinite(x);
                    S[j * ld + i] = x;
                }
        } else {
            // S(i, j) = A(j, i): row i of S is column i of the stored matrix (coalesced reads)
            for (int i = warp; i < m; i += nwarps)
                for (int j = lane; j < n; j += 32) {
                    const T x = a[(size_t)i * lda + j];
                    nonfinite |= !isfinite(x);
                    S[j * ld + i] = x;
                }
        }
        if (__syncthreads_or(nonfinite) && tid == 0) info[b] = BSVD_INFO_NONFINITE;

        // ---- factorisation: v_i = house(R(i:m, i)); R = (I - 2 v v^T) R ----
        house_factor_smem(S, ld, diag, m, n);

        // ---- R: strict upper part from S, diagonal from diag, zeros below ----
        if (R) {
            T* r_out = R[b];
            for (int j = warp; j < n; j += nwarps)
                for (int i = lane; i < n; i += 32)
                    r_out[r_trans ? (size_t)i * ldr + j : (size_t)j * ldr + i] =
                        i < j ? S[j * ld + i] : (i == j ? diag[j] : T(0));
        }
        __syncthreads();

        // ---- Q = H_0 ... H_{n-1} [I; 0] ----
        if (Q && m <= 32 * QROWS) {
            // column j of Q is H_0 H_1 ... H_j e_j (H_i e_j = e_j for i > j): every column on its own,
            // one warp per column, in registers (rows lane + 32 t), with no barrier
            T* q_out = Q[b];
            for (int j = warp; j < n; j += nwarps) {
                T q[QROWS];
#pragma unroll
                for (int t = 0; t < QROWS; ++t) q[t] = (lane + 32 * t == j) ? T(1) : T(0);
                for (int i = j; i >= 0; --i) {
                    const T* v = S + (size_t)i * ld;
                    T w = T(0);
#pragma unroll
                    for (int t = 0; t < QROWS; ++t) {
                        const int r = lane + 32 * t;
                        if (r >= i && r < m) w = fma(v[r], q[t], w);
                    }
                    w = T(2) * warp_sum(w);
#pragma unroll
                    for (int t = 0; t < QROWS; ++t) {
                        const int r = lane + 32 * t;
                        if (r >= i && r < m) q[t] = fma(-w, v[r], q[t]);
                    }
                }
#pragma unroll
                for (int t = 0; t < QROWS; ++t) {
                    const int r = lane + 32 * t;
                    if (r < m) q_out[(size_t)j * ldq + r] = q[t];
                }
            }
        } else if (Q) {
            // taller matrices: backward accumulation in place
            for (int i = n - 1; i >= 0; --i) {
                const T* col = S + i * ld;
                for (int j = i + 1 + warp; j < n; j += nwarps) {
                    T* cj = S + j * ld;
                    T w = T(0);
                    for (int r = i + lane; r < m; r += 32) w += col[r] * cj[r];
                    w = T(2) * warp_sum(w);
                    for (int r = i + lane; r < m; r += 32) cj[r] -= w * col[r];
                }
                const T v0 = col[i];
                __syncthreads();
                // column i of Q: H_i e_i = e_i - 2 v0 v on rows >= i, zero above
                for (int r = tid; r < m; r += blockDim.x) {
                    const T vr = S[i * ld + r];
                    S[i * ld + r] = r < i ? T(0) : ((r == i ? T(1) : T(0)) - T(2) * v0 * vr);
                }
                __syncthreads();
            }
            T* q_out = Q[b];
            for (int j = warp; j < n; j += nwarps)
                for (int i = lane; i < m; i += 32) q_out[(size_t)j * ldq + i] = S[j * ld + i];
        }
        __syncthreads();
    }
}

template <typename T>
int launch_qr(int batch, int max_m, int max_n, void* const* A, const int* M, const int* N, const int* LDA,
              void* const* Q, const int* LDQ, void* const* R, const int* LDR, int* info, cudaStream_t st,
              ItemList wl, bool r_transposed, const int* a_trans)
{
    const size_t smem = ((size_t)(max_m | 1) * max_n + max_n) * sizeof(T);
    const int threads = max_n <= 32 ? 128 : 256;
    // rows per lane of the register Q formation from the batch's row bound
    auto kern = max_m <= 32 ? qr_kernel<T, 1> : (max_m <= 64 ? qr_kernel<T, 2> : (max_m <= 128 ? qr_kernel<T, 4>
                                                                                             : qr_kernel<T, 8>));
    if (smem > 48 * 1024) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return BSVD_ERR_CUDA;
    }
    const int grid = item_grid(kern, threads, smem, wl, batch, st);
    if (grid == 0) return BSVD_ERR_CUDA;
    kern<<<grid, threads, smem, st>>>(batch, max_m, max_n, (T* const*)A, M, N, LDA, (T* const*)Q, LDQ, (T* const*)R,
                                      LDR, info, wl, r_transposed ? 1 : 0, a_trans);
    return cudaGetLastError() == cudaSuccess ? BSVD_SUCCESS : BSVD_ERR_CUDA;
}

template int launch_qr<float>(int, int, int, void* const*, const int*, const int*, const int*, void* const*,
                              const int*, void* const*, const int*, int*, cudaStream_t, ItemList, bool, const int*);
template int launch_qr<double>(int, int, int, void* const*, const int*, const int*, const int*, void* const*,
                               const int*, void* const*, const int*, int*, cudaStream_t, ItemList, bool, const int*);

}  // namespace bsvd
