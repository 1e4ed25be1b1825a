// jacobi_smem.cu -- one-sided Jacobi SVD with the matrix resident in shared memory
// (Algorithm 2, Section 2.2; shared-memory kernel of Section 5).
//
// One CTA per matrix.  The working matrix W (m x n, or A^T when m < n) and the accumulated
// rotations V live in shared memory for the whole factorisation, so global memory is touched
// once to load A and once to store U, S, V.  Each round-robin step (Section 5) processes
// n/2 disjoint column pairs in parallel; a pair is owned by a group of G consecutive lanes, each
// holding up to MAXR rows of both columns in registers (several rows per thread with a serial
// partial sum, then a shuffle reduction inside the group -- Section 5's advice to put as few
// threads as possible on a pair).  The three Gram entries, the rotation test and (c, s) are
// computed redundantly by the G lanes, the columns are rotated in registers and written back.
// A CTA-wide count of rotations per sweep decides convergence.  Finally sigma_j = ||w_j||,
// U = W / sigma, and a rank computed per column scatters S, U, V in descending order.
#include <cuda_runtime.h>

#include "common.cuh"
#include "launch.cuh"

namespace bsvd {

template <typename T, typename P, int G, int MAXR>
__global__ void __launch_bounds__(80 * G > 1024 ? 1024 : 80 * G) jacobi_smem_kernel(int batch, int max_mm, int max_np, T* const* A, const int* M, const int* N,
                                   const int* LDA, T* const* Sout, T* const* U, const int* LDU, T* const* V,
                                   const int* LDV, double tol_in, int max_sweeps, int* info, long long* rot_out,
                                   ItemList wl)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ldw = max_mm | 1;  // odd leading dimensions spread columns over the banks
    const int ldv = max_np | 1;
    T* W = reinterpret_cast<T*>(smem_raw);
    T* Vs = W + (size_t)ldw * max_np;
    T* sig = Vs + (size_t)ldv * max_np;
    int* rank = reinterpret_cast<int*>(sig + max_np);

    const int tid = threadIdx.x;
    const int slot = tid / G;        // pair slot
    const int gl = tid % G;          // lane inside the pair group
    const int nthreads = blockDim.x;

    for (int b = item_first(wl, batch); b >= 0; b = item_next(wl, batch, b)) {
        const int m = M[b], n = N[b], lda = LDA[b];
        const bool tr = m < n;
        const int mm = tr ? n : m;   // working rows
        const int nn = tr ? m : n;   // working columns (k)
        const int np = nn + (nn & 1);
        const bool wantU = U != nullptr, wantV = V != nullptr;
        const int ldu = wantU ? LDU[b] : 1, ldvo = wantV ? LDV[b] : 1;
        const bool bad = m < 0 || n < 0 || mm > max_mm || np > max_np || lda < (m > 1 ? m : 1) ||
                         (wantU && ldu < (m > 1 ? m : 1)) || (wantV && ldvo < (n > 1 ? n : 1)) ||
                         (mm + G - 1) / G > MAXR;
        if (bad) {
            if (tid == 0) info[b] = BSVD_INFO_BAD_SHAPE;
            continue;
        }
        if (nn == 0) {
            if (tid == 0) {
                info[b] = 0;
                if (rot_out) rot_out[b] = 0;
            }
            continue;
        }
        // the V factor of the working matrix is the output U when transposed
        const bool accV = tr ? wantU : wantV;

        // ---- load W (coalesced along columns of A), zero the padding column, V = I ----
        const T* a = A[b];
        // kRun loads per thread in flight before their stores (a shared store between two global
        // loads would make each load wait for the previous one's data)
        constexpr int kRun = 8;
        const int tot = mm * nn;
        for (int e0 = 0; e0 < tot; e0 += kRun * nthreads) {
            T x[kRun];
#pragma unroll
            for (int u = 0; u < kRun; ++u) {
                const int e = e0 + tid + u * nthreads;
                x[u] = T(0);
                if (e < tot) {
                    if (!tr) {
                        const int j = e / mm, i = e - j * mm;
                        x[u] = a[(size_t)j * lda + i];
                    } else {   // W(i, j) = A(j, i): read A by columns
                        const int i = e / nn, j = e - i * nn;
                        x[u] = a[(size_t)i * lda + j];
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < kRun; ++u) {
                const int e = e0 + tid + u * nthreads;
                if (e < tot) {
                    if (!tr) {
                        const int j = e / mm, i = e - j * mm;
                        W[j * ldw + i] = x[u];
                    } else {
                        const int i = e / nn, j = e - i * nn;
                        W[j * ldw + i] = x[u];
                    }
                }
            }
        }
        if (np != nn)
            for (int i = tid; i < mm; i += nthreads) W[nn * ldw + i] = T(0);
        if (accV)
            for (int e = tid; e < np * np; e += nthreads) {
                const int j = e / np, i = e - j * np;
                Vs[j * ldv + i] = i == j ? T(1) : T(0);
            }
        __syncthreads();

        const P tol = tol_in > 0.0 ? P(tol_in) : P(dsqrt(double(mm)) * Unit<T>::value);
        const int sweeps_cap = max_sweeps > 0 ? max_sweeps : 30;
        const int rpl = (mm + G - 1) / G;  // rows per lane
        int sweep = 0;
        bool converged = false;
        long long total_rot = 0;

        while (sweep < sweeps_cap) {
            int rot_sweep = 0;
            for (int step = 0; step < np - 1; ++step) {
                // every lane runs the reduction (idle slots with zeros) so that the group
                // shuffles always see full warps
                const bool active = slot < np / 2;
                int p = 0, q = 0;
                if (active) round_robin_pair(np, step, slot, p, q);
                T x[MAXR], y[MAXR];
                P al = P(0), be = P(0), ga = P(0);
#pragma unroll
                for (int k = 0; k < MAXR; ++k) {
                    const int r = gl + k * G;
                    x[k] = T(0);
                    y[k] = T(0);
                    if (active && k < rpl && r < mm) {
                        x[k] = W[p * ldw + r];
                        y[k] = W[q * ldw + r];
                        al += P(x[k]) * P(x[k]);
                        be += P(y[k]) * P(y[k]);
                        ga += P(x[k]) * P(y[k]);
                    }
                }
                al = group_sum<G>(al);
                be = group_sum<G>(be);
                ga = group_sum<G>(ga);
                P c, s;
                const bool rotated = active && q < nn && jacobi_rotation<P>(al, be, ga, tol, c, s);
                if (rotated) {
                    const T ct = T(c), st = T(s);
#pragma unroll
                    for (int k = 0; k < MAXR; ++k) {
                        const int r = gl + k * G;
                        if (k < rpl && r < mm) {
                            W[p * ldw + r] = ct * x[k] - st * y[k];
                            W[q * ldw + r] = st * x[k] + ct * y[k];
                        }
                    }
                    if (accV) {
                        for (int r = gl; r < nn; r += G) {
                            const T vx = Vs[p * ldv + r], vy = Vs[q * ldv + r];
                            Vs[p * ldv + r] = ct * vx - st * vy;
                            Vs[q * ldv + r] = st * vx + ct * vy;
                        }
                    }
                }
                rot_sweep += __syncthreads_count(rotated && gl == 0);
            }
            ++sweep;
            total_rot += rot_sweep;
            if (rot_sweep == 0) {
                converged = true;
                break;
            }
        }

        // ---- sigma_j = ||w_j|| ----
        for (int j0 = 0; j0 < nn; j0 += nthreads / G) {  // uniform trip count for the shuffles
            const int j = j0 + slot;
            P ss = P(0);
            if (j < nn)
                for (int r = gl; r < mm; r += G) ss += P(W[j * ldw + r]) * P(W[j * ldw + r]);
            ss = group_sum<G>(ss);
            if (gl == 0 && j < nn) sig[j] = T(dsqrt(ss));
        }
        __syncthreads();
        // ---- descending rank, ties in column order ----
        for (int j = tid; j < nn; j += nthreads) {
            const T sj = sig[j];
            int r = 0;
            for (int i = 0; i < nn; ++i) {
                const T si = sig[i];
                r += (si > sj) || (si == sj && i < j);
            }
            rank[j] = r;
        }
        __syncthreads();

        // ---- outputs: S; left vectors W/sigma; right vectors V (swapped when transposed) ----
        T* s_out = Sout[b];
        for (int j = tid; j < nn; j += nthreads) s_out[rank[j]] = sig[j];
        T* uw = tr ? (wantV ? V[b] : nullptr) : (wantU ? U[b] : nullptr);  // receives W / sigma
        const int lduw = tr ? ldvo : ldu;
        T* vw = tr ? (wantU ? U[b] : nullptr) : (wantV ? V[b] : nullptr);  // receives Vs
        const int ldvw = tr ? ldu : ldvo;
        if (uw) {
            for (int e = tid; e < mm * nn; e += nthreads) {
                const int j = e / mm, i = e - j * mm;
                const T sj = sig[j];
                uw[(size_t)rank[j] * lduw + i] = sj > T(0) ? W[j * ldw + i] / sj : T(0);
            }
        }
        if (vw) {
            for (int e = tid; e < nn * nn; e += nthreads) {
                const int j = e / nn, i = e - j * nn;
                vw[(size_t)rank[j] * ldvw + i] = Vs[j * ldv + i];
            }
        }
        if (tid == 0) {
            bool finite = true;
            for (int i = 0; i < nn; ++i) finite = finite && isfinite(sig[i]);
            info[b] = !finite ? BSVD_INFO_NONFINITE : (converged ? sweep : BSVD_INFO_NOT_CONVERGED + sweep);
            if (rot_out) rot_out[b] = total_rot;
        }
        __syncthreads();
    }
}

// shared memory bytes for a launch with working sizes max_mm x max_np
template <typename T>
static size_t jacobi_smem_bytes(int max_mm, int max_np)
{
    return ((size_t)(max_mm | 1) * max_np + (size_t)(max_np | 1) * max_np + max_np) * sizeof(T) +
           (size_t)max_np * sizeof(int) + 16;
}

template <typename T, typename P, int G, int MAXR>
static int launch_g(int batch, int max_mm, int max_np, void* const* A, const int* M, const int* N, const int* LDA,
                    void* const* S, void* const* U, const int* LDU, void* const* V, const int* LDV, double tol,
                    int max_sweeps, int* info, long long* rot, cudaStream_t st, ItemList wl)
{
    auto kern = jacobi_smem_kernel<T, P, G, MAXR>;
    const size_t smem = jacobi_smem_bytes<T>(max_mm, max_np);
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return BSVD_ERR_CUDA;
    const int threads = (max_np / 2) * G < 32 ? 32 : (max_np / 2) * G;
    const int grid = item_grid(kern, threads, smem, wl, batch, st);
    if (grid == 0) return BSVD_ERR_CUDA;
    kern<<<grid, threads, smem, st>>>(batch, max_mm, max_np, (T* const*)A, M, N, LDA, (T* const*)S, (T* const*)U, LDU,
                                      (T* const*)V, LDV, tol, max_sweeps, info, rot, wl);
    return cudaGetLastError() == cudaSuccess ? BSVD_SUCCESS : BSVD_ERR_CUDA;
}

// Picks the lanes-per-pair G so that every lane holds at most 16 rows.
template <typename T>
int launch_jacobi_smem(int batch, int max_m, int max_n, void* const* A, const int* M, const int* N, const int* LDA,
                       void* const* S, void* const* U, const int* LDU, void* const* V, const int* LDV, double tol,
                       int max_sweeps, int* info, long long* rot, cudaStream_t st, ItemList wl, bool p64)
{
    if (sizeof(T) == 4) {  // FP32 up to 128 x 128: the columns in registers (jacobi_rx.cu)
        const int rc = launch_jacobi_rx(batch, max_m, max_n, A, M, N, LDA, S, U, LDU, V, LDV, tol, max_sweeps, info,
                                        rot, st, wl, p64);
        if (rc != BSVD_ERR_UNSUPPORTED) return rc;
    }
    const int max_mm = max_m > max_n ? max_m : max_n;
    const int max_nn = max_m > max_n ? max_n : max_m;
    const int max_np = (max_nn + 1) & ~1;
    const int maxk_lim = sizeof(T) == 4 ? 160 : 64;  // and the matrix and V must fit in shared memory
    if (max_mm > 256 || max_nn > maxk_lim) return BSVD_ERR_UNSUPPORTED;
    if (max_np == 0) return launch_g<T, T, 1, 16>(batch, max_mm, 2, A, M, N, LDA, S, U, LDU, V, LDV, tol, max_sweeps,
                                                 info, rot, st, wl);
    if (jacobi_smem_bytes<T>(max_mm, max_np) > 220 * 1024) return BSVD_ERR_UNSUPPORTED;
    int g = 1;
    while (g * 16 < max_mm) g *= 2;
    if ((max_np / 2) * g > 1024) {
        // more than 1024 threads at 16 rows per lane: 8 lanes per pair with up to 24 rows each
        if (max_mm > 8 * 24 || (max_np / 2) * 8 > 1024) return BSVD_ERR_UNSUPPORTED;
        return p64 && sizeof(T) == 4
                   ? launch_g<T, double, 8, 24>(batch, max_mm, max_np, A, M, N, LDA, S, U, LDU, V, LDV, tol,
                                                max_sweeps, info, rot, st, wl)
                   : launch_g<T, T, 8, 24>(batch, max_mm, max_np, A, M, N, LDA, S, U, LDU, V, LDV, tol, max_sweeps,
                                           info, rot, st, wl);
    }
#define BSVD_LAUNCH_G(GG)                                                                                          \
    return p64 && sizeof(T) == 4                                                                                   \
               ? launch_g<T, double, GG, 16>(batch, max_mm, max_np, A, M, N, LDA, S, U, LDU, V, LDV, tol, max_sweeps, \
                                             info, rot, st, wl)                                                   \
               : launch_g<T, T, GG, 16>(batch, max_mm, max_np, A, M, N, LDA, S, U, LDU, V, LDV, tol, max_sweeps, info,  \
                                        rot, st, wl)
    switch (g) {
        case 1: BSVD_LAUNCH_G(1);
        case 2: BSVD_LAUNCH_G(2);
        case 4: BSVD_LAUNCH_G(4);
        case 8: BSVD_LAUNCH_G(8);
        default: BSVD_LAUNCH_G(16);
    }
#undef BSVD_LAUNCH_G
}

template int launch_jacobi_smem<float>(int, int, int, void* const*, const int*, const int*, const int*, void* const*,
                                       void* const*, const int*, void* const*, const int*, double, int, int*,
                                       long long*, cudaStream_t, ItemList, bool);
template int launch_jacobi_smem<double>(int, int, int, void* const*, const int*, const int*, const int*,
                                        void* const*, void* const*, const int*, void* const*, const int*, double, int,
                                        int*, long long*, cudaStream_t, ItemList, bool);

}  // namespace bsvd
