// jacobi_rx.cu -- one-sided Jacobi SVD of FP32 matrices up to 128 x 128 with the columns resident
// in registers and the pair exchange through shared memory (Algorithm 2, Section 2.2; the
// shared-memory kernel of Section 5, re-arranged for sm_103a).
//
// The shared tier (jacobi_smem.cu) keeps W and V in shared memory and streams both columns of every
// pair through registers at every step: eight shared-memory accesses per row of a pair, which bound
// it by shared-memory bandwidth.  Here each pair slot's G lanes keep their rows of the slot's two W
// columns and two V columns in registers for the whole factorisation.  The pair ordering is the
// odd-even transposition with exchange of the register tier (2 NS positions, every processed pair
// swaps positions, 2 NS steps per sweep), so between steps exactly one column per slot moves to the
// neighbouring slot: it is written to a double-buffered exchange area in shared memory and read back
// by the neighbour after the step's one barrier.  A row of a pair then costs one shared store and one
// shared load for W and the same for V, half the traffic of the shared tier, and the rotation's
// arithmetic runs on registers.
//
// Layout: slot s (0 <= s < NS = np / 2) has lanes s G .. s G + G - 1; lane g holds rows g + G k of
// its columns (k < RW for W, k < RV for V).  Even steps pair positions (2s, 2s + 1), odd steps
// (2s + 1, 2s + 2); on odd steps the wrap slot NS - 1, holding positions 2 NS - 1 and 0, idles.
#include <cuda_runtime.h>

#include "common.cuh"
#include "launch.cuh"

namespace bsvd {

namespace {

constexpr int kRxG = 8;  // lanes per pair slot

template <int RW>
struct RxDims {
    static constexpr int ldx = RW * kRxG + 8;  // exchange row stride: slots 8 banks apart
};

}  // namespace

// P: precision of the rotation parameters and the rotation test (T, or double for FP32 data)
template <typename T, typename P, int RW, int RV>
__global__ void __launch_bounds__(64 * kRxG, 1)
    jacobi_rx_kernel(int batch, int max_mm, int max_np, T* const* A, const int* M, const int* N, const int* LDA,
                     T* const* Sout, T* const* U, const int* LDU, T* const* V, const int* LDV, double tol_in,
                     int max_sweeps, int* info, long long* rot_out, ItemList wl)
{
    constexpr int G = kRxG;
    constexpr int LDW = RxDims<RW>::ldx;   // exchange stride, W rows
    constexpr int LDV_ = RxDims<RV>::ldx;  // exchange stride, V rows
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nslot_max = max_np / 2;
    T* xw = reinterpret_cast<T*>(smem_raw);               // [2][nslot_max][LDW]
    T* xv = xw + (size_t)2 * nslot_max * LDW;             // [2][nslot_max][LDV_]
    int* xc = reinterpret_cast<int*>(xv + (size_t)2 * nslot_max * LDV_);  // [2][nslot_max] column ids
    T* sig = reinterpret_cast<T*>(xc + 2 * nslot_max);   // [max_np] singular values by column id
    int* rank = reinterpret_cast<int*>(sig + max_np);     // [max_np]

    const int tid = threadIdx.x;
    const int s = tid / G;  // slot
    const int g = tid % G;  // lane in the slot

    for (int b = item_first(wl, batch); b >= 0; b = item_next(wl, batch, b)) {
        const int m = M[b], n = N[b], lda = LDA[b];
        const bool tr = m < n;
        const int mm = tr ? n : m;  // working rows
        const int nn = tr ? m : n;  // working columns
        const int np = nn + (nn & 1);
        const int ns = np / 2;      // slots of this matrix
        const bool wantU = U != nullptr, wantV = V != nullptr;
        const int ldu = wantU ? LDU[b] : 1, ldvo = wantV ? LDV[b] : 1;
        const bool bad = m < 0 || n < 0 || mm > max_mm || np > max_np || mm > RW * G || np > RV * G ||
                         lda < (m > 1 ? m : 1) || (wantU && ldu < (m > 1 ? m : 1)) ||
                         (wantV && ldvo < (n > 1 ? n : 1));
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
        const bool accV = tr ? wantU : wantV;
        const bool live = s < ns;

        // ---- W (A, or A^T) and V = I into registers; the padding column is zero ----
        T wl_[RW], wr_[RW], vl_[RV], vr_[RV];
        int colL = 2 * s, colR = 2 * s + 1;
        const T* a = A[b];
#pragma unroll
        for (int k = 0; k < RW; ++k) {
            const int r = g + G * k;
            T x = T(0), y = T(0);
            if (live && r < mm) {
                if (!tr) {
                    if (colL < nn) x = a[(size_t)colL * lda + r];
                    if (colR < nn) y = a[(size_t)colR * lda + r];
                } else {
                    if (colL < nn) x = a[(size_t)r * lda + colL];
                    if (colR < nn) y = a[(size_t)r * lda + colR];
                }
            }
            wl_[k] = x;
            wr_[k] = y;
        }
#pragma unroll
        for (int k = 0; k < RV; ++k) {
            const int r = g + G * k;
            vl_[k] = (r == colL) ? T(1) : T(0);
            vr_[k] = (r == colR) ? T(1) : T(0);
        }

        const P tol = tol_in > 0.0 ? P(tol_in) : P(dsqrt(double(mm)) * Unit<T>::value);
        const int sweeps_cap = max_sweeps > 0 ? max_sweeps : 30;
        int sweep = 0;
        bool converged = false;
        long long total_rot = 0;
        int par = 0;  // exchange buffer of this step

        while (sweep < sweeps_cap) {
            int rot_sweep = 0;
            for (int st = 0; st < 2 * ns; ++st) {
                const bool odd = st & 1;
                const bool wrap = s == ns - 1;
                // Gram entries of the slot's pair over this lane's rows, then over the slot's lanes
                T al = T(0), be = T(0), ga = T(0);
#pragma unroll
                for (int k = 0; k < RW; ++k) {
                    al = fma(wl_[k], wl_[k], al);
                    be = fma(wr_[k], wr_[k], be);
                    ga = fma(wl_[k], wr_[k], ga);
                }
                al = group_sum<G>(al);
                be = group_sum<G>(be);
                ga = group_sum<G>(ga);
                P c, sn;
                const bool rotated = live && !(odd && wrap) && jacobi_rotation<P>(P(al), P(be), P(ga), tol, c, sn);
                if (rotated) {
                    const T ct = T(c), st_ = T(sn);
#pragma unroll
                    for (int k = 0; k < RW; ++k) {
                        const T x = wl_[k], y = wr_[k];
                        wl_[k] = ct * x - st_ * y;
                        wr_[k] = st_ * x + ct * y;
                    }
                    if (accV) {
#pragma unroll
                        for (int k = 0; k < RV; ++k) {
                            const T x = vl_[k], y = vr_[k];
                            vl_[k] = ct * x - st_ * y;
                            vr_[k] = st_ * x + ct * y;
                        }
                    }
                }
                // exchange, first half: the column that leaves the slot goes to the exchange area
                T* ow = xw + ((size_t)par * nslot_max + s) * LDW;
                T* ov = xv + ((size_t)par * nslot_max + s) * LDV_;
                if (live) {
                    // even -> odd: the right column moves one slot down; odd -> even: the left column
                    // moves one slot up, except the wrap slot's right column (it did not rotate)
                    const bool send_right = !odd || wrap;
                    if (send_right) {
#pragma unroll
                        for (int k = 0; k < RW; ++k) ow[g + G * k] = wr_[k];
                        if (accV) {
#pragma unroll
                            for (int k = 0; k < RV; ++k) ov[g + G * k] = vr_[k];
                        }
                        if (g == 0) xc[par * nslot_max + s] = colR;
                    } else {
#pragma unroll
                        for (int k = 0; k < RW; ++k) ow[g + G * k] = wl_[k];
                        if (accV) {
#pragma unroll
                            for (int k = 0; k < RV; ++k) ov[g + G * k] = vl_[k];
                        }
                        if (g == 0) xc[par * nslot_max + s] = colL;
                    }
                }
                rot_sweep += __syncthreads_count(rotated && g == 0);
                // second half: the neighbour's column comes in
                if (live) {
                    if (!odd) {
                        const int src = s + 1 == ns ? 0 : s + 1;
                        const T* iw = xw + ((size_t)par * nslot_max + src) * LDW;
                        const T* iv = xv + ((size_t)par * nslot_max + src) * LDV_;
#pragma unroll
                        for (int k = 0; k < RW; ++k) wr_[k] = iw[g + G * k];
                        if (accV) {
#pragma unroll
                            for (int k = 0; k < RV; ++k) vr_[k] = iv[g + G * k];
                        }
                        colR = xc[par * nslot_max + src];
                    } else {
                        const int src = s == 0 ? ns - 1 : s - 1;
                        const T* iw = xw + ((size_t)par * nslot_max + src) * LDW;
                        const T* iv = xv + ((size_t)par * nslot_max + src) * LDV_;
                        if (wrap) {  // the wrap slot keeps its left column as the right one
#pragma unroll
                            for (int k = 0; k < RW; ++k) wr_[k] = wl_[k];
                            if (accV) {
#pragma unroll
                                for (int k = 0; k < RV; ++k) vr_[k] = vl_[k];
                            }
                            colR = colL;
                        }
#pragma unroll
                        for (int k = 0; k < RW; ++k) wl_[k] = iw[g + G * k];
                        if (accV) {
#pragma unroll
                            for (int k = 0; k < RV; ++k) vl_[k] = iv[g + G * k];
                        }
                        colL = xc[par * nslot_max + src];
                    }
                }
                par ^= 1;
            }
            ++sweep;
            total_rot += rot_sweep;
            if (rot_sweep == 0) {
                converged = true;
                break;
            }
        }

        // ---- sigma_j = ||w_j||, by column id ----
        {
            T sl = T(0), sr = T(0);
#pragma unroll
            for (int k = 0; k < RW; ++k) {
                sl = fma(wl_[k], wl_[k], sl);
                sr = fma(wr_[k], wr_[k], sr);
            }
            sl = group_sum<G>(sl);
            sr = group_sum<G>(sr);
            if (live && g == 0) {
                if (colL < nn) sig[colL] = dsqrt(sl);
                if (colR < nn) sig[colR] = dsqrt(sr);
            }
        }
        __syncthreads();
        // ---- descending rank, ties in column order ----
        for (int j = tid; j < nn; j += blockDim.x) {
            const T sj = sig[j];
            int r = 0;
            for (int i = 0; i < nn; ++i) {
                const T si = sig[i];
                r += (si > sj) || (si == sj && i < j);
            }
            rank[j] = r;
        }
        __syncthreads();

        // ---- outputs from the registers: S; left vectors W / sigma; right vectors V (swapped when
        // the working matrix is A^T) ----
        T* s_out = Sout[b];
        for (int j = tid; j < nn; j += blockDim.x) s_out[rank[j]] = sig[j];
        T* uw = tr ? (wantV ? V[b] : nullptr) : (wantU ? U[b] : nullptr);  // receives W / sigma
        const int lduw = tr ? ldvo : ldu;
        T* vw = tr ? (wantU ? U[b] : nullptr) : (wantV ? V[b] : nullptr);  // receives V
        const int ldvw = tr ? ldu : ldvo;
        if (live) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int col = h ? colR : colL;
                if (col >= nn) continue;
                const int rk = rank[col];
                const T sj = sig[col];
                const T inv = sj > T(0) ? T(1) / sj : T(0);
                if (uw) {
#pragma unroll
                    for (int k = 0; k < RW; ++k) {
                        const int r = g + G * k;
                        if (r < mm) uw[(size_t)rk * lduw + r] = (h ? wr_[k] : wl_[k]) * inv;
                    }
                }
                if (vw) {
#pragma unroll
                    for (int k = 0; k < RV; ++k) {
                        const int r = g + G * k;
                        if (r < nn) vw[(size_t)rk * ldvw + r] = h ? vr_[k] : vl_[k];
                    }
                }
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

// shared memory of a launch: two exchange buffers for W and V rows, column ids, sigma and ranks
template <typename T, int RW, int RV>
static size_t jacobi_rx_bytes(int max_np)
{
    const int ns = max_np / 2;
    return ((size_t)2 * ns * RxDims<RW>::ldx + (size_t)2 * ns * RxDims<RV>::ldx) * sizeof(T) +
           (size_t)2 * ns * sizeof(int) + (size_t)max_np * (sizeof(T) + sizeof(int)) + 16;
}

template <typename T, typename P, int RW, int RV>
static int launch_rx(int batch, int max_mm, int max_np, void* const* A, const int* M, const int* N, const int* LDA,
                     void* const* S, void* const* U, const int* LDU, void* const* V, const int* LDV, double tol,
                     int max_sweeps, int* info, long long* rot, cudaStream_t st, ItemList wl)
{
    auto kern = jacobi_rx_kernel<T, P, RW, RV>;
    const size_t smem = jacobi_rx_bytes<T, RW, RV>(max_np);
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return BSVD_ERR_CUDA;
    const int threads = (max_np / 2) * kRxG < 32 ? 32 : (max_np / 2) * kRxG;
    const int grid = item_grid(kern, threads, smem, wl, batch, st);
    if (grid == 0) return BSVD_ERR_CUDA;
    kern<<<grid, threads, smem, st>>>(batch, max_mm, max_np, (T* const*)A, M, N, LDA, (T* const*)S, (T* const*)U, LDU,
                                      (T* const*)V, LDV, tol, max_sweeps, info, rot, wl);
    return cudaGetLastError() == cudaSuccess ? BSVD_SUCCESS : BSVD_ERR_CUDA;
}

// FP32 matrices with max(m, n) <= 128 (16 rows of W and of V per lane; more rows would exceed the
// 128 registers a thread has at 512 threads).  Returns BSVD_ERR_UNSUPPORTED for other shapes (the
// caller then takes the shared tier).
int launch_jacobi_rx(int batch, int max_m, int max_n, void* const* A, const int* M, const int* N, const int* LDA,
                     void* const* S, void* const* U, const int* LDU, void* const* V, const int* LDV, double tol,
                     int max_sweeps, int* info, long long* rot, cudaStream_t st, ItemList wl, bool p64)
{
    const int max_mm = max_m > max_n ? max_m : max_n;
    const int max_nn = max_m > max_n ? max_n : max_m;
    const int max_np = (max_nn + 1) & ~1;
    if (max_mm > 16 * kRxG || max_np > 16 * kRxG || max_np < 2) return BSVD_ERR_UNSUPPORTED;
    return p64 ? launch_rx<float, double, 16, 16>(batch, max_mm, max_np, A, M, N, LDA, S, U, LDU, V, LDV, tol,
                                                  max_sweeps, info, rot, st, wl)
               : launch_rx<float, float, 16, 16>(batch, max_mm, max_np, A, M, N, LDA, S, U, LDU, V, LDV, tol,
                                                 max_sweeps, info, rot, st, wl);
}

}  // namespace bsvd
