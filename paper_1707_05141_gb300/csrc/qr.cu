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
        // each lane loads kLoadRun elements of a column into registers before storing any of them,
        // so that their global loads are in flight together (a store to shared memory between two
        // loads would make each load wait for the previous one's data)
        constexpr int kLoadRun = 8;
        if (!at) {
            for (int j = warp; j < n; j += nwarps)
                for (int i0 = 0; i0 < m; i0 += 32 * kLoadRun) {
                    T x[kLoadRun];
#pragma unroll
                    for (int u = 0; u < kLoadRun; ++u) {
                        const int i = i0 + lane + 32 * u;
                        x[u] = i < m ? a[(size_t)j * lda + i] : T(0);
                    }
#pragma unroll
                    for (int u = 0; u < kLoadRun; ++u) {
                        const int i = i0 + lane + 32 * u;
                        if (i < m) {
                            nonfinite |= !isfinite(x[u]);
                            S[j * ld + i] = x[u];
                        }
                    }
                }
        } else {
            // S(i, j) = A(j, i): row i of S is column i of the stored matrix (coalesced reads)
            for (int i = warp; i < m; i += nwarps)
                for (int j0 = 0; j0 < n; j0 += 32 * kLoadRun) {
                    T x[kLoadRun];
#pragma unroll
                    for (int u = 0; u < kLoadRun; ++u) {
                        const int j = j0 + lane + 32 * u;
                        x[u] = j < n ? a[(size_t)i * lda + j] : T(0);
                    }
#pragma unroll
                    for (int u = 0; u < kLoadRun; ++u) {
                        const int j = j0 + lane + 32 * u;
                        if (j < n) {
                            nonfinite |= !isfinite(x[u]);
                            S[j * ld + i] = x[u];
                        }
                    }
                }
        }
        if (__syncthreads_or(nonfinite) && tid == 0) info[b] = BSVD_INFO_NONFINITE;

        // ---- factorisation: v_i = house(R(i:m, i)); R = (I - 2 v v^T) R ----
        if (max_m <= 32 * QROWS)
            house_factor_smem_rows<T, QROWS>(S, ld, diag, m, n);
        else
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
            // in registers (rows lane + 32 t), with no barrier.  A warp carries QC columns
            // (j, j + nwarps, ...) at once: each reflector is read once for all of them, and their
            // QC shuffle reductions are independent, so their latencies overlap.
            constexpr int QC = 4;
            T* q_out = Q[b];
            for (int j0 = warp; j0 < n; j0 += nwarps * QC) {
                T q[QC][QROWS];
                int jc[QC];
#pragma unroll
                for (int c = 0; c < QC; ++c) {
                    jc[c] = j0 + c * nwarps;
#pragma unroll
                    for (int t = 0; t < QROWS; ++t) q[c][t] = (lane + 32 * t == jc[c]) ? T(1) : T(0);
                }
                int jtop = jc[0];
#pragma unroll
                for (int c = 1; c < QC; ++c)
                    if (jc[c] < n) jtop = jc[c];
                for (int i = jtop; i >= 0; --i) {
                    const T* v = S + (size_t)i * ld;
                    T vr[QROWS];
#pragma unroll
                    for (int t = 0; t < QROWS; ++t) {
                        const int r = lane + 32 * t;
                        vr[t] = (r >= i && r < m) ? v[r] : T(0);
                    }
                    T w[QC];
#pragma unroll
                    for (int c = 0; c < QC; ++c) {
                        w[c] = T(0);
#pragma unroll
                        for (int t = 0; t < QROWS; ++t) w[c] = fma(vr[t], q[c][t], w[c]);
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                        for (int c = 0; c < QC; ++c) w[c] += __shfl_xor_sync(0xffffffffu, w[c], o);
#pragma unroll
                    for (int c = 0; c < QC; ++c) {
                        // H_i leaves column j unchanged for i > j (and columns past n do not exist)
                        const T wc = (i <= jc[c] && jc[c] < n) ? T(-2) * w[c] : T(0);
#pragma unroll
                        for (int t = 0; t < QROWS; ++t) q[c][t] = fma(wc, vr[t], q[c][t]);
                    }
                }
#pragma unroll
                for (int c = 0; c < QC; ++c) {
                    if (jc[c] >= n) break;
#pragma unroll
                    for (int t = 0; t < QROWS; ++t) {
                        const int r = lane + 32 * t;
                        if (r < m) q_out[(size_t)jc[c] * ldq + r] = q[c][t];
                    }
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

// ------------------------------------------------------------------------------------------------
// Warp-per-matrix form for narrow panels (n <= 32 CPL, m <= ROWS): lane l holds columns l + 32 c
// (c < CPL) of the matrix in registers, so the product M^T v of a reflector is, for every column,
// one dot product inside its lane: no reduction across lanes and no barrier across warps.  Each
// warp owns a shared tile (column-major, ROWS x 32 CPL) that stages the coalesced loads and the
// stores of Q and keeps the reflectors: at step i the lane that owns column i writes it into tile
// column i, the warp turns it into v_i there (norm by a shuffle reduction), and every lane then
// reads v_i as a broadcast.  Q is formed in the registers by backward accumulation,
// Q = H_0 (H_1 (... H_{n-1} [I; 0])), where step i changes only the columns j >= i.
// ------------------------------------------------------------------------------------------------

// next item of this warp (first == true: its first one), or -1; every lane of the warp calls it
__device__ __forceinline__ int warp_item(const ItemList& wl, int batch, int prev, bool first)
{
    const int wpb = blockDim.x >> 5;
    if (wl.idx == nullptr) {
        const long long nb = first ? (long long)blockIdx.x * wpb + (threadIdx.x >> 5)
                                   : (long long)prev + (long long)gridDim.x * wpb;
        return nb < batch ? (int)nb : -1;
    }
    unsigned long long pos = 0;
    if ((threadIdx.x & 31) == 0) pos = atomicAdd(wl.claim, 1ull);
    pos = __shfl_sync(0xffffffffu, pos, 0);
    return pos < (unsigned long long)*wl.count ? wl.idx[pos] : -1;
}

template <typename T, int ROWS>
struct WarpQrTile {
    static constexpr int kVec = 16 / (int)sizeof(T);                  // elements per 16-byte access
    static constexpr int kLd = ROWS + (sizeof(T) == 4 ? 4 : 2);       // 16-byte chunks of 8 lanes' columns in distinct banks
};

template <typename T, int N>
__device__ __forceinline__ void ld_vec(const T* p, T (&v)[N]);
template <>
__device__ __forceinline__ void ld_vec<float, 4>(const float* p, float (&v)[4])
{
    const float4 x = *reinterpret_cast<const float4*>(p);
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
}
template <>
__device__ __forceinline__ void ld_vec<double, 2>(const double* p, double (&v)[2])
{
    const double2 x = *reinterpret_cast<const double2*>(p);
    v[0] = x.x; v[1] = x.y;
}
__device__ __forceinline__ void st_vec(float* p, float a, float b, float c, float d)
{
    *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}

// p[0:ROWS] = col (16-byte stores)
template <typename T, int ROWS>
__device__ __forceinline__ void warp_store_column(T* p, const T (&col)[ROWS])
{
#pragma unroll
    for (int q = 0; q < ROWS / WarpQrTile<T, ROWS>::kVec; ++q) {
        if constexpr (sizeof(T) == 4)
            st_vec(reinterpret_cast<float*>(p) + q * 4, col[q * 4], col[q * 4 + 1], col[q * 4 + 2], col[q * 4 + 3]);
        else
            *reinterpret_cast<double2*>(p + q * 2) = make_double2(col[q * 2], col[q * 2 + 1]);
    }
}

// col -= 2 (v . col) v for the reflector v of step i in shared memory (zero above row i).  Rows go
// in groups of 16: a group wholly above row i is skipped, and inside a group the code is straight
// (its shared loads run ahead of the FMAs).  The branch per group also bounds how far the loads
// are hoisted, and with them the registers they hold.
template <typename T, int ROWS>
__device__ __forceinline__ void warp_apply(const T* v, T (&col)[ROWS], int i)
{
    constexpr int VEC = WarpQrTile<T, ROWS>::kVec;
    constexpr int GR = 16;        // rows per group
    constexpr int G = GR / VEC;  // chunks per group
    constexpr int NACC = 8;
    T acc[NACC];
#pragma unroll
    for (int k = 0; k < NACC; ++k) acc[k] = T(0);
#pragma unroll
    for (int g = 0; g < ROWS / GR; ++g) {
        if (GR * (g + 1) <= i) continue;
#pragma unroll
        for (int q = g * G; q < (g + 1) * G; ++q) {
            T vv[VEC];
            ld_vec(v + q * VEC, vv);
#pragma unroll
            for (int e = 0; e < VEC; ++e)
                acc[(q * VEC + e) % NACC] = fma(vv[e], col[q * VEC + e], acc[(q * VEC + e) % NACC]);
        }
    }
#pragma unroll
    for (int k = NACC / 2; k > 0; k >>= 1)
#pragma unroll
        for (int t = 0; t < k; ++t) acc[t] += acc[t + k];
    const T w = T(-2) * acc[0];
#pragma unroll
    for (int g = 0; g < ROWS / GR; ++g) {
        if (GR * (g + 1) <= i) continue;
#pragma unroll
        for (int q = g * G; q < (g + 1) * G; ++q) {
            T vv[VEC];
            ld_vec(v + q * VEC, vv);
#pragma unroll
            for (int e = 0; e < VEC; ++e) col[q * VEC + e] = fma(w, vv[e], col[q * VEC + e]);
        }
    }
}

// 4- or 8-byte asynchronous copy global -> shared; src_bytes = 0 writes zero
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* dst, const T* src, bool valid)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    const int n = valid ? (int)sizeof(T) : 0;
    if constexpr (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// CTAs per SM the register allocation is capped for: the 128-row FP32 form fits three (12 warps)
// in 170 registers with a few bytes of spill outside the loops; the others keep the compiler's
// allocation
template <typename T, int ROWS, int CPL>
struct QrWarpMinBlocks {
    static constexpr int value = (sizeof(T) == 4 && ROWS == 128 && CPL == 1) ? 3 : 1;
};

template <typename T, int ROWS, int CPL>
__global__ void __launch_bounds__(128, QrWarpMinBlocks<T, ROWS, CPL>::value) qr_warp_kernel(int batch, int max_m, int max_n, T* const* A, const int* M,
                                                      const int* N, const int* LDA, T* const* Q, const int* LDQ,
                                                      T* const* R, const int* LDR, int* info, ItemList wl, int r_trans,
                                                      const int* a_trans)
{
    constexpr int NC = 32 * CPL;
    constexpr int VEC = WarpQrTile<T, ROWS>::kVec;
    constexpr int LDT = WarpQrTile<T, ROWS>::kLd;
    constexpr int NR = ROWS / 32;  // rows per lane when the warp works on one column
    static_assert(CPL == 1 || CPL == 2, "one or two columns per lane");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    T* tile = reinterpret_cast<T*>(smem_raw) + (size_t)(threadIdx.x >> 5) * LDT * NC;
    T a[CPL][ROWS];
    T rdiag[CPL];

    for (int b = warp_item(wl, batch, -1, true); b >= 0; b = warp_item(wl, batch, b, false)) {
        const int m = M[b], n = N[b], lda = LDA[b];
        const bool at = a_trans && a_trans[b];  // factor A^T: the stored matrix is n x m, ld lda
        const int ldq = Q ? LDQ[b] : m, ldr = R ? LDR[b] : n;
        const bool bad = m < 0 || n < 0 || m < n || m > max_m || n > max_n ||
                         lda < ((at ? n : m) > 1 ? (at ? n : m) : 1) || (Q && ldq < (m > 1 ? m : 1)) ||
                         (R && ldr < (n > 1 ? n : 1));
        if (bad) {
            if (lane == 0) info[b] = BSVD_INFO_BAD_SHAPE;
            continue;
        }
        if (lane == 0) info[b] = 0;
        if (n == 0) continue;
        const T* ain = A[b];
        int nonfinite = 0;
        if (!at) {
            // column j, rows lane + 32 t: coalesced asynchronous copies, all in flight at once;
            // rows >= m zero-filled
            __syncwarp();
            for (int j = 0; j < n; ++j) {
#pragma unroll
                for (int t = 0; t < NR; ++t) {
                    const int r = lane + 32 * t;
                    cp_async_elem(tile + j * LDT + r, r < m ? ain + (size_t)j * lda + r : ain, r < m);
                }
            }
            cp_async_wait_all();
            __syncwarp();
#pragma unroll
            for (int c = 0; c < CPL; ++c) {
                const int j = lane + 32 * c;
#pragma unroll
                for (int q = 0; q < ROWS / VEC; ++q) {
                    T vv[VEC];
                    if (j < n) ld_vec(tile + (size_t)j * LDT + q * VEC, vv);
#pragma unroll
                    for (int e = 0; e < VEC; ++e) {
                        a[c][q * VEC + e] = j < n ? vv[e] : T(0);
                        nonfinite |= !isfinite(a[c][q * VEC + e]);
                    }
                }
            }
        } else {
            // S(r, j) = stored(j, r) at r lda + j: for a fixed row the lanes read consecutive columns
#pragma unroll
            for (int c = 0; c < CPL; ++c) {
                const int j = lane + 32 * c;
#pragma unroll
                for (int r = 0; r < ROWS; ++r) {
                    const T x = (j < n && r < m) ? ain[(size_t)r * lda + j] : T(0);
                    nonfinite |= !isfinite(x);
                    a[c][r] = x;
                }
            }
        }
        if (__any_sync(0xffffffffu, nonfinite) && lane == 0) info[b] = BSVD_INFO_NONFINITE;
        __syncwarp();

        // ---- factorisation ----
#pragma unroll
        for (int c = 0; c < CPL; ++c) rdiag[c] = T(0);
        for (int i = 0; i < n; ++i) {
            T* v = tile + (size_t)i * LDT;
            if (lane == (i & 31)) {
                // two explicit arms (CPL <= 2) keep the register index static
                if (i < 32)
                    warp_store_column<T, ROWS>(v, a[0]);
                else
                    warp_store_column<T, ROWS>(v, a[CPL - 1]);
            }
            __syncwarp();
            // v_i = house(S(i:m, i)) in place, zero above row i; R(i, i) = -sign(x_0) ||x||
            const T x0 = v[i];
            T xs[NR];
            T ss = T(0);
#pragma unroll
            for (int t = 0; t < NR; ++t) {
                const int r = lane * NR + t;
                xs[t] = r >= i ? v[r] : T(0);
                ss = fma(xs[t], xs[t], ss);
            }
            ss = warp_sum(ss);
            const T alpha = dsqrt(ss);
            const T sg = x0 >= T(0) ? T(1) : T(-1);
            // ||x + sign(x0) alpha e1||^2 = 2 alpha (alpha + |x0|); a zero column gives v = 0
            const T inv = alpha > T(0) ? drsqrt(T(2) * alpha * (alpha + dabs(x0))) : T(0);
            __syncwarp();
#pragma unroll
            for (int t = 0; t < NR; ++t) {
                const int r = lane * NR + t;
                v[r] = (r == i ? x0 + sg * alpha : xs[t]) * inv;
            }
            if (lane == (i & 31)) {
                if (i < 32)
                    rdiag[0] = alpha > T(0) ? -sg * alpha : T(0);
                else
                    rdiag[CPL - 1] = alpha > T(0) ? -sg * alpha : T(0);
            }
            __syncwarp();
#pragma unroll
            for (int c = 0; c < CPL; ++c) {
                const int j = lane + 32 * c;
                if (j > i && j < n) warp_apply<T, ROWS>(v, a[c], i);
            }
        }

        // ---- R (n x n): rows above the diagonal of column j sit in lane j's registers ----
        if (R) {
            T* r_out = R[b];
#pragma unroll
            for (int c = 0; c < CPL; ++c) {
                const int j = lane + 32 * c;
                if (j < n) {
#pragma unroll
                    for (int r = 0; r < (NC < ROWS ? NC : ROWS); ++r) {  // n <= m <= ROWS
                        if (r >= n) break;
                        const T x = r < j ? a[c][r] : (r == j ? rdiag[c] : T(0));
                        r_out[r_trans ? (size_t)r * ldr + j : (size_t)j * ldr + r] = x;
                    }
                }
            }
        }

        // ---- Q = H_0 ... H_{n-1} [I; 0], column j in lane j's registers ----
        if (Q) {
#pragma unroll
            for (int c = 0; c < CPL; ++c)
#pragma unroll
                for (int r = 0; r < ROWS; ++r) a[c][r] = r == lane + 32 * c ? T(1) : T(0);
            for (int i = n - 1; i >= 0; --i) {
                const T* v = tile + (size_t)i * LDT;
#pragma unroll
                for (int c = 0; c < CPL; ++c) {
                    const int j = lane + 32 * c;
                    if (j >= i && j < n) warp_apply<T, ROWS>(v, a[c], i);
                }
            }
            __syncwarp();  // every lane has finished reading the reflectors
#pragma unroll
            for (int c = 0; c < CPL; ++c) {
                const int j = lane + 32 * c;
                if (j < n) warp_store_column<T, ROWS>(tile + (size_t)j * LDT, a[c]);
            }
            __syncwarp();
            T* q_out = Q[b];
#pragma unroll 2
            for (int j = 0; j < n; ++j)
#pragma unroll
                for (int t = 0; t < NR; ++t) {
                    const int r = lane + 32 * t;
                    if (r < m) q_out[(size_t)j * ldq + r] = tile[j * LDT + r];
                }
        }
        __syncwarp();  // the tile is reused by the next item
    }
}

template <typename T>
int launch_qr(int batch, int max_m, int max_n, void* const* A, const int* M, const int* N, const int* LDA,
              void* const* Q, const int* LDQ, void* const* R, const int* LDR, int* info, cudaStream_t st,
              ItemList wl, bool r_transposed, const int* a_trans)
{
    // narrow panels: one warp per matrix, the matrix in registers (lane = column)
    constexpr int kRegRows = sizeof(T) == 4 ? 128 : 64;  // register budget: ROWS x CPL elements per lane
    if (max_n <= 64 && max_m <= kRegRows && (max_n <= 32 || max_m <= kRegRows / 2)) {
        void (*kern)(int, int, int, T* const*, const int*, const int*, const int*, T* const*, const int*, T* const*,
                     const int*, int*, ItemList, int, const int*);
        size_t smem;
        if (max_n > 32) {
            kern = qr_warp_kernel<T, kRegRows / 2, 2>;
            smem = (size_t)WarpQrTile<T, kRegRows / 2>::kLd * 64 * sizeof(T);
        } else if (max_m <= 32) {
            kern = qr_warp_kernel<T, 32, 1>;
            smem = (size_t)WarpQrTile<T, 32>::kLd * 32 * sizeof(T);
        } else if (max_m <= 64) {
            kern = qr_warp_kernel<T, 64, 1>;
            smem = (size_t)WarpQrTile<T, 64>::kLd * 32 * sizeof(T);
        } else {
            kern = qr_warp_kernel<T, kRegRows, 1>;
            smem = (size_t)WarpQrTile<T, kRegRows>::kLd * 32 * sizeof(T);
        }
        constexpr int kWarps = 4;
        smem *= kWarps;
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return BSVD_ERR_CUDA;
        int grid;
        if (wl.idx == nullptr) {
            grid = ceil_div(batch < 1 ? 1 : batch, kWarps);
        } else {
            grid = item_grid(kern, 32 * kWarps, smem, wl, ceil_div(batch < 1 ? 1 : batch, kWarps), st);
            if (grid == 0) return BSVD_ERR_CUDA;
        }
        kern<<<grid, 32 * kWarps, smem, st>>>(batch, max_m, max_n, (T* const*)A, M, N, LDA, (T* const*)Q, LDQ,
                                              (T* const*)R, LDR, info, wl, r_transposed ? 1 : 0, a_trans);
        return cudaGetLastError() == cudaSuccess ? BSVD_SUCCESS : BSVD_ERR_CUDA;
    }
    const size_t smem = ((size_t)(max_m | 1) * max_n + max_n) * sizeof(T);
    // wide panels run one CTA per SM (the matrix fills shared memory): 16 warps hide the latency of
    // the per-column reductions better than 8
    // rows per lane of the register Q formation from the batch's row bound
    auto kern = max_m <= 32 ? qr_kernel<T, 1> : (max_m <= 64 ? qr_kernel<T, 2> : (max_m <= 128 ? qr_kernel<T, 4>
                                                                                             : qr_kernel<T, 8>));
    int threads = max_n <= 32 ? 128 : (max_n <= 64 ? 256 : 512);
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) return BSVD_ERR_CUDA;
    while (threads > fa.maxThreadsPerBlock && threads > 128) threads /= 2;  // the kernel's registers allow fewer
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
