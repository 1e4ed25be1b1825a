// qr_blocked.cu -- batched blocked Householder QR of large matrices in global memory, and the
// block-Jacobi SVD preconditioned by it.
//
// Blocked QR (Algorithm 1 in 32-column panels; the larger factorisations of Section 3.2).  The
// working matrix X (A, or A^T when m < n: mm x nn with mm >= nn) is factored panel by panel:
//   panel  the (mm - j0) x 32 panel is factored on chip by the Householder kernel's shared-memory
//          factorisation (unit-norm reflectors v_c with H_c = I - 2 v_c v_c^T stored in place at and
//          below the diagonal, R above it, R's diagonal aside), and the panel's compact WY factor T
//          is formed: H_0 ... H_31 = I - V T V^T with T upper triangular, T(c, c) = 2,
//          T(0:c, c) = -2 T(0:c, 0:c) V(:, 0:c)^T v_c;
//   update the trailing columns C = X(j0:, j0+32:) <- (I - V T V^T)^T C = C - V T^T (V^T C), in
//          32-column tiles, rows streamed through shared memory in chunks (any mm).
// Preconditioned block Jacobi (the QR preconditioning Section 6.3 names as future work; the same
// effect as the register tier's preconditioning, at the block level).  With X = Q R, the block tier
// runs on R^T (nn x nn, lower triangular, rows graded like the singular values): R^T = U~ S V~^T
// gives X = (Q V~) S U~^T, so X's right vectors are U~ and its left ones Q V~ = H_0 ... H_{nn-1} V~,
// formed by applying the panels' block reflectors, last panel first, to [V~; 0].
#include <cuda_runtime.h>

#include "common.cuh"
#include "house.cuh"
#include "launch.cuh"

namespace bsvd {

namespace {

constexpr int kPw = 32;    // panel width
constexpr int kCh = 128;   // rows per chunk of the block-reflector application

// shared memory of qb_apply_kernel: V and C chunks (32 x (kCh + 1)), V^T C and T (32 x 33)
template <typename T>
constexpr size_t qb_apply_smem() { return sizeof(T) * (2 * kPw * (kCh + 1) + 2 * kPw * (kPw + 1)); }

struct QbLayout {
    size_t off_ptr, off_int, off_X, off_T, off_rd, off_Rt, off_inner, inner_bytes, total;
    size_t strideX, strideT, strideRd, strideRt;   // elements per matrix
};

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// svd = false: the blocked QR alone (no R^T, no block-Jacobi workspace)
template <typename T>
QbLayout qb_layout(int batch, int max_m, int max_n, int bw, int method, bool svd = true)
{
    QbLayout L;
    const size_t mm = max_m > max_n ? max_m : max_n, nn = max_m > max_n ? max_n : max_m;
    const size_t P = (nn + kPw - 1) / kPw;
    L.strideX = mm * nn;
    L.strideT = P * kPw * kPw;
    L.strideRd = nn;
    L.strideRt = svd ? nn * nn : 0;
    size_t o = 0;
    L.off_ptr = o;
    o = al256(o + sizeof(void*) * (size_t)batch * 3);
    L.off_int = o;
    o = al256(o + sizeof(int) * (size_t)batch * 8);
    L.off_X = o;
    o = al256(o + sizeof(T) * L.strideX * batch);
    L.off_T = o;
    o = al256(o + sizeof(T) * L.strideT * batch);
    L.off_rd = o;
    o = al256(o + sizeof(T) * L.strideRd * batch);
    L.off_Rt = o;
    o = al256(o + sizeof(T) * L.strideRt * batch);
    L.off_inner = o;
    L.inner_bytes = svd ? block_jacobi_workspace<T>(batch, (int)nn, (int)nn, bw, method & 0xff) : 0;
    o = al256(o + L.inner_bytes);
    L.total = o;
    return L;
}

// per-matrix integers: 0 mm, 1 nn, 2 bad, 3 ld of X's left-vector output, 4 ld of its right-vector
// output, 5 n2 (nn, or 0 when bad: the inner call's sizes), 6 ld of R^T
struct QbInts {
    int *mm, *nn, *bad, *ldL, *ldR, *n2, *ldRt;
};

template <typename T>
struct QbPtrs {
    T **Rt, **XL, **XR;
};

template <typename T>
__device__ __forceinline__ T* qb_X(unsigned char* ws, const QbLayout& L, int b)
{
    return reinterpret_cast<T*>(ws + L.off_X) + (size_t)b * L.strideX;
}

// setup: shapes, X = A or A^T (ld mm), the inner call's pointer and size arrays
template <typename T>
__global__ void __launch_bounds__(256) qb_setup_kernel(int batch, int max_mm, int max_nn, T* const* A, const int* M,
                                                       const int* N, const int* LDA, T* const* U, const int* LDU,
                                                       T* const* V, const int* LDV, unsigned char* ws, QbLayout L,
                                                       QbInts I, QbPtrs<T> Pp, int* info)
{
    const int b = blockIdx.x;
    const int m = M[b], n = N[b], lda = LDA[b], ldu = LDU[b], ldv = LDV[b];
    const bool tr = m < n;
    const int mm = tr ? n : m, nn = tr ? m : n;
    const bool bad = m < 0 || n < 0 || mm > max_mm || nn > max_nn || lda < (m > 1 ? m : 1) ||
                     ldu < (m > 1 ? m : 1) || ldv < (n > 1 ? n : 1);
    if (threadIdx.x == 0) {
        I.mm[b] = bad ? 0 : mm;
        I.nn[b] = bad ? 0 : nn;
        I.bad[b] = bad ? 1 : 0;
        I.n2[b] = bad ? 0 : nn;
        I.ldRt[b] = nn > 1 ? nn : 1;
        I.ldL[b] = tr ? ldv : ldu;
        I.ldR[b] = tr ? ldu : ldv;
        Pp.Rt[b] = reinterpret_cast<T*>(ws + L.off_Rt) + (size_t)b * L.strideRt;
        Pp.XL[b] = tr ? V[b] : U[b];
        Pp.XR[b] = tr ? U[b] : V[b];
        if (bad) info[b] = BSVD_INFO_BAD_SHAPE;
    }
    if (bad) return;
    T* X = qb_X<T>(ws, L, b);
    const T* a = A[b];
    for (size_t e = threadIdx.x; e < (size_t)mm * nn; e += blockDim.x) {
        const int j = (int)(e / mm), i = (int)(e - (size_t)j * mm);
        X[e] = tr ? a[(size_t)i * lda + j] : a[(size_t)j * lda + i];
    }
}

// panel p: factor X(j0:mm, j0:j0+32) on chip, write reflectors and R back, form T
template <typename T>
__global__ void __launch_bounds__(256) qb_panel_kernel(int p, unsigned char* ws, QbLayout L, QbInts I)
{
    extern __shared__ __align__(16) unsigned char qb_sm[];
    const int b = blockIdx.x;
    const int mm = I.mm[b], nn = I.nn[b];
    const int j0 = p * kPw;
    if (j0 >= nn) return;
    const int rows = mm - j0;                          // >= nn - j0 >= 1
    const int mr = rows > kPw ? rows : kPw;            // factored height (zero rows below `rows`)
    const int ld = mr | 1;
    T* S = reinterpret_cast<T*>(qb_sm);
    T* diag = S + (size_t)ld * kPw;
    T* G = diag + kPw;                                 // V^T V, 32 x 33
    T* Ts = G + kPw * (kPw + 1);                       // T, 32 x 33
    T* X = qb_X<T>(ws, L, b);
    for (int e = threadIdx.x; e < ld * kPw; e += blockDim.x) {
        const int c = e / ld, r = e - c * ld;
        S[e] = (r < rows && j0 + c < nn) ? X[(size_t)(j0 + c) * mm + j0 + r] : T(0);
    }
    __syncthreads();
    house_factor_smem(S, ld, diag, mr, kPw);
    __syncthreads();
    for (int e = threadIdx.x; e < rows * kPw; e += blockDim.x) {
        const int c = e / rows, r = e - c * rows;
        if (j0 + c < nn) X[(size_t)(j0 + c) * mm + j0 + r] = S[(size_t)c * ld + r];
    }
    T* rd = reinterpret_cast<T*>(ws + L.off_rd) + (size_t)b * L.strideRd;
    if (threadIdx.x < kPw && j0 + (int)threadIdx.x < nn) rd[j0 + threadIdx.x] = diag[threadIdx.x];
    // G = V^T V with V(r, c) = S(r, c) for r >= c, 0 above; one warp per entry group
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int e = warp; e < kPw * kPw; e += nw) {
        const int i = e / kPw, j = e - i * kPw;
        if (j < i) continue;                           // symmetric: the upper triangle is enough
        T s = T(0);
        for (int r = j + lane; r < mr; r += 32) s += S[(size_t)i * ld + r] * S[(size_t)j * ld + r];
        s = warp_sum(s);
        if (lane == 0) G[i * (kPw + 1) + j] = s;       // G(i, j), i <= j
    }
    for (int e = threadIdx.x; e < kPw * (kPw + 1); e += blockDim.x) Ts[e] = T(0);
    __syncthreads();
    // T column by column: T(c, c) = 2, T(0:c, c) = -2 T(0:c, 0:c) G(0:c, c)
    for (int c = 0; c < kPw; ++c) {
        if (threadIdx.x < (unsigned)c) {
            const int i = threadIdx.x;
            T s = T(0);
            for (int k = i; k < c; ++k) s += Ts[k * (kPw + 1) + i] * G[k * (kPw + 1) + c];  // T(i, k) G(k, c)
            Ts[c * (kPw + 1) + i] = T(-2) * s;                                              // T(i, c)
        }
        if (threadIdx.x == 0) Ts[c * (kPw + 1) + c] = T(2);
        __syncthreads();
    }
    T* Tg = reinterpret_cast<T*>(ws + L.off_T) + (size_t)b * L.strideT + (size_t)p * kPw * kPw;
    for (int e = threadIdx.x; e < kPw * kPw; e += blockDim.x) {
        const int c = e / kPw, i = e - c * kPw;
        Tg[e] = Ts[c * (kPw + 1) + i];                 // column-major T(i, c)
    }
}

// block reflector of panel p applied to 32 columns of C (rows j0 .. mm-1):
//   trans = 1: C <- (I - V T V^T)^T C = C - V T^T (V^T C)   (the QR's trailing update; C in X)
//   trans = 0: C <- (I - V T V^T) C   = C - V T (V^T C)     (forming Q V~ or Q; C in the output)
// One CTA per (matrix, 32-column tile); tile t covers columns c0_base + 32 t ...; rows in chunks of
// kCh through shared memory, twice.
template <typename T>
__global__ void __launch_bounds__(256) qb_apply_kernel(int p, int trans, int tiles, unsigned char* ws, QbLayout L,
                                                       QbInts I, T* const* Cp, const int* LDC, int c0_base)
{
    extern __shared__ __align__(16) unsigned char ap_sm[];
    T(*Vs)[kCh + 1] = reinterpret_cast<T(*)[kCh + 1]>(ap_sm);                       // V chunk (column i, row r)
    T(*Cs)[kCh + 1] = Vs + kPw;                                                    // C chunk
    T(*Ws)[kPw + 1] = reinterpret_cast<T(*)[kPw + 1]>(Cs + kPw);                   // V^T C, then op(T) V^T C
    T(*Tsm)[kPw + 1] = Ws + kPw;                                                   // T (column c, row i)
    const int b = blockIdx.x / tiles, t = blockIdx.x - b * tiles;
    const int mm = I.mm[b], nn = I.nn[b];
    const int j0 = p * kPw;
    if (j0 >= nn) return;
    // columns of C: trailing update X(:, j0+32+32t ..), the left vectors' columns 32t .., or Q's
    // columns j0 + 32t .. (those left of j0 are still e_c there, which the panel leaves alone)
    const int c0 = c0_base + kPw * t;
    if (c0 >= nn) return;
    const int ncol = nn - c0 < kPw ? nn - c0 : kPw;
    const int vcols = nn - j0 < kPw ? nn - j0 : kPw;   // reflectors of this panel (zero beyond)
    T* C = Cp ? Cp[b] : qb_X<T>(ws, L, b);
    const int ldc = Cp ? LDC[b] : mm;
    const T* X = qb_X<T>(ws, L, b);
    const T* Tg = reinterpret_cast<const T*>(ws + L.off_T) + (size_t)b * L.strideT + (size_t)p * kPw * kPw;
    const int tid = threadIdx.x;
    for (int e = tid; e < kPw * kPw; e += 256) Tsm[e / kPw][e % kPw] = Tg[e];
    // thread's 2 x 2 block of the 32 x 32 product: rows 2 ti, 2 ti + 1, columns 2 tj, 2 tj + 1
    const int ti = tid & 15, tj = tid >> 4;
    T w00 = T(0), w01 = T(0), w10 = T(0), w11 = T(0);
    const int rows = mm - j0;
    for (int r0 = 0; r0 < rows; r0 += kCh) {
        __syncthreads();
        for (int e = tid; e < kPw * kCh; e += 256) {
            const int c = e / kCh, r = e - c * kCh;
            const int gr = j0 + r0 + r;                // row of X / C
            T v = T(0), x = T(0);
            if (r0 + r < rows) {
                if (c < vcols && r0 + r >= c) v = X[(size_t)(j0 + c) * mm + gr];
                if (c < ncol) x = C[(size_t)(c0 + c) * ldc + gr];
            }
            Vs[c][r] = v;
            Cs[c][r] = x;
        }
        __syncthreads();
        const int rn = rows - r0 < kCh ? rows - r0 : kCh;
        for (int r = 0; r < rn; ++r) {
            const T va = Vs[2 * ti][r], vb = Vs[2 * ti + 1][r];
            const T xa = Cs[2 * tj][r], xb = Cs[2 * tj + 1][r];
            w00 = fma(va, xa, w00);
            w01 = fma(va, xb, w01);
            w10 = fma(vb, xa, w10);
            w11 = fma(vb, xb, w11);
        }
    }
    Ws[2 * tj][2 * ti] = w00;
    Ws[2 * tj + 1][2 * ti] = w01;
    Ws[2 * tj][2 * ti + 1] = w10;
    Ws[2 * tj + 1][2 * ti + 1] = w11;
    __syncthreads();
    // op(T) W: row i of op(T) is column i of T (trans) or row i of T (no trans)
    T y00 = T(0), y01 = T(0), y10 = T(0), y11 = T(0);
    for (int k = 0; k < kPw; ++k) {
        const T ta = trans ? Tsm[2 * ti][k] : Tsm[k][2 * ti];
        const T tb = trans ? Tsm[2 * ti + 1][k] : Tsm[k][2 * ti + 1];
        const T xa = Ws[2 * tj][k], xb = Ws[2 * tj + 1][k];
        y00 = fma(ta, xa, y00);
        y01 = fma(ta, xb, y01);
        y10 = fma(tb, xa, y10);
        y11 = fma(tb, xb, y11);
    }
    __syncthreads();
    Ws[2 * tj][2 * ti] = y00;
    Ws[2 * tj + 1][2 * ti] = y01;
    Ws[2 * tj][2 * ti + 1] = y10;
    Ws[2 * tj + 1][2 * ti + 1] = y11;
    // C -= V (op(T) V^T C), chunk by chunk again
    for (int r0 = 0; r0 < rows; r0 += kCh) {
        __syncthreads();
        for (int e = tid; e < kPw * kCh; e += 256) {
            const int c = e / kCh, r = e - c * kCh;
            const int gr = j0 + r0 + r;
            T v = T(0), x = T(0);
            if (r0 + r < rows) {
                if (c < vcols && r0 + r >= c) v = X[(size_t)(j0 + c) * mm + gr];
                if (c < ncol) x = C[(size_t)(c0 + c) * ldc + gr];
            }
            Vs[c][r] = v;
            Cs[c][r] = x;
        }
        __syncthreads();
        const int rn = rows - r0 < kCh ? rows - r0 : kCh;
        // thread: row r = tid % kCh, columns (tid / kCh) * 16 .. + 15
        const int r = tid % kCh, cb = (tid / kCh) * (kPw / 2);
        if (r < rn) {
#pragma unroll 4
            for (int j = 0; j < kPw / 2; ++j) {
                const int c = cb + j;
                if (c >= ncol) break;
                T acc = Cs[c][r];
                for (int i = 0; i < kPw; ++i) acc = fma(-Vs[i][r], Ws[c][i], acc);
                C[(size_t)(c0 + c) * ldc + j0 + r0 + r] = acc;
            }
        }
    }
}

// R^T (nn x nn, lower triangular) from X's strict upper part and the diagonal
template <typename T>
__global__ void __launch_bounds__(256) qb_rt_kernel(unsigned char* ws, QbLayout L, QbInts I)
{
    const int b = blockIdx.x;
    const int mm = I.mm[b], nn = I.nn[b];
    const T* X = qb_X<T>(ws, L, b);
    const T* rd = reinterpret_cast<const T*>(ws + L.off_rd) + (size_t)b * L.strideRd;
    T* Rt = reinterpret_cast<T*>(ws + L.off_Rt) + (size_t)b * L.strideRt;
    for (size_t e = threadIdx.x; e < (size_t)nn * nn; e += blockDim.x) {
        const int j = (int)(e / nn), i = (int)(e - (size_t)j * nn);   // Rt(i, j) = R(j, i)
        Rt[e] = i > j ? X[(size_t)i * mm + j] : (i == j ? rd[i] : T(0));
    }
}

// the left vectors [V~; 0]: rows nn .. mm-1 zeroed; bad shapes marked again (the inner call saw
// them as empty)
template <typename T>
__global__ void __launch_bounds__(256) qb_mid_kernel(QbInts I, QbPtrs<T> Pp, int* info)
{
    const int b = blockIdx.x;
    if (I.bad[b]) {
        if (threadIdx.x == 0) info[b] = BSVD_INFO_BAD_SHAPE;
        return;
    }
    const int mm = I.mm[b], nn = I.nn[b], ld = I.ldL[b];
    if (mm == nn) return;
    T* XL = Pp.XL[b];
    for (size_t e = threadIdx.x; e < (size_t)(mm - nn) * nn; e += blockDim.x) {
        const int j = (int)(e / (mm - nn)), i = nn + (int)(e - (size_t)j * (mm - nn));
        XL[(size_t)j * ld + i] = T(0);
    }
}

// ---- the blocked QR as an entry of its own (A = Q R of matrices beyond the shared-memory kernel) ----

// setup: shapes (m >= n), X = A (ld m); a bad shape gets mm = nn = 0, so every later stage skips it
template <typename T>
__global__ void __launch_bounds__(256) qbq_setup_kernel(int max_mm, int max_nn, T* const* A, const int* M,
                                                        const int* N, const int* LDA, T* const* Q, const int* LDQ,
                                                        T* const* R, const int* LDR, unsigned char* ws, QbLayout L,
                                                        QbInts I, int* info)
{
    const int b = blockIdx.x;
    const int m = M[b], n = N[b], lda = LDA[b];
    const int ldq = Q ? LDQ[b] : 1, ldr = R ? LDR[b] : 1;
    const bool bad = m < 0 || n < 0 || m < n || m > max_mm || n > max_nn || lda < (m > 1 ? m : 1) ||
                     (Q && ldq < (m > 1 ? m : 1)) || (R && ldr < (n > 1 ? n : 1));
    if (threadIdx.x == 0) {
        I.mm[b] = bad ? 0 : m;
        I.nn[b] = bad ? 0 : n;
        I.bad[b] = bad ? 1 : 0;
        info[b] = bad ? BSVD_INFO_BAD_SHAPE : 0;
    }
    if (bad) return;
    T* X = qb_X<T>(ws, L, b);
    const T* a = A[b];
    for (size_t e = threadIdx.x; e < (size_t)m * n; e += blockDim.x) {
        const int j = (int)(e / m), i = (int)(e - (size_t)j * m);
        X[e] = a[(size_t)j * lda + i];
    }
}

// R (n x n: X's strict upper triangle, the diagonal from rd, exact zeros below) and Q = [I; 0]
// (m x n), which the panels' block reflectors then turn into H_0 ... H_{n-1} [I; 0]
template <typename T>
__global__ void __launch_bounds__(256) qbq_out_kernel(T* const* Q, const int* LDQ, T* const* R, const int* LDR,
                                                      unsigned char* ws, QbLayout L, QbInts I)
{
    const int b = blockIdx.x;
    const int mm = I.mm[b], nn = I.nn[b];
    if (nn == 0) return;
    const T* X = qb_X<T>(ws, L, b);
    const T* rd = reinterpret_cast<const T*>(ws + L.off_rd) + (size_t)b * L.strideRd;
    if (R) {
        T* r = R[b];
        const int ldr = LDR[b];
        for (size_t e = threadIdx.x; e < (size_t)nn * nn; e += blockDim.x) {
            const int j = (int)(e / nn), i = (int)(e - (size_t)j * nn);
            r[(size_t)j * ldr + i] = i < j ? X[(size_t)j * mm + i] : (i == j ? rd[i] : T(0));
        }
    }
    if (Q) {
        T* q = Q[b];
        const int ldq = LDQ[b];
        for (size_t e = threadIdx.x; e < (size_t)mm * nn; e += blockDim.x) {
            const int j = (int)(e / mm), i = (int)(e - (size_t)j * mm);
            q[(size_t)j * ldq + i] = i == j ? T(1) : T(0);
        }
    }
}

}  // namespace

template <typename T>
size_t block_jacobi_qr_workspace(int batch, int max_m, int max_n, int bw, int method)
{
    return qb_layout<T>(batch, max_m, max_n, bw, method).total;
}

template <typename T>
int launch_block_jacobi_qr(int batch, int max_m, int max_n, int bw, int method, void* const* A, const int* M,
                           const int* N, const int* LDA, void* const* S, void* const* U, const int* LDU,
                           void* const* V, const int* LDV, double tol, int max_sweeps, int* info, long long* rot,
                           void* ws_v, size_t ws_bytes, cudaStream_t st)
{
    const int mm = max_m > max_n ? max_m : max_n, nn = max_m > max_n ? max_n : max_m;
    const int ldp = (mm > kPw ? mm : kPw) | 1;
    const size_t panel_smem = sizeof(T) * ((size_t)ldp * kPw + kPw + 2 * kPw * (kPw + 1));
    if (panel_smem > 200 * 1024) return BSVD_ERR_UNSUPPORTED;
    const QbLayout L = qb_layout<T>(batch, max_m, max_n, bw, method);
    if (ws_bytes < L.total) return BSVD_ERR_WORKSPACE;
    unsigned char* ws = static_cast<unsigned char*>(ws_v);
    QbPtrs<T> Pp;
    T** pp = reinterpret_cast<T**>(ws + L.off_ptr);
    Pp.Rt = pp;
    Pp.XL = pp + batch;
    Pp.XR = pp + 2 * (size_t)batch;
    QbInts I;
    int* ip = reinterpret_cast<int*>(ws + L.off_int);
    int** slots[7] = {&I.mm, &I.nn, &I.bad, &I.ldL, &I.ldR, &I.n2, &I.ldRt};
    for (int i = 0; i < 7; ++i) *slots[i] = ip + (size_t)i * batch;
    qb_setup_kernel<T><<<batch, 256, 0, st>>>(batch, mm, nn, (T* const*)A, M, N, LDA, (T* const*)U, LDU, (T* const*)V,
                                              LDV, ws, L, I, Pp, info);
    if (cudaGetLastError() != cudaSuccess) return BSVD_ERR_CUDA;
    if (panel_smem > 48 * 1024 &&
        cudaFuncSetAttribute(qb_panel_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)panel_smem) !=
            cudaSuccess)
        return BSVD_ERR_CUDA;
    constexpr size_t apply_smem = qb_apply_smem<T>();
    if (apply_smem > 48 * 1024 &&
        cudaFuncSetAttribute(qb_apply_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)apply_smem) !=
            cudaSuccess)
        return BSVD_ERR_CUDA;
    const int P = (nn + kPw - 1) / kPw;
    const int tiles = P;   // 32-column tiles of nn
    for (int p = 0; p < P; ++p) {
        qb_panel_kernel<T><<<batch, 256, panel_smem, st>>>(p, ws, L, I);
        if (p + 1 < P)
            qb_apply_kernel<T><<<batch * (P - p - 1), 256, apply_smem, st>>>(p, 1, P - p - 1, ws, L, I, nullptr,
                                                                              nullptr, p * kPw + kPw);
        if (cudaGetLastError() != cudaSuccess) return BSVD_ERR_CUDA;
    }
    qb_rt_kernel<T><<<batch, 256, 0, st>>>(ws, L, I);
    if (cudaGetLastError() != cudaSuccess) return BSVD_ERR_CUDA;
    // block Jacobi on R^T: its left vectors U~ are X's right vectors, its right vectors V~ go to the
    // top of X's left-vector output
    const int inner_method = method & ~BSVD_BLOCK_QR_PRECONDITION;
    int rc = launch_block_jacobi<T>(batch, nn, nn, bw, inner_method, (void* const*)Pp.Rt, I.n2, I.n2, I.ldRt, S,
                                    (void* const*)Pp.XR, I.ldR, (void* const*)Pp.XL, I.ldL, tol, max_sweeps, info, rot,
                                    ws + L.off_inner, L.inner_bytes, st);
    if (rc != BSVD_SUCCESS) return rc;
    qb_mid_kernel<T><<<batch, 256, 0, st>>>(I, Pp, info);
    // X's left vectors: Q [V~; 0] = H_0 ... H_{nn-1} [V~; 0], last panel first
    for (int p = P - 1; p >= 0; --p) {
        qb_apply_kernel<T><<<batch * tiles, 256, apply_smem, st>>>(p, 0, tiles, ws, L, I, Pp.XL, I.ldL, 0);
        if (cudaGetLastError() != cudaSuccess) return BSVD_ERR_CUDA;
    }
    return BSVD_SUCCESS;
}

// the blocked QR alone: X = A, panels and trailing updates, then R and Q = H_0 ... H_{n-1} [I; 0]
// (panel p's block reflector applied, last panel first, to Q's columns from p's first on)
// (bounds of 0 are taken as 1, as the launcher does)
template <typename T>
size_t qr_blocked_workspace(int batch, int max_m, int max_n)
{
    return qb_layout<T>(batch, max_m > 1 ? max_m : 1, max_n > 1 ? max_n : 1, 32, 0, false).total;
}

template <typename T>
int launch_qr_blocked(int batch, int max_m, int max_n, void* const* A, const int* M, const int* N, const int* LDA,
                      void* const* Q, const int* LDQ, void* const* R, const int* LDR, int* info, void* ws_v,
                      size_t ws_bytes, cudaStream_t st)
{
    if (qr_blocked_max_rows<T>() < max_m) return BSVD_ERR_UNSUPPORTED;
    const int ldp = (max_m > kPw ? max_m : kPw) | 1;
    const size_t panel_smem = sizeof(T) * ((size_t)ldp * kPw + kPw + 2 * kPw * (kPw + 1));
    const QbLayout L = qb_layout<T>(batch, max_m, max_n, 32, 0, false);
    if (ws_bytes < L.total) return BSVD_ERR_WORKSPACE;
    unsigned char* ws = static_cast<unsigned char*>(ws_v);
    QbInts I;
    int* ip = reinterpret_cast<int*>(ws + L.off_int);
    int** slots[7] = {&I.mm, &I.nn, &I.bad, &I.ldL, &I.ldR, &I.n2, &I.ldRt};
    for (int i = 0; i < 7; ++i) *slots[i] = ip + (size_t)i * batch;
    qbq_setup_kernel<T><<<batch, 256, 0, st>>>(max_m, max_n, (T* const*)A, M, N, LDA, (T* const*)Q, LDQ, (T* const*)R,
                                               LDR, ws, L, I, info);
    if (cudaGetLastError() != cudaSuccess) return BSVD_ERR_CUDA;
    if (panel_smem > 48 * 1024 &&
        cudaFuncSetAttribute(qb_panel_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)panel_smem) !=
            cudaSuccess)
        return BSVD_ERR_CUDA;
    constexpr size_t apply_smem = qb_apply_smem<T>();
    if (apply_smem > 48 * 1024 &&
        cudaFuncSetAttribute(qb_apply_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)apply_smem) !=
            cudaSuccess)
        return BSVD_ERR_CUDA;
    const int P = (max_n + kPw - 1) / kPw;
    for (int p = 0; p < P; ++p) {
        qb_panel_kernel<T><<<batch, 256, panel_smem, st>>>(p, ws, L, I);
        if (p + 1 < P)
            qb_apply_kernel<T><<<batch * (P - p - 1), 256, apply_smem, st>>>(p, 1, P - p - 1, ws, L, I, nullptr,
                                                                              nullptr, p * kPw + kPw);
        if (cudaGetLastError() != cudaSuccess) return BSVD_ERR_CUDA;
    }
    qbq_out_kernel<T><<<batch, 256, 0, st>>>((T* const*)Q, LDQ, (T* const*)R, LDR, ws, L, I);
    if (cudaGetLastError() != cudaSuccess) return BSVD_ERR_CUDA;
    if (Q) {
        for (int p = P - 1; p >= 0; --p) {
            qb_apply_kernel<T><<<batch * (P - p), 256, apply_smem, st>>>(p, 0, P - p, ws, L, I, (T* const*)Q, LDQ,
                                                                          p * kPw);
            if (cudaGetLastError() != cudaSuccess) return BSVD_ERR_CUDA;
        }
    }
    return BSVD_SUCCESS;
}

// rows of the tallest matrix whose 32-column panel fits on chip (200 KiB of shared memory)
template <typename T>
int qr_blocked_max_rows()
{
    const size_t fixed = sizeof(T) * (kPw + 2 * kPw * (kPw + 1));
    const size_t ld = (200 * 1024 - fixed) / (sizeof(T) * kPw);   // largest ld with the panel in 200 KiB
    return (int)(ld % 2 ? ld : ld - 1);                          // ld = rows | 1
}

template size_t block_jacobi_qr_workspace<float>(int, int, int, int, int);
template size_t block_jacobi_qr_workspace<double>(int, int, int, int, int);
template int launch_block_jacobi_qr<float>(int, int, int, int, int, void* const*, const int*, const int*, const int*,
                                           void* const*, void* const*, const int*, void* const*, const int*, double,
                                           int, int*, long long*, void*, size_t, cudaStream_t);
template int launch_block_jacobi_qr<double>(int, int, int, int, int, void* const*, const int*, const int*,
                                            const int*, void* const*, void* const*, const int*, void* const*,
                                            const int*, double, int, int*, long long*, void*, size_t, cudaStream_t);

template size_t qr_blocked_workspace<float>(int, int, int);
template size_t qr_blocked_workspace<double>(int, int, int);
template int qr_blocked_max_rows<float>();
template int qr_blocked_max_rows<double>();
template int launch_qr_blocked<float>(int, int, int, void* const*, const int*, const int*, const int*, void* const*,
                                      const int*, void* const*, const int*, int*, void*, size_t, cudaStream_t);
template int launch_qr_blocked<double>(int, int, int, void* const*, const int*, const int*, const int*, void* const*,
                                       const int*, void* const*, const int*, int*, void*, size_t, cudaStream_t);

}  // namespace bsvd
