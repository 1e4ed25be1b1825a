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
// A panel too tall for one CTA's shared memory is factored by a thread-block cluster of up to 8
// CTAs, each holding a slab of its rows: per column, the CTAs' partial sums of squares, then their
// partial products with the panel's other columns, are exchanged through distributed shared memory
// (two cluster barriers), every CTA forming the same reflector from the same sums.
// Preconditioned block Jacobi (the QR preconditioning Section 6.3 names as future work; the same
// effect as the register tier's preconditioning, at the block level).  With X = Q R, the block tier
// runs on R^T (nn x nn, lower triangular, rows graded like the singular values): R^T = U~ S V~^T
// gives X = (Q V~) S U~^T, so X's right vectors are U~ and its left ones Q V~ = H_0 ... H_{nn-1} V~,
// formed by applying the panels' block reflectors, last panel first, to [V~; 0].
#include <cooperative_groups.h>
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
    constexpr int kRun = 8;   // each thread's loads in flight together, then its shared stores
    for (int e0 = 0; e0 < ld * kPw; e0 += kRun * (int)blockDim.x) {
        T x[kRun];
#pragma unroll
        for (int u = 0; u < kRun; ++u) {
            const int e = e0 + threadIdx.x + u * blockDim.x;
            const int c = e / ld, r = e - c * ld;
            x[u] = (e < ld * kPw && r < rows && j0 + c < nn) ? X[(size_t)(j0 + c) * mm + j0 + r] : T(0);
        }
#pragma unroll
        for (int u = 0; u < kRun; ++u) {
            const int e = e0 + threadIdx.x + u * blockDim.x;
            if (e < ld * kPw) S[e] = x[u];
        }
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
    // a chunk of V and of C: each thread's loads in flight together, then its shared stores (a
    // store between two loads would make each load wait for the previous one's data)
    constexpr int PE = (kPw * kCh) / 256;
    auto stage = [&](int r0) {
        T v[PE], x[PE];
#pragma unroll
        for (int q = 0; q < PE; ++q) {
            const int e = tid + 256 * q;
            const int c = e / kCh, r = e - c * kCh;
            const int gr = j0 + r0 + r;                // row of X / C
            v[q] = T(0);
            x[q] = T(0);
            if (r0 + r < rows) {
                if (c < vcols && r0 + r >= c) v[q] = X[(size_t)(j0 + c) * mm + gr];
                if (c < ncol) x[q] = C[(size_t)(c0 + c) * ldc + gr];
            }
        }
#pragma unroll
        for (int q = 0; q < PE; ++q) {
            const int e = tid + 256 * q;
            const int c = e / kCh, r = e - c * kCh;
            Vs[c][r] = v[q];
            Cs[c][r] = x[q];
        }
    };
    for (int r0 = 0; r0 < rows; r0 += kCh) {
        __syncthreads();
        stage(r0);
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
        stage(r0);
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

// ---- tall panels: one thread-block cluster per matrix, a slab of the panel's rows per CTA ----

namespace cg = cooperative_groups;

constexpr int kClusterMax = 8;   // CTAs per cluster (the portable maximum)

// dynamic shared memory of the cluster panel kernel for slabs of up to `slab` rows:
// S (slab | 1) x 32, diag, partial Gram (32 x 33), G and T (32 x 33 each), part/xq (2 + 2),
// wpart (2 x 32)
template <typename T>
size_t qb_cpanel_smem(int slab)
{
    return sizeof(T) * ((size_t)(slab | 1) * kPw + kPw + 3 * kPw * (kPw + 1) + 4 + 2 * kPw);
}

template <typename T>
__device__ __forceinline__ T qb_block_sum(T v, T* red)
{
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    T s = T(0);
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    __syncthreads();
    return s;   // in thread 0
}

// panel p of matrix blockIdx.x / cs, CTA `rank` of its cluster holding panel rows
// [rank * slab, rank * slab + nr): Householder reflectors of the panel's columns (Algorithm 1, the
// same reflectors and signs as the one-CTA factorisation), R, and the compact WY factor T
template <typename T>
__global__ void __launch_bounds__(256) qb_panel_cluster_kernel(int p, int cs, unsigned char* ws, QbLayout L, QbInts I)
{
    extern __shared__ __align__(16) unsigned char qc_sm[];
    __shared__ T red[8];
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int b = blockIdx.x / cs;
    const int mm = I.mm[b], nn = I.nn[b];
    const int j0 = p * kPw;
    if (j0 >= nn) return;   // the whole cluster (one matrix) leaves together
    const int rows = mm - j0;
    const int slab = ((rows + cs - 1) / cs) > kPw ? (rows + cs - 1) / cs : kPw;   // CTA 0 holds rows 0 .. 31
    const int lds = slab | 1;
    const int r0 = rank * slab;
    const int nr = rows - r0 < 0 ? 0 : (rows - r0 > slab ? slab : rows - r0);
    const int vcols = nn - j0 < kPw ? nn - j0 : kPw;
    T* S = reinterpret_cast<T*>(qc_sm);
    T* diag = S + (size_t)lds * kPw;
    T* Gp = diag + kPw;                 // this CTA's partial V^T V
    T* G = Gp + kPw * (kPw + 1);        // the cluster's sum (CTA 0)
    T* Ts = G + kPw * (kPw + 1);        // T (CTA 0)
    T* part = Ts + kPw * (kPw + 1);     // [2]: partial sum of squares of the current column
    T* xq = part + 2;                   // [2]: the column's diagonal entry (CTA 0)
    T* wpart = xq + 2;                  // [2][32]: partial products with the columns to its right
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    T* X = qb_X<T>(ws, L, b);
    constexpr int kRun = 8;   // each thread's loads in flight together, then its shared stores
    for (int e0 = 0; e0 < nr * kPw; e0 += kRun * (int)blockDim.x) {
        T x[kRun];
#pragma unroll
        for (int u = 0; u < kRun; ++u) {
            const int e = e0 + tid + u * blockDim.x;
            const int c = e / (nr > 0 ? nr : 1), lr = e - c * nr;
            x[u] = (e < nr * kPw && j0 + c < nn) ? X[(size_t)(j0 + c) * mm + j0 + r0 + lr] : T(0);
        }
#pragma unroll
        for (int u = 0; u < kRun; ++u) {
            const int e = e0 + tid + u * blockDim.x;
            if (e < nr * kPw) {
                const int c = e / nr, lr = e - c * nr;
                S[c * lds + lr] = x[u];
            }
        }
    }
    __syncthreads();
    for (int i = 0; i < vcols; ++i) {
        const int par = i & 1;
        T* col = S + (size_t)i * lds;
        // this CTA's share of ||x||^2 over the panel rows at and below i
        T ss = T(0);
        for (int lr = tid; lr < nr; lr += blockDim.x)
            if (r0 + lr >= i) ss += col[lr] * col[lr];
        ss = qb_block_sum(ss, red);
        if (tid == 0) {
            part[par] = ss;
            if (rank == 0) xq[par] = col[i];
        }
        cluster.sync();
        // every CTA forms the same reflector from the same sums (added in rank order)
        T tot = T(0);
        for (int q = 0; q < cs; ++q) tot += *cluster.map_shared_rank(part + par, q);
        const T x0 = *cluster.map_shared_rank(xq + par, 0);
        const T alpha = dsqrt(tot);
        const T sg = x0 >= T(0) ? T(1) : T(-1);
        const T inv = alpha > T(0) ? drsqrt(T(2) * alpha * (alpha + dabs(x0))) : T(0);
        for (int lr = tid; lr < nr; lr += blockDim.x) {
            const int pr = r0 + lr;
            if (pr >= i) col[lr] = (pr == i ? x0 + sg * alpha : col[lr]) * inv;
        }
        if (rank == 0 && tid == 0) diag[i] = -sg * alpha;
        __syncthreads();
        // this CTA's share of v^T (column j) for the panel's columns right of i (a warp per column)
        for (int j = i + 1 + warp; j < vcols; j += 8) {
            const T* cj = S + (size_t)j * lds;
            T d = T(0);
            for (int lr = lane; lr < nr; lr += 32)
                if (r0 + lr >= i) d += col[lr] * cj[lr];
            d = warp_sum(d);
            if (lane == 0) wpart[par * kPw + j] = d;
        }
        cluster.sync();
        for (int j = i + 1 + warp; j < vcols; j += 8) {
            T w = T(0);
            for (int q = 0; q < cs; ++q) w += *cluster.map_shared_rank(wpart + par * kPw + j, q);
            w *= T(2);
            T* cj = S + (size_t)j * lds;
            for (int lr = lane; lr < nr; lr += 32)
                if (r0 + lr >= i) cj[lr] -= w * col[lr];
        }
        __syncthreads();
    }
    // this CTA's share of V^T V (V(r, c) = S(r, c) at and below the panel's diagonal)
    for (int e = warp; e < kPw * kPw; e += 8) {
        const int i = e / kPw, j = e - i * kPw;
        if (j < i) continue;
        T s = T(0);
        if (j < vcols)
            for (int lr = lane; lr < nr; lr += 32)
                if (r0 + lr >= j) s += S[(size_t)i * lds + lr] * S[(size_t)j * lds + lr];
        s = warp_sum(s);
        if (lane == 0) Gp[i * (kPw + 1) + j] = s;
    }
    cluster.sync();
    if (rank == 0) {
        for (int e = tid; e < kPw * (kPw + 1); e += blockDim.x) {
            T s = T(0);
            for (int q = 0; q < cs; ++q) s += *cluster.map_shared_rank(Gp + e, q);
            G[e] = s;
            Ts[e] = T(0);
        }
        __syncthreads();
        for (int c = 0; c < kPw; ++c) {   // T(c, c) = 2, T(0:c, c) = -2 T(0:c, 0:c) G(0:c, c)
            if (tid < c) {
                T s = T(0);
                for (int k = tid; k < c; ++k) s += Ts[k * (kPw + 1) + tid] * G[k * (kPw + 1) + c];
                Ts[c * (kPw + 1) + tid] = T(-2) * s;
            }
            if (tid == 0) Ts[c * (kPw + 1) + c] = T(2);
            __syncthreads();
        }
        T* Tg = reinterpret_cast<T*>(ws + L.off_T) + (size_t)b * L.strideT + (size_t)p * kPw * kPw;
        for (int e = tid; e < kPw * kPw; e += blockDim.x) {
            const int c = e / kPw, i = e - c * kPw;
            Tg[e] = Ts[c * (kPw + 1) + i];
        }
        T* rd = reinterpret_cast<T*>(ws + L.off_rd) + (size_t)b * L.strideRd;
        if (tid < vcols) rd[j0 + tid] = diag[tid];
    }
    for (int e = tid; e < nr * kPw; e += blockDim.x) {
        const int c = e / nr, lr = e - c * nr;
        if (j0 + c < nn) X[(size_t)(j0 + c) * mm + j0 + r0 + lr] = S[c * lds + lr];
    }
    cluster.sync();   // no CTA leaves while CTA 0 may still read its shared memory
}

}  // namespace

// rows of the tallest panel one CTA factors: its 32 columns in 200 KiB of shared memory
template <typename T>
static int qr_blocked_cta_rows()
{
    const size_t fixed = sizeof(T) * (kPw + 2 * kPw * (kPw + 1));
    const size_t ld = (200 * 1024 - fixed) / (sizeof(T) * kPw);   // largest ld with the panel in 200 KiB
    return (int)(ld % 2 ? ld : ld - 1);                          // ld = rows | 1
}

// rows of one cluster CTA's slab, the same way
template <typename T>
static int qb_cluster_slab_rows()
{
    const size_t fixed = qb_cpanel_smem<T>(1) - sizeof(T) * kPw;   // everything but S
    const size_t ld = (200 * 1024 - fixed) / (sizeof(T) * kPw);
    return (int)(ld % 2 ? ld : ld - 1);
}

// the tallest matrix the blocked QR factors: a cluster of 8 slabs
template <typename T>
int qr_blocked_max_rows()
{
    return kClusterMax * qb_cluster_slab_rows<T>();
}

// panels of every matrix: one CTA per panel when a 32-column panel of max_m rows fits in its shared
// memory, else a cluster of ceil(max_m / rows_per_cta) CTAs (at most 8)
template <typename T>
static int qb_launch_panel(int p, int batch, int max_m, unsigned char* ws, const QbLayout& L, const QbInts& I,
                           cudaStream_t st)
{
    const int one = qr_blocked_cta_rows<T>();
    if (max_m <= one) {
        const int ldp = (max_m > kPw ? max_m : kPw) | 1;
        const size_t panel_smem = sizeof(T) * ((size_t)ldp * kPw + kPw + 2 * kPw * (kPw + 1));
        if (panel_smem > 48 * 1024 &&
            cudaFuncSetAttribute(qb_panel_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)panel_smem) !=
                cudaSuccess)
            return BSVD_ERR_CUDA;
        qb_panel_kernel<T><<<batch, 256, panel_smem, st>>>(p, ws, L, I);
        return cudaGetLastError() == cudaSuccess ? BSVD_SUCCESS : BSVD_ERR_CUDA;
    }
    const int per = qb_cluster_slab_rows<T>();
    const int cs = (max_m + per - 1) / per;
    if (cs > kClusterMax) return BSVD_ERR_UNSUPPORTED;
    const int slab = (max_m + cs - 1) / cs;
    const size_t smem = qb_cpanel_smem<T>(slab > kPw ? slab : kPw);
    if (cudaFuncSetAttribute(qb_panel_cluster_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return BSVD_ERR_CUDA;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(batch * cs));
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, qb_panel_cluster_kernel<T>, p, cs, ws, L, I) != cudaSuccess) return BSVD_ERR_CUDA;
    return cudaGetLastError() == cudaSuccess ? BSVD_SUCCESS : BSVD_ERR_CUDA;
}

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
    if (mm > qr_blocked_max_rows<T>()) return BSVD_ERR_UNSUPPORTED;
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
    constexpr size_t apply_smem = qb_apply_smem<T>();
    if (apply_smem > 48 * 1024 &&
        cudaFuncSetAttribute(qb_apply_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)apply_smem) !=
            cudaSuccess)
        return BSVD_ERR_CUDA;
    const int P = (nn + kPw - 1) / kPw;
    const int tiles = P;   // 32-column tiles of nn
    for (int p = 0; p < P; ++p) {
        const int rc = qb_launch_panel<T>(p, batch, mm, ws, L, I, st);
        if (rc != BSVD_SUCCESS) return rc;
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
    constexpr size_t apply_smem = qb_apply_smem<T>();
    if (apply_smem > 48 * 1024 &&
        cudaFuncSetAttribute(qb_apply_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)apply_smem) !=
            cudaSuccess)
        return BSVD_ERR_CUDA;
    const int P = (max_n + kPw - 1) / kPw;
    for (int p = 0; p < P; ++p) {
        const int rc = qb_launch_panel<T>(p, batch, max_m, ws, L, I, st);
        if (rc != BSVD_SUCCESS) return rc;
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
