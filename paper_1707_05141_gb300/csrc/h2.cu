// h2.cu -- truncation of an H^2 nested row basis on the GPU (Section 8.2: the compression phase of
// the paper's hierarchical-matrix application, one level of the tree at a time).
//
// Input: a binary basis tree of depth d -- explicit leaf bases U_i (m_i x k) and, for every
// non-root node c, a transfer matrix E_c (k x k) with U_p = diag(U_{2p}, U_{2p+1}) [E_{2p}; E_{2p+1}].
// Nodes are numbered in heap order: node i of level l is g = 2^l - 1 + i.
//   leaves  one batched Jacobi SVD of all leaves, U_i = Q S W^T; the rank k~ is the smallest whose
//           discarded tail sqrt(sum_{j >= k~} s_j^2) is within eps ||U_i||_F; U~_i = Q(:, 0:k~) and the
//           projection T_i = U~_i^T U_i = S~ W~^T;
//   level   for l = d, ..., 1, every parent p at level l - 1 (children c1 = 2p, c2 = 2p + 1):
//           TE_p = [T_{c1} E_{c1}; T_{c2} E_{c2}] ((k~_{c1} + k~_{c2}) x k), one batched Jacobi SVD
//           of all TE_p of the level, truncated as above; E~_{c1}, E~_{c2} are the first k~_{c1}
//           and the next k~_{c2} rows of Q~, and T_p = S~ W~^T.
// The SVDs are the library's register tier (shared tier where the register tier does not fit);
// the products, truncations and copies are small kernels, one CTA per node.
#include <cuda_runtime.h>

#include "common.cuh"
#include "launch.cuh"

namespace bsvd {

namespace {

struct H2Layout {
    size_t off_ptr, off_int, off_leafQ, off_leafS, off_leafW, off_te, off_q, off_s, off_w, total;
    size_t leafQ, kS, kW, te;   // elements per node
};

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

template <typename T>
H2Layout h2_layout(int depth, int k, int max_leaf_m)
{
    H2Layout L;
    const size_t nl = (size_t)1 << depth, nin = nl - 1, nodes = 2 * nl - 1;
    const size_t mk = (size_t)(max_leaf_m > k ? max_leaf_m : k);
    L.leafQ = mk * k;
    L.kS = (size_t)k;
    L.kW = (size_t)k * k;
    L.te = (size_t)2 * k * k;
    size_t o = 0;
    L.off_ptr = o;
    o = al256(o + sizeof(void*) * nodes * 4);  // A, U, S, V pointers of every node's SVD
    L.off_int = o;
    o = al256(o + sizeof(int) * nodes * 5);    // rows, cols, ld of A, ld of U, ld of V
    L.off_leafQ = o;
    o = al256(o + sizeof(T) * L.leafQ * nl);
    L.off_leafS = o;
    o = al256(o + sizeof(T) * L.kS * nl);
    L.off_leafW = o;
    o = al256(o + sizeof(T) * L.kW * nl);
    L.off_te = o;
    o = al256(o + sizeof(T) * L.te * (nin > 0 ? nin : 1));
    L.off_q = o;
    o = al256(o + sizeof(T) * L.te * (nin > 0 ? nin : 1));
    L.off_s = o;
    o = al256(o + sizeof(T) * L.kS * (nin > 0 ? nin : 1));
    L.off_w = o;
    o = al256(o + sizeof(T) * L.kW * (nin > 0 ? nin : 1));
    L.total = o;
    return L;
}

template <typename T>
struct H2Arrays {
    T **A, **U, **S, **V;            // per node (heap order): the SVD's operands
    int *rows, *cols, *lda, *ldu, *ldv;
};

template <typename T>
H2Arrays<T> h2_arrays(unsigned char* ws, const H2Layout& L, int nodes)
{
    H2Arrays<T> a;
    T** p = reinterpret_cast<T**>(ws + L.off_ptr);
    a.A = p;
    a.U = p + nodes;
    a.S = p + 2 * (size_t)nodes;
    a.V = p + 3 * (size_t)nodes;
    int* q = reinterpret_cast<int*>(ws + L.off_int);
    a.rows = q;
    a.cols = q + nodes;
    a.lda = q + 2 * (size_t)nodes;
    a.ldu = q + 3 * (size_t)nodes;
    a.ldv = q + 4 * (size_t)nodes;
    return a;
}

// setup: the SVD operands of every node (leaves: the caller's bases; inner nodes: TE in the workspace)
template <typename T>
__global__ void h2_setup_kernel(int depth, int k, int max_leaf_m, T* const* leaf, const int* leaf_m,
                                const int* leaf_ld, unsigned char* ws, H2Layout L, H2Arrays<T> a, int* info)
{
    const int nl = 1 << depth, nodes = 2 * nl - 1;
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nodes) return;
    if (g >= nl - 1) {   // leaf i = g - (2^d - 1)
        const int i = g - (nl - 1);
        const int m = leaf_m[i], ld = leaf_ld[i];
        const bool bad = m < 0 || m > max_leaf_m || ld < (m > 1 ? m : 1);
        a.A[g] = leaf[i];
        a.rows[g] = bad ? -1 : m;   // a negative size: the SVD flags the leaf, its rank is 0
        a.cols[g] = k;
        a.lda[g] = ld > 1 ? ld : 1;
        const int mm = m > k ? m : k;
        a.U[g] = reinterpret_cast<T*>(ws + L.off_leafQ) + (size_t)i * L.leafQ;
        a.ldu[g] = mm > 1 ? mm : 1;
        a.S[g] = reinterpret_cast<T*>(ws + L.off_leafS) + (size_t)i * L.kS;
        a.V[g] = reinterpret_cast<T*>(ws + L.off_leafW) + (size_t)i * L.kW;
        a.ldv[g] = k > 1 ? k : 1;
        info[g] = bad ? BSVD_INFO_BAD_SHAPE : 0;
    } else {             // inner node: TE_g (rows set per level), 2k x k buffers
        a.A[g] = reinterpret_cast<T*>(ws + L.off_te) + (size_t)g * L.te;
        a.rows[g] = 0;
        a.cols[g] = k;
        a.lda[g] = 2 * k;
        a.U[g] = reinterpret_cast<T*>(ws + L.off_q) + (size_t)g * L.te;
        a.ldu[g] = 2 * k;
        a.S[g] = reinterpret_cast<T*>(ws + L.off_s) + (size_t)g * L.kS;
        a.V[g] = reinterpret_cast<T*>(ws + L.off_w) + (size_t)g * L.kW;
        a.ldv[g] = k > 1 ? k : 1;
        info[g] = 0;
    }
}

// truncation rank of a node: the smallest r with sum_{j >= r} s_j^2 <= eps^2 sum_j s_j^2 (FP64 sums)
template <typename T>
__device__ __forceinline__ int h2_rank(const T* s, int n, double eps)
{
    double tot = 0.0;
    for (int j = 0; j < n; ++j) tot += (double)s[j] * (double)s[j];
    const double thr = eps * eps * tot;
    double tail = 0.0;
    int r = n;
    for (int j = n - 1; j >= 0; --j) {
        const double t2 = tail + (double)s[j] * (double)s[j];
        if (t2 > thr) break;
        tail = t2;
        r = j;
    }
    return r;
}

// finish of the nodes g0 .. g0 + cnt - 1 after their SVD: rank, T = S~ W~^T (k~ x k, ld k), and
// the truncated left factor -- the new leaf (leaves) or the children's new transfers (inner nodes)
template <typename T>
__global__ void __launch_bounds__(256) h2_finish_kernel(int g0, int depth, int k, double eps, H2Arrays<T> a,
                                                        T* const* new_leaf, const int* new_leaf_ld,
                                                        T* const* new_transfer, T* const* Tout, int* rank,
                                                        int* info)
{
    __shared__ int kt;
    const int g = g0 + blockIdx.x;
    const int nl = 1 << depth;
    const bool leaf = g >= nl - 1;
    if (info[g] == BSVD_INFO_BAD_SHAPE || info[g] == BSVD_INFO_NONFINITE) {
        if (threadIdx.x == 0) rank[g] = 0;
        return;
    }
    const int rows = a.rows[g] > 0 ? a.rows[g] : 0, cols = a.cols[g];
    const int kmin = rows < cols ? rows : cols;
    const T* S = a.S[g];
    if (threadIdx.x == 0) {
        kt = h2_rank(S, kmin, eps);
        rank[g] = kt;
    }
    __syncthreads();
    const int r = kt;
    // T = S~ W~^T: T(i, c) = s_i W(c, i), k~ x k, ld k
    const T* W = a.V[g];
    const int ldw = a.ldv[g];
    T* t = Tout[g];
    for (int e = threadIdx.x; e < r * k; e += blockDim.x) {
        const int c = e / r, i = e - c * r;
        t[(size_t)c * k + i] = c < cols ? S[i] * W[(size_t)i * ldw + c] : T(0);
    }
    const T* Q = a.U[g];
    const int ldq = a.ldu[g];
    if (leaf) {
        const int li = g - (nl - 1);
        T* u = new_leaf[li];
        const int ldn = new_leaf_ld[li];
        for (int e = threadIdx.x; e < r * rows; e += blockDim.x) {
            const int c = e / rows, i = e - c * rows;
            u[(size_t)c * ldn + i] = Q[(size_t)c * ldq + i];
        }
    } else {
        // children c1 = 2g + 1, c2 = 2g + 2 (heap order); their ranks split Q~'s rows
        const int c1 = 2 * g + 1, c2 = 2 * g + 2;
        const int r1 = rank[c1], r2 = rank[c2];
        T* e1 = new_transfer[c1];
        T* e2 = new_transfer[c2];
        for (int e = threadIdx.x; e < r * (r1 + r2); e += blockDim.x) {
            const int c = e / (r1 + r2), i = e - c * (r1 + r2);
            const T v = Q[(size_t)c * ldq + i];
            if (i < r1) e1[(size_t)c * k + i] = v;
            else e2[(size_t)c * k + (i - r1)] = v;
        }
    }
}

// TE_p = [T_{c1} E_{c1}; T_{c2} E_{c2}] for the parents g0 .. g0 + cnt - 1 (one CTA each)
template <typename T>
__global__ void __launch_bounds__(256) h2_te_kernel(int g0, int k, T* const* E, T* const* Tout, const int* rank,
                                                    H2Arrays<T> a, int* info)
{
    extern __shared__ __align__(16) unsigned char h2_sm[];
    T* Es = reinterpret_cast<T*>(h2_sm);              // E_c, k x (k + 1)
    T* Ts = Es + (size_t)k * (k + 1);                 // T_c, k x (k + 1)
    const int g = g0 + blockIdx.x;
    const int c1 = 2 * g + 1, c2 = 2 * g + 2;
    const int r1 = rank[c1], r2 = rank[c2];
    T* te = a.A[g];
    const int ld = a.lda[g];
    if (threadIdx.x == 0) a.rows[g] = r1 + r2;   // a flagged child has rank 0
    for (int h = 0; h < 2; ++h) {
        const int c = h ? c2 : c1, r = h ? r2 : r1, off = h ? r1 : 0;
        __syncthreads();
        const T* e = E[c];
        const T* t = Tout[c];
        for (int x = threadIdx.x; x < k * k; x += blockDim.x) {
            const int col = x / k, row = x - col * k;
            Es[row * (k + 1) + col] = e[(size_t)col * k + row];   // E(row, col), ld k
            Ts[row * (k + 1) + col] = row < r ? t[(size_t)col * k + row] : T(0);
        }
        __syncthreads();
        for (int x = threadIdx.x; x < r * k; x += blockDim.x) {
            const int col = x / r, row = x - col * r;
            T s = T(0);
            for (int j = 0; j < k; ++j) s = fma(Ts[row * (k + 1) + j], Es[j * (k + 1) + col], s);
            te[(size_t)col * ld + off + row] = s;
        }
    }
}

// batched SVD of the nodes g0 .. g0 + cnt - 1: the register tier, or the shared tier where the
// register tier does not hold the bounds
template <typename T>
int h2_svd(int g0, int cnt, int max_rows, int k, const H2Arrays<T>& a, int* info, long long* rot, cudaStream_t st)
{
    void* const* A = (void* const*)(a.A + g0);
    void* const* U = (void* const*)(a.U + g0);
    void* const* S = (void* const*)(a.S + g0);
    void* const* V = (void* const*)(a.V + g0);
    long long* r = rot ? rot + g0 : nullptr;
    int rc = launch_jacobi_reg<T>(cnt, max_rows, k, 0, A, a.rows + g0, a.cols + g0, a.lda + g0, S, U, a.ldu + g0, V,
                                  a.ldv + g0, 0.0, 0, info + g0, r, st);
    if (rc == BSVD_ERR_UNSUPPORTED)
        rc = launch_jacobi_smem<T>(cnt, max_rows, k, A, a.rows + g0, a.cols + g0, a.lda + g0, S, U, a.ldu + g0, V,
                                   a.ldv + g0, 0.0, 0, info + g0, r, st);
    return rc;
}

}  // namespace

template <typename T>
size_t h2_truncate_workspace(int depth, int k, int max_leaf_m)
{
    return h2_layout<T>(depth, k, max_leaf_m).total;
}

template <typename T>
int launch_h2_truncate(int depth, int k, int max_leaf_m, void* const* leaf, const int* leaf_m, const int* leaf_ld,
                       void* const* transfer, double eps, void* const* new_leaf, const int* new_leaf_ld,
                       void* const* new_transfer, void* const* Tout, int* rank, int* info, long long* rot,
                       void* ws_v, size_t ws_bytes, cudaStream_t st)
{
    const H2Layout L = h2_layout<T>(depth, k, max_leaf_m);
    if (ws_bytes < L.total) return BSVD_ERR_WORKSPACE;
    unsigned char* ws = static_cast<unsigned char*>(ws_v);
    const int nl = 1 << depth, nodes = 2 * nl - 1;
    H2Arrays<T> a = h2_arrays<T>(ws, L, nodes);
    h2_setup_kernel<T><<<(nodes + 127) / 128, 128, 0, st>>>(depth, k, max_leaf_m, (T* const*)leaf, leaf_m, leaf_ld,
                                                            ws, L, a, info);
    if (cudaGetLastError() != cudaSuccess) return BSVD_ERR_CUDA;
    // leaves
    int rc = h2_svd<T>(nl - 1, nl, max_leaf_m, k, a, info, rot, st);
    if (rc) return rc;
    h2_finish_kernel<T><<<nl, 256, 0, st>>>(nl - 1, depth, k, eps, a, (T* const*)new_leaf, new_leaf_ld,
                                            (T* const*)new_transfer, (T* const*)Tout, rank, info);
    if (cudaGetLastError() != cudaSuccess) return BSVD_ERR_CUDA;
    const size_t te_smem = 2 * sizeof(T) * (size_t)k * (k + 1);
    if (te_smem > 48 * 1024 &&
        cudaFuncSetAttribute(h2_te_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)te_smem) !=
            cudaSuccess)
        return BSVD_ERR_CUDA;
    // levels d-1 .. 0: the parents of level l + 1
    for (int l = depth - 1; l >= 0; --l) {
        const int g0 = (1 << l) - 1, cnt = 1 << l;
        h2_te_kernel<T><<<cnt, 256, te_smem, st>>>(g0, k, (T* const*)transfer, (T* const*)Tout, rank, a, info);
        if (cudaGetLastError() != cudaSuccess) return BSVD_ERR_CUDA;
        rc = h2_svd<T>(g0, cnt, 2 * k, k, a, info, rot, st);
        if (rc) return rc;
        h2_finish_kernel<T><<<cnt, 256, 0, st>>>(g0, depth, k, eps, a, (T* const*)new_leaf, new_leaf_ld,
                                                 (T* const*)new_transfer, (T* const*)Tout, rank, info);
        if (cudaGetLastError() != cudaSuccess) return BSVD_ERR_CUDA;
    }
    return BSVD_SUCCESS;
}

template size_t h2_truncate_workspace<float>(int, int, int);
template size_t h2_truncate_workspace<double>(int, int, int);
template int launch_h2_truncate<float>(int, int, int, void* const*, const int*, const int*, void* const*, double,
                                       void* const*, const int*, void* const*, void* const*, int*, int*, long long*,
                                       void*, size_t, cudaStream_t);
template int launch_h2_truncate<double>(int, int, int, void* const*, const int*, const int*, void* const*, double,
                                        void* const*, const int*, void* const*, void* const*, int*, int*, long long*,
                                        void*, size_t, cudaStream_t);

}  // namespace bsvd
