// block_jacobi.cu -- batched one-sided block Jacobi SVD for matrices that live in global memory
// (Algorithm 3, Section 6).
//
// The working matrix W (A, or A^T when m < n, copied into the caller's U or V output) is split into
// nb column blocks of width bw.  A sweep visits every block pair once in round-robin order (nb - 1
// steps of nb/2 disjoint pairs, Section 5's ordering applied to blocks); a matrix with fewer
// blocks than the batch's largest runs its own steps and idles in the rest.  Every step runs
// batched stages over the pairs of the matrices not yet converged (device item lists: the GRAM
// test lists the pairs that rotate, and only those reach the later stages):
//   GRAM   : G = [W_i W_j]^T [W_i W_j] (2bw x 2bw) -- on the tensor cores for FP32 with bw = 32
//            (TF32 operands split in a high and a low part, FP32 accumulation in tensor memory),
//            by FP32 dot products otherwise -- then e_l = the largest |G_pq| / sqrt(G_pp G_qq),
//            evaluated in FP64 (the paper's scaledOffdiag, Section 6.1).  A pair with e_l <= tol
//            is already orthogonal and is skipped by the next stages.
//   DIRECT : [W_i W_j] = Q R by the batched Householder QR, and R goes to the inner SVD instead of
//            G (Section 6.2): robust for ill-conditioned blocks, where G loses the small singular
//            values (Section 6.3).
//   inner  : one-sided Jacobi of the 2bw x 2bw G (or R) with the register-tier kernel, which
//            returns the rotation X (GRAM: the QR-preconditioned variant's U = Q V_w, the
//            eigenvectors of G; DIRECT: the right singular vectors of R).
//   polish : one Newton-Schulz step makes X orthogonal to rounding level (see bj_polish_kernel).
//   update : [W_i W_j] <- [W_i W_j] X (GRAM) or <- Q U_R diag(S_R) (DIRECT), and
//            [V_i V_j] <- [V_i V_j] X, in FP32 on 128-row tiles staged in shared memory.
// A matrix whose sweep rotated nothing is converged (the paper's "final sweep performs no
// rotations"); it leaves the lists.  Finally sigma_j = ||w_j||, U = W / sigma and the columns of
// U and V are sorted by descending sigma in place (cycle-following permutation).
#include <cuda_runtime.h>

#include <cstddef>

#include "common.cuh"
#include "launch.cuh"
#include "tcgen05.cuh"

namespace bsvd {

// ------------------------------------------------------------------------------------------------
// workspace layout (all offsets 256-byte aligned)
// ------------------------------------------------------------------------------------------------
struct BjLayout {
    int batch, npairs, bw, mm_max;
    size_t n_items;                   // batch * npairs
    size_t off_G, off_X, off_S, off_UR, off_P;           // per-item matrices
    size_t off_pG, off_pX, off_pS, off_pUR, off_pP;      // pointer arrays (item order)
    size_t off_m, off_n, off_ld, off_ldp, off_info;      // int arrays per item
    size_t off_state;                                    // per-matrix state
    size_t off_mlist, off_plist;                         // live matrices, rotating pair items
    size_t off_ctr;                                      // BjCounters
    size_t off_ver, off_pv;                              // block versions, pair test records
    size_t npv;                                          // pair records per matrix
    int retest;                                          // 1: re-test every pair every sweep
    size_t total;
};

// claim counters of the persistent stage kernels and the lengths of the two live lists
struct BjCounters {
    unsigned long long claim[8];  // gram, pack, polish, update, QR, inner SVD
    int pcount;                   // rotating pairs of the current step (plist)
    int mcount;                   // matrices not yet converged (mlist)
    int timeouts;                 // tensor-core completion waits that gave up (0 in a valid run)
    int pad;
};
constexpr size_t kStepCounterBytes = offsetof(BjCounters, mcount);  // claims + pcount: zeroed every step

struct BjState {
    int mm, nn, nblk, converged;
    int sweeps, rot_sweep, pad0, pad1;
    long long rotations;
    double emax;
};

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Pair selection by the recorded tests.  Every block carries a version, bumped when a rotating pair
// that contains it is decided (its update follows in the same step, and no other pair of the step
// touches it).  A pair whose test found it orthogonal records the two versions; while neither block
// changes its Gram matrix -- and so its test -- would come out the same, so the pair is not formed
// or tested again.  The choice is exact: results equal those of re-testing every pair.
struct BjPairRecord {
    int* ver;       // the two blocks' versions
    unsigned* rec;  // the pair's record: (version i << 16) | version j when found orthogonal, else ~0
    unsigned key;   // the current versions, packed the same way
};

__device__ __forceinline__ BjPairRecord bj_pair_record(unsigned char* ws, const BjLayout& L, int b, int bi, int bj)
{
    const int nbp = 2 * L.npairs;
    int* ver = reinterpret_cast<int*>(ws + L.off_ver) + (size_t)b * nbp;
    unsigned* rec = nullptr;   // (no pair: bi == bj when the item is not live)
    if (bi < bj) {
        const size_t idx = (size_t)bi * nbp - (size_t)bi * (bi + 1) / 2 + (size_t)(bj - bi - 1);
        rec = reinterpret_cast<unsigned*>(ws + L.off_pv) + (size_t)b * L.npv + idx;
    }
    return BjPairRecord{ver, rec, ((unsigned)ver[bi] << 16) | ((unsigned)ver[bj] & 0xffffu)};
}

template <typename T>
static BjLayout bj_layout(int batch, int max_m, int max_n, int bw, bool direct)
{
    BjLayout L;
    const int mm = max_m > max_n ? max_m : max_n;
    const int nn = max_m > max_n ? max_n : max_m;
    int nblk = (nn + bw - 1) / bw;
    if (nblk < 2) nblk = 2;
    nblk += nblk & 1;
    L.batch = batch;
    L.npairs = nblk / 2;
    L.bw = bw;
    L.mm_max = mm > 2 * bw ? mm : 2 * bw;  // rows of a packed pair (zero-padded to at least 2bw)
    L.n_items = (size_t)batch * L.npairs;
    const size_t k2 = (size_t)(2 * bw) * (2 * bw);
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = align256(o + bytes);
        return at;
    };
    L.off_G = take(L.n_items * k2 * sizeof(T));
    L.off_X = take(L.n_items * k2 * sizeof(T));
    L.off_S = take(L.n_items * 2 * bw * sizeof(T));
    L.off_UR = take(direct ? L.n_items * k2 * sizeof(T) : 0);
    L.off_P = take(direct ? L.n_items * (size_t)(mm > 2 * bw ? mm : 2 * bw) * 2 * bw * sizeof(T) : 0);
    L.off_pG = take(L.n_items * sizeof(void*));
    L.off_pX = take(L.n_items * sizeof(void*));
    L.off_pS = take(L.n_items * sizeof(void*));
    L.off_pUR = take(L.n_items * sizeof(void*));
    L.off_pP = take(L.n_items * sizeof(void*));
    L.off_m = take(L.n_items * sizeof(int));
    L.off_n = take(L.n_items * sizeof(int));
    L.off_ld = take(L.n_items * sizeof(int));
    L.off_ldp = take(L.n_items * sizeof(int));
    L.off_info = take(L.n_items * sizeof(int));
    L.off_state = take((size_t)batch * sizeof(BjState));
    L.off_mlist = take((size_t)batch * sizeof(int));
    L.off_plist = take(L.n_items * sizeof(int));
    L.off_ctr = take(sizeof(BjCounters));
    L.npv = (size_t)(2 * L.npairs) * (2 * L.npairs - 1) / 2;
    L.off_ver = take((size_t)batch * 2 * L.npairs * sizeof(int));
    L.off_pv = take((size_t)batch * L.npv * sizeof(unsigned));
    L.retest = 0;
    L.total = o;
    return L;
}

// ------------------------------------------------------------------------------------------------
// setup: working copy, V = I, per-item pointer arrays
// ------------------------------------------------------------------------------------------------
template <typename T>
__global__ void bj_setup_kernel(int batch, int max_mm, int max_nn, int bw, int npairs, T* const* A, const int* M,
                                const int* N, const int* LDA, T* const* U, const int* LDU, T* const* V,
                                const int* LDV, unsigned char* ws, BjLayout L, int* info)
{
    const int b = blockIdx.x;
    if (b >= batch) return;
    BjState* st = reinterpret_cast<BjState*>(ws + L.off_state) + b;
    const int m = M[b], n = N[b], lda = LDA[b];
    const bool tr = m < n;
    const int mm = tr ? n : m, nn = tr ? m : n;
    const int ldu = LDU[b], ldv = LDV[b];
    const bool bad = m < 0 || n < 0 || mm > max_mm || nn > max_nn || lda < (m > 1 ? m : 1) ||
                     ldu < (m > 1 ? m : 1) || ldv < (n > 1 ? n : 1);
    T* Wk = tr ? V[b] : U[b];  // working matrix mm x nn
    const int ldw = tr ? ldv : ldu;
    T* Vk = tr ? U[b] : V[b];  // accumulated rotations nn x nn
    const int ldvk = tr ? ldu : ldv;
    if (threadIdx.x == 0) {
        st->mm = bad ? 0 : mm;
        st->nn = bad ? 0 : nn;
        st->nblk = (nn + bw - 1) / bw;
        st->converged = (bad || nn == 0) ? 1 : 0;
        st->sweeps = 0;
        st->rot_sweep = 0;
        st->rotations = 0;
        st->emax = 0.0;
        info[b] = bad ? BSVD_INFO_BAD_SHAPE : 0;
        if (!st->converged) {
            BjCounters* C = reinterpret_cast<BjCounters*>(ws + L.off_ctr);
            reinterpret_cast<int*>(ws + L.off_mlist)[atomicAdd(&C->mcount, 1)] = b;
        }
    }
    // per-item pointers into the workspace
    for (int k = threadIdx.x; k < npairs; k += blockDim.x) {
        const size_t it = (size_t)b * npairs + k;
        const size_t k2 = (size_t)(2 * bw) * (2 * bw);
        T* G = reinterpret_cast<T*>(ws + L.off_G) + it * k2;
        T* X = reinterpret_cast<T*>(ws + L.off_X) + it * k2;
        T* S = reinterpret_cast<T*>(ws + L.off_S) + it * 2 * bw;
        T* UR = reinterpret_cast<T*>(ws + L.off_UR) + it * k2;
        T* P = reinterpret_cast<T*>(ws + L.off_P) + it * (size_t)L.mm_max * 2 * bw;
        reinterpret_cast<T**>(ws + L.off_pG)[it] = G;
        reinterpret_cast<T**>(ws + L.off_pX)[it] = X;
        reinterpret_cast<T**>(ws + L.off_pS)[it] = S;
        reinterpret_cast<T**>(ws + L.off_pUR)[it] = UR;
        reinterpret_cast<T**>(ws + L.off_pP)[it] = P;
        reinterpret_cast<int*>(ws + L.off_m)[it] = 0;
        reinterpret_cast<int*>(ws + L.off_n)[it] = 0;
        reinterpret_cast<int*>(ws + L.off_ld)[it] = 2 * bw;
        reinterpret_cast<int*>(ws + L.off_ldp)[it] = mm > 1 ? mm : 1;
    }
    {
        int* ver = reinterpret_cast<int*>(ws + L.off_ver) + (size_t)b * 2 * npairs;
        unsigned* rec = reinterpret_cast<unsigned*>(ws + L.off_pv) + (size_t)b * L.npv;
        for (int k = threadIdx.x; k < 2 * npairs; k += blockDim.x) ver[k] = 0;
        for (size_t k = threadIdx.x; k < L.npv; k += blockDim.x) rec[k] = ~0u;
    }
    if (bad) return;
    const T* a = A[b];
    for (size_t e = threadIdx.x; e < (size_t)mm * nn; e += blockDim.x) {
        const int j = (int)(e / mm), i = (int)(e - (size_t)j * mm);
        Wk[(size_t)j * ldw + i] = tr ? a[(size_t)i * lda + j] : a[(size_t)j * lda + i];
    }
    for (size_t e = threadIdx.x; e < (size_t)nn * nn; e += blockDim.x) {
        const int j = (int)(e / nn), i = (int)(e - (size_t)j * nn);
        Vk[(size_t)j * ldvk + i] = i == j ? T(1) : T(0);
    }
}

// column block (blk, column offset c in [0, 2bw)) -> global column, or -1 when past nn
__device__ __forceinline__ int bj_col(int bi, int bj, int bw, int c, int nn)
{
    const int blk = c < bw ? bi : bj;
    const int col = blk * bw + (c < bw ? c : c - bw);
    return col < nn ? col : -1;
}

// ------------------------------------------------------------------------------------------------
// GRAM stage: G = A_ij^T A_ij with FP32 dot products; FP64 scaled off-diagonal test
// ------------------------------------------------------------------------------------------------
template <typename T, int K2>  // K2 = 2 bw
__device__ __forceinline__ void bj_gram_item(int it, int batch, int npairs, int step, int bw, T* const* U,
                                             const int* LDU, T* const* V, const int* LDV, const int* M,
                                             const int* N, unsigned char* ws, const BjLayout& L, double tol)
{
    constexpr int RC = 32;                 // rows per staged chunk
    constexpr int TPO = (K2 * K2) / 256;   // outputs per thread
    __shared__ T xs[K2][RC + 1];
    __shared__ T gd[K2];
    __shared__ double red[8];
    const int b = it / npairs, k = it - b * npairs;
    BjState* st = reinterpret_cast<BjState*>(ws + L.off_state) + b;
    int* im = reinterpret_cast<int*>(ws + L.off_m);
    int* in = reinterpret_cast<int*>(ws + L.off_n);
    const int mm = st->mm, nn = st->nn, nblk = st->nblk;
    const int nbp = nblk + (nblk & 1);
    int bi = 0, bj = 0;
    if (k < nbp / 2 && step < nbp - 1) round_robin_pair(nbp, step, k, bi, bj);
    // pairs with the virtual block (odd nb) are skipped, except for a single block, which is
    // orthogonalised internally through its pair with the empty block; a matrix with fewer blocks
    // than the batch's largest runs its own nbp - 1 steps of each sweep and idles in the rest
    const bool live = !st->converged && step < nbp - 1 && k < nbp / 2 && (bj < nblk || nblk == 1) && bi * bw < nn;
    const BjPairRecord pr = bj_pair_record(ws, L, b, bi, bj);
    if (!live || (!L.retest && pr.rec && *pr.rec == pr.key)) {   // no pair, or unchanged since found orthogonal
        if (threadIdx.x == 0) im[it] = in[it] = 0;
        return;
    }
    const bool tr = M[b] < N[b];
    const T* W = tr ? V[b] : U[b];
    const int ldw = tr ? LDV[b] : LDU[b];
    T* G = reinterpret_cast<T* const*>(ws + L.off_pG)[it];
    const int tid = threadIdx.x;
    // thread tile: TPO consecutive outputs of one column block
    const int o0 = tid * TPO;
    const int gc = o0 / K2, gr0 = o0 % K2;  // output column gc, rows gr0 .. gr0 + TPO - 1
    T acc[TPO];
#pragma unroll
    for (int q = 0; q < TPO; ++q) acc[q] = T(0);
    for (int r0 = 0; r0 < mm; r0 += RC) {
        // the thread's loads of the chunk in flight together, then its shared stores
        constexpr int PL = (K2 * RC) / 256;
        T xl[PL];
#pragma unroll
        for (int q = 0; q < PL; ++q) {
            const int e = tid + 256 * q;
            const int c = e / RC, r = e % RC;
            const int col = bj_col(bi, bj, bw, c, nn);
            xl[q] = (col >= 0 && r0 + r < mm) ? W[(size_t)col * ldw + r0 + r] : T(0);
        }
#pragma unroll
        for (int q = 0; q < PL; ++q) {
            const int e = tid + 256 * q;
            xs[e / RC][e % RC] = xl[q];
        }
        __syncthreads();
#pragma unroll 4
        for (int r = 0; r < RC; ++r) {
            const T y = xs[gc][r];
#pragma unroll
            for (int q = 0; q < TPO; ++q) acc[q] = fma(xs[gr0 + q][r], y, acc[q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < TPO; ++q) G[(size_t)gc * K2 + gr0 + q] = acc[q];
    if (gr0 <= gc && gc < gr0 + TPO) gd[gc] = acc[gc - gr0];
    __syncthreads();
    // e_l = max |G_pq| / sqrt(G_pp G_qq), FP64
    double e = 0.0;
#pragma unroll
    for (int q = 0; q < TPO; ++q) {
        const int r = gr0 + q;
        if (r == gc) continue;
        const double dp = (double)gd[r], dq = (double)gd[gc];
        if (dp > 0.0 && dq > 0.0) {
            const double v = fabs((double)acc[q]) / sqrt(dp * dq);
            e = v > e ? v : e;
        }
    }
    for (int o = 16; o > 0; o >>= 1) e = fmax(e, __shfl_xor_sync(0xffffffffu, e, o));
    if ((tid & 31) == 0) red[tid >> 5] = e;
    __syncthreads();
    if (tid == 0) {
        double em = 0.0;
        for (int w = 0; w < 8; ++w) em = fmax(em, red[w]);
        const bool rot = em > tol;
        im[it] = rot ? K2 : 0;
        in[it] = rot ? K2 : 0;
        if (rot) {
            atomicAdd(&st->rot_sweep, 1);
            BjCounters* C = reinterpret_cast<BjCounters*>(ws + L.off_ctr);
            reinterpret_cast<int*>(ws + L.off_plist)[atomicAdd(&C->pcount, 1)] = it;
            ++pr.ver[bi];
            ++pr.ver[bj];
        } else if (pr.rec) {
            *pr.rec = pr.key;
        }
        // emax of the matrix over the sweep, as ordered bits of a non-negative double
        atomicMax(reinterpret_cast<unsigned long long*>(&st->emax), (unsigned long long)__double_as_longlong(em));
    }
}

// persistent over the pairs of the live matrices (mlist); appends the rotating pairs to plist
template <typename T, int K2>
__global__ void __launch_bounds__(256) bj_gram_kernel(int batch, int npairs, int step, int bw, T* const* U,
                                                      const int* LDU, T* const* V, const int* LDV, const int* M,
                                                      const int* N, unsigned char* ws, BjLayout L, double tol)
{
    BjCounters* C = reinterpret_cast<BjCounters*>(ws + L.off_ctr);
    const int* mlist = reinterpret_cast<const int*>(ws + L.off_mlist);
    const long long items = (long long)C->mcount * npairs;
    for (long long j = next_work(&C->claim[0]); j < items; j = next_work(&C->claim[0])) {
        const int b = mlist[j / npairs], k = (int)(j % npairs);
        bj_gram_item<T, K2>(b * npairs + k, batch, npairs, step, bw, U, LDU, V, LDV, M, N, ws, L, tol);
    }
}

// ------------------------------------------------------------------------------------------------
// DIRECT stage: pack a live pair [W_i W_j] into a contiguous buffer for its QR.  Which pairs are
// live is decided by the GRAM kernel's test, run first: FP32 dot products of the columns
// themselves and the FP64 scaled off-diagonal, the same test for both methods.
// ------------------------------------------------------------------------------------------------
template <typename T, int K2>
__device__ __forceinline__ void bj_pack_item(int it, int batch, int npairs, int step, int bw, T* const* U,
                                             const int* LDU, T* const* V, const int* LDV, const int* M,
                                             const int* N, unsigned char* ws, const BjLayout& L)
{
    const int b = it / npairs, k = it - b * npairs;
    BjState* st = reinterpret_cast<BjState*>(ws + L.off_state) + b;
    int* im = reinterpret_cast<int*>(ws + L.off_m);
    int* in = reinterpret_cast<int*>(ws + L.off_n);
    const int mm = st->mm, nn = st->nn, nblk = st->nblk;
    const int nbp = nblk + (nblk & 1);
    if (in[it] == 0) return;  // the pair test (GRAM kernel, run first) found it orthogonal
    int bi, bj;
    round_robin_pair(nbp, step, k, bi, bj);
    const bool tr = M[b] < N[b];
    const T* W = tr ? V[b] : U[b];
    const int ldw = tr ? LDV[b] : LDU[b];
    T* P = reinterpret_cast<T* const*>(ws + L.off_pP)[it];
    // rows are zero-padded to at least K2 so that the pair's QR is of a tall matrix: the padding
    // changes neither R nor the product A_ij V_R on the real rows
    const int mp = mm > K2 ? mm : K2;
    for (int c = threadIdx.x >> 5; c < K2; c += blockDim.x >> 5) {
        const int col = bj_col(bi, bj, bw, c, nn);
        for (int r = threadIdx.x & 31; r < mp; r += 32)
            P[(size_t)c * mp + r] = (col >= 0 && r < mm) ? W[(size_t)col * ldw + r] : T(0);
    }
    if (threadIdx.x == 0) {
        im[it] = mp;
        in[it] = K2;
        reinterpret_cast<int*>(ws + L.off_ldp)[it] = mp;
    }
}

template <typename T, int K2>
__global__ void __launch_bounds__(256) bj_pack_kernel(int batch, int npairs, int step, int bw, T* const* U,
                                                      const int* LDU, T* const* V, const int* LDV, const int* M,
                                                      const int* N, unsigned char* ws, BjLayout L)
{
    BjCounters* C = reinterpret_cast<BjCounters*>(ws + L.off_ctr);
    const int* plist = reinterpret_cast<const int*>(ws + L.off_plist);
    const long long items = C->pcount;
    for (long long j = next_work(&C->claim[1]); j < items; j = next_work(&C->claim[1]))
        bj_pack_item<T, K2>(plist[j], batch, npairs, step, bw, U, LDU, V, LDV, M, N, ws, L);
}

// ------------------------------------------------------------------------------------------------
// polish: one Newton-Schulz step X <- X - X (X^T X - I) / 2 towards the orthogonal polar factor.
// X (the inner SVD's accumulated rotation, a product of hundreds of plane rotations) is orthogonal
// only to ~25 u; V multiplies ~150 of them per column, so their errors would add up.  After the
// step ||X^T X - I|| is at the rounding level of one product.
// ------------------------------------------------------------------------------------------------
// BI consecutive shared-memory values at an address aligned to their size, in the widest loads
template <typename T, int BI>
__device__ __forceinline__ void ld_shared_run(const T* p, T (&v)[BI])
{
    constexpr int bytes = BI * (int)sizeof(T);
    if constexpr (bytes % 16 == 0) {
#pragma unroll
        for (int i = 0; i < bytes / 16; ++i) {
            if constexpr (sizeof(T) == 4) {
                const float4 x = reinterpret_cast<const float4*>(p)[i];
                v[4 * i] = x.x;
                v[4 * i + 1] = x.y;
                v[4 * i + 2] = x.z;
                v[4 * i + 3] = x.w;
            } else {
                const double2 x = reinterpret_cast<const double2*>(p)[i];
                v[2 * i] = x.x;
                v[2 * i + 1] = x.y;
            }
        }
    } else if constexpr (bytes == 8 && sizeof(T) == 4) {
        const float2 x = *reinterpret_cast<const float2*>(p);
        v[0] = x.x;
        v[1] = x.y;
    } else {
#pragma unroll
        for (int i = 0; i < BI; ++i) v[i] = p[i];
    }
}

// shared memory of the polish: X twice (row-major and column-major) and E, rows padded to 16 bytes
template <typename T, int K2>
constexpr size_t bj_polish_smem() { return 3 * sizeof(T) * (size_t)K2 * (K2 + 16 / sizeof(T)); }

template <typename T, int K2>
__device__ __forceinline__ void bj_polish_item(T* X, unsigned char* pol_sm)
{
    constexpr int LD = K2 + 16 / (int)sizeof(T);   // padded row (16-byte multiple)
    constexpr int BI = K2 / 16;                     // each thread: a BI x BI block of the 16 x 16 grid
    constexpr int VE = 16 / (int)sizeof(T);         // elements per 16-byte global load
    T* xr = reinterpret_cast<T*>(pol_sm);           // xr[k * LD + c] = X(k, c) (row-major)
    T* xc = xr + K2 * LD;                           // xc[k * LD + r] = X(r, k) (column-major)
    T* es = xc + K2 * LD;                           // es[k * LD + c] = E(k, c), E = X^T X - I
    const int tid = threadIdx.x;
    // X in 16-byte loads, all in flight (X is K2 x K2 column-major, contiguous, 256-byte aligned)
#pragma unroll
    for (int q = 0; q < (K2 * K2) / (VE * 256); ++q) {
        const int e = tid + 256 * q;
        const int c = e / (K2 / VE), r = (e - c * (K2 / VE)) * VE;
        T v[VE];
        if constexpr (sizeof(T) == 4) {
            const float4 x = reinterpret_cast<const float4*>(X)[e];
            v[0] = x.x;
            v[1] = x.y;
            v[2] = x.z;
            v[3] = x.w;
        } else {
            const double2 x = reinterpret_cast<const double2*>(X)[e];
            v[0] = x.x;
            v[1] = x.y;
        }
#pragma unroll
        for (int i = 0; i < VE; ++i) {
            xc[c * LD + r + i] = v[i];
            xr[(r + i) * LD + c] = v[i];
        }
    }
    __syncthreads();
    const int i0 = (tid & 15) * BI, j0 = (tid >> 4) * BI;
    T acc[BI][BI];
#pragma unroll
    for (int i = 0; i < BI; ++i)
#pragma unroll
        for (int j = 0; j < BI; ++j) acc[i][j] = T(0);
    // E(i, j) = sum_k X(k, i) X(k, j) - [i == j]
#pragma unroll 4
    for (int k = 0; k < K2; ++k) {
        T a[BI], bv[BI];
        ld_shared_run<T, BI>(xr + k * LD + i0, a);
        ld_shared_run<T, BI>(xr + k * LD + j0, bv);
#pragma unroll
        for (int i = 0; i < BI; ++i)
#pragma unroll
            for (int j = 0; j < BI; ++j) acc[i][j] = fma(a[i], bv[j], acc[i][j]);
    }
#pragma unroll
    for (int i = 0; i < BI; ++i)
#pragma unroll
        for (int j = 0; j < BI; ++j) es[(i0 + i) * LD + j0 + j] = acc[i][j] - (i0 + i == j0 + j ? T(1) : T(0));
    __syncthreads();
    // X(r, c) <- X(r, c) - 0.5 sum_k X(r, k) E(k, c), rows i0.., columns j0..
#pragma unroll
    for (int i = 0; i < BI; ++i)
#pragma unroll
        for (int j = 0; j < BI; ++j) acc[i][j] = T(0);
#pragma unroll 4
    for (int k = 0; k < K2; ++k) {
        T a[BI], ev[BI];
        ld_shared_run<T, BI>(xc + k * LD + i0, a);
        ld_shared_run<T, BI>(es + k * LD + j0, ev);
#pragma unroll
        for (int i = 0; i < BI; ++i)
#pragma unroll
            for (int j = 0; j < BI; ++j) acc[i][j] = fma(a[i], ev[j], acc[i][j]);
    }
#pragma unroll
    for (int j = 0; j < BI; ++j)
#pragma unroll
        for (int i = 0; i < BI; ++i)
            X[(size_t)(j0 + j) * K2 + i0 + i] = xc[(j0 + j) * LD + i0 + i] - T(0.5) * acc[i][j];
    __syncthreads();  // the shared buffers are reused by the next item
}

// GRAM polishes the rotation X; DIRECT polishes both factors of R's SVD: V_R (the rotation of V)
// and U_R (W <- Q U_R S_R), since W's columns are only as orthogonal as Q U_R
template <typename T, int K2>
__global__ void __launch_bounds__(256) bj_polish_kernel(unsigned char* ws, BjLayout L, int direct)
{
    extern __shared__ __align__(16) unsigned char pol_sm[];
    BjCounters* C = reinterpret_cast<BjCounters*>(ws + L.off_ctr);
    const int* plist = reinterpret_cast<const int*>(ws + L.off_plist);
    const int* in = reinterpret_cast<const int*>(ws + L.off_n);
    const long long items = C->pcount;
    for (long long j = next_work(&C->claim[2]); j < items; j = next_work(&C->claim[2])) {
        const int it = plist[j];
        if (in[it] == 0) continue;
        bj_polish_item<T, K2>(reinterpret_cast<T* const*>(ws + L.off_pX)[it], pol_sm);
        if (direct) bj_polish_item<T, K2>(reinterpret_cast<T* const*>(ws + L.off_pUR)[it], pol_sm);
    }
}

// ------------------------------------------------------------------------------------------------
// update stage: dst rows <- src rows (r x 2bw) * X (2bw x 2bw) [* diag(S)]
//   GRAM  : src = dst = [W_i W_j] (in place, row tiles), X = accumulated rotation of G
//   DIRECT: src = Q (packed), X = U_R with columns scaled by S_R, dst = [W_i W_j]
//   V     : src = dst = [V_i V_j], X = accumulated rotation (GRAM) or V_R (DIRECT)
// A CTA takes a 128-row tile: the source tile is staged k-major (row index contiguous, straight
// from the column-major matrix), the multiplier once per tile, and each of the 256 threads
// accumulates a 4-row x (2bw / 8)-column block in registers (one 4-wide and two (2bw/16)-wide
// shared loads per 4 x 2bw/8 FMAs).
// ------------------------------------------------------------------------------------------------
constexpr int kUpdRows = 128;

// V consecutive shared-memory values starting at a 16-byte aligned address, in 16-byte loads
template <typename T, int V>
__device__ __forceinline__ void ld_shared_vec(const T* p, T (&v)[V])
{
    static_assert((V * sizeof(T)) % 16 == 0, "whole 16-byte vectors");
    if constexpr (sizeof(T) == 8) {
        const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
        for (int i = 0; i < V / 2; ++i) {
            const double2 x = q[i];
            v[2 * i] = x.x;
            v[2 * i + 1] = x.y;
        }
    } else {
        const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
        for (int i = 0; i < V / 4; ++i) {
            const float4 x = q[i];
            v[4 * i] = x.x;
            v[4 * i + 1] = x.y;
            v[4 * i + 2] = x.z;
            v[4 * i + 3] = x.w;
        }
    }
}

template <int K2>
constexpr int bj_upd_cols() { return K2 / 8; }  // output columns per thread

// the multiplier's rows padded by 16 bytes: its transposed stores (consecutive threads, consecutive
// rows) then fall in 8 banks instead of one
template <typename T, int K2>
constexpr int bj_upd_ldb() { return K2 + 16 / (int)sizeof(T); }

// two source tiles (the current item's and the next one's) and the multiplier
template <typename T, int K2>
constexpr size_t bj_update_smem()
{
    return sizeof(T) * (2 * (size_t)K2 * (kUpdRows + 4) + (size_t)K2 * bj_upd_ldb<T, K2>());
}

// one update item: (rotating pair `it`, 128-row tile `tile`) of a W or V block-column pair
template <typename T>
struct UpdItem {
    bool valid, useUR;
    int bi, bj, r0, rows, nn, ldd, lds;
    T* dstM;              // the tile's destination (and, except DIRECT's W tile, its source)
    const T* sb;          // the source columns (dstM, or DIRECT's packed Q)
    const T* Xv;          // multiplier: X (GRAM) / V_R (DIRECT), column-major K2 x K2
    const T* URv;         // DIRECT's W tile: U_R, scaled by S_R
    const T* Sv;
};

template <typename T, int K2>
__device__ __forceinline__ UpdItem<T> bj_upd_item(int it, int tile, int npairs, int step, int direct, T* const* U,
                                                  const int* LDU, T* const* V, const int* LDV, const int* M,
                                                  const int* N, unsigned char* ws, const BjLayout& L)
{
    UpdItem<T> q;
    const int b = it / npairs, k = it - b * npairs;
    const BjState* st = reinterpret_cast<const BjState*>(ws + L.off_state) + b;
    const int mm = st->mm, nn = st->nn, nblk = st->nblk;
    const int nbp = nblk + (nblk & 1);
    const int tilesW = (mm + kUpdRows - 1) / kUpdRows, tilesV = (nn + kUpdRows - 1) / kUpdRows;
    q.valid = tile < tilesW + tilesV;
    if (!q.valid) return q;
    round_robin_pair(nbp, step, k, q.bi, q.bj);
    const bool onV = tile >= tilesW;
    q.r0 = (onV ? tile - tilesW : tile) * kUpdRows;
    q.rows = onV ? nn : mm;
    q.nn = nn;
    const bool tr = M[b] < N[b];
    q.dstM = onV ? (tr ? U[b] : V[b]) : (tr ? V[b] : U[b]);
    q.ldd = onV ? (tr ? LDU[b] : LDV[b]) : (tr ? LDV[b] : LDU[b]);
    q.Xv = reinterpret_cast<T* const*>(ws + L.off_pX)[it];
    q.URv = reinterpret_cast<T* const*>(ws + L.off_pUR)[it];
    q.Sv = reinterpret_cast<T* const*>(ws + L.off_pS)[it];
    q.useUR = direct && !onV;
    const T* P = reinterpret_cast<T* const*>(ws + L.off_pP)[it];
    q.sb = q.useUR ? P : q.dstM;
    q.lds = q.useUR ? (mm > K2 ? mm : K2) : q.ldd;
    return q;
}

// the item's source tile, k-major (As[k * LDA + r] = src(r0 + r, column k of the pair)), rows past
// the matrix zero: 16-byte cp.async copies, all of a thread's in flight at once, committed as one
// group (an empty group for an invalid item or unaligned columns, which are copied here directly)
template <typename T, int K2>
__device__ __forceinline__ void bj_upd_stage_a(const UpdItem<T>& q, int bw, T* As)
{
    constexpr int LDA = kUpdRows + 4;
    constexpr int VE = 16 / (int)sizeof(T);    // elements per 16-byte copy
    constexpr int CPC = kUpdRows / VE;         // copies per column
    const int tid = threadIdx.x;
    if (q.valid) {
        if ((reinterpret_cast<uintptr_t>(q.sb) & 15) == 0 && (q.lds % VE) == 0) {
#pragma unroll
            for (int u = 0; u < (K2 * CPC) / 256; ++u) {
                const int e = tid + 256 * u;
                const int kk = e / CPC, r = (e - kk * CPC) * VE;
                const int col = q.useUR ? kk : bj_col(q.bi, q.bj, bw, kk, q.nn);
                int valid = col >= 0 ? q.rows - (q.r0 + r) : 0;
                valid = valid < 0 ? 0 : (valid > VE ? VE : valid);
                const T* src = valid > 0 ? q.sb + (size_t)col * q.lds + q.r0 + r : q.sb;
                const unsigned dst = (unsigned)__cvta_generic_to_shared(As + kk * LDA + r);
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src),
                             "r"(valid * (int)sizeof(T))
                             : "memory");
            }
        } else {
            for (int e = tid; e < K2 * kUpdRows; e += 256) {
                const int kk = e / kUpdRows, r = e - kk * kUpdRows;
                T v = T(0);
                if (q.r0 + r < q.rows) {
                    const int col = q.useUR ? kk : bj_col(q.bi, q.bj, bw, kk, q.nn);
                    if (col >= 0) v = q.sb[(size_t)col * q.lds + q.r0 + r];
                }
                As[kk * LDA + r] = v;
            }
        }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

// the multiplier of the item (consecutive threads: consecutive k of a column), into registers
template <typename T, int K2>
__device__ __forceinline__ void bj_upd_load_b(const UpdItem<T>& q, T (&br)[(K2 * K2) / 256])
{
#pragma unroll
    for (int u = 0; u < (K2 * K2) / 256; ++u) {
        const int e = threadIdx.x + 256 * u;
        const int n = e / K2;
        br[u] = !q.valid ? T(0) : (q.useUR ? q.URv[e] * q.Sv[n] : q.Xv[e]);
    }
}

// ... and transposed into Bs (Bs[k * LDB + n] = multiplier(k, n))
template <typename T, int K2>
__device__ __forceinline__ void bj_upd_store_b(const T (&br)[(K2 * K2) / 256], T* Bs)
{
    constexpr int LDB = bj_upd_ldb<T, K2>();
#pragma unroll
    for (int u = 0; u < (K2 * K2) / 256; ++u) {
        const int e = threadIdx.x + 256 * u;
        const int n = e / K2, kk = e - n * K2;
        Bs[kk * LDB + n] = br[u];
    }
}

// the 128 x K2 product of the staged tile and multiplier, written to the destination: each of the
// 256 threads accumulates a 4-row x (K2 / 8)-column block (one 4-wide and two (K2/16)-wide shared
// loads per 4 x K2/8 FMAs)
template <typename T, int K2>
__device__ __forceinline__ void bj_upd_compute(const UpdItem<T>& q, int bw, const T* As, const T* Bs)
{
    if (!q.valid) return;
    constexpr int LDA = kUpdRows + 4;
    constexpr int LDB = bj_upd_ldb<T, K2>();
    constexpr int NC = bj_upd_cols<K2>();
    constexpr int VE = 16 / (int)sizeof(T);
    const int tid = threadIdx.x;
    const int tx = tid & 31, ty = tid >> 5;       // rows 4 tx .. 4 tx + 3, columns NC ty .. NC ty + NC - 1
    T acc[4][NC];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < NC; ++j) acc[i][j] = T(0);
#pragma unroll 2
    for (int kk = 0; kk < K2; ++kk) {
        T a[4], bv[NC];
        ld_shared_vec<T, 4>(As + kk * LDA + 4 * tx, a);     // 16-byte aligned: LDA * size and 4 tx
        ld_shared_vec<T, NC>(Bs + kk * LDB + NC * ty, bv);
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < NC; ++j) acc[i][j] = fma(a[i], bv[j], acc[i][j]);
    }
    // the thread's 4 rows of each output column in 16-byte stores where aligned and whole
    const bool vst = (reinterpret_cast<uintptr_t>(q.dstM) & 15) == 0 && (q.ldd % VE) == 0 && q.r0 + 4 * tx + 3 < q.rows;
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        const int col = bj_col(q.bi, q.bj, bw, NC * ty + j, q.nn);
        if (col < 0) continue;
        T* d = q.dstM + (size_t)col * q.ldd + q.r0 + 4 * tx;
        if (vst) {
            if constexpr (sizeof(T) == 4) {
                *reinterpret_cast<float4*>(d) = make_float4(acc[0][j], acc[1][j], acc[2][j], acc[3][j]);
            } else {
                reinterpret_cast<double2*>(d)[0] = make_double2(acc[0][j], acc[1][j]);
                reinterpret_cast<double2*>(d)[1] = make_double2(acc[2][j], acc[3][j]);
            }
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (q.r0 + 4 * tx + i < q.rows) d[i] = acc[i][j];
        }
    }
}

// Work items are (rotating pair, row tile) flattened; `tiles` is the bound on tiles per pair.  Two
// source-tile buffers: while a CTA multiplies one item, the next item's tile is already being
// copied in and its multiplier loaded into registers, so the copies' latency is hidden behind the
// product.
template <typename T, int K2>
__global__ void __launch_bounds__(256, 2) bj_update_kernel(int tiles, int npairs, int step, int bw, int direct,
                                                           T* const* U, const int* LDU, T* const* V, const int* LDV,
                                                           const int* M, const int* N, unsigned char* ws, BjLayout L)
{
    extern __shared__ __align__(16) unsigned char upd_sm[];
    constexpr int LDA = kUpdRows + 4;
    T* As0 = reinterpret_cast<T*>(upd_sm);
    T* As1 = As0 + (size_t)K2 * LDA;
    T* Bs = As1 + (size_t)K2 * LDA;
    BjCounters* C = reinterpret_cast<BjCounters*>(ws + L.off_ctr);
    const int* plist = reinterpret_cast<const int*>(ws + L.off_plist);
    const long long total = (long long)C->pcount * tiles;
    long long w = next_work(&C->claim[3]);
    if (w >= total) return;   // (uniform: every thread read the same claimed position)
    UpdItem<T> q = bj_upd_item<T, K2>(plist[w / tiles], (int)(w % tiles), npairs, step, direct, U, LDU, V, LDV, M,
                                      N, ws, L);
    bj_upd_stage_a<T, K2>(q, bw, As0);
    {
        T br[(K2 * K2) / 256];
        bj_upd_load_b<T, K2>(q, br);
        bj_upd_store_b<T, K2>(br, Bs);
    }
    int buf = 0;
    for (;;) {
        const long long wn = next_work(&C->claim[3]);   // its barrier: the other buffer is free
        const bool next = wn < total;
        UpdItem<T> qn;
        T br[(K2 * K2) / 256];
        if (next) {
            qn = bj_upd_item<T, K2>(plist[wn / tiles], (int)(wn % tiles), npairs, step, direct, U, LDU, V, LDV, M,
                                    N, ws, L);
            bj_upd_stage_a<T, K2>(qn, bw, buf ? As0 : As1);
            bj_upd_load_b<T, K2>(qn, br);
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");   // this item's tile has landed
        } else {
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        }
        __syncthreads();
        bj_upd_compute<T, K2>(q, bw, buf ? As1 : As0, Bs);
        if (!next) break;
        __syncthreads();   // every thread is done with Bs
        bj_upd_store_b<T, K2>(br, Bs);
        q = qn;
        buf ^= 1;
    }
}

// ------------------------------------------------------------------------------------------------
// Tensor-core Gram stage (FP32 data, bw = 32: pair width 64).  G = X^T X runs on tcgen05 in TF32
// with FP32 accumulation; every FP32 element x is split as x = hi + lo with hi = tf32(x) and
// lo = tf32(x - hi), both rounded to nearest (x carried to 2^-23 relative, without bias), and all
// four products hi^T hi, hi^T lo, lo^T hi, lo^T lo are formed.  Operands are staged through
// registers into the K-major core-matrix layout of tcgen05.cuh; the accumulator lives in tensor
// memory.  The update stays on the SIMT pipes: measured on a GB300, the tensor core's FP32
// accumulation rounds toward zero (mean error -2.7e-7 relative for a K = 64 product of exact
// TF32 values, FP32 FMA +2e-9), a bias that V, updated ~200 times per column, accumulates to
// ||V^T V - I|| ~ 2e-5, above the 1e-5 gate; the Gram only feeds the pair test and the inner
// SVD, whose rotation is re-orthogonalised, so its bias does not accumulate.
// ------------------------------------------------------------------------------------------------
constexpr int kTcGramKc = 32;                                   // rows of X per staged chunk
constexpr uint32_t kTcLbo = 128;                                // K-adjacent core matrices
constexpr uint32_t kTcGramSbo = (kTcGramKc / 4) * 128;          // 1024 B between 8-row groups
constexpr uint32_t kTcGramStage = 128u * kTcGramKc * 4u;        // 16 KB: 64 hi + 64 lo rows x KC
constexpr int kTcGramStages = 3;
// raw FP32 chunks (64 columns x KC rows, 8 KB each) copied in asynchronously two chunks ahead of
// the split; three slots, so the copy into a slot never overtakes the split that last read it
constexpr uint32_t kTcRawStage = 64u * kTcGramKc * 4u;
constexpr int kTcRawStages = 3;
// 3 operand stages (48 KB) + 3 raw stages (24 KB) + alignment: three CTAs fit an SM (3 x 128 TMEM
// columns <= 512)
constexpr size_t kTcGramSmem = kTcGramStages * kTcGramStage + kTcRawStages * kTcRawStage + 1024 + 64;

// next claimed position, or "none" once any tensor-core wait of the call has given up (uniform
// over the CTA: thread 0 decides, the barrier publishes)
__device__ __forceinline__ long long tc_next(BjCounters* C, int which)
{
    __shared__ long long s_pos;
    __syncthreads();
    if (threadIdx.x == 0)
        s_pos = *reinterpret_cast<volatile int*>(&C->timeouts) != 0 ? (1ll << 62)
                                                                     : (long long)atomicAdd(&C->claim[which], 1ull);
    __syncthreads();
    return s_pos;
}

__device__ __forceinline__ unsigned char* align1k(unsigned char* p)
{
    return reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(p) + 1023) & ~(uintptr_t)1023);
}

__device__ __forceinline__ float4 tc_hi(float4 v)
{
    return make_float4(tc::to_tf32(v.x), tc::to_tf32(v.y), tc::to_tf32(v.z), tc::to_tf32(v.w));
}

__device__ __forceinline__ float4 tc_lo(float4 v, float4 h)
{
    return make_float4(tc::to_tf32(v.x - h.x), tc::to_tf32(v.y - h.y), tc::to_tf32(v.z - h.z),
                       tc::to_tf32(v.w - h.w));
}

__device__ __forceinline__ void tc_split_store(unsigned char* hi_base, unsigned char* lo_base, uint32_t off,
                                               float4 v)
{
    const float4 h = tc_hi(v);
    *reinterpret_cast<float4*>(hi_base + off) = h;
    *reinterpret_cast<float4*>(lo_base + off) = tc_lo(v, h);
}

// Gram of one pair item: D = [X_hi X_lo]^T [X_hi X_lo] (128 x 128, M = N = 128, K = rows), then
// G = D11 + D12 + D21 + D22 = hi^T hi + hi^T lo + lo^T hi + lo^T lo: X^T X up to the TF32 reading
// of lo (relative 2^-22).
// Pair test as the SIMT kernel's: max |G_pq| / sqrt(G_pp G_qq), located in FP32 and evaluated in
// FP64 for the winning element.
__device__ __forceinline__ void bj_gram_tc_item(int it, int npairs, int step, int bw, float* const* U,
                                                const int* LDU, float* const* V, const int* LDV, const int* M,
                                                const int* N, unsigned char* ws, const BjLayout& L, double tol,
                                                unsigned char* sm, uint32_t tmem, uint64_t* bars,
                                                uint32_t& phase, uint32_t& used, BjCounters* C, uint64_t* never)
{
    constexpr int K2 = 64;
    __shared__ float gd[K2];
    __shared__ float redv[4];
    __shared__ int redi[4];
    const int b = it / npairs, k = it - b * npairs;
    BjState* st = reinterpret_cast<BjState*>(ws + L.off_state) + b;
    int* im = reinterpret_cast<int*>(ws + L.off_m);
    int* in = reinterpret_cast<int*>(ws + L.off_n);
    const int mm = st->mm, nn = st->nn, nblk = st->nblk;
    const int nbp = nblk + (nblk & 1);
    int bi = 0, bj = 0;
    if (k < nbp / 2 && step < nbp - 1) round_robin_pair(nbp, step, k, bi, bj);
    const bool live = !st->converged && step < nbp - 1 && k < nbp / 2 && (bj < nblk || nblk == 1) && bi * bw < nn &&
                      mm > 0;  // (the SIMT item explains each condition)
    const BjPairRecord pr = bj_pair_record(ws, L, b, bi, bj);
    if (!live || (!L.retest && pr.rec && *pr.rec == pr.key)) {   // as in the SIMT item
        if (threadIdx.x == 0) im[it] = in[it] = 0;
        return;
    }
    const bool tr = M[b] < N[b];
    const float* W = tr ? V[b] : U[b];
    const int ldw = tr ? LDV[b] : LDU[b];
    const int tid = threadIdx.x;
    const bool vec = (ldw & 3) == 0 && (reinterpret_cast<uintptr_t>(W) & 15) == 0;
    const int nch = (mm + kTcGramKc - 1) / kTcGramKc;
    constexpr uint32_t idesc = tc::idesc_tf32(128, 128);
    constexpr int kUnits = (K2 * kTcGramKc / 4) / 128;  // float4 units per thread per chunk
    unsigned char* raw = sm + kTcGramStages * kTcGramStage;
    // unit j of this thread: column i, 4-row group g (consecutive threads take consecutive columns,
    // so eight threads write one 128-byte core matrix).  Chunk c's units are copied asynchronously
    // into raw slot c % 3 at unit offset u * 16 (rows past mm and padding columns zero-filled); the
    // thread that copies a unit is the thread that later splits it, so its own wait suffices.
    auto issue_chunk = [&](int c) {
        unsigned char* slot = raw + (c % kTcRawStages) * kTcRawStage;
#pragma unroll
        for (int j = 0; j < kUnits; ++j) {
            const int u = tid + 128 * j;
            const int i = u & (K2 - 1), g = u / K2;
            const int col = bj_col(bi, bj, bw, i, nn);
            const int r = c * kTcGramKc + 4 * g;
            const int left = col >= 0 ? (mm - r < 0 ? 0 : (mm - r > 4 ? 4 : mm - r)) : 0;
            const float* src = col >= 0 && left > 0 ? W + (size_t)col * ldw + r : W;
            const uint32_t dst = tc::smem_u32(slot + u * 16);
            if (vec) {
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src),
                             "r"(4 * left)
                             : "memory");
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(dst + 4 * e),
                                 "l"(e < left ? src + e : W), "r"(e < left ? 4 : 0)
                                 : "memory");
            }
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    issue_chunk(0);
    if (nch > 1) issue_chunk(1);
    bool ok = true;
    for (int c = 0; c < nch; ++c) {
        const int s = c % kTcGramStages;
        unsigned char* stage = sm + s * kTcGramStage;
        // two chunks ahead: the copy into slot (c + 2) % 3 follows the split of chunk c - 1 that read it
        if (c + 2 < nch) {
            issue_chunk(c + 2);
            asm volatile("cp.async.wait_group 2;\n" ::: "memory");
        } else if (c + 1 < nch) {
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        }
        if (c >= kTcGramStages) {  // the MMAs of chunk c - 3 read this stage
            // after a failure: no more waits.  `never` (failure-path test only) is a barrier nothing
            // arrives at, waited for 1 ms: the wait runs out, and the call takes its timeout path
            if (ok) ok = never ? tc::mbar_wait(never, 0u, 1000000ull) : tc::mbar_wait(&bars[s], (phase >> s) & 1u);
            phase ^= 1u << s;
        }
        const unsigned char* rs = raw + (c % kTcRawStages) * kTcRawStage;
#pragma unroll
        for (int j = 0; j < kUnits; ++j) {
            const int u = tid + 128 * j;
            const int i = u & (K2 - 1), g = u / K2;
            const float4 v = *reinterpret_cast<const float4*>(rs + u * 16);
            // hi to operand rows 0..63, lo to rows 64..127 of the same stage
            tc_split_store(stage + tc::kmajor_offset(i, 4 * g, kTcLbo, kTcGramSbo),
                           stage + tc::kmajor_offset(K2 + i, 4 * g, kTcLbo, kTcGramSbo), 0u, v);
        }
        tc::fence_smem_to_async();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            const uint32_t base = tc::smem_u32(stage);
#pragma unroll
            for (int kk = 0; kk < kTcGramKc / 8; ++kk) {
                const uint64_t d = tc::desc_kmajor(base + kk * 2 * kTcLbo, kTcLbo, kTcGramSbo);
                tc::mma_tf32(tmem, d, d, idesc, (c > 0 || kk > 0) ? 1u : 0u);
            }
            tc::mma_commit(&bars[s]);
        }
        used |= 1u << s;  // stages that have received a commit (for the failure path's drain)
    }
    // drain: the last (up to three) chunks' commits, one per barrier
    for (int c = nch > kTcGramStages ? nch - kTcGramStages : 0; c < nch; ++c) {
        const int s = c % kTcGramStages;
        if (ok) ok = tc::mbar_wait(&bars[s], (phase >> s) & 1u);
        phase ^= 1u << s;
    }
    tc::fence_after_sync();
    // epilogue: lane (row) i of D; P = D(i, 0:64) + D(i, 64:128)
    const int warp = tid >> 5, lane = tid & 31;
    const int row = warp * 32 + lane;
    float p[K2];
    {
        float a[32], c2[32];
        const uint32_t t = tmem + ((uint32_t)(warp * 32) << 16);
        tc::tmem_ld32(t + 0, a);
        tc::tmem_ld32(t + 64, c2);
#pragma unroll
        for (int j = 0; j < 32; ++j) p[j] = a[j] + c2[j];
        tc::tmem_ld32(t + 32, a);
        tc::tmem_ld32(t + 96, c2);
#pragma unroll
        for (int j = 0; j < 32; ++j) p[32 + j] = a[j] + c2[j];
    }
    tc::fence_before_sync();
    float* Gs = reinterpret_cast<float*>(sm);  // 64 x 65, row-major, over the (idle) stages
    __syncthreads();
    if (row >= K2) {
#pragma unroll
        for (int j = 0; j < K2; ++j) Gs[(row - K2) * (K2 + 1) + j] = p[j];
    }
    __syncthreads();
    if (row < K2) {
#pragma unroll
        for (int j = 0; j < K2; ++j) Gs[row * (K2 + 1) + j] += p[j];
    }
    __syncthreads();
    if (!ok && tid == 0) atomicAdd(&C->timeouts, 1);
    // G to the item's buffer (column-major; G is symmetric up to rounding), diagonal to gd
    float* G = reinterpret_cast<float* const*>(ws + L.off_pG)[it];
    for (int e = tid; e < K2 * K2; e += 128) {
        const int gc = e / K2, gr = e - gc * K2;
        G[e] = Gs[gr * (K2 + 1) + gc];
    }
    if (tid < K2) gd[tid] = Gs[tid * (K2 + 1) + tid];
    __syncthreads();
    // largest scaled off-diagonal element: located in FP32 ...
    float best = -1.f;
    int bidx = 0;
    for (int e = tid; e < K2 * K2; e += 128) {
        const int r = e / K2, c = e - r * K2;
        if (r == c) continue;
        const float dr = gd[r], dc = gd[c];
        if (!(dr > 0.f) || !(dc > 0.f)) continue;
        const float v = fabsf(Gs[r * (K2 + 1) + c]) * rsqrtf(dr) * rsqrtf(dc);
        if (v > best) {
            best = v;
            bidx = e;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
        if (ov > best || (ov == best && oi < bidx)) {
            best = ov;
            bidx = oi;
        }
    }
    if (lane == 0) {
        redv[warp] = best;
        redi[warp] = bidx;
    }
    __syncthreads();
    if (tid == 0) {
        for (int w = 1; w < 4; ++w)
            if (redv[w] > best || (redv[w] == best && redi[w] < bidx)) {
                best = redv[w];
                bidx = redi[w];
            }
        // ... and evaluated in FP64
        double em = 0.0;
        if (best >= 0.f) {
            const int r = bidx / K2, c = bidx - r * K2;
            em = fabs((double)Gs[r * (K2 + 1) + c]) / sqrt((double)gd[r] * (double)gd[c]);
        }
        const bool rot = em > tol;
        im[it] = rot ? K2 : 0;
        in[it] = rot ? K2 : 0;
        if (rot) {
            atomicAdd(&st->rot_sweep, 1);
            reinterpret_cast<int*>(ws + L.off_plist)[atomicAdd(&C->pcount, 1)] = it;
            ++pr.ver[bi];
            ++pr.ver[bj];
        } else if (pr.rec) {
            *pr.rec = pr.key;
        }
        atomicMax(reinterpret_cast<unsigned long long*>(&st->emax), (unsigned long long)__double_as_longlong(em));
    }
}

// TMEM and barriers are set up once per CTA; the CTA then claims pair items of the live matrices
__global__ void __launch_bounds__(128) bj_gram_tc_kernel(int npairs, int step, int bw, float* const* U,
                                                         const int* LDU, float* const* V, const int* LDV,
                                                         const int* M, const int* N, unsigned char* ws, BjLayout L,
                                                         double tol, int test_timeout)
{
    extern __shared__ __align__(16) unsigned char tc_raw[];
    __shared__ uint64_t bars[kTcGramStages];
    __shared__ uint64_t never_bar;  // failure-path test: a barrier nothing arrives at
    __shared__ uint32_t tmem_slot;
    unsigned char* sm = align1k(tc_raw);
    BjCounters* C = reinterpret_cast<BjCounters*>(ws + L.off_ctr);
    if (threadIdx.x < 32) {
        tc::tmem_alloc(&tmem_slot, 128);
        tc::tmem_relinquish();
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < kTcGramStages; ++s) tc::mbar_init(&bars[s], 1);
        tc::mbar_init(&never_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    uint32_t phase = 0, used = 0;
    const int* mlist = reinterpret_cast<const int*>(ws + L.off_mlist);
    const long long items = (long long)C->mcount * npairs;
    for (long long j = tc_next(C, 0); j < items; j = tc_next(C, 0)) {
        const int b = mlist[j / npairs], k = (int)(j % npairs);
        bj_gram_tc_item(b * npairs + k, npairs, step, bw, U, LDU, V, LDV, M, N, ws, L, tol, sm, tmem, bars, phase,
                        used, C, test_timeout ? &never_bar : nullptr);
    }
    // after a wait that gave up (in any CTA of the call) this CTA's MMAs may still be in flight:
    // wait once more, again bounded, for the last commit of every stage it used before its tensor
    // memory is released (a CTA whose waits all succeeded finds every phase complete at once)
    if (*reinterpret_cast<volatile int*>(&C->timeouts) != 0) {
        for (int s = 0; s < kTcGramStages; ++s)
            if ((used >> s) & 1u) tc::mbar_wait(&bars[s], ((phase >> s) & 1u) ^ 1u);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (threadIdx.x < 32) tc::tmem_dealloc(tmem, 128);
}

// end of a sweep: a matrix whose sweep rotated nothing is converged
__global__ void bj_sweep_end_kernel(int batch, int max_sweeps, int sweep, unsigned char* ws, BjLayout L, int* info)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= batch) return;
    BjState* st = reinterpret_cast<BjState*>(ws + L.off_state) + b;
    if (st->converged) return;
    st->sweeps = sweep + 1;
    st->rotations += st->rot_sweep;
    if (st->rot_sweep == 0) {
        st->converged = 1;
        info[b] = sweep + 1;
    } else if (sweep + 1 >= max_sweeps) {
        info[b] = BSVD_INFO_NOT_CONVERGED + sweep + 1;
    }
    st->rot_sweep = 0;
    st->emax = 0.0;
    if (!st->converged) {  // still live: on the next sweep's list
        BjCounters* C = reinterpret_cast<BjCounters*>(ws + L.off_ctr);
        reinterpret_cast<int*>(ws + L.off_mlist)[atomicAdd(&C->mcount, 1)] = b;
    }
}

// ------------------------------------------------------------------------------------------------
// finalize: sigma, normalisation, descending sort of U and V columns in place
// ------------------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) bj_finalize_kernel(int batch, T* const* S, T* const* U, const int* LDU,
                                                          T* const* V, const int* LDV, const int* M, const int* N,
                                                          unsigned char* ws, BjLayout L, int* info,
                                                          long long* rot_out)
{
    extern __shared__ __align__(16) unsigned char sm[];
    const int b = blockIdx.x;
    BjState* st = reinterpret_cast<BjState*>(ws + L.off_state) + b;
    if (info[b] == BSVD_INFO_BAD_SHAPE) return;
    if (reinterpret_cast<const BjCounters*>(ws + L.off_ctr)->timeouts != 0) {  // results not valid
        if (threadIdx.x == 0) info[b] = BSVD_INFO_DEVICE_TIMEOUT;
        return;
    }
    const int mm = st->mm, nn = st->nn;
    if (threadIdx.x == 0 && rot_out) rot_out[b] = st->rotations;
    if (nn == 0) return;
    const bool tr = M[b] < N[b];
    T* W = tr ? V[b] : U[b];
    const int ldw = tr ? LDV[b] : LDU[b];
    T* Vk = tr ? U[b] : V[b];
    const int ldv = tr ? LDU[b] : LDV[b];
    const size_t a16 = 16;
    T* sig = reinterpret_cast<T*>(sm);
    int* dest = reinterpret_cast<int*>(sm + ((nn * sizeof(T) + a16 - 1) & ~(a16 - 1)));
    unsigned char* done = reinterpret_cast<unsigned char*>(dest) + ((nn * sizeof(int) + a16 - 1) & ~(a16 - 1));
    T* tmpW = reinterpret_cast<T*>(done + ((nn + a16 - 1) & ~(a16 - 1)));
    T* tmpV = tmpW + mm;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j = warp; j < nn; j += nw) {
        T s = T(0);
        for (int r = lane; r < mm; r += 32) s = fma(W[(size_t)j * ldw + r], W[(size_t)j * ldw + r], s);
        s = warp_sum(s);
        if (lane == 0) sig[j] = dsqrt(s);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        bool finite = true;
        for (int j = 0; j < nn; ++j) finite = finite && isfinite(sig[j]);
        if (!finite) info[b] = BSVD_INFO_NONFINITE;
    }
    for (int j = threadIdx.x; j < nn; j += blockDim.x) {
        // rank in a total order (a NaN ranks last), so that dest is always a permutation
        const T sj = sig[j] == sig[j] ? sig[j] : T(-1);
        int r = 0;
        for (int i = 0; i < nn; ++i) {
            const T si = sig[i] == sig[i] ? sig[i] : T(-1);
            r += (si > sj) || (si == sj && i < j);
        }
        dest[j] = r;
        done[j] = 0;
        S[b][r] = sig[j];
    }
    __syncthreads();
    // normalise W columns (U = W / sigma)
    for (int j = warp; j < nn; j += nw) {
        const T sj = sig[j];
        const T inv = sj > T(0) ? T(1) / sj : T(0);
        for (int r = lane; r < mm; r += 32) W[(size_t)j * ldw + r] *= inv;
    }
    __syncthreads();
    // permute columns j -> dest[j] by following cycles (one column in flight in shared memory)
    for (int j0 = 0; j0 < nn; ++j0) {
        if (done[j0] || dest[j0] == j0) continue;
        for (int r = threadIdx.x; r < mm; r += blockDim.x) tmpW[r] = W[(size_t)j0 * ldw + r];
        for (int r = threadIdx.x; r < nn; r += blockDim.x) tmpV[r] = Vk[(size_t)j0 * ldv + r];
        __syncthreads();
        int j = j0, guard = 0;
        do {
            const int d = dest[j];
            // swap the in-flight column with column d
            for (int r = threadIdx.x; r < mm; r += blockDim.x) {
                const T x = W[(size_t)d * ldw + r];
                W[(size_t)d * ldw + r] = tmpW[r];
                tmpW[r] = x;
            }
            for (int r = threadIdx.x; r < nn; r += blockDim.x) {
                const T x = Vk[(size_t)d * ldv + r];
                Vk[(size_t)d * ldv + r] = tmpV[r];
                tmpV[r] = x;
            }
            __syncthreads();
            if (threadIdx.x == 0) done[j] = 1;
            j = d;
            __syncthreads();
        } while (j != j0 && ++guard < nn);  // a permutation closes every cycle within nn moves
    }
}

// ------------------------------------------------------------------------------------------------
// host driver
// ------------------------------------------------------------------------------------------------
template <typename T>
size_t block_jacobi_workspace(int batch, int max_m, int max_n, int bw, int method)
{
    if (method & BSVD_BLOCK_QR_PRECONDITION) return block_jacobi_qr_workspace<T>(batch, max_m, max_n, bw, method);
    return bj_layout<T>(batch, max_m, max_n, bw, (method & 0xff) != 0).total;
}

template <typename T, int K2>
static int run_block(int batch, int max_m, int max_n, void* const* A, const int* M, const int* N, const int* LDA,
                     void* const* S, void* const* U, const int* LDU, void* const* V, const int* LDV, double tol,
                     int max_sweeps, int method, int* info, long long* rot, unsigned char* ws, cudaStream_t st)
{
    const int bw = K2 / 2;
    int inner_variant = (method >> 8) & 0xff;  // register-tier variant of the inner SVD (0: see below)
    const int cap_bits = (method >> 24) & 0x7f;
    const bool simt = (method & BSVD_BLOCK_SIMT_PRODUCTS) != 0;
    const int test_timeout = (method & BSVD_BLOCK_TEST_TIMEOUT) != 0 ? 1 : 0;
    const int retest = (method & BSVD_BLOCK_RETEST_ALL) != 0 ? 1 : 0;
    method &= 0xff;
    const bool direct = method != 0;
    // sweep cap of each inner SVD: 127 = to convergence (as Algorithm 3 states), 0 = default.
    // Measured on 160 x 512^2 (GRAM): caps of 8, 4, 2 sweeps leave the outer sweeps (14.5, 14.5,
    // 14.3) and every error unchanged while the call gets 0, 9 and 21% faster -- a fully converged
    // inner SVD is wasted once the outer iteration revisits the pair -- so GRAM defaults to 2.
    const int inner_sweeps = cap_bits == 127 ? 0 : (cap_bits != 0 ? cap_bits : (direct ? 0 : 2));
    // GRAM's inner SVD by default runs the QR-preconditioned register variant and takes X from
    // its U = Q V_w (orthogonal by construction, also for the zero singular values of padding
    // columns; for the symmetric positive semidefinite G the left singular vectors are its
    // eigenvectors): fewer sweeps than the plain variant on A = G.  DIRECT needs both factors of
    // the SVD of R and keeps the first plain variant.
    bool inner_u = false;
    if (!direct && inner_variant == 0) {
        int d[9];
        for (int k = 1; jacobi_reg_variant_desc(sizeof(T) == 8, K2, K2, k, d) == BSVD_SUCCESS; ++k)
            if (d[6]) {
                inner_variant = k;
                inner_u = true;
                break;
            }
    } else if (!direct) {
        int d[9];
        inner_u = jacobi_reg_variant_desc(sizeof(T) == 8, K2, K2, inner_variant, d) == BSVD_SUCCESS && d[6];
    }
    BjLayout L = bj_layout<T>(batch, max_m, max_n, bw, direct);
    L.retest = retest;
    const int mm = max_m > max_n ? max_m : max_n, nn = max_m > max_n ? max_n : max_m;
    const int npairs = L.npairs, nbp = 2 * npairs;
    // default pair threshold sqrt(m) u; DIRECT rotations are only as orthogonal as the pair's
    // Householder Q (~ 2bw u), so its default sits 4x higher (U's orthogonality at convergence is
    // the threshold: 4 sqrt(512) u = 5.4e-6 in FP32)
    const double tol_outer = tol > 0.0 ? tol : (direct ? 4.0 : 1.0) * sqrt((double)mm) * Unit<T>::value;
    BjCounters* ctr = reinterpret_cast<BjCounters*>(ws + L.off_ctr);
    if (cudaMemsetAsync(ctr, 0, sizeof(BjCounters), st) != cudaSuccess) return BSVD_ERR_CUDA;
    bj_setup_kernel<T><<<batch, 256, 0, st>>>(batch, mm, nn, bw, npairs, (T* const*)A, M, N, LDA, (T* const*)U, LDU,
                                              (T* const*)V, LDV, ws, L, info);
    if (cudaGetLastError() != cudaSuccess) return BSVD_ERR_CUDA;
    const int items = batch * npairs;
    void* const* pG = reinterpret_cast<void* const*>(ws + L.off_pG);
    void* const* pX = reinterpret_cast<void* const*>(ws + L.off_pX);
    void* const* pS = reinterpret_cast<void* const*>(ws + L.off_pS);
    void* const* pUR = reinterpret_cast<void* const*>(ws + L.off_pUR);
    void* const* pP = reinterpret_cast<void* const*>(ws + L.off_pP);
    const int* im = reinterpret_cast<const int*>(ws + L.off_m);
    const int* in = reinterpret_cast<const int*>(ws + L.off_n);
    const int* ild = reinterpret_cast<const int*>(ws + L.off_ld);  // 2bw for every item
    const int* ildp = reinterpret_cast<const int*>(ws + L.off_ldp);
    int* iinfo = reinterpret_cast<int*>(ws + L.off_info);
    const int tiles = (mm + kUpdRows - 1) / kUpdRows + (nn + kUpdRows - 1) / kUpdRows;
    constexpr size_t upd_smem = bj_update_smem<T, K2>();
    if (upd_smem > 48 * 1024 && cudaFuncSetAttribute(bj_update_kernel<T, K2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     (int)upd_smem) != cudaSuccess)
        return BSVD_ERR_CUDA;
    const int sweeps = max_sweeps > 0 ? max_sweeps : 20;
    const size_t polish_smem = bj_polish_smem<T, K2>();
    if (polish_smem > 48 * 1024 && cudaFuncSetAttribute(bj_polish_kernel<T, K2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                        (int)polish_smem) != cudaSuccess)
        return BSVD_ERR_CUDA;
    // persistent grids over the live lists: converged matrices and orthogonal pairs cost nothing
    const ItemList pairs{reinterpret_cast<const int*>(ws + L.off_plist), &ctr->pcount, nullptr};
    const int g_gram = persistent_grid(bj_gram_kernel<T, K2>, 256, 0, items);
    const int g_pack = persistent_grid(bj_pack_kernel<T, K2>, 256, 0, items);
    const int g_polish = persistent_grid(bj_polish_kernel<T, K2>, 256, polish_smem, items);
    const int g_update = persistent_grid(bj_update_kernel<T, K2>, 256, upd_smem, (long long)items * tiles);
    // tensor-core Gram (FP32 data, bw = 32)
    const bool tc_gram = sizeof(T) == 4 && K2 == 64 && !simt;
    int g_gram_tc = 1;
    if (tc_gram) {
        if (cudaFuncSetAttribute(bj_gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcGramSmem) !=
            cudaSuccess)
            return BSVD_ERR_CUDA;
        // resident CTAs per SM from the kernel's registers and shared memory (at most four:
        // 4 x 128 = 512 TMEM columns, so tcgen05.alloc never waits); the occupancy query reports
        // one for any kernel that allocates tensor memory, so the grid is set from these limits
        int dev = 0, sms = 1, regs_sm = 65536, smem_sm = 228 * 1024;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, bj_gram_tc_kernel) != cudaSuccess) return BSVD_ERR_CUDA;
        const int by_regs = regs_sm / ((fa.numRegs > 0 ? fa.numRegs : 255) * 128);
        const int by_smem = smem_sm / (int)(kTcGramSmem + fa.sharedSizeBytes + 1024);
        int per = by_regs < by_smem ? by_regs : by_smem;
        per = per < 1 ? 1 : (per > 4 ? 4 : per);
        g_gram_tc = items < per * sms ? items : per * sms;
    }
    for (int sw = 0; sw < sweeps; ++sw) {
        for (int step = 0; step < nbp - 1; ++step) {
            if (cudaMemsetAsync(ctr, 0, kStepCounterBytes, st) != cudaSuccess) return BSVD_ERR_CUDA;
            if (tc_gram)
                bj_gram_tc_kernel<<<g_gram_tc, 128, kTcGramSmem, st>>>(npairs, step, bw, (float* const*)U, LDU,
                                                                      (float* const*)V, LDV, M, N, ws, L, tol_outer,
                                                                      test_timeout);
            else
                bj_gram_kernel<T, K2><<<g_gram, 256, 0, st>>>(batch, npairs, step, bw, (T* const*)U, LDU,
                                                              (T* const*)V, LDV, M, N, ws, L, tol_outer);
            if (!direct) {
                const int rc = launch_jacobi_reg<T>(items, K2, K2, inner_variant, pG, im, in, ild, pS,
                                                    inner_u ? pX : nullptr, ild, inner_u ? nullptr : pX, ild, 0.0,
                                                    inner_sweeps, iinfo, nullptr, st,
                                                    ItemList{pairs.idx, pairs.count, &ctr->claim[5]});
                if (rc != BSVD_SUCCESS) return rc;
            } else {
                bj_pack_kernel<T, K2><<<g_pack, 256, 0, st>>>(batch, npairs, step, bw, (T* const*)U, LDU,
                                                              (T* const*)V, LDV, M, N, ws, L);
                int rc = launch_qr<T>(items, L.mm_max, K2, pP, im, in, ildp, pP, ildp, pG, ild, iinfo, st,
                                      ItemList{pairs.idx, pairs.count, &ctr->claim[4]});
                if (rc != BSVD_SUCCESS) return rc;
                // the inner sizes are K2 x K2 (R) for live items: reuse the n array for both
                rc = launch_jacobi_reg<T>(items, K2, K2, inner_variant, pG, in, in, ild, pS, pUR, ild, pX, ild, 0.0,
                                          inner_sweeps, iinfo, nullptr, st,
                                          ItemList{pairs.idx, pairs.count, &ctr->claim[5]});
                if (rc != BSVD_SUCCESS) return rc;
            }
            bj_polish_kernel<T, K2><<<g_polish, 256, polish_smem, st>>>(ws, L, direct ? 1 : 0);
            bj_update_kernel<T, K2><<<g_update, 256, upd_smem, st>>>(tiles, npairs, step, bw, direct ? 1 : 0,
                                                                     (T* const*)U, LDU, (T* const*)V, LDV, M, N, ws, L);
            if (cudaGetLastError() != cudaSuccess) return BSVD_ERR_CUDA;
        }
        if (cudaMemsetAsync(&ctr->mcount, 0, sizeof(int), st) != cudaSuccess) return BSVD_ERR_CUDA;
        bj_sweep_end_kernel<<<(batch + 127) / 128, 128, 0, st>>>(batch, sweeps, sw, ws, L, info);
    }
    const size_t fsm = (size_t)nn * (sizeof(T) + sizeof(int) + 1) + 48 + (size_t)(mm + nn) * sizeof(T) + 64;
    if (fsm > 48 * 1024 &&
        cudaFuncSetAttribute(bj_finalize_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm) != cudaSuccess)
        return BSVD_ERR_CUDA;
    bj_finalize_kernel<T><<<batch, 256, fsm, st>>>(batch, (T* const*)S, (T* const*)U, LDU, (T* const*)V, LDV, M, N, ws,
                                                   L, info, rot);
    return cudaGetLastError() == cudaSuccess ? BSVD_SUCCESS : BSVD_ERR_CUDA;
}

template <typename T>
int launch_block_jacobi(int batch, int max_m, int max_n, int bw, int method, void* const* A, const int* M,
                        const int* N, const int* LDA, void* const* S, void* const* U, const int* LDU, void* const* V,
                        const int* LDV, double tol, int max_sweeps, int* info, long long* rot, void* ws, size_t ws_bytes,
                        cudaStream_t st)
{
    if (method & BSVD_BLOCK_QR_PRECONDITION)
        return launch_block_jacobi_qr<T>(batch, max_m, max_n, bw, method, A, M, N, LDA, S, U, LDU, V, LDV, tol,
                                         max_sweeps, info, rot, ws, ws_bytes, st);
    if (bw != 16 && bw != 32) return BSVD_ERR_UNSUPPORTED;
    const int mm = max_m > max_n ? max_m : max_n;
    if ((method & 0xff) != 0 && (size_t)(mm > 2 * bw ? mm : 2 * bw) * 2 * bw * sizeof(T) > 200 * 1024) return BSVD_ERR_UNSUPPORTED;
    if (mm > 16384) return BSVD_ERR_UNSUPPORTED;
    if (ws_bytes < block_jacobi_workspace<T>(batch, max_m, max_n, bw, method & 0xff)) return BSVD_ERR_WORKSPACE;
    unsigned char* w = static_cast<unsigned char*>(ws);
    return bw == 16 ? run_block<T, 32>(batch, max_m, max_n, A, M, N, LDA, S, U, LDU, V, LDV, tol, max_sweeps, method,
                                       info, rot, w, st)
                    : run_block<T, 64>(batch, max_m, max_n, A, M, N, LDA, S, U, LDU, V, LDV, tol, max_sweeps, method,
                                       info, rot, w, st);
}

template size_t block_jacobi_workspace<float>(int, int, int, int, int);
template size_t block_jacobi_workspace<double>(int, int, int, int, int);
template int launch_block_jacobi<float>(int, int, int, int, int, void* const*, const int*, const int*, const int*,
                                        void* const*, void* const*, const int*, void* const*, const int*, double, int,
                                        int*, long long*, void*, size_t, cudaStream_t);
template int launch_block_jacobi<double>(int, int, int, int, int, void* const*, const int*, const int*, const int*,
                                         void* const*, void* const*, const int*, void* const*, const int*, double, int,
                                         int*, long long*, void*, size_t, cudaStream_t);

}  // namespace bsvd
