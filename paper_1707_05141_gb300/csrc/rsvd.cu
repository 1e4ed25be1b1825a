// rsvd.cu -- batched randomized truncated SVD (Algorithm 4, Section 7), FP32 or FP64.
//
// Every block b (m x n, any shape up to 256 x 256) is processed by one batched pipeline, all
// blocks at once, sizes per block:
//   plan     ||A||_F (FP64 sums), l = k + p for a fixed rank k (Algorithm 4 as stated), else
//            hint + p; a block whose l reaches min(m, n), or passes the sample cap (160 columns
//            in FP32, 128 with tensor-core sampling, 64 in FP64: the small SVD stays in the
//            register / shared tiers), is full
//            rank: it skips the randomized steps and is factored directly at the end.
//   sample   Y = A [Omega | Omega_probe]: Omega (n x l) and 8 probe columns are generated on the
//            fly from Philox (no Omega in memory), one batched GEMM.
//   range    [Q, ~] = qr(Y);  q power steps: Z = A^T Q, Qz = qr(Z), Y = A Qz, Q = qr(Y)
//            (randomized subspace iteration, the robust variant Section 7 mentions).
//   project  B^T = A^T Q (n x l), [Q_B, R_B] = qr(B^T)   (Section 7, phase 2).
//   small    SVD of R_B^T by one-sided Jacobi (register tier for l <= 64, shared tier to 160):
//            R_B^T = U_R S V_R^T, so A ~ Q B = Q R_B^T Q_B^T and U = Q U_R, V = Q_B V_R (the QR
//            writes R_B transposed; one-sided Jacobi on the lower-triangular R_B^T, whose rows are
//            graded like the singular values, converges in fewer sweeps than on R_B: the same
//            effect as the register tier's QR preconditioning).
//   estimate posterior error of the rank-l approximation from the probes (Halko et al. 4.3):
//            est^2 = mean_j ||A w_j - U S V^T w_j||^2.  In tolerance mode, if est > (eps / 2)
//            ||A||_F the block gets p more samples in the next round (the adaptive range
//            finder); past the sample cap it falls back to the full SVD.  A fixed-rank block
//            is done after its one round (the estimate is still reported).
//   finish   tolerance mode: the smallest k with sum_{i >= k} s_i^2 <= (0.95 eps)^2 ||A||_F^2 -
//            4 est^2 (FP64 sums, Section 8.2's relative Frobenius truncation); fixed rank: k;
//            first k columns of U, V and k values of S to the caller.
// Full-rank blocks: min(m, n) <= 64 by A = Q R (A^T when m < n), the register-tier SVD of R^T and
// a batched GEMM for the Q side; up to 128 (FP32) by the shared tier; above by the block-Jacobi
// tier on R^T of a blocked Householder QR.  FP64 runs every stage in FP64 (the Gaussian samples too).
// Every stage runs over a device list of the blocks it concerns.
#include <cuda_runtime.h>

#include "common.cuh"
#include "launch.cuh"
#include "philox.cuh"

namespace bsvd {

constexpr int kProbes = 8;     // probe columns of the posterior estimate
constexpr int kLCapMax = 160;  // largest sample cap (FP32)
constexpr int kMaxDim = 256;

// sample cap (the small l x l SVD stays in the register / shared tiers) and the largest min(m, n)
// the shared tier takes for a full-rank block, per element type
template <typename T> struct RsCap;
template <> struct RsCap<float> { static constexpr int l = 160, smem = 128; };
template <> struct RsCap<double> { static constexpr int l = 64, smem = 64; };

enum { RS_RSVD = 0, RS_FULL = 1, RS_DONE = 2 };

// full-rank blocks above the shared tier: GRAM block Jacobi on R^T of a blocked Householder QR
// (about half the outer sweeps of the block tier on A)
constexpr int kBlockMethod = BSVD_BLOCK_GRAM | BSVD_BLOCK_QR_PRECONDITION;
enum { RSF_FALLBACK = 1, RSF_FROM_FULL = 2, RSF_NO_SCRATCH = 4 };

struct RsState {
    int m, n, k;       // k = min(m, n)
    int ell;           // current number of samples
    int mode;          // RS_*
    int rank, flags, rounds;
    int fixed;         // fixed rank (> 0), or 0: tolerance mode
    int cap;           // sample cap of this call (RsCap<T>::l, or less)
    double eps;        // relative Frobenius tolerance of this block
    double norm2;      // ||A||_F^2
    double est2;       // posterior estimate of ||A - U S V^T||_F^2 (rank ell)
    long long off;     // scratch offset (elements)
    long long size;    // scratch size (elements)
};

// FP64 copies of the small SVD's operands (R, U, V: l64 x l64 each, sigma), l64 = min(l, 64), in
// doubles; FP32 runs keep them after their own pieces for the FP64 small SVD (BSVD_RSVD_SMALL_FP64)
__host__ __device__ inline long long rs_small64_doubles(long long l)
{
    const long long l64 = l < 64 ? l : 64;
    auto al = [](long long x) { return (x + 255) & ~255ll; };
    return 3 * al(l64 * l64) + al(l64);
}

// per-block scratch (elements of the run's type, size bytes each) for bounds m, n and sample cap lcap
__host__ __device__ inline long long rs_scratch_elems(int m, int n, int lcap, int size)
{
    const long long k = m < n ? m : n;
    const long long l = k < lcap ? k : lcap;
    const long long a = 255;  // 256-element alignment of every piece
    auto al = [&](long long x) { return (x + a) & ~a; };
    const long long base = al((long long)m * (l + kProbes)) + al((long long)n * l) + al((long long)n * l) +
                           3 * al(l * l) + al(k) + al((long long)m * k) + al((long long)n * k);
    return base + (size == 4 ? 2 * rs_small64_doubles(l) : 0);
}

// pointer / size arrays handed to the batched QR, Jacobi and GEMM stages
template <typename T>
struct RsArrays {
    T** pY;        // m x (l + probes), ld m          (Y, then Q in its first l columns)
    T** pZ;        // n x l, ld n                     (Z, then Qz)
    T** pBt;       // n x l, ld n                     (B^T, then Q_B)
    T** pR;        // l x l, ld l                     (R of each QR; R_B^T for the small SVD)
    T** pUp;       // l x l, ld l                     (U_R of R_B^T)
    T** pVp;       // l x l, ld l                     (V_R of R_B^T)
    T** pS;        // k                               (singular values)
    T** pUw;       // m x k, ld m                     (U before truncation)
    T** pVw;       // n x k, ld n                     (V before truncation)
    int *m_act, *n_act, *l_act, *lp_act;  // sizes for active randomized blocks (0 otherwise)
    int *l_reg, *l_smem;                  // l for the small SVD: register tier (l <= 64) / shared
    int *ld_m, *ld_n, *ld_l;
    int *m_reg, *n_reg;                   // full-rank blocks with min(m, n) <= 64: QR sizes max(m, n),
                                          // min(m, n) (0 otherwise)
    int *m_smem, *n_smem;                 // ... for the shared tier
    int *m_blk, *n_blk;                   // ... for the block tier (min(m, n) > 128)
    int* info;                            // scratch info of the inner stages
    // full-rank blocks with min(m, n) <= 64 (A = Q R, or A^T = Q R when m < n; SVD of R^T = U~ S V~^T):
    T** pQf;       // Q (max(m,n) x min(m,n), ld max(m,n)): pY, or pBt for A^T
    T** pCf;       // Q V~: U (pUw) for A, V (pVw) for A^T
    T** pDf;       // U~: V (pVw) for A, U (pUw) for A^T
    // FP64 copies for the small SVD in FP64 (FP32 runs): R, U, V (l x l, ld l) and sigma
    double **pR64, **pU64, **pV64, **pS64;
    int *qtr, *ld_q;                      // factor A^T; max(m, n)
    // item lists (see ItemList) built with the arrays: blocks sampling in this round, split by
    // the tier of their small SVD; full-rank blocks of the QR path and of the shared tier
    int *list_act, *list_lreg, *list_lsmem, *list_reg, *list_smem;
    // size-binned lists (RB_* bins, `batch` entries each): the QR and small-SVD stages are launched
    // once per bin with that bin's bounds, so small blocks get the shared memory and threads of
    // their own size (occupancy), not those of the batch's largest
    int* binned;
    int* cnt;                             // list lengths: RL_* then the bins; cnt[kTimeoutSlot]: timeouts
    RsState* st;
};
enum { RL_ACT = 0, RL_LREG, RL_LSMEM, RL_REG, RL_SMEM, RL_COUNT };
// bins: rows (m or n; max(m, n) on the full-rank path) in (0, 64], (64, 128], (128, ...); columns
// (l, or k) in (0, 32], (32, 64], (64, ...)
constexpr int kRowBins = 3, kColBins = 3;
constexpr int RB_QY = RL_COUNT;                         // QR of Y (m x l): 9 bins
constexpr int RB_QZ = RB_QY + kRowBins * kColBins;      // QR of Z and B^T (n x l): 9 bins
constexpr int RB_LREG = RB_QZ + kRowBins * kColBins;    // small SVD, register tier (l <= 32, <= 64)
constexpr int RB_FQR = RB_LREG + 2;                     // full-rank QR path: QR of A (max(m,n) x k), 3 x 3 bins
constexpr int RB_FSVD = RB_FQR + kRowBins * kColBins;   // ... and the SVD of R^T, register tier (k <= 32, <= 64)
constexpr int RB_LSM = RB_FSVD + 2;                     // small SVD, shared tier (l <= 128, above)
constexpr int RB_END = RB_LSM + 2;
constexpr int kBins = RB_END - RL_COUNT;
constexpr int kCounters = 64;                           // list lengths and flags (ints)
constexpr int kTimeoutSlot = kCounters - 1;
static_assert(RB_END <= kTimeoutSlot, "counter slots");

__host__ __device__ inline int rs_row_bin(int r) { return r <= 64 ? 0 : (r <= 128 ? 1 : 2); }
__host__ __device__ inline int rs_col_bin(int c) { return c <= 32 ? 0 : (c <= 64 ? 1 : 2); }
__host__ __device__ inline int rs_row_bound(int b) { return 64 << b; }
__host__ __device__ inline int rs_col_bound(int b) { return 32 << b; }

// ------------------------------------------------------------------------------------------------
// batched GEMM  C (M x N) = op(A) (M x K) * B (K x N), per-block sizes, element type T.
// op(A) = A (column-major, lda) or A^T; B either from memory (column-major, ldb) or, when
// OMEGA, the Gaussian sampling stream: columns c < nOmega from stream 0, the rest from the
// probe stream 1 (column c - nOmega).
// 64 x 64 output tile per CTA, 256 threads with a 4 x 4 register tile, K staged 16 at a time.
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ void lds4(const float* p, float (&r)[4])
{
    const float4 v = *reinterpret_cast<const float4*>(p);
    r[0] = v.x;
    r[1] = v.y;
    r[2] = v.z;
    r[3] = v.w;
}
__device__ __forceinline__ void lds4(const double* p, double (&r)[4])
{
    const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
    r[0] = a.x;
    r[1] = a.y;
    r[2] = b.x;
    r[3] = b.y;
}
__device__ __forceinline__ void gauss4t(unsigned long long seed, uint32_t idx, uint32_t tag, uint32_t g, uint32_t c,
                                        float (&z)[4])
{
    const float4 v = gauss4(seed, idx, tag, g, c);
    z[0] = v.x;
    z[1] = v.y;
    z[2] = v.z;
    z[3] = v.w;
}
__device__ __forceinline__ void gauss4t(unsigned long long seed, uint32_t idx, uint32_t tag, uint32_t g, uint32_t c,
                                        double (&z)[4])
{
    const Gauss4d v = gauss4d(seed, idx, tag, g, c);
    z[0] = v.x;
    z[1] = v.y;
    z[2] = v.z;
    z[3] = v.w;
}

template <typename T, bool TRANS_A, bool OMEGA>
__device__ __forceinline__ void gemm_tile(int b, int tm, int tn, T* const* A, const int* LDA, T* const* B,
                                          const int* LDB, T* const* C, const int* LDC, const int* M, const int* N,
                                          const int* K, const int* NOMEGA, unsigned long long seed)
{
    constexpr int BM = 64, BN = 64, BK = 16;
    __shared__ __align__(16) T As[BK][BM + 4];
    __shared__ __align__(16) T Bs[BK][BN + 4];
    const int Mb = M[b], Nb = N[b], Kb = K[b];
    const int m0 = tm * BM, n0 = tn * BN;
    if (Mb <= 0 || Nb <= 0 || m0 >= Mb || n0 >= Nb) return;
    const T* a = A[b];
    const int lda = LDA[b];
    const T* bm = OMEGA ? nullptr : B[b];
    const int ldb = OMEGA ? 0 : LDB[b];
    const int nom = OMEGA ? NOMEGA[b] : 0;
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;  // 16 x 16 threads, 4 x 4 outputs each
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
    for (int k0 = 0; k0 < Kb; k0 += BK) {
        // A tile: op(A)(m0 + i, k0 + kk), and the B tile B(k0 + kk, n0 + j): each thread's global
        // loads are issued together before any of its shared stores (a store between two loads
        // would make each load wait for the previous one's data)
        constexpr int PA = (BM * BK) / 256, PB = (BK * BN) / 256;
        T xa[PA], xb[PB];
#pragma unroll
        for (int q = 0; q < PA; ++q) {
            const int e = tid + 256 * q;
            int i, kk;
            if (!TRANS_A) {
                i = e % BM;
                kk = e / BM;  // consecutive threads walk down a column of A
            } else {
                kk = e % BK;
                i = e / BK;   // consecutive threads walk down a column of A (= a row of A^T)
            }
            const int gi = m0 + i, gk = k0 + kk;
            xa[q] = (gi < Mb && gk < Kb) ? (TRANS_A ? a[(size_t)gi * lda + gk] : a[(size_t)gk * lda + gi]) : T(0);
        }
        if (!OMEGA) {
#pragma unroll
            for (int q = 0; q < PB; ++q) {
                const int e = tid + 256 * q;
                const int kk = e % BK, j = e / BK;
                const int gk = k0 + kk, gj = n0 + j;
                xb[q] = (gk < Kb && gj < Nb) ? bm[(size_t)gj * ldb + gk] : T(0);
            }
        }
#pragma unroll
        for (int q = 0; q < PA; ++q) {
            const int e = tid + 256 * q;
            const int i = !TRANS_A ? e % BM : e / BK, kk = !TRANS_A ? e / BM : e % BK;
            As[kk][i] = xa[q];
        }
        if (!OMEGA) {
#pragma unroll
            for (int q = 0; q < PB; ++q) {
                const int e = tid + 256 * q;
                Bs[e % BK][e / BK] = xb[q];
            }
        } else {
            // 4 rows per Philox call: BK / 4 = 4 groups x 64 columns = 256 calls, one per thread
            const int g = tid & 3, j = tid >> 2;
            const int gj = n0 + j;
            const int gk0 = k0 + 4 * g;
            T z[4] = {T(0), T(0), T(0), T(0)};
            if (gj < Nb && gk0 < Kb) {
                const bool probe = gj >= nom;
                gauss4t(seed, (uint32_t)b, probe ? 1u : 0u, (uint32_t)(gk0 >> 2), (uint32_t)(probe ? gj - nom : gj), z);
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) Bs[4 * g + r][j] = gk0 + r < Kb ? z[r] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T ar[4], br[4];
            lds4(&As[kk][ty * 4], ar);
            lds4(&Bs[kk][tx * 4], br);
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(ar[i], br[j], acc[i][j]);
        }
        __syncthreads();
    }
    T* c = C[b];
    const int ldc = LDC[b];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int gj = n0 + tx * 4 + j;
        if (gj >= Nb) continue;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int gi = m0 + ty * 4 + i;
            if (gi < Mb) c[(size_t)gj * ldc + gi] = acc[i][j];
        }
    }
}

// persistent over a list of matrices; a CTA computes every output tile of the matrix it claims
template <typename T, bool TRANS_A, bool OMEGA>
__global__ void __launch_bounds__(256) gemm_batched_kernel(ItemList wl, T* const* A, const int* LDA, T* const* B,
                                                           const int* LDB, T* const* C, const int* LDC, const int* M,
                                                           const int* N, const int* K, const int* NOMEGA,
                                                           unsigned long long seed)
{
    for (int b = list_item(wl); b >= 0; b = list_item(wl)) {
        const int tn_count = (N[b] + 63) / 64, tiles = ((M[b] + 63) / 64) * tn_count;
        for (int t = 0; t < tiles; ++t)
            gemm_tile<T, TRANS_A, OMEGA>(b, t / tn_count, t % tn_count, A, LDA, B, LDB, C, LDC, M, N, K, NOMEGA, seed);
    }
}

template <bool TRANS_A, bool OMEGA, typename T>
static int gemm(int batch, ItemList wl, T* const* A, const int* LDA, T* const* B, const int* LDB, T* const* C,
                const int* LDC, const int* M, const int* N, const int* K, const int* NOM, unsigned long long seed,
                cudaStream_t st)
{
    const int grid = item_grid(gemm_batched_kernel<T, TRANS_A, OMEGA>, 256, 0, wl, batch, st);
    if (grid == 0) return BSVD_ERR_CUDA;
    gemm_batched_kernel<T, TRANS_A, OMEGA><<<grid, 256, 0, st>>>(wl, A, LDA, B, LDB, C, LDC, M, N, K, NOM, seed);
    return cudaGetLastError() == cudaSuccess ? BSVD_SUCCESS : BSVD_ERR_CUDA;
}

// ------------------------------------------------------------------------------------------------
// plan: sizes, tolerance, mode, ||A||_F^2, first sample count, scratch sizes
// ------------------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) rs_plan_kernel(int batch, int max_m, int max_n, T* const* A, const int* M,
                                                      const int* N, const int* LDA, const int* fixed, const int* hint,
                                                      const double* tol_arr, double tol, int p, int cap, RsState* st,
                                                      int* info)
{
    const int b = blockIdx.x;
    const int m = M[b], n = N[b], lda = LDA[b];
    const double eps = tol_arr ? tol_arr[b] : tol;
    const bool bad = m < 0 || n < 0 || m > max_m || n > max_n || lda < (m > 1 ? m : 1) || !(eps >= 0.0 && eps < 1.0);
    __shared__ double red[8];
    double s = 0.0;
    if (!bad) {
        const T* a = A[b];
        for (int j = 0; j < n; ++j)
            for (int i = threadIdx.x; i < m; i += blockDim.x) {
                const double x = a[(size_t)j * lda + i];
                s += x * x;
            }
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        RsState r;
        r.m = bad ? 0 : m;
        r.n = bad ? 0 : n;
        r.k = bad ? 0 : (m < n ? m : n);
        int f = fixed ? fixed[b] : 0;
        f = f < 0 ? 0 : (f > kMaxDim ? kMaxDim : f);
        int h = f > 0 ? f : (hint ? hint[b] : 0);
        h = h < 0 ? 0 : (h > kMaxDim ? kMaxDim : h);  // a hint at or above min(m, n) already means full rank
        int l = h + p;
        if (l < 1) l = 1;
        r.ell = l;
        r.mode = bad || r.k == 0 ? RS_DONE : ((l >= r.k || l > cap) ? RS_FULL : RS_RSVD);
        r.cap = cap;
        r.rank = 0;
        r.flags = 0;
        r.rounds = 0;
        r.fixed = f;
        r.eps = bad ? 0.0 : eps;
        r.norm2 = t;
        r.est2 = 0.0;
        r.off = 0;
        // a NaN or infinity in A makes ||A||_F^2 non-finite: flagged, not processed
        const bool nonfinite = !bad && !isfinite(t);
        if (nonfinite) {
            r.m = r.n = r.k = 0;
            r.mode = RS_DONE;
        }
        r.size = bad || nonfinite ? 0 : rs_scratch_elems(m, n, RsCap<T>::l, (int)sizeof(T));
        st[b] = r;
        info[b] = bad ? BSVD_INFO_BAD_SHAPE : (nonfinite ? BSVD_INFO_NONFINITE : 0);
    }
}

// exclusive scan of the scratch sizes (one CTA; batch up to millions in a strided loop); a block
// whose pieces would end past the workspace's capacity is not processed (flag, no writes)
__global__ void __launch_bounds__(1024) rs_scan_kernel(int batch, RsState* st, long long capacity, int* info)
{
    __shared__ long long part[1024];
    const int per = (batch + blockDim.x - 1) / blockDim.x;
    const int b0 = threadIdx.x * per;
    long long s = 0;
    for (int b = b0; b < b0 + per && b < batch; ++b) s += st[b].size;
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = 1; o < (int)blockDim.x; o <<= 1) {
        const long long v = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    long long base = threadIdx.x ? part[threadIdx.x - 1] : 0;
    for (int b = b0; b < b0 + per && b < batch; ++b) {
        st[b].off = base;
        base += st[b].size;
        if (base > capacity && st[b].mode != RS_DONE) {
            st[b].mode = RS_DONE;
            st[b].flags |= RSF_NO_SCRATCH;
            info[b] = BSVD_INFO_NO_SCRATCH;
        }
    }
}

// pointers and per-stage sizes; `final` selects the full-rank pass instead of a sampling round
template <typename T>
__global__ void rs_arrays_kernel(int batch, T* scratch, RsArrays<T> ar, int final)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= batch) return;
    const RsState s = ar.st[b];
    const int m = s.m, n = s.n, k = s.k;
    const int lcap = k < RsCap<T>::l ? k : RsCap<T>::l;
    const long long a = 255;
    auto al = [&](long long x) { return (x + a) & ~a; };
    T* base = scratch + s.off;
    long long o = 0;
    ar.pY[b] = base + o;   o += al((long long)m * (lcap + kProbes));
    ar.pZ[b] = base + o;   o += al((long long)n * lcap);
    ar.pBt[b] = base + o;  o += al((long long)n * lcap);
    ar.pR[b] = base + o;   o += al((long long)lcap * lcap);
    ar.pUp[b] = base + o;  o += al((long long)lcap * lcap);
    ar.pVp[b] = base + o;  o += al((long long)lcap * lcap);
    ar.pS[b] = base + o;   o += al(k);
    ar.pUw[b] = base + o;  o += al((long long)m * k);
    ar.pVw[b] = base + o;  o += al((long long)n * k);
    if (sizeof(T) == 4) {  // 1 KB-aligned: base and every piece are multiples of 256 elements
        const long long l64 = lcap < 64 ? lcap : 64;
        const long long p2 = ((l64 * l64 + 255) & ~255ll);
        double* d = reinterpret_cast<double*>(base + o);
        ar.pR64[b] = d;
        ar.pU64[b] = d + p2;
        ar.pV64[b] = d + 2 * p2;
        ar.pS64[b] = d + 3 * p2;
    }
    const bool act = !final && s.mode == RS_RSVD;
    const int l = act ? s.ell : 0;
    ar.m_act[b] = act ? m : 0;
    ar.n_act[b] = act ? n : 0;
    ar.l_act[b] = l;
    ar.lp_act[b] = act ? l + kProbes : 0;
    ar.l_reg[b] = l <= 64 ? l : 0;
    ar.l_smem[b] = l > 64 ? l : 0;
    ar.ld_m[b] = m > 1 ? m : 1;
    ar.ld_n[b] = n > 1 ? n : 1;
    ar.ld_l[b] = l > 1 ? l : 1;
    const bool full = final && s.mode == RS_FULL;
    const int mm = m > n ? m : n;
    // the QR path: A = Q R, the SVD of R^T (register tier for k <= 64, shared tier above), Q V~
    const bool reg = full && k <= RsCap<T>::smem;
    const bool blk = full && k > RsCap<T>::smem;
    const bool smem = reg && k > 64;  // its SVD of R^T in the shared tier
    const bool wide = m < n;
    ar.m_reg[b] = reg ? mm : 0;
    ar.n_reg[b] = reg ? k : 0;
    ar.qtr[b] = wide ? 1 : 0;
    ar.ld_q[b] = mm > 1 ? mm : 1;
    ar.pQf[b] = wide ? ar.pBt[b] : ar.pY[b];
    ar.pCf[b] = wide ? ar.pVw[b] : ar.pUw[b];
    ar.pDf[b] = wide ? ar.pUw[b] : ar.pVw[b];
    if (reg) ar.ld_l[b] = k > 1 ? k : 1;
    ar.m_smem[b] = 0;
    ar.n_smem[b] = 0;
    ar.m_blk[b] = blk ? m : 0;
    ar.n_blk[b] = blk ? n : 0;
    auto bin_push = [&](int which) {
        const int bi = which - RL_COUNT;
        ar.binned[(size_t)bi * batch + atomicAdd(&ar.cnt[which], 1)] = b;
    };
    if (act) {
        ar.list_act[atomicAdd(&ar.cnt[RL_ACT], 1)] = b;
        bin_push(RB_QY + rs_row_bin(m) * kColBins + rs_col_bin(l));
        bin_push(RB_QZ + rs_row_bin(n) * kColBins + rs_col_bin(l));
        if (l <= 64) {
            ar.list_lreg[atomicAdd(&ar.cnt[RL_LREG], 1)] = b;
            bin_push(RB_LREG + (l <= 32 ? 0 : 1));
        } else {
            ar.list_lsmem[atomicAdd(&ar.cnt[RL_LSMEM], 1)] = b;
            bin_push(RB_LSM + (l <= 128 ? 0 : 1));
        }
    }
    if (reg) {
        ar.list_reg[atomicAdd(&ar.cnt[RL_REG], 1)] = b;
        bin_push(RB_FQR + rs_row_bin(mm) * kColBins + rs_col_bin(k));
        if (!smem) bin_push(RB_FSVD + (k <= 32 ? 0 : 1));
    }
    if (smem) ar.list_smem[atomicAdd(&ar.cnt[RL_SMEM], 1)] = b;
}

// ------------------------------------------------------------------------------------------------
// posterior estimate and the next round's decision (one CTA per active block)
//   E = A Wp - Uw diag(S) (Vw^T Wp)  with A Wp = the probe columns of Y (kept since sampling)
// ------------------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void rs_estimate_item(int b, const RsArrays<T>& ar, unsigned long long seed, int p)
{
    __shared__ T t[kLCapMax][kProbes];   // S (Vw^T Wp)
    __shared__ double red[8];
    RsState* s = ar.st + b;
    if (s->mode != RS_RSVD) return;
    const int m = s->m, n = s->n, l = s->ell;
    const T* Vw = ar.pVw[b];
    const T* Uw = ar.pUw[b];
    const T* S = ar.pS[b];
    const T* Y = ar.pY[b];
    // the probe columns Wp (n x 8), four rows per Philox call
    __shared__ T wp[kMaxDim][kProbes];
    for (int e = threadIdx.x; e < ((n + 3) / 4) * kProbes; e += blockDim.x) {
        const int g = e / kProbes, j = e % kProbes;
        T z[4];
        gauss4t(seed, (uint32_t)b, 1u, (uint32_t)g, (uint32_t)j, z);
#pragma unroll
        for (int r = 0; r < 4; ++r)
            if (4 * g + r < n) wp[4 * g + r][j] = z[r];
    }
    __syncthreads();
    // t(c, j) = S_c * sum_r Vw(r, c) Wp(r, j); one warp per (c, j) pair
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int cj = warp; cj < l * kProbes; cj += 8) {
        const int c = cj / kProbes, j = cj % kProbes;
        T acc = T(0);
        for (int r = lane; r < n; r += 32) acc = fma(Vw[(size_t)c * n + r], wp[r][j], acc);
        acc = warp_sum(acc);
        if (lane == 0) t[c][j] = acc * S[c];
    }
    __syncthreads();
    double e = 0.0;
    for (int ij = threadIdx.x; ij < m * kProbes; ij += blockDim.x) {
        const int i = ij % m, j = ij / m;
        T v = Y[(size_t)(l + j) * m + i];
        for (int c = 0; c < l; ++c) v = fma(-Uw[(size_t)c * m + i], t[c][j], v);
        e += (double)v * (double)v;
    }
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if (lane == 0) red[warp] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < 8; ++w) tot += red[w];
        const double est2 = tot / kProbes;
        s->est2 = est2;
        s->rounds += 1;
        if (s->fixed > 0 || est2 <= 0.25 * s->eps * s->eps * s->norm2) {
            s->mode = RS_DONE;  // fixed rank, or range accepted: finish from this round's factors
        } else {
            const int next = s->ell + p;
            if (next >= s->k || next > s->cap) {
                s->mode = RS_FULL;
                s->est2 = 0.0;
                s->flags |= RSF_FALLBACK;
            } else {
                s->ell = next;
            }
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(256) rs_estimate_kernel(ItemList wl, RsArrays<T> ar, unsigned long long seed, int p)
{
    for (int b = list_item(wl); b >= 0; b = list_item(wl)) rs_estimate_item<T>(b, ar, seed, p);
}

// U~ (k x k, ld k) to the side the GEMM does not write (QR path of the full-rank blocks)
template <typename T>
__global__ void __launch_bounds__(256) rs_copy_kernel(ItemList wl, RsArrays<T> ar)
{
    for (int b = list_item(wl); b >= 0; b = list_item(wl)) {
        const int k = ar.n_reg[b];
        const T* src = ar.pUp[b];
        T* dst = ar.pDf[b];
        for (int e = threadIdx.x; e < k * k; e += blockDim.x) dst[e] = src[e];
    }
}

// FP32 <-> FP64 copies of the small SVD's operands (l = L[b] rows and columns, leading dimension l)
__global__ void __launch_bounds__(256) rs_widen_kernel(ItemList wl, const int* L, float* const* src,
                                                       double* const* dst)
{
    for (int b = list_item(wl); b >= 0; b = list_item(wl)) {
        const int l = L[b];
        const float* s = src[b];
        double* d = dst[b];
        for (int e = threadIdx.x; e < l * l; e += blockDim.x) d[e] = (double)s[e];
    }
}

__global__ void __launch_bounds__(256) rs_narrow_kernel(ItemList wl, const int* L, double* const* S64,
                                                        double* const* U64, double* const* V64, float* const* S,
                                                        float* const* U, float* const* V)
{
    for (int b = list_item(wl); b >= 0; b = list_item(wl)) {
        const int l = L[b];
        for (int e = threadIdx.x; e < l * l; e += blockDim.x) {
            U[b][e] = (float)U64[b][e];
            V[b][e] = (float)V64[b][e];
        }
        for (int e = threadIdx.x; e < l; e += blockDim.x) S[b][e] = (float)S64[b][e];
    }
}

// blocks still sampling after the last round fall back to the full SVD
__global__ void rs_fallback_kernel(int batch, RsState* st)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < batch && st[b].mode == RS_RSVD) {
        st[b].mode = RS_FULL;
        st[b].est2 = 0.0;
        st[b].flags |= RSF_FALLBACK;
    }
}

// ------------------------------------------------------------------------------------------------
// finish: truncation rank and the copy of the first k columns to the caller
// ------------------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) rs_finish_kernel(RsArrays<T> ar, T* const* dU, const int* LDU, T* const* dS,
                                                        T* const* dV, const int* LDV, const int* kmax, int* rank_out,
                                                        float* err_est, int* samples, int* info)
{
    __shared__ int kk;
    const int b = blockIdx.x;
    RsState* s = ar.st + b;
    if (info[b] == BSVD_INFO_BAD_SHAPE) return;
    if (ar.cnt[kTimeoutSlot] != 0) {  // a tensor-core completion wait gave up: the call's results are invalid
        if (threadIdx.x == 0) info[b] = BSVD_INFO_DEVICE_TIMEOUT;
        return;
    }
    if (info[b] == BSVD_INFO_NONFINITE) {
        if (threadIdx.x == 0) rank_out[b] = 0;
        return;
    }
    const int m = s->m, n = s->n;
    if (s->flags & RSF_NO_SCRATCH) return;
    const bool from_full = s->mode == RS_FULL;
    const int ncol = from_full ? s->k : s->ell;  // columns available: all k, or the l samples
    const T* S = ar.pS[b];
    if (threadIdx.x == 0) {
        int k = ncol;
        if (s->fixed > 0) {
            k = s->fixed < ncol ? s->fixed : ncol;  // Algorithm 4: the first k of k + p columns
        } else {
            // smallest k with sum_{i >= k} S_i^2 <= (0.95 eps)^2 ||A||^2 - 4 est^2: the 8-probe
            // estimate of the range error is trusted to a factor 2 (its relative spread is about
            // sqrt(2/8)), and 5% of eps is left for the factorisation's own residual
            const double eps = s->eps;
            double thr = 0.9025 * eps * eps * s->norm2 - 4.0 * s->est2;
            if (thr < 0.0) thr = 0.0;
            double tail = 0.0;
            for (int i = ncol - 1; i >= 0; --i) {
                const double t2 = tail + (double)S[i] * (double)S[i];
                if (t2 > thr) break;
                tail = t2;
                k = i;
            }
        }
        const int cap = kmax[b];
        int fl = (s->flags & RSF_FALLBACK) ? BSVD_INFO_FALLBACK : 0;
        if (k > cap) {
            fl |= BSVD_INFO_RANK_CAPPED;
            k = cap;
        }
        kk = k;
        s->rank = k;
        rank_out[b] = k;
        if (err_est) err_est[b] = s->norm2 > 0.0 ? (float)sqrt(s->est2 / s->norm2) : 0.f;
        if (samples) samples[b] = ncol;
        info[b] = fl | s->rounds;
    }
    __syncthreads();
    const int k = kk;
    const T* Uw = ar.pUw[b];
    const T* Vw = ar.pVw[b];
    T* u = dU[b];
    T* v = dV[b];
    const int ldu = LDU[b], ldv = LDV[b];
    for (int c = 0; c < k; ++c) {
        for (int i = threadIdx.x; i < m; i += blockDim.x) u[(size_t)c * ldu + i] = Uw[(size_t)c * m + i];
        for (int i = threadIdx.x; i < n; i += blockDim.x) v[(size_t)c * ldv + i] = Vw[(size_t)c * n + i];
    }
    for (int c = threadIdx.x; c < k; c += blockDim.x) dS[b][c] = S[c];
}

// ------------------------------------------------------------------------------------------------
// host driver
// ------------------------------------------------------------------------------------------------
struct RsFixed {
    size_t off_state, off_ptr, off_int, off_ctr, off_bjws, bj_bytes, off_scratch;
};

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr int kPtrArrays = 16, kIntArrays = 24;  // the last four pointer arrays hold FP64 pointers

template <typename T>
static RsFixed rs_fixed(int batch, int max_m, int max_n)
{
    RsFixed F;
    size_t o = 0;
    F.off_state = o;
    o = al256(o + sizeof(RsState) * (size_t)batch);
    F.off_ptr = o;
    o = al256(o + sizeof(T*) * (size_t)batch * kPtrArrays);
    F.off_int = o;
    o = al256(o + sizeof(int) * (size_t)batch * (kIntArrays + kBins));
    F.off_ctr = o;
    o = al256(o + sizeof(unsigned long long) * 8 + sizeof(int) * kCounters);  // claim counters, list lengths
    F.off_bjws = o;
    const int kmx = max_m < max_n ? max_m : max_n;
    F.bj_bytes = kmx > RsCap<T>::smem ? block_jacobi_workspace<T>(batch, max_m, max_n, 32, kBlockMethod) : 0;
    o = al256(o + F.bj_bytes);
    F.off_scratch = o;
    return F;
}

template <typename T>
size_t rsvd_workspace(int batch, int max_m, int max_n, const int* h_m, const int* h_n)
{
    const RsFixed F = rs_fixed<T>(batch, max_m, max_n);
    size_t el = 0;
    for (int b = 0; b < batch; ++b) {
        const int m = h_m ? h_m[b] : max_m, n = h_n ? h_n[b] : max_n;
        el += (size_t)rs_scratch_elems(m < 0 ? 0 : m, n < 0 ? 0 : n, RsCap<T>::l, (int)sizeof(T));
    }
    return F.off_scratch + al256(el * sizeof(T));
}

// The small SVD of the listed blocks in FP64: R (l x l FP32, ld l, l = L[b] <= 64) widened, the
// FP64 register tier, U, V, sigma narrowed back to FP32 (FP32 runs only)
template <typename T>
static int small_svd_fp64(int batch, int lmax, const int* L, ItemList wl, const RsArrays<T>& ar, cudaStream_t st)
{
    if constexpr (sizeof(T) != 4) {
        return BSVD_ERR_UNSUPPORTED;
    } else {
        const int gw = item_grid(rs_widen_kernel, 256, 0, wl, batch, st);
        if (gw == 0) return BSVD_ERR_CUDA;
        rs_widen_kernel<<<gw, 256, 0, st>>>(wl, L, ar.pR, ar.pR64);
        if (cudaGetLastError() != cudaSuccess) return BSVD_ERR_CUDA;
        const int rc = launch_jacobi_reg<double>(batch, lmax, lmax, 0, (void* const*)ar.pR64, L, L, L,
                                                 (void* const*)ar.pS64, (void* const*)ar.pU64, L,
                                                 (void* const*)ar.pV64, L, 0.0, 0, ar.info, nullptr, st, wl);
        if (rc) return rc;
        const int gn = item_grid(rs_narrow_kernel, 256, 0, wl, batch, st);
        if (gn == 0) return BSVD_ERR_CUDA;
        rs_narrow_kernel<<<gn, 256, 0, st>>>(wl, L, ar.pS64, ar.pU64, ar.pV64, ar.pS, ar.pUp, ar.pVp);
        return cudaGetLastError() == cudaSuccess ? BSVD_SUCCESS : BSVD_ERR_CUDA;
    }
}

template <typename T>
int launch_rsvd(int batch, int max_m, int max_n, void* const* A, const int* M, const int* N, const int* LDA,
                const int* fixed, const int* hint, const double* tol_arr, double tol, const int* kmax, int p, int q,
                int rounds, unsigned long long seed, int flags, void* const* dU, const int* LDU, void* const* dS,
                void* const* dV, const int* LDV, int* rank_out, float* err_est, int* samples, int* info, void* ws,
                size_t ws_bytes, cudaStream_t st)
{
    if (max_m > kMaxDim || max_n > kMaxDim) return BSVD_ERR_UNSUPPORTED;
    const RsFixed F = rs_fixed<T>(batch, max_m, max_n);
    if (ws_bytes < F.off_scratch) return BSVD_ERR_WORKSPACE;
    unsigned char* w = static_cast<unsigned char*>(ws);
    RsArrays<T> ar;
    ar.st = reinterpret_cast<RsState*>(w + F.off_state);
    T** pp = reinterpret_cast<T**>(w + F.off_ptr);
    T*** slots[12] = {&ar.pY, &ar.pZ, &ar.pBt, &ar.pR, &ar.pUp, &ar.pVp, &ar.pS, &ar.pUw, &ar.pVw,
                      &ar.pQf, &ar.pCf, &ar.pDf};
    for (int i = 0; i < 12; ++i) *slots[i] = pp + (size_t)i * batch;
    double** dp = reinterpret_cast<double**>(pp + (size_t)12 * batch);
    ar.pR64 = dp;
    ar.pU64 = dp + batch;
    ar.pV64 = dp + 2 * (size_t)batch;
    ar.pS64 = dp + 3 * (size_t)batch;
    // the small SVDs (of R_B^T, and of R^T on the full-rank QR path) in FP64: FP32 runs only
    const bool small64 = sizeof(T) == 4 && (flags & BSVD_RSVD_SMALL_FP64) != 0;
    // the sampling product on the tensor cores: FP32 runs only
    const bool tc_sample = sizeof(T) == 4 && (flags & BSVD_RSVD_TC_SAMPLING) != 0;
    // sample cap of this call: the tensor-core sampling kernel takes l <= 128
    const int lcap_run = tc_sample && RsCap<T>::l > 128 ? 128 : RsCap<T>::l;
    int* ip = reinterpret_cast<int*>(w + F.off_int);
    int** islots[kIntArrays] = {&ar.m_act, &ar.n_act, &ar.l_act, &ar.lp_act, &ar.l_reg, &ar.l_smem,
                                &ar.ld_m, &ar.ld_n, &ar.ld_l, &ar.m_reg, &ar.n_reg, &ar.m_smem,
                                &ar.n_smem, &ar.m_blk, &ar.n_blk, &ar.info, &ar.list_act, &ar.list_lreg,
                                &ar.list_lsmem, &ar.list_reg, &ar.list_smem, &ar.qtr, &ar.ld_q, nullptr};
    for (int i = 0; i < kIntArrays; ++i)
        if (islots[i]) *islots[i] = ip + (size_t)i * batch;
    ar.binned = ip + (size_t)kIntArrays * batch;
    T* scratch = reinterpret_cast<T*>(w + F.off_scratch);
    unsigned long long* claim = reinterpret_cast<unsigned long long*>(w + F.off_ctr);  // one launch at a time
    ar.cnt = reinterpret_cast<int*>(claim + 8);
    auto listed = [&](const int* idx, int which) { return ItemList{idx, ar.cnt + which, claim}; };
    auto bin_list = [&](int which) {
        return ItemList{ar.binned + (size_t)(which - RL_COUNT) * batch, ar.cnt + which, claim};
    };
    const long long capacity = (long long)((ws_bytes - F.off_scratch) / sizeof(T));

    // tensor-core waits that gave up (the round memsets clear only the list lengths)
    if (cudaMemsetAsync(ar.cnt + kTimeoutSlot, 0, sizeof(int), st) != cudaSuccess) return BSVD_ERR_CUDA;
    rs_plan_kernel<T><<<batch, 256, 0, st>>>(batch, max_m, max_n, (T* const*)A, M, N, LDA, fixed, hint, tol_arr, tol,
                                             p, lcap_run, ar.st, info);
    rs_scan_kernel<<<1, 1024, 0, st>>>(batch, ar.st, capacity, info);
    if (cudaGetLastError() != cudaSuccess) return BSVD_ERR_CUDA;
    const int tb = (batch + 127) / 128;
    T* const* fA = (T* const*)A;
    const int mx = max_m, nx = max_n;
    const int kx = mx < nx ? mx : nx;
    const int lx = kx < lcap_run ? kx : lcap_run;
    int rc = BSVD_SUCCESS;
    const ItemList act = listed(ar.list_act, RL_ACT);
    // QR of the active blocks' m x l (rows = M) or n x l (rows = N) panels, one launch per size bin
    // that the batch's bounds can populate
    auto qr_binned = [&](int base, int rows_max, T** P, const int* rows, const int* ldp, bool r_t) {
        for (int rb = 0; rb < kRowBins; ++rb) {
            if (rb > 0 && rs_row_bound(rb - 1) >= rows_max) break;
            for (int cb = 0; cb < kColBins; ++cb) {
                if (cb > 0 && rs_col_bound(cb - 1) >= lx) break;
                // the last bins have no upper bound: they take the batch's bounds
                const int rbd = rb < kRowBins - 1 && rs_row_bound(rb) < rows_max ? rs_row_bound(rb) : rows_max;
                if (cb > 0 && rs_col_bound(cb - 1) >= rbd) continue;  // l <= rows: no block in this bin
                int cbd = cb < kColBins - 1 && rs_col_bound(cb) < lx ? rs_col_bound(cb) : lx;
                if (cbd > rbd) cbd = rbd;
                const int e = launch_qr<T>(batch, rbd, cbd, (void* const*)P, rows, ar.l_act, ldp, (void* const*)P,
                                           ldp, (void* const*)ar.pR, ar.ld_l, ar.info, st,
                                           bin_list(base + rb * kColBins + cb), r_t);
                if (e) return e;
            }
        }
        return (int)BSVD_SUCCESS;
    };
    for (int r = 0; r < rounds && rc == BSVD_SUCCESS && lx > 0; ++r) {
        if (cudaMemsetAsync(ar.cnt, 0, sizeof(int) * RB_END, st) != cudaSuccess) return BSVD_ERR_CUDA;
        rs_arrays_kernel<T><<<tb, 128, 0, st>>>(batch, scratch, ar, 0);
        // sample: Y = A [Omega | probes]
        if constexpr (sizeof(T) == 4) {
            if (tc_sample)
                rc = launch_rs_sample_tc(batch, act, fA, LDA, ar.pY, ar.m_act, ar.n_act, ar.l_act, seed,
                                         ar.cnt + kTimeoutSlot, st);
        }
        if (!tc_sample)
            rc = gemm<false, true, T>(batch, act, fA, LDA, nullptr, nullptr, ar.pY, ar.ld_m, ar.m_act, ar.lp_act,
                                      ar.n_act, ar.l_act, seed, st);
        if (rc) break;
        rc = qr_binned(RB_QY, mx, ar.pY, ar.m_act, ar.ld_m, false);
        if (rc) break;
        // q power steps: Z = A^T Q, Qz = qr(Z), Y = A Qz, Q = qr(Y)
        for (int it = 0; it < q && rc == BSVD_SUCCESS; ++it) {
            rc = gemm<true, false, T>(batch, act, fA, LDA, ar.pY, ar.ld_m, ar.pZ, ar.ld_n, ar.n_act, ar.l_act, ar.m_act,
                                      nullptr, seed, st);
            if (rc) break;
            rc = qr_binned(RB_QZ, nx, ar.pZ, ar.n_act, ar.ld_n, false);
            if (rc) break;
            rc = gemm<false, false, T>(batch, act, fA, LDA, ar.pZ, ar.ld_n, ar.pY, ar.ld_m, ar.m_act, ar.l_act,
                                       ar.n_act, nullptr, seed, st);
            if (rc) break;
            rc = qr_binned(RB_QY, mx, ar.pY, ar.m_act, ar.ld_m, false);
        }
        if (rc) break;
        // project: B^T = A^T Q, [Q_B, R_B] = qr(B^T)
        rc = gemm<true, false, T>(batch, act, fA, LDA, ar.pY, ar.ld_m, ar.pBt, ar.ld_n, ar.n_act, ar.l_act, ar.m_act,
                                  nullptr, seed, st);
        if (rc) break;
        rc = qr_binned(RB_QZ, nx, ar.pBt, ar.n_act, ar.ld_n, true);
        if (rc) break;
        // small SVD of R_B^T (l x l): register tier up to 64, shared tier above; with
        // BSVD_RSVD_SMALL_FP64 the register-tier ones in FP64 (operands widened, results narrowed)
        // and the shared-tier ones with FP64 rotation parameters
        for (int cb = 0; cb < 2 && rc == BSVD_SUCCESS; ++cb) {  // l in (0, 32], (32, 64]
            if (cb > 0 && lx <= 32) break;
            const int lr = (32 << cb) < lx ? (32 << cb) : lx;
            const ItemList wl = bin_list(RB_LREG + cb);
            rc = small64 ? small_svd_fp64(batch, lr, ar.l_reg, wl, ar, st)
                         : launch_jacobi_reg<T>(batch, lr, lr, 0, (void* const*)ar.pR, ar.l_reg, ar.l_reg, ar.ld_l,
                                                (void* const*)ar.pS, (void* const*)ar.pUp, ar.ld_l,
                                                (void* const*)ar.pVp, ar.ld_l, 0.0, 0, ar.info, nullptr, st, wl);
        }
        if (rc) break;
        // l in (64, 128] (FP32: the columns-in-registers form of the shared tier) and above 128
        for (int cb = 0; cb < 2 && rc == BSVD_SUCCESS; ++cb) {
            if (lx <= (cb ? 128 : 64)) break;
            const int lb = cb == 0 && lx > 128 ? 128 : lx;
            rc = launch_jacobi_smem<T>(batch, lb, lb, (void* const*)ar.pR, ar.l_smem, ar.l_smem, ar.ld_l,
                                       (void* const*)ar.pS, (void* const*)ar.pUp, ar.ld_l, (void* const*)ar.pVp,
                                       ar.ld_l, 0.0, 0, ar.info, nullptr, st, bin_list(RB_LSM + cb), small64);
        }
        if (rc) break;
        // U = Q U_R, V = Q_B V_R
        rc = gemm<false, false, T>(batch, act, ar.pY, ar.ld_m, ar.pUp, ar.ld_l, ar.pUw, ar.ld_m, ar.m_act, ar.l_act,
                                   ar.l_act, nullptr, seed, st);
        if (rc) break;
        rc = gemm<false, false, T>(batch, act, ar.pBt, ar.ld_n, ar.pVp, ar.ld_l, ar.pVw, ar.ld_n, ar.n_act, ar.l_act,
                                   ar.l_act, nullptr, seed, st);
        if (rc) break;
        const int ge = item_grid(rs_estimate_kernel<T>, 256, 0, act, batch, st);
        if (ge == 0) return BSVD_ERR_CUDA;
        rs_estimate_kernel<T><<<ge, 256, 0, st>>>(act, ar, seed, p);
        if (cudaGetLastError() != cudaSuccess) rc = BSVD_ERR_CUDA;
    }
    if (rc) return rc;
    // full-rank blocks, and blocks whose estimate never passed, by the direct Jacobi tiers
    rs_fallback_kernel<<<tb, 128, 0, st>>>(batch, ar.st);
    if (cudaMemsetAsync(ar.cnt, 0, sizeof(int) * RB_END, st) != cudaSuccess) return BSVD_ERR_CUDA;
    rs_arrays_kernel<T><<<tb, 128, 0, st>>>(batch, scratch, ar, 1);
    if (cudaGetLastError() != cudaSuccess) return BSVD_ERR_CUDA;
    const int mm_x = mx > nx ? mx : nx;
    if (kx > 0) {
        // min(m, n) <= 128 (FP32; 64 in FP64): A (A^T when m < n) = Q R with R written transposed,
        // the SVD of R^T = U~ S V~^T (R^T: the preconditioned form; register tier for k <= 64, shared
        // tier above), then A = (Q V~) S U~^T: the Q side by the batched GEMM, U~ copied
        const ItemList qlist = listed(ar.list_reg, RL_REG);
        const int kq = kx < RsCap<T>::smem ? kx : RsCap<T>::smem;
        for (int rb = 0; rb < kRowBins; ++rb) {  // QR of A (A^T): max(m, n) x k, by size bin
            if (rb > 0 && rs_row_bound(rb - 1) >= mm_x) break;
            const int rbd = rb < kRowBins - 1 && rs_row_bound(rb) < mm_x ? rs_row_bound(rb) : mm_x;
            for (int cb = 0; cb < kColBins; ++cb) {
                if (cb > 0 && rs_col_bound(cb - 1) >= kq) break;
                if (cb > 0 && rs_col_bound(cb - 1) >= rbd) continue;  // k <= rows
                int cbd = cb < kColBins - 1 && rs_col_bound(cb) < kq ? rs_col_bound(cb) : kq;
                if (cbd > rbd) cbd = rbd;
                rc = launch_qr<T>(batch, rbd, cbd, A, ar.m_reg, ar.n_reg, LDA, (void* const*)ar.pQf, ar.ld_q,
                                  (void* const*)ar.pR, ar.ld_l, ar.info, st, bin_list(RB_FQR + rb * kColBins + cb),
                                  true, ar.qtr);
                if (rc) return rc;
            }
        }
        const int kr = kq < 64 ? kq : 64;
        for (int cb = 0; cb < 2; ++cb) {  // SVD of R^T: k x k, register tier by size bin
            if (cb > 0 && kr <= 32) break;
            const int kb = (32 << cb) < kr ? (32 << cb) : kr;
            const ItemList wl = bin_list(RB_FSVD + cb);
            rc = small64 ? small_svd_fp64(batch, kb, ar.n_reg, wl, ar, st)
                         : launch_jacobi_reg<T>(batch, kb, kb, 0, (void* const*)ar.pR, ar.n_reg, ar.n_reg, ar.ld_l,
                                                (void* const*)ar.pS, (void* const*)ar.pUp, ar.ld_l,
                                                (void* const*)ar.pVp, ar.ld_l, 0.0, 0, ar.info, nullptr, st, wl);
            if (rc) return rc;
        }
        if (kq > 64) {  // 64 < k <= 128: the SVD of R^T in the shared tier
            rc = launch_jacobi_smem<T>(batch, kq, kq, (void* const*)ar.pR, ar.n_reg, ar.n_reg, ar.ld_l,
                                       (void* const*)ar.pS, (void* const*)ar.pUp, ar.ld_l, (void* const*)ar.pVp,
                                       ar.ld_l, 0.0, 0, ar.info, nullptr, st, listed(ar.list_smem, RL_SMEM), small64);
            if (rc) return rc;
        }
        rc = gemm<false, false, T>(batch, qlist, ar.pQf, ar.ld_q, ar.pVp, ar.ld_l, ar.pCf, ar.ld_q, ar.m_reg, ar.n_reg,
                                   ar.n_reg, nullptr, seed, st);
        if (rc) return rc;
        {
            const int gc = item_grid(rs_copy_kernel<T>, 256, 0, qlist, batch, st);
            if (gc == 0) return BSVD_ERR_CUDA;
            rs_copy_kernel<T><<<gc, 256, 0, st>>>(qlist, ar);
            if (cudaGetLastError() != cudaSuccess) return BSVD_ERR_CUDA;
        }
        if (kx > RsCap<T>::smem) {
            // the block tier keeps its own list of live matrices: blocks not routed to it are 0 x 0
            rc = launch_block_jacobi<T>(batch, mx, nx, 32, kBlockMethod, A, ar.m_blk, ar.n_blk, LDA, (void* const*)ar.pS,
                                        (void* const*)ar.pUw, ar.ld_m, (void* const*)ar.pVw, ar.ld_n, 0.0, 0, ar.info,
                                        nullptr, w + F.off_bjws, F.bj_bytes, st);
            if (rc) return rc;
        }
    }
    rs_finish_kernel<T><<<batch, 256, 0, st>>>(ar, (T* const*)dU, LDU, (T* const*)dS, (T* const*)dV, LDV, kmax,
                                               rank_out, err_est, samples, info);
    return cudaGetLastError() == cudaSuccess ? BSVD_SUCCESS : BSVD_ERR_CUDA;
}

template size_t rsvd_workspace<float>(int, int, int, const int*, const int*);
template size_t rsvd_workspace<double>(int, int, int, const int*, const int*);
template int launch_rsvd<float>(int, int, int, void* const*, const int*, const int*, const int*, const int*,
                                const int*, const double*, double, const int*, int, int, int, unsigned long long, int,
                                void* const*, const int*, void* const*, void* const*, const int*, int*, float*, int*,
                                int*, void*, size_t, cudaStream_t);
template int launch_rsvd<double>(int, int, int, void* const*, const int*, const int*, const int*, const int*,
                                 const int*, const double*, double, const int*, int, int, int, unsigned long long, int,
                                 void* const*, const int*, void* const*, void* const*, const int*, int*, float*, int*,
                                 int*, void*, size_t, cudaStream_t);

}  // namespace bsvd
