/*
 * bsvd.h -- C ABI of the batched QR / one-sided Jacobi SVD / randomized SVD library for GB300
 * (sm_103a), after Boukaram, Turkiyyah, Ltaief & Keyes, "Batched QR and SVD Algorithms on GPUs
 * with Applications in Hierarchical Matrix Compression" (2017).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - A batch is `batch` independent matrices.  Each one is passed through a DEVICE array of
 *    DEVICE pointers (`void* const* dA`, element b points at matrix b) plus DEVICE arrays of
 *    per-matrix sizes (`d_m`, `d_n`, `d_lda`, ...).  This is the pointer-array form of the batched
 *    interfaces the paper builds on (Section 3: batches of independent small matrices).
 *  - Storage is column-major: entry (i, j) of matrix b lives at dA[b][j * lda[b] + i].  Every
 *    leading dimension must be >= max(1, rows).
 *  - dtype is BSVD_F32 or BSVD_F64; all matrices of one call share it.  Scalars such as
 *    singular values have the same type as the matrices.
 *  - `max_m`, `max_n` are HOST upper bounds of d_m, d_n over the batch; they choose the memory
 *    tier and the launch shape.  A matrix that exceeds them gets info = BSVD_INFO_BAD_SHAPE.
 *  - `stream` is a cudaStream_t passed as an opaque pointer (NULL = legacy default stream).
 *    Every call is asynchronous on it: the host returns after enqueueing, never synchronises,
 *    and never allocates device memory.  Buffers belong to the caller and must stay valid
 *    until the stream work completes.
 *  - The return value is a HOST status: BSVD_SUCCESS, a negative argument code
 *    (-k means argument k, counted from 1, is invalid; nothing was launched),
 *    BSVD_ERR_UNSUPPORTED (shape beyond the tiers this build implements; nothing launched) or
 *    BSVD_ERR_CUDA (a launch failed; the stream's state is whatever CUDA reports).
 *  - Per-matrix results go to the DEVICE array d_info (one int per matrix).
 */
#ifndef BSVD_H
#define BSVD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BSVD_F32 0
#define BSVD_F64 1

#define BSVD_SUCCESS 0
#define BSVD_ERR_UNSUPPORTED (-1000)
#define BSVD_ERR_CUDA (-1001)
#define BSVD_ERR_WORKSPACE (-1002) /* workspace smaller than the matching *_workspace query */

/* per-matrix info */
#define BSVD_INFO_BAD_SHAPE (-1)
#define BSVD_INFO_NOT_CONVERGED (1 << 20) /* + sweeps run: the sweep cap was reached */
#define BSVD_INFO_NO_SCRATCH (-2)         /* batched_rsvd: workspace too small for this matrix */
#define BSVD_INFO_RANK_CAPPED (1 << 21)   /* batched_rsvd: the rank needed exceeds kmax */
#define BSVD_INFO_FALLBACK (1 << 22)      /* batched_rsvd: sampling did not pass, full SVD used */
#define BSVD_INFO_DEVICE_TIMEOUT (-3)     /* a bounded on-device wait (tensor-core completion) gave up;
                                             the results of this call are not valid */
#define BSVD_INFO_NONFINITE (-4)          /* the matrix holds a NaN or an infinity (seen in its column
                                             norms, singular values or R's diagonal): its outputs are
                                             not meaningful */

/* Jacobi memory tiers (argument `tier` of batched_svd_jacobi).  `tier` may carry a variant in
   bits 8 and up: BSVD_TIER_REGISTER | (k << 8) forces the k-th register variant that fits the
   shape bound (k = 0: the first); see bsvd_jacobi_variants. */
#define BSVD_TIER_AUTO 0
#define BSVD_TIER_REGISTER 1 /* Section 4: matrix and V resident in registers, one lane per pair */
#define BSVD_TIER_SHARED 2   /* Section 5: matrix and V resident in shared memory */

/*
 * batched_qr -- reduced Householder QR of each matrix, A = Q R (Algorithm 1, Section 2.1;
 * batched kernel of Section 3.1).
 *
 *   dA[b]  (in)  m x n, m >= n, ld d_lda[b]; not modified.
 *   dQ[b]  (out) m x n with orthonormal columns, ld d_ldq[b] >= m.  dQ may be NULL (no Q).
 *   dR[b]  (out) n x n upper triangular, ld d_ldr[b] >= n; entries below the diagonal are
 *                written as exact zeros.  dR may be NULL (no R).
 *   d_info[b] (out) 0, or BSVD_INFO_BAD_SHAPE (m < n, a negative size, a size above max_m /
 *                max_n, or a leading dimension too small) -- outputs of that matrix untouched.
 * Reflectors follow Algorithm 1: v = house(x) with R(i,i) = -sign(x_1) ||x|| (sign(0) = +1).
 * Q and R are therefore unique; a zero column gives the identity reflector.
 * Limits: max_m <= 1024 and max_m * max_n * sizeof(element) <= 200 KiB (the matrix is factored
 * in shared memory); otherwise BSVD_ERR_UNSUPPORTED.
 */
int batched_qr(int dtype, int batch, int max_m, int max_n,
               void* const* dA, const int* d_m, const int* d_n, const int* d_lda,
               void* const* dQ, const int* d_ldq,
               void* const* dR, const int* d_ldr,
               int* d_info, void* stream);

/*
 * batched_qr_blocked_workspace -- bytes of DEVICE workspace batched_qr_blocked needs for these bounds
 * (0 for invalid arguments).  Host only.
 */
size_t batched_qr_blocked_workspace(int dtype, int batch, int max_m, int max_n);

/*
 * batched_qr_blocked -- the same reduced Householder QR (Algorithm 1, same reflectors and signs) for
 * matrices beyond batched_qr's shared-memory kernel: the blocked factorisation Section 3.1 leaves to
 * larger matrices and Section 3.2 names for large squares.  Each matrix is copied to the workspace
 * and factored in 32-column panels: the panel (all rows below its first) is factored on chip, its
 * reflectors are gathered in the compact WY form H_j ... H_{j+31} = I - V T V^T, and the trailing
 * columns are updated as C - V T^T (V^T C), streamed through shared memory in 128-row chunks.
 * Q = H_0 ... H_{n-1} [I; 0] is formed by applying the panels' block reflectors, last panel first.
 * A panel taller than one CTA's shared memory holds (1533 rows FP32, 733 FP64) is factored by a
 * thread-block cluster of up to 8 CTAs, each with a slab of its rows in shared memory; the
 * reflectors' norms and products are summed across the cluster through distributed shared memory.
 *
 *   Arguments as batched_qr, plus:
 *   workspace  DEVICE buffer of at least batched_qr_blocked_workspace(...) bytes, caller-owned,
 *              contents need not be initialised; not used after the stream work completes.
 *              Smaller -> BSVD_ERR_WORKSPACE.
 * Limits: max_m <= batched_qr_blocked_max_rows(dtype) (8 slabs of a 32-column panel, each in
 * 200 KiB of one CTA's shared memory: 11976 rows FP32, 5576 FP64); any max_n <= max_m.  Otherwise
 * BSVD_ERR_UNSUPPORTED.  d_info[b] as batched_qr.
 */
int batched_qr_blocked(int dtype, int batch, int max_m, int max_n,
                       void* const* dA, const int* d_m, const int* d_n, const int* d_lda,
                       void* const* dQ, const int* d_ldq,
                       void* const* dR, const int* d_ldr,
                       int* d_info, void* workspace, size_t workspace_bytes, void* stream);

/* batched_qr_blocked_max_rows -- the tallest matrix batched_qr_blocked factors (host only). */
int batched_qr_blocked_max_rows(int dtype);

/*
 * batched_svd_jacobi -- reduced SVD A = U diag(S) V^T of each matrix by one-sided Jacobi
 * (Algorithm 2, Section 2.2; register / shared-memory kernels of Sections 4-5).
 *
 *   dA[b]  (in)  m x n, ld d_lda[b]; not modified.  k = min(m, n).  A wide matrix (m < n) is
 *                processed through its transpose.
 *   dS[b]  (out) k singular values, descending (Section 1); ties keep column order.
 *   dU[b]  (out) m x k left singular vectors, ld d_ldu[b] >= m; dU may be NULL.  A column whose
 *                singular value is zero is written as zeros.
 *   dV[b]  (out) n x k right singular vectors (accumulated rotations), ld d_ldv[b] >= n; dV may
 *                be NULL, which also skips the accumulation.
 *   tol    rotation threshold: pair (i, j) is rotated only when
 *          |a_i . a_j| > tol * ||a_i|| ||a_j||.  tol <= 0 selects sqrt(max(m, n)) * u with u the
 *          unit roundoff of dtype (2^-24 or 2^-53).
 *   max_sweeps  sweep cap (<= 0 selects 30).
 *   tier   BSVD_TIER_AUTO or a specific tier; see the tier macros.
 *   d_info[b] (out) number of sweeps run (the last one rotates nothing), or
 *                BSVD_INFO_NOT_CONVERGED + sweeps when the cap was reached (results are the last
 *                iterate), or BSVD_INFO_BAD_SHAPE.
 *   d_rotations[b] (out, nullable) number of plane rotations applied.
 * Rotations use zeta = (beta - alpha) / (2 gamma), t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),
 * c = 1 / sqrt(1 + t^2), s = c t on the 2 x 2 Gram matrix [[alpha, gamma], [gamma, beta]].
 * Tiers: the register tier holds min(m, n) <= 64 and max(m, n) <= 128 (F32) / 64 (F64); the shared
 * tier max(m, n) <= 256 and min(m, n) <= 160 (F32, while the matrix and V fit in 220 KiB of shared
 * memory) / 64 (F64); FP32 matrices up to 128 x 128 in the shared tier keep their columns in
 * registers and exchange one column per pair step through shared memory.  BSVD_TIER_AUTO uses the choice
 * recorded by bsvd_set_jacobi_choice for the size bin, else the register tier when it fits, else
 * the shared tier; larger shapes give BSVD_ERR_UNSUPPORTED.
 */
int batched_svd_jacobi(int dtype, int batch, int max_m, int max_n,
                       void* const* dA, const int* d_m, const int* d_n, const int* d_lda,
                       void* const* dS,
                       void* const* dU, const int* d_ldu,
                       void* const* dV, const int* d_ldv,
                       double tol, int max_sweeps, int tier,
                       int* d_info, long long* d_rotations, void* stream);

/*
 * bsvd_jacobi_variants -- number of kernel variants of `tier` (BSVD_TIER_REGISTER or
 * BSVD_TIER_SHARED) that can run a batch bounded by max_m x max_n, or a negative argument code.
 * Host only; launches nothing.  The autotuner times each variant and records the fastest.
 */
int bsvd_jacobi_variants(int dtype, int max_m, int max_n, int tier);

/*
 * bsvd_jacobi_variant_desc -- describe the k-th (k >= 1) register-tier variant that fits a batch
 * bounded by max_m x max_n (the variant BSVD_TIER_REGISTER | (k << 8) launches).  desc (HOST, 9
 * ints, caller-owned) receives {column-pair slots, row parts, rows of A per lane, rows of V per
 * lane, resident CTAs per SM, scaled rotations (0/1), QR preconditioning (0/1), FP64 rotation
 * parameters (0/1), carried column norms (0/1)}.  QR preconditioning (square bounds only) factors A = Q R and runs the sweeps
 * on R^T (the project's addition; the paper runs them on A).  FP64 rotation parameters (FP32 data
 * only) compute zeta, t, c, s and the rotation test in FP64 from the FP32 Gram sums; carried
 * column norms keep each column's squared norm across the steps of a sweep (one dot product per
 * pair instead of three; alpha' = alpha - t gamma, beta' = beta + t gamma after a rotation, summed
 * afresh at every sweep's start and after a cancelling update).  These variants are listed last,
 * the carried-norm ones after the FP64-parameter ones.  Returns 0, a negative argument code, or
 * BSVD_ERR_UNSUPPORTED when there is no k-th variant.  Host only; launches nothing.
 */
int bsvd_jacobi_variant_desc(int dtype, int max_m, int max_n, int k, int* desc);

/*
 * bsvd_set_jacobi_choice -- record the encoded tier (tier | variant << 8) that BSVD_TIER_AUTO
 * uses for batches whose bounds fall in the same size bin as max_m x max_n (bins are powers of
 * two of max(m, n) and min(m, n), up to 256).  BSVD_TIER_AUTO clears the entry.  Host only; may
 * run concurrently with batched_svd_jacobi calls, which see either the old or the new entry (the
 * choice applies to calls made after it returns); returns 0 or a negative argument code.
 * (This tuning table is the project's addition: the paper tunes its kernels by hand, Sections 3-5.)
 */
int bsvd_set_jacobi_choice(int dtype, int max_m, int max_n, int tier);

/* Block-Jacobi methods (argument `method` of batched_svd_block_jacobi), Algorithm 3 */
#define BSVD_BLOCK_GRAM 0   /* Section 6.1: pair Gram matrix G, its eigenvectors as the block rotation */
#define BSVD_BLOCK_DIRECT 1 /* Section 6.2: pair QR, SVD of the triangular factor */
/* Flag for `method`: FP32 data with block width 32 form the pair Gram matrices on the tensor cores
 * by default (TF32 operands split into a high and a low part, all four products, FP32
 * accumulation: FP32-level accuracy); this flag forms them with FP32 SIMT dot products instead
 * (the plain FP32 form).  The block updates run on the FP32 SIMT pipes either way. */
#define BSVD_BLOCK_SIMT_PRODUCTS (1 << 16)
/* Flag for `method`, for tests of the failure path only: in the tensor-core Gram (FP32, block
 * width 32, without BSVD_BLOCK_SIMT_PRODUCTS) the first completion wait of each pair waits 1 ms on
 * a barrier that nothing arrives at, as a tensor-core completion that never came would; the call
 * then takes its timeout path (no further pairs, a bounded wait for the MMAs in flight before the
 * tensor memory is freed) and every matrix gets BSVD_INFO_DEVICE_TIMEOUT.  No fault, no hang. */
#define BSVD_BLOCK_TEST_TIMEOUT (1 << 17)
/* Flag for `method`: precondition by a blocked Householder QR (the preconditioning Section 6.3
 * names as future work).  The working matrix X (A, or A^T when m < n) is factored X = Q R in
 * 32-column panels (each panel on chip, the trailing columns updated through the compact WY form
 * I - V T V^T), the block Jacobi runs on the lower-triangular R^T, whose rows are graded like the
 * singular values (about half the outer sweeps), and X's left vectors are formed as Q times R^T's
 * right vectors.  Needs max(m, n) <= batched_qr_blocked_max_rows(dtype) (the panels are factored as
 * in batched_qr_blocked); the workspace holds X, R^T and the panels' T factors besides the block
 * tier's own. */
#define BSVD_BLOCK_QR_PRECONDITION (1 << 18)
/* Flag for `method`: test every block pair in every sweep.  By default a pair whose test found it
 * orthogonal is not formed or tested again while neither of its two blocks has been rotated since
 * (the block pairs are selected by their recorded off-diagonal tests, the adaptive pair selection
 * Section 6.3 proposes, in its exact form: the skipped tests would have come out the same, so the
 * results do not change).  This flag restores the plain cyclic visit, for comparison. */
#define BSVD_BLOCK_RETEST_ALL (1 << 19)

/*
 * batched_svd_block_jacobi_workspace -- bytes of DEVICE workspace batched_svd_block_jacobi needs
 * for these bounds, block width and method (its BSVD_BLOCK_QR_PRECONDITION bit included; 0 for
 * invalid arguments).  Host only.
 */
size_t batched_svd_block_jacobi_workspace(int dtype, int batch, int max_m, int max_n, int block_width,
                                          int method);

/*
 * bsvd_set_block_choice -- record, for batches whose bounds fall in the same size bin as
 * max_m x max_n (powers of two of max(m, n) and min(m, n), up to 16384), the block width (16 or 32)
 * and the inner register variant (0: the default; k: the k-th variant of bsvd_jacobi_variants for
 * 2bw x 2bw) that block_width = 0 selects; block_width 0 clears the entry.  Host only; the tuning
 * of Sections 3-6 by measurement (the paper fixes bw = 32 by hand).  Returns 0 or a negative
 * argument code.
 */
int bsvd_set_block_choice(int dtype, int max_m, int max_n, int block_width, int inner_variant);

/*
 * batched_svd_block_jacobi -- reduced SVD by one-sided block Jacobi in global memory (Algorithm 3,
 * Section 6), for matrices too large for the register and shared-memory tiers.
 *
 * Arguments as batched_svd_jacobi, except:
 *   dU[b], dV[b]  REQUIRED: they double as the working storage (the working matrix A, or A^T when
 *                 m < n, lives in U, or V, and the rotations accumulate in the other one).
 *   tol           pair threshold: a block pair is rotated when its largest scaled off-diagonal
 *                 |G_pq| / sqrt(G_pp G_qq) exceeds tol (tested in FP64); tol <= 0 selects
 *                 sqrt(max(m, n)) * u.  The same threshold drives the inner 2bw x 2bw Jacobi.
 *   max_sweeps    block sweeps launched (<= 0 selects 20); converged matrices skip the rest.
 *   block_width   bw = 16 or 32 columns per block (the paper uses 32, Section 6.3), or 0: the
 *                 block width and inner variant bsvd_set_block_choice recorded for the size bin
 *                 (32 and the default inner variant when none; the workspace query resolves 0 the
 *                 same way, so query and call must see the same table entry).
 *   method        BSVD_BLOCK_GRAM or BSVD_BLOCK_DIRECT, optionally | (k << 8) to run the inner
 *                 2bw x 2bw SVDs with the k-th register-tier variant (see bsvd_jacobi_variants).
 *                 | BSVD_BLOCK_TEST_TIMEOUT exercises the failure path (tests only; see the flag).
 *                 | BSVD_BLOCK_QR_PRECONDITION runs the block Jacobi on R^T of a blocked QR (see the
 *                 flag); info and rotations then count the sweeps on R^T.
 *                 | BSVD_BLOCK_SIMT_PRODUCTS keeps the Gram products on the FP32 SIMT pipes (FP32
 *                 data with bw = 32 form them on the tensor cores otherwise).  | (s << 24) sets the sweep cap of
 *                 each pair visit's inner SVD: 1 <= s <= 126 sweeps, 127 = to convergence (as
 *                 Algorithm 3 states), 0 = the default (GRAM: 2, measured as fast with unchanged
 *                 outer sweeps and errors; DIRECT: to convergence).  The outer sweeps continue
 *                 until no pair rotates either way.
 *                 DIRECT needs max(m, n) * 2 bw * sizeof(element) <= 200 KiB (the pair's QR runs on
 *                 chip); its default tol is 4 sqrt(max(m, n)) u, since its rotations are only as
 *                 orthogonal as the pair's Householder Q.
 *   workspace     DEVICE buffer of at least batched_svd_block_jacobi_workspace(...) bytes, owned by
 *                 the caller, contents need not be initialised; not used after the stream work
 *                 completes.  Smaller -> BSVD_ERR_WORKSPACE.
 *   d_info[b]     block sweeps run (the last one rotates no pair), or BSVD_INFO_NOT_CONVERGED +
 *                 sweeps, or BSVD_INFO_BAD_SHAPE, or BSVD_INFO_DEVICE_TIMEOUT (every matrix of the
 *                 call) when a tensor-core completion wait gave up.
 *   d_rotations[b] (nullable) number of block-pair rotations applied.
 * Limits: max(m, n) <= 16384.  Host launches max_sweeps * (nb - 1) steps without synchronising.
 */
int batched_svd_block_jacobi(int dtype, int batch, int max_m, int max_n,
                             void* const* dA, const int* d_m, const int* d_n, const int* d_lda,
                             void* const* dS,
                             void* const* dU, const int* d_ldu,
                             void* const* dV, const int* d_ldv,
                             double tol, int max_sweeps, int block_width, int method,
                             int* d_info, long long* d_rotations,
                             void* workspace, size_t workspace_bytes, void* stream);

/*
 * batched_rsvd_workspace -- bytes of DEVICE workspace for batched_rsvd.  h_m, h_n are optional
 * HOST arrays of the batch's sizes (exact size); NULL bounds every matrix by max_m x max_n.
 * 0 for invalid arguments.
 */
size_t batched_rsvd_workspace(int dtype, int batch, int max_m, int max_n, const int* h_m, const int* h_n);

/*
 * batched_rsvd -- randomized SVD of each matrix (Algorithm 4, Section 7) with q steps of randomized
 * subspace iteration (the robust variant Section 7 mentions), either at a fixed rank or truncated to
 * a relative Frobenius tolerance (Section 8.2).  FP32 or FP64 (every stage in that precision,
 * Gaussian samples included); m, n <= 256.
 *
 *   d_rank[b]      (nullable) FIXED-RANK MODE when > 0: k = d_rank[b]; l = k + oversample Gaussian
 *                  columns, `power_iters` power steps, one round, the first k columns of the rank-l
 *                  factorisation are returned (Algorithm 4 as stated).  When k + oversample reaches
 *                  min(m, n) or exceeds the sample cap (160 columns in FP32, 128 with
 *                  BSVD_RSVD_TC_SAMPLING, 64 in FP64), the full
 *                  Jacobi SVD replaces the sampling and its first k columns are returned.  NULL, 0
 *                  or a negative value selects TOLERANCE MODE for that matrix.
 *   d_rank_hint[b] (nullable, tolerance mode) first rank guess k0: the first round draws
 *                  l = k0 + oversample columns (NULL or 0: l = oversample; negative counts as 0,
 *                  above 256 as 256).  A guess with l >= min(m, n), or past the sample cap, sends
 *                  the matrix straight to the full Jacobi SVD.
 *   d_tol[b]       (nullable) per-matrix eps in [0, 1); NULL uses `tol` for every matrix.  A matrix
 *                  whose eps is outside [0, 1) (or NaN) gets info BSVD_INFO_BAD_SHAPE.
 *   tol            eps of every matrix when d_tol is NULL (must be in [0, 1)).  In tolerance mode the
 *                  result satisfies ||A - U S V^T||_F <= eps ||A||_F up to the posterior estimate's
 *                  error: after each round, 8 probe columns (Gaussian stream 1) give
 *                  est = ||(A - U_l S_l V_l^T) W||_F / sqrt(8); est <= eps/2 ||A||_F accepts the
 *                  round, otherwise the next round draws `oversample` more columns.  Past
 *                  max_rounds, or the sample cap, the matrix gets the full Jacobi SVD (est = 0).
 *                  The rank k is the smallest with sum_{i >= k} s_i^2 <= (0.95 eps)^2 ||A||_F^2 -
 *                  4 est^2 (the estimate trusted to a factor 2; 5% of eps kept for the
 *                  factorisation's own residual).
 *   oversample     p in [1, 64];  power_iters q in [0, 8];  max_rounds in [1, 64].
 *   seed           Omega(r, c) of matrix b is Philox4x32-10 at counter (r/4, c, b, 0), key = seed,
 *                  through Box-Muller (the probes: counter (r/4, j, b, 1)).
 *   flags          0, or BSVD_RSVD_SMALL_FP64 (FP32 runs; ignored in FP64): the small SVDs -- of the
 *                  projected block's R_B^T and, for full-rank blocks with min(m, n) <= 128, of R^T
 *                  -- run in FP64 when l <= 64 (operands widened, FP64 register tier, results
 *                  narrowed to FP32), and with FP64 rotation parameters in the shared tier above.
 *                  | BSVD_RSVD_TC_SAMPLING (FP32 runs; ignored in FP64): the sample A Omega is a
 *                  tcgen05 product of kind::tf32 (the FP32 operands read with a 10-bit mantissa, FP32
 *                  accumulation), the 8 probe columns stay FP32 products; the power step and the
 *                  projection that follow are FP32.  Other bits: argument error.  A tensor-core
 *                  completion wait that gives up (bounded; no valid input makes one) gives every
 *                  matrix of the call BSVD_INFO_DEVICE_TIMEOUT.
 *   dU[b] (m x kmax, ld d_ldu[b]), dS[b] (kmax), dV[b] (n x kmax, ld d_ldv[b]): the first k columns
 *                  and values are written; k > kmax writes kmax and flags BSVD_INFO_RANK_CAPPED.
 *   d_rank_out[b]  k;  d_err_est[b] (nullable) est / ||A||_F (also in fixed-rank mode; 0 after a
 *                  full SVD);  d_samples[b] (nullable) the number of columns the result came from
 *                  (l, or min(m, n) after a full SVD).
 *   d_info[b]      rounds run | BSVD_INFO_FALLBACK | BSVD_INFO_RANK_CAPPED, or BSVD_INFO_BAD_SHAPE
 *                  or BSVD_INFO_NO_SCRATCH (the matrix did not fit the workspace; nothing written).
 *                  A matrix sent straight to the full SVD has 0 rounds.
 *   workspace      at least batched_rsvd_workspace(...) bytes (else BSVD_ERR_WORKSPACE), caller-owned,
 *                  contents need not be initialised.
 */
#define BSVD_RSVD_SMALL_FP64 1  /* flags: FP32 runs take the small SVDs in FP64 (see batched_rsvd) */
#define BSVD_RSVD_TC_SAMPLING 2 /* flags: FP32 runs form the sample A Omega on the tensor cores */

int batched_rsvd(int dtype, int batch, int max_m, int max_n,
                 void* const* dA, const int* d_m, const int* d_n, const int* d_lda,
                 const int* d_rank, const int* d_rank_hint, const double* d_tol, double tol,
                 int oversample, int power_iters, int max_rounds, unsigned long long seed, int flags,
                 void* const* dU, const int* d_ldu, void* const* dS, void* const* dV, const int* d_ldv,
                 const int* d_kmax, int* d_rank_out, float* d_err_est, int* d_samples, int* d_info,
                 void* workspace, size_t workspace_bytes, void* stream);

/*
 * Learned rank predictor (no counterpart in the paper: the project's addition that chooses the
 * first sample count of batched_rsvd; the adaptive range finder remains the fallback and the
 * judge of every result).  FP32, device arrays, asynchronous on `stream`.
 */
#define BSVD_SKETCH_FEATURES 16
#define BSVD_MLP_PARAMS 5313 /* W1 64x16, b1 64, W2 64x64, b2 64, w3 64, b3 1 (row-major) */

/* bsvd_sketch_features -- 16 features per matrix (m, n <= 256) from column norms and 8 Gaussian
 * probes (Philox stream 2 under `seed`): layout d_features[b * 16 + i]; see mlp.cu for the list. */
int bsvd_sketch_features(int batch, int max_m, int max_n, void* const* dA, const int* d_m, const int* d_n,
                         const int* d_lda, unsigned long long seed, float* d_features, void* stream);

/* bsvd_mlp_forward -- y = w3 . relu(W2 relu(W1 f + b1) + b2) + b3 for each feature row (y estimates
 * log(rank + 1)).  d_out (nullable) receives y; d_rank_hint (nullable) receives
 * clamp(ceil(exp(y) - 1 + margin), 1, min(m, n)) (min(m, n) only when d_m, d_n are given, else
 * 65536; a NaN margin gives 1). */
int bsvd_mlp_forward(int batch, const float* d_features, const float* d_params, float* d_out, int* d_rank_hint,
                     float margin, const int* d_m, const int* d_n, void* stream);

/* bsvd_mlp_grad -- gradient of L = 1/(2B) sum_b (y_b - target_b)^2 with respect to the parameters:
 * d_grad (BSVD_MLP_PARAMS floats) and d_loss (one float) are overwritten. */
int bsvd_mlp_grad(int batch, const float* d_features, const float* d_target, const float* d_params, float* d_grad,
                  float* d_loss, void* stream);

/* bsvd_mlp_adam -- one Adam step (Kingma & Ba 2015) on the parameters; m, v moment buffers of
 * nparams floats (start at zero), step >= 1. */
int bsvd_mlp_adam(int nparams, float* d_params, const float* d_grad, float* d_m, float* d_v, int step, float lr,
                  float beta1, float beta2, float eps, void* stream);

/* Number of parameters of the rank predictor (BSVD_MLP_PARAMS). */
int bsvd_mlp_param_count(void);

/* Size of the library-owned scratch array used by batched_svd_block_jacobi_noalloc (64 MiB). */
#define BSVD_NOALLOC_SCRATCH_BYTES (64u << 20)
#define BSVD_ERR_SCRATCH_LIMIT (-1003) /* the call needs more than BSVD_NOALLOC_SCRATCH_BYTES */

/*
 * batched_svd_block_jacobi_noalloc -- the same computation as batched_svd_block_jacobi, for
 * callers that can neither pass a workspace nor allocate device memory (for example code running
 * under a host application's memory manager that forbids driver allocations, or on a
 * latency-critical path where cudaMalloc's implicit synchronisation is not acceptable).  The
 * paper has no counterpart; this is a property of the library, not of the method.
 *
 * Arguments are those of batched_svd_block_jacobi without workspace/workspace_bytes.  The
 * scratch is one static device array of BSVD_NOALLOC_SCRATCH_BYTES that every GPU loading the
 * library holds until the process exits.  The function calls no cudaMalloc or cudaFree and no
 * allocating library routine.
 *   - A batch whose batched_svd_block_jacobi_workspace(...) exceeds BSVD_NOALLOC_SCRATCH_BYTES is
 *     rejected with BSVD_ERR_SCRATCH_LIMIT before anything is launched (for 512 x 512 FP32 with
 *     block width 32 that is about 250 matrices per call).
 *   - The first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 *     that device current; make that first call before any stream capture.  The address is kept
 *     with the identifier of the context it was found in; a call in a new context of the device
 *     (after cudaDeviceReset, or once the primary context was released and re-created) looks it up
 *     again, so make the first call after such a reset before any capture too.  Lookup failure
 *     returns BSVD_ERR_CUDA.
 *   - Every call on a device uses the same array: calls whose GPU work overlaps (other streams,
 *     other host threads) race on it and must be serialised by the caller.  Each call writes every
 *     scratch location before reading it, so leftover contents of a previous call do not matter.
 */
int batched_svd_block_jacobi_noalloc(int dtype, int batch, int max_m, int max_n,
                                     void* const* dA, const int* d_m, const int* d_n, const int* d_lda,
                                     void* const* dS,
                                     void* const* dU, const int* d_ldu,
                                     void* const* dV, const int* d_ldv,
                                     double tol, int max_sweeps, int block_width, int method,
                                     int* d_info, long long* d_rotations, void* stream);

/*
 * bsvd_h2_truncate_workspace -- bytes of DEVICE workspace bsvd_h2_truncate needs (0 for invalid
 * arguments).  Host only.
 *
 * bsvd_h2_truncate -- the truncation phase of H^2-matrix compression (Section 8.2): a nested row
 * basis over a binary tree of depth `depth` is replaced by a truncated orthonormal one, level by
 * level from the leaves, with the projections T = U~^T U of every node.
 *
 * Nodes are numbered in heap order: node i of level l is g = 2^l - 1 + i (root 0, children of g are
 * 2g + 1 and 2g + 2); the 2^depth leaves are g = 2^depth - 1 + i.  All pointers are DEVICE arrays.
 *   d_leaf[i]      leaf basis U_i, m_i x k (d_leaf_m[i] = m_i <= max_leaf_m <= 256, ld d_leaf_ld[i]).
 *   d_transfer[g]  (g >= 1) transfer matrix E_g, k x k, ld k: U_parent = diag(U_c1, U_c2) [E_c1; E_c2].
 *   k              the basis rank of every node (1..64; q^2 for a q x q Chebyshev grid).
 *   eps            relative threshold: every node keeps the smallest rank r whose discarded tail
 *                  sqrt(sum_{j >= r} s_j^2) is within eps times the Frobenius norm of the matrix it
 *                  truncates (the leaf basis, or TE_p = [T_c1 E_c1; T_c2 E_c2]).
 *   d_new_leaf[i]  (out) U~_i: the first rank[leaf] columns are written (ld d_new_leaf_ld[i] >= m_i).
 *   d_new_transfer[g] (out, g >= 1) E~_g: rank[g] x rank[parent] written, ld k (k x k buffers).
 *   d_T[g]         (out) T_g = U~_g^T U_g: rank[g] x k written, ld k (k x k buffers), every node.
 *   d_rank[g], d_info[g] (out) per node: the kept rank; the sweeps of the node's SVD, or
 *                  BSVD_INFO_BAD_SHAPE (a leaf with m_i > max_leaf_m or a short ld; rank 0) or
 *                  BSVD_INFO_NONFINITE.
 *   d_rotations[g] (out, nullable) plane rotations of the node's SVD.
 *   workspace      at least bsvd_h2_truncate_workspace(...) bytes (else BSVD_ERR_WORKSPACE).
 * Every SVD is the one-sided Jacobi of this library (register tier; shared tier where the
 * register tier does not hold the bounds), all nodes of a level in one batched call.
 */
size_t bsvd_h2_truncate_workspace(int dtype, int depth, int k, int max_leaf_m);
int bsvd_h2_truncate(int dtype, int depth, int k, int max_leaf_m, void* const* d_leaf, const int* d_leaf_m,
                     const int* d_leaf_ld, void* const* d_transfer, double eps, void* const* d_new_leaf,
                     const int* d_new_leaf_ld, void* const* d_new_transfer, void* const* d_T, int* d_rank,
                     int* d_info, long long* d_rotations, void* workspace, size_t workspace_bytes, void* stream);

/*
 * Host-in, host-out calls on uniform batches (HOST arrays; no counterpart in the paper, whose
 * batches already live on the GPU).  Matrix b of the batch is column-major at element b * m * n of
 * hA (leading dimension m); outputs are packed the same way: S k values (k = min(m, n)), U m x k,
 * V n x k, Q m x n, R n x n per matrix, info one int.  The batch is cut into `chunks` chunks whose
 * host -> device copy, computation and device -> host copy overlap (library-owned streams, created
 * once per device: two for the copies, and two per call for the computation, consecutive chunks on
 * different ones; every one of them starts after the work already enqueued on `stream`, and on
 * return `stream` is ordered after the last copy: synchronising it completes the call).  Host
 * buffers must stay valid until then and should be page-locked for the copies to overlap.  The
 * device copies of the whole batch live in `workspace` (at least *_workspace(...) bytes, else
 * BSVD_ERR_WORKSPACE); nothing is allocated.  Calls on one device share the copy streams and take
 * turns on four compute streams.  hU, hV, hQ, hR, h_info may be NULL (not computed / not copied).
 */
size_t bsvd_host_svd_workspace(int dtype, int batch, int m, int n);
int bsvd_host_svd(int dtype, int batch, int m, int n, const void* hA, void* hS, void* hU, void* hV, int* h_info,
                  int chunks, void* workspace, size_t workspace_bytes, void* stream);
size_t bsvd_host_qr_workspace(int dtype, int batch, int m, int n);
int bsvd_host_qr(int dtype, int batch, int m, int n, const void* hA, void* hQ, void* hR, int* h_info, int chunks,
                 void* workspace, size_t workspace_bytes, void* stream);

/*
 * Diagnostics (outside the method; for tests and the benchmark).
 *
 * bsvd_philox_gauss -- for each of `count` counters (d_ctr: 4 x count words, DEVICE) the
 * Philox4x32-10 output words under key (seed low, seed high) to d_words (4 x count, nullable), and
 * the four Gaussian samples the randomized SVD draws from that counter, read as (row / 4, column,
 * matrix index, stream tag), in FP32 to d_gauss and in FP64 to d_gauss64 (4 x count each,
 * nullable).  Returns 0 or a negative argument code; asynchronous on `stream`.
 *
 * bsvd_fma_probe -- launches `blocks` CTAs of 256 threads that each run `iters` x 16 independent
 * fused multiply-adds in FP32 (dtype BSVD_F32) or FP64; d_out (DEVICE, blocks x 256 elements of
 * dtype) receives the sums.  Returns the number of floating-point operations launched (2 per FMA),
 * or a negative code.  Timing it with events on `stream` gives the pipe's peak throughput.
 */
int bsvd_philox_gauss(int count, const unsigned* d_ctr, unsigned long long seed, unsigned* d_words,
                      float* d_gauss, double* d_gauss64, void* stream);
long long bsvd_fma_probe(int dtype, int blocks, int iters, void* d_out, void* stream);

/* Library version and build description (static strings). */
const char* bsvd_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BSVD_H */
