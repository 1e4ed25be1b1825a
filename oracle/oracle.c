/*
 * oracle.c -- plain, slow FP64 CPU reference for the batched Householder QR, the one-sided Jacobi
 * SVD and the randomized SVD of Boukaram, Turkiyyah, Ltaief & Keyes, "Batched QR and SVD
 * Algorithms on GPUs with Applications in Hierarchical Matrix Compression" (2017).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package's smoke check and the benchmark's CPU
 * baseline leg load this library.  It shares no code, header or constant with the CUDA library,
 * and neither side includes or links the other.
 *
 * Everything is FP64, column-major with an explicit leading dimension, one matrix per call,
 * written for a reader to check against the paper by eye: no blocking, no fusion, no reordering
 * beyond what each algorithm states.  The batch drivers at the end only spread independent
 * matrices over POSIX threads.
 *
 * Readings of the paper where it is silent (each one also listed in the design notes):
 *  - house(x): v = x + sign(x1) ||x|| e1 with sign(0) = +1, normalised to unit length so that
 *    the reflector is I - 2 v v^T as Algorithm 1 writes it; a zero x gives v = 0 (identity).
 *  - rot(G) in Algorithm 2: the Rutishauser form zeta = (beta - alpha) / (2 gamma),
 *    t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), c = 1 / sqrt(1 + t^2), s = c t, applied as
 *    [a_i, a_j] <- [c a_i - s a_j, s a_i + c a_j]; a pair is skipped when
 *    |gamma| <= tol sqrt(alpha beta) or when alpha or beta is zero.
 *  - pair order: row-cyclic (i < j lexicographic), the serial order of Section 4.
 *  - convergence: a sweep that performs no rotation; at most max_sweeps sweeps.
 *  - singular values sorted descending (Section 1), ties kept in column order.
 *  - right singular vectors by accumulating the rotations on the identity (Section 2.2).
 *  - randomized SVD to a tolerance: Algorithm 4 in rounds of p samples, judged by an 8-probe
 *    posterior estimate (Halko, Martinsson & Tropp 2011, Sec. 4.3-4.4), with a full-SVD fallback
 *    and a budgeted truncation; the constants are stated beside orc_rsvd_adaptive.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define AT(A, ld, i, j) ((A)[(size_t)(j) * (size_t)(ld) + (size_t)(i)])

#define ORC_NOT_CONVERGED (1 << 20)

/* ---------------------------------------------------------------------------------------------
 * small helpers
 * ------------------------------------------------------------------------------------------- */

/* 2-norm of x, scaled by max |x_i| so that squares cannot overflow or underflow. */
double orc_nrm2(int len, const double* x, int inc)
{
    double scale = 0.0, ssq = 0.0;
    for (int i = 0; i < len; ++i) {
        double a = fabs(x[(size_t)i * inc]);
        if (a > scale) scale = a;
    }
    if (scale == 0.0) return 0.0;
    for (int i = 0; i < len; ++i) {
        double r = x[(size_t)i * inc] / scale;
        ssq += r * r;
    }
    return scale * sqrt(ssq);
}

/* C = op(A) * op(B), plain triple loop; op = transpose when the flag is set.
   op(A) is p x r, op(B) is r x q, C is p x q. */
void orc_gemm(int ta, int tb, int p, int q, int r,
              const double* A, int lda, const double* B, int ldb, double* C, int ldc)
{
    for (int j = 0; j < q; ++j)
        for (int i = 0; i < p; ++i) {
            double acc = 0.0;
            for (int l = 0; l < r; ++l) {
                double a = ta ? AT(A, lda, l, i) : AT(A, lda, i, l);
                double b = tb ? AT(B, ldb, j, l) : AT(B, ldb, l, j);
                acc += a * b;
            }
            AT(C, ldc, i, j) = acc;
        }
}

/* ---------------------------------------------------------------------------------------------
 * Householder QR -- Algorithm 1 (Section 2.1)
 * ------------------------------------------------------------------------------------------- */

/* house(x): unit v with (I - 2 v v^T) x = -sign(x1) ||x|| e1; v = 0 when x = 0. */
void orc_house(int len, const double* x, double* v)
{
    double alpha = orc_nrm2(len, x, 1);
    if (alpha == 0.0) {
        for (int i = 0; i < len; ++i) v[i] = 0.0;
        return;
    }
    for (int i = 0; i < len; ++i) v[i] = x[i];
    v[0] += (x[0] >= 0.0 ? alpha : -alpha);
    double nv = orc_nrm2(len, v, 1);
    for (int i = 0; i < len; ++i) v[i] /= nv;
}

/* Reduced QR of an m x n matrix, m >= n >= 0, exactly as Algorithm 1: start from [Q, R] = [I, A];
   for each column i: v = house(R(i)) on rows i..m-1, R = (I - 2vv^T) R, Q = Q (I - 2vv^T).
   Outputs the first n columns of Q (m x n) and the leading n x n upper triangle of R (entries
   below the diagonal stored as exact zeros).  Returns 0, or -1 for a bad shape. */
int orc_qr(int m, int n, const double* A, int lda, double* Q, int ldq, double* R, int ldr)
{
    if (m < 0 || n < 0 || m < n || lda < m || ldq < m || ldr < n) return -1;
    if (n == 0) return 0;
    double* Rw = (double*)malloc(sizeof(double) * (size_t)m * n);
    double* Qw = (double*)malloc(sizeof(double) * (size_t)m * m);
    double* v = (double*)malloc(sizeof(double) * (size_t)m);
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < m; ++i) AT(Rw, m, i, j) = AT(A, lda, i, j);
    for (int j = 0; j < m; ++j)
        for (int i = 0; i < m; ++i) AT(Qw, m, i, j) = (i == j) ? 1.0 : 0.0;

    for (int i = 0; i < n; ++i) {
        /* v = house(R(i)), zero above row i */
        for (int r = 0; r < i; ++r) v[r] = 0.0;
        orc_house(m - i, &AT(Rw, m, i, i), v + i);
        /* R = (I - 2 v v^T) R */
        for (int j = 0; j < n; ++j) {
            double w = 0.0;
            for (int r = 0; r < m; ++r) w += v[r] * AT(Rw, m, r, j);
            for (int r = 0; r < m; ++r) AT(Rw, m, r, j) -= 2.0 * w * v[r];
        }
        /* Q = Q (I - 2 v v^T) */
        for (int r = 0; r < m; ++r) {
            double w = 0.0;
            for (int c = 0; c < m; ++c) w += AT(Qw, m, r, c) * v[c];
            for (int c = 0; c < m; ++c) AT(Qw, m, r, c) -= 2.0 * w * v[c];
        }
    }
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < m; ++i) AT(Q, ldq, i, j) = AT(Qw, m, i, j);
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) AT(R, ldr, i, j) = (i <= j) ? AT(Rw, m, i, j) : 0.0;
    free(Rw);
    free(Qw);
    free(v);
    return 0;
}

/* ---------------------------------------------------------------------------------------------
 * One-sided Jacobi SVD -- Algorithm 2 (Section 2.2)
 * ------------------------------------------------------------------------------------------- */

/* rot(G) for G = [[alpha, gamma], [gamma, beta]]: returns 0 (no rotation) or 1 with (c, s). */
int orc_rot(double alpha, double beta, double gamma, double tol, double* c, double* s)
{
    if (alpha == 0.0 || beta == 0.0) return 0;
    if (fabs(gamma) <= tol * sqrt(alpha) * sqrt(beta)) return 0;
    double zeta = (beta - alpha) / (2.0 * gamma);
    double t;
    if (fabs(zeta) > 1e150)
        t = 0.5 / zeta; /* 1 / (|zeta| + sqrt(1 + zeta^2)) -> 1 / (2 |zeta|), sign(zeta) kept */
    else
        t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
    *c = 1.0 / sqrt(1.0 + t * t);
    *s = *c * t;
    return 1;
}

/* Cyclic one-sided Jacobi on W (m x n, m >= n, overwritten) accumulating V (n x n).
   Returns the number of sweeps run (the last one performs no rotation) or
   ORC_NOT_CONVERGED + max_sweeps. */
static int jacobi_core(int m, int n, double* W, int ldw, double* V, int ldv, double tol,
                       int max_sweeps, long long* rotations)
{
    long long rots = 0;
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) AT(V, ldv, i, j) = (i == j) ? 1.0 : 0.0;
    int sweep = 0;
    int converged = 0;
    while (sweep < max_sweeps) {
        int rot_this_sweep = 0;
        for (int i = 0; i < n - 1; ++i)
            for (int j = i + 1; j < n; ++j) {
                /* G = A_ij^T A_ij */
                double alpha = 0.0, beta = 0.0, gamma = 0.0;
                for (int r = 0; r < m; ++r) {
                    double ai = AT(W, ldw, r, i), aj = AT(W, ldw, r, j);
                    alpha += ai * ai;
                    beta += aj * aj;
                    gamma += ai * aj;
                }
                double c, s;
                if (!orc_rot(alpha, beta, gamma, tol, &c, &s)) continue;
                /* A_ij = A_ij R, and the same on V */
                for (int r = 0; r < m; ++r) {
                    double ai = AT(W, ldw, r, i), aj = AT(W, ldw, r, j);
                    AT(W, ldw, r, i) = c * ai - s * aj;
                    AT(W, ldw, r, j) = s * ai + c * aj;
                }
                for (int r = 0; r < n; ++r) {
                    double vi = AT(V, ldv, r, i), vj = AT(V, ldv, r, j);
                    AT(V, ldv, r, i) = c * vi - s * vj;
                    AT(V, ldv, r, j) = s * vi + c * vj;
                }
                ++rot_this_sweep;
            }
        ++sweep;
        rots += rot_this_sweep;
        if (rot_this_sweep == 0) {
            converged = 1;
            break;
        }
    }
    if (rotations) *rotations = rots;
    return converged ? sweep : ORC_NOT_CONVERGED + sweep;
}

/* Reduced SVD A = U diag(S) V^T of an m x n matrix by Algorithm 2.  k = min(m, n):
   S (k), U (m x k), V (n x k); U or V may be NULL.  A wide matrix (m < n) is handled through its
   transpose.  tol <= 0 selects sqrt(max(m, n)) * 2^-53.  Returns the sweep count (or
   ORC_NOT_CONVERGED + sweeps), or -1 for a bad shape. */
int orc_jacobi_svd(int m, int n, const double* A, int lda, double tol, int max_sweeps,
                   double* S, double* U, int ldu, double* V, int ldv, long long* rotations)
{
    if (m < 0 || n < 0 || lda < (m > 0 ? m : 1)) return -1;
    int tr = (m < n);
    int mm = tr ? n : m, nn = tr ? m : n; /* working shape, mm >= nn */
    if (tol <= 0.0) tol = sqrt((double)mm) * ldexp(1.0, -53);
    if (rotations) *rotations = 0;
    if (nn == 0) return 0;
    double* W = (double*)malloc(sizeof(double) * (size_t)mm * nn);
    double* Vw = (double*)malloc(sizeof(double) * (size_t)nn * nn);
    for (int j = 0; j < nn; ++j)
        for (int i = 0; i < mm; ++i) AT(W, mm, i, j) = tr ? AT(A, lda, j, i) : AT(A, lda, i, j);

    int info = jacobi_core(mm, nn, W, mm, Vw, nn, tol, max_sweeps, rotations);

    /* sigma_j = ||w_j||, u_j = w_j / sigma_j, then a stable descending sort */
    double* sig = (double*)malloc(sizeof(double) * nn);
    int* perm = (int*)malloc(sizeof(int) * nn);
    for (int j = 0; j < nn; ++j) {
        sig[j] = orc_nrm2(mm, &AT(W, mm, 0, j), 1);
        perm[j] = j;
    }
    for (int a = 1; a < nn; ++a) { /* insertion sort: stable */
        int p = perm[a];
        int b = a - 1;
        while (b >= 0 && sig[perm[b]] < sig[p]) {
            perm[b + 1] = perm[b];
            --b;
        }
        perm[b + 1] = p;
    }
    double* Ul = tr ? V : U; /* left vectors of the working matrix */
    int ldul = tr ? ldv : ldu;
    double* Vr = tr ? U : V;
    int ldvr = tr ? ldu : ldv;
    for (int q = 0; q < nn; ++q) {
        int j = perm[q];
        S[q] = sig[j];
        if (Ul) {
            for (int i = 0; i < mm; ++i)
                AT(Ul, ldul, i, q) = (sig[j] > 0.0) ? AT(W, mm, i, j) / sig[j] : 0.0;
        }
        if (Vr) {
            for (int i = 0; i < nn; ++i) AT(Vr, ldvr, i, q) = AT(Vw, nn, i, j);
        }
    }
    free(sig);
    free(perm);
    free(W);
    free(Vw);
    return info;
}

/* ---------------------------------------------------------------------------------------------
 * Counter-based random numbers for the sampling matrix Omega (Section 7: Omega = Rand(n, k+p)).
 * Philox4x32-10 from its published definition (Salmon, Moraes, Dror & Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC 2011): ten rounds of two 32x32->64 multiplies, key bumped by
 * the Weyl constants between rounds.  Normals by Box & Muller (1958).
 * ------------------------------------------------------------------------------------------- */

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * x2;
        uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)p1;
        uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)p0;
        x0 = y0;
        x1 = y1;
        x2 = y2;
        x3 = y3;
    }
    out[0] = x0;
    out[1] = x1;
    out[2] = x2;
    out[3] = x3;
}

/* Gaussian entry (row, col) of the sampling stream `tag` of matrix `index` under `seed`:
   counter (row / 4, col, index, tag), key (seed low word, seed high word); the four words give
   two Box-Muller pairs (w0, w1) -> rows 4g, 4g+1 and (w2, w3) -> rows 4g+2, 4g+3, with uniforms
   u = (w + 1/2) 2^-32 and z = sqrt(-2 ln u_a) (cos, sin)(2 pi u_b). */
double orc_gauss(uint64_t seed, uint32_t index, uint32_t tag, uint32_t row, uint32_t col)
{
    uint32_t ctr[4] = {row >> 2, col, index, tag};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    int sub = row & 3;
    uint32_t wa = w[(sub >> 1) * 2], wb = w[(sub >> 1) * 2 + 1];
    double ua = ((double)wa + 0.5) * ldexp(1.0, -32);
    double ub = ((double)wb + 0.5) * ldexp(1.0, -32);
    double r = sqrt(-2.0 * log(ua));
    double th = 2.0 * 3.14159265358979323846 * ub;
    return (sub & 1) ? r * sin(th) : r * cos(th);
}

/* Omega(row, c) for c in [c0, c0 + cols), n rows, column-major into O (ld = n). */
void orc_omega(uint64_t seed, uint32_t index, uint32_t tag, int n, int c0, int cols, double* O)
{
    for (int c = 0; c < cols; ++c)
        for (int r = 0; r < n; ++r) AT(O, n, r, c) = orc_gauss(seed, index, tag, (uint32_t)r, (uint32_t)(c0 + c));
}

/* ---------------------------------------------------------------------------------------------
 * Randomized SVD -- Algorithm 4 (Section 7), with q steps of randomized subspace (power)
 * iteration as the more robust variant Section 7 mentions (each product followed by a QR, as in
 * Halko, Martinsson & Tropp 2011, Alg. 4.4).
 * ------------------------------------------------------------------------------------------- */

/* Orthonormal basis Q (m x l) of range(A Omega) after q power steps.  Needs l <= min(m, n). */
int orc_range_basis(int m, int n, const double* A, int lda, const double* Omega, int l, int q,
                    double* Q)
{
    double* Y = (double*)malloc(sizeof(double) * (size_t)m * l);
    double* Z = (double*)malloc(sizeof(double) * (size_t)n * l);
    double* Qz = (double*)malloc(sizeof(double) * (size_t)n * l);
    double* Rt = (double*)malloc(sizeof(double) * (size_t)l * l);
    orc_gemm(0, 0, m, l, n, A, lda, Omega, n, Y, m);          /* Y = A Omega      */
    int rc = orc_qr(m, l, Y, m, Q, m, Rt, l);                 /* [Q, R_y] = qr(Y) */
    for (int it = 0; it < q && rc == 0; ++it) {
        orc_gemm(1, 0, n, l, m, A, lda, Q, m, Z, n);          /* Z = A^T Q        */
        rc = orc_qr(n, l, Z, n, Qz, n, Rt, l);
        if (rc) break;
        orc_gemm(0, 0, m, l, n, A, lda, Qz, n, Y, m);         /* Y = A qr(Z).Q    */
        rc = orc_qr(m, l, Y, m, Q, m, Rt, l);
    }
    free(Y);
    free(Z);
    free(Qz);
    free(Rt);
    return rc;
}

/* Given the basis Q (m x l): B = Q^T A; [Q_B, R_B] = qr(B^T); [U_R, S, V_R] = svd(R_B^T);
   U = Q U_R (m x l), V = Q_B V_R (n x l).  Returns the Jacobi info of the small SVD. */
int orc_rsvd_finish(int m, int n, const double* A, int lda, const double* Q, int l,
                    double* U, double* S, double* V)
{
    double* B = (double*)malloc(sizeof(double) * (size_t)l * n);
    double* Bt = (double*)malloc(sizeof(double) * (size_t)n * l);
    double* QB = (double*)malloc(sizeof(double) * (size_t)n * l);
    double* RB = (double*)malloc(sizeof(double) * (size_t)l * l);
    double* RBt = (double*)malloc(sizeof(double) * (size_t)l * l);
    double* UR = (double*)malloc(sizeof(double) * (size_t)l * l);
    double* VR = (double*)malloc(sizeof(double) * (size_t)l * l);
    orc_gemm(1, 0, l, n, m, Q, m, A, lda, B, l);              /* B = Q^T A        */
    for (int j = 0; j < l; ++j)
        for (int i = 0; i < n; ++i) AT(Bt, n, i, j) = AT(B, l, j, i);
    orc_qr(n, l, Bt, n, QB, n, RB, l);                        /* [Q_B, R_B] = qr(B^T) */
    for (int j = 0; j < l; ++j)
        for (int i = 0; i < l; ++i) AT(RBt, l, i, j) = AT(RB, l, j, i);
    int info = orc_jacobi_svd(l, l, RBt, l, -1.0, 60, S, UR, l, VR, l, NULL);
    orc_gemm(0, 0, m, l, l, Q, m, UR, l, U, m);               /* U = Q U_R   */
    orc_gemm(0, 0, n, l, l, QB, n, VR, l, V, n);              /* V = Q_B V_R */
    free(B);
    free(Bt);
    free(QB);
    free(RB);
    free(RBt);
    free(UR);
    free(VR);
    return info;
}

/* Fixed-width randomized SVD: Omega = the first l columns of sampling stream 0 of `index`.
   U (m x l), S (l), V (n x l).  Needs 1 <= l <= min(m, n).  Returns the small SVD's info or -1. */
int orc_rsvd(int m, int n, const double* A, int lda, uint64_t seed, uint32_t index, int l, int q,
             double* U, double* S, double* V)
{
    if (l < 1 || l > m || l > n) return -1;
    double* Om = (double*)malloc(sizeof(double) * (size_t)n * l);
    double* Q = (double*)malloc(sizeof(double) * (size_t)m * l);
    orc_omega(seed, index, 0, n, 0, l, Om);
    int rc = orc_range_basis(m, n, A, lda, Om, l, q, Q);
    int info = rc ? -1 : orc_rsvd_finish(m, n, A, lda, Q, l, U, S, V);
    free(Om);
    free(Q);
    return info;
}

/* Truncation rank (Section 8.2): the smallest k with sqrt(sum_{i >= k} S_i^2) <= eps * normA,
   S descending; the tail sums run from the smallest value up. */
int orc_trunc_rank(int len, const double* S, double normA, double eps)
{
    double thr = eps * normA;
    double thr2 = thr * thr;
    double tail = 0.0;
    int k = len;
    for (int i = len - 1; i >= 0; --i) {
        double t = tail + S[i] * S[i];
        if (t > thr2) break;
        tail = t;
        k = i;
    }
    return k;
}

/* ---------------------------------------------------------------------------------------------
 * Adaptive randomized SVD to a relative Frobenius tolerance.  Section 7 runs Algorithm 4 with a
 * fixed sample count; the adaptive form follows Halko, Martinsson & Tropp (2011), Sec. 4.3-4.4,
 * which the paper cites for the method: a posterior estimate of the range error decides whether
 * more samples are drawn.  The constants are the library's reading of it:
 *  - r = 8 probe columns w_j, Gaussian stream 1 of the matrix (stream 0 is Omega);
 *  - est^2 = (1/r) sum_j ||(A - U S V^T) w_j||^2 (unbiased for ||A - U S V^T||_F^2);
 *  - a round with l samples is accepted when est <= (eps / 2) ||A||_F;
 *  - otherwise l grows by p; when l would reach min(m, n) or exceed lcap, or after max_rounds
 *    rounds, the matrix takes the full Jacobi SVD (est = 0 then);
 *  - the rank is the smallest k with sum_{i >= k} s_i^2 <= (0.95 eps)^2 ||A||_F^2 - 4 est^2 (the
 *    estimate trusted to a factor 2 in est, 5% of eps kept for the factorisation's own error).
 * ------------------------------------------------------------------------------------------- */

#define ORC_PROBES 8

/* est^2 = (1/r) sum_j ||A w_j - U diag(S) V^T w_j||^2 for the first r columns w_j of stream 1 of
   `index` (U m x l, S l, V n x l, column-major with ld m and n). */
double orc_post_est2(int m, int n, const double* A, int lda, const double* U, const double* S,
                     const double* V, int l, uint64_t seed, uint32_t index, int r)
{
    double* W = (double*)malloc(sizeof(double) * (size_t)n * (r > 0 ? r : 1));
    double* AW = (double*)malloc(sizeof(double) * (size_t)m * (r > 0 ? r : 1));
    double* VW = (double*)malloc(sizeof(double) * (size_t)(l > 0 ? l : 1) * (r > 0 ? r : 1));
    orc_omega(seed, index, 1, n, 0, r, W);
    orc_gemm(0, 0, m, r, n, A, lda, W, n, AW, m);     /* A W       */
    if (l > 0) orc_gemm(1, 0, l, r, n, V, n, W, n, VW, l); /* V^T W     */
    double sum = 0.0;
    for (int j = 0; j < r; ++j)
        for (int i = 0; i < m; ++i) {
            double e = AT(AW, m, i, j);
            for (int c = 0; c < l; ++c) e -= AT(U, m, i, c) * S[c] * AT(VW, l, c, j);
            sum += e * e;
        }
    free(W);
    free(AW);
    free(VW);
    return r > 0 ? sum / r : 0.0;
}

/* Truncation with the estimate's budget: the smallest k (<= len) with
   sum_{i >= k} S_i^2 <= (0.95 eps)^2 normA2 - 4 est2 (a negative budget keeps all len values). */
int orc_budget_rank(int len, const double* S, double normA2, double eps, double est2)
{
    double thr = 0.95 * 0.95 * eps * eps * normA2 - 4.0 * est2;
    if (thr < 0.0) thr = 0.0;
    double tail = 0.0;
    int k = len;
    for (int i = len - 1; i >= 0; --i) {
        double t = tail + S[i] * S[i];
        if (t > thr) break;
        tail = t;
        k = i;
    }
    return k;
}

/* Adaptive randomized SVD of one m x n matrix (1 <= m, n).  hint: first rank guess (clamped to
   [0, 256]); the first round draws l = hint + p columns.  q power steps per round.
   Outputs (caller-allocated, k = min(m, n)): U (m x k), S (k), V (n x k) -- the first `samples`
   columns are filled -- and res[6] = {rank, samples, rounds, fallback (0/1), est2 (as double),
   ||A||_F^2}; est2_round (max_rounds, nullable) receives each round's estimate.
   Returns 0, or -1 for bad arguments. */
int orc_rsvd_adaptive(int m, int n, const double* A, int lda, uint64_t seed, uint32_t index,
                      int hint, double eps, int p, int q, int max_rounds, int lcap,
                      double* U, double* S, double* V, double* res, double* est2_round)
{
    if (m < 1 || n < 1 || lda < m || p < 1 || max_rounds < 1) return -1;
    int k = m < n ? m : n;
    double norm2 = 0.0;
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < m; ++i) norm2 += AT(A, lda, i, j) * AT(A, lda, i, j);
    if (hint < 0) hint = 0;
    if (hint > 256) hint = 256;
    int l = hint + p;
    int full = (l >= k || l > lcap);
    int rounds = 0, fallback = 0, accepted = 0;
    double est2 = 0.0;
    for (int r = 0; r < max_rounds && !full && !accepted; ++r) {
        orc_rsvd(m, n, A, lda, seed, index, l, q, U, S, V);
        est2 = orc_post_est2(m, n, A, lda, U, S, V, l, seed, index, ORC_PROBES);
        if (est2_round) est2_round[r] = est2;
        rounds += 1;
        if (est2 <= 0.25 * eps * eps * norm2) {
            accepted = 1;
        } else if (l + p >= k || l + p > lcap) {
            full = 1;
            fallback = 1;
        } else {
            l += p;
        }
    }
    if (!full && !accepted) { /* rounds exhausted */
        full = 1;
        fallback = 1;
    }
    int samples = l;
    if (full) {
        orc_jacobi_svd(m, n, A, lda, -1.0, 60, S, U, m, V, n, NULL);
        est2 = 0.0;
        samples = k;
    }
    res[0] = orc_budget_rank(samples, S, norm2, eps, est2);
    res[1] = samples;
    res[2] = rounds;
    res[3] = fallback;
    res[4] = est2;
    res[5] = norm2;
    return 0;
}

/* Fixed-rank randomized SVD (Algorithm 4 as stated: k + p samples, q power steps, the first k
   columns kept).  When k + p reaches min(m, n) or exceeds lcap, the full Jacobi SVD replaces the
   sampling.  U (m x min(m,n)), S, V (n x min(m,n)) caller-allocated; the first k columns are the
   result.  Returns the number of samples used (k + p, or min(m, n)), or -1. */
int orc_rsvd_rank(int m, int n, const double* A, int lda, uint64_t seed, uint32_t index, int k,
                  int p, int q, int lcap, double* U, double* S, double* V)
{
    int kk = m < n ? m : n;
    if (m < 1 || n < 1 || lda < m || k < 1 || p < 0) return -1;
    int l = k + p;
    if (l >= kk || l > lcap) {
        orc_jacobi_svd(m, n, A, lda, -1.0, 60, S, U, m, V, n, NULL);
        return kk;
    }
    orc_rsvd(m, n, A, lda, seed, index, l, q, U, S, V);
    return l;
}

/* ---------------------------------------------------------------------------------------------
 * Batch drivers: independent matrices spread over threads (no arithmetic here).
 * ------------------------------------------------------------------------------------------- */

typedef struct {
    int count;
    int next;
    pthread_mutex_t mu;
    void (*fn)(void*, int);
    void* ctx;
} pool_t;

static void* pool_worker(void* arg)
{
    pool_t* p = (pool_t*)arg;
    for (;;) {
        pthread_mutex_lock(&p->mu);
        int b = p->next++;
        pthread_mutex_unlock(&p->mu);
        if (b >= p->count) break;
        p->fn(p->ctx, b);
    }
    return NULL;
}

static void parallel_for(int nthreads, int count, void (*fn)(void*, int), void* ctx)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pool_t p;
    p.count = count;
    p.next = 0;
    p.fn = fn;
    p.ctx = ctx;
    pthread_mutex_init(&p.mu, NULL);
    if (nthreads == 1) {
        pool_worker(&p);
    } else {
        pthread_t th[256];
        for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, pool_worker, &p);
        for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    }
    pthread_mutex_destroy(&p.mu);
}

typedef struct {
    const int *m, *n;
    const double* A;
    const long long* offA;
    double *Q, *R;
    const long long *offQ, *offR;
    int* info;
} qr_ctx;

static void qr_one(void* c_, int b)
{
    qr_ctx* c = (qr_ctx*)c_;
    int m = c->m[b], n = c->n[b];
    c->info[b] = orc_qr(m, n, c->A + c->offA[b], m > 0 ? m : 1, c->Q + c->offQ[b], m > 0 ? m : 1,
                        c->R + c->offR[b], n > 0 ? n : 1);
}

/* Batched QR: matrix b is m[b] x n[b] at A + offA[b] (ld = m[b]); Q (m x n, ld m) and
   R (n x n, ld n) at their offsets. */
void orc_qr_batch(int batch, const int* m, const int* n, const double* A, const long long* offA,
                  double* Q, const long long* offQ, double* R, const long long* offR, int* info,
                  int nthreads)
{
    qr_ctx c = {m, n, A, offA, Q, R, offQ, offR, info};
    parallel_for(nthreads, batch, qr_one, &c);
}

typedef struct {
    const int *m, *n;
    const double* A;
    const long long* offA;
    double tol;
    int max_sweeps;
    double *S, *U, *V;
    const long long *offS, *offU, *offV;
    int* info;
    long long* rot;
} svd_ctx;

static void svd_one(void* c_, int b)
{
    svd_ctx* c = (svd_ctx*)c_;
    int m = c->m[b], n = c->n[b];
    c->info[b] = orc_jacobi_svd(m, n, c->A + c->offA[b], m > 0 ? m : 1, c->tol, c->max_sweeps,
                                c->S + c->offS[b], c->U ? c->U + c->offU[b] : NULL, m > 0 ? m : 1,
                                c->V ? c->V + c->offV[b] : NULL, n > 0 ? n : 1,
                                c->rot ? c->rot + b : NULL);
}

/* Batched Jacobi SVD: U (m x k, ld m), V (n x k, ld n), S (k), k = min(m, n). */
void orc_svd_batch(int batch, const int* m, const int* n, const double* A, const long long* offA,
                   double tol, int max_sweeps, double* S, const long long* offS, double* U,
                   const long long* offU, double* V, const long long* offV, int* info,
                   long long* rotations, int nthreads)
{
    svd_ctx c = {m, n, A, offA, tol, max_sweeps, S, U, V, offS, offU, offV, info, rotations};
    parallel_for(nthreads, batch, svd_one, &c);
}
