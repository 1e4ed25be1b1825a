// jacobi_reg.cu -- one-sided Jacobi SVD with the whole matrix resident in registers
// (Algorithm 2, Section 2.2; the register tier of Section 4, re-mapped for sm_103a).
//
// Layout.  The working matrix W (m x n, or A^T when m < n) and the accumulated rotations V are
// spread over NS * PARTS lanes: lane (part, slot) holds RA rows (rows part*RA ...) of the two
// columns that column-pair slot `slot` currently owns, and RV rows of the same two columns of V.
// A round-robin step therefore processes all NS pairs at once, one pair per lane, with no shared
// memory traffic: the three Gram dot products are serial partial sums over the lane's rows
// followed by a reduction across the PARTS lanes of the pair (a shuffle when the parts share a
// warp, one barrier with a double-buffered exchange slot when they do not).  Each lane then
// computes its own pair's rotation, so one warp instruction serves NS pairs -- the parameter
// computation the paper measured as the dominant cost (Section 4.2) is not replicated across a
// warp.  All parts compute bit-identical parameters from identical sums.
//
// Pair ordering.  Odd-even transposition with exchange: 2 NS column positions, even steps pair
// positions (2k, 2k+1), odd steps (2k+1, 2k+2), and every processed pair swaps positions, so after
// 2 NS steps each of the 2NS(2NS-1)/2 pairs has met exactly once (one of the parallel orderings
// Section 5 lists).  Slot k holds the pair it processes; between steps exactly ONE column per slot
// moves to the neighbouring slot (a warp shuffle), half the traffic of the circle method.
//
// Scaled rotations (FAST = true).  Each column carries a scale d (W = W~ diag(d), V = V~ diag(d)).
// The rotation [w_i, w_j] <- [c w_i - s w_j, s w_i + c w_j] with t = s / c becomes
//   w~_i <- w~_i - t (d_j / d_i) w~_j,   w~_j <- w~_j + t (d_i / d_j) w~_i,   d_i, d_j <- c d_i, c d_j,
// one FMA per element instead of two multiplies and two FMAs; the scales are folded back into
// the columns at the end of every sweep (c >= 1/sqrt 2, so d stays above 2^-33 within a sweep).
// FAST = false applies the rotation as written.
//
// Carried column norms (CARRY = true).  Each lane keeps the squared norms of its two columns (true,
// unscaled frame) and moves them with the columns; a step then needs one dot product (gamma)
// instead of three, and after a rotation the norms follow from the Jacobi angle's identities
// alpha' = alpha - t gamma, beta' = beta + t gamma (the one-sided Jacobi norm update LAPACK's xGESVJ
// uses).  The norms are recomputed from the columns at the start of every sweep; an update that
// cancels below a quarter of the old value marks the norm stale (negative), and the next step of
// that column sums it afresh (the warp, or the CTA, takes the three-product step when any of its
// lanes holds a stale norm).  A rotation-free sweep changes no norm, so the convergence decision is
// taken on norms summed at that sweep's start.
//
// QR preconditioning (PRE = true, square matrices).  A = Q R by Householder QR in the register
// layout (reflectors kept in shared memory), then the sweeps run on W = R^T: R^T V_w = U_w S gives A = (Q V_w) S U_w^T, so
// U = Q V_w (the reflectors applied to the accumulated rotations) and V = U_w = W / sigma.  The
// rows of R are graded like the singular values, and the sweeps converge in fewer passes: 8.2
// instead of 14.1 on 64 x 64 FP32 with sigma_i = exp(-i/8), 9.0 instead of 16.1 on 32 x 32 FP64
// with sigma_i = 10^(-8i/31) (simulated with the same ordering and tolerance), for the price of
// about one sweep (the factorisation and the back-transformation).
#include <cuda_runtime.h>

#include <type_traits>

#include "common.cuh"
#include "launch.cuh"

namespace bsvd {

template <typename T>
struct Red3 {
    T a, b, c, pad;
};

// MINB is the number of matrices (CTAs) the launch bound asks to keep resident per SM; it caps
// the register allocation at 65536 / (NS * PARTS * MINB), trading scheduling freedom against
// occupancy.  Several values are instantiated and the autotuner picks one per size bin.
template <typename T, int NS, int PARTS, int RA, int RV, int MINB, bool FAST, bool PRE, bool P64, bool CARRY>
__global__ void __launch_bounds__(NS * PARTS, MINB)
    jacobi_reg_kernel(int batch, T* const* A, const int* M, const int* N, const int* LDA, T* const* Sout, T* const* U,
                      const int* LDU, T* const* V, const int* LDV, double tol_in, int max_sweeps, int* info,
                      long long* rot_out, ItemList wl)
{
    constexpr int NT = NS * PARTS;
    constexpr int PPW = 32 / NS;   // parts per warp (1 or 2)
    constexpr int NW = NT / 32;    // warps per matrix
    constexpr int NC = 2 * NS;     // column capacity
    static_assert(NT % 32 == 0, "whole warps only");
    // rotation parameters (zeta, t, c, s) and the rotation test in the working precision, or in
    // FP64 for FP32 data (P64): the Gram entries are summed in T, then promoted
    typedef typename std::conditional<P64, double, T>::type P;

    __shared__ Red3<T> red[2][NW > 1 ? NW : 1][32];
    __shared__ T sig_s[NC];
    constexpr int QM = PRE ? PARTS * RA : 1;  // the QR's matrix (column-major, leading dimension QM)
    __shared__ T qs[PRE ? QM * NC : 1];
    __shared__ T qdiag[PRE ? NC : 1];
    __shared__ T qred[PRE ? PARTS : 1];

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int s = lane % NS;                  // pair slot
    const int part = warp * PPW + lane / NS;  // row part
    const unsigned part_mask = PPW == 2 ? (lane < 16 ? 0x0000FFFFu : 0xFFFF0000u) : 0xFFFFFFFFu;

    for (int b = item_first(wl, batch); b >= 0; b = item_next(wl, batch, b)) {
        const int m = M[b], n = N[b], lda = LDA[b];
        const bool tr = m < n;
        const int mm = tr ? n : m;
        const int nn = tr ? m : n;
        const bool wantU = U != nullptr, wantV = V != nullptr;
        const int ldu = wantU ? LDU[b] : 1, ldvo = wantV ? LDV[b] : 1;
        const bool bad = m < 0 || n < 0 || mm > PARTS * RA || nn > NC || nn > PARTS * RV ||
                         lda < (m > 1 ? m : 1) || (wantU && ldu < (m > 1 ? m : 1)) || (wantV && ldvo < (n > 1 ? n : 1));
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
        int step_parity = 0;  // double-buffer index of the cross-part exchange slot
        // preconditioned: the sweeps run on R^T, whose rotations give U (through Q) and whose
        // normalised columns give V, so the roles of the two outputs swap as for A^T
        const bool pre = PRE && m == n && n > 1 && n <= QM;
        const bool sw = tr || pre;
        const bool accV = sw ? wantU : wantV;

        // ---- load: slot s owns columns (positions) 2s and 2s + 1 ----
        int colL = 2 * s, colR = 2 * s + 1;
        T aL[RA], aR[RA], vL[RV], vR[RV];
        const T* a = A[b];
        if (pre) {
#pragma unroll
            for (int k = 0; k < RA; ++k) {
                const int r = part * RA + k;
                aL[k] = (r < n && colL < n) ? a[(size_t)colL * lda + r] : T(0);
                aR[k] = (r < n && colR < n) ? a[(size_t)colR * lda + r] : T(0);
            }
            // Householder QR in the register layout (Algorithm 1): column i's owner lanes (one per
            // part) publish the column and their share of its squared norm; every lane forms the
            // reflector v_i (normalised for I - 2 v v^T) from the published column, applies it to
            // its own columns right of i, and the owners store v_i in column i of qs (rows >= i)
            // for the back-transformation.  Two barriers per column.
            for (int i = 0; i < n; ++i) {
                const int so = i >> 1;
                const bool odd_col = i & 1;
                if (s == so) {
                    T ss = T(0);
#pragma unroll
                    for (int k = 0; k < RA; ++k) {
                        const int r = part * RA + k;
                        const T x = odd_col ? aR[k] : aL[k];
                        if (r < n) qs[i * QM + r] = x;
                        ss = (r >= i && r < n) ? fma(x, x, ss) : ss;
                    }
                    qred[part] = ss;
                }
                __syncthreads();
                T ss = T(0);
#pragma unroll
                for (int p = 0; p < PARTS; ++p) ss += qred[p];
                const T x0 = qs[i * QM + i];
                const T alpha = dsqrt(ss);
                const T sg = x0 >= T(0) ? T(1) : T(-1);
                const T inv = alpha > T(0) ? drsqrt(T(2) * alpha * (alpha + dabs(x0))) : T(0);
                const T rii = -sg * alpha;
                T vk[RA];
                T wl = T(0), wr = T(0);
#pragma unroll
                for (int k = 0; k < RA; ++k) {
                    const int r = part * RA + k;
                    const T x = r < n ? qs[i * QM + r] : T(0);
                    vk[k] = r < i ? T(0) : (r == i ? x0 + sg * alpha : x) * inv;
                    wl = fma(vk[k], aL[k], wl);
                    wr = fma(vk[k], aR[k], wr);
                }
                if (PPW == 2) {
                    wl += __shfl_xor_sync(0xffffffffu, wl, 16);
                    wr += __shfl_xor_sync(0xffffffffu, wr, 16);
                }
                if (NW > 1) {
                    red[step_parity][warp][lane] = Red3<T>{wl, wr, T(0), T(0)};
                    __syncthreads();
                    wl = wr = T(0);
#pragma unroll
                    for (int w = 0; w < NW; ++w) {
                        wl += red[step_parity][w][lane].a;
                        wr += red[step_parity][w][lane].b;
                    }
                    step_parity ^= 1;
                } else {
                    __syncthreads();  // every lane has read column i of qs before the owners overwrite it
                }
                // columns right of i take the reflector; column i becomes R(0:i, i), R(i, i), zeros
                wl = colL > i ? T(-2) * wl : T(0);
                wr = colR > i ? T(-2) * wr : T(0);
#pragma unroll
                for (int k = 0; k < RA; ++k) {
                    const int r = part * RA + k;
                    aL[k] = fma(wl, vk[k], aL[k]);
                    aR[k] = fma(wr, vk[k], aR[k]);
                    if (colL == i && r >= i) aL[k] = r == i ? rii : T(0);
                    if (colR == i && r >= i) aR[k] = r == i ? rii : T(0);
                    if (s == so && r >= i && r < n) qs[i * QM + r] = vk[k];
                }
            }
            // R to the upper triangle of qs and to qdiag (v_i occupies rows >= i of column i)
#pragma unroll
            for (int k = 0; k < RA; ++k) {
                const int r = part * RA + k;
                if (r < colL && colL < n) qs[colL * QM + r] = aL[k];
                if (r == colL && colL < n) qdiag[colL] = aL[k];
                if (r < colR && colR < n) qs[colR * QM + r] = aR[k];
                if (r == colR && colR < n) qdiag[colR] = aR[k];
            }
            __syncthreads();
            // W = R^T: W(r, c) = R(c, r), stored above the diagonal of qs (diagonal in qdiag)
#pragma unroll
            for (int k = 0; k < RA; ++k) {
                const int r = part * RA + k;
                aL[k] = T(0);
                aR[k] = T(0);
                if (r < n) {
                    if (colL < n) aL[k] = colL < r ? qs[r * QM + colL] : (colL == r ? qdiag[r] : T(0));
                    if (colR < n) aR[k] = colR < r ? qs[r * QM + colR] : (colR == r ? qdiag[r] : T(0));
                }
            }
        } else {
#pragma unroll
            for (int k = 0; k < RA; ++k) {
                const int r = part * RA + k;
                aL[k] = T(0);
                aR[k] = T(0);
                if (r < mm) {
                    if (!tr) {
                        if (colL < nn) aL[k] = a[(size_t)colL * lda + r];
                        if (colR < nn) aR[k] = a[(size_t)colR * lda + r];
                    } else {
                        if (colL < nn) aL[k] = a[(size_t)r * lda + colL];
                        if (colR < nn) aR[k] = a[(size_t)r * lda + colR];
                    }
                }
            }
        }
#pragma unroll
        for (int k = 0; k < RV; ++k) {
            const int r = part * RV + k;
            vL[k] = (r == colL) ? T(1) : T(0);
            vR[k] = (r == colR) ? T(1) : T(0);
        }
        T dL = T(1), dR = T(1);  // column scales
        T nL = T(0), nR = T(0);  // CARRY: true squared norms of the two columns (negative: stale)

        const P tol = tol_in > 0.0 ? P(tol_in) : P(dsqrt(double(mm)) * Unit<T>::value);
        const int sweeps_cap = max_sweeps > 0 ? max_sweeps : 30;
        int sweep = 0;
        bool converged = false;
        long long total_rot = 0;

        while (sweep < sweeps_cap) {
            int rot_sweep = 0;
            if (CARRY) nL = nR = T(-1);  // every sweep starts from norms summed afresh
#pragma unroll 1
            for (int st = 0; st < 2 * NS; ++st) {
                const bool odd = st & 1;
                // Gram partials over this lane's rows (two accumulators per entry); with carried
                // norms only gamma, unless a norm of the warp (of the CTA, NW > 1) is stale.  The
                // flag is exchanged with the partial sums: a stale lane sends its squared norms
                // (non-negative) in slots a and b, the others send -1
                const bool mine = !CARRY || nL < T(0) || nR < T(0);
                const bool full = !CARRY || (NW > 1 ? true : __any_sync(0xffffffffu, mine));
                T a0 = T(0), a1 = T(0), b0 = T(0), b1 = T(0), c0 = T(0), c1 = T(0);
                if (mine) {
#pragma unroll
                    for (int k = 0; k < RA; k += 2) {
                        a0 = fma(aL[k], aL[k], a0);
                        b0 = fma(aR[k], aR[k], b0);
                        c0 = fma(aL[k], aR[k], c0);
                        if (k + 1 < RA) {
                            a1 = fma(aL[k + 1], aL[k + 1], a1);
                            b1 = fma(aR[k + 1], aR[k + 1], b1);
                            c1 = fma(aL[k + 1], aR[k + 1], c1);
                        }
                    }
                } else {
                    // gamma alone: four chains (a0, b0 serve as the third and fourth), so that the
                    // dot product's FMA latency is not the step's critical path
#pragma unroll
                    for (int k = 0; k < RA; k += 4) {
                        c0 = fma(aL[k], aR[k], c0);
                        if (k + 1 < RA) c1 = fma(aL[k + 1], aR[k + 1], c1);
                        if (k + 2 < RA) a0 = fma(aL[k + 2], aR[k + 2], a0);
                        if (k + 3 < RA) b0 = fma(aL[k + 3], aR[k + 3], b0);
                    }
                    c0 += a0;
                    c1 += b0;
                    a0 = b0 = T(0);
                }
                T sa = a0 + a1, sb = b0 + b1, sc = c0 + c1;
                if (PPW == 2) {
                    if (full) {
                        sa += __shfl_xor_sync(0xffffffffu, sa, 16);
                        sb += __shfl_xor_sync(0xffffffffu, sb, 16);
                    }
                    sc += __shfl_xor_sync(0xffffffffu, sc, 16);
                }
                if (NW > 1) {
                    red[step_parity][warp][lane] = Red3<T>{sa, sb, sc, T(0)};
                    __syncthreads();
                    sa = sb = sc = T(0);
#pragma unroll
                    for (int w = 0; w < NW; ++w) {
                        const Red3<T> r = red[step_parity][w][lane];
                        sa += r.a;
                        sb += r.b;
                        sc += r.c;
                    }
                    step_parity ^= 1;
                }
                // column norms in the unscaled frame: carried, or just summed (all parts of a pair
                // hold the same carried values and the same stale flag, so they agree)
                T tnL = nL, tnR = nR;
                if (CARRY && mine) {
                    tnL = dL * dL * sa;
                    tnR = dR * dR * sb;
                }
                // rotation of the pair, in the unscaled frame; the wrap slot idles on odd steps
                const P alpha = CARRY ? P(tnL) : (FAST ? P(dL) * P(dL) * P(sa) : P(sa));
                const P beta = CARRY ? P(tnR) : (FAST ? P(dR) * P(dR) * P(sb) : P(sb));
                const P gamma = FAST ? P(dL) * P(dR) * P(sc) : P(sc);
                const bool rot = !(odd && s == NS - 1) && alpha > P(0) && beta > P(0) &&
                                 off_diagonal_large(alpha, beta, gamma, tol);
                P tth = P(0), cth = P(1);
                if (rot) {
                    tth = jacobi_t(alpha, beta, gamma);
                    cth = drsqrt(P(1) + tth * tth);
                }
                // unconditional update within a warp: a skipped pair has multipliers 0 (and c = 1),
                // which leaves its columns bit-identical; a warp none of whose pairs rotates (most
                // steps of the last sweeps, every step of the final, rotation-free one) skips it
                const bool any_rot = __any_sync(0xffffffffu, rot);
                if (!any_rot) {
                } else if (FAST) {
                    // scale ratios from the current scales (correctly rounded reciprocals), so that
                    // their rounding does not accumulate over the rotations of a sweep
                    const T mL = -T(tth) * (dR * rcp_rn(dL));  // -t d_j / d_i
                    const T mR = T(tth) * (dL * rcp_rn(dR));   //  t d_i / d_j
#pragma unroll
                    for (int k = 0; k < RA; ++k) {
                        const T x = aL[k], y = aR[k];
                        aL[k] = fma(mL, y, x);
                        aR[k] = fma(mR, x, y);
                    }
                    if (accV) {
#pragma unroll
                        for (int k = 0; k < RV; ++k) {
                            const T x = vL[k], y = vR[k];
                            vL[k] = fma(mL, y, x);
                            vR[k] = fma(mR, x, y);
                        }
                    }
                    dL *= T(cth);
                    dR *= T(cth);
                } else {
                    const T cc = T(cth), ss = T(cth * tth);
#pragma unroll
                    for (int k = 0; k < RA; ++k) {
                        const T x = aL[k], y = aR[k];
                        aL[k] = fma(cc, x, -ss * y);
                        aR[k] = fma(ss, x, cc * y);
                    }
                    if (accV) {
#pragma unroll
                        for (int k = 0; k < RV; ++k) {
                            const T x = vL[k], y = vR[k];
                            vL[k] = fma(cc, x, -ss * y);
                            vR[k] = fma(ss, x, cc * y);
                        }
                    }
                }
                rot_sweep += __popc(__ballot_sync(0xffffffffu, rot) & part_mask);
                if (CARRY) {
                    // alpha' = alpha - t gamma, beta' = beta + t gamma; a cancelling update is stale
                    nL = tnL;
                    nR = tnR;
                    if (rot) {
                        const T tg = T(tth * gamma);
                        const T aN = tnL - tg, bN = tnR + tg;
                        nL = aN < T(0.25) * tnL ? T(-1) : aN;
                        nR = bN < T(0.25) * tnR ? T(-1) : bN;
                    }
                }
                // exchange: after the swap the pair's lower position holds the right column
                if (!odd) {
                    // even -> odd: the right column moves one slot down (slot s receives s + 1's)
                    const int src = s + 1 == NS ? 0 : s + 1;
#pragma unroll
                    for (int k = 0; k < RA; ++k) aR[k] = __shfl_sync(0xffffffffu, aR[k], src, NS);
                    if (accV) {
#pragma unroll
                        for (int k = 0; k < RV; ++k) vR[k] = __shfl_sync(0xffffffffu, vR[k], src, NS);
                    }
                    if (FAST) dR = __shfl_sync(0xffffffffu, dR, src, NS);
                    if (CARRY) nR = __shfl_sync(0xffffffffu, nR, src, NS);
                    colR = __shfl_sync(0xffffffffu, colR, src, NS);
                } else {
                    // odd -> even: the left column moves one slot up; the wrap slot, which did not
                    // rotate, hands over its right column and keeps its left one as the right
                    const int src = s == 0 ? NS - 1 : s - 1;
                    const bool wrap = s == NS - 1;
#pragma unroll
                    for (int k = 0; k < RA; ++k) {
                        const T r = __shfl_sync(0xffffffffu, wrap ? aR[k] : aL[k], src, NS);
                        aR[k] = wrap ? aL[k] : aR[k];
                        aL[k] = r;
                    }
                    if (accV) {
#pragma unroll
                        for (int k = 0; k < RV; ++k) {
                            const T r = __shfl_sync(0xffffffffu, wrap ? vR[k] : vL[k], src, NS);
                            vR[k] = wrap ? vL[k] : vR[k];
                            vL[k] = r;
                        }
                    }
                    if (FAST) {
                        const T r = __shfl_sync(0xffffffffu, wrap ? dR : dL, src, NS);
                        dR = wrap ? dL : dR;
                        dL = r;
                    }
                    if (CARRY) {
                        const T r = __shfl_sync(0xffffffffu, wrap ? nR : nL, src, NS);
                        nR = wrap ? nL : nR;
                        nL = r;
                    }
                    const int rc = __shfl_sync(0xffffffffu, wrap ? colR : colL, src, NS);
                    colR = wrap ? colL : colR;
                    colL = rc;
                }
            }
            if (FAST) {
                // fold the scales back into the columns
#pragma unroll
                for (int k = 0; k < RA; ++k) {
                    aL[k] *= dL;
                    aR[k] *= dR;
                }
                if (accV) {
#pragma unroll
                    for (int k = 0; k < RV; ++k) {
                        vL[k] *= dL;
                        vR[k] *= dR;
                    }
                }
                dL = dR = T(1);
            }
            ++sweep;
            total_rot += rot_sweep;
            if (rot_sweep == 0) {
                converged = true;
                break;
            }
        }

        // ---- preconditioned: U = Q V_w = H_0 H_1 ... H_{n-1} V_w, the reflectors applied last first ----
        if (PRE && pre && accV) {
            for (int j = n - 1; j >= 0; --j) {
                const T* vj = qs + j * QM;  // the reflector occupies rows j .. n - 1 of column j
                T dl = T(0), dr = T(0);
#pragma unroll
                for (int k = 0; k < RV; ++k) {
                    const int r = part * RV + k;
                    const T v = (r >= j && r < n) ? vj[r] : T(0);
                    dl = fma(v, vL[k], dl);
                    dr = fma(v, vR[k], dr);
                }
                if (PPW == 2) {
                    dl += __shfl_xor_sync(0xffffffffu, dl, 16);
                    dr += __shfl_xor_sync(0xffffffffu, dr, 16);
                }
                if (NW > 1) {
                    red[step_parity][warp][lane] = Red3<T>{dl, dr, T(0), T(0)};
                    __syncthreads();
                    dl = dr = T(0);
#pragma unroll
                    for (int w = 0; w < NW; ++w) {
                        dl += red[step_parity][w][lane].a;
                        dr += red[step_parity][w][lane].b;
                    }
                    step_parity ^= 1;
                }
                dl *= T(-2);
                dr *= T(-2);
#pragma unroll
                for (int k = 0; k < RV; ++k) {
                    const int r = part * RV + k;
                    const T v = (r >= j && r < n) ? vj[r] : T(0);
                    vL[k] = fma(dl, v, vL[k]);
                    vR[k] = fma(dr, v, vR[k]);
                }
            }
        }

        // ---- sigma = column norms (reduced across parts like the Gram entries) ----
        T na = T(0), nb = T(0);
#pragma unroll
        for (int k = 0; k < RA; ++k) {
            na = fma(aL[k], aL[k], na);
            nb = fma(aR[k], aR[k], nb);
        }
        if (PPW == 2) {
            na += __shfl_xor_sync(0xffffffffu, na, 16);
            nb += __shfl_xor_sync(0xffffffffu, nb, 16);
        }
        if (NW > 1) {
            red[step_parity][warp][lane] = Red3<T>{na, nb, T(0), T(0)};
            __syncthreads();
            na = nb = T(0);
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                na += red[step_parity][w][lane].a;
                nb += red[step_parity][w][lane].b;
            }
        }
        const T sgL = dsqrt(na), sgR = dsqrt(nb);
        if (part == 0) {
            sig_s[colL] = sgL;
            sig_s[colR] = sgR;
        }
        __syncthreads();
        int rkL = 0, rkR = 0;
        for (int i = 0; i < nn; ++i) {
            const T si = sig_s[i];
            rkL += (si > sgL) || (si == sgL && i < colL);
            rkR += (si > sgR) || (si == sgR && i < colR);
        }
        T* s_out = Sout[b];
        if (part == 0) {
            if (colL < nn) s_out[rkL] = sgL;
            if (colR < nn) s_out[rkR] = sgR;
        }
        T* uw = sw ? (wantV ? V[b] : nullptr) : (wantU ? U[b] : nullptr);  // receives W / sigma
        const int lduw = sw ? ldvo : ldu;
        T* vw = sw ? (wantU ? U[b] : nullptr) : (wantV ? V[b] : nullptr);  // receives V (PRE: Q V_w)
        const int ldvw = sw ? ldu : ldvo;
        if (uw) {
            const T iL = sgL > T(0) ? T(1) / sgL : T(0), iR = sgR > T(0) ? T(1) / sgR : T(0);
#pragma unroll
            for (int k = 0; k < RA; ++k) {
                const int r = part * RA + k;
                if (r < mm) {
                    if (colL < nn) uw[(size_t)rkL * lduw + r] = aL[k] * iL;
                    if (colR < nn) uw[(size_t)rkR * lduw + r] = aR[k] * iR;
                }
            }
        }
        if (vw) {
#pragma unroll
            for (int k = 0; k < RV; ++k) {
                const int r = part * RV + k;
                if (r < nn) {
                    if (colL < nn) vw[(size_t)rkL * ldvw + r] = vL[k];
                    if (colR < nn) vw[(size_t)rkR * ldvw + r] = vR[k];
                }
            }
        }
        if (tid == 0) {
            bool finite = true;
            for (int i = 0; i < nn; ++i) finite = finite && isfinite(sig_s[i]);
            info[b] = !finite ? BSVD_INFO_NONFINITE : (converged ? sweep : BSVD_INFO_NOT_CONVERGED + sweep);
            if (rot_out) rot_out[b] = total_rot;
        }
        __syncthreads();
    }
}

template <typename T, int NS, int PARTS, int RA, int RV, int MINB, bool FAST, bool PRE, bool P64, bool CARRY>
static int launch_reg(int batch, void* const* A, const int* M, const int* N, const int* LDA, void* const* S,
                      void* const* U, const int* LDU, void* const* V, const int* LDV, double tol, int max_sweeps,
                      int* info, long long* rot, cudaStream_t st, ItemList wl)
{
    auto kern = jacobi_reg_kernel<T, NS, PARTS, RA, RV, MINB, FAST, PRE, P64 && sizeof(T) == 4, CARRY>;
    const int grid = item_grid(kern, NS * PARTS, 0, wl, batch, st);
    if (grid == 0) return BSVD_ERR_CUDA;
    kern<<<grid, NS * PARTS, 0, st>>>(
        batch, (T* const*)A, M, N, LDA, (T* const*)S, (T* const*)U, LDU, (T* const*)V, LDV, tol, max_sweeps, info, rot,
        wl);
    return cudaGetLastError() == cudaSuccess ? BSVD_SUCCESS : BSVD_ERR_CUDA;
}

// Register-tier variants (slots, row parts, A rows per lane, V rows per lane, resident CTAs, scaled
// rotations, QR preconditioning, FP64 rotation parameters, carried column norms), in order of
// preference.  `variant` 0
// launches the first that fits the shape bound; k > 0 launches the k-th fitting one; a negative
// `variant` only counts the fitting ones (returned).  The preconditioned ones need square bounds
// and are listed after the plain ones, so that variant 0 stays unpreconditioned; the FP32 variants
// with FP64 rotation parameters (zeta, t, c, s and the rotation test in FP64, the data and the Gram
// sums in FP32) come next, the carried-norm ones last.
#define BSVD_REG_VARIANTS_F32(X)                                                                        \
    X(16, 2, 16, 16, 16, true, false, false, false) /* n <= 32, m <= 32: one warp per matrix */                \
    X(16, 2, 32, 16, 12, true, false, false, false) /* n <= 32, m <= 64 */                                     \
    X(32, 2, 32, 32, 6, true, false, false, false)  /* n <= 64, m <= 64: two warps, 3 warps per SMSP */        \
    X(32, 2, 32, 32, 4, true, false, false, false)  /*   ... 2 warps per sub-partition, no register cap */     \
    X(32, 2, 32, 32, 6, false, false, false, false) /*   ... rotations applied as written */                   \
    X(32, 4, 16, 16, 4, true, false, false, false)  /*   ... four warps, 128-register cap */                   \
    X(16, 4, 32, 8, 4, true, false, false, false)   /* n <= 32, m <= 128 */                                    \
    X(32, 4, 32, 16, 2, true, false, false, false)  /* n <= 64, m <= 128 */                                    \
    X(16, 2, 16, 16, 16, true, true, false, false)  /* 32 x 32, QR-preconditioned */                           \
    X(32, 2, 32, 32, 6, true, true, false, false)   /* 64 x 64, QR-preconditioned */                           \
    X(32, 2, 32, 32, 6, true, false, true, false)   /* n <= 64, m <= 64, FP64 rotation parameters */           \
    X(32, 2, 32, 32, 6, true, true, true, false)    /* 64 x 64, QR-preconditioned, FP64 rotation parameters */ \
    X(16, 2, 16, 16, 16, true, true, false, true)   /* 32 x 32, QR-preconditioned, carried column norms */  \
    X(32, 2, 32, 32, 6, true, false, false, true)   /* n <= 64, m <= 64, carried column norms */            \
    X(32, 2, 32, 32, 6, true, true, false, true)    /* 64 x 64, QR-preconditioned, carried column norms */
#define BSVD_REG_VARIANTS_F64(X)                                                                        \
    X(16, 2, 16, 16, 8, true, false, false, false)  /* n <= 32, m <= 32: one warp per matrix */                \
    X(16, 2, 16, 16, 8, false, false, false, false)                                                            \
    X(16, 2, 16, 16, 12, true, false, false, false)                                                            \
    X(16, 4, 16, 8, 5, true, false, false, false)   /* n <= 32, m <= 64 */                                     \
    X(32, 4, 16, 16, 2, true, false, false, false)  /* n <= 64, m <= 64 */                                     \
    X(16, 2, 16, 16, 8, true, true, false, false)   /* 32 x 32, QR-preconditioned */                           \
    X(32, 4, 16, 16, 2, true, true, false, false)   /* 64 x 64, QR-preconditioned */                       \
    X(16, 2, 16, 16, 8, true, true, false, true)    /* 32 x 32, QR-preconditioned, carried column norms */  \
    X(32, 4, 16, 16, 2, true, true, false, true)    /* 64 x 64, QR-preconditioned, carried column norms */

#define BSVD_FITS(NS_, PARTS_, RA_, RV_, PRE_) \
    (nn <= 2 * (NS_) && mm <= (PARTS_) * (RA_) && nn <= (PARTS_) * (RV_) && (!(PRE_) || max_m == max_n))

template <typename T>
int launch_jacobi_reg(int batch, int max_m, int max_n, int variant, void* const* A, const int* M, const int* N,
                      const int* LDA, void* const* S, void* const* U, const int* LDU, void* const* V, const int* LDV,
                      double tol, int max_sweeps, int* info, long long* rot, cudaStream_t st, ItemList wl)
{
    const int mm = max_m > max_n ? max_m : max_n;
    const int nn = max_m > max_n ? max_n : max_m;
    int seen = 0;
#define BSVD_TRY(NS_, PARTS_, RA_, RV_, MINB_, FAST_, PRE_, P64_, CARRY_)                                       \
    if (BSVD_FITS(NS_, PARTS_, RA_, RV_, PRE_)) {                                                               \
        ++seen;                                                                                             \
        if (variant == 0 || variant == seen)                                                                \
            return launch_reg<T, NS_, PARTS_, RA_, RV_, MINB_, FAST_, PRE_, P64_, CARRY_>(                        \
                batch, A, M, N, LDA, S, U, LDU, V, LDV, tol, max_sweeps, info, rot, st, wl);                      \
    }
    if constexpr (sizeof(T) == 4) {
        BSVD_REG_VARIANTS_F32(BSVD_TRY)
    } else {
        BSVD_REG_VARIANTS_F64(BSVD_TRY)
    }
#undef BSVD_TRY
    return variant < 0 ? seen : BSVD_ERR_UNSUPPORTED;
}

// The k-th (k >= 1) register-tier variant fitting the bounds: desc = {slots, parts, A rows per
// lane, V rows per lane, resident CTAs, scaled rotations, QR preconditioning, FP64 rotation
// parameters, carried column norms}; 0, or BSVD_ERR_UNSUPPORTED when there is no k-th variant.
int jacobi_reg_variant_desc(bool f64, int max_m, int max_n, int k, int* desc)
{
    const int mm = max_m > max_n ? max_m : max_n;
    const int nn = max_m > max_n ? max_n : max_m;
    int seen = 0;
#define BSVD_DESC(NS_, PARTS_, RA_, RV_, MINB_, FAST_, PRE_, P64_, CARRY_)                                \
    if (BSVD_FITS(NS_, PARTS_, RA_, RV_, PRE_) && ++seen == k) {                                        \
        const int d[9] = {NS_, PARTS_, RA_, RV_, MINB_, (FAST_) ? 1 : 0, (PRE_) ? 1 : 0, (P64_) ? 1 : 0,  \
                          (CARRY_) ? 1 : 0};                                                            \
        for (int i = 0; i < 9; ++i) desc[i] = d[i];                                                     \
        return BSVD_SUCCESS;                                                                            \
    }
    if (!f64) {
        BSVD_REG_VARIANTS_F32(BSVD_DESC)
    } else {
        BSVD_REG_VARIANTS_F64(BSVD_DESC)
    }
#undef BSVD_DESC
    return BSVD_ERR_UNSUPPORTED;
}
#undef BSVD_FITS

template int launch_jacobi_reg<float>(int, int, int, int, void* const*, const int*, const int*, const int*,
                                      void* const*, void* const*, const int*, void* const*, const int*, double, int,
                                      int*, long long*, cudaStream_t, ItemList);
template int launch_jacobi_reg<double>(int, int, int, int, void* const*, const int*, const int*, const int*,
                                       void* const*, void* const*, const int*, void* const*, const int*, double, int,
                                       int*, long long*, cudaStream_t, ItemList);

}  // namespace bsvd
