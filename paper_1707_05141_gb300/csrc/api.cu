// api.cu -- the extern "C" boundary declared in include/bsvd.h: host-side argument checks, tier
// selection and launches on the caller's stream.  No device allocation, no synchronisation.
#include <cuda_runtime.h>

#include <atomic>

#include "common.cuh"
#include "launch.cuh"

using namespace bsvd;

namespace {

// Autotuning table: for each (dtype, size bin of max(m, n), size bin of min(m, n)) the encoded
// tier | variant << 8 that BSVD_TIER_AUTO uses.  0 = not tuned (built-in preference order).
// Entries are atomics so that recording a choice may race with calls that read it (relaxed
// order: a call sees the old or the new entry, each a complete choice).
constexpr int kBins = 9;  // bins 0..8 cover sizes <= 1, 2, 4, ..., 256
std::atomic<int> g_choice[2][kBins][kBins];

int size_bin(int x)
{
    int b = 0;
    while ((1 << b) < x && b < kBins - 1) ++b;
    return b;
}

// Block-tier table: for each (dtype, bin of max(m, n), bin of min(m, n)) up to 16384 the block width
// | inner register variant << 8 that block_width = 0 selects.  0 = not tuned (width 32, default
// inner variant).
constexpr int kBlockBins = 15;   // sizes <= 1, 2, 4, ..., 16384
std::atomic<int> g_block_choice[2][kBlockBins][kBlockBins];

int block_bin(int x)
{
    int b = 0;
    while ((1 << b) < x && b < kBlockBins - 1) ++b;
    return b;
}

// block_width 0: the recorded choice for this size bin (its inner variant joins `method` unless the
// caller named one); returns the block width to use
int resolve_block_choice(int dtype, int max_m, int max_n, int block_width, int* method)
{
    if (block_width != 0) return block_width;
    const int mm = max_m > max_n ? max_m : max_n, nn = max_m > max_n ? max_n : max_m;
    const int c = g_block_choice[dtype == BSVD_F64][block_bin(mm)][block_bin(nn)].load(std::memory_order_relaxed);
    if (c == 0) return 32;
    if (((*method >> 8) & 0xff) == 0) *method |= (c >> 8 & 0xff) << 8;
    return c & 0xff;
}

template <typename T>
int svd_dispatch(int batch, int max_m, int max_n, int tier, void* const* dA, const int* d_m, const int* d_n,
                 const int* d_lda, void* const* dS, void* const* dU, const int* d_ldu, void* const* dV, const int* d_ldv,
                 double tol, int max_sweeps, int* d_info, long long* d_rot, cudaStream_t st)
{
    int base = tier & 0xff, variant = tier >> 8;
    if (base == BSVD_TIER_AUTO) {
        const int mm = max_m > max_n ? max_m : max_n, nn = max_m > max_n ? max_n : max_m;
        const int c = g_choice[sizeof(T) == 8][size_bin(mm)][size_bin(nn)].load(std::memory_order_relaxed);
        if (c) {
            base = c & 0xff;
            variant = c >> 8;
        }
    }
    if (base == BSVD_TIER_AUTO || base == BSVD_TIER_REGISTER) {
        const int rc = launch_jacobi_reg<T>(batch, max_m, max_n, variant, dA, d_m, d_n, d_lda, dS, dU, d_ldu, dV,
                                            d_ldv, tol, max_sweeps, d_info, d_rot, st);
        if (rc != BSVD_ERR_UNSUPPORTED || base == BSVD_TIER_REGISTER) return rc;
    }
    return launch_jacobi_smem<T>(batch, max_m, max_n, dA, d_m, d_n, d_lda, dS, dU, d_ldu, dV, d_ldv, tol,
                                 max_sweeps, d_info, d_rot, st);
}

}  // namespace

extern "C" {

const char* bsvd_version(void)
{
    return "bsvd-gb300 0.6 (sm_103a; batched Householder QR, register/shared/block one-sided Jacobi SVD with QR "
           "preconditioning (register and block level) and a tcgen05 block Gram, fixed-rank and adaptive "
           "randomized SVD, H2 basis truncation, learned rank predictor)";
}

int batched_qr(int dtype, int batch, int max_m, int max_n, void* const* dA, const int* d_m, const int* d_n,
               const int* d_lda, void* const* dQ, const int* d_ldq, void* const* dR, const int* d_ldr, int* d_info,
               void* stream)
{
    if (dtype != BSVD_F32 && dtype != BSVD_F64) return -1;
    if (batch < 0) return -2;
    if (max_m < 0) return -3;
    if (max_n < 0 || max_n > max_m) return -4;
    if (batch == 0) return BSVD_SUCCESS;
    if (!dA) return -5;
    if (!d_m) return -6;
    if (!d_n) return -7;
    if (!d_lda) return -8;
    if (dQ && !d_ldq) return -10;
    if (dR && !d_ldr) return -12;
    if (!d_info) return -13;
    const size_t es = dtype == BSVD_F32 ? 4 : 8;
    if (max_m > 1024 || (size_t)max_m * max_n * es > 200 * 1024) return BSVD_ERR_UNSUPPORTED;
    if (max_n == 0) max_n = 1;
    if (max_m == 0) max_m = 1;
    cudaStream_t st = (cudaStream_t)stream;
    return dtype == BSVD_F32 ? launch_qr<float>(batch, max_m, max_n, dA, d_m, d_n, d_lda, dQ, d_ldq, dR, d_ldr, d_info, st)
                             : launch_qr<double>(batch, max_m, max_n, dA, d_m, d_n, d_lda, dQ, d_ldq, dR, d_ldr, d_info, st);
}

size_t batched_qr_blocked_workspace(int dtype, int batch, int max_m, int max_n)
{
    if ((dtype != BSVD_F32 && dtype != BSVD_F64) || batch < 0 || max_m < 0 || max_n < 0 || max_n > max_m) return 0;
    return dtype == BSVD_F32 ? qr_blocked_workspace<float>(batch, max_m, max_n)
                             : qr_blocked_workspace<double>(batch, max_m, max_n);
}

int batched_qr_blocked_max_rows(int dtype)
{
    if (dtype != BSVD_F32 && dtype != BSVD_F64) return -1;
    return dtype == BSVD_F32 ? qr_blocked_max_rows<float>() : qr_blocked_max_rows<double>();
}

int batched_qr_blocked(int dtype, int batch, int max_m, int max_n, void* const* dA, const int* d_m, const int* d_n,
                       const int* d_lda, void* const* dQ, const int* d_ldq, void* const* dR, const int* d_ldr,
                       int* d_info, void* workspace, size_t workspace_bytes, void* stream)
{
    if (dtype != BSVD_F32 && dtype != BSVD_F64) return -1;
    if (batch < 0) return -2;
    if (max_m < 0) return -3;
    if (max_n < 0 || max_n > max_m) return -4;
    if (batch == 0) return BSVD_SUCCESS;
    if (!dA) return -5;
    if (!d_m) return -6;
    if (!d_n) return -7;
    if (!d_lda) return -8;
    if (dQ && !d_ldq) return -10;
    if (dR && !d_ldr) return -12;
    if (!d_info) return -13;
    if (!workspace) return -14;
    if (max_m > batched_qr_blocked_max_rows(dtype)) return BSVD_ERR_UNSUPPORTED;
    if (max_n == 0) max_n = 1;
    if (max_m == 0) max_m = 1;
    cudaStream_t st = (cudaStream_t)stream;
    return dtype == BSVD_F32 ? launch_qr_blocked<float>(batch, max_m, max_n, dA, d_m, d_n, d_lda, dQ, d_ldq, dR, d_ldr,
                                                        d_info, workspace, workspace_bytes, st)
                             : launch_qr_blocked<double>(batch, max_m, max_n, dA, d_m, d_n, d_lda, dQ, d_ldq, dR,
                                                         d_ldr, d_info, workspace, workspace_bytes, st);
}

int batched_svd_jacobi(int dtype, int batch, int max_m, int max_n, void* const* dA, const int* d_m, const int* d_n,
                       const int* d_lda, void* const* dS, void* const* dU, const int* d_ldu, void* const* dV,
                       const int* d_ldv, double tol, int max_sweeps, int tier, int* d_info, long long* d_rotations,
                       void* stream)
{
    if (dtype != BSVD_F32 && dtype != BSVD_F64) return -1;
    if (batch < 0) return -2;
    if (max_m < 0) return -3;
    if (max_n < 0) return -4;
    if ((tier & 0xff) != BSVD_TIER_AUTO && (tier & 0xff) != BSVD_TIER_REGISTER && (tier & 0xff) != BSVD_TIER_SHARED)
        return -16;
    if ((tier & 0xff) == BSVD_TIER_SHARED && (tier >> 8) != 0) return -16;
    if (batch == 0) return BSVD_SUCCESS;
    if (!dA) return -5;
    if (!d_m) return -6;
    if (!d_n) return -7;
    if (!d_lda) return -8;
    if (!dS) return -9;
    if (dU && !d_ldu) return -11;
    if (dV && !d_ldv) return -13;
    if (!(tol == tol)) return -14;  // NaN
    if (!d_info) return -17;
    cudaStream_t st = (cudaStream_t)stream;
    return dtype == BSVD_F32 ? svd_dispatch<float>(batch, max_m, max_n, tier, dA, d_m, d_n, d_lda, dS, dU, d_ldu, dV,
                                                   d_ldv, tol, max_sweeps, d_info, d_rotations, st)
                             : svd_dispatch<double>(batch, max_m, max_n, tier, dA, d_m, d_n, d_lda, dS, dU, d_ldu, dV,
                                                    d_ldv, tol, max_sweeps, d_info, d_rotations, st);
}

int bsvd_jacobi_variant_desc(int dtype, int max_m, int max_n, int k, int* desc)
{
    if (dtype != BSVD_F32 && dtype != BSVD_F64) return -1;
    if (max_m < 0) return -2;
    if (max_n < 0) return -3;
    if (k < 1) return -4;
    if (!desc) return -5;
    return jacobi_reg_variant_desc(dtype == BSVD_F64, max_m, max_n, k, desc);
}

int bsvd_jacobi_variants(int dtype, int max_m, int max_n, int tier)
{
    if (dtype != BSVD_F32 && dtype != BSVD_F64) return -1;
    if (max_m < 0) return -2;
    if (max_n < 0) return -3;
    if (tier == BSVD_TIER_REGISTER)
        return dtype == BSVD_F32 ? launch_jacobi_reg<float>(0, max_m, max_n, -1, nullptr, nullptr, nullptr, nullptr,
                                                            nullptr, nullptr, nullptr, nullptr, nullptr, 0.0, 0,
                                                            nullptr, nullptr, nullptr)
                                 : launch_jacobi_reg<double>(0, max_m, max_n, -1, nullptr, nullptr, nullptr, nullptr,
                                                             nullptr, nullptr, nullptr, nullptr, nullptr, 0.0, 0,
                                                             nullptr, nullptr, nullptr);
    if (tier == BSVD_TIER_SHARED) {
        const int mm = max_m > max_n ? max_m : max_n, nn = max_m > max_n ? max_n : max_m;
        return (mm <= 256 && nn <= (dtype == BSVD_F32 ? 128 : 64)) ? 1 : 0;
    }
    return -4;
}

int bsvd_set_jacobi_choice(int dtype, int max_m, int max_n, int tier)
{
    if (dtype != BSVD_F32 && dtype != BSVD_F64) return -1;
    if (max_m < 0 || max_m > 256) return -2;
    if (max_n < 0 || max_n > 256) return -3;
    const int base = tier & 0xff;
    if (base != BSVD_TIER_AUTO && base != BSVD_TIER_REGISTER && base != BSVD_TIER_SHARED) return -4;
    const int mm = max_m > max_n ? max_m : max_n, nn = max_m > max_n ? max_n : max_m;
    g_choice[dtype == BSVD_F64][size_bin(mm)][size_bin(nn)].store(base == BSVD_TIER_AUTO ? 0 : tier,
                                                                 std::memory_order_relaxed);
    return BSVD_SUCCESS;
}

int bsvd_set_block_choice(int dtype, int max_m, int max_n, int block_width, int inner_variant)
{
    if (dtype != BSVD_F32 && dtype != BSVD_F64) return -1;
    if (max_m < 0 || max_m > 16384) return -2;
    if (max_n < 0 || max_n > 16384) return -3;
    if (block_width != 0 && block_width != 16 && block_width != 32) return -4;
    if (inner_variant < 0 || inner_variant > 255 || (block_width == 0 && inner_variant != 0)) return -5;
    const int mm = max_m > max_n ? max_m : max_n, nn = max_m > max_n ? max_n : max_m;
    g_block_choice[dtype == BSVD_F64][block_bin(mm)][block_bin(nn)].store(
        block_width == 0 ? 0 : (block_width | inner_variant << 8), std::memory_order_relaxed);
    return BSVD_SUCCESS;
}

size_t batched_svd_block_jacobi_workspace(int dtype, int batch, int max_m, int max_n, int block_width, int method)
{
    if ((dtype != BSVD_F32 && dtype != BSVD_F64) || batch < 0 || max_m < 0 || max_n < 0) return 0;
    block_width = resolve_block_choice(dtype, max_m, max_n, block_width, &method);
    const int base = method & 0xff;
    if ((block_width != 16 && block_width != 32) || (base != BSVD_BLOCK_GRAM && base != BSVD_BLOCK_DIRECT)) return 0;
    const int m2 = base | (method & BSVD_BLOCK_QR_PRECONDITION);
    return dtype == BSVD_F32 ? block_jacobi_workspace<float>(batch, max_m, max_n, block_width, m2)
                             : block_jacobi_workspace<double>(batch, max_m, max_n, block_width, m2);
}

int batched_svd_block_jacobi(int dtype, int batch, int max_m, int max_n, void* const* dA, const int* d_m,
                             const int* d_n, const int* d_lda, void* const* dS, void* const* dU, const int* d_ldu,
                             void* const* dV, const int* d_ldv, double tol, int max_sweeps, int block_width,
                             int method, int* d_info, long long* d_rotations, void* workspace, size_t workspace_bytes,
                             void* stream)
{
    if (dtype != BSVD_F32 && dtype != BSVD_F64) return -1;
    if (batch < 0) return -2;
    if (max_m < 0) return -3;
    if (max_n < 0) return -4;
    if (batch == 0) return BSVD_SUCCESS;
    if (!dA) return -5;
    if (!d_m) return -6;
    if (!d_n) return -7;
    if (!d_lda) return -8;
    if (!dS) return -9;
    if (!dU) return -10;
    if (!d_ldu) return -11;
    if (!dV) return -12;
    if (!d_ldv) return -13;
    if (!(tol == tol)) return -14;
    if (block_width != 0 && block_width != 16 && block_width != 32) return -16;
    block_width = resolve_block_choice(dtype, max_m, max_n, block_width, &method);
    if ((method & 0xff) != BSVD_BLOCK_GRAM && (method & 0xff) != BSVD_BLOCK_DIRECT) return -17;
    // method bits: 0-7 method, 8-15 inner variant, 16 SIMT Gram products, 17 failure-path test,
    // 18 QR preconditioning, 19 re-test every pair, 24-30 inner sweep cap
    if (method & ~(0xffff | BSVD_BLOCK_SIMT_PRODUCTS | BSVD_BLOCK_TEST_TIMEOUT | BSVD_BLOCK_QR_PRECONDITION |
                   BSVD_BLOCK_RETEST_ALL | (0x7f << 24)))
        return -17;
    if (!d_info) return -18;
    if (!workspace) return -20;
    cudaStream_t st = (cudaStream_t)stream;
    return dtype == BSVD_F32
               ? launch_block_jacobi<float>(batch, max_m, max_n, block_width, method, dA, d_m, d_n, d_lda, dS, dU, d_ldu,
                                            dV, d_ldv, tol, max_sweeps, d_info, d_rotations, workspace, workspace_bytes, st)
               : launch_block_jacobi<double>(batch, max_m, max_n, block_width, method, dA, d_m, d_n, d_lda, dS, dU,
                                             d_ldu, dV, d_ldv, tol, max_sweeps, d_info, d_rotations, workspace,
                                             workspace_bytes, st);
}

size_t batched_rsvd_workspace(int dtype, int batch, int max_m, int max_n, const int* h_m, const int* h_n)
{
    if ((dtype != BSVD_F32 && dtype != BSVD_F64) || batch < 0 || max_m < 0 || max_n < 0 || max_m > 256 ||
        max_n > 256)
        return 0;
    return dtype == BSVD_F32 ? rsvd_workspace<float>(batch, max_m, max_n, h_m, h_n)
                             : rsvd_workspace<double>(batch, max_m, max_n, h_m, h_n);
}

int batched_rsvd(int dtype, int batch, int max_m, int max_n, void* const* dA, const int* d_m, const int* d_n,
                 const int* d_lda, const int* d_rank, const int* d_rank_hint, const double* d_tol, double tol,
                 int oversample, int power_iters, int max_rounds, unsigned long long seed, int flags, void* const* dU,
                 const int* d_ldu, void* const* dS, void* const* dV, const int* d_ldv, const int* d_kmax,
                 int* d_rank_out, float* d_err_est, int* d_samples, int* d_info, void* workspace,
                 size_t workspace_bytes, void* stream)
{
    if (dtype != BSVD_F32 && dtype != BSVD_F64) return -1;
    if (batch < 0) return -2;
    if (max_m < 0) return -3;
    if (max_n < 0) return -4;
    if (batch == 0) return BSVD_SUCCESS;
    if (max_m > 256 || max_n > 256) return BSVD_ERR_UNSUPPORTED;
    if (!dA) return -5;
    if (!d_m) return -6;
    if (!d_n) return -7;
    if (!d_lda) return -8;
    if (!(tol >= 0.0 && tol < 1.0)) return -12;
    if (oversample < 1 || oversample > 64) return -13;
    if (power_iters < 0 || power_iters > 8) return -14;
    if (max_rounds < 1 || max_rounds > 64) return -15;
    if (flags & ~(BSVD_RSVD_SMALL_FP64 | BSVD_RSVD_TC_SAMPLING)) return -17;
    if (!dU) return -18;
    if (!d_ldu) return -19;
    if (!dS) return -20;
    if (!dV) return -21;
    if (!d_ldv) return -22;
    if (!d_kmax) return -23;
    if (!d_rank_out) return -24;
    if (!d_info) return -27;
    if (!workspace) return -28;
    cudaStream_t st = (cudaStream_t)stream;
    return dtype == BSVD_F32
               ? launch_rsvd<float>(batch, max_m, max_n, dA, d_m, d_n, d_lda, d_rank, d_rank_hint, d_tol, tol, d_kmax,
                                    oversample, power_iters, max_rounds, seed, flags, dU, d_ldu, dS, dV, d_ldv, d_rank_out,
                                    d_err_est, d_samples, d_info, workspace, workspace_bytes, st)
               : launch_rsvd<double>(batch, max_m, max_n, dA, d_m, d_n, d_lda, d_rank, d_rank_hint, d_tol, tol,
                                     d_kmax, oversample, power_iters, max_rounds, seed, flags, dU, d_ldu, dS, dV, d_ldv,
                                     d_rank_out, d_err_est, d_samples, d_info, workspace, workspace_bytes, st);
}

size_t bsvd_h2_truncate_workspace(int dtype, int depth, int k, int max_leaf_m)
{
    if ((dtype != BSVD_F32 && dtype != BSVD_F64) || depth < 0 || depth > 20 || k < 1 || k > 64 || max_leaf_m < 0 ||
        max_leaf_m > 256)
        return 0;
    return dtype == BSVD_F32 ? h2_truncate_workspace<float>(depth, k, max_leaf_m)
                             : h2_truncate_workspace<double>(depth, k, max_leaf_m);
}

int bsvd_h2_truncate(int dtype, int depth, int k, int max_leaf_m, void* const* d_leaf, const int* d_leaf_m,
                     const int* d_leaf_ld, void* const* d_transfer, double eps, void* const* d_new_leaf,
                     const int* d_new_leaf_ld, void* const* d_new_transfer, void* const* d_T, int* d_rank,
                     int* d_info, long long* d_rotations, void* workspace, size_t workspace_bytes, void* stream)
{
    if (dtype != BSVD_F32 && dtype != BSVD_F64) return -1;
    if (depth < 0 || depth > 20) return -2;
    if (k < 1 || k > 64) return -3;
    if (max_leaf_m < 0 || max_leaf_m > 256 || (dtype == BSVD_F64 && max_leaf_m > 256)) return -4;
    if (!d_leaf) return -5;
    if (!d_leaf_m) return -6;
    if (!d_leaf_ld) return -7;
    if (depth > 0 && !d_transfer) return -8;
    if (!(eps >= 0.0 && eps < 1.0)) return -9;
    if (!d_new_leaf) return -10;
    if (!d_new_leaf_ld) return -11;
    if (depth > 0 && !d_new_transfer) return -12;
    if (!d_T) return -13;
    if (!d_rank) return -14;
    if (!d_info) return -15;
    if (!workspace) return -17;
    cudaStream_t st = (cudaStream_t)stream;
    return dtype == BSVD_F32
               ? launch_h2_truncate<float>(depth, k, max_leaf_m, d_leaf, d_leaf_m, d_leaf_ld, d_transfer, eps,
                                           d_new_leaf, d_new_leaf_ld, d_new_transfer, d_T, d_rank, d_info, d_rotations,
                                           workspace, workspace_bytes, st)
               : launch_h2_truncate<double>(depth, k, max_leaf_m, d_leaf, d_leaf_m, d_leaf_ld, d_transfer, eps,
                                            d_new_leaf, d_new_leaf_ld, d_new_transfer, d_T, d_rank, d_info, d_rotations,
                                            workspace, workspace_bytes, st);
}

}  // extern "C"
