// launch.cuh -- the library's internal launchers, shared by the C boundary (api.cu) and the
// composed drivers (block_jacobi.cu, rsvd.cu).  Every launcher takes device pointer / size arrays
// of one batch, enqueues on `st` and returns a BSVD_* status; `wl` restricts the launch to a device
// list of items (see ItemList).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace bsvd {

template <typename T>
int launch_qr(int batch, int max_m, int max_n, void* const* A, const int* M, const int* N, const int* LDA,
              void* const* Q, const int* LDQ, void* const* R, const int* LDR, int* info, cudaStream_t st,
              ItemList wl = all_items(), bool r_transposed = false,  // r_transposed: R^T written to R
              const int* a_trans = nullptr);  // a_trans[b] != 0: factor A^T (stored n x m, ld LDA)
template <typename T>
int launch_jacobi_reg(int batch, int max_m, int max_n, int variant, void* const* A, const int* M, const int* N,
                      const int* LDA, void* const* S, void* const* U, const int* LDU, void* const* V, const int* LDV,
                      double tol, int max_sweeps, int* info, long long* rot, cudaStream_t st,
                      ItemList wl = all_items());
int jacobi_reg_variant_desc(bool f64, int max_m, int max_n, int k, int* desc);
template <typename T>
int launch_jacobi_smem(int batch, int max_m, int max_n, void* const* A, const int* M, const int* N, const int* LDA,
                       void* const* S, void* const* U, const int* LDU, void* const* V, const int* LDV, double tol,
                       int max_sweeps, int* info, long long* rot, cudaStream_t st, ItemList wl = all_items(),
                       bool p64 = false);  // p64: FP32 data, FP64 rotation parameters
// the register-resident form of the shared tier (FP32, max(m, n) <= 128); BSVD_ERR_UNSUPPORTED otherwise
int launch_jacobi_rx(int batch, int max_m, int max_n, void* const* A, const int* M, const int* N, const int* LDA,
                     void* const* S, void* const* U, const int* LDU, void* const* V, const int* LDV, double tol,
                     int max_sweeps, int* info, long long* rot, cudaStream_t st, ItemList wl, bool p64);
template <typename T>
size_t block_jacobi_workspace(int batch, int max_m, int max_n, int bw, int method);  // method: base | QR flag
template <typename T>
size_t block_jacobi_qr_workspace(int batch, int max_m, int max_n, int bw, int method);
template <typename T>
int launch_block_jacobi_qr(int batch, int max_m, int max_n, int bw, int method, void* const* A, const int* M,
                           const int* N, const int* LDA, void* const* S, void* const* U, const int* LDU,
                           void* const* V, const int* LDV, double tol, int max_sweeps, int* info, long long* rot,
                           void* ws, size_t ws_bytes, cudaStream_t st);
// the blocked Householder QR of matrices beyond the shared-memory kernel (qr_blocked.cu)
template <typename T>
size_t qr_blocked_workspace(int batch, int max_m, int max_n);
template <typename T>
int qr_blocked_max_rows();
template <typename T>
int launch_qr_blocked(int batch, int max_m, int max_n, void* const* A, const int* M, const int* N, const int* LDA,
                      void* const* Q, const int* LDQ, void* const* R, const int* LDR, int* info, void* ws,
                      size_t ws_bytes, cudaStream_t st);
template <typename T>
int launch_block_jacobi(int batch, int max_m, int max_n, int bw, int method, void* const* A, const int* M,
                        const int* N, const int* LDA, void* const* S, void* const* U, const int* LDU, void* const* V,
                        const int* LDV, double tol, int max_sweeps, int* info, long long* rot, void* ws, size_t ws_bytes,
                        cudaStream_t st);
template <typename T>
size_t rsvd_workspace(int batch, int max_m, int max_n, const int* h_m, const int* h_n);
template <typename T>
int launch_rsvd(int batch, int max_m, int max_n, void* const* A, const int* M, const int* N, const int* LDA,
                const int* fixed, const int* hint, const double* tol_arr, double tol, const int* kmax, int p, int q,
                int rounds, unsigned long long seed, int flags, void* const* dU, const int* LDU, void* const* dS,
                void* const* dV, const int* LDV, int* rank_out, float* err_est, int* samples, int* info, void* ws,
                size_t ws_bytes, cudaStream_t st);

template <typename T>
size_t h2_truncate_workspace(int depth, int k, int max_leaf_m);
template <typename T>
int launch_h2_truncate(int depth, int k, int max_leaf_m, void* const* leaf, const int* leaf_m, const int* leaf_ld,
                       void* const* transfer, double eps, void* const* new_leaf, const int* new_leaf_ld,
                       void* const* new_transfer, void* const* Tout, int* rank, int* info, long long* rot, void* ws,
                       size_t ws_bytes, cudaStream_t st);

// Y(:, 0:l) = A Omega on the tensor cores (TF32, FP32 accumulation), Y(:, l:l+8) = A W in FP32
// (randomized SVD sampling, FP32 data, m, n <= 256, l <= 128, Y with leading dimension m)
int launch_rs_sample_tc(int batch, ItemList wl, float* const* A, const int* LDA, float* const* Y, const int* M,
                        const int* N, const int* L, unsigned long long seed, int* timeouts, cudaStream_t st);

}  // namespace bsvd
