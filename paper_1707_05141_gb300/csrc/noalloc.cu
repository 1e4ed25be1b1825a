// noalloc.cu -- an allocation-free variant of batched_svd_block_jacobi.
//
// Some callers cannot hand the library a workspace, nor call cudaMalloc themselves: code that runs
// under a host application's own memory manager that forbids direct driver allocations, or on a
// latency-critical path where cudaMalloc (which may synchronise the device) is not acceptable.
// For them this entry point keeps its scratch in a fixed-size array in device memory that belongs
// to the library, so a call needs nothing beyond the caller's inputs and outputs.
//
// The array is a file-scope __device__ object: every GPU that loads this library holds it until
// the process exits.  In host code its name is only a stand-in, not a device address, so the
// first call on each device, with that device current, looks the address up with
// cudaGetSymbolAddress and remembers it for that device, together with the identifier of the
// context it belongs to.  A later call in another context of that device (after cudaDeviceReset,
// or a primary context released and created again) looks the address up again instead of using
// a stale one.
#include <cuda.h>  // context types only; the driver functions are reached through the runtime
#include <cuda_runtime.h>

#include <mutex>

#include "common.cuh"

namespace bsvd {
template <typename T>
size_t block_jacobi_workspace(int batch, int max_m, int max_n, int bw, int method);
template <typename T>
int launch_block_jacobi(int batch, int max_m, int max_n, int bw, int method, void* const* A, const int* M,
                        const int* N, const int* LDA, void* const* S, void* const* U, const int* LDU, void* const* V,
                        const int* LDV, double tol, int max_sweeps, int* info, long long* rot, void* ws, size_t ws_bytes,
                        cudaStream_t st);
}  // namespace bsvd

namespace {

constexpr size_t kScratchBytes = (size_t)BSVD_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices];                 // device address of g_scratch on each device, once looked up
unsigned long long g_ctx_id[kMaxDevices];  // identifier of the context that address belongs to

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

// Identifier of the calling thread's current context (unique for the life of the process), or 0
// when there is none or it cannot be read.  Called with g_mu held.
unsigned long long current_context_id()
{
    static bool resolved = false;
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    if (!resolved) {
        resolved = true;
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f);
    }
    if (!get_current || !get_id) return 0;
    CUcontext c = nullptr;
    if (get_current(&c) != CUDA_SUCCESS || !c) return 0;
    unsigned long long id = 0;
    return get_id(c, &id) == CUDA_SUCCESS ? id : 0;
}

// Device address of the scratch array on the current device (nullptr on failure).  Looked up once
// per device and context; when the context identifier cannot be read, looked up on every call.
void* scratch_address()
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lock(g_mu);
    const unsigned long long id = current_context_id();
    if (!g_addr[dev] || id == 0 || id != g_ctx_id[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess) return nullptr;
        g_addr[dev] = p;
        g_ctx_id[dev] = current_context_id();  // the lookup makes the device's primary context current
    }
    return g_addr[dev];
}

}  // namespace

extern "C" {

int batched_svd_block_jacobi_noalloc(int dtype, int batch, int max_m, int max_n, void* const* dA, const int* d_m,
                                     const int* d_n, const int* d_lda, void* const* dS, void* const* dU,
                                     const int* d_ldu, void* const* dV, const int* d_ldv, double tol, int max_sweeps,
                                     int block_width, int method, int* d_info, long long* d_rotations, void* stream)
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
    if (block_width != 16 && block_width != 32) return -16;
    if ((method & 0xff) != BSVD_BLOCK_GRAM && (method & 0xff) != BSVD_BLOCK_DIRECT) return -17;
    // method bits: 0-7 method, 8-15 inner variant, 16 SIMT Gram products, 17 failure-path test,
    // 18 QR preconditioning, 24-30 inner sweep cap
    if (method & ~(0xffff | BSVD_BLOCK_SIMT_PRODUCTS | BSVD_BLOCK_TEST_TIMEOUT | BSVD_BLOCK_QR_PRECONDITION |
                   BSVD_BLOCK_RETEST_ALL | (0x7f << 24)))
        return -17;
    if (!d_info) return -18;
    const size_t need = dtype == BSVD_F32
                            ? bsvd::block_jacobi_workspace<float>(batch, max_m, max_n, block_width,
                                                                  method & (0xff | BSVD_BLOCK_QR_PRECONDITION))
                            : bsvd::block_jacobi_workspace<double>(batch, max_m, max_n, block_width,
                                                                   method & (0xff | BSVD_BLOCK_QR_PRECONDITION));
    if (need > kScratchBytes) return BSVD_ERR_SCRATCH_LIMIT;
    void* ws = scratch_address();
    if (!ws) return BSVD_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    return dtype == BSVD_F32
               ? bsvd::launch_block_jacobi<float>(batch, max_m, max_n, block_width, method, dA, d_m, d_n, d_lda, dS, dU,
                                                  d_ldu, dV, d_ldv, tol, max_sweeps, d_info, d_rotations, ws,
                                                  kScratchBytes, st)
               : bsvd::launch_block_jacobi<double>(batch, max_m, max_n, block_width, method, dA, d_m, d_n, d_lda, dS,
                                                   dU, d_ldu, dV, d_ldv, tol, max_sweeps, d_info, d_rotations, ws,
                                                   kScratchBytes, st);
}

}  // extern "C"
