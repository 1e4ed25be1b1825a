// host_pipeline.cu -- host-in, host-out batched QR and Jacobi SVD of uniform batches, with the
// copies overlapped with the computation.
//
// The paper's routines take batches already resident on the GPU; a caller whose matrices live in
// host memory would otherwise copy everything in, compute, and copy everything out in three serial
// phases.  Here the batch is cut into chunks: chunk c is copied in on one stream, computed on a
// compute stream and copied out on another, so that the transfer of chunk c + 1 and the read-back
// of chunk c - 1 run while chunk c is computed; consecutive chunks are computed on two different
// streams, so one chunk's last wave overlaps the next chunk's first.  The device copies of the whole
// batch live in the caller's workspace; the streams and the events are the library's own (created
// once per device and reused), every stream starts after the caller's earlier work, and the
// caller's stream waits for the last read-back, so synchronising it covers the whole call.  Host
// buffers should be page-locked for the copies to overlap.
#include <cuda_runtime.h>

#include <mutex>
#include <vector>

#include "common.cuh"

namespace {

constexpr int kMaxDevices = 64;

struct HostPipe {
    cudaStream_t s_in = nullptr, s_out = nullptr;
    cudaStream_t s_comp[4] = {nullptr, nullptr, nullptr, nullptr};  // compute streams (two per call, in turn)
    int next_pair = 0;
    std::vector<cudaEvent_t> ev;  // 2 per chunk (copied in, computed) + start + done
};
std::mutex g_pipe_mu;
HostPipe g_pipe[kMaxDevices];

// copy streams and at least `nev` events of the current device (nullptr on failure)
HostPipe* host_pipe(int nev)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    HostPipe& p = g_pipe[dev];
    if (!p.s_in && cudaStreamCreateWithFlags(&p.s_in, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
    if (!p.s_out && cudaStreamCreateWithFlags(&p.s_out, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
    for (int i = 0; i < 4; ++i)
        if (!p.s_comp[i] && cudaStreamCreateWithFlags(&p.s_comp[i], cudaStreamNonBlocking) != cudaSuccess)
            return nullptr;
    while ((int)p.ev.size() < nev) {
        cudaEvent_t e;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return nullptr;
        p.ev.push_back(e);
    }
    return &p;
}

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// device layout of one uniform batch: `na` matrices per item (inputs then outputs), each of the
// given element count, then the pointer arrays (one per matrix kind) and the size arrays
struct HostLayout {
    size_t off[6];        // element arrays (bytes)
    size_t cnt[6];        // elements per matrix of each kind
    size_t off_ptr, off_int, total;
    int kinds;
};

HostLayout host_layout(int batch, size_t es, const size_t* per, int kinds)
{
    HostLayout L;
    L.kinds = kinds;
    size_t o = 0;
    for (int i = 0; i < kinds; ++i) {
        L.cnt[i] = per[i];
        L.off[i] = o;
        o = al256(o + es * per[i] * (size_t)batch);
    }
    L.off_ptr = o;
    o = al256(o + sizeof(void*) * (size_t)batch * kinds);
    L.off_int = o;
    o = al256(o + sizeof(int) * (size_t)batch * 8);
    L.total = o;
    return L;
}

// pointer arrays (matrix b of kind i at base_i + b * cnt_i elements) and constant size arrays
__global__ void host_setup_kernel(int batch, int kinds, unsigned char* ws, HostLayout L, size_t es, int a0, int a1,
                                  int a2, int a3, int a4, int a5, int a6, int a7)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= batch) return;
    void** p = reinterpret_cast<void**>(ws + L.off_ptr);
    for (int i = 0; i < kinds; ++i) p[(size_t)i * batch + b] = ws + L.off[i] + es * L.cnt[i] * (size_t)b;
    int* q = reinterpret_cast<int*>(ws + L.off_int);
    const int v[8] = {a0, a1, a2, a3, a4, a5, a6, a7};
    for (int i = 0; i < 8; ++i) q[(size_t)i * batch + b] = v[i];
}

// one chunked host -> device -> host pass; `compute(c0, c1, s)` enqueues the batched call for
// matrices c0 .. c1 - 1 on stream s; kinds [0, nin) are copied in, [nin, kinds) copied out (plus the
// info array).  Chunks alternate between two of the library's compute streams, so the last wave of
// one chunk's kernel shares the GPU with the first waves of the next instead of leaving SMs idle;
// the next call of the library takes the other two streams.
template <typename F>
int host_run(int batch, int chunks, const HostLayout& L, size_t es, unsigned char* ws, const void* const* host,
             int nin, int* h_info, int* d_info, cudaStream_t st, F compute)
{
    if (chunks < 1) chunks = 1;
    if (chunks > batch) chunks = batch;
    const int step = (batch + chunks - 1) / chunks;
    const int nch = (batch + step - 1) / step;
    std::lock_guard<std::mutex> lock(g_pipe_mu);
    HostPipe* P = host_pipe(2 * nch + 2);
    if (!P) return BSVD_ERR_CUDA;
    cudaEvent_t ev_start = P->ev[2 * nch], ev_done = P->ev[2 * nch + 1];
    // the copy streams start after the caller's earlier work (and after the pointer setup)
    if (cudaEventRecord(ev_start, st) != cudaSuccess) return BSVD_ERR_CUDA;
    if (cudaStreamWaitEvent(P->s_in, ev_start, 0) != cudaSuccess) return BSVD_ERR_CUDA;
    if (cudaStreamWaitEvent(P->s_out, ev_start, 0) != cudaSuccess) return BSVD_ERR_CUDA;
    cudaStream_t sc[2] = {P->s_comp[P->next_pair], P->s_comp[P->next_pair + 1]};
    P->next_pair ^= 2;
    for (int i = 0; i < 2; ++i)
        if (cudaStreamWaitEvent(sc[i], ev_start, 0) != cudaSuccess) return BSVD_ERR_CUDA;
    for (int c = 0; c < nch; ++c) {
        const int c0 = c * step, c1 = c0 + step < batch ? c0 + step : batch;
        const size_t nb = (size_t)(c1 - c0);
        for (int i = 0; i < nin; ++i) {
            const size_t bytes = es * L.cnt[i] * nb, from = es * L.cnt[i] * (size_t)c0;
            if (cudaMemcpyAsync(ws + L.off[i] + from, static_cast<const unsigned char*>(host[i]) + from, bytes,
                                cudaMemcpyHostToDevice, P->s_in) != cudaSuccess)
                return BSVD_ERR_CUDA;
        }
        cudaEvent_t ev_in = P->ev[2 * c], ev_comp = P->ev[2 * c + 1];
        if (cudaEventRecord(ev_in, P->s_in) != cudaSuccess) return BSVD_ERR_CUDA;
        cudaStream_t cs = sc[c & 1];
        if (cudaStreamWaitEvent(cs, ev_in, 0) != cudaSuccess) return BSVD_ERR_CUDA;
        const int rc = compute(c0, c1, cs);
        if (rc != BSVD_SUCCESS) return rc;
        if (cudaEventRecord(ev_comp, cs) != cudaSuccess) return BSVD_ERR_CUDA;
        if (cudaStreamWaitEvent(P->s_out, ev_comp, 0) != cudaSuccess) return BSVD_ERR_CUDA;
        for (int i = nin; i < L.kinds; ++i) {
            if (!host[i]) continue;
            const size_t bytes = es * L.cnt[i] * nb, from = es * L.cnt[i] * (size_t)c0;
            if (cudaMemcpyAsync(static_cast<unsigned char*>(const_cast<void*>(host[i])) + from,
                                ws + L.off[i] + from, bytes, cudaMemcpyDeviceToHost, P->s_out) != cudaSuccess)
                return BSVD_ERR_CUDA;
        }
        if (h_info && cudaMemcpyAsync(h_info + c0, d_info + c0, sizeof(int) * nb, cudaMemcpyDeviceToHost, P->s_out) !=
                          cudaSuccess)
            return BSVD_ERR_CUDA;
    }
    // the caller's stream completes only after the last read-back (which follows every chunk's
    // computation)
    if (cudaEventRecord(ev_done, P->s_out) != cudaSuccess) return BSVD_ERR_CUDA;
    if (cudaStreamWaitEvent(st, ev_done, 0) != cudaSuccess) return BSVD_ERR_CUDA;
    return BSVD_SUCCESS;
}

bool host_args_ok(int dtype, int batch, int m, int n) { return (dtype == BSVD_F32 || dtype == BSVD_F64) && batch >= 0 && m >= 0 && n >= 0; }

HostLayout svd_layout(int dtype, int batch, int m, int n)
{
    const size_t k = m < n ? m : n;
    const size_t per[5] = {(size_t)m * n, k, (size_t)m * k, (size_t)n * k, 1};  // A, S, U, V, info (ints)
    return host_layout(batch, dtype == BSVD_F32 ? 4 : 8, per, 5);
}

HostLayout qr_layout(int dtype, int batch, int m, int n)
{
    const size_t per[4] = {(size_t)m * n, (size_t)m * n, (size_t)n * n, 1};     // A, Q, R, info (ints)
    return host_layout(batch, dtype == BSVD_F32 ? 4 : 8, per, 4);
}

}  // namespace

extern "C" {

size_t bsvd_host_svd_workspace(int dtype, int batch, int m, int n)
{
    if (!host_args_ok(dtype, batch, m, n)) return 0;
    return svd_layout(dtype, batch, m, n).total;
}

int bsvd_host_svd(int dtype, int batch, int m, int n, const void* hA, void* hS, void* hU, void* hV, int* h_info,
                  int chunks, void* workspace, size_t workspace_bytes, void* stream)
{
    if (dtype != BSVD_F32 && dtype != BSVD_F64) return -1;
    if (batch < 0) return -2;
    if (m < 0) return -3;
    if (n < 0) return -4;
    if (batch == 0) return BSVD_SUCCESS;
    if (!hA) return -5;
    if (!hS) return -6;
    if (!workspace) return -11;
    const HostLayout L = svd_layout(dtype, batch, m, n);
    if (workspace_bytes < L.total) return BSVD_ERR_WORKSPACE;
    unsigned char* ws = static_cast<unsigned char*>(workspace);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t es = dtype == BSVD_F32 ? 4 : 8;
    const int k = m < n ? m : n;
    // the info array is the fifth kind (its elements are ints: one per matrix, es bytes reserved)
    host_setup_kernel<<<(batch + 127) / 128, 128, 0, st>>>(batch, 4, ws, L, es, m, n, m > 1 ? m : 1, k, 1,
                                                          m > 1 ? m : 1, n > 1 ? n : 1, 0);
    if (cudaGetLastError() != cudaSuccess) return BSVD_ERR_CUDA;
    void** p = reinterpret_cast<void**>(ws + L.off_ptr);
    int* q = reinterpret_cast<int*>(ws + L.off_int);
    int* d_info = reinterpret_cast<int*>(ws + L.off[4]);
    const void* host[4] = {hA, hS, hU, hV};
    HostLayout Lc = L;
    Lc.kinds = 4;
    return host_run(batch, chunks, Lc, es, ws, host, 1, h_info, d_info, st, [&](int c0, int c1, cudaStream_t cs) {
        const int nb = c1 - c0;
        return batched_svd_jacobi(dtype, nb, m, n, p + c0, q + c0, q + (size_t)batch + c0,
                                  q + 2 * (size_t)batch + c0, p + (size_t)batch + c0,
                                  hU ? p + 2 * (size_t)batch + c0 : nullptr, q + 5 * (size_t)batch + c0,
                                  hV ? p + 3 * (size_t)batch + c0 : nullptr, q + 6 * (size_t)batch + c0, 0.0, 0,
                                  BSVD_TIER_AUTO, d_info + c0, nullptr, cs);
    });
}

size_t bsvd_host_qr_workspace(int dtype, int batch, int m, int n)
{
    if (!host_args_ok(dtype, batch, m, n)) return 0;
    return qr_layout(dtype, batch, m, n).total;
}

int bsvd_host_qr(int dtype, int batch, int m, int n, const void* hA, void* hQ, void* hR, int* h_info, int chunks,
                 void* workspace, size_t workspace_bytes, void* stream)
{
    if (dtype != BSVD_F32 && dtype != BSVD_F64) return -1;
    if (batch < 0) return -2;
    if (m < 0) return -3;
    if (n < 0 || n > m) return -4;
    if (batch == 0) return BSVD_SUCCESS;
    if (!hA) return -5;
    if (!workspace) return -10;
    const HostLayout L = qr_layout(dtype, batch, m, n);
    if (workspace_bytes < L.total) return BSVD_ERR_WORKSPACE;
    unsigned char* ws = static_cast<unsigned char*>(workspace);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t es = dtype == BSVD_F32 ? 4 : 8;
    host_setup_kernel<<<(batch + 127) / 128, 128, 0, st>>>(batch, 3, ws, L, es, m, n, m > 1 ? m : 1, m > 1 ? m : 1,
                                                          n > 1 ? n : 1, 0, 0, 0);
    if (cudaGetLastError() != cudaSuccess) return BSVD_ERR_CUDA;
    void** p = reinterpret_cast<void**>(ws + L.off_ptr);
    int* q = reinterpret_cast<int*>(ws + L.off_int);
    int* d_info = reinterpret_cast<int*>(ws + L.off[3]);
    const void* host[3] = {hA, hQ, hR};
    HostLayout Lc = L;
    Lc.kinds = 3;
    return host_run(batch, chunks, Lc, es, ws, host, 1, h_info, d_info, st, [&](int c0, int c1, cudaStream_t cs) {
        const int nb = c1 - c0;
        return batched_qr(dtype, nb, m, n, p + c0, q + c0, q + (size_t)batch + c0, q + 2 * (size_t)batch + c0,
                          hQ ? p + (size_t)batch + c0 : nullptr, q + 3 * (size_t)batch + c0,
                          hR ? p + 2 * (size_t)batch + c0 : nullptr, q + 4 * (size_t)batch + c0, d_info + c0, cs);
    });
}

}  // extern "C"
