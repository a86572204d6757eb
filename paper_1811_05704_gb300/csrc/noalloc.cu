// noalloc.cu -- amg_spmv_dot_noalloc: the product y = A x with x.y, using a
// fixed scratch area in device global memory instead of allocating one.
//
// Who needs this: callers that must not allocate device memory once they are
// running -- a latency-critical loop that cannot afford the allocator's locks
// and possible device synchronisation, a process whose device memory is
// entirely reserved up front by another allocator (a framework's caching
// pool), or an environment whose rules forbid dynamic allocation after
// initialisation.  amg_spmv_dot allocates its scratch with cudaMallocAsync on
// every call; this entry point instead uses g_noalloc_scratch below, a static
// array that every GPU loading the library holds until the process exits.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "amg_internal.h"

namespace amg {

// Scratch layout: two arrays of kNoallocMaxBlocks per-block partial sums,
// then the block counter and the error word.
constexpr int kNoallocMaxBlocks = 1 << 16;
constexpr size_t kNoallocBytes = 2 * (size_t)kNoallocMaxBlocks * sizeof(double) + 2 * sizeof(unsigned int);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

// The array's name in host code is a host-side stand-in, not a device
// address: its address on each device is looked up once, with that device
// current, and cached here.
static std::mutex g_noalloc_mutex;
static void* g_noalloc_addr[64] = {nullptr};

static unsigned char* noalloc_scratch_on_current_device() {
    int dev = 0;
    AMG_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) fail(AMG_ERR_INVALID_ARG, "device ordinal above 63");
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            fail(AMG_ERR_CUDA, std::string("cudaGetSymbolAddress of the static scratch: ") +
                                   cudaGetErrorString(e));
        }
        g_noalloc_addr[dev] = p;
    }
    return static_cast<unsigned char*>(g_noalloc_addr[dev]);
}

amg_status spmv_dot_noalloc(const amg_csr* A, const double* x, double* y, double* dot, void* stream) {
    if (!A || !A->on_device || !A->row_ptr || !A->col || !A->val || !x || !y || !dot || x == y)
        fail(AMG_ERR_INVALID_ARG, "bad arguments (the matrix must be on the device)");
    if (A->n < 1 || A->n >= (1LL << 31) - 1 || A->nnz < 0 || A->nnz >= (1LL << 31) - 1)
        fail(AMG_ERR_INVALID_ARG, "n must be in [1, 2^31) and nnz in [0, 2^31)");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int32_t n = (int32_t)A->n;
    const double avg = (double)A->nnz / (double)n;
    int rpb = kRowsPerBlock;
    while (rpb > 1 && rpb * avg > kTileNnz) rpb >>= 1;
    const int64_t nb = ((int64_t)n + rpb - 1) / rpb;
    if (nb > kNoallocMaxBlocks)
        fail(AMG_ERR_TOO_LARGE, "matrix needs " + std::to_string(nb) + " row blocks; the static scratch of "
                                "amg_spmv_dot_noalloc holds " + std::to_string(kNoallocMaxBlocks));

    unsigned char* base = noalloc_scratch_on_current_device();
    double* partial = reinterpret_cast<double*>(base);
    unsigned int* counter = reinterpret_cast<unsigned int*>(base + 2 * (size_t)kNoallocMaxBlocks * sizeof(double));
    int* err = reinterpret_cast<int*>(counter + 1);
    // the array keeps the previous call's contents: clear counter and error word
    AMG_CUDA(cudaMemsetAsync(counter, 0, 2 * sizeof(unsigned int), s));
    launch_validate_csr(n, A->nnz, A->row_ptr, err, s);
    int herr = 0;
    AMG_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    AMG_CUDA(cudaStreamSynchronize(s));
    if (herr) fail(AMG_ERR_INVALID_ARG, "row_ptr is not a valid CSR row pointer");
    Reduce red;
    red.partial = partial;
    red.stride = kNoallocMaxBlocks;
    red.counter = counter;
    red.out = dot;
    red.fin = FIN_NONE;
    launch_spmv_dot_uniform(n, n, A->row_ptr, A->col, A->val, x, y, rpb, red, err, s);
    AMG_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    AMG_CUDA(cudaStreamSynchronize(s));
    if (herr) fail(AMG_ERR_INVALID_ARG, "column index out of range");
    return AMG_OK;
}

}  // namespace amg
