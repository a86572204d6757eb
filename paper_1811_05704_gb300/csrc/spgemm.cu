// spgemm.cu -- the Galerkin product A_{i+1} = R_i (A_i P_i) of Algorithm 1
// on the GPU, as two row-wise sparse products C = A B.
//
// Row i of C is accumulated in a hash table in shared memory: a warp per row
// (table of kWarpSlots) while the row has at most kWarpSlots/2 distinct
// columns, else a block per row (table of kBlockSlots).  The symbolic pass
// counts distinct columns exactly; the numeric pass accumulates
//     c_ij = ((0 + a_ik1 b_k1j) + a_ik2 b_k2j) + ...
// over the nonzeros of row i of A in ascending k, with explicit
// round-to-nearest multiply and add (no FMA contraction): the lanes of a step
// handle distinct columns of one row of B, and steps are ordered by a warp or
// block barrier.  The result is therefore independent of scheduling and equal
// bit for bit to the sequential row-by-row product.  Columns are sorted by a
// rank sort before they are written.  Numerical zeros are kept (the pattern is
// structural).
#include <cuda_runtime.h>

#include "amg_internal.h"

namespace amg {

namespace {

constexpr int kWarpSlots = 1024;   // per warp; used while distinct <= 512
constexpr int kWarpCap = kWarpSlots / 2;
constexpr int kBlockSlots = 8192;  // per block; used while distinct <= 4096
constexpr int kBlockCap = kBlockSlots / 2;
constexpr int kBlockThreads = 512;
constexpr int kWarpsPerBlock = 4;
constexpr int kEmpty = -1;

__device__ __forceinline__ unsigned slot_of(int key, unsigned mask) {
    return ((unsigned)key * 2654435761u) & mask;
}

// Insert key; returns the slot, or -1 if the probe sequence found no room
// (cannot happen while the load stays below the table size, but the loop is
// bounded and the caller raises an error flag instead of spinning).
__device__ __forceinline__ int insert(int* keys, unsigned mask, int key, bool& added) {
    unsigned h = slot_of(key, mask);
    added = false;
    for (unsigned probe = 0; probe <= mask; ++probe) {
        const int prev = atomicCAS(keys + h, kEmpty, key);
        if (prev == kEmpty) { added = true; return (int)h; }
        if (prev == key) return (int)h;
        h = (h + 1) & mask;
    }
    return -1;
}

// error bits: 1 = table overflow (probe failed), 2 = row too wide, 4 = nnz overflow

// ------------------------------------------------------------- symbolic
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
k_sym_warp(int32_t m, const int32_t* __restrict__ ap, const int32_t* __restrict__ ac,
           const int32_t* __restrict__ bp, const int32_t* __restrict__ bc,
           int32_t* __restrict__ count, int32_t* __restrict__ big, int32_t* __restrict__ nbig,
           int* __restrict__ err) {
    __shared__ int keys[kWarpsPerBlock][kWarpSlots];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = blockIdx.x * kWarpsPerBlock + warp;
    if (row >= m) return;
    int* tab = keys[warp];
    for (int i = lane; i < kWarpSlots; i += 32) tab[i] = kEmpty;
    __syncwarp();
    int distinct = 0;
    bool overflow = false;
    for (int ka = ap[row]; ka < ap[row + 1] && !overflow; ++ka) {
        const int k = ac[ka];
        const int b0 = bp[k], b1 = bp[k + 1];
        for (int kb = b0; kb < b1; kb += 32) {
            bool added = false;
            if (kb + lane < b1) {
                if (insert(tab, kWarpSlots - 1, bc[kb + lane], added) < 0) atomicOr(err, 1);
            }
            distinct += __popc(__ballot_sync(0xffffffffu, added));
            __syncwarp();
            if (distinct > kWarpCap) { overflow = true; break; }
        }
    }
    if (lane == 0) {
        if (overflow) {
            count[row] = -1;
            big[atomicAdd(nbig, 1)] = row;
        } else {
            count[row] = distinct;
        }
    }
}

__global__ void __launch_bounds__(kBlockThreads)
k_sym_block(const int32_t* __restrict__ rows, const int32_t* __restrict__ ap,
            const int32_t* __restrict__ ac, const int32_t* __restrict__ bp,
            const int32_t* __restrict__ bc, int32_t* __restrict__ count, int* __restrict__ err) {
    extern __shared__ int smem[];
    int* tab = smem;
    __shared__ int distinct;
    const int row = rows[blockIdx.x];
    for (int i = threadIdx.x; i < kBlockSlots; i += kBlockThreads) tab[i] = kEmpty;
    if (threadIdx.x == 0) distinct = 0;
    __syncthreads();
    for (int ka = ap[row]; ka < ap[row + 1]; ++ka) {
        const int k = ac[ka];
        for (int kb = bp[k] + threadIdx.x; kb < bp[k + 1]; kb += kBlockThreads) {
            bool added = false;
            if (insert(tab, kBlockSlots - 1, bc[kb], added) < 0) atomicOr(err, 1);
            if (added) atomicAdd(&distinct, 1);
        }
        __syncthreads();
        const int seen = distinct;
        __syncthreads();  // every thread has read `distinct` before the next step adds to it
        if (seen > kBlockCap) break;
    }
    if (threadIdx.x == 0) {
        if (distinct > kBlockCap) atomicOr(err, 2);
        count[row] = distinct;
    }
}

// exclusive scan of counts into ptr (m + 1 entries) by one block
__global__ void __launch_bounds__(1024)
k_scan(int32_t m, const int32_t* __restrict__ count, int32_t* __restrict__ ptr,
       int* __restrict__ err) {
    __shared__ long long part[1024];
    const int t = threadIdx.x;
    const int64_t chunk = ((int64_t)m + 1023) / 1024;
    const int64_t b = t * chunk, e = min((int64_t)m, b + chunk);
    long long s = 0;
    for (int64_t i = b; i < e; ++i) s += count[i];
    part[t] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {  // inclusive Hillis-Steele
        long long v = (t >= o) ? part[t - o] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    long long run = (t == 0) ? 0 : part[t - 1];
    if (part[1023] >= (1LL << 31) - 1) {
        if (t == 0) atomicOr(err, 4);
        return;
    }
    for (int64_t i = b; i < e; ++i) {
        ptr[i] = (int32_t)run;
        run += count[i];
    }
    if (t == 1023) ptr[m] = (int32_t)part[1023];
}

// -------------------------------------------------------------- numeric
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
k_num_warp(int32_t m, const int32_t* __restrict__ ap, const int32_t* __restrict__ ac,
           const double* __restrict__ av, const int32_t* __restrict__ bp,
           const int32_t* __restrict__ bc, const double* __restrict__ bv,
           const int32_t* __restrict__ count, const int32_t* __restrict__ cp,
           int32_t* __restrict__ cc, double* __restrict__ cv, int* __restrict__ err) {
    extern __shared__ unsigned char raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = blockIdx.x * kWarpsPerBlock + warp;
    if (row >= m) return;
    if (count[row] < 0 || count[row] > kWarpCap) return;  // handled by the block kernel
    double* vals = reinterpret_cast<double*>(raw) + warp * kWarpSlots;
    int* keys = reinterpret_cast<int*>(reinterpret_cast<double*>(raw) + kWarpsPerBlock * kWarpSlots) +
                warp * (kWarpSlots + kWarpCap);
    int* lst = keys + kWarpSlots;  // compacted slot list, kWarpCap entries
    for (int i = lane; i < kWarpSlots; i += 32) { keys[i] = kEmpty; vals[i] = 0.0; }
    __syncwarp();
    for (int ka = ap[row]; ka < ap[row + 1]; ++ka) {
        const int k = ac[ka];
        const double a = av[ka];
        const int b0 = bp[k], b1 = bp[k + 1];
        for (int kb = b0 + lane; kb < b1; kb += 32) {  // distinct columns: no two lanes share a slot
            bool added;
            const int sl = insert(keys, kWarpSlots - 1, bc[kb], added);
            if (sl < 0) atomicOr(err, 1);
            else vals[sl] = __dadd_rn(vals[sl], __dmul_rn(a, bv[kb]));
        }
        __syncwarp();  // orders the steps: each slot sees its products in ascending k
    }
    // compact occupied slots (in slot order), then rank-sort by column
    int base = 0;
    for (int i0 = 0; i0 < kWarpSlots; i0 += 32) {
        const bool occ = keys[i0 + lane] != kEmpty;
        const unsigned msk = __ballot_sync(0xffffffffu, occ);
        const int pos = base + __popc(msk & ((1u << lane) - 1u));
        if (occ && pos < kWarpCap) lst[pos] = i0 + lane;
        base += __popc(msk);
    }
    __syncwarp();
    const int n = base;
    const int out0 = cp[row];
    if (n != count[row] || n > kWarpCap) {  // symbolic and numeric disagree: write nothing
        if (lane == 0) atomicOr(err, 1);
        return;
    }
    for (int e = lane; e < n; e += 32) {
        const int key = keys[lst[e]];
        int rank = 0;
        for (int j = 0; j < n; ++j) rank += keys[lst[j]] < key;
        cc[out0 + rank] = key;
        cv[out0 + rank] = vals[lst[e]];
    }
}

__global__ void __launch_bounds__(kBlockThreads)
k_num_block(const int32_t* __restrict__ rows, const int32_t* __restrict__ ap,
            const int32_t* __restrict__ ac, const double* __restrict__ av,
            const int32_t* __restrict__ bp, const int32_t* __restrict__ bc,
            const double* __restrict__ bv, const int32_t* __restrict__ cp,
            int32_t* __restrict__ cc, double* __restrict__ cv, int* __restrict__ err) {
    extern __shared__ unsigned char raw[];
    double* vals = reinterpret_cast<double*>(raw);
    int* keys = reinterpret_cast<int*>(vals + kBlockSlots);
    int* lst = keys + kBlockSlots;  // kBlockCap entries
    __shared__ int wbase[kBlockThreads / 32 + 1];
    const int row = rows[blockIdx.x];
    for (int i = threadIdx.x; i < kBlockSlots; i += kBlockThreads) { keys[i] = kEmpty; vals[i] = 0.0; }
    __syncthreads();
    for (int ka = ap[row]; ka < ap[row + 1]; ++ka) {
        const int k = ac[ka];
        const double a = av[ka];
        for (int kb = bp[k] + threadIdx.x; kb < bp[k + 1]; kb += kBlockThreads) {
            bool added;
            const int sl = insert(keys, kBlockSlots - 1, bc[kb], added);
            if (sl < 0) atomicOr(err, 1);
            else vals[sl] = __dadd_rn(vals[sl], __dmul_rn(a, bv[kb]));
        }
        __syncthreads();
    }
    // compact: chunks of kBlockThreads slots, warp ballots + a block prefix
    int total = 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i0 = 0; i0 < kBlockSlots; i0 += kBlockThreads) {
        const bool occ = keys[i0 + threadIdx.x] != kEmpty;
        const unsigned msk = __ballot_sync(0xffffffffu, occ);
        if (lane == 0) wbase[warp] = __popc(msk);
        __syncthreads();
        if (threadIdx.x == 0) {
            int s = 0;
            for (int w = 0; w < kBlockThreads / 32; ++w) { const int c = wbase[w]; wbase[w] = s; s += c; }
            wbase[kBlockThreads / 32] = s;
        }
        __syncthreads();
        if (occ) {
            const int pos = total + wbase[warp] + __popc(msk & ((1u << lane) - 1u));
            if (pos < kBlockCap) lst[pos] = i0 + threadIdx.x;
        }
        total += wbase[kBlockThreads / 32];
        __syncthreads();
    }
    const int n = min(total, kBlockCap);
    const int out0 = cp[row];
    if (total != cp[row + 1] - cp[row]) { if (threadIdx.x == 0) atomicOr(err, 1); return; }
    for (int e = threadIdx.x; e < n; e += kBlockThreads) {
        const int key = keys[lst[e]];
        int rank = 0;
        for (int j = 0; j < n; ++j) rank += keys[lst[j]] < key;
        cc[out0 + rank] = key;
        cv[out0 + rank] = vals[lst[e]];
    }
}

}  // namespace

void device_spgemm(const DevCsr& A, const DevCsr& B, DevCsr& C, cudaStream_t s) {
    const int32_t m = A.nrows;
    C.nrows = m;
    C.ncols = B.ncols;
    int32_t* count = dev_alloc<int32_t>(m > 0 ? m : 1);
    int32_t* big = dev_alloc<int32_t>(m > 0 ? m : 1);
    int32_t* nbig = dev_alloc<int32_t>(1);
    int* err = dev_alloc<int>(1);
    AMG_CUDA(cudaMemsetAsync(nbig, 0, sizeof(int32_t), s));
    AMG_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    C.ptr = dev_alloc<int32_t>(m + 1 + kPad);
    AMG_CUDA(cudaMemsetAsync(C.ptr, 0, (m + 1 + kPad) * sizeof(int32_t), s));

    const unsigned wgrid = (unsigned)((m + kWarpsPerBlock - 1) / kWarpsPerBlock);
    if (m > 0) {
        k_sym_warp<<<wgrid, kWarpsPerBlock * 32, 0, s>>>(m, A.ptr, A.col, B.ptr, B.col, count, big,
                                                          nbig, err);
        AMG_CUDA(cudaGetLastError());
    }
    int32_t hbig = 0;
    AMG_CUDA(cudaMemcpyAsync(&hbig, nbig, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    AMG_CUDA(cudaStreamSynchronize(s));
    const size_t sym_smem = kBlockSlots * sizeof(int);
    const size_t num_block_smem = kBlockSlots * (sizeof(double) + sizeof(int)) + kBlockCap * sizeof(int);
    const size_t num_warp_smem = kWarpsPerBlock * (kWarpSlots * (sizeof(double) + sizeof(int)) +
                                                   kWarpCap * sizeof(int));
    if (hbig > 0) {
        AMG_CUDA(cudaFuncSetAttribute(k_sym_block, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)sym_smem));
        k_sym_block<<<hbig, kBlockThreads, sym_smem, s>>>(big, A.ptr, A.col, B.ptr, B.col, count, err);
        AMG_CUDA(cudaGetLastError());
    }
    k_scan<<<1, 1024, 0, s>>>(m, count, C.ptr, err);
    AMG_CUDA(cudaGetLastError());
    int32_t nnz = 0;
    int herr = 0;
    AMG_CUDA(cudaMemcpyAsync(&nnz, C.ptr + m, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    AMG_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    AMG_CUDA(cudaStreamSynchronize(s));
    auto cleanup = [&]() { dev_free(count); dev_free(big); dev_free(nbig); dev_free(err); };
    if (herr) {
        cleanup();
        dev_free(C.ptr);
        C.ptr = nullptr;
        if (herr & 4) fail(AMG_ERR_TOO_LARGE, "Galerkin product has more than 2^31 nonzeros");
        fail(AMG_ERR_TOO_LARGE, "Galerkin product row wider than 4096 columns");
    }
    C.nnz = nnz;
    C.col = dev_alloc<int32_t>(nnz + kPad);
    C.val = dev_alloc<double>(nnz + kPad);
    AMG_CUDA(cudaMemsetAsync(C.col, 0, (nnz + kPad) * sizeof(int32_t), s));
    AMG_CUDA(cudaMemsetAsync(C.val, 0, (nnz + kPad) * sizeof(double), s));
    if (m > 0) {
        AMG_CUDA(cudaFuncSetAttribute(k_num_warp, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)num_warp_smem));
        k_num_warp<<<wgrid, kWarpsPerBlock * 32, num_warp_smem, s>>>(
            m, A.ptr, A.col, A.val, B.ptr, B.col, B.val, count, C.ptr, C.col, C.val, err);
        AMG_CUDA(cudaGetLastError());
    }
    if (hbig > 0) {
        AMG_CUDA(cudaFuncSetAttribute(k_num_block, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)num_block_smem));
        k_num_block<<<hbig, kBlockThreads, num_block_smem, s>>>(big, A.ptr, A.col, A.val, B.ptr,
                                                                B.col, B.val, C.ptr, C.col, C.val, err);
        AMG_CUDA(cudaGetLastError());
    }
    AMG_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    AMG_CUDA(cudaStreamSynchronize(s));
    cleanup();
    if (herr) fail(AMG_ERR_CUDA, "sparse product numeric phase inconsistent with its symbolic phase");
}

}  // namespace amg
