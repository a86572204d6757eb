// spgemm.cu -- the Galerkin product A_{i+1} = R_i (A_i P_i) of Algorithm 1
// on the GPU, as two row-wise sparse products C = A B.
//
// Row i of C is accumulated in a hash table in shared memory: a warp per row
// (table of kWarpSlots) while the row has at most kWarpSlots/2 distinct
// columns, else a block per row (table of kBlockSlots) while it has at most
// kBlockSlots/2; wider rows (the dense coarse levels of problems with strong
// coefficient jumps) go to a block with a dense accumulator of all columns in
// global memory (L2-resident at the sizes where it occurs).  The symbolic pass
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

#include <algorithm>
#include <vector>

#include "amg_internal.h"

namespace amg {

namespace {

constexpr int kWarpSlots = 1024;   // per warp; used while distinct <= 512
constexpr int kWarpCap = kWarpSlots / 2;
constexpr int kBlockSlots = 8192;  // per block; used while distinct <= 4096
constexpr int kBlockCap = kBlockSlots / 2;
constexpr int kBlockThreads = 512;
constexpr int kWarpsPerBlock = 4;
constexpr int kSmallSlots = 128;   // small-row instances: per warp, used while distinct <= 64
constexpr int kSmallCap = kSmallSlots / 2;
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

// error bit 1: table overflow (probe failed) or symbolic and numeric disagree

// ------------------------------------------------------------- symbolic
// A warp per row.  Two instances: SMALL (128-slot tables, 8 warps a block)
// takes the rows whose bound on distinct columns (the sum of the lengths of
// the rows of B they touch) is at most 64 -- nearly every row of the finest
// levels -- with many warps resident per SM; the large one (1024-slot
// tables) takes the others.
// The large instance runs over the list of rows the small one passed on
// (`lst`, *nlst entries, a warp each), and lists the rows it finds to have
// more than kSmallCap distinct columns for the large numeric instance
// (`mid`, *nmid).
template <bool SMALL>
__global__ void __launch_bounds__((SMALL ? 8 : kWarpsPerBlock) * 32)
k_sym_warp(int32_t m, const int32_t* __restrict__ ap, const int32_t* __restrict__ ac,
           const int32_t* __restrict__ bp, const int32_t* __restrict__ bc,
           int32_t* __restrict__ count, int32_t* __restrict__ big, int32_t* __restrict__ nbig,
           int32_t* __restrict__ lst, int32_t* __restrict__ nlst, int32_t* __restrict__ mid,
           int32_t* __restrict__ nmid, int* __restrict__ err) {
    constexpr int WARPS = SMALL ? 8 : kWarpsPerBlock;
    constexpr int SLOTS = SMALL ? kSmallSlots : kWarpSlots;
    constexpr int CAP = SMALL ? kSmallCap : kWarpCap;
    __shared__ int keys[WARPS][SLOTS];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int* tab = keys[warp];
    const int nrows = SMALL ? m : *nlst;
    for (int w = blockIdx.x * WARPS + warp; w < nrows; w += (SMALL ? nrows : gridDim.x * WARPS)) {
    const int row = SMALL ? w : lst[w];
    // the row has at most `bound` distinct columns: a table of twice that
    // (at least 32 slots) is all that has to be cleared
    int bound = 0;
    for (int ka = ap[row] + lane; ka < ap[row + 1]; ka += 32) bound += bp[ac[ka] + 1] - bp[ac[ka]];
    for (int o = 16; o > 0; o >>= 1) bound += __shfl_xor_sync(0xffffffffu, bound, o);
    if (SMALL && bound > kSmallCap) {  // for the large instance
        if (lane == 0) lst[atomicAdd(nlst, 1)] = row;
        continue;
    }
    int slots = 32;
    while (slots < SLOTS && slots < 2 * bound) slots <<= 1;
    const unsigned mask = (unsigned)slots - 1u;
    for (int i = lane; i < slots; i += 32) tab[i] = kEmpty;
    __syncwarp();
    int distinct = 0;
    bool overflow = false;
    for (int ka = ap[row]; ka < ap[row + 1] && !overflow; ++ka) {
        const int k = ac[ka];
        const int b0 = bp[k], b1 = bp[k + 1];
        for (int kb = b0; kb < b1; kb += 32) {
            bool added = false;
            if (kb + lane < b1) {
                if (insert(tab, mask, bc[kb + lane], added) < 0) atomicOr(err, 1);
            }
            distinct += __popc(__ballot_sync(0xffffffffu, added));
            __syncwarp();
            if (distinct > CAP) { overflow = true; break; }
        }
    }
    if (lane == 0) {
        if (overflow) {
            count[row] = -1;
            big[atomicAdd(nbig, 1)] = row;
        } else {
            count[row] = distinct;
            if (!SMALL && distinct > kSmallCap) mid[atomicAdd(nmid, 1)] = row;
        }
    }
    __syncwarp();
    }
}

__global__ void __launch_bounds__(kBlockThreads)
k_sym_block(const int32_t* __restrict__ rows, const int32_t* __restrict__ ap,
            const int32_t* __restrict__ ac, const int32_t* __restrict__ bp,
            const int32_t* __restrict__ bc, int32_t* __restrict__ count,
            int32_t* __restrict__ wide, int32_t* __restrict__ nwide) {
    extern __shared__ int smem[];
    int* tab = smem;
    __shared__ int distinct, full;
    const int row = rows[blockIdx.x];
    for (int i = threadIdx.x; i < kBlockSlots; i += kBlockThreads) tab[i] = kEmpty;
    if (threadIdx.x == 0) { distinct = 0; full = 0; }
    __syncthreads();
    for (int ka = ap[row]; ka < ap[row + 1]; ++ka) {
        const int k = ac[ka];
        for (int kb = bp[k] + threadIdx.x; kb < bp[k + 1]; kb += kBlockThreads) {
            bool added = false;
            if (insert(tab, kBlockSlots - 1, bc[kb], added) < 0) full = 1;  // table full: a wide row
            if (added) atomicAdd(&distinct, 1);
        }
        __syncthreads();
        const bool stop = distinct > kBlockCap || full;
        __syncthreads();  // every thread has read `distinct` before the next step adds to it
        if (stop) break;
    }
    if (threadIdx.x == 0) {
        if (distinct > kBlockCap || full) {
            count[row] = -1;
            wide[atomicAdd(nwide, 1)] = row;
        } else {
            count[row] = distinct;
        }
    }
}

// Sum of v over the block (blockDim.x a multiple of 32, at most 1024); the
// total in every thread.
__device__ __forceinline__ int block_sum_int(int v, int* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    int t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    return t;
}

// Exclusive prefix of v over the block in thread order; *total gets the sum.
__device__ __forceinline__ int block_excl_scan_int(int v, int* sh, int* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    __syncthreads();
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    int before = 0, all = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        if (w < warp) before += sh[w];
        all += sh[w];
    }
    *total = all;
    return before + x - v;
}

// Wide rows, symbolic: a block per row (grid-stride over the wide rows) marks
// the columns it meets in a bit set of all ncols columns (per block, zero on
// entry and left zero), then counts them.
__global__ void __launch_bounds__(kBlockThreads)
k_sym_wide(int32_t nwide, const int32_t* __restrict__ rows, const int32_t* __restrict__ ap,
           const int32_t* __restrict__ ac, const int32_t* __restrict__ bp,
           const int32_t* __restrict__ bc, unsigned* __restrict__ scratch, int64_t words,
           int32_t* __restrict__ count) {
    __shared__ int sh[kBlockThreads / 32];
    unsigned* mark = scratch + (int64_t)blockIdx.x * words;
    for (int w = blockIdx.x; w < nwide; w += gridDim.x) {
        const int row = rows[w];
        for (int ka = ap[row]; ka < ap[row + 1]; ++ka) {
            const int k = ac[ka];
            for (int kb = bp[k] + threadIdx.x; kb < bp[k + 1]; kb += kBlockThreads) {
                const int c = bc[kb];
                atomicOr(mark + (c >> 5), 1u << (c & 31));
            }
        }
        __syncthreads();
        int local = 0;
        for (int64_t i = threadIdx.x; i < words; i += kBlockThreads) {
            local += __popc(mark[i]);
            mark[i] = 0u;
        }
        const int total = block_sum_int(local, sh);
        if (threadIdx.x == 0) count[row] = total;
        __syncthreads();
    }
}

// -------------------------------------------------------------- numeric
template <bool SMALL>
__global__ void __launch_bounds__((SMALL ? 8 : kWarpsPerBlock) * 32)
k_num_warp(int32_t m, const int32_t* __restrict__ ap, const int32_t* __restrict__ ac,
           const double* __restrict__ av, const int32_t* __restrict__ bp,
           const int32_t* __restrict__ bc, const double* __restrict__ bv,
           const int32_t* __restrict__ count, const int32_t* __restrict__ mid, const int32_t* __restrict__ nmid,
           const int32_t* __restrict__ cp, int32_t* __restrict__ cc, double* __restrict__ cv,
           int* __restrict__ err) {
    constexpr int WARPS = SMALL ? 8 : kWarpsPerBlock;
    constexpr int SLOTS = SMALL ? kSmallSlots : kWarpSlots;
    constexpr int CAP = SMALL ? kSmallCap : kWarpCap;
    extern __shared__ unsigned char raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // rows of at most kSmallCap columns go to the small instance (over all
    // rows), rows of up to kWarpCap to the large one (over the list the
    // symbolic phase made), longer ones to the block kernels
    const int nrows = SMALL ? m : *nmid;
    for (int w = blockIdx.x * WARPS + warp; w < nrows; w += (SMALL ? nrows : gridDim.x * WARPS)) {
    const int row = SMALL ? w : mid[w];
    if (count[row] < 0 || count[row] > CAP) continue;
    double* vals = reinterpret_cast<double*>(raw) + warp * SLOTS;
    int* keys = reinterpret_cast<int*>(reinterpret_cast<double*>(raw) + WARPS * SLOTS) + warp * (SLOTS + CAP);
    int* lst = keys + SLOTS;  // compacted slot list, CAP entries
    // a table of twice the row's column count (at least 32 slots)
    int slots = 32;
    while (slots < SLOTS && slots < 2 * count[row]) slots <<= 1;
    const unsigned mask = (unsigned)slots - 1u;
    for (int i = lane; i < slots; i += 32) { keys[i] = kEmpty; vals[i] = 0.0; }
    __syncwarp();
    for (int ka = ap[row]; ka < ap[row + 1]; ++ka) {
        const int k = ac[ka];
        const double a = av[ka];
        const int b0 = bp[k], b1 = bp[k + 1];
        for (int kb = b0 + lane; kb < b1; kb += 32) {  // distinct columns: no two lanes share a slot
            bool added;
            const int sl = insert(keys, mask, bc[kb], added);
            if (sl < 0) atomicOr(err, 1);
            else vals[sl] = __dadd_rn(vals[sl], __dmul_rn(a, bv[kb]));
        }
        __syncwarp();  // orders the steps: each slot sees its products in ascending k
    }
    // compact occupied slots (in slot order), then rank-sort by column
    int base = 0;
    for (int i0 = 0; i0 < slots; i0 += 32) {
        const bool occ = keys[i0 + lane] != kEmpty;
        const unsigned msk = __ballot_sync(0xffffffffu, occ);
        const int pos = base + __popc(msk & ((1u << lane) - 1u));
        if (occ && pos < CAP) lst[pos] = i0 + lane;
        base += __popc(msk);
    }
    __syncwarp();
    const int n = base;
    const int out0 = cp[row];
    if (n != count[row] || n > CAP) {  // symbolic and numeric disagree: write nothing
        if (lane == 0) atomicOr(err, 1);
        continue;
    }
    for (int e = lane; e < n; e += 32) {
        const int key = keys[lst[e]];
        int rank = 0;
        for (int j = 0; j < n; ++j) rank += keys[lst[j]] < key;
        cc[out0 + rank] = key;
        cv[out0 + rank] = vals[lst[e]];
    }
    __syncwarp();
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
    if (cp[row + 1] - cp[row] > kBlockCap) return;  // a wide row: handled by k_num_wide
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

// Wide rows, numeric: the products of step k (one row of B, distinct
// columns) go straight to a dense accumulator of all ncols columns, steps
// ordered by a block barrier, so every entry sums its products in ascending
// k exactly as the hash kernels do.  The occupied columns are then written in
// ascending order (a scan over the bit set) and the accumulator and the bit
// set are cleared for the next row.
__global__ void __launch_bounds__(kBlockThreads)
k_num_wide(int32_t nwide, const int32_t* __restrict__ rows, const int32_t* __restrict__ ap,
           const int32_t* __restrict__ ac, const double* __restrict__ av,
           const int32_t* __restrict__ bp, const int32_t* __restrict__ bc,
           const double* __restrict__ bv, double* __restrict__ acc_scratch,
           unsigned* __restrict__ mark_scratch, int32_t ncols, int64_t words,
           const int32_t* __restrict__ cp, int32_t* __restrict__ cc, double* __restrict__ cv,
           int* __restrict__ err) {
    __shared__ int sh[kBlockThreads / 32];
    double* acc = acc_scratch + (int64_t)blockIdx.x * ncols;
    unsigned* mark = mark_scratch + (int64_t)blockIdx.x * words;
    for (int w = blockIdx.x; w < nwide; w += gridDim.x) {
        const int row = rows[w];
        for (int ka = ap[row]; ka < ap[row + 1]; ++ka) {
            const int k = ac[ka];
            const double a = av[ka];
            for (int kb = bp[k] + threadIdx.x; kb < bp[k + 1]; kb += kBlockThreads) {
                const int c = bc[kb];
                acc[c] = __dadd_rn(acc[c], __dmul_rn(a, bv[kb]));
                atomicOr(mark + (c >> 5), 1u << (c & 31));
            }
            __syncthreads();
        }
        const int out0 = cp[row], width = cp[row + 1] - cp[row];
        int written = 0;
        for (int64_t base = 0; base < words; base += kBlockThreads) {
            const int64_t i = base + threadIdx.x;
            const unsigned m = (i < words) ? mark[i] : 0u;
            int chunk = 0;
            int pos = written + block_excl_scan_int(__popc(m), sh, &chunk);
            for (unsigned bits = m; bits; bits &= bits - 1u) {
                const int c = (int)(i * 32) + __ffs(bits) - 1;
                if (pos < width) {
                    cc[out0 + pos] = c;
                    cv[out0 + pos] = acc[c];
                }
                acc[c] = 0.0;
                ++pos;
            }
            if (i < words) mark[i] = 0u;
            written += chunk;
        }
        if (threadIdx.x == 0 && written != width) atomicOr(err, 1);
        __syncthreads();
    }
}

}  // namespace

// Device temporaries of one product, stream-ordered on the product's stream
// and freed when it goes out of scope (also when an error is thrown); the
// output arrays are freed too unless kept.
struct SpgemmScratch {
    cudaStream_t s = nullptr;
    std::vector<void*> tmp;
    DevCsr* out = nullptr;
    bool keep = false;
    template <typename T>
    T* get(size_t n) {
        T* p = dev_alloc_async<T>(n, s);
        tmp.push_back(p);
        return p;
    }
    ~SpgemmScratch() {
        for (void* p : tmp) dev_free_async(p, s);
        if (out && !keep) {
            dev_free_async(out->ptr, s);
            dev_free_async(out->col, s);
            dev_free_async(out->val, s);
            out->ptr = nullptr;
            out->col = nullptr;
            out->val = nullptr;
        }
    }
};

void device_spgemm(const DevCsr& A, const DevCsr& B, DevCsr& C, cudaStream_t s) {
    const int32_t m = A.nrows;
    C.nrows = m;
    C.ncols = B.ncols;
    C.ptr = nullptr;
    C.col = nullptr;
    C.val = nullptr;
    SpgemmScratch S;
    S.s = s;
    S.out = &C;
    int32_t* count = S.get<int32_t>(m > 0 ? m : 1);
    int32_t* big = S.get<int32_t>(m > 0 ? m : 1);
    int32_t* nbig = S.get<int32_t>(4);  // [0]: rows for the block kernels, [1]: wide rows,
                                        // [2]: rows for the large symbolic, [3]: the large numeric warp kernel
    int32_t* wide = S.get<int32_t>(m > 0 ? m : 1);
    int32_t* lst = S.get<int32_t>(m > 0 ? m : 1);
    int32_t* mid = S.get<int32_t>(m > 0 ? m : 1);
    int* err = S.get<int>(1);
    AMG_CUDA(cudaMemsetAsync(nbig, 0, 4 * sizeof(int32_t), s));
    AMG_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    C.ptr = dev_alloc_async<int32_t>(m + 1 + kPad, s);
    AMG_CUDA(cudaMemsetAsync(C.ptr, 0, (m + 1 + kPad) * sizeof(int32_t), s));

    const unsigned sgrid = (unsigned)((m + 7) / 8);
    if (m > 0) {
        k_sym_warp<true><<<sgrid, 8 * 32, 0, s>>>(m, A.ptr, A.col, B.ptr, B.col, count, big, nbig, lst,
                                                   nbig + 2, mid, nbig + 3, err);
        AMG_CUDA(cudaGetLastError());
        int32_t hl = 0;  // rows for the large instance: a warp each
        AMG_CUDA(cudaMemcpyAsync(&hl, nbig + 2, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        AMG_CUDA(cudaStreamSynchronize(s));
        if (hl > 0)
            k_sym_warp<false><<<(unsigned)((hl + kWarpsPerBlock - 1) / kWarpsPerBlock), kWarpsPerBlock * 32, 0, s>>>(
                m, A.ptr, A.col, B.ptr, B.col, count, big, nbig, lst, nbig + 2, mid, nbig + 3, err);
        AMG_CUDA(cudaGetLastError());
    }
    int32_t hbig = 0;
    AMG_CUDA(cudaMemcpyAsync(&hbig, nbig, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    AMG_CUDA(cudaStreamSynchronize(s));
    const size_t sym_smem = kBlockSlots * sizeof(int);
    const size_t num_block_smem = kBlockSlots * (sizeof(double) + sizeof(int)) + kBlockCap * sizeof(int);
    const size_t num_warp_smem = kWarpsPerBlock * (kWarpSlots * (sizeof(double) + sizeof(int)) +
                                                   kWarpCap * sizeof(int));
    const size_t num_small_smem = 8 * (kSmallSlots * (sizeof(double) + sizeof(int)) + kSmallCap * sizeof(int));
    if (hbig > 0) {
        AMG_CUDA(cudaFuncSetAttribute(k_sym_block, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)sym_smem));
        k_sym_block<<<hbig, kBlockThreads, sym_smem, s>>>(big, A.ptr, A.col, B.ptr, B.col, count, wide,
                                                          nbig + 1);
        AMG_CUDA(cudaGetLastError());
    }
    // wide rows: a dense bit set (symbolic) and accumulator (numeric) per block
    int32_t hwide = 0;
    if (hbig > 0) {
        AMG_CUDA(cudaMemcpyAsync(&hwide, nbig + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        AMG_CUDA(cudaStreamSynchronize(s));
    }
    const int64_t words = ((int64_t)C.ncols + 31) / 32;
    int wgrid_wide = 0;
    if (hwide > 0) {
        int dev = 0, sms = 0;
        AMG_CUDA(cudaGetDevice(&dev));
        AMG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const int64_t per_block = (int64_t)C.ncols * 8 + words * 4;
        const int64_t cap = std::max<int64_t>(1, (int64_t(1) << 30) / per_block);  // <= 1 GiB of scratch
        wgrid_wide = (int)std::min<int64_t>(std::min<int64_t>(hwide, 2 * (int64_t)sms), cap);
        unsigned* mark = S.get<unsigned>((size_t)(wgrid_wide * words));
        AMG_CUDA(cudaMemsetAsync(mark, 0, (size_t)(wgrid_wide * words) * sizeof(unsigned), s));
        k_sym_wide<<<wgrid_wide, kBlockThreads, 0, s>>>(hwide, wide, A.ptr, A.col, B.ptr, B.col, mark, words,
                                                        count);
        AMG_CUDA(cudaGetLastError());
    }
    int herr = 0;
    AMG_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    AMG_CUDA(cudaStreamSynchronize(s));
    if (herr) fail(AMG_ERR_CUDA, "sparse product symbolic phase: hash table overflow");
    const int64_t nnz = dev_exclusive_scan(count, C.ptr, m, s);  // TOO_LARGE above 2^31 - 1
    C.nnz = nnz;
    C.col = dev_alloc_async<int32_t>(nnz + kPad, s);
    C.val = dev_alloc_async<double>(nnz + kPad, s);
    AMG_CUDA(cudaMemsetAsync(C.col, 0, (nnz + kPad) * sizeof(int32_t), s));
    AMG_CUDA(cudaMemsetAsync(C.val, 0, (nnz + kPad) * sizeof(double), s));
    if (m > 0) {
        AMG_CUDA(cudaFuncSetAttribute(k_num_warp<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)num_warp_smem));
        k_num_warp<true><<<sgrid, 8 * 32, num_small_smem, s>>>(
            m, A.ptr, A.col, A.val, B.ptr, B.col, B.val, count, mid, nbig + 3, C.ptr, C.col, C.val, err);
        int32_t hm = 0;
        AMG_CUDA(cudaMemcpyAsync(&hm, nbig + 3, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        AMG_CUDA(cudaStreamSynchronize(s));
        if (hm > 0)
            k_num_warp<false><<<(unsigned)((hm + kWarpsPerBlock - 1) / kWarpsPerBlock), kWarpsPerBlock * 32,
                                num_warp_smem, s>>>(m, A.ptr, A.col, A.val, B.ptr, B.col, B.val, count, mid, nbig + 3,
                                                    C.ptr, C.col, C.val, err);
        AMG_CUDA(cudaGetLastError());
    }
    if (hbig > 0) {
        AMG_CUDA(cudaFuncSetAttribute(k_num_block, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)num_block_smem));
        k_num_block<<<hbig, kBlockThreads, num_block_smem, s>>>(big, A.ptr, A.col, A.val, B.ptr,
                                                                B.col, B.val, C.ptr, C.col, C.val, err);
        AMG_CUDA(cudaGetLastError());
    }
    if (hwide > 0) {
        double* acc = S.get<double>((size_t)wgrid_wide * C.ncols);
        unsigned* mark = S.get<unsigned>((size_t)(wgrid_wide * words));
        AMG_CUDA(cudaMemsetAsync(acc, 0, (size_t)wgrid_wide * C.ncols * sizeof(double), s));
        AMG_CUDA(cudaMemsetAsync(mark, 0, (size_t)(wgrid_wide * words) * sizeof(unsigned), s));
        k_num_wide<<<wgrid_wide, kBlockThreads, 0, s>>>(hwide, wide, A.ptr, A.col, A.val, B.ptr, B.col, B.val,
                                                        acc, mark, (int32_t)C.ncols, words, C.ptr, C.col,
                                                        C.val, err);
        AMG_CUDA(cudaGetLastError());
    }
    AMG_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    AMG_CUDA(cudaStreamSynchronize(s));
    if (herr) fail(AMG_ERR_CUDA, "sparse product numeric phase inconsistent with its symbolic phase");
    S.keep = true;
}

}  // namespace amg
