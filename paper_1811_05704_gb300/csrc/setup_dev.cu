// setup_dev.cu -- the smoothed-aggregation set-up of one level on the GPU
// (Algorithm 1 up to the Galerkin product, which spgemm.cu provides).
//
// Every step computes exactly what the host set-up (setup_host.cpp) computes,
// bit for bit: the same strength decisions, the same aggregates with the same
// ids, the same prolongation values.  Floating-point steps use explicit
// round-to-nearest operations (__dmul_rn, __dadd_rn, ...) in the host's
// order, so that no multiply-add is contracted; sums that the host forms left
// to right are formed left to right by one thread.
//
// The ordered passes of the aggregation (pass 1 seeds an aggregate at node i
// only if its whole strong neighbourhood is still free when i's turn comes;
// pass 3 lets a free node seed an aggregate with its free neighbours, in row
// order) are the lexicographically first solutions of their rules.  They are
// computed here by dataflow over the nodes: warps take chunks of 32
// consecutive nodes from a counter in increasing order, and a node decides as
// soon as the nodes below it that it depends on have decided.  The lowest
// undecided node always belongs to a running warp and depends only on decided
// nodes, so the computation always progresses; every wait is still bounded
// in time and reported through an error flag.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "amg_internal.h"

namespace amg {

namespace {

constexpr int kT = 256;  // threads per block of the row kernels

// ------------------------------------------------------------ temporaries
// Stream-ordered device temporaries of one set-up step, freed on scope exit.
struct Tmp {
    cudaStream_t s;
    std::vector<void*> ptrs;
    explicit Tmp(cudaStream_t st) : s(st) {}
    template <typename T>
    T* get(size_t n) {
        T* p = dev_alloc_async<T>(n > 0 ? n : 1, s);
        ptrs.push_back(p);
        return p;
    }
    ~Tmp() {
        for (void* p : ptrs) dev_free_async(p, s);
    }
};

unsigned grid_for(int64_t n, int per = kT) {
    const int64_t g = (n + per - 1) / per;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, 1 << 20));
}

template <typename T>
T read1(const T* d, cudaStream_t s) {
    T v;
    AMG_CUDA(cudaMemcpyAsync(&v, d, sizeof(T), cudaMemcpyDeviceToHost, s));
    AMG_CUDA(cudaStreamSynchronize(s));
    return v;
}

// ------------------------------------------------------------------ scan
// Exclusive prefix sums of int32 counts into int32 offsets (n + 1 entries),
// in three steps: per-block totals, a scan of the totals by one block, then
// the per-block scans with their offsets.  *overflow (device) is set if the
// total does not fit below 2^31 - 1.
constexpr int kScanPer = 2048;  // elements per block (8 per thread)

__global__ void __launch_bounds__(kT) k_scan_totals(int64_t n, const int32_t* __restrict__ in,
                                                    long long* __restrict__ tot) {
    __shared__ long long sh[kT / 32];
    const int64_t b = (int64_t)blockIdx.x * kScanPer;
    long long s = 0;
    for (int64_t i = b + threadIdx.x; i < min(n, b + kScanPer); i += kT) s += in[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int w = 0; w < kT / 32; ++w) t += sh[w];
        tot[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(1024) k_scan_block_totals(int nb, long long* __restrict__ tot,
                                                            int* __restrict__ overflow) {
    __shared__ long long part[1024];
    const int t = threadIdx.x;
    const int chunk = (nb + 1023) / 1024;
    const int b = t * chunk, e = min(nb, b + chunk);
    long long s = 0;
    for (int i = b; i < e; ++i) s += tot[i];
    part[t] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const long long v = (t >= o) ? part[t - o] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    long long run = (t == 0) ? 0 : part[t - 1];
    for (int i = b; i < e; ++i) {
        const long long v = tot[i];
        tot[i] = run;
        run += v;
    }
    if (t == 1023) {
        tot[nb] = part[1023];
        if (part[1023] >= (1LL << 31) - 1) *overflow = 1;
    }
}

__global__ void __launch_bounds__(kT) k_scan_apply(int64_t n, const int32_t* __restrict__ in,
                                                   const long long* __restrict__ tot, int nb,
                                                   int32_t* __restrict__ out) {
    __shared__ long long sh[kT / 32];
    constexpr int per = kScanPer / kT;
    const int64_t b = (int64_t)blockIdx.x * kScanPer + (int64_t)threadIdx.x * per;
    long long v[per];
    long long s = 0;
#pragma unroll
    for (int u = 0; u < per; ++u) {
        v[u] = (b + u < n) ? in[b + u] : 0;
        s += v[u];
    }
    // exclusive prefix of the per-thread sums over the block
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long x = s;
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    long long before = 0;
    for (int w = 0; w < warp; ++w) before += sh[w];
    long long run = tot[blockIdx.x] + before + x - s;
#pragma unroll
    for (int u = 0; u < per; ++u) {
        if (b + u < n) out[b + u] = (int32_t)run;
        run += v[u];
    }
    if (blockIdx.x == nb - 1 && threadIdx.x == kT - 1) out[n] = (int32_t)tot[nb];
}

}  // namespace

// out[0..n] = exclusive prefix of in[0..n-1]; returns out[n] (the total).
int64_t dev_exclusive_scan(const int32_t* in, int32_t* out, int64_t n, cudaStream_t s) {
    Tmp t(s);
    const int nb = (int)std::max<int64_t>(1, (n + kScanPer - 1) / kScanPer);
    long long* tot = t.get<long long>(nb + 1);
    int* overflow = t.get<int>(1);
    AMG_CUDA(cudaMemsetAsync(overflow, 0, sizeof(int), s));
    k_scan_totals<<<nb, kT, 0, s>>>(n, in, tot);
    k_scan_block_totals<<<1, 1024, 0, s>>>(nb, tot, overflow);
    k_scan_apply<<<nb, kT, 0, s>>>(n, in, tot, nb, out);
    AMG_CUDA(cudaGetLastError());
    if (read1(overflow, s)) fail(AMG_ERR_TOO_LARGE, "set-up array (or Galerkin product) with more than 2^31 entries");
    return read1(out + n, s);
}

namespace {

// ------------------------------------------------------ segmented sorting
// Rows of a CSR-like array sorted by key, carrying a payload.  Rows of up to
// kShortSort entries are sorted by one thread (insertion sort); longer rows
// by a block with a bitonic sort of (key, payload) pairs packed in 64 bits,
// in shared memory up to kSmemSort entries and in a global scratch slice
// beyond.  Keys are non-negative int32 and distinct within a row.
constexpr int kShortSort = 32;
constexpr int kSmemSort = 4096;
constexpr int kSortThreads = 512;

__global__ void __launch_bounds__(kT) k_sort_short_rows(int64_t n, const int32_t* __restrict__ ptr,
                                                        int32_t* __restrict__ key, int32_t* __restrict__ pay,
                                                        int32_t* __restrict__ long_rows,
                                                        int32_t* __restrict__ nlong) {
    const int64_t r = (int64_t)blockIdx.x * kT + threadIdx.x;
    if (r >= n) return;
    const int b = ptr[r], e = ptr[r + 1];
    if (e - b > kShortSort) {
        long_rows[atomicAdd(nlong, 1)] = (int32_t)r;
        return;
    }
    for (int i = b + 1; i < e; ++i) {
        const int32_t k = key[i], p = pay[i];
        int j = i - 1;
        while (j >= b && key[j] > k) {
            key[j + 1] = key[j];
            pay[j + 1] = pay[j];
            --j;
        }
        key[j + 1] = k;
        pay[j + 1] = p;
    }
}

// bitonic sort of buf[0..m) (m a power of two) by the whole block
__device__ void block_bitonic(unsigned long long* buf, int m) {
    for (int k = 2; k <= m; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < m; i += blockDim.x) {
                const int p = i ^ j;
                if (p > i) {
                    const unsigned long long a = buf[i], c = buf[p];
                    const bool up = (i & k) == 0;
                    if ((a > c) == up) {
                        buf[i] = c;
                        buf[p] = a;
                    }
                }
            }
            __syncthreads();
        }
}

__global__ void __launch_bounds__(kSortThreads) k_sort_long_rows(const int32_t* __restrict__ rows, int nrows,
                                                                  const int32_t* __restrict__ ptr,
                                                                  int32_t* __restrict__ key, int32_t* __restrict__ pay,
                                                                  unsigned long long* __restrict__ scratch,
                                                                  int scratch_len) {
    extern __shared__ unsigned long long sbuf[];
    for (int w = blockIdx.x; w < nrows; w += gridDim.x) {
        const int r = rows[w];
        const int b = ptr[r], len = ptr[r + 1] - b;
        int m = 1;
        while (m < len) m <<= 1;
        unsigned long long* buf = (m <= kSmemSort) ? sbuf : scratch + (size_t)blockIdx.x * scratch_len;
        for (int i = threadIdx.x; i < m; i += blockDim.x)
            buf[i] = (i < len) ? ((unsigned long long)(uint32_t)key[b + i] << 32) | (uint32_t)pay[b + i]
                               : ~0ull;
        __syncthreads();
        block_bitonic(buf, m);
        for (int i = threadIdx.x; i < len; i += blockDim.x) {
            key[b + i] = (int32_t)(buf[i] >> 32);
            pay[b + i] = (int32_t)(buf[i] & 0xffffffffu);
        }
        __syncthreads();
    }
}

// Raises the long-row kernels' shared-memory limit (defined below them).
void allow_sort_smem();

void dev_sort_rows(int64_t n, const int32_t* ptr, int32_t* key, int32_t* pay, cudaStream_t s) {
    if (n == 0) return;
    Tmp t(s);
    int32_t* rows = t.get<int32_t>(n);
    int32_t* nlong = t.get<int32_t>(1);
    AMG_CUDA(cudaMemsetAsync(nlong, 0, sizeof(int32_t), s));
    k_sort_short_rows<<<grid_for(n), kT, 0, s>>>(n, ptr, key, pay, rows, nlong);
    AMG_CUDA(cudaGetLastError());
    const int hl = read1(nlong, s);
    if (hl == 0) return;
    // longest of the long rows, for the scratch of rows beyond shared memory
    std::vector<int32_t> lr(hl);
    AMG_CUDA(cudaMemcpyAsync(lr.data(), rows, hl * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    std::vector<int32_t> hp(n + 1);
    AMG_CUDA(cudaMemcpyAsync(hp.data(), ptr, (n + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    AMG_CUDA(cudaStreamSynchronize(s));
    int longest = 0;
    for (int32_t r : lr) longest = std::max(longest, hp[r + 1] - hp[r]);
    int m = 1;
    while (m < longest) m <<= 1;
    int dev = 0, sms = 0;
    AMG_CUDA(cudaGetDevice(&dev));
    AMG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int grid = std::min(hl, 2 * sms);
    unsigned long long* scratch = nullptr;
    int scratch_len = 0;
    if (m > kSmemSort) {
        scratch_len = m;
        scratch = t.get<unsigned long long>((size_t)grid * m);
    }
    const size_t smem = (size_t)std::min(m, kSmemSort) * sizeof(unsigned long long);
    allow_sort_smem();
    k_sort_long_rows<<<grid, kSortThreads, smem, s>>>(rows, hl, ptr, key, pay, scratch, scratch_len);
    AMG_CUDA(cudaGetLastError());
}

// --------------------------------------------------------- sorted transpose
// T = M^T for an n x ncols pattern (ptr, col) restricted to the entries with
// keep[k] != 0 (all if keep is null), with `with_diag` adding the entry (i, i)
// to every row i < min(n, ncols) first; rows of T sorted ascending.  perm[q]
// (optional) receives, for entry q of T, the index k of the entry of M it
// came from (-1 for an added diagonal).
__global__ void __launch_bounds__(kT) k_tr_count(int64_t n, int64_t ncols, const int32_t* __restrict__ ptr,
                                                 const int32_t* __restrict__ col, const uint8_t* __restrict__ keep,
                                                 int with_diag, int32_t* __restrict__ cnt) {
    const int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x;
    if (i >= n) return;
    if (with_diag && i < ncols) atomicAdd(cnt + i, 1);
    for (int k = ptr[i]; k < ptr[i + 1]; ++k)
        if (!keep || keep[k]) atomicAdd(cnt + col[k], 1);
}

__global__ void __launch_bounds__(kT) k_tr_fill(int64_t n, int64_t ncols, const int32_t* __restrict__ ptr,
                                                const int32_t* __restrict__ col, const uint8_t* __restrict__ keep,
                                                int with_diag, int32_t* __restrict__ cursor,
                                                int32_t* __restrict__ tcol, int32_t* __restrict__ perm) {
    const int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x;
    if (i >= n) return;
    if (with_diag && i < ncols) {
        const int q = atomicAdd(cursor + i, 1);
        tcol[q] = (int32_t)i;
        perm[q] = -1;
    }
    for (int k = ptr[i]; k < ptr[i + 1]; ++k)
        if (!keep || keep[k]) {
            const int q = atomicAdd(cursor + col[k], 1);
            tcol[q] = (int32_t)i;
            perm[q] = k;
        }
}

struct DevPattern {
    int32_t* ptr = nullptr;  // ncols + 1
    int32_t* col = nullptr;
    int32_t* perm = nullptr;
    int64_t nnz = 0;
};

// allocates T's arrays in `t` (freed with it) unless `keep_alloc` is given
void dev_transpose_pattern(int64_t n, int64_t ncols, const int32_t* ptr, const int32_t* col,
                           const uint8_t* keep, bool with_diag, int64_t max_nnz, DevPattern& T, Tmp& t,
                           cudaStream_t s) {
    Tmp w(s);
    int32_t* cnt = w.get<int32_t>(ncols);
    AMG_CUDA(cudaMemsetAsync(cnt, 0, ncols * sizeof(int32_t), s));
    T.ptr = t.get<int32_t>(ncols + 1 + kPad);
    AMG_CUDA(cudaMemsetAsync(T.ptr, 0, (ncols + 1 + kPad) * sizeof(int32_t), s));
    if (n > 0) k_tr_count<<<grid_for(n), kT, 0, s>>>(n, ncols, ptr, col, keep, with_diag ? 1 : 0, cnt);
    AMG_CUDA(cudaGetLastError());
    T.nnz = dev_exclusive_scan(cnt, T.ptr, ncols, s);
    if (T.nnz > max_nnz) fail(AMG_ERR_CUDA, "transposed pattern larger than its source");
    T.col = t.get<int32_t>(T.nnz + kPad);
    T.perm = t.get<int32_t>(T.nnz + kPad);
    AMG_CUDA(cudaMemcpyAsync(cnt, T.ptr, ncols * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    if (n > 0)
        k_tr_fill<<<grid_for(n), kT, 0, s>>>(n, ncols, ptr, col, keep, with_diag ? 1 : 0, cnt, T.col, T.perm);
    AMG_CUDA(cudaGetLastError());
    dev_sort_rows(ncols, T.ptr, T.col, T.perm, s);
}

// ------------------------------------------------------------- diagonal
// dg[i] = a_ii (binary search of the sorted row); the lowest row without a
// nonzero diagonal is recorded in *bad (initialised to n).
__global__ void __launch_bounds__(kT) k_diag(int64_t n, const int32_t* __restrict__ ptr,
                                             const int32_t* __restrict__ col, const double* __restrict__ val,
                                             double* __restrict__ dg, int* __restrict__ bad) {
    const int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x;
    if (i >= n) return;
    int lo = ptr[i], hi = ptr[i + 1];
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (col[mid] < i) lo = mid + 1;
        else hi = mid;
    }
    const double d = (lo < ptr[i + 1] && col[lo] == i) ? val[lo] : 0.0;
    dg[i] = d;
    if (d == 0.0) atomicMin(bad, (int)i);
}

// Smoother diagonal: damped Jacobi omega / a_ii, or SPAI-0 a_ii / sum_j a_ij^2
// (the squares summed in column order).
__global__ void __launch_bounds__(kT) k_smoother_diag(int64_t n, const int32_t* __restrict__ ptr,
                                                      const double* __restrict__ val, const double* __restrict__ dg,
                                                      int spai0, double omega, double* __restrict__ d) {
    const int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x;
    if (i >= n) return;
    if (spai0) {
        double s2 = 0.0;
        for (int k = ptr[i]; k < ptr[i + 1]; ++k) s2 = __dadd_rn(s2, __dmul_rn(val[k], val[k]));
        d[i] = __ddiv_rn(dg[i], s2);
    } else {
        d[i] = __ddiv_rn(omega, dg[i]);
    }
}

// vald[k] = a_ij d_j
__global__ void __launch_bounds__(kT) k_scale_cols(int64_t nnz, const int32_t* __restrict__ col,
                                                   const double* __restrict__ val, const double* __restrict__ d,
                                                   double* __restrict__ out) {
    const int64_t k = (int64_t)blockIdx.x * kT + threadIdx.x;
    if (k < nnz) out[k] = __dmul_rn(val[k], d[col[k]]);
}

// Strength of connection (Vanek, Mandel and Brezina 1996, cited in Sec. 3):
// j != i is strong for i iff a_ij^2 > eps^2 |a_ii a_jj|, from row i.  Also
// the number of strong entries of each row.
__global__ void __launch_bounds__(kT) k_strength(int64_t n, const int32_t* __restrict__ ptr,
                                                 const int32_t* __restrict__ col, const double* __restrict__ val,
                                                 const double* __restrict__ dg, double e2,
                                                 uint8_t* __restrict__ strong, int32_t* __restrict__ deg) {
    const int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x;
    if (i >= n) return;
    const double di = dg[i];
    int cnt = 0;
    for (int k = ptr[i]; k < ptr[i + 1]; ++k) {
        const int j = col[k];
        const double a = val[k];
        const bool st = (j != i) && (__dmul_rn(a, a) > __dmul_rn(e2, fabs(__dmul_rn(di, dg[j]))));
        strong[k] = st;
        cnt += st;
    }
    deg[i] = cnt;
}


// ------------------------------------------------------------ aggregation
constexpr int kUndecided = 0, kRoot = 1, kOut = 2;  // pass-1 / pass-3 node states
constexpr int kRes = 8;                              // pass 1: resources checked together
constexpr int kNotFree = 3;                          // pass 3: aggregated before pass 3

__device__ __forceinline__ int ld_relaxed(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(int* p, int v) {
    asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait budget of the dataflow passes: a node that waits longer than this for
// the nodes below it gives up, raises the abort flag (every other waiting
// node then gives up at once) and the host reports an error.
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s

// Pass 0 and eligibility for pass 1: a node without strong neighbours is a
// singleton aggregate; a node can seed in pass 1 only if it has strong
// neighbours and none of them is a singleton (which pass 0 aggregated).
__global__ void __launch_bounds__(kT) k_pass1_init(int64_t n, const int32_t* __restrict__ ptr,
                                                   const int32_t* __restrict__ col,
                                                   const uint8_t* __restrict__ strong,
                                                   const int32_t* __restrict__ deg, int* __restrict__ state,
                                                   int32_t* __restrict__ single) {
    const int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x;
    if (i >= n) return;
    bool elig = deg[i] > 0;
    for (int k = ptr[i]; k < ptr[i + 1] && elig; ++k)
        if (strong[k] && deg[col[k]] == 0) elig = false;
    state[i] = elig ? kUndecided : kOut;
    single[i] = deg[i] == 0;
}

// Pass 1: node i seeds an aggregate (state kRoot) iff no lower seed r claimed
// any node of i's closed strong neighbourhood {i} + N_i, i.e. iff for every
// j in {i} + N_i every candidate r < i of j (the nodes r with j in {r} + N_r:
// the sorted list tcol[tptr[j] ..]) did not seed.  cursor[j] counts the
// leading candidates of j known not to seed, so each list is walked once
// overall.  A candidate that seeded makes i kOut at once.
__global__ void __launch_bounds__(kT) k_pass1(int n, const int32_t* __restrict__ ptr,
                                              const int32_t* __restrict__ col, const uint8_t* __restrict__ strong,
                                              const int32_t* __restrict__ tptr, const int32_t* __restrict__ tcol,
                                              int* state, int* cursor, unsigned* next, int* abort_flag,
                                              int* err) {
    const int lane = threadIdx.x & 31;
    for (;;) {
        int base = 0;
        if (lane == 0) base = (int)atomicAdd(next, 32u);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= n) break;
        const int i = base + lane;
        if (i < n && ld_relaxed(state + i) == kUndecided) {
            const unsigned long long t0 = now_ns();
            const int kb = ptr[i], ke = ptr[i + 1];
            // resources before kpos are known to be clear for i (their
            // cursors reached i, and cannot pass it before i decides): a
            // retry starts at the first one that was not
            int kpos = kb - 1;
            for (unsigned spin = 0;; ++spin) {
                bool blocked = false, out = false;
                // resources in batches of kRes: their list heads, cursors,
                // candidates and states are loaded together (independent
                // loads), then each resource is resolved, walking further
                // only past candidates that did not seed
                for (int k0 = kpos; k0 < ke && !out; k0 += kRes) {
                    int jj[kRes], tb[kRes], len[kRes], c0[kRes], rr[kRes], st[kRes];
#pragma unroll
                    for (int u = 0; u < kRes; ++u) {
                        const int k = k0 + u;
                        jj[u] = (k < kb) ? i : (k < ke && strong[k]) ? col[k] : -1;
                    }
#pragma unroll
                    for (int u = 0; u < kRes; ++u) {
                        tb[u] = len[u] = c0[u] = 0;
                        if (jj[u] >= 0) {
                            tb[u] = tptr[jj[u]];
                            len[u] = tptr[jj[u] + 1] - tb[u];
                            c0[u] = ld_relaxed(cursor + jj[u]);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < kRes; ++u)
                        rr[u] = (jj[u] >= 0 && c0[u] < len[u]) ? tcol[tb[u] + c0[u]] : i;
#pragma unroll
                    for (int u = 0; u < kRes; ++u) st[u] = (rr[u] < i) ? ld_relaxed(state + rr[u]) : kUndecided;
                    for (int u = 0; u < kRes && !out; ++u) {
                        if (jj[u] < 0) continue;
                        int c = c0[u], r = rr[u], sr = st[u];
                        for (;;) {
                            if (c >= len[u]) {  // i is in every candidate list it walks: cannot happen
                                atomicOr(err, 1);
                                out = true;
                                break;
                            }
                            if (r >= i) break;
                            if (sr == kOut) {
                                ++c;
                                if (c < len[u]) {
                                    r = tcol[tb[u] + c];
                                    sr = (r < i) ? ld_relaxed(state + r) : kUndecided;
                                }
                                continue;
                            }
                            if (sr == kRoot) out = true;
                            else blocked = true;
                            break;
                        }
                        if (c > c0[u]) atomicMax(cursor + jj[u], c);
                        if (!blocked && !out) kpos = k0 + u + 1;
                    }
                }
                if (out) { st_relaxed(state + i, kOut); break; }
                if (!blocked) { st_relaxed(state + i, kRoot); break; }
                if (ld_relaxed(abort_flag)) break;
                if ((spin & 31) == 31 && now_ns() - t0 > kWaitNs) {
                    atomicExch(abort_flag, 1);
                    break;
                }
                __nanosleep(100);
            }
        }
        __syncwarp();
    }
}

// Aggregate ids after pass 1: singletons first (ids in row order), then the
// pass-1 seeds in row order; a seed's strong neighbours join it.
__global__ void __launch_bounds__(kT) k_pass1_assign(int64_t n, const int32_t* __restrict__ ptr,
                                                     const int32_t* __restrict__ col,
                                                     const uint8_t* __restrict__ strong,
                                                     const int* __restrict__ state,
                                                     const int32_t* __restrict__ single,
                                                     const int32_t* __restrict__ single_id,
                                                     const int32_t* __restrict__ root_id, int32_t nsingle,
                                                     int32_t* __restrict__ agg) {
    const int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x;
    if (i >= n) return;
    if (single[i]) agg[i] = single_id[i];
    if (state[i] == kRoot) {
        const int32_t id = nsingle + root_id[i];
        agg[i] = id;
        for (int k = ptr[i]; k < ptr[i + 1]; ++k)
            if (strong[k]) agg[col[k]] = id;
    }
}

__global__ void __launch_bounds__(kT) k_flag_eq(int64_t n, const int* __restrict__ state, int v,
                                                int32_t* __restrict__ flag) {
    const int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x;
    if (i < n) flag[i] = state[i] == v;
}

// Pass 2: a node left free by pass 1 joins the aggregate (as assigned after
// pass 1) of its strong neighbour with the largest |a_ij| / sqrt(|a_ii a_jj|),
// the first such neighbour in column order on ties.
__global__ void __launch_bounds__(kT) k_pass2(int64_t n, const int32_t* __restrict__ ptr,
                                              const int32_t* __restrict__ col, const double* __restrict__ val,
                                              const uint8_t* __restrict__ strong, const double* __restrict__ dg,
                                              const int32_t* __restrict__ after1, int32_t* __restrict__ agg,
                                              int* __restrict__ state3) {
    const int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x;
    if (i >= n) return;
    int32_t a = after1[i];
    if (a == -1) {
        double best = -1.0;
        const double di = dg[i];
        for (int k = ptr[i]; k < ptr[i + 1]; ++k) {
            if (!strong[k]) continue;
            const int j = col[k];
            const int32_t aj = after1[j];
            if (aj == -1) continue;
            const double c = __ddiv_rn(fabs(val[k]), __dsqrt_rn(fabs(__dmul_rn(di, dg[j]))));
            if (c > best) {
                best = c;
                a = aj;
            }
        }
    }
    agg[i] = a;
    state3[i] = (a == -1) ? kUndecided : kNotFree;
}

// Pass 3: in row order, a node still free seeds an aggregate with its free
// strong neighbours.  Node i seeds (kRoot) iff no lower seed r has i as a
// strong neighbour; otherwise it joins the lowest such seed (owner[i]).  The
// candidates r < i with i in N_r are read in ascending order from the sorted
// transposed list of node i (which also holds i itself).
__global__ void __launch_bounds__(kT) k_pass3(int n, const int32_t* __restrict__ tptr,
                                              const int32_t* __restrict__ tcol, int* state3,
                                              int32_t* __restrict__ owner, unsigned* next, int* abort_flag) {
    const int lane = threadIdx.x & 31;
    for (;;) {
        int base = 0;
        if (lane == 0) base = (int)atomicAdd(next, 32u);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= n) break;
        const int i = base + lane;
        if (i < n && ld_relaxed(state3 + i) == kUndecided) {
            const unsigned long long t0 = now_ns();
            int claim = -1;
            bool gave_up = false;
            for (int c = tptr[i]; c < tptr[i + 1] && claim < 0 && !gave_up; ++c) {
                const int r = tcol[c];
                if (r >= i) break;
                for (unsigned spin = 0;; ++spin) {
                    const int st = ld_relaxed(state3 + r);
                    if (st == kRoot) { claim = r; break; }
                    if (st != kUndecided) break;
                    if (ld_relaxed(abort_flag)) { gave_up = true; break; }
                    if ((spin & 31) == 31 && now_ns() - t0 > kWaitNs) {
                        atomicExch(abort_flag, 1);
                        gave_up = true;
                        break;
                    }
                    __nanosleep(100);
                }
            }
            if (!gave_up) {
                owner[i] = claim;
                st_relaxed(state3 + i, claim < 0 ? kRoot : kOut);
            }
        }
        __syncwarp();
    }
}

__global__ void __launch_bounds__(kT) k_pass3_assign(int64_t n, const int* __restrict__ state3,
                                                     const int32_t* __restrict__ owner,
                                                     const int32_t* __restrict__ root3_id, int32_t base,
                                                     int32_t* __restrict__ agg) {
    const int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x;
    if (i >= n) return;
    const int st = state3[i];
    if (st == kRoot) agg[i] = base + root3_id[i];
    else if (st == kOut) agg[i] = base + root3_id[owner[i]];
}


// ----------------------------------------------------------- prolongation
// Smoothed prolongation P = (I - omega D_F^{-1} A_F) P_t (setup_host.cpp
// states the reading): t_i = 1/sqrt(|agg(i)|); aF_ii = a_ii minus the weak
// entries of row i summed in column order; rho = max_i (row sum of |A_F| in
// column order) / |aF_ii|, omega = (4/3)/rho; P_ij = [j == agg(i)] t_i -
// (omega / aF_ii) s_ij, s_ij = sum over the kept entries k of row i in column
// order with agg(k) = j of aF_ik t_k.  Kept entries: the diagonal and the
// strong ones.
__global__ void __launch_bounds__(kT) k_agg_sizes(int64_t n, const int32_t* __restrict__ agg,
                                                  int32_t* __restrict__ size) {
    const int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x;
    if (i < n) atomicAdd(size + agg[i], 1);
}

__global__ void __launch_bounds__(kT) k_filtered(int64_t n, const int32_t* __restrict__ ptr,
                                                 const int32_t* __restrict__ col, const double* __restrict__ val,
                                                 const uint8_t* __restrict__ strong, const double* __restrict__ dg,
                                                 const int32_t* __restrict__ agg, const int32_t* __restrict__ size,
                                                 double* __restrict__ t, double* __restrict__ dF,
                                                 unsigned long long* __restrict__ rho_bits) {
    const int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x;
    // non-negative doubles order like their bit patterns: the maximum is taken
    // on those, per warp by shuffles, then one atomic per warp
    unsigned long long bits = 0ull;
    if (i < n) {
        t[i] = __ddiv_rn(1.0, __dsqrt_rn((double)size[agg[i]]));
        double weak = 0.0;
        for (int k = ptr[i]; k < ptr[i + 1]; ++k)
            if (col[k] != i && !strong[k]) weak = __dadd_rn(weak, val[k]);
        const double f = __dsub_rn(dg[i], weak);
        dF[i] = f;
        double row = 0.0;
        for (int k = ptr[i]; k < ptr[i + 1]; ++k) {
            if (col[k] == i) row = __dadd_rn(row, fabs(f));
            else if (strong[k]) row = __dadd_rn(row, fabs(val[k]));
        }
        bits = (unsigned long long)__double_as_longlong(__ddiv_rn(row, fabs(f)));
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long b = __shfl_xor_sync(0xffffffffu, bits, o);
        bits = b > bits ? b : bits;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(rho_bits, bits);
}

__global__ void k_omega(const unsigned long long* __restrict__ rho_bits, double* __restrict__ omega) {
    *omega = __ddiv_rn(4.0 / 3.0, __longlong_as_double((long long)*rho_bits));
}

// Short rows (at most kShortP nonzeros of A): one thread per row collects the
// coarse columns in first-seen order with their sums s_ij (each formed in
// column order), then sorts them by column.  FILL = false counts them only.
constexpr int kShortP = 96;

template <bool FILL>
__global__ void __launch_bounds__(kT) k_prolong_short(int64_t n, const int32_t* __restrict__ ptr,
                                                      const int32_t* __restrict__ col,
                                                      const double* __restrict__ val,
                                                      const uint8_t* __restrict__ strong,
                                                      const int32_t* __restrict__ agg, const double* __restrict__ t,
                                                      const double* __restrict__ dF,
                                                      const double* __restrict__ omega,
                                                      int32_t* __restrict__ count, const int32_t* __restrict__ pptr,
                                                      int32_t* __restrict__ pcol, double* __restrict__ pval,
                                                      int32_t* __restrict__ long_rows, int32_t* __restrict__ nlong) {
    const int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x;
    if (i >= n) return;
    const int b = ptr[i], e = ptr[i + 1];
    if (e - b > kShortP) {
        if (!FILL) long_rows[atomicAdd(nlong, 1)] = (int32_t)i;
        return;
    }
    int32_t cc[kShortP + 1];
    double ss[kShortP + 1];
    int m = 0;
    const int32_t own = agg[i];
    cc[m] = own;
    ss[m++] = 0.0;
    for (int k = b; k < e; ++k) {
        const int j = col[k];
        if (j != i && !strong[k]) continue;
        const int32_t c = agg[j];
        int q = 0;
        while (q < m && cc[q] != c) ++q;
        if (q == m) {
            cc[m] = c;
            ss[m++] = 0.0;
        }
        if (FILL) {
            const double a = (j == i) ? dF[i] : val[k];
            ss[q] = __dadd_rn(ss[q], __dmul_rn(a, t[j]));
        }
    }
    if constexpr (!FILL) {
        count[i] = m;
    } else {
        for (int x = 1; x < m; ++x) {  // insertion sort by column
            const int32_t c = cc[x];
            const double v = ss[x];
            int y = x - 1;
            while (y >= 0 && cc[y] > c) {
                cc[y + 1] = cc[y];
                ss[y + 1] = ss[y];
                --y;
            }
            cc[y + 1] = c;
            ss[y + 1] = v;
        }
        const double w = __ddiv_rn(*omega, dF[i]);
        const double ti = t[i];
        int o = pptr[i];
        for (int q = 0; q < m; ++q, ++o) {
            pcol[o] = cc[q];
            pval[o] = __dsub_rn(cc[q] == own ? ti : 0.0, __dmul_rn(w, ss[q]));
        }
    }
}

// Long rows: a block per row sorts the kept entries by (coarse column, column
// position) -- so each coarse column's terms stay in column order -- then a
// thread per distinct coarse column forms its sum.  Rows longer than
// kSmemSort sort in a global scratch slice of the block.
template <bool FILL>
__global__ void __launch_bounds__(kSortThreads) k_prolong_long(
    const int32_t* __restrict__ rows, int nrows, const int32_t* __restrict__ ptr,
    const int32_t* __restrict__ col, const double* __restrict__ val, const uint8_t* __restrict__ strong,
    const int32_t* __restrict__ agg, const double* __restrict__ t, const double* __restrict__ dF,
    const double* __restrict__ omega, int32_t* __restrict__ count, const int32_t* __restrict__ pptr,
    int32_t* __restrict__ pcol, double* __restrict__ pval, unsigned long long* __restrict__ scratch,
    int scratch_len) {
    extern __shared__ unsigned long long sbuf[];
    __shared__ int wsum[kSortThreads / 32];
    for (int w = blockIdx.x; w < nrows; w += gridDim.x) {
        const int i = rows[w];
        const int b = ptr[i], len = ptr[i + 1] - b;
        int m = 1;
        while (m < len) m <<= 1;
        unsigned long long* buf = (m <= kSmemSort) ? sbuf : scratch + (size_t)blockIdx.x * scratch_len;
        for (int q = threadIdx.x; q < m; q += blockDim.x) {
            unsigned long long key = ~0ull;
            if (q < len) {
                const int j = col[b + q];
                if (j == i || strong[b + q]) key = ((unsigned long long)(uint32_t)agg[j] << 32) | (uint32_t)q;
            }
            buf[q] = key;
        }
        __syncthreads();
        block_bitonic(buf, m);
        // distinct coarse columns: the first entry of each run of equal keys
        // (high halves); kept entries come first, dropped ones sort last
        int before = 0;  // runs that start in earlier chunks of the block
        for (int q0 = 0; q0 < m; q0 += blockDim.x) {
            const int q = q0 + threadIdx.x;
            const unsigned long long kq = (q < m) ? buf[q] : ~0ull;
            const bool start = kq != ~0ull && (q == 0 || (buf[q - 1] >> 32) != (kq >> 32));
            // block-wide exclusive count of starts
            const unsigned bal = __ballot_sync(0xffffffffu, start);
            const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
            if (lane == 0) wsum[warp] = __popc(bal);
            __syncthreads();
            int off = before;
            int chunk_total = 0;
            for (int x = 0; x < (int)(blockDim.x >> 5); ++x) {
                if (x < warp) off += wsum[x];
                chunk_total += wsum[x];
            }
            off += __popc(bal & ((1u << lane) - 1u));
            if (FILL && start) {
                const int32_t c = (int32_t)(kq >> 32);
                double sum = 0.0;
                for (int z = q; z < m && (buf[z] >> 32) == (kq >> 32); ++z) {
                    const int k = b + (int)(buf[z] & 0xffffffffu);
                    const int j = col[k];
                    const double a = (j == i) ? dF[i] : val[k];
                    sum = __dadd_rn(sum, __dmul_rn(a, t[j]));
                }
                const double wgt = __ddiv_rn(*omega, dF[i]);
                const int o = pptr[i] + off;
                pcol[o] = c;
                pval[o] = __dsub_rn(c == agg[i] ? t[i] : 0.0, __dmul_rn(wgt, sum));
            }
            before += chunk_total;
            __syncthreads();
        }
        if (!FILL && threadIdx.x == 0) count[i] = before;
        __syncthreads();
    }
}

// The long-row kernels' shared-memory limit is raised once, to the largest
// size any launch asks for: set-ups on several host threads at once (the
// server) must not change a kernel's attribute between another thread's
// setting and its launch.
void allow_sort_smem() {
    static const bool done = [] {
        const int bytes = kSmemSort * (int)sizeof(unsigned long long);
        AMG_CUDA(cudaFuncSetAttribute(k_sort_long_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
        AMG_CUDA(cudaFuncSetAttribute(k_prolong_long<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
        AMG_CUDA(cudaFuncSetAttribute(k_prolong_long<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
        return true;
    }();
    (void)done;
}

__global__ void __launch_bounds__(kT) k_gather_vals(int64_t nnz, const int32_t* __restrict__ perm,
                                                    const double* __restrict__ src, double* __restrict__ dst) {
    const int64_t q = (int64_t)blockIdx.x * kT + threadIdx.x;
    if (q < nnz) dst[q] = src[perm[q]];
}


// ---------------------------------------------- fused restriction operator
// M = R - (R A) D on the pattern of R A (which contains R's: A has its
// diagonal): row c of M merges row c of R into row c of R A.
__global__ void __launch_bounds__(kT) k_fused_restriction(int64_t m, const int32_t* __restrict__ rptr,
                                                          const int32_t* __restrict__ rcol,
                                                          const double* __restrict__ rval,
                                                          const int32_t* __restrict__ mptr,
                                                          const int32_t* __restrict__ mcol,
                                                          double* __restrict__ mval, const double* __restrict__ d,
                                                          int* __restrict__ err) {
    const int64_t c = (int64_t)blockIdx.x * kT + threadIdx.x;
    if (c >= m) return;
    int q = rptr[c];
    const int qe = rptr[c + 1];
    for (int k = mptr[c]; k < mptr[c + 1]; ++k) {
        const int j = mcol[k];
        double r = 0.0;
        if (q < qe && rcol[q] == j) r = rval[q++];
        mval[k] = __dsub_rn(r, __dmul_rn(mval[k], d[j]));
    }
    if (q != qe) atomicOr(err, 1);  // an entry of R outside the pattern of R A: cannot happen
}

}  // namespace

// ============================================================ entry points
void dev_diagonal(const DevCsr& A, double* dg, cudaStream_t s) {
    Tmp t(s);
    int* bad = t.get<int>(1);
    const int n = A.nrows;
    AMG_CUDA(cudaMemcpyAsync(bad, &n, sizeof(int), cudaMemcpyHostToDevice, s));
    k_diag<<<grid_for(n), kT, 0, s>>>(n, A.ptr, A.col, A.val, dg, bad);
    AMG_CUDA(cudaGetLastError());
    const int b = read1(bad, s);
    if (b < n) fail(AMG_ERR_INVALID_ARG, "zero or missing diagonal in row " + std::to_string(b));
}

void dev_smoother_diag(const DevCsr& A, const double* dg, const amg_params& prm, double* d, cudaStream_t s) {
    k_smoother_diag<<<grid_for(A.nrows), kT, 0, s>>>(A.nrows, A.ptr, A.val, dg,
                                                     prm.smoother == AMG_SMOOTHER_SPAI0 ? 1 : 0, prm.jacobi_omega, d);
    AMG_CUDA(cudaGetLastError());
}

void dev_scale_columns(const DevCsr& A, const double* d, double* out, cudaStream_t s) {
    if (A.nnz > 0) k_scale_cols<<<grid_for(A.nnz), kT, 0, s>>>(A.nnz, A.col, A.val, d, out);
    AMG_CUDA(cudaGetLastError());
}

namespace {

// Blocks for the dataflow passes: enough warps to keep many chunks of nodes
// in flight; the passes do not need their blocks to be resident together.
unsigned dataflow_grid() {
    int dev = 0, sms = 0;
    AMG_CUDA(cudaGetDevice(&dev));
    AMG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    return (unsigned)(4 * sms);
}

}  // namespace

int64_t dev_aggregate(const DevCsr& A, const double* dg, double eps, int32_t* agg, uint8_t* strong,
                      cudaStream_t s) {
    const int64_t n = A.nrows;
    Tmp t(s);
    int32_t* deg = t.get<int32_t>(n);
    k_strength<<<grid_for(n), kT, 0, s>>>(n, A.ptr, A.col, A.val, dg, eps * eps, strong, deg);
    AMG_CUDA(cudaGetLastError());
    // candidate lists: node j's list holds j and every r with j strong for r
    DevPattern T;
    dev_transpose_pattern(n, n, A.ptr, A.col, strong, true, A.nnz + n, T, t, s);
    int* state = t.get<int>(n);
    int32_t* single = t.get<int32_t>(n);
    int32_t* single_id = t.get<int32_t>(n + 1);
    int32_t* flag = t.get<int32_t>(n);
    int32_t* root_id = t.get<int32_t>(n + 1);
    int* cursor = t.get<int>(n);
    unsigned* next = t.get<unsigned>(2);
    int* abort_flag = t.get<int>(2);
    int* err = abort_flag + 1;
    AMG_CUDA(cudaMemsetAsync(cursor, 0, n * sizeof(int), s));
    AMG_CUDA(cudaMemsetAsync(next, 0, 2 * sizeof(unsigned), s));
    AMG_CUDA(cudaMemsetAsync(abort_flag, 0, 2 * sizeof(int), s));
    k_pass1_init<<<grid_for(n), kT, 0, s>>>(n, A.ptr, A.col, strong, deg, state, single);
    const int64_t nsingle = dev_exclusive_scan(single, single_id, n, s);
    k_pass1<<<dataflow_grid(), kT, 0, s>>>((int)n, A.ptr, A.col, strong, T.ptr, T.col, state, cursor, next,
                                            abort_flag, err);
    AMG_CUDA(cudaGetLastError());
    {
        int h[2];
        AMG_CUDA(cudaMemcpyAsync(h, abort_flag, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
        AMG_CUDA(cudaStreamSynchronize(s));
        if (h[0] || h[1]) fail(AMG_ERR_CUDA, "device aggregation (pass 1) did not complete");
    }
    k_flag_eq<<<grid_for(n), kT, 0, s>>>(n, state, kRoot, flag);
    const int64_t n1 = dev_exclusive_scan(flag, root_id, n, s);
    int32_t* after1 = t.get<int32_t>(n);
    AMG_CUDA(cudaMemsetAsync(after1, 0xff, n * sizeof(int32_t), s));  // -1
    k_pass1_assign<<<grid_for(n), kT, 0, s>>>(n, A.ptr, A.col, strong, state, single, single_id, root_id,
                                              (int32_t)nsingle, after1);
    // pass 2 writes agg and the pass-3 states
    k_pass2<<<grid_for(n), kT, 0, s>>>(n, A.ptr, A.col, A.val, strong, dg, after1, agg, state);
    k_pass3<<<dataflow_grid(), kT, 0, s>>>((int)n, T.ptr, T.col, state, flag /* owner */, next + 1,
                                            abort_flag);
    AMG_CUDA(cudaGetLastError());
    if (read1(abort_flag, s)) fail(AMG_ERR_CUDA, "device aggregation (pass 3) did not complete");
    int32_t* owner = flag;
    int32_t* flag3 = single;  // no longer needed
    k_flag_eq<<<grid_for(n), kT, 0, s>>>(n, state, kRoot, flag3);
    int32_t* root3_id = root_id;
    const int64_t n3 = dev_exclusive_scan(flag3, root3_id, n, s);
    k_pass3_assign<<<grid_for(n), kT, 0, s>>>(n, state, owner, root3_id, (int32_t)(nsingle + n1), agg);
    AMG_CUDA(cudaGetLastError());
    return nsingle + n1 + n3;
}

// Allocates P's arrays (stream-ordered, kPad padding, zero-filled).
void dev_prolongation(const DevCsr& A, const double* dg, const uint8_t* strong, const int32_t* agg,
                      int64_t nagg, DevCsr& P, double& omega, cudaStream_t s) {
    const int64_t n = A.nrows;
    Tmp t(s);
    int32_t* size = t.get<int32_t>(nagg);
    AMG_CUDA(cudaMemsetAsync(size, 0, nagg * sizeof(int32_t), s));
    k_agg_sizes<<<grid_for(n), kT, 0, s>>>(n, agg, size);
    double* tv = t.get<double>(n);
    double* dF = t.get<double>(n);
    unsigned long long* rho = t.get<unsigned long long>(1);
    double* om = t.get<double>(1);
    AMG_CUDA(cudaMemsetAsync(rho, 0, sizeof(unsigned long long), s));
    k_filtered<<<grid_for(n), kT, 0, s>>>(n, A.ptr, A.col, A.val, strong, dg, agg, size, tv, dF, rho);
    k_omega<<<1, 1, 0, s>>>(rho, om);
    AMG_CUDA(cudaGetLastError());
    int32_t* count = t.get<int32_t>(n);
    int32_t* long_rows = t.get<int32_t>(n);
    int32_t* nlong = t.get<int32_t>(1);
    AMG_CUDA(cudaMemsetAsync(nlong, 0, sizeof(int32_t), s));
    k_prolong_short<false><<<grid_for(n), kT, 0, s>>>(n, A.ptr, A.col, A.val, strong, agg, tv, dF, om, count,
                                                      nullptr, nullptr, nullptr, long_rows, nlong);
    AMG_CUDA(cudaGetLastError());
    const int hl = read1(nlong, s);
    // the long rows' kernel: shared-memory sort up to kSmemSort entries
    int m = 1, grid = 0;
    unsigned long long* scratch = nullptr;
    size_t smem = 0;
    if (hl > 0) {
        std::vector<int32_t> hp(n + 1);
        std::vector<int32_t> lr(hl);
        AMG_CUDA(cudaMemcpyAsync(hp.data(), A.ptr, (n + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        AMG_CUDA(cudaMemcpyAsync(lr.data(), long_rows, hl * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        AMG_CUDA(cudaStreamSynchronize(s));
        int longest = 0;
        for (int32_t r : lr) longest = std::max(longest, hp[r + 1] - hp[r]);
        while (m < longest) m <<= 1;
        int dev = 0, sms = 0;
        AMG_CUDA(cudaGetDevice(&dev));
        AMG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        grid = std::min(hl, 2 * sms);
        if (m > kSmemSort) scratch = t.get<unsigned long long>((size_t)grid * m);
        smem = (size_t)std::min(m, kSmemSort) * sizeof(unsigned long long);
        allow_sort_smem();
        k_prolong_long<false><<<grid, kSortThreads, smem, s>>>(long_rows, hl, A.ptr, A.col, A.val, strong, agg, tv,
                                                               dF, om, count, nullptr, nullptr, nullptr, scratch,
                                                               m > kSmemSort ? m : 0);
        AMG_CUDA(cudaGetLastError());
    }
    P.nrows = (int32_t)n;
    P.ncols = (int32_t)nagg;
    P.ptr = dev_alloc_async<int32_t>(n + 1 + kPad, s);
    AMG_CUDA(cudaMemsetAsync(P.ptr, 0, (n + 1 + kPad) * sizeof(int32_t), s));
    P.nnz = dev_exclusive_scan(count, P.ptr, n, s);
    P.col = dev_alloc_async<int32_t>(P.nnz + kPad, s);
    P.val = dev_alloc_async<double>(P.nnz + kPad, s);
    AMG_CUDA(cudaMemsetAsync(P.col, 0, (P.nnz + kPad) * sizeof(int32_t), s));
    AMG_CUDA(cudaMemsetAsync(P.val, 0, (P.nnz + kPad) * sizeof(double), s));
    k_prolong_short<true><<<grid_for(n), kT, 0, s>>>(n, A.ptr, A.col, A.val, strong, agg, tv, dF, om, nullptr,
                                                     P.ptr, P.col, P.val, nullptr, nullptr);
    if (hl > 0)
        k_prolong_long<true><<<grid, kSortThreads, smem, s>>>(long_rows, hl, A.ptr, A.col, A.val, strong, agg, tv,
                                                              dF, om, nullptr, P.ptr, P.col, P.val, scratch,
                                                              m > kSmemSort ? m : 0);
    AMG_CUDA(cudaGetLastError());
    omega = read1(om, s);
}

// R = P^T with columns ascending (Sec. 2).  Allocates R's arrays.
void dev_transpose(const DevCsr& P, DevCsr& R, cudaStream_t s) {
    Tmp t(s);
    DevPattern T;
    dev_transpose_pattern(P.nrows, P.ncols, P.ptr, P.col, nullptr, false, P.nnz, T, t, s);
    R.nrows = P.ncols;
    R.ncols = P.nrows;
    R.nnz = T.nnz;
    R.ptr = dev_alloc_async<int32_t>(R.nrows + 1 + kPad, s);
    R.col = dev_alloc_async<int32_t>(R.nnz + kPad, s);
    R.val = dev_alloc_async<double>(R.nnz + kPad, s);
    AMG_CUDA(cudaMemsetAsync(R.col + R.nnz, 0, kPad * sizeof(int32_t), s));
    AMG_CUDA(cudaMemsetAsync(R.val + R.nnz, 0, kPad * sizeof(double), s));
    AMG_CUDA(cudaMemcpyAsync(R.ptr, T.ptr, (R.nrows + 1 + kPad) * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    AMG_CUDA(cudaMemcpyAsync(R.col, T.col, R.nnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    if (R.nnz > 0) k_gather_vals<<<grid_for(R.nnz), kT, 0, s>>>(R.nnz, T.perm, P.val, R.val);
    AMG_CUDA(cudaGetLastError());
    AMG_CUDA(cudaStreamSynchronize(s));
}

void dev_fused_restriction(const DevCsr& R, const double* d, DevCsr& M, cudaStream_t s) {
    Tmp t(s);
    int* err = t.get<int>(1);
    AMG_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    k_fused_restriction<<<grid_for(M.nrows), kT, 0, s>>>(M.nrows, R.ptr, R.col, R.val, M.ptr, M.col, M.val, d, err);
    AMG_CUDA(cudaGetLastError());
    if (read1(err, s)) fail(AMG_ERR_CUDA, "fused restriction: R outside the pattern of R A");
}

}  // namespace amg
