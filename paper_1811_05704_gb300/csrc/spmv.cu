// spmv.cu -- the solve-phase kernels.
//
// One CSR SpMV engine serves every step of the V-cycle (Algorithm 2) and the
// Krylov products: a block takes a run of rows (a precomputed row block, or
// a uniform split), streams their values and column indices through shared
// memory in tiles of kTileNnz products with fully coalesced, evict-first
// loads, gathers x through L2, and reduces each row in column order -- one
// thread per row for short rows, one warp per row for long ones.  What
// differs between the steps is only the gathered operand and the epilogue
// ("Epi" functors below), so the smoother, the residual and the dot products
// are fused into the product instead of costing extra passes over HBM:
//   presmooth+residual   x = d f,  t = f - A x       (Alg. 2 pre-relaxation, residual)
//   restrict             f_c = R t                    (Alg. 2 restriction)
//   prolong+correct      x += P x_c                   (Alg. 2 interpolation)
//   postsmooth           y = x + d (f - A x) [, w.y]  (Alg. 2 post-relaxation)
//   residual             r = f - A x, r.r, f.f
//   spmv+dot             q = A p, p.q                 (Krylov product)
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <atomic>

#include <algorithm>
#include <type_traits>

#include "amg_internal.h"
#include "device_common.cuh"
#include "epilogues.cuh"

namespace amg {

// ---------------------------------------------------- streaming engine
// Persistent, warp-specialised CSR kernel.  The matrix is split into tiles
// (consecutive rows, at most kTileNnz nonzeros and kRowsPerBlock rows); CTA b
// owns a contiguous run of tiles.  One producer lane streams each tile's row
// pointers, column indices and values into a shared-memory ring of stages
// with bulk asynchronous copies (cp.async.bulk, completion counted on an
// mbarrier, evict-first in L2 so that the gathered vectors stay resident);
// eight consumer warps take `vw` lanes per row, gather the operand through
// L2, reduce the row with shuffles and run the epilogue.  With programmatic
// dependent launch the producer fetches its first tiles -- constant matrix
// data -- before waiting for the previous kernel, so consecutive kernels of
// the solve overlap their pipeline fill with the predecessor's tail.
constexpr int kCons = kConsumers;

// Ring depth and resident CTAs per SM.  Every kernel keeps a ring of 2
// stages.  A float64 stage is about 34 KB, and three CTAs fit an SM; the
// float32 and bfloat16 stages (at most about 24 KB) fit four CTAs (their
// registers then fit 56 per thread).  More CTAs hide more of the gather
// latency than a deeper ring: measured on the 150^3 V-cycles, four float32
// CTAs of 2 stages beat three of 3, and three float64 CTAs of 2 stages beat
// two of 3 (FP64 solve 8.92 -> 8.72 ms; 200^3 variable coefficients 626 ->
// 588 ms).  Long-row tiles (RMAX = 128, chosen at set-up for large matrices
// with long rows, such as the fused restriction operators) hold
// kLongTileNnz nonzeros, about 50 KB a stage in float64, so two such CTAs
// fit an SM; they leave room for fewer lanes per row (fewer shuffle steps on
// the float64 pipe).
template <int RMAX>
__host__ __device__ constexpr int tile_nnz() { return RMAX == 128 ? kLongTileNnz : kTileNnz; }
template <typename VT, int RMAX>
__host__ __device__ constexpr int stages() { return 2; }
template <typename VT>
__host__ __device__ constexpr int stream_ctas() { return sizeof(VT) >= 8 ? 3 : kStreamCtasMax; }

__device__ int g_dev_err;  // bit 2: a pipeline wait gave up (see mbar_wait)

// Nonzero spans are copied from a start rounded down, and to an end rounded
// up, to a multiple of nz_align elements, so that both the column indices and
// the values start and end on 16-byte boundaries.
template <typename VT>
__host__ __device__ constexpr int nz_align() { return sizeof(VT) >= 4 ? 4 : 16 / (int)sizeof(VT); }

// Bytes per element of an epilogue's row-indexed vector k in shared memory:
// the epilogue's vslot(k) if it declares one (it must be at least vbytes(k)
// for every instance), else 8.
template <typename Epi, typename = void>
struct VecSlots {
    __host__ __device__ static constexpr int at(int) { return 8; }
};
template <typename Epi>
struct VecSlots<Epi, std::void_t<decltype(Epi::vslot(0))>> {
    __host__ __device__ static constexpr int at(int k) { return Epi::vslot(k); }
};

template <typename VT, int RMAX, typename Epi>
struct StreamLayout {
    static constexpr int NV = Epi::nvec;
    static constexpr int rp_n = RMAX + 8;       // row pointers of the tile (+ alignment slack)
    static constexpr int nz_n = tile_nnz<RMAX>() + 2 * nz_align<VT>();  // nonzeros of the tile (+ alignment slack)
    static constexpr int vec_n = RMAX + 8;      // rows of a row-indexed vector slice (+ alignment slack)
    static constexpr size_t rp_bytes = (size_t)rp_n * 4;
    static constexpr size_t col_bytes = (size_t)nz_n * 4;
    static constexpr size_t val_bytes = (size_t)nz_n * sizeof(VT);
    __host__ __device__ static constexpr size_t vec_bytes(int k) {
        return ((size_t)vec_n * VecSlots<Epi>::at(k) + 15) / 16 * 16;
    }
    __host__ __device__ static constexpr size_t vec_off(int k) {
        size_t o = 0;
        for (int j = 0; j < k; ++j) o += vec_bytes(j);
        return o;
    }
    static constexpr size_t stage = rp_bytes + col_bytes + val_bytes + vec_off(NV);
    static constexpr size_t header = 128;
    static constexpr size_t total = header + stages<VT, RMAX>() * stage;
    static_assert(rp_bytes % 16 == 0 && col_bytes % 16 == 0 && val_bytes % 16 == 0 && stage % 16 == 0,
                  "bulk-copy destinations must stay 16-byte aligned");
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity), "r"(100000u)  // suspend up to 100 us per poll
        : "memory");
    return ok != 0;
}
// Bounded wait: each poll suspends for at most 100 us, and after kPolls polls
// (2^15 in the kernels: at most about 3.3 s) the wait gives up, records bit 2
// in g_dev_err and returns false instead of spinning forever.
template <uint32_t kPolls>
__device__ __forceinline__ bool mbar_wait_n(uint64_t* b, uint32_t parity) {
    for (uint32_t i = 0; i < kPolls; ++i)
        if (mbar_try(b, parity)) return true;
    atomicOr(&g_dev_err, 4);
    return false;
}
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity) { return mbar_wait_n<1u << 15>(b, parity); }
__device__ __forceinline__ uint64_t evict_first_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
// bulk global -> shared copy; dst, src 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                         uint64_t pol) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1], %2, [%3], %4;" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
        : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

constexpr int kGatherBatch = 4;

// sum -/+ the products of nonzeros k, k + vw, ... < ke, in that order; the
// columns, values and gathered operands of kGatherBatch nonzeros at a time
// are loaded before any is accumulated.
template <int SIGN, typename acc_t, typename VT, typename Epi>
__device__ __forceinline__ acc_t row_batched(acc_t sum, int k, int ke, int vw, const VT* vs, const int* cs,
                                             const Epi& epi) {
    for (; k < ke; k += kGatherBatch * vw) {
        int c[kGatherBatch];
        acc_t a[kGatherBatch], x[kGatherBatch];
#pragma unroll
        for (int u = 0; u < kGatherBatch; ++u) {
            const bool in = k + u * vw < ke;
            c[u] = in ? cs[k + u * vw] : 0;
            a[u] = in ? (acc_t)vs[k + u * vw] : acc_t(0);
        }
#pragma unroll
        for (int u = 0; u < kGatherBatch; ++u) x[u] = (k + u * vw < ke) ? epi.xg(c[u]) : acc_t(0);
#pragma unroll
        for (int u = 0; u < kGatherBatch; ++u) {
            if (k + u * vw < ke) {
                if constexpr (SIGN < 0) sum -= a[u] * x[u];
                else sum += a[u] * x[u];
            }
        }
    }
    return sum;
}

template <typename VT, typename Epi, int RMAX>
__global__ void __launch_bounds__(kCons + 32, stream_ctas<VT>())
k_stream(const int32_t* __restrict__ ptr, const int32_t* __restrict__ col,
         const VT* __restrict__ val, const int2* __restrict__ tiles, int ntiles, int vw, Epi epi,
         Reduce red, const int* __restrict__ skip) {
    using acc_t = typename Epi::acc_t;
    constexpr int NV = Epi::nvec;
    using L = StreamLayout<VT, RMAX, Epi>;
    constexpr int kStages = stages<VT, RMAX>();  // at most 3: the 128-byte header holds their barriers
    extern __shared__ __align__(128) unsigned char sm[];
    uint64_t* full = reinterpret_cast<uint64_t*>(sm);
    uint64_t* empty = full + kStages;
    int4* info = reinterpret_cast<int4*>(sm + 64);
    auto stage_of = [&](int s) { return sm + L::header + s * L::stage; };
    auto rp_of = [&](int s) { return reinterpret_cast<int*>(stage_of(s)); };
    auto col_of = [&](int s) { return reinterpret_cast<int*>(stage_of(s) + L::rp_bytes); };
    auto val_of = [&](int s) { return reinterpret_cast<VT*>(stage_of(s) + L::rp_bytes + L::col_bytes); };
    auto vec_of = [&](int s, int k) {
        return stage_of(s) + L::rp_bytes + L::col_bytes + L::val_bytes + L::vec_off(k);
    };

    const int tid = threadIdx.x;
    const int t0 = (int)((long long)ntiles * blockIdx.x / gridDim.x);
    const int t1 = (int)((long long)ntiles * (blockIdx.x + 1) / gridDim.x);
    const int count = t1 - t0;
    const int first = min(kStages, count);
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kCons / 32);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    pdl_trigger();

    double d0 = 0.0, d1 = 0.0;
    bool stop = false;  // set by an earlier kernel; the same value in every block of the grid
    if (tid >= kCons) {
        if (tid != kCons) {
            pdl_wait();
            stop = skip && *(volatile const int*)skip;
        } else {  // producer lane
            const uint64_t pol = evict_first_policy();
            int2 cur = tiles[t0], nxt = tiles[t0 + 1];
            // matrix arrays stream once (evict first); the row-indexed vectors
            // are copied with the default policy
            auto issue = [&](int i) {
                const int s = i % kStages;
                const int ar = cur.x & ~3, re = (nxt.x + 1 + 3) & ~3, vre = (nxt.x + 3) & ~3;
                constexpr int na = nz_align<VT>();
                const int ak = cur.y & ~(na - 1), ke = (nxt.y + na - 1) & ~(na - 1);
                info[s] = make_int4(cur.x, nxt.x, ar, ak);
                const uint32_t brp = (uint32_t)(re - ar) * 4u;
                const uint32_t bnz = (uint32_t)(ke - ak);
                uint32_t bytes = brp + bnz * (4u + (uint32_t)sizeof(VT));
                for (int k = 0; k < NV; ++k) bytes += (uint32_t)(vre - ar) * (uint32_t)epi.vbytes(k);
                mbar_arrive_tx(&full[s], bytes);
                bulk_g2s(rp_of(s), ptr + ar, brp, &full[s], pol);
                if (bnz) {
                    bulk_g2s(col_of(s), col + ak, bnz * 4u, &full[s], pol);
                    bulk_g2s(val_of(s), val + ak, bnz * (uint32_t)sizeof(VT), &full[s], pol);
                }
                for (int k = 0; k < NV; ++k) {
                        const uint32_t vb = (uint32_t)epi.vbytes(k);
                        bulk_g2s(vec_of(s, k), static_cast<const unsigned char*>(epi.vptr(k)) + (size_t)ar * vb,
                                 (uint32_t)(vre - ar) * vb, &full[s]);
                    }
                cur = nxt;
                if (i + 2 <= count) nxt = tiles[t0 + i + 2];
            };
            // Without row-indexed vectors a tile depends only on the constant
            // matrix: fetch the first tiles before waiting for the preceding
            // kernel.  With vectors (written by earlier kernels) wait first.
            int issued = 0;
            if (NV == 0) {
                for (; issued < first; ++issued) issue(issued);
            }
            pdl_wait();
            stop = skip && *(volatile const int*)skip;
            if (!stop)
                for (int i = issued; i < count; ++i) {
                    if (i >= kStages && !mbar_wait(&empty[i % kStages], ((i / kStages) - 1) & 1)) break;
                    issue(i);
                }
        }
    } else {
        pdl_wait();
        stop = skip && *(volatile const int*)skip;
        const int n = stop ? (NV == 0 ? first : 0) : count;  // tiles the producer issues
        const int grp = tid / vw, lane = tid - grp * vw;
        const int ngroups = kCons / vw;
        for (int i = 0; i < n; ++i) {
            const int s = i % kStages;
            if (!mbar_wait(&full[s], (i / kStages) & 1)) break;
            if (!stop) {
                const int4 inf = info[s];
                const int* rp = rp_of(s);
                const int* cs = col_of(s);
                const VT* vs = val_of(s);
                VecTile vt;
#pragma unroll
                for (int k = 0; k < 4; ++k) vt.base[k] = (k < NV) ? vec_of(s, k) : nullptr;
                vt.row0 = inf.z;
                const int nrows = inf.y - inf.x;
                if (nrows > ngroups) {
                    // two consumer passes in this tile (short rows): take the
                    // rows of both passes together, so that each lane has the
                    // gathers of two rows in flight at once
                    for (int rb = 0; rb < nrows; rb += 2 * ngroups) {  // same trip count in every lane
                        const int rowA = inf.x + rb + grp, rowB = rowA + ngroups;
                        const bool actA = rb + grp < nrows, actB = rb + ngroups + grp < nrows;
                        typename Epi::Pre preA{}, preB{};
                        acc_t sumA = acc_t(0), sumB = acc_t(0);
                        if (lane == 0) {
                            if (actA) preA = epi.load(rowA, vt);
                            if (actB) preB = epi.load(rowB, vt);
                            if constexpr (Seeding<Epi>::sign != 0) {
                                if (actA) sumA = epi.seed(preA);
                                if (actB) sumB = epi.seed(preB);
                            }
                        }
                        int kA = 0, keA = 0, kB = 0, keB = 0;
                        if (actA) { kA = rp[rowA - inf.z] - inf.w + lane; keA = rp[rowA + 1 - inf.z] - inf.w; }
                        if (actB) { kB = rp[rowB - inf.z] - inf.w + lane; keB = rp[rowB + 1 - inf.z] - inf.w; }
#pragma unroll 2
                        for (;;) {
                            const bool a = kA < keA, b = kB < keB;
                            if (!a && !b) break;
                            if constexpr (Seeding<Epi>::sign < 0) {
                                if (a) sumA -= (acc_t)vs[kA] * epi.xg(cs[kA]);
                                if (b) sumB -= (acc_t)vs[kB] * epi.xg(cs[kB]);
                            } else {
                                if (a) sumA += (acc_t)vs[kA] * epi.xg(cs[kA]);
                                if (b) sumB += (acc_t)vs[kB] * epi.xg(cs[kB]);
                            }
                            kA += vw;
                            kB += vw;
                        }
                        for (int o = vw >> 1; o > 0; o >>= 1) {
                            sumA += __shfl_xor_sync(0xffffffffu, sumA, o, vw);
                            sumB += __shfl_xor_sync(0xffffffffu, sumB, o, vw);
                        }
                        if (lane == 0) {
                            if (actA) epi.store(rowA, sumA, preA, d0, d1);
                            if (actB) epi.store(rowB, sumB, preB, d0, d1);
                        }
                    }
                } else
                for (int rb = 0; rb < nrows; rb += ngroups) {  // same trip count in every lane
                    const int row = inf.x + rb + grp;
                    const bool active = rb + grp < nrows;
                    typename Epi::Pre pre{};
                    acc_t sum = acc_t(0);
                    if (active && lane == 0) {
                        pre = epi.load(row, vt);
                        if constexpr (Seeding<Epi>::sign != 0) sum = epi.seed(pre);
                    }
                    if (active) {
                        const int kb = rp[row - inf.z] - inf.w, ke = rp[row + 1 - inf.z] - inf.w;
                        if constexpr (!std::is_same<acc_t, double>::value) {
                            // float32 kernels are bound by gather latency, not
                            // by a pipe: a lane loads the columns and values
                            // of up to kGatherBatch of its nonzeros, issues
                            // their gathers together, then accumulates them
                            // in order (the same order as one at a time)
                            sum = row_batched<Seeding<Epi>::sign>(sum, kb + lane, ke, vw, vs, cs, epi);
                        } else if constexpr (Seeding<Epi>::sign < 0) {
#pragma unroll 4
                            for (int k = kb + lane; k < ke; k += vw) sum -= (acc_t)vs[k] * epi.xg(cs[k]);
                        } else {
#pragma unroll 4
                            for (int k = kb + lane; k < ke; k += vw) sum += (acc_t)vs[k] * epi.xg(cs[k]);
                        }
                    }
                    for (int o = vw >> 1; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o, vw);
                    if (active && lane == 0) epi.store(row, sum, pre, d0, d1);
                }
            }
            __syncwarp();
            if ((tid & 31) == 0) mbar_arrive(&empty[s]);
        }
    }
    if constexpr (Epi::ndot > 0) {
        if (!stop) {  // a skipped kernel contributes no dot products
            __syncthreads();  // every tile consumed: the ring is free for the block sums
            reduce_finalize_sh<Epi::ndot>(red, d0, d1, reinterpret_cast<double*>(sm + L::header));
        }
    }
}

// ------------------------------------------------------ row-chunk engine
// Fallback for matrices with a row longer than one tile, and the
// bounds-checked standalone product: a block takes a run of rows, stages the
// products of kTileNnz nonzeros at a time in shared memory and reduces each
// row in column order (a thread per row, or a warp per row for long rows).
template <typename VT>
__device__ __forceinline__ VT ld_stream(const VT* p) { return __ldcs(p); }

template <typename VT, typename Epi, bool CHECK>
__global__ void __launch_bounds__(kThreads)
k_spmv(const int32_t* __restrict__ ptr, const int32_t* __restrict__ col,
       const VT* __restrict__ val, const int32_t* __restrict__ blk, int32_t nrows,
       int32_t ncols, int rpb, Epi epi, Reduce red, const int* __restrict__ skip,
       int* __restrict__ err) {
    using acc_t = typename Epi::acc_t;
    if (skip && *skip) return;
    __shared__ acc_t prod[kTileNnz];
    __shared__ acc_t rowsum[kRowsPerBlock];
    __shared__ int rp[kRowsPerBlock + 1];

    const int tid = threadIdx.x;
    int r0, r1;
    if (blk) {
        r0 = blk[blockIdx.x];
        r1 = blk[blockIdx.x + 1];
    } else {
        r0 = blockIdx.x * rpb;
        r1 = min(r0 + rpb, nrows);
    }
    const int nr = r1 - r0;
    for (int i = tid; i <= nr; i += kThreads) rp[i] = ptr[r0 + i];
    if (tid < kRowsPerBlock) rowsum[tid] = acc_t(0);
    __syncthreads();
    const int k0 = rp[0], k1 = rp[nr];
    const bool warp_rows = (k1 - k0) >= 24 * nr;  // long rows: a warp per row
    typename Epi::Pre pre{};
    VecTile vt;
#pragma unroll
    for (int k = 0; k < 4; ++k)
        vt.base[k] = (k < Epi::nvec) ? static_cast<const unsigned char*>(epi.vptr(k)) : nullptr;
    vt.row0 = 0;
    if (tid < nr) pre = epi.load(r0 + tid, vt);

    acc_t acc = acc_t(0);
    for (int c0 = k0; c0 < k1; c0 += kTileNnz) {
        const int c1 = min(c0 + kTileNnz, k1);
        for (int base = c0 + tid; base < c1; base += 4 * kThreads) {
            int cc[4];
            VT vv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int k = base + u * kThreads;
                if (k < c1) {
                    cc[u] = ld_stream(col + k);
                    vv[u] = ld_stream(val + k);
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int k = base + u * kThreads;
                if (k < c1) {
                    int c = cc[u];
                    if (CHECK && (unsigned)c >= (unsigned)ncols) {
                        atomicOr(err, 2);
                        c = 0;
                        vv[u] = VT(0);
                    }
                    prod[k - c0] = (acc_t)vv[u] * epi.xg(c);
                }
            }
        }
        __syncthreads();
        if (!warp_rows) {
            if (tid < nr) {
                const int a = max(rp[tid], c0), b = min(rp[tid + 1], c1);
                for (int k = a; k < b; ++k) acc += prod[k - c0];
            }
        } else {
            const int lane = tid & 31, warp = tid >> 5;
            for (int rr = warp; rr < nr; rr += kThreads / 32) {
                const int a = max(rp[rr], c0), b = min(rp[rr + 1], c1);
                acc_t v = acc_t(0);
                for (int k = a + lane; k < b; k += 32) v += prod[k - c0];
                v = warp_sum(v);
                if (lane == 0) rowsum[rr] += v;
            }
        }
        __syncthreads();
    }
    if (warp_rows) acc = (tid < nr) ? rowsum[tid] : acc_t(0);

    double d0 = 0.0, d1 = 0.0;
    if (tid < nr) {
        // this engine sums the row first; a seeded epilogue gets seed -/+ sum
        if constexpr (Seeding<Epi>::sign < 0) acc = epi.seed(pre) - acc;
        if constexpr (Seeding<Epi>::sign > 0) acc = epi.seed(pre) + acc;
        epi.store(r0 + tid, acc, pre, d0, d1);
    }
    if constexpr (Epi::ndot > 0) reduce_finalize<Epi::ndot>(red, d0, d1);
}

// ------------------------------------------------------- long-row engine
// Matrices with a row longer than a streaming tile (the dense coarse levels
// that aggregation leaves on problems with strongly varying coefficients:
// hundreds to thousands of nonzeros a row).  A group of vw lanes (a warp, or
// half of one) takes a row; its lanes stride through the row's nonzeros with
// coalesced, evict-first column and value loads, keep kRowBatch gathers in
// flight each, accumulate with fused multiply-adds (one float64 operation a
// nonzero, against a product and an add in the row-chunk engine) and reduce
// with shuffles; the group's first lane runs the epilogue.  Groups take rows
// round-robin, so a long row holds up only its own group (no tile barrier
// couples it to other rows).  Rows of more than brow_min nonzeros (a few
// nearly dense rows on the smallest levels; brow_min is set per matrix at
// set-up) would leave one group far behind the rest; the whole block takes
// those first, from a list made at set-up.
constexpr int kRowBatch = 8;

// sum -/+ the products of nonzeros k, k + step, ... < ke, kRowBatch at a time
template <int SIGN, typename acc_t, typename VT, typename Epi>
__device__ __forceinline__ acc_t row_partial(acc_t sum, int k, int ke, int step, const int32_t* __restrict__ col,
                                             const VT* __restrict__ val, const Epi& epi) {
    for (; k + (kRowBatch - 1) * step < ke; k += kRowBatch * step) {
        int c[kRowBatch];
        acc_t a[kRowBatch], x[kRowBatch];
#pragma unroll
        for (int u = 0; u < kRowBatch; ++u) {
            c[u] = ld_stream(col + k + u * step);
            a[u] = (acc_t)ld_stream(val + k + u * step);
        }
#pragma unroll
        for (int u = 0; u < kRowBatch; ++u) x[u] = epi.xg(c[u]);
#pragma unroll
        for (int u = 0; u < kRowBatch; ++u) {
            if constexpr (SIGN < 0) sum -= a[u] * x[u];
            else sum += a[u] * x[u];
        }
    }
    for (; k < ke; k += step) {
        const acc_t a = (acc_t)ld_stream(val + k);
        if constexpr (SIGN < 0) sum -= a * epi.xg(ld_stream(col + k));
        else sum += a * epi.xg(ld_stream(col + k));
    }
    return sum;
}

template <typename VT, typename Epi>
__global__ void __launch_bounds__(kThreads)
k_rows(const int32_t* __restrict__ ptr, const int32_t* __restrict__ col, const VT* __restrict__ val,
       int32_t nrows, int vw, const int32_t* __restrict__ brows, int32_t nbrows, int32_t brow_min, Epi epi,
       Reduce red,
       const int* __restrict__ skip) {
    using acc_t = typename Epi::acc_t;
    constexpr int SIGN = Seeding<Epi>::sign;
    __shared__ acc_t part[kThreads / 32];
    if (skip && *(volatile const int*)skip) return;
    VecTile vt;
#pragma unroll
    for (int k = 0; k < 4; ++k)
        vt.base[k] = (k < Epi::nvec) ? static_cast<const unsigned char*>(epi.vptr(k)) : nullptr;
    vt.row0 = 0;
    double d0 = 0.0, d1 = 0.0;
    // the longest rows, a block each
    for (int i = blockIdx.x; i < nbrows; i += gridDim.x) {
        const int row = __ldg(brows + i);
        typename Epi::Pre pre{};
        acc_t sum = acc_t(0);
        if (threadIdx.x == 0) {
            pre = epi.load(row, vt);
            if constexpr (SIGN != 0) sum = epi.seed(pre);
        }
        sum = row_partial<SIGN>(sum, __ldg(ptr + row) + (int)threadIdx.x, __ldg(ptr + row + 1), kThreads, col,
                                val, epi);
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = sum;
        __syncthreads();
        if (threadIdx.x == 0) {
            acc_t t = part[0];
            for (int w = 1; w < kThreads / 32; ++w) t += part[w];
            epi.store(row, t, pre, d0, d1);
        }
        __syncthreads();
    }
    // the other rows, a group of vw lanes each; every lane of a warp runs the
    // same number of iterations (the shuffles need the whole warp): rows past
    // the end, and rows of the list above, are inactive
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & (vw - 1);
    const int group = tid / vw, ngroups = (gridDim.x * blockDim.x) / vw;
    const int rounds = (nrows + ngroups - 1) / ngroups;
    for (int it = 0; it < rounds; ++it) {
        const int row = group + it * ngroups;
        int kb = 0, ke = 0;
        bool active = false;
        if (row < nrows) {
            kb = __ldg(ptr + row);
            ke = __ldg(ptr + row + 1);
            active = ke - kb <= brow_min;
            if (!active) kb = ke = 0;
        }
        typename Epi::Pre pre{};
        acc_t sum = acc_t(0);
        if (active && lane == 0) {
            pre = epi.load(row, vt);
            if constexpr (SIGN != 0) sum = epi.seed(pre);
        }
        sum = row_partial<SIGN>(sum, kb + lane, ke, vw, col, val, epi);
        for (int o = vw >> 1; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o, vw);
        if (active && lane == 0) epi.store(row, sum, pre, d0, d1);
    }
    if constexpr (Epi::ndot > 0) reduce_finalize<Epi::ndot>(red, d0, d1);
}

static std::atomic<int> g_sm_count{0};
// set by the thread that issues the launches (several host threads may each
// drive a solve on their own stream)
static thread_local bool g_pdl = true;

void set_stream_options(bool pdl) { g_pdl = pdl; }

int stream_grid(int ntiles, int ctas_per_sm) {
    int sms = g_sm_count.load();
    if (sms == 0) {
        int dev = 0;
        AMG_CUDA(cudaGetDevice(&dev));
        AMG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        g_sm_count.store(sms);
    }
    return std::max(1, std::min(ntiles, ctas_per_sm * sms));
}

// Check of the bounded wait: one block waits on a pipeline barrier that no
// copy or thread ever completes, with the streaming kernels' wait limited to
// 2^12 polls (at most about 0.4 s).  Every thread gives up, bit 2 of the
// device error word is set, and the kernel returns.
__global__ void k_wait_unfilled() {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    mbar_wait_n<1u << 12>(&bar, 0);
}

int check_wait_limit(double* seconds) {
    read_and_clear_dev_err();  // start from a clear error word
    cudaEvent_t e0, e1;
    AMG_CUDA(cudaEventCreate(&e0));
    AMG_CUDA(cudaEventCreate(&e1));
    AMG_CUDA(cudaEventRecord(e0, 0));
    k_wait_unfilled<<<1, 32>>>();
    AMG_CUDA(cudaGetLastError());
    AMG_CUDA(cudaEventRecord(e1, 0));
    AMG_CUDA(cudaEventSynchronize(e1));
    float ms = 0.0f;
    AMG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    AMG_CUDA(cudaEventDestroy(e0));
    AMG_CUDA(cudaEventDestroy(e1));
    if (seconds) *seconds = ms * 1e-3;
    return read_and_clear_dev_err();
}

int* dev_err_ptr() {
    void* p = nullptr;
    AMG_CUDA(cudaGetSymbolAddress(&p, g_dev_err));
    return static_cast<int*>(p);
}

void enqueue_dev_err_copy(int* host_dst, cudaStream_t s) {
    AMG_CUDA(cudaMemcpyFromSymbolAsync(host_dst, g_dev_err, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
}

int read_and_clear_dev_err() {
    int v = 0, z = 0;
    AMG_CUDA(cudaMemcpyFromSymbol(&v, g_dev_err, sizeof(int)));
    if (v) AMG_CUDA(cudaMemcpyToSymbol(g_dev_err, &z, sizeof(int)));
    return v;
}

template <typename VT, typename Epi, int RMAX>
static void launch_stream(const DevCsr& A, const VT* val, const Epi& epi, const Reduce& red,
                          const int* skip, cudaStream_t s) {
    const size_t smem = StreamLayout<VT, RMAX, Epi>::total;
    // once per template instance (thread-safe static initialisation): the
    // shared-memory limit, and the CTAs per SM the grid is sized for -- the
    // resident count the device reports, at most stream_ctas<VT>(), so that
    // the persistent grid is one wave.  Kernels that can hold more than two
    // CTAs per SM ask for the largest shared-memory carveout; the float64
    // kernels keep the default, whose larger L1 serves their gathers.
    static const int ctas = [smem] {
        AMG_CUDA(cudaFuncSetAttribute(k_stream<VT, Epi, RMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
        if (stream_ctas<VT>() > 2)
            AMG_CUDA(cudaFuncSetAttribute(k_stream<VT, Epi, RMAX>,
                                          cudaFuncAttributePreferredSharedMemoryCarveout, 100));
        int per_sm = 0;
        AMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_stream<VT, Epi, RMAX>, kCons + 32,
                                                               smem));
        return std::max(1, std::min(per_sm, stream_ctas<VT>()));
    }();
    const int grid = stream_grid(A.ntiles, ctas);
    if (Epi::ndot > 0 && grid > red.stride) fail(AMG_ERR_TOO_LARGE, "reduction buffer smaller than the grid");
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kCons + 32);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    // Products of small matrices (the coarse levels: L2-resident, bound by
    // launch and dependency latency) always overlap their start with the
    // predecessor's tail; the others only with use_pdl.  Measured on 150^3
    // Poisson, FP64: 8.384 -> 8.363 ms with it below 2^21 nonzeros, 8.368 ms
    // below 2^23, slower for every kernel (8.72 against 8.62 ms).
    cfg.numAttrs = (g_pdl || A.nnz < kPdlAlwaysNnz) ? 1 : 0;
    AMG_CUDA(cudaLaunchKernelEx(&cfg, k_stream<VT, Epi, RMAX>, (const int32_t*)A.ptr, (const int32_t*)A.col,
                                val, (const int2*)A.tiles, (int)A.ntiles, (int)A.vw, epi, red, skip));
}

template <typename VT, typename Epi>
static void launch_rows(const DevCsr& A, const VT* val, const Epi& epi, const Reduce& red,
                        const int* skip, cudaStream_t s) {
    static const int per_sm = [] {
        int b = 0;
        AMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_rows<VT, Epi>, kThreads, 0));
        return std::max(1, b);
    }();
    const int vw = A.rows_vw, per_block = kThreads / vw;
    int grid = stream_grid((int)std::min<int64_t>(((int64_t)A.nrows + per_block - 1) / per_block, 1 << 30), per_sm);
    if (Epi::ndot > 0) grid = std::min(grid, red.stride);
    // launched in plain stream order, without programmatic dependent launch:
    // with it (the kernel triggering its dependents at the start, like the
    // streaming engine) the 200^3 variable-coefficient FP64 solve took 748
    // instead of 506 ms
    k_rows<VT, Epi><<<grid, kThreads, 0, s>>>(A.ptr, A.col, val, (int32_t)A.nrows, vw, A.brows, A.nbrows,
                                              A.brow_min, epi, red, skip);
    AMG_CUDA(cudaGetLastError());
}

template <typename VT, typename Epi>
static void run(const DevCsr& A, const VT* val, const Epi& epi, const Reduce& red,
                const int* skip, cudaStream_t s) {
    if (A.nrows == 0) return;
    if (A.tiles) {
        if (A.nz_cap == kLongTileNnz) launch_stream<VT, Epi, 128>(A, val, epi, red, skip, s);
        else if (A.rows_cap <= 256) launch_stream<VT, Epi, 256>(A, val, epi, red, skip, s);
        else launch_stream<VT, Epi, 512>(A, val, epi, red, skip, s);
        return;
    }
    // the long-row engine for float64 values only: the float kernels are
    // not bound by a pipe, and there the row-chunk engine measured faster
    // (200^3 variable coefficients, FP32 V-cycle 273 against 303 ms)
    if (A.rows_vw && sizeof(VT) >= 8) {
        launch_rows(A, val, epi, red, skip, s);
        return;
    }
    if (Epi::ndot > 0 && A.nblk > red.stride) fail(AMG_ERR_TOO_LARGE, "reduction buffer smaller than the grid");
    k_spmv<VT, Epi, false><<<A.nblk, kThreads, 0, s>>>(A.ptr, A.col, val, A.blk, A.nrows, A.ncols,
                                                        0, epi, red, skip, nullptr);
    AMG_CUDA(cudaGetLastError());
}

void launch_spmv(const DevCsr& A, const double* x, double* y, const int* skip, cudaStream_t s) {
    run(A, A.val, EpiY{x, y}, Reduce{}, skip, s);
}

void launch_spmv_dot(const DevCsr& A, const double* x, const double* w, double* y,
                     const Reduce& r, const int* skip, cudaStream_t s) {
    run(A, A.val, EpiYDot{x, w ? w : x, y}, r, skip, s);
}

void launch_residual_plain(const DevCsr& A, const double* f, const double* x, double* t,
                           const int* skip, cudaStream_t s) {
    run(A, A.val, EpiRes0{f, x, t}, Reduce{}, skip, s);
}

void launch_spmv_dot2(const DevCsr& A, const double* x, const double* w, double* y,
                      const Reduce& r, const int* skip, cudaStream_t s) {
    run(A, A.val, EpiYDot2{x, w, y}, r, skip, s);
}

void launch_presmooth_residual(const DevCsr& A, const double* d, const double* f, double* x,
                               double* t, const int* skip, cudaStream_t s) {
    run(A, A.vald, EpiPre{d, f, x, t}, Reduce{}, skip, s);
}

void launch_smooth(const DevCsr& A, const double* d, const double* f, const double* x, double* y,
                   const double* w, const Reduce* r, const int* skip, cudaStream_t s) {
    if (r && w == f) run(A, A.val, EpiSmoothDotF{d, f, x, y}, *r, skip, s);
    else if (r) run(A, A.val, EpiSmooth<true>{d, f, x, y, w}, *r, skip, s);
    else run(A, A.val, EpiSmooth<false>{d, f, x, y, nullptr}, Reduce{}, skip, s);
}

void launch_residual(const DevCsr& A, const double* f, const double* x, double* r, double* r2,
                     const Reduce& red, const int* skip, cudaStream_t s, float* r32) {
    if (r32) run(A, A.val, EpiResid<true>{f, x, r, r2, r32}, red, skip, s);
    else run(A, A.val, EpiResid<false>{f, x, r, r2, nullptr}, red, skip, s);
}

void launch_prolong_add(const DevCsr& P, const double* xc, double* x, const int* skip,
                        cudaStream_t s) {
    run(P, P.val, EpiProlong{xc, x}, Reduce{}, skip, s);
}
void launch_prolong_pre(const DevCsr& P, const double* d, const double* f, const double* xc, double* x,
                        const int* skip, cudaStream_t s) {
    run(P, P.val, EpiProlongPre{d, f, xc, x}, Reduce{}, skip, s);
}

static const __nv_bfloat16* bf16_of(const uint16_t* p) { return reinterpret_cast<const __nv_bfloat16*>(p); }

// The float32 V-cycle kernels read bfloat16-stored values when the matrix has
// them (AMG_PRECISION_BF16), else float32 values.
template <typename Epi>
static void run32(const DevCsr& A, const float* v32, const uint16_t* v16, const Epi& epi, const Reduce& red,
                  const int* skip, cudaStream_t s) {
    if (v16) run(A, bf16_of(v16), epi, red, skip, s);
    else run(A, v32, epi, red, skip, s);
}

void launch_spmv_f32(const DevCsr& A, const float* x, float* y, const int* skip, cudaStream_t s) {
    run32(A, A.val32, A.val16, EpiY32{x, y}, Reduce{}, skip, s);
}

void launch_presmooth_residual_f32(const DevCsr& A, const float* d, const float* f32,
                                   const double* f64, float* x, float* t, const int* skip,
                                   cudaStream_t s) {
    if (f64) run32(A, A.vald32, A.vald16, EpiPre32<true>{d, nullptr, f64, x, t}, Reduce{}, skip, s);
    else run32(A, A.vald32, A.vald16, EpiPre32<false>{d, f32, nullptr, x, t}, Reduce{}, skip, s);
}

template <bool DOT>
static void smooth_f32(const DevCsr& A, const EpiSmooth32<DOT, false, false>& e, const Reduce& r,
                       const int* skip, cudaStream_t s) {
    // the float64 input and output, where given, select the instantiation
    if (e.f64 && e.y64)
        run32(A, A.val32, A.val16, EpiSmooth32<DOT, true, true>{e.d, nullptr, e.f64, e.x, nullptr, e.y64, e.w}, r,
              skip, s);
    else if (e.f64)
        run32(A, A.val32, A.val16, EpiSmooth32<DOT, true, false>{e.d, nullptr, e.f64, e.x, e.y32, nullptr, e.w}, r,
              skip, s);
    else if (e.y64)
        run32(A, A.val32, A.val16, EpiSmooth32<DOT, false, true>{e.d, e.f32, nullptr, e.x, nullptr, e.y64, e.w}, r,
              skip, s);
    else
        run32(A, A.val32, A.val16, e, r, skip, s);
}

void launch_smooth_f32(const DevCsr& A, const float* d, const float* f32, const double* f64,
                       const float* x, float* y32, double* y64, const double* w,
                       const Reduce* r, const int* skip, cudaStream_t s) {
    if (r) smooth_f32<true>(A, EpiSmooth32<true, false, false>{d, f32, f64, x, y32, y64, w}, *r, skip, s);
    else smooth_f32<false>(A, EpiSmooth32<false, false, false>{d, f32, f64, x, y32, y64, nullptr}, Reduce{}, skip, s);
}

void launch_prolong_add_f32(const DevCsr& P, const float* xc, float* x, const int* skip,
                            cudaStream_t s) {
    run32(P, P.val32, P.val16, EpiProlong32{xc, x}, Reduce{}, skip, s);
}

void launch_prolong_pre_f32(const DevCsr& P, const float* d, const float* f, const float* xc, float* x,
                            const int* skip, cudaStream_t s) {
    run32(P, P.val32, P.val16, EpiProlongPre32{d, f, xc, x}, Reduce{}, skip, s);
}

// Standalone product on a caller's device CSR: uniform row split (no
// schedule to build), column indices bounds-checked (a bad index sets bit 1
// of *err and contributes zero).
void launch_spmv_dot_uniform(int32_t n, int32_t ncols, const int32_t* ptr, const int32_t* col,
                             const double* val, const double* x, double* y, int rows_per_block,
                             const Reduce& r, int* err_flag, cudaStream_t s) {
    const int64_t nb = (n + rows_per_block - 1) / rows_per_block;
    if (nb > r.stride) fail(AMG_ERR_TOO_LARGE, "reduction buffer smaller than the grid");
    k_spmv<double, EpiYDot, true><<<(unsigned)nb, kThreads, 0, s>>>(
        ptr, col, val, nullptr, n, ncols, rows_per_block, EpiYDot{x, x, y}, r, nullptr, err_flag);
    AMG_CUDA(cudaGetLastError());
}

// --------------------------------------------------------- vector kernels
int vec_grid(int64_t n) {
    const int64_t per = (int64_t)kThreads * 4;
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + per - 1) / per, 152 * 8));
}

__global__ void k_fill(double* x, double v, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        x[i] = v;
}

// Vector kernels run a grid-stride loop that takes kVecBatch elements a
// thread at a time (i, i + stride, ...): ld(i, v) loads element i's inputs
// for all of them before op(i, v) uses any, so that a thread keeps
// kVecBatch times the loads in flight.  op runs in element order, so sums
// accumulate in the same order as one element at a time.  (On 150^3 the
// update kernels measured about the same either way: they are held by the
// float64 pipe, two operations an element, and the reduction at their end.)
constexpr int kVecBatch = 4;
template <int NV, typename Ld, typename Op>
__device__ __forceinline__ void vec_batched(int64_t n, Ld ld, Op op) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i0 < n; i0 += kVecBatch * stride) {
        double v[kVecBatch][NV];
#pragma unroll
        for (int u = 0; u < kVecBatch; ++u) {
            const int64_t i = i0 + u * stride;
            if (i < n) ld(i, v[u]);
        }
#pragma unroll
        for (int u = 0; u < kVecBatch; ++u) {
            const int64_t i = i0 + u * stride;
            if (i < n) op(i, v[u]);
        }
    }
}

// CG's x update is deferred by one kernel: the update of iteration k,
// x += alpha_k p_k, runs in the p update of iteration k + 1 (which reads p_k
// anyway), or in k_cg_xfinal after the loop.  The iterates are the same,
// operation for operation; the residual update no longer reads p and x nor
// writes x, 8 bytes a row less per iteration.
//   p update:  x += alpha_x p (if pending); p = z + beta p
__global__ void __launch_bounds__(kThreads)
k_cg_pupdate(const KState* __restrict__ st, const double* __restrict__ z, double* __restrict__ p,
             double* __restrict__ x, int64_t n) {
    if (st->halt) return;
    const double beta = st->beta, ax = st->alpha_x;
    if (ax != 0.0) {
        vec_batched<3>(n, [&](int64_t i, double* v) { v[0] = p[i]; v[1] = z[i]; v[2] = x[i]; },
                       [&](int64_t i, const double* v) {
                           x[i] = v[2] + ax * v[0];
                           p[i] = v[1] + beta * v[0];
                       });
    } else {
        vec_batched<2>(n, [&](int64_t i, double* v) { v[0] = p[i]; v[1] = z[i]; },
                       [&](int64_t i, const double* v) { p[i] = v[1] + beta * v[0]; });
    }
}

// The pending x update after the loop (whatever ended it).
__global__ void __launch_bounds__(kThreads)
k_cg_xfinal(const KState* __restrict__ st, const double* __restrict__ p, double* __restrict__ x, int64_t n) {
    const double ax = st->alpha_x;
    if (ax == 0.0) return;
    vec_batched<2>(n, [&](int64_t i, double* v) { v[0] = p[i]; v[1] = x[i]; },
                   [&](int64_t i, const double* v) { x[i] = v[1] + ax * v[0]; });
}

// r -= alpha q with r.r.  F32: also write the updated vector rounded to
// float32 (the input of a float32 V-cycle); a template parameter, so that the
// float64 solve's kernel has no conversion on its float64 pipe.
template <bool F32>
__global__ void __launch_bounds__(kThreads)
k_cg_update(Reduce red, const double* __restrict__ q, double* __restrict__ r, float* __restrict__ r32,
            int64_t n) {
    if (red.st->halt) return;
    const double alpha = red.st->alpha;
    double acc = 0.0;
    vec_batched<2>(n, [&](int64_t i, double* v) { v[0] = r[i]; v[1] = q[i]; },
                   [&](int64_t i, const double* v) {
                       const double t = v[0] - alpha * v[1];
                       r[i] = t;
                       if constexpr (F32) r32[i] = (float)t;
                       acc += t * t;
                   });
    reduce_finalize<1>(red, acc, 0.0);
}

template <bool F32>  // as k_cg_update
__global__ void __launch_bounds__(kThreads)
k_bi_pupdate(const KState* __restrict__ st, const double* __restrict__ r, const double* __restrict__ v,
             double* __restrict__ p, float* __restrict__ p32, int64_t n) {
    if (st->halt) return;
    const double beta = st->beta, omega = st->omega;
    vec_batched<3>(n, [&](int64_t i, double* e) { e[0] = r[i]; e[1] = p[i]; e[2] = v[i]; },
                   [&](int64_t i, const double* e) {
                       const double pv = e[0] + beta * (e[1] - omega * e[2]);
                       p[i] = pv;
                       if constexpr (F32) p32[i] = (float)pv;
                   });
}

template <bool F32>  // as k_cg_update
__global__ void __launch_bounds__(kThreads)
k_bi_s(Reduce red, const double* __restrict__ r, const double* __restrict__ v,
       double* __restrict__ sv, float* __restrict__ s32, int64_t n) {
    if (red.st->halt) return;
    const double alpha = red.st->alpha;
    double acc = 0.0;
    vec_batched<2>(n, [&](int64_t i, double* e) { e[0] = r[i]; e[1] = v[i]; },
                   [&](int64_t i, const double* e) {
                       const double s = e[0] - alpha * e[1];
                       sv[i] = s;
                       if constexpr (F32) s32[i] = (float)s;
                       acc += s * s;
                   });
    reduce_finalize<1>(red, acc, 0.0);
}

__global__ void __launch_bounds__(kThreads)
k_bi_update(Reduce red, const double* __restrict__ rh, const double* __restrict__ ph,
            const double* __restrict__ sh, const double* __restrict__ sv,
            const double* __restrict__ t, double* __restrict__ x, double* __restrict__ r,
            int64_t n) {
    const KState* st = red.st;
    if (st->halt && !st->half) return;
    const double alpha = st->alpha;
    if (st->half) {  // converged on ||s||: x += alpha p^ and stop
        vec_batched<2>(n, [&](int64_t i, double* e) { e[0] = x[i]; e[1] = ph[i]; },
                       [&](int64_t i, const double* e) { x[i] = e[0] + alpha * e[1]; });
        return;
    }
    const double omega = st->omega;
    double a = 0.0, b = 0.0;
    vec_batched<6>(n,
                   [&](int64_t i, double* e) {
                       e[0] = x[i]; e[1] = ph[i]; e[2] = sh[i]; e[3] = sv[i]; e[4] = t[i]; e[5] = rh[i];
                   },
                   [&](int64_t i, const double* e) {
                       x[i] = e[0] + (alpha * e[1] + omega * e[2]);
                       const double v = e[3] - omega * e[4];
                       r[i] = v;
                       a += v * v;
                       b += e[5] * v;
                   });
    reduce_finalize<2>(red, a, b);
}

__global__ void __launch_bounds__(kThreads)
k_dot2(Reduce red, const double* __restrict__ a, const double* __restrict__ b,
       const double* __restrict__ c, const double* __restrict__ d, int64_t n,
       const int* __restrict__ skip) {
    if (skip && *skip) return;
    double s0 = 0.0, s1 = 0.0;
    if (c)
        vec_batched<4>(n, [&](int64_t i, double* e) { e[0] = a[i]; e[1] = b[i]; e[2] = c[i]; e[3] = d[i]; },
                       [&](int64_t i, const double* e) {
                           s0 += e[0] * e[1];
                           s1 += e[2] * e[3];
                       });
    else
        vec_batched<2>(n, [&](int64_t i, double* e) { e[0] = a[i]; e[1] = b[i]; },
                       [&](int64_t i, const double* e) { s0 += e[0] * e[1]; });
    reduce_finalize<2>(red, s0, s1);
}

// Coarsest level: x = A_L^{-1} f, one warp per row of the dense inverse.
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_coarse(const double* __restrict__ inv, int n, const T* __restrict__ f, T* __restrict__ x,
         const int* __restrict__ skip) {
    if (skip && *skip) return;
    const int lane = threadIdx.x & 31;
    const int row = blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
    if (row >= n) return;
    const double* a = inv + (int64_t)row * n;
    double s = 0.0;
    for (int j = lane; j < n; j += 32) s += a[j] * (double)f[j];
    s = warp_sum(s);
    if (lane == 0) x[row] = (T)s;
}

__global__ void k_scale(const double* __restrict__ d, const double* __restrict__ f,
                        double* __restrict__ x, int64_t n, const int* __restrict__ skip) {
    if (skip && *skip) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        x[i] = d[i] * f[i];
}

void launch_scale(const double* d, const double* f, double* x, int64_t n, const int* skip,
                  cudaStream_t s) {
    k_scale<<<vec_grid(n), kThreads, 0, s>>>(d, f, x, n, skip);
    AMG_CUDA(cudaGetLastError());
}

__global__ void k_to_f32(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

// float64 -> bfloat16, one rounding to nearest even
__global__ void k_to_bf16(const double* __restrict__ a, __nv_bfloat16* __restrict__ b, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        b[i] = __double2bfloat16(a[i]);
}

// Structure check of a caller's device CSR before the standalone product:
// bit 0 of *err is set if row_ptr[0] != 0, row_ptr decreases, or
// row_ptr[n] != nnz.
__global__ void k_validate(int32_t n, int64_t nnz, const int32_t* __restrict__ ptr,
                           int* __restrict__ err) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int v = ptr[i];
        bool ok = (v >= 0) && (v <= nnz);
        if (i == 0) ok = ok && (v == 0);
        if (i == n) ok = ok && (v == nnz);
        if (i < n) ok = ok && (ptr[i + 1] >= v);
        if (!ok) atomicOr(err, 1);
    }
}

// Grid of a batched vector kernel K: one wave of the blocks that fit on the
// SMs (K's registers decide how many), or fewer when n needs fewer for
// kVecBatch elements a thread.  With a fixed 8 blocks an SM, kernels whose
// registers allow 4 or 5 ran in two uneven waves.
template <auto K>
static int vec_grid_k(int64_t n) {
    static const int per_sm = [] {
        int b = 0;
        AMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, K, kThreads, 0));
        return std::max(1, b);
    }();
    const int64_t per = (int64_t)kThreads * kVecBatch;
    const int64_t g = std::min<int64_t>((n + per - 1) / per, stream_grid(1 << 30, per_sm));
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, vec_grid(n)));  // within the reduction buffer
}

void launch_fill(double* x, double v, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    k_fill<<<vec_grid(n), kThreads, 0, s>>>(x, v, n);
    AMG_CUDA(cudaGetLastError());
}

void launch_cg_pupdate(KState* st, const double* z, double* p, double* x, int64_t n, cudaStream_t s) {
    k_cg_pupdate<<<vec_grid_k<k_cg_pupdate>(n), kThreads, 0, s>>>(st, z, p, x, n);
    AMG_CUDA(cudaGetLastError());
}

void launch_cg_xfinal(KState* st, const double* p, double* x, int64_t n, cudaStream_t s) {
    k_cg_xfinal<<<vec_grid_k<k_cg_xfinal>(n), kThreads, 0, s>>>(st, p, x, n);
    AMG_CUDA(cudaGetLastError());
}

void launch_cg_update(const Reduce& r, const double* q, double* rv, int64_t n, cudaStream_t s, float* r32) {
    if (r32) k_cg_update<true><<<vec_grid_k<k_cg_update<true>>(n), kThreads, 0, s>>>(r, q, rv, r32, n);
    else k_cg_update<false><<<vec_grid_k<k_cg_update<false>>(n), kThreads, 0, s>>>(r, q, rv, nullptr, n);
    AMG_CUDA(cudaGetLastError());
}

void launch_bi_pupdate(KState* st, const double* r, const double* v, double* p, int64_t n,
                       cudaStream_t s, float* p32) {
    if (p32) k_bi_pupdate<true><<<vec_grid_k<k_bi_pupdate<true>>(n), kThreads, 0, s>>>(st, r, v, p, p32, n);
    else k_bi_pupdate<false><<<vec_grid_k<k_bi_pupdate<false>>(n), kThreads, 0, s>>>(st, r, v, p, nullptr, n);
    AMG_CUDA(cudaGetLastError());
}

void launch_bi_s(const Reduce& red, const double* r, const double* v, double* sv, int64_t n,
                 cudaStream_t s, float* s32) {
    if (s32) k_bi_s<true><<<vec_grid_k<k_bi_s<true>>(n), kThreads, 0, s>>>(red, r, v, sv, s32, n);
    else k_bi_s<false><<<vec_grid_k<k_bi_s<false>>(n), kThreads, 0, s>>>(red, r, v, sv, nullptr, n);
    AMG_CUDA(cudaGetLastError());
}

void launch_bi_update(const Reduce& red, const double* rh, const double* ph, const double* sh,
                      const double* sv, const double* t, double* x, double* rv, int64_t n,
                      cudaStream_t s) {
    k_bi_update<<<vec_grid_k<k_bi_update>(n), kThreads, 0, s>>>(red, rh, ph, sh, sv, t, x, rv, n);
    AMG_CUDA(cudaGetLastError());
}

void launch_dot2(const Reduce& red, const double* a, const double* b, const double* c,
                 const double* d, int64_t n, const int* skip, cudaStream_t s) {
    k_dot2<<<vec_grid_k<k_dot2>(n), kThreads, 0, s>>>(red, a, b, c, d, n, skip);
    AMG_CUDA(cudaGetLastError());
}

void launch_coarse_solve(const double* inv, int32_t n, const double* f, double* x,
                         const int* skip, cudaStream_t s) {
    const int rows_per_block = kThreads / 32;
    k_coarse<double><<<(n + rows_per_block - 1) / rows_per_block, kThreads, 0, s>>>(inv, n, f, x, skip);
    AMG_CUDA(cudaGetLastError());
}

void launch_coarse_solve_f32(const double* inv, int32_t n, const float* f, float* x,
                             const int* skip, cudaStream_t s) {
    const int rows_per_block = kThreads / 32;
    k_coarse<float><<<(n + rows_per_block - 1) / rows_per_block, kThreads, 0, s>>>(inv, n, f, x, skip);
    AMG_CUDA(cudaGetLastError());
}

void launch_copy_to_bf16(const double* a, uint16_t* b, int64_t n, cudaStream_t s) {
    if (n == 0) return;
    const unsigned grid = (unsigned)std::min<int64_t>((n + 255) / 256, 65535);
    k_to_bf16<<<grid, 256, 0, s>>>(a, reinterpret_cast<__nv_bfloat16*>(b), n);
    AMG_CUDA(cudaGetLastError());
}

void launch_copy_to_f32(const double* a, float* b, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    k_to_f32<<<vec_grid(n), kThreads, 0, s>>>(a, b, n);
    AMG_CUDA(cudaGetLastError());
}

void launch_validate_csr(int32_t n, int64_t nnz, const int32_t* ptr, int* err, cudaStream_t s) {
    k_validate<<<vec_grid(n + 1), kThreads, 0, s>>>(n, nnz, ptr, err);
    AMG_CUDA(cudaGetLastError());
}

}  // namespace amg
