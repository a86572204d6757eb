// tail.cu -- the small coarse levels of the V-cycle in one launch.
//
// Below a few million nonzeros a level's sparse products take a few
// microseconds of memory traffic but each separate launch costs about as much
// again in launch and pipeline-fill latency.  The tail kernel therefore runs
// Algorithm 2 from level ls down to the coarsest level and back up to ls as a
// list of phases -- pre-sweep + residual, restriction, dense coarsest solve,
// prolongation + correction, post-sweep -- in one launch of a single
// thread-block cluster (16 CTAs of 1024 threads where the device allows, else
// 8), with the cluster's hardware barrier between phases: all CTAs of a
// cluster are resident together, so the barrier needs no spinning on global
// memory, and its release/acquire semantics at cluster scope make each
// phase's global-memory results visible to the next.  The data of these
// levels is small enough to stay in L2, so rows are read with plain loads by
// warps (vw lanes per row) rather than streamed.
#include <cuda_runtime.h>

#include <algorithm>

#include "amg_internal.h"
#include "device_common.cuh"

namespace amg {

constexpr int kTailThreads = 1024;

// Every thread of every CTA of the cluster arrives; the wait returns once all
// have arrived (hardware barrier, no polling loop).
__device__ __forceinline__ void cluster_barrier() {
    asm volatile(
        "barrier.cluster.arrive.release.aligned;\n"
        "barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

// Nonzeros a lane loads before it gathers: a lane issues the column and value
// loads of up to kTailBatch nonzeros of its row, then their gathers, then the
// multiply-adds, so that a row costs a few dependent L2 round trips rather
// than one per nonzero.
constexpr int kTailBatch = 8;

template <typename VT, typename T>
__global__ void __launch_bounds__(kTailThreads, 1)
k_tail(const TailPhase* __restrict__ phases, int nph, const int* __restrict__ skip) {
    if (skip && *skip) return;  // the same flag value in every block: uniform
    // the phase table, copied once into shared memory
    extern __shared__ __align__(16) unsigned char tail_sm[];
    TailPhase* ph = reinterpret_cast<TailPhase*>(tail_sm);
    {
        const int words = nph * (int)(sizeof(TailPhase) / 4);
        const uint32_t* src = reinterpret_cast<const uint32_t*>(phases);
        uint32_t* dst = reinterpret_cast<uint32_t*>(tail_sm);
        for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nw = (int)((gridDim.x * blockDim.x) >> 5);
    for (int p = 0; p < nph; ++p) {
        const TailPhase& P = ph[p];
        const T* f = static_cast<const T*>(P.f);
        const T* xin = static_cast<const T*>(P.xin);
        const T* d = static_cast<const T*>(P.d);
        T* out1 = static_cast<T*>(P.out1);
        T* out2 = static_cast<T*>(P.out2);
        const int op = P.op, n = P.n;
        if (op == TAIL_COARSE) {  // x = A_L^{-1} f, a warp per row of the dense inverse
            const int ncols = P.ncols;
            for (int r = gw; r < n; r += nw) {
                const double* a = P.inv + (int64_t)r * ncols;
                double s = 0.0;
                for (int j = lane; j < ncols; j += 32) s += a[j] * (double)f[j];
                s = warp_sum(s);
                if (lane == 0) out1[r] = (T)s;
            }
        } else {
            const int32_t* ptr = P.ptr;
            const int32_t* col = P.col;
            const VT* val = static_cast<const VT*>(P.val);
            const int vw = P.vw, per = 32 / vw;
            const int sub = lane / vw, l2 = lane - sub * vw;
            // gathered operand: f for the pre-sweep (values already scaled by
            // d_j), the input vector otherwise
            const T* g = (op == TAIL_PRE) ? f : xin;
            for (int rb = gw * per; rb < n; rb += nw * per) {  // same trip count in the warp
                const int r = rb + sub;
                const bool act = r < n;
                // the row's epilogue operands, loaded ahead of the product
                T e0 = T(0), e1 = T(0), e2 = T(0);
                if (act && l2 == 0) {
                    if (op == TAIL_PRE) { e0 = f[r]; e1 = d[r]; }
                    else if (op == TAIL_PROLONG) e0 = out1[r];
                    else if (op == TAIL_POST) { e0 = xin[r]; e1 = d[r]; e2 = f[r]; }
                }
                const int kb = act ? ptr[r] : 0, ke = act ? ptr[r + 1] : 0;
                T s = T(0);
                for (int k0 = kb + l2; k0 < ke; k0 += vw * kTailBatch) {
                    int c[kTailBatch];
                    VT v[kTailBatch];
#pragma unroll
                    for (int u = 0; u < kTailBatch; ++u) {
                        const int k = k0 + u * vw;
                        c[u] = k < ke ? col[k] : 0;
                        v[u] = k < ke ? val[k] : VT(0);
                    }
#pragma unroll
                    for (int u = 0; u < kTailBatch; ++u)
                        if (k0 + u * vw < ke) s += (T)v[u] * g[c[u]];
                }
                for (int o = vw >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, vw);
                if (act && l2 == 0) {
                    switch (op) {
                        case TAIL_PRE:
                            out1[r] = e1 * e0;  // x = d f
                            out2[r] = e0 - s;   // t = f - A x
                            break;
                        case TAIL_SPMV: out1[r] = s; break;
                        case TAIL_PROLONG: out1[r] = e0 + s; break;
                        case TAIL_POST: out1[r] = e0 + e1 * (e2 - s); break;
                        default: break;
                    }
                }
            }
        }
        if (p + 1 < nph) cluster_barrier();
    }
}

// Cluster size: 16 CTAs where the device can place such a cluster of this
// kernel, else 8 (the portable size).
template <typename VT, typename T>
static int tail_cluster_size() {
    static const int size = [] {
        AMG_CUDA(cudaFuncSetAttribute(k_tail<VT, T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(16);
        cfg.blockDim = dim3(kTailThreads);
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 16;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int clusters = 0;
        if (cudaOccupancyMaxActiveClusters(&clusters, k_tail<VT, T>, &cfg) != cudaSuccess) {
            cudaGetLastError();
            clusters = 0;
        }
        return clusters > 0 ? 16 : 8;
    }();
    return size;
}

template <typename VT, typename T>
static void launch_tail_t(const TailPlan& plan, const int* skip, cudaStream_t s) {
    const int c = tail_cluster_size<VT, T>();
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(c);
    cfg.blockDim = dim3(kTailThreads);
    cfg.dynamicSmemBytes = (size_t)plan.nph * sizeof(TailPhase);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = c;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    AMG_CUDA(cudaLaunchKernelEx(&cfg, k_tail<VT, T>, (const TailPhase*)plan.phases, plan.nph, skip));
}

void launch_tail(const TailPlan& plan, bool f32, const int* skip, cudaStream_t s) {
    if (f32) launch_tail_t<float, float>(plan, skip, s);
    else launch_tail_t<double, double>(plan, skip, s);
}

}  // namespace amg
