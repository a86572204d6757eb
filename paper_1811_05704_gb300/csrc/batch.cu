// batch.cu -- one persistent kernel solving many independent systems.
//
// A CTA takes the next system from a device work queue and runs its whole
// preconditioned CG (the same recurrences, stopping test and restart rule as
// the single-system solve) with block-level barriers between steps and
// fixed-order block reductions; the V-cycle (Algorithm 2) works level by
// level on the system's packed hierarchy, in float32 or float64.  Systems
// finish at different iteration counts; the queue keeps every SM busy until
// the last one ends.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "batch.h"
#include "device_common.cuh"

namespace amg {

namespace {

// Sum over the block, the same total in every thread (fixed order).  The
// values are transposed through shared memory and warp 0 adds them lane by
// lane over the warps, then across its lanes with shuffles: nwarps + 4
// float64 add instructions issued by one warp, against a shuffle butterfly in
// every warp plus nwarps adds in every thread (each float64 warp instruction
// holds the SM's float64 pipe for 16 cycles on GB300).  sh: blockDim.x + 1
// doubles.
constexpr int kMaxBatchThreads = 1024;
__device__ __forceinline__ double block_allsum(double v, double* sh) {
    const int tid = threadIdx.x, lane = tid & 31, nt = blockDim.x;
    __syncthreads();  // the previous call's total has been read
    sh[tid] = v;
    __syncthreads();
    if (tid < 32) {
        double t = sh[lane];
        for (int w = 32; w < nt; w += 32) t += sh[w + lane];
        t = warp_sum(t);
        if (lane == 0) sh[nt] = t;
    }
    __syncthreads();
    return sh[nt];
}

// row i of a CSR matrix times a gathered vector, summed in column order.  The
// columns and values of up to kRowBatch nonzeros are loaded, then their
// operands gathered, before any is accumulated: a short row costs one
// dependent round trip per step instead of one per nonzero.
constexpr int kRowBatch = 8;
template <typename VT, typename XT, typename AT>
__device__ __forceinline__ AT row_dot(const int32_t* __restrict__ ptr, const int32_t* __restrict__ col,
                                      const VT* __restrict__ val, const XT* __restrict__ x, int i) {
    const int kb = ptr[i], ke = ptr[i + 1];
    AT s = AT(0);
    for (int k = kb; k < ke; k += kRowBatch) {
        int c[kRowBatch];
        AT a[kRowBatch], g[kRowBatch];
#pragma unroll
        for (int u = 0; u < kRowBatch; ++u) {
            const bool in = k + u < ke;
            c[u] = in ? col[k + u] : 0;
            a[u] = in ? (AT)val[k + u] : AT(0);
        }
#pragma unroll
        for (int u = 0; u < kRowBatch; ++u) g[u] = (k + u < ke) ? (AT)x[c[u]] : AT(0);
#pragma unroll
        for (int u = 0; u < kRowBatch; ++u)
            if (k + u < ke) s += a[u] * g[u];
    }
    return s;
}

// z = M r (one V-cycle, zero initial guess on every level) and returns the
// block-wide r.z.  T is the V-cycle type; r and z are float64.  rT is r in
// the V-cycle type (float32: r rounded once by the kernel step that wrote r,
// so that the finest level does not convert r's entries at every gather).
template <typename T>
__device__ double vcycle_block(const BSys& S, const double* __restrict__ r, const T* __restrict__ rT,
                               double* __restrict__ z, double* sh) {
    const int L = S.nlev;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    if (L == 1) {  // M = A^{-1}
        double rz = 0.0;
        for (int i = warp; i < S.nc; i += nw) {
            const double* a = S.inv + (int64_t)i * S.nc;
            double s = 0.0;
            for (int j = lane; j < S.nc; j += 32) s += a[j] * r[j];
            s = warp_sum(s);
            if (lane == 0) { z[i] = s; rz += r[i] * s; }
        }
        return block_allsum(rz, sh);
    }
    for (int l = 0; l < L - 1; ++l) {
        const BLevel& v = S.lev[l];
        const T* vald = static_cast<const T*>(v.Avald);
        const T* d = static_cast<const T*>(v.d);
        T* x = static_cast<T*>(v.x);
        T* t = static_cast<T*>(v.t);
        if (l == 0) {
            for (int i = tid; i < v.n; i += nt) {
                const T s = row_dot<T, T, T>(v.Aptr, v.Acol, vald, rT, i);
                const T fi = rT[i];
                x[i] = d[i] * fi;
                t[i] = fi - s;
            }
        } else {
            const T* f = static_cast<const T*>(v.f);
            for (int i = tid; i < v.n; i += nt) {
                const T s = row_dot<T, T, T>(v.Aptr, v.Acol, vald, f, i);
                const T fi = f[i];
                x[i] = d[i] * fi;
                t[i] = fi - s;
            }
        }
        __syncthreads();
        T* fc = static_cast<T*>(S.lev[l + 1].f);
        const T* rv = static_cast<const T*>(v.Rval);
        for (int c = tid; c < v.nc; c += nt) fc[c] = row_dot<T, T, T>(v.Rptr, v.Rcol, rv, t, c);
        __syncthreads();
    }
    {  // coarsest: x = A_L^{-1} f, a warp per row, float64 accumulation
        const BLevel& c = S.lev[L - 1];
        const T* f = static_cast<const T*>(c.f);
        T* x = static_cast<T*>(c.x);
        for (int i = warp; i < S.nc; i += nw) {
            const double* a = S.inv + (int64_t)i * S.nc;
            double s = 0.0;
            for (int j = lane; j < S.nc; j += 32) s += a[j] * (double)f[j];
            s = warp_sum(s);
            if (lane == 0) x[i] = (T)s;
        }
        __syncthreads();
    }
    double rz = 0.0;
    for (int l = L - 2; l >= 0; --l) {
        const BLevel& v = S.lev[l];
        const T* xc = static_cast<const T*>((l + 1 == L - 1) ? S.lev[l + 1].x : S.lev[l + 1].y);
        T* x = static_cast<T*>(v.x);
        const T* pv = static_cast<const T*>(v.Pval);
        for (int i = tid; i < v.n; i += nt) x[i] += row_dot<T, T, T>(v.Pptr, v.Pcol, pv, xc, i);
        __syncthreads();
        const T* av = static_cast<const T*>(v.Aval);
        const T* d = static_cast<const T*>(v.d);
        if (l == 0) {
            for (int i = tid; i < v.n; i += nt) {
                const T s = row_dot<T, T, T>(v.Aptr, v.Acol, av, x, i);
                const double zi = (double)(x[i] + d[i] * (rT[i] - s));
                z[i] = zi;
                rz += r[i] * zi;
            }
        } else {
            const T* f = static_cast<const T*>(v.f);
            T* y = static_cast<T*>(v.y);
            for (int i = tid; i < v.n; i += nt) {
                const T s = row_dot<T, T, T>(v.Aptr, v.Acol, av, x, i);
                y[i] = x[i] + d[i] * (f[i] - s);
            }
        }
        __syncthreads();
    }
    return block_allsum(rz, sh);
}

// Preconditioned CG on one system (block-wide), the same recurrences and
// rules as the single-system solve.
template <typename T>
__device__ void cg_block(const BSys& S, const double* __restrict__ f, double* __restrict__ x, double rtol,
                         int maxiter, BResult* res, double* sh) {
    const int n = S.n, tid = threadIdx.x, nt = blockDim.x;
    double* r = S.r;
    double* z = S.z;
    double* p = S.p;
    double* q = S.q;
    // r in the V-cycle type, written wherever r is: for a float32 V-cycle the
    // finest level's y (unused on that level), else r itself
    T* rT = nullptr;
    if constexpr (std::is_same<T, double>::value) rT = r;
    else if (S.nlev > 1) rT = static_cast<T*>(S.lev[0].y);
    auto put = [&](int i, double v) {
        r[i] = v;
        if constexpr (!std::is_same<T, double>::value) {
            if (rT) rT[i] = (T)v;
        }
    };
    // r = f - A x, ||r||, ||f||
    double a = 0.0, b = 0.0;
    for (int i = tid; i < n; i += nt) {
        const double v = f[i] - row_dot<double, double, double>(S.ptr, S.col, S.val, x, i);
        put(i, v);
        a += v * v;
        b += f[i] * f[i];
    }
    double rr = block_allsum(a, sh);
    const double nf = sqrt(block_allsum(b, sh));
    int it = 0, status = AMG_OK;
    if (nf == 0.0) {
        for (int i = tid; i < n; i += nt) x[i] = 0.0;
        if (tid == 0) { res->iters = 0; res->status = AMG_OK; res->relres = 0.0; }
        return;
    }
    double relres = sqrt(rr) / nf;
    if (!isfinite(relres)) {
        if (tid == 0) { res->iters = 0; res->status = AMG_ERR_INVALID_ARG; res->relres = relres; }
        return;
    }
    for (int attempt = 0; attempt < 64; ++attempt) {
        if (relres <= rtol || it >= maxiter) break;
        double res_k = relres, rho = 0.0;
        bool first = true;
        while (res_k > rtol && it < maxiter) {
            const double rho_new = vcycle_block<T>(S, r, rT, z, sh);
            if (!(rho_new > 0.0) || !isfinite(rho_new)) { status = AMG_ERR_BREAKDOWN; break; }
            const double beta = first ? 0.0 : rho_new / rho;
            rho = rho_new;
            first = false;
            if (beta == 0.0)  // first direction: p = z (whatever p held before)
                for (int i = tid; i < n; i += nt) p[i] = z[i];
            else
                for (int i = tid; i < n; i += nt) p[i] = z[i] + beta * p[i];
            __syncthreads();
            double pq = 0.0;
            for (int i = tid; i < n; i += nt) {
                const double v = row_dot<double, double, double>(S.ptr, S.col, S.val, p, i);
                q[i] = v;
                pq += p[i] * v;
            }
            pq = block_allsum(pq, sh);
            if (!(pq > 0.0) || !isfinite(pq)) { status = AMG_ERR_BREAKDOWN; break; }
            const double alpha = rho / pq;
            double s2 = 0.0;
            for (int i = tid; i < n; i += nt) {
                x[i] += alpha * p[i];
                const double v = r[i] - alpha * q[i];
                put(i, v);
                s2 += v * v;
            }
            res_k = sqrt(block_allsum(s2, sh)) / nf;
            ++it;
        }
        // true residual; restart from it if it misses rtol
        double t2 = 0.0;
        for (int i = tid; i < n; i += nt) {
            const double v = f[i] - row_dot<double, double, double>(S.ptr, S.col, S.val, x, i);
            put(i, v);
            t2 += v * v;
        }
        relres = sqrt(block_allsum(t2, sh)) / nf;
        if (status != AMG_OK) break;
    }
    if (status == AMG_OK && relres > rtol) status = AMG_ERR_NOT_CONVERGED;
    if (tid == 0) { res->iters = it; res->status = status; res->relres = relres; }
}

template <typename T>
__global__ void k_batch_cg(const BSys* __restrict__ sys, const int* __restrict__ order, int nsys,
                           const int64_t* __restrict__ row_off, unsigned int* queue, const double* f,
                           double* x, double rtol, int maxiter, BResult* res) {
    __shared__ double sh[kMaxBatchThreads + 1];
    __shared__ int next;
    for (;;) {
        if (threadIdx.x == 0) next = (int)atomicAdd(queue, 1u);
        __syncthreads();
        const int k = next;
        __syncthreads();
        if (k >= nsys) return;
        const int s = order[k];
        const BSys& S = sys[s];
        const int64_t o = row_off[s];
        cg_block<T>(S, f + o, x + o, rtol, maxiter, res + s, sh);
        __syncthreads();
    }
}

}  // namespace

int batch_max_threads(bool vcycle_f32) {
    cudaFuncAttributes fa;
    AMG_CUDA(cudaFuncGetAttributes(&fa, vcycle_f32 ? (const void*)k_batch_cg<float> : (const void*)k_batch_cg<double>));
    return fa.maxThreadsPerBlock;
}

void launch_batch_cg(const BSys* sys, const int* order, int nsys, const int64_t* row_off,
                     unsigned int* queue, const double* f, double* x, double rtol, int maxiter,
                     bool vcycle_f32, BResult* res, int threads, int ctas_per_sm, cudaStream_t s) {
    int dev = 0, sms = 0;
    AMG_CUDA(cudaGetDevice(&dev));
    AMG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cudaFuncAttributes fa;
    AMG_CUDA(cudaFuncGetAttributes(&fa, vcycle_f32 ? (const void*)k_batch_cg<float> : (const void*)k_batch_cg<double>));
    if (threads > fa.maxThreadsPerBlock) fail(AMG_ERR_INVALID_ARG, "schedule exceeds the kernel's block size limit");
    const int grid = std::max(1, std::min(nsys, sms * ctas_per_sm));
    AMG_CUDA(cudaMemsetAsync(queue, 0, sizeof(unsigned int), s));
    if (vcycle_f32)
        k_batch_cg<float><<<grid, threads, 0, s>>>(sys, order, nsys, row_off, queue, f, x, rtol, maxiter, res);
    else
        k_batch_cg<double><<<grid, threads, 0, s>>>(sys, order, nsys, row_off, queue, f, x, rtol, maxiter, res);
    AMG_CUDA(cudaGetLastError());
}

}  // namespace amg
