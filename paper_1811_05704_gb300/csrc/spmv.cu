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
#include <cuda_runtime.h>

#include <algorithm>

#include "amg_internal.h"
#include "device_common.cuh"

namespace amg {

// ------------------------------------------------------------ epilogues
// Each epilogue provides: acc_t, ndot (dot products it contributes), xg(c)
// (the gathered operand for column c) and store(r, s, d0, d1).
struct EpiY {
    using acc_t = double;
    static constexpr int ndot = 0;
    const double* __restrict__ x;
    double* __restrict__ y;
    __device__ double xg(int c) const { return __ldg(x + c); }
    __device__ void store(int r, double s, double&, double&) const { y[r] = s; }
};

struct EpiYDot {  // y = A x, dot w.y
    using acc_t = double;
    static constexpr int ndot = 1;
    const double* __restrict__ x;
    const double* __restrict__ w;
    double* __restrict__ y;
    __device__ double xg(int c) const { return __ldg(x + c); }
    __device__ void store(int r, double s, double& d0, double&) const {
        y[r] = s;
        d0 = __ldg(w + r) * s;
    }
};

struct EpiRes0 {  // t = f - A x
    using acc_t = double;
    static constexpr int ndot = 0;
    const double* __restrict__ f;
    const double* __restrict__ x;
    double* __restrict__ t;
    __device__ double xg(int c) const { return __ldg(x + c); }
    __device__ void store(int r, double s, double&, double&) const { t[r] = __ldg(f + r) - s; }
};

struct EpiYDot2 {  // y = A x, dots y.y and y.w
    using acc_t = double;
    static constexpr int ndot = 2;
    const double* __restrict__ x;
    const double* __restrict__ w;
    double* __restrict__ y;
    __device__ double xg(int c) const { return __ldg(x + c); }
    __device__ void store(int r, double s, double& d0, double& d1) const {
        y[r] = s;
        d0 = s * s;
        d1 = s * __ldg(w + r);
    }
};

struct EpiPre {  // x = d f ; t = f - A x   (first pre-sweep from zero + residual)
    using acc_t = double;
    static constexpr int ndot = 0;
    const double* __restrict__ d;
    const double* __restrict__ f;
    double* __restrict__ x;
    double* __restrict__ t;
    __device__ double xg(int c) const { return __ldg(d + c) * __ldg(f + c); }
    __device__ void store(int r, double s, double&, double&) const {
        const double fr = __ldg(f + r);
        x[r] = __ldg(d + r) * fr;
        t[r] = fr - s;
    }
};

template <bool DOT>
struct EpiSmooth {  // y = x + d (f - A x) ; optional w.y
    using acc_t = double;
    static constexpr int ndot = DOT ? 1 : 0;
    const double* __restrict__ d;
    const double* __restrict__ f;
    const double* __restrict__ x;
    double* __restrict__ y;
    const double* __restrict__ w;
    __device__ double xg(int c) const { return __ldg(x + c); }
    __device__ void store(int r, double s, double& d0, double&) const {
        const double v = __ldg(x + r) + __ldg(d + r) * (__ldg(f + r) - s);
        y[r] = v;
        if (DOT) d0 = __ldg(w + r) * v;
    }
};

struct EpiResid {  // r = f - A x (optionally also into r2), dots r.r and f.f
    using acc_t = double;
    static constexpr int ndot = 2;
    const double* __restrict__ f;
    const double* __restrict__ x;
    double* __restrict__ r;
    double* __restrict__ r2;
    __device__ double xg(int c) const { return __ldg(x + c); }
    __device__ void store(int i, double s, double& d0, double& d1) const {
        const double fi = __ldg(f + i);
        const double v = fi - s;
        r[i] = v;
        if (r2) r2[i] = v;
        d0 = v * v;
        d1 = fi * fi;
    }
};

struct EpiProlong {  // x += P xc
    using acc_t = double;
    static constexpr int ndot = 0;
    const double* __restrict__ xc;
    double* __restrict__ x;
    __device__ double xg(int c) const { return __ldg(xc + c); }
    __device__ void store(int r, double s, double&, double&) const { x[r] += s; }
};

// float32 V-cycle epilogues: level vectors in float32; on the finest level the
// right-hand side (the Krylov vector) is read in float64 and the output is
// written in float64.
struct EpiY32 {
    using acc_t = float;
    static constexpr int ndot = 0;
    const float* __restrict__ x;
    float* __restrict__ y;
    __device__ float xg(int c) const { return __ldg(x + c); }
    __device__ void store(int r, float s, double&, double&) const { y[r] = s; }
};

struct EpiPre32 {
    using acc_t = float;
    static constexpr int ndot = 0;
    const float* __restrict__ d;
    const float* __restrict__ f32;   // level rhs (levels >= 1)
    const double* __restrict__ f64;  // finest-level rhs (Krylov vector), or null
    float* __restrict__ x;
    float* __restrict__ t;
    __device__ float fv(int c) const { return f64 ? (float)__ldg(f64 + c) : __ldg(f32 + c); }
    __device__ float xg(int c) const { return __ldg(d + c) * fv(c); }
    __device__ void store(int r, float s, double&, double&) const {
        const float fr = fv(r);
        x[r] = __ldg(d + r) * fr;
        t[r] = fr - s;
    }
};

template <bool DOT>
struct EpiSmooth32 {
    using acc_t = float;
    static constexpr int ndot = DOT ? 1 : 0;
    const float* __restrict__ d;
    const float* __restrict__ f32;
    const double* __restrict__ f64;
    const float* __restrict__ x;
    float* __restrict__ y32;   // level output (levels >= 1)
    double* __restrict__ y64;  // finest-level output, or null
    const double* __restrict__ w;
    __device__ float fv(int c) const { return f64 ? (float)__ldg(f64 + c) : __ldg(f32 + c); }
    __device__ float xg(int c) const { return __ldg(x + c); }
    __device__ void store(int r, float s, double& d0, double&) const {
        const float v = __ldg(x + r) + __ldg(d + r) * (fv(r) - s);
        if (y64) y64[r] = (double)v;
        else y32[r] = v;
        if (DOT) d0 = __ldg(w + r) * (double)v;
    }
};

struct EpiProlong32 {
    using acc_t = float;
    static constexpr int ndot = 0;
    const float* __restrict__ xc;
    float* __restrict__ x;
    __device__ float xg(int c) const { return __ldg(xc + c); }
    __device__ void store(int r, float s, double&, double&) const { x[r] += s; }
};

// -------------------------------------------------------------- engine
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

    acc_t acc = acc_t(0);
    for (int c0 = k0; c0 < k1; c0 += kTileNnz) {
        const int c1 = min(c0 + kTileNnz, k1);
        // gather: products of this tile into shared memory, 4 loads in flight
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
    if (tid < nr) epi.store(r0 + tid, acc, d0, d1);
    if constexpr (Epi::ndot > 0) reduce_finalize(red, d0, d1);
}

template <typename VT, typename Epi>
static void run(const DevCsr& A, const VT* val, const Epi& epi, const Reduce& red,
                const int* skip, cudaStream_t s) {
    if (A.nrows == 0) return;
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
    run(A, A.val, EpiPre{d, f, x, t}, Reduce{}, skip, s);
}

void launch_smooth(const DevCsr& A, const double* d, const double* f, const double* x, double* y,
                   const double* w, const Reduce* r, const int* skip, cudaStream_t s) {
    if (r) run(A, A.val, EpiSmooth<true>{d, f, x, y, w}, *r, skip, s);
    else run(A, A.val, EpiSmooth<false>{d, f, x, y, nullptr}, Reduce{}, skip, s);
}

void launch_residual(const DevCsr& A, const double* f, const double* x, double* r, double* r2,
                     const Reduce& red, const int* skip, cudaStream_t s) {
    run(A, A.val, EpiResid{f, x, r, r2}, red, skip, s);
}

void launch_prolong_add(const DevCsr& P, const double* xc, double* x, const int* skip,
                        cudaStream_t s) {
    run(P, P.val, EpiProlong{xc, x}, Reduce{}, skip, s);
}

void launch_spmv_f32(const DevCsr& A, const float* x, float* y, const int* skip, cudaStream_t s) {
    run(A, A.val32, EpiY32{x, y}, Reduce{}, skip, s);
}

void launch_presmooth_residual_f32(const DevCsr& A, const float* d, const float* f32,
                                   const double* f64, float* x, float* t, const int* skip,
                                   cudaStream_t s) {
    run(A, A.val32, EpiPre32{d, f32, f64, x, t}, Reduce{}, skip, s);
}

void launch_smooth_f32(const DevCsr& A, const float* d, const float* f32, const double* f64,
                       const float* x, float* y32, double* y64, const double* w,
                       const Reduce* r, const int* skip, cudaStream_t s) {
    if (r) run(A, A.val32, EpiSmooth32<true>{d, f32, f64, x, y32, y64, w}, *r, skip, s);
    else run(A, A.val32, EpiSmooth32<false>{d, f32, f64, x, y32, y64, nullptr}, Reduce{}, skip, s);
}

void launch_prolong_add_f32(const DevCsr& P, const float* xc, float* x, const int* skip,
                            cudaStream_t s) {
    run(P, P.val32, EpiProlong32{xc, x}, Reduce{}, skip, s);
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

__global__ void k_cg_pupdate(const KState* __restrict__ st, const double* __restrict__ z,
                             double* __restrict__ p, int64_t n) {
    if (st->halt) return;
    const double beta = st->beta;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = z[i] + beta * p[i];
}

__global__ void __launch_bounds__(kThreads)
k_cg_update(Reduce red, const double* __restrict__ p, const double* __restrict__ q,
            double* __restrict__ x, double* __restrict__ r, int64_t n) {
    if (red.st->halt) return;
    const double alpha = red.st->alpha;
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        x[i] += alpha * p[i];
        const double v = r[i] - alpha * q[i];
        r[i] = v;
        acc += v * v;
    }
    reduce_finalize(red, acc, 0.0);
}

__global__ void k_bi_pupdate(const KState* __restrict__ st, const double* __restrict__ r,
                             const double* __restrict__ v, double* __restrict__ p, int64_t n) {
    if (st->halt) return;
    const double beta = st->beta, omega = st->omega;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = r[i] + beta * (p[i] - omega * v[i]);
}

__global__ void __launch_bounds__(kThreads)
k_bi_s(Reduce red, const double* __restrict__ r, const double* __restrict__ v,
       double* __restrict__ sv, int64_t n) {
    if (red.st->halt) return;
    const double alpha = red.st->alpha;
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double s = r[i] - alpha * v[i];
        sv[i] = s;
        acc += s * s;
    }
    reduce_finalize(red, acc, 0.0);
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
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
             i += (int64_t)gridDim.x * blockDim.x)
            x[i] += alpha * ph[i];
        return;
    }
    const double omega = st->omega;
    double a = 0.0, b = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        x[i] += alpha * ph[i] + omega * sh[i];
        const double v = sv[i] - omega * t[i];
        r[i] = v;
        a += v * v;
        b += rh[i] * v;
    }
    reduce_finalize(red, a, b);
}

__global__ void __launch_bounds__(kThreads)
k_dot2(Reduce red, const double* __restrict__ a, const double* __restrict__ b,
       const double* __restrict__ c, const double* __restrict__ d, int64_t n,
       const int* __restrict__ skip) {
    if (skip && *skip) return;
    double s0 = 0.0, s1 = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        s0 += a[i] * b[i];
        if (c) s1 += c[i] * d[i];
    }
    reduce_finalize(red, s0, s1);
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

void launch_fill(double* x, double v, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    k_fill<<<vec_grid(n), kThreads, 0, s>>>(x, v, n);
    AMG_CUDA(cudaGetLastError());
}

void launch_cg_pupdate(KState* st, const double* z, double* p, int64_t n, cudaStream_t s) {
    k_cg_pupdate<<<vec_grid(n), kThreads, 0, s>>>(st, z, p, n);
    AMG_CUDA(cudaGetLastError());
}

void launch_cg_update(const Reduce& r, const double* p, const double* q, double* x, double* rv,
                      int64_t n, cudaStream_t s) {
    k_cg_update<<<vec_grid(n), kThreads, 0, s>>>(r, p, q, x, rv, n);
    AMG_CUDA(cudaGetLastError());
}

void launch_bi_pupdate(KState* st, const double* r, const double* v, double* p, int64_t n,
                       cudaStream_t s) {
    k_bi_pupdate<<<vec_grid(n), kThreads, 0, s>>>(st, r, v, p, n);
    AMG_CUDA(cudaGetLastError());
}

void launch_bi_s(const Reduce& red, const double* r, const double* v, double* sv, int64_t n,
                 cudaStream_t s) {
    k_bi_s<<<vec_grid(n), kThreads, 0, s>>>(red, r, v, sv, n);
    AMG_CUDA(cudaGetLastError());
}

void launch_bi_update(const Reduce& red, const double* rh, const double* ph, const double* sh,
                      const double* sv, const double* t, double* x, double* rv, int64_t n,
                      cudaStream_t s) {
    k_bi_update<<<vec_grid(n), kThreads, 0, s>>>(red, rh, ph, sh, sv, t, x, rv, n);
    AMG_CUDA(cudaGetLastError());
}

void launch_dot2(const Reduce& red, const double* a, const double* b, const double* c,
                 const double* d, int64_t n, const int* skip, cudaStream_t s) {
    k_dot2<<<vec_grid(n), kThreads, 0, s>>>(red, a, b, c, d, n, skip);
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
