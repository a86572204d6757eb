// device_common.cuh -- block reductions and the on-device Krylov scalar
// updates run by the last block of a dot-producing kernel.
#pragma once

#include <cuda_runtime.h>

#include "amg_internal.h"

namespace amg {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the block (blockDim.x a multiple of 32) in a fixed order; the
// result is valid in thread 0.  `sh` needs blockDim.x/32 doubles.
__device__ __forceinline__ double block_sum(double v, double* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0) {
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    }
    return t;
}

__device__ __forceinline__ void set_loop(const Reduce& red, int cond) {
    red.st->cond = cond;
    if (red.set_cond) cudaGraphSetConditional((cudaGraphConditionalHandle)red.cond_handle, cond ? 1u : 0u);
}

__device__ __forceinline__ void breakdown(const Reduce& red) {
    KState* st = red.st;
    st->status = AMG_ERR_BREAKDOWN;
    st->halt = 1;
    st->skip2 = 1;
    set_loop(red, 0);
}

__device__ __forceinline__ bool bad(double v) { return !isfinite(v); }

// Krylov scalar recurrences, executed by one thread once the dot products of
// the current kernel are complete.  CG follows preconditioned CG (Saad,
// Alg. 9.1); BiCGStab the right-preconditioned form (Saad, Alg. 7.7).
static __device__ void finalize(const Reduce& red, double a, double b) {
    KState* st = red.st;
    switch (red.fin) {
        case FIN_NONE:
            if (red.out) *red.out = a;
            else { st->dots[0] = a; st->dots[1] = b; }
            break;
        case FIN_INIT:
        case FIN_BI_INIT: {
            const double nf = sqrt(b);
            st->nf = nf;
            st->first = 1;
            st->half = 0;
            st->skip2 = 0;
            if (nf == 0.0) {
                st->zero_rhs = 1;
                st->res = 0.0;
                st->halt = 1;
                set_loop(red, 0);
                break;
            }
            st->res = sqrt(a) / nf;
            int cond = (st->res > st->rtol) && (st->it < st->maxiter) && !st->halt;
            if (red.fin == FIN_BI_INIT) {
                st->rho_prev = 1.0;
                st->alpha = 1.0;
                st->omega = 1.0;
                st->rho = a;  // shadow residual = r, so rh.r = r.r
                st->beta = st->rho;
                if (cond && (st->rho == 0.0 || bad(st->rho))) { breakdown(red); break; }
            }
            if (!cond) st->halt = 1;
            set_loop(red, cond);
            break;
        }
        case FIN_CG_RHO: {
            if (!(a > 0.0) || bad(a)) { breakdown(red); break; }
            st->beta = st->first ? 0.0 : a / st->rho;
            st->rho = a;
            st->first = 0;
            break;
        }
        case FIN_CG_ALPHA: {
            // the p update before this product applied the pending x update
            st->alpha_x = 0.0;
            if (!(a > 0.0) || bad(a)) { breakdown(red); break; }
            st->alpha = st->rho / a;
            st->alpha_x = st->alpha;  // x += alpha p, applied by the next p update or after the loop
            break;
        }
        case FIN_CG_RES: {
            st->it += 1;
            st->res = sqrt(a) / st->nf;
            set_loop(red, (st->res > st->rtol) && (st->it < st->maxiter));
            break;
        }
        case FIN_TRUE:
            st->relres = (st->nf > 0.0) ? sqrt(a) / st->nf : 0.0;
            break;
        case FIN_BI_ALPHA: {
            if (a == 0.0 || bad(a)) { breakdown(red); break; }
            st->alpha = st->rho / a;
            break;
        }
        case FIN_BI_HALF: {
            st->it += 1;
            const double rs = sqrt(a) / st->nf;
            if (rs <= st->rtol) {
                st->half = 1;
                st->skip2 = 1;
                st->res = rs;
                set_loop(red, 0);
            }
            break;
        }
        case FIN_BI_OMEGA: {
            if (a == 0.0 || bad(a)) { breakdown(red); break; }
            const double om = b / a;
            if (om == 0.0 || bad(om)) { breakdown(red); break; }
            st->omega = om;
            break;
        }
        case FIN_BI_RES: {
            st->rho_prev = st->rho;
            st->rho = b;
            st->res = sqrt(a) / st->nf;
            const int cond = (st->res > st->rtol) && (st->it < st->maxiter);
            if (cond && (st->rho == 0.0 || bad(st->rho))) { breakdown(red); break; }
            st->beta = (st->rho / st->rho_prev) * (st->alpha / st->omega);
            set_loop(red, cond);
            break;
        }
        default:
            break;
    }
}

// Block sums of a (and, for ND = 2, of b) in a fixed order, valid in thread
// 0.  The block's values are transposed through shared memory: warp w < ND
// adds its sum's column lane by lane over the warps, then reduces its 32
// lanes with shuffles -- nwarps + 4 float64 add instructions a sum, issued by
// one warp.  A shuffle butterfly in every warp issues 5 a warp and nwarps
// more; on GB300 every float64 warp instruction holds the SM's float64 pipe
// for 16 cycles, and the dot-producing kernels end with all their blocks
// reducing at once.  sh: ND * blockDim.x doubles of shared memory
// (blockDim.x a multiple of 32), free again when the call returns.
template <int ND>
__device__ __forceinline__ void block_sums(double a, double b, double* sh, double& ta, double& tb) {
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
    sh[tid] = a;
    if (ND > 1) sh[nt + tid] = b;
    __syncthreads();
    double t = 0.0;
    if (warp < ND) {
        const double* c = sh + warp * nt + lane;
        t = c[0];
        for (int w = 32; w < nt; w += 32) t += c[w];
        t = warp_sum(t);
    }
    __syncthreads();  // every column read
    if (ND > 1 && tid == 32) sh[0] = t;
    if (ND > 1) __syncthreads();
    ta = t;
    tb = ND > 1 ? sh[0] : 0.0;
    if (ND > 1) __syncthreads();  // sh[0] read before anyone reuses sh
}

// Per-block partial sums -> partial[], and the last block to finish sums the
// partials in index order and runs finalize().  Deterministic for a given
// grid size.  Must be reached by every thread of every block of the grid.
// ND: the number of dot products (1: b is ignored and finalize gets 0).
// sh: ND * blockDim.x doubles of shared memory.
template <int ND>
static __device__ void reduce_finalize_sh(const Reduce& red, double a, double b, double* sh) {
    static_assert(ND == 1 || ND == 2, "one or two dot products");
    __shared__ int last;
    double ta, tb;
    block_sums<ND>(a, b, sh, ta, tb);
    if (threadIdx.x == 0) {
        red.partial[blockIdx.x] = ta;
        if (ND > 1) red.partial[red.stride + blockIdx.x] = tb;
        // release: this block's partials are visible before its ticket;
        // acquire: the last block sees every block's partials (the barrier
        // below passes that on to its other threads).  Measured against a
        // full fence and a relaxed atomic: 150^3 FP64 solve 8.384 -> 8.361 ms.
        unsigned int ticket;
        asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(ticket) : "l"(red.counter) : "memory");
        last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    double sa = 0.0, sb = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
        sa += __ldcg(red.partial + i);
        if (ND > 1) sb += __ldcg(red.partial + red.stride + i);
    }
    block_sums<ND>(sa, sb, sh, ta, tb);
    if (threadIdx.x == 0) {
        *red.counter = 0u;
        finalize(red, ta, tb);
    }
}

// The same with a static scratch, for kernels of at most kThreads threads.
template <int ND>
static __device__ void reduce_finalize(const Reduce& red, double a, double b) {
    __shared__ double sh[ND * kThreads];
    reduce_finalize_sh<ND>(red, a, b, sh);
}

}  // namespace amg
