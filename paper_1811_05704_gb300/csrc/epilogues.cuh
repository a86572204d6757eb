// epilogues.cuh -- what each step of the solve does around one sparse row
// product s_i = sum_j a_ij g(x_j).  An epilogue provides
//   acc_t         accumulation type
//   ndot          number of dot products it contributes (0..2)
//   xg(c)         the gathered operand g for column c
//   Pre load(i)   row-indexed inputs of row i (loaded before the row product,
//                 so their latency overlaps the gathers)
//   store(i, s, pre, d0, d1)   write the outputs of row i, set dot terms
#pragma once

#include <cuda_runtime.h>

namespace amg {

struct Empty {};

struct EpiY {  // y = A x
    using acc_t = double;
    using Pre = Empty;
    static constexpr int ndot = 0;
    const double* __restrict__ x;
    double* __restrict__ y;
    __device__ double xg(int c) const { return __ldg(x + c); }
    __device__ Pre load(int) const { return {}; }
    __device__ void store(int r, double s, const Pre&, double&, double&) const { y[r] = s; }
};

struct EpiYDot {  // y = A x, dot w.y
    using acc_t = double;
    struct Pre { double w; };
    static constexpr int ndot = 1;
    const double* __restrict__ x;
    const double* __restrict__ w;
    double* __restrict__ y;
    __device__ double xg(int c) const { return __ldg(x + c); }
    __device__ Pre load(int r) const { return {__ldg(w + r)}; }
    __device__ void store(int r, double s, const Pre& p, double& d0, double&) const {
        y[r] = s;
        d0 = p.w * s;
    }
};

struct EpiYDot2 {  // y = A x, dots y.y and y.w
    using acc_t = double;
    struct Pre { double w; };
    static constexpr int ndot = 2;
    const double* __restrict__ x;
    const double* __restrict__ w;
    double* __restrict__ y;
    __device__ double xg(int c) const { return __ldg(x + c); }
    __device__ Pre load(int r) const { return {__ldg(w + r)}; }
    __device__ void store(int r, double s, const Pre& p, double& d0, double& d1) const {
        y[r] = s;
        d0 = s * s;
        d1 = s * p.w;
    }
};

struct EpiRes0 {  // t = f - A x
    using acc_t = double;
    struct Pre { double f; };
    static constexpr int ndot = 0;
    const double* __restrict__ f;
    const double* __restrict__ x;
    double* __restrict__ t;
    __device__ double xg(int c) const { return __ldg(x + c); }
    __device__ Pre load(int r) const { return {__ldg(f + r)}; }
    __device__ void store(int r, double s, const Pre& p, double&, double&) const { t[r] = p.f - s; }
};

struct EpiPre {  // x = d f ; t = f - A x   (first pre-sweep from zero, then the residual)
    using acc_t = double;
    struct Pre { double d, f; };
    static constexpr int ndot = 0;
    const double* __restrict__ d;
    const double* __restrict__ f;
    double* __restrict__ x;
    double* __restrict__ t;
    __device__ double xg(int c) const { return __ldg(d + c) * __ldg(f + c); }
    __device__ Pre load(int r) const { return {__ldg(d + r), __ldg(f + r)}; }
    __device__ void store(int r, double s, const Pre& p, double&, double&) const {
        x[r] = p.d * p.f;
        t[r] = p.f - s;
    }
};

template <bool DOT>
struct EpiSmooth {  // y = x + d (f - A x) ; optional w.y
    using acc_t = double;
    struct Pre { double x, d, f, w; };
    static constexpr int ndot = DOT ? 1 : 0;
    const double* __restrict__ d;
    const double* __restrict__ f;
    const double* __restrict__ x;
    double* __restrict__ y;
    const double* __restrict__ w;
    __device__ double xg(int c) const { return __ldg(x + c); }
    __device__ Pre load(int r) const {
        return {__ldg(x + r), __ldg(d + r), __ldg(f + r), DOT ? __ldg(w + r) : 0.0};
    }
    __device__ void store(int r, double s, const Pre& p, double& d0, double&) const {
        const double v = p.x + p.d * (p.f - s);
        y[r] = v;
        if (DOT) d0 = p.w * v;
    }
};

struct EpiResid {  // r = f - A x (optionally also into r2), dots r.r and f.f
    using acc_t = double;
    struct Pre { double f; };
    static constexpr int ndot = 2;
    const double* __restrict__ f;
    const double* __restrict__ x;
    double* __restrict__ r;
    double* __restrict__ r2;
    __device__ double xg(int c) const { return __ldg(x + c); }
    __device__ Pre load(int i) const { return {__ldg(f + i)}; }
    __device__ void store(int i, double s, const Pre& p, double& d0, double& d1) const {
        const double v = p.f - s;
        r[i] = v;
        if (r2) r2[i] = v;
        d0 = v * v;
        d1 = p.f * p.f;
    }
};

struct EpiProlong {  // x += P xc
    using acc_t = double;
    struct Pre { double x; };
    static constexpr int ndot = 0;
    const double* __restrict__ xc;
    double* __restrict__ x;
    __device__ double xg(int c) const { return __ldg(xc + c); }
    __device__ Pre load(int r) const { return {x[r]}; }
    __device__ void store(int r, double s, const Pre& p, double&, double&) const { x[r] = p.x + s; }
};

// float32 V-cycle: level vectors and matrix values in float32, float32
// accumulation; on the finest level the right-hand side (the Krylov vector)
// is read in float64 and the output written in float64.
struct EpiY32 {
    using acc_t = float;
    using Pre = Empty;
    static constexpr int ndot = 0;
    const float* __restrict__ x;
    float* __restrict__ y;
    __device__ float xg(int c) const { return __ldg(x + c); }
    __device__ Pre load(int) const { return {}; }
    __device__ void store(int r, float s, const Pre&, double&, double&) const { y[r] = s; }
};

struct EpiPre32 {
    using acc_t = float;
    struct Pre { float d, f; };
    static constexpr int ndot = 0;
    const float* __restrict__ d;
    const float* __restrict__ f32;   // level rhs (levels >= 1)
    const double* __restrict__ f64;  // finest-level rhs, or null
    float* __restrict__ x;
    float* __restrict__ t;
    __device__ float fv(int c) const { return f64 ? (float)__ldg(f64 + c) : __ldg(f32 + c); }
    __device__ float xg(int c) const { return __ldg(d + c) * fv(c); }
    __device__ Pre load(int r) const { return {__ldg(d + r), fv(r)}; }
    __device__ void store(int r, float s, const Pre& p, double&, double&) const {
        x[r] = p.d * p.f;
        t[r] = p.f - s;
    }
};

template <bool DOT>
struct EpiSmooth32 {
    using acc_t = float;
    struct Pre { float x, d, f; double w; };
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
    __device__ Pre load(int r) const {
        return {__ldg(x + r), __ldg(d + r), fv(r), DOT ? __ldg(w + r) : 0.0};
    }
    __device__ void store(int r, float s, const Pre& p, double& d0, double&) const {
        const float v = p.x + p.d * (p.f - s);
        if (y64) y64[r] = (double)v;
        else y32[r] = v;
        if (DOT) d0 = p.w * (double)v;
    }
};

struct EpiProlong32 {
    using acc_t = float;
    struct Pre { float x; };
    static constexpr int ndot = 0;
    const float* __restrict__ xc;
    float* __restrict__ x;
    __device__ float xg(int c) const { return __ldg(xc + c); }
    __device__ Pre load(int r) const { return {x[r]}; }
    __device__ void store(int r, float s, const Pre& p, double&, double&) const { x[r] = p.x + s; }
};

}  // namespace amg
