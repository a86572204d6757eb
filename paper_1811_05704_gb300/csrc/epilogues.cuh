// epilogues.cuh -- what each step of the solve does around one sparse row
// product s_i = sum_j a_ij g(x_j).  An epilogue provides
//   acc_t             accumulation type
//   ndot              number of dot products it contributes (0..2)
//   nvec, vptr(k), vbytes(k)
//                     row-indexed input vectors (internal, padded buffers)
//                     ... and optionally vslot(k), a compile-time bound on
//                     vbytes(k) that sizes the vector's shared-memory slot
//                     (8 bytes when absent)
//                     that the streaming engine copies into shared memory with
//                     the tile; an epilogue that reads caller memory by row
//                     (the residual of the initial guess) lists none and
//                     loads it directly
//   xg(c)             the gathered operand g for column c
//   Pre load(i, vt)   row-indexed inputs of row i (from the tile's copies)
//   store(i, s, pre, d0, d1)   write the outputs of row i and add its dot
//                     terms to the running sums d0, d1 (a fused multiply-add
//                     each; an epilogue with fewer than two dots leaves the
//                     unused sums alone, so they cost no float64 add)
// and optionally
//   kSeed, seed(pre)  seeded accumulation for outputs of the form seed - s
//                     (kSeed = -1: a residual f - A x) or seed + s (kSeed =
//                     +1: a correction x + P xc).  The engines then start the
//                     row's accumulator at seed(pre) and subtract or add the
//                     products (each a fused multiply-add), and store()
//                     receives that value instead of s.  This saves one
//                     float64 add per row, which counts on GB300, whose
//                     float64 pipe is nearly as busy as its HBM in these
//                     kernels.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

namespace amg {

// Row-indexed vector slices of one tile: vector k, row i lives at
// base[k] + (i - row0) * elem.  For the row-chunk engine base[k] is the
// global vector itself and row0 = 0.
struct VecTile {
    const unsigned char* base[4];
    int row0;
    template <typename T>
    __device__ __forceinline__ T at(int k, int i) const {
        return reinterpret_cast<const T*>(base[k])[i - row0];
    }
};

struct Empty {};

template <typename Epi, typename = void>
struct Seeding {
    static constexpr int sign = 0;
};
template <typename Epi>
struct Seeding<Epi, std::void_t<decltype(Epi::kSeed)>> {
    static constexpr int sign = Epi::kSeed;
};

struct EpiY {  // y = A x
    using acc_t = double;
    using Pre = Empty;
    static constexpr int ndot = 0, nvec = 0;
    const double* __restrict__ x;
    double* __restrict__ y;
    __device__ const void* vptr(int) const { return nullptr; }
    __device__ int vbytes(int) const { return 8; }
    __device__ double xg(int c) const { return __ldg(x + c); }
    __device__ Pre load(int, const VecTile&) const { return {}; }
    __device__ void store(int r, double s, const Pre&, double&, double&) const { y[r] = s; }
};

struct EpiYDot {  // y = A x, dot w.y
    using acc_t = double;
    struct Pre { double w; };
    static constexpr int ndot = 1, nvec = 1;
    const double* __restrict__ x;
    const double* __restrict__ w;
    double* __restrict__ y;
    __device__ const void* vptr(int) const { return w; }
    __device__ int vbytes(int) const { return 8; }
    __device__ double xg(int c) const { return __ldg(x + c); }
    __device__ Pre load(int r, const VecTile& v) const { return {v.at<double>(0, r)}; }
    __device__ void store(int r, double s, const Pre& p, double& d0, double&) const {
        y[r] = s;
        d0 = fma(p.w, s, d0);
    }
};

struct EpiYDot2 {  // y = A x, dots y.y and y.w
    using acc_t = double;
    struct Pre { double w; };
    static constexpr int ndot = 2, nvec = 1;
    const double* __restrict__ x;
    const double* __restrict__ w;
    double* __restrict__ y;
    __device__ const void* vptr(int) const { return w; }
    __device__ int vbytes(int) const { return 8; }
    __device__ double xg(int c) const { return __ldg(x + c); }
    __device__ Pre load(int r, const VecTile& v) const { return {v.at<double>(0, r)}; }
    __device__ void store(int r, double s, const Pre& p, double& d0, double& d1) const {
        y[r] = s;
        d0 = fma(s, s, d0);
        d1 = fma(s, p.w, d1);
    }
};

struct EpiRes0 {  // t = f - A x
    using acc_t = double;
    struct Pre { double f; };
    static constexpr int ndot = 0, nvec = 1;
    const double* __restrict__ f;
    const double* __restrict__ x;
    double* __restrict__ t;
    __device__ const void* vptr(int) const { return f; }
    __device__ int vbytes(int) const { return 8; }
    __device__ double xg(int c) const { return __ldg(x + c); }
    __device__ Pre load(int r, const VecTile& v) const { return {v.at<double>(0, r)}; }
    static constexpr int kSeed = -1;
    __device__ double seed(const Pre& p) const { return p.f; }
    __device__ void store(int r, double res, const Pre&, double&, double&) const { t[r] = res; }
};

// x = d f ; t = f - A x, the first pre-sweep from zero and the residual.  The
// matrix passed with this epilogue holds a_ij d_j (values scaled by the
// smoother diagonal at setup), so that A (d f) needs one gather, of f.
struct EpiPre {
    using acc_t = double;
    struct Pre { double d, f; };
    static constexpr int ndot = 0, nvec = 2;
    const double* __restrict__ d;
    const double* __restrict__ f;
    double* __restrict__ x;
    double* __restrict__ t;
    __device__ const void* vptr(int k) const { return k == 0 ? (const void*)d : (const void*)f; }
    __device__ int vbytes(int) const { return 8; }
    __device__ double xg(int c) const { return __ldg(f + c); }
    __device__ Pre load(int r, const VecTile& v) const { return {v.at<double>(0, r), v.at<double>(1, r)}; }
    static constexpr int kSeed = -1;
    __device__ double seed(const Pre& p) const { return p.f; }
    __device__ void store(int r, double res, const Pre& p, double&, double&) const {
        x[r] = p.d * p.f;
        t[r] = res;
    }
};

template <bool DOT>
struct EpiSmooth {  // y = x + d (f - A x) ; optional w.y
    using acc_t = double;
    struct Pre { double x, d, f, w; };
    static constexpr int ndot = DOT ? 1 : 0, nvec = DOT ? 4 : 3;
    const double* __restrict__ d;
    const double* __restrict__ f;
    const double* __restrict__ x;
    double* __restrict__ y;
    const double* __restrict__ w;
    __device__ const void* vptr(int k) const {
        return k == 0 ? (const void*)x : k == 1 ? (const void*)d : k == 2 ? (const void*)f : (const void*)w;
    }
    __device__ int vbytes(int) const { return 8; }
    __device__ double xg(int c) const { return __ldg(x + c); }
    __device__ Pre load(int r, const VecTile& v) const {
        return {v.at<double>(0, r), v.at<double>(1, r), v.at<double>(2, r), DOT ? v.at<double>(3, r) : 0.0};
    }
    static constexpr int kSeed = -1;
    __device__ double seed(const Pre& p) const { return p.f; }
    __device__ void store(int r, double res, const Pre& p, double& d0, double&) const {
        const double val = p.x + p.d * res;
        y[r] = val;
        if (DOT) d0 = fma(p.w, val, d0);
    }
};

// y = x + d (f - A x) and f.y: the finest-level post-sweep, whose right-hand
// side is the Krylov residual that the dot product pairs with.
struct EpiSmoothDotF {
    using acc_t = double;
    struct Pre { double x, d, f; };
    static constexpr int ndot = 1, nvec = 3;
    const double* __restrict__ d;
    const double* __restrict__ f;
    const double* __restrict__ x;
    double* __restrict__ y;
    __device__ const void* vptr(int k) const {
        return k == 0 ? (const void*)x : k == 1 ? (const void*)d : (const void*)f;
    }
    __device__ int vbytes(int) const { return 8; }
    __device__ double xg(int c) const { return __ldg(x + c); }
    __device__ Pre load(int r, const VecTile& v) const {
        return {v.at<double>(0, r), v.at<double>(1, r), v.at<double>(2, r)};
    }
    static constexpr int kSeed = -1;
    __device__ double seed(const Pre& p) const { return p.f; }
    __device__ void store(int r, double res, const Pre& p, double& d0, double&) const {
        const double val = p.x + p.d * res;
        y[r] = val;
        d0 = fma(p.f, val, d0);
    }
};

// r = f - A x (optionally also into r2, and with F32 rounded to float32 into
// r32), dots r.r and f.f.  f and x may be the caller's buffers, so f is read
// directly (no shared-memory copy).
template <bool F32>
struct EpiResid {
    using acc_t = double;
    struct Pre { double f; };
    static constexpr int ndot = 2, nvec = 0;
    const double* __restrict__ f;
    const double* __restrict__ x;
    double* __restrict__ r;
    double* __restrict__ r2;
    float* __restrict__ r32;  // optional: r rounded to float32 (input of a float32 V-cycle)
    __device__ const void* vptr(int) const { return nullptr; }
    __device__ int vbytes(int) const { return 8; }
    __device__ double xg(int c) const { return __ldg(x + c); }
    __device__ Pre load(int i, const VecTile&) const { return {__ldg(f + i)}; }
    static constexpr int kSeed = -1;
    __device__ double seed(const Pre& p) const { return p.f; }
    __device__ void store(int i, double v, const Pre& p, double& d0, double& d1) const {
        r[i] = v;
        if (r2) r2[i] = v;
        if constexpr (F32) r32[i] = (float)v;
        d0 = fma(v, v, d0);
        d1 = fma(p.f, p.f, d1);
    }
};

struct EpiProlong {  // x += P xc
    using acc_t = double;
    struct Pre { double x; };
    static constexpr int ndot = 0, nvec = 1;
    const double* __restrict__ xc;
    double* __restrict__ x;
    __device__ const void* vptr(int) const { return x; }
    __device__ int vbytes(int) const { return 8; }
    __device__ double xg(int c) const { return __ldg(xc + c); }
    __device__ Pre load(int r, const VecTile& v) const { return {v.at<double>(0, r)}; }
    static constexpr int kSeed = +1;
    __device__ double seed(const Pre& p) const { return p.x; }
    __device__ void store(int r, double xs, const Pre&, double&, double&) const { x[r] = xs; }
};

// x = d f + P xc: the prolongation and correction of a level whose first
// pre-sweep (x = d f from zero) was folded into the fused restriction
// operator; the pre-sweep's x is formed here, as the seed of the product.
struct EpiProlongPre {
    using acc_t = double;
    struct Pre { double d, f; };
    static constexpr int ndot = 0, nvec = 2;
    const double* __restrict__ d;
    const double* __restrict__ f;
    const double* __restrict__ xc;
    double* __restrict__ x;
    __device__ const void* vptr(int k) const { return k == 0 ? (const void*)d : (const void*)f; }
    __device__ int vbytes(int) const { return 8; }
    __device__ double xg(int c) const { return __ldg(xc + c); }
    __device__ Pre load(int r, const VecTile& v) const { return {v.at<double>(0, r), v.at<double>(1, r)}; }
    static constexpr int kSeed = +1;
    __device__ double seed(const Pre& p) const { return p.d * p.f; }
    __device__ void store(int r, double xs, const Pre&, double&, double&) const { x[r] = xs; }
};

// float32 V-cycle: level vectors and matrix values in float32, float32
// accumulation; on the finest level the right-hand side (the Krylov vector)
// is read in float64 and the output written in float64.
struct EpiY32 {
    using acc_t = float;
    using Pre = Empty;
    static constexpr int ndot = 0, nvec = 0;
    const float* __restrict__ x;
    float* __restrict__ y;
    __device__ const void* vptr(int) const { return nullptr; }
    __device__ int vbytes(int) const { return 4; }
    __device__ float xg(int c) const { return __ldg(x + c); }
    __device__ Pre load(int, const VecTile&) const { return {}; }
    __device__ void store(int r, float s, const Pre&, double&, double&) const { y[r] = s; }
};

// F64: the level's right-hand side is the float64 Krylov vector (finest
// level), else a float32 level vector.  The choice is a template parameter so
// that the kernels of the other levels contain no float64 conversion at all
// (on GB300 a conversion from float64 occupies the float64 pipe like a
// multiply-add).
template <bool F64>
struct EpiPre32 {  // as EpiPre, with matrix values a_ij d_j in float32
    using acc_t = float;
    struct Pre { float d, f; };
    static constexpr int ndot = 0, nvec = 2;
    const float* __restrict__ d;
    const float* __restrict__ f32;   // level rhs (F64 false)
    const double* __restrict__ f64;  // finest-level rhs (F64 true)
    float* __restrict__ x;
    float* __restrict__ t;
    __device__ const void* vptr(int k) const {
        if (k == 0) return d;
        if constexpr (F64) return f64;
        else return f32;
    }
    __device__ int vbytes(int k) const { return (k == 1 && F64) ? 8 : 4; }
    __host__ __device__ static constexpr int vslot(int k) { return (k == 1 && F64) ? 8 : 4; }
    __device__ float xg(int c) const {
        if constexpr (F64) return (float)__ldg(f64 + c);
        else return __ldg(f32 + c);
    }
    __device__ Pre load(int r, const VecTile& v) const {
        if constexpr (F64) return {v.at<float>(0, r), (float)v.at<double>(1, r)};
        else return {v.at<float>(0, r), v.at<float>(1, r)};
    }
    __device__ void store(int r, float s, const Pre& p, double&, double&) const {
        x[r] = p.d * p.f;
        t[r] = p.f - s;
    }
};

// F64IN: the right-hand side is the float64 Krylov vector; F64OUT: the output
// is written in float64 (the finest level's z); otherwise float32 level
// vectors (see EpiPre32 for why these are template parameters).
template <bool DOT, bool F64IN, bool F64OUT>
struct EpiSmooth32 {
    using acc_t = float;
    struct Pre { float x, d, f; double w; };
    static constexpr int ndot = DOT ? 1 : 0, nvec = DOT ? 4 : 3;
    const float* __restrict__ d;
    const float* __restrict__ f32;
    const double* __restrict__ f64;
    const float* __restrict__ x;
    float* __restrict__ y32;   // level output (F64OUT false)
    double* __restrict__ y64;  // finest-level output (F64OUT true)
    const double* __restrict__ w;
    __device__ const void* vptr(int k) const {
        if (k == 0) return x;
        if (k == 1) return d;
        if (k == 2) {
            if constexpr (F64IN) return f64;
            else return f32;
        }
        return w;
    }
    __device__ int vbytes(int k) const { return (k == 3 || (k == 2 && F64IN)) ? 8 : 4; }
    __host__ __device__ static constexpr int vslot(int k) { return (k == 3 || (k == 2 && F64IN)) ? 8 : 4; }
    __device__ float xg(int c) const { return __ldg(x + c); }
    __device__ Pre load(int r, const VecTile& v) const {
        float f;
        if constexpr (F64IN) f = (float)v.at<double>(2, r);
        else f = v.at<float>(2, r);
        double w = 0.0;
        if constexpr (DOT) w = v.at<double>(3, r);
        return {v.at<float>(0, r), v.at<float>(1, r), f, w};
    }
    __device__ void store(int r, float s, const Pre& p, double& d0, double&) const {
        const float val = p.x + p.d * (p.f - s);
        if constexpr (F64OUT) y64[r] = (double)val;
        else y32[r] = val;
        if constexpr (DOT) d0 = fma(p.w, (double)val, d0);
    }
};

struct EpiProlongPre32 {  // as EpiProlongPre, float32 vectors
    using acc_t = float;
    struct Pre { float d, f; };
    static constexpr int ndot = 0, nvec = 2;
    const float* __restrict__ d;
    const float* __restrict__ f;
    const float* __restrict__ xc;
    float* __restrict__ x;
    __device__ const void* vptr(int k) const { return k == 0 ? (const void*)d : (const void*)f; }
    __device__ int vbytes(int) const { return 4; }
    __host__ __device__ static constexpr int vslot(int) { return 4; }
    __device__ float xg(int c) const { return __ldg(xc + c); }
    __device__ Pre load(int r, const VecTile& v) const { return {v.at<float>(0, r), v.at<float>(1, r)}; }
    __device__ void store(int r, float s, const Pre& p, double&, double&) const { x[r] = p.d * p.f + s; }
};

struct EpiProlong32 {
    using acc_t = float;
    struct Pre { float x; };
    static constexpr int ndot = 0, nvec = 1;
    const float* __restrict__ xc;
    float* __restrict__ x;
    __device__ const void* vptr(int) const { return x; }
    __device__ int vbytes(int) const { return 4; }
    __host__ __device__ static constexpr int vslot(int) { return 4; }
    __device__ float xg(int c) const { return __ldg(xc + c); }
    __device__ Pre load(int r, const VecTile& v) const { return {v.at<float>(0, r)}; }
    __device__ void store(int r, float s, const Pre& p, double&, double&) const { x[r] = p.x + s; }
};

}  // namespace amg
