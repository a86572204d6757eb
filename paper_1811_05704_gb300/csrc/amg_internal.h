// amg_internal.h -- declarations shared by the library's translation units.
// Not part of the public ABI (include/amg.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/amg.h"

namespace amg {

// ----------------------------------------------------------------- errors
struct Error {
    amg_status status;
    std::string msg;
};
// Throwing is internal only; every extern "C" entry point catches and turns
// the exception into a status + thread-local message.
[[noreturn]] void fail(amg_status st, const std::string& msg);
void cuda_check(cudaError_t e, const char* what);
#define AMG_CUDA(call) ::amg::cuda_check((call), #call)

// ------------------------------------------------------------ host CSR
struct HostCsr {
    int64_t nrows = 0, ncols = 0;
    std::vector<int32_t> ptr;  // nrows + 1
    std::vector<int32_t> col;
    std::vector<double> val;
    int64_t nnz() const { return ptr.empty() ? 0 : ptr.back(); }
};

// Host part of the setup (setup_host.cpp).  Each function implements one
// step of smoothed aggregation; see the comments there for the readings.
std::vector<double> host_diagonal(const HostCsr& A);  // fails on a zero / missing diagonal
void host_validate(const HostCsr& A);                  // CSR structure checks
int64_t host_aggregate(const HostCsr& A, const std::vector<double>& dg, double eps,
                       std::vector<int32_t>& agg);
void host_prolongation(const HostCsr& A, const std::vector<double>& dg, double eps,
                       const std::vector<int32_t>& agg, int64_t nagg, HostCsr& P,
                       double& omega);
void host_transpose(const HostCsr& P, HostCsr& R);
void host_smoother_diag(const HostCsr& A, const std::vector<double>& dg, const amg_params& prm,
                        std::vector<double>& d);
void host_dense_inverse(const HostCsr& A, std::vector<double>& inv);  // row-major n x n
std::vector<int32_t> host_row_blocks(const std::vector<int32_t>& ptr, int rows_cap, int nnz_cap);
// streaming-engine tiles: (row, nonzero) boundaries and lanes per row; empty
// if a row has more than nnz_cap nonzeros
std::vector<int32_t> host_tiles(const std::vector<int32_t>& ptr, int nnz_cap, int rows_cap_max,
                                int& vw, int& rows_cap);

// Algorithmic bytes of one Krylov iteration on a hierarchy with these level
// sizes (rows, nonzeros of A_l, nonzeros of P_l): every array a kernel reads
// or writes counted once per kernel, the gathered vector once; int32 columns
// and row pointers, V-cycle values of the precision's width (8, 4 or 2
// bytes) with level vectors of 8 or 4 bytes; the outer product q = A p and
// the Krylov vector updates in float64.  CG: one V-cycle, one product and
// the updates of x, r, p; BiCGStab: two of each and its longer updates.
struct LevelSizes {
    int64_t n, nnz, nnz_p;
    int64_t nnz_m = 0;  // nonzeros of the fused restriction operator (0: not used)
};
// cg_x_deferred: the single-system CG applies x += alpha p inside the next
// p update (64 bytes a row of Krylov updates); the batched CG updates x with
// r (72 bytes a row).
double krylov_iteration_bytes(const std::vector<LevelSizes>& lev, int precision, int solver,
                              bool cg_x_deferred);

// ---------------------------------------------------------- device CSR
// Row-block schedule: block b of the SpMV kernel covers rows
// [blk[b], blk[b+1]); at most kRowsPerBlock rows and (unless a single row)
// at most kTileNnz nonzeros, so one block's products fit one shared tile.
constexpr int kThreads = 256;
constexpr int kRowsPerBlock = 256;
constexpr int kTileNnz = 2048;
constexpr int kLongTileNnz = 4096;  // long-row tiles of the streaming engine (at most 128 rows)
constexpr int kConsumers = 256;  // consumer threads per CTA of the streaming engine
constexpr int kBlockRowNnz = 2048;  // long-row engine: rows this long or shorter never take a whole block
constexpr int64_t kPdlAlwaysNnz = (int64_t)1 << 21;  // products below this size always use programmatic dependent launch

struct DevCsr {
    int32_t nrows = 0, ncols = 0;
    int64_t nnz = 0;
    int32_t* ptr = nullptr;
    int32_t* col = nullptr;
    double* val = nullptr;
    float* val32 = nullptr;  // float32 copy (mixed-precision V-cycle), optional
    int32_t* blk = nullptr;  // row-block schedule (row-chunk engine)
    int32_t nblk = 0;
    int2* tiles = nullptr;   // streaming-engine tiles {first row, first nonzero}, ntiles + 1
    int32_t ntiles = 0;      // 0: some row is longer than a tile, use the row-chunk engine
    int32_t vw = 1;          // lanes per row in the streaming engine
    int32_t rows_cap = 256;  // most rows in one tile (256, or 512 for P and R; 128 for long-row tiles)
    int32_t nz_cap = kTileNnz;  // most nonzeros in one tile (kTileNnz, or kLongTileNnz)
    int32_t rows_vw = 0;        // > 0 (no tiles): the long-row engine, with this many lanes a row
    int32_t* brows = nullptr;   // long-row engine: rows of more than brow_min nonzeros, a block each
    int32_t nbrows = 0, brow_min = 0;
    double* vald = nullptr;  // a_ij d_j: values scaled by the smoother diagonal (level A only)
    float* vald32 = nullptr;
    // bfloat16 copies of val and vald (bit patterns; mixed-precision V-cycle
    // with bfloat16-stored values), optional; used instead of val32 and
    // vald32 when present
    uint16_t* val16 = nullptr;
    uint16_t* vald16 = nullptr;
};
// Device CSR arrays carry kPad readable elements past their end (row_ptr
// past n + 1, col/val past nnz): the streaming engine copies 16-byte-aligned
// spans that may overrun the last row by up to three elements.
constexpr int kPad = 8;

// ------------------------------------------------------- Krylov state
// Lives in device memory; scalars of the Krylov recurrences are computed on
// the device by the last block of the kernel that produced the dot products.
struct KState {
    double rtol;
    int maxiter;
    int it;
    int status;      // 0 ok, AMG_ERR_BREAKDOWN
    int halt;        // stop everything (breakdown, or nothing to do)
    int skip2;       // BiCGStab: skip the second half of the step
    int half;        // BiCGStab: converged at the half step
    int first;       // CG: next beta is 0
    int cond;        // last loop condition value
    int zero_rhs;    // ||f|| == 0
    double nf;       // ||f||
    double res;      // recurrence residual / ||f||
    double relres;   // true residual / ||f|| (after the loop)
    double rho, rho_prev, alpha, omega, beta;
    double alpha_x;  // CG: x += alpha_x p not yet applied (0: none pending)
    double dots[4];
};

// What the last block of a dot-producing kernel does with the sums.
enum Fin : int {
    FIN_NONE = 0,    // store dots into st->dots
    FIN_INIT,        // dots: (r.r, f.f): nf, res, loop condition
    FIN_CG_RHO,      // dot: r.z -> beta, rho
    FIN_CG_ALPHA,    // dot: p.q -> alpha
    FIN_CG_RES,      // dot: r.r -> it++, res, loop condition
    FIN_TRUE,        // dot: r.r of the true residual -> relres
    FIN_BI_INIT,     // dots: (r.r, f.f): as FIN_INIT plus rho = r.r, beta
    FIN_BI_ALPHA,    // dot: rh.v -> alpha
    FIN_BI_HALF,     // dot: s.s -> it++, half-step test
    FIN_BI_OMEGA,    // dots: (t.t, t.s) -> omega
    FIN_BI_RES,      // dots: (r.r, rh.r) -> rho, beta, res, loop condition
};

struct Reduce {
    double* partial = nullptr;      // two arrays of `stride` per-block sums
    int stride = 0;                 // >= grid size of any kernel using this buffer
    unsigned int* counter = nullptr;
    KState* st = nullptr;
    int fin = FIN_NONE;
    int set_cond = 0;               // call cudaGraphSetConditional (graph launches only)
    unsigned long long cond_handle = 0;
    double* out = nullptr;          // FIN_NONE with out != nullptr: write dot[0] there
};
constexpr int kMaxReduceBlocks = 1 << 22;  // sanity cap on a reducing grid

// ------------------------------------------------------------ launchers
// SpMV-engine kernels (spmv.cu).  `skip` (may be null): if *skip != 0 the
// kernel returns at once (device-side early exit inside graph loops).
// y = A x
void launch_spmv(const DevCsr& A, const double* x, double* y, const int* skip, cudaStream_t s);
// y = A x and dot(w, y) reduced through r (w = x if null)
void launch_spmv_dot(const DevCsr& A, const double* x, const double* w, double* y,
                     const Reduce& r, const int* skip, cudaStream_t s);
// y = A x and dots (y.y, y.w)
void launch_spmv_dot2(const DevCsr& A, const double* x, const double* w, double* y,
                      const Reduce& r, const int* skip, cudaStream_t s);
// t = f - A x (no dots)
void launch_residual_plain(const DevCsr& A, const double* f, const double* x, double* t,
                           const int* skip, cudaStream_t s);
// x = d f (elementwise)
void launch_scale(const double* d, const double* f, double* x, int64_t n, const int* skip,
                  cudaStream_t s);
int vec_grid(int64_t n);
int stream_grid(int ntiles, int ctas_per_sm);  // persistent grid of the streaming engine
constexpr int kStreamCtasMax = 4;             // most resident streaming CTAs per SM (any value type)
void set_stream_options(bool pdl);
int read_and_clear_dev_err();
void enqueue_dev_err_copy(int* host_dst, cudaStream_t s);
// standalone, uniform rows-per-block schedule, bounds-checked columns
void launch_spmv_dot_uniform(int32_t n, int32_t ncols, const int32_t* ptr, const int32_t* col,
                             const double* val, const double* x, double* y, int rows_per_block,
                             const Reduce& r, int* err_flag, cudaStream_t s);
// x = d f, t = f - A x
void launch_presmooth_residual(const DevCsr& A, const double* d, const double* f, double* x,
                               double* t, const int* skip, cudaStream_t s);
// y = x + d (f - A x), optional dot(w, y)
void launch_smooth(const DevCsr& A, const double* d, const double* f, const double* x, double* y,
                   const double* w, const Reduce* r, const int* skip, cudaStream_t s);
// r = f - A x with dots (r.r, f.f); optional copy of r to r2
void launch_residual(const DevCsr& A, const double* f, const double* x, double* r, double* r2,
                     const Reduce& red, const int* skip, cudaStream_t s, float* r32 = nullptr);
// x += P xc
void launch_prolong_add(const DevCsr& P, const double* xc, double* x, const int* skip,
                        cudaStream_t s);
// x = d f + P xc (the level's pre-sweep folded into the fused restriction)
void launch_prolong_pre(const DevCsr& P, const double* d, const double* f, const double* xc, double* x,
                        const int* skip, cudaStream_t s);

// float32 V-cycle variants (mixed precision)
void launch_spmv_f32(const DevCsr& A, const float* x, float* y, const int* skip, cudaStream_t s);
void launch_presmooth_residual_f32(const DevCsr& A, const float* d, const float* f32,
                                   const double* f64, float* x, float* t, const int* skip,
                                   cudaStream_t s);
void launch_smooth_f32(const DevCsr& A, const float* d, const float* f32, const double* f64,
                       const float* x, float* y32, double* y64, const double* w,
                       const Reduce* r, const int* skip, cudaStream_t s);
void launch_prolong_add_f32(const DevCsr& P, const float* xc, float* x, const int* skip,
                            cudaStream_t s);
void launch_prolong_pre_f32(const DevCsr& P, const float* d, const float* f, const float* xc, float* x,
                            const int* skip, cudaStream_t s);

// vector kernels
void launch_fill(double* x, double v, int64_t n, cudaStream_t s);
void launch_cg_pupdate(KState* st, const double* z, double* p, double* x, int64_t n, cudaStream_t s);
void launch_cg_xfinal(KState* st, const double* p, double* x, int64_t n, cudaStream_t s);
void launch_cg_update(const Reduce& r, const double* q, double* rv, int64_t n, cudaStream_t s,
                      float* r32 = nullptr);
void launch_bi_pupdate(KState* st, const double* r, const double* v, double* p, int64_t n,
                       cudaStream_t s, float* p32 = nullptr);
void launch_bi_s(const Reduce& red, const double* r, const double* v, double* sv, int64_t n,
                 cudaStream_t s, float* s32 = nullptr);
void launch_bi_update(const Reduce& red, const double* rh, const double* ph, const double* sh,
                      const double* sv, const double* t, double* x, double* rv, int64_t n,
                      cudaStream_t s);
void launch_dot2(const Reduce& red, const double* a, const double* b, const double* c,
                 const double* d, int64_t n, const int* skip, cudaStream_t s);
void launch_coarse_solve(const double* inv, int32_t n, const double* f, double* x,
                         const int* skip, cudaStream_t s);
void launch_coarse_solve_f32(const double* inv, int32_t n, const float* f, float* x,
                             const int* skip, cudaStream_t s);
void launch_copy_to_f32(const double* a, float* b, int64_t n, cudaStream_t s);
void launch_copy_to_bf16(const double* a, uint16_t* b, int64_t n, cudaStream_t s);
void launch_validate_csr(int32_t n, int64_t nnz, const int32_t* ptr, int* err, cudaStream_t s);

// Small coarse levels in one cooperative launch (tail.cu).
enum TailOp : int { TAIL_PRE = 0, TAIL_SPMV = 1, TAIL_COARSE = 2, TAIL_PROLONG = 3, TAIL_POST = 4 };
struct TailPhase {
    int op;             // TailOp
    int n;              // rows
    int vw;             // lanes per row
    int ncols;          // columns of the dense inverse (TAIL_COARSE)
    const int32_t* ptr;
    const int32_t* col;
    const void* val;    // matrix values (scaled by d_j for TAIL_PRE)
    const double* inv;  // dense inverse (TAIL_COARSE)
    const void* d;      // smoother diagonal
    const void* f;      // right-hand side of the level
    const void* xin;    // gathered input vector
    void* out1;
    void* out2;
};
struct TailPlan {
    TailPhase* phases = nullptr;  // device array
    int nph = 0;
};
void launch_tail(const TailPlan& plan, bool f32, const int* skip, cudaStream_t s);
int* dev_err_ptr();
// Runs the bounded-wait check kernel on the current device; returns the device
// error word it left (cleared afterwards) and the kernel's duration.
int check_wait_limit(double* seconds);

// Device set-up of one level (setup_dev.cu); the same results, bit for bit,
// as the host functions above.  dev_prolongation and dev_transpose allocate
// the output matrix's arrays (stream-ordered, kPad padding).
void dev_diagonal(const DevCsr& A, double* dg, cudaStream_t s);  // fails on a zero / missing diagonal
void dev_smoother_diag(const DevCsr& A, const double* dg, const amg_params& prm, double* d, cudaStream_t s);
void dev_scale_columns(const DevCsr& A, const double* d, double* out, cudaStream_t s);  // a_ij d_j
int64_t dev_aggregate(const DevCsr& A, const double* dg, double eps, int32_t* agg, uint8_t* strong,
                      cudaStream_t s);
void dev_prolongation(const DevCsr& A, const double* dg, const uint8_t* strong, const int32_t* agg,
                      int64_t nagg, DevCsr& P, double& omega, cudaStream_t s);
void dev_transpose(const DevCsr& P, DevCsr& R, cudaStream_t s);
// M holds R A (from device_spgemm); its values become those of R - (R A) D.
void dev_fused_restriction(const DevCsr& R, const double* d, DevCsr& M, cudaStream_t s);

// out[0..n] = exclusive prefix sums of in[0..n-1] (setup_dev.cu); returns the
// total; fails with TOO_LARGE if it reaches 2^31 - 1.
int64_t dev_exclusive_scan(const int32_t* in, int32_t* out, int64_t n, cudaStream_t s);

// Galerkin product on the device (spgemm.cu): C = A B, pattern structural,
// entries accumulated in ascending order of the inner index.
// C's arrays are stream-ordered allocations on s (free with dev_free_async).
void device_spgemm(const DevCsr& A, const DevCsr& B, DevCsr& C, cudaStream_t s);

// device memory helpers
template <typename T>
T* dev_alloc(size_t count);
void dev_free(void* p);
// Stream-ordered device memory (the device's default memory pool): freeing
// does not synchronise the device, so set-ups and frees on one stream do not
// stall solves running on other streams.  Memory from dev_alloc_async is
// freed with dev_free_async.
void* dev_alloc_async_bytes(size_t bytes, cudaStream_t s);
template <typename T>
T* dev_alloc_async(size_t count, cudaStream_t s) {
    return static_cast<T*>(dev_alloc_async_bytes(count * sizeof(T), s));
}
void dev_free_async(void* p, cudaStream_t s);

}  // namespace amg
