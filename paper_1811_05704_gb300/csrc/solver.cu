// solver.cu -- hierarchy construction (Algorithm 1), the V-cycle (Algorithm 2)
// and the Krylov loops, issued either as one CUDA graph per solve (a
// device-side while-node runs the iterations; the loop condition is set by
// the kernel that computes the residual norm) or as host-driven launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstring>

#include "amg_internal.h"
#include "host_parallel.h"
#include "handle.h"

namespace amg {

// ------------------------------------------------------------ memory
template <typename T>
static T* halloc(amg_handle* h, size_t count) {
    T* p = dev_alloc_async<T>(count > 0 ? count : 1, h->stream);
    h->dev_allocs.push_back(p);
    h->dev_bytes += (int64_t)(count > 0 ? count : 1) * (int64_t)sizeof(T);
    return p;
}

static void track(amg_handle* h, const DevCsr& D) {
    h->dev_allocs.push_back(D.ptr);
    h->dev_allocs.push_back(D.col);
    h->dev_allocs.push_back(D.val);
    h->dev_bytes += (int64_t)(D.nrows + 1 + kPad) * 4 + (D.nnz + kPad) * 12;
}

static void schedule(amg_handle* h, const std::vector<int32_t>& ptr, DevCsr& D, int rows_cap_max,
                     bool allow_long = false) {
    const std::vector<int32_t> blk = host_row_blocks(ptr, kRowsPerBlock, kTileNnz);
    D.nblk = (int32_t)blk.size() - 1;
    D.blk = halloc<int32_t>(h, blk.size());
    AMG_CUDA(cudaMemcpyAsync(D.blk, blk.data(), blk.size() * sizeof(int32_t), cudaMemcpyHostToDevice, h->stream));
    int vw = 1, rows_cap = kRowsPerBlock;
    // long-row tiles for the fused restriction operators of a float64
    // V-cycle (allow_long) and the level matrices of a float64 hierarchy,
    // when the matrix is large and its rows long: at least 24 nonzeros a row
    // and enough nonzeros for about two tiles per persistent CTA.  Long-row
    // tiles hold twice the nonzeros, so the same rows get half the lanes
    // each: fewer float64 shuffle adds and epilogue instructions a row.
    // Measured on 150^3 Poisson: the finest operator's product (75 nonzeros
    // a row, 4 lanes instead of 8) 115 -> 102 us; level 1 (32 a row, 2 lanes
    // instead of 4) with them, the FP64 solve 8.46 -> 8.38 ms.  On the dense
    // coarse levels of the 200^3 variable-coefficient problem (130-2,000
    // nonzeros a row) and in the float V-cycles the shallower ring cost more
    // than the fewer lanes saved.
    const int64_t nnz = ptr.back(), nr = (int64_t)ptr.size() - 1;
    const bool long_rows = (allow_long || h->prm.precision == AMG_PRECISION_FP64) &&
                           rows_cap_max == kRowsPerBlock && nr > 0 && nnz >= 24 * nr &&
                           nnz >= (int64_t)kLongTileNnz * 600;
    const int nz_cap = long_rows ? kLongTileNnz : kTileNnz;
    // Float64 values on a matrix of long, irregular rows (at least 32
    // nonzeros a row on average, a row of at least three times the mean, and
    // at least 2^20 nonzeros; the smallest levels' products, a few tiles,
    // measured faster in the streaming engine:
    // the coarse levels and fused operators of problems with strongly varying
    // coefficients) take the long-row engine instead of tiles, whose
    // consumers wait for a tile's longest row.  Measured on 200^3 variable
    // coefficients: level 2 (43 a row, longest 282) 308 -> 248 us, level 3
    // (133, longest 1,167) 504 -> 382 us, the FP64 solve 449 -> 415 ms.  On
    // 150^3 Poisson, whose levels hold rows within twice their mean, tiles
    // stay faster (the solve 8.62 against 8.84 ms with the engine from 40
    // nonzeros a row).
    int64_t longest = 0;
    for (int64_t i = 0; i < nr; ++i) longest = std::max<int64_t>(longest, ptr[i + 1] - ptr[i]);
    const bool irregular = h->prm.precision == AMG_PRECISION_FP64 && nr > 0 && nnz >= 32 * nr &&
                           longest * nr >= 3 * nnz && nnz >= (int64_t)1 << 20;
    const std::vector<int32_t> tiles =
        irregular ? std::vector<int32_t>() : host_tiles(ptr, nz_cap, long_rows ? 128 : rows_cap_max, vw, rows_cap);
    D.tiles = nullptr;
    D.ntiles = 0;
    D.rows_vw = 0;
    if (tiles.empty() && h->prm.use_stream && nr > 0) {
        // a row longer than a tile, or irregular rows: the long-row engine
        // (float64 values; float values take the row-chunk engine).  Rows of more than
        // brow_min nonzeros (kBlockRowNnz, or four times the mean row if that
        // is more) take a block each; the others a group of lanes sized for
        // about one batch of kRowBatch (8) nonzeros a lane.  Measured on the
        // 200^3 variable-coefficient levels: with a block for every row over
        // kBlockRowNnz, levels of 1,100-2,000 nonzeros a row ran 25% slower
        // than with none; levels of 700-860 a row, a few rows of 6,500-8,100,
        // ran 45% faster
        D.brow_min = (int32_t)std::max<int64_t>(kBlockRowNnz, 4 * nnz / nr);
        std::vector<int32_t> brows;
        int64_t small_nnz = 0;
        for (int64_t i = 0; i < nr; ++i) {
            if (ptr[i + 1] - ptr[i] > D.brow_min) brows.push_back((int32_t)i);
            else small_nnz += ptr[i + 1] - ptr[i];
        }
        const double avg = (double)small_nnz / (double)std::max<int64_t>(1, nr - (int64_t)brows.size());
        int lanes = 1;
        while (lanes < 32 && 8.0 * lanes < avg) lanes *= 2;
        D.rows_vw = lanes;
        D.nbrows = (int32_t)brows.size();
        D.brows = nullptr;
        if (!brows.empty()) {
            D.brows = halloc<int32_t>(h, brows.size());
            AMG_CUDA(cudaMemcpyAsync(D.brows, brows.data(), brows.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                                     h->stream));
        }
    }
    if (!tiles.empty() && h->prm.use_stream) {
        // every tile must fit the shared-memory slots of the kernel instance
        // that run() picks for it (RMAX rows, nz_cap nonzeros)
        const int rmax = long_rows ? 128 : (rows_cap <= kRowsPerBlock ? kRowsPerBlock : 2 * kRowsPerBlock);
        for (size_t t = 0; t + 3 < tiles.size(); t += 2)
            if (tiles[t + 2] - tiles[t] > rmax || tiles[t + 3] - tiles[t + 1] > nz_cap)
                fail(AMG_ERR_TOO_LARGE, "streaming tile exceeds its kernel's row or nonzero slots");
        D.ntiles = (int32_t)tiles.size() / 2 - 1;
        D.vw = vw;
        D.rows_cap = rows_cap;
        D.nz_cap = nz_cap;
        int32_t* t = halloc<int32_t>(h, tiles.size());
        AMG_CUDA(cudaMemcpyAsync(t, tiles.data(), tiles.size() * sizeof(int32_t), cudaMemcpyHostToDevice, h->stream));
        D.tiles = reinterpret_cast<int2*>(t);
    }
}

static void make_f32(amg_handle* h, DevCsr& D) {
    if (h->prm.precision == AMG_PRECISION_BF16) {
        D.val16 = halloc<uint16_t>(h, D.nnz + kPad);
        AMG_CUDA(cudaMemsetAsync(D.val16, 0, (D.nnz + kPad) * sizeof(uint16_t), h->stream));
        launch_copy_to_bf16(D.val, D.val16, D.nnz, h->stream);
        return;
    }
    D.val32 = halloc<float>(h, D.nnz + kPad);
    AMG_CUDA(cudaMemsetAsync(D.val32, 0, (D.nnz + kPad) * sizeof(float), h->stream));
    launch_copy_to_f32(D.val, D.val32, D.nnz, h->stream);
}

static void upload(amg_handle* h, const HostCsr& H, DevCsr& D, int rows_cap_max) {
    D.nrows = (int32_t)H.nrows;
    D.ncols = (int32_t)H.ncols;
    D.nnz = H.nnz();
    D.ptr = halloc<int32_t>(h, H.nrows + 1 + kPad);
    D.col = halloc<int32_t>(h, D.nnz + kPad);
    D.val = halloc<double>(h, D.nnz + kPad);
    AMG_CUDA(cudaMemsetAsync(D.ptr, 0, (H.nrows + 1 + kPad) * sizeof(int32_t), h->stream));
    AMG_CUDA(cudaMemsetAsync(D.col, 0, (D.nnz + kPad) * sizeof(int32_t), h->stream));
    AMG_CUDA(cudaMemsetAsync(D.val, 0, (D.nnz + kPad) * sizeof(double), h->stream));
    AMG_CUDA(cudaMemcpyAsync(D.ptr, H.ptr.data(), (H.nrows + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, h->stream));
    AMG_CUDA(cudaMemcpyAsync(D.col, H.col.data(), D.nnz * sizeof(int32_t), cudaMemcpyHostToDevice, h->stream));
    AMG_CUDA(cudaMemcpyAsync(D.val, H.val.data(), D.nnz * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    schedule(h, H.ptr, D, rows_cap_max);
}

static void download(const DevCsr& D, HostCsr& H, cudaStream_t s) {
    H.nrows = D.nrows;
    H.ncols = D.ncols;
    H.ptr.resize(D.nrows + 1);
    H.col.resize(D.nnz);
    H.val.resize(D.nnz);
    AMG_CUDA(cudaMemcpyAsync(H.ptr.data(), D.ptr, (D.nrows + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    AMG_CUDA(cudaMemcpyAsync(H.col.data(), D.col, D.nnz * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    AMG_CUDA(cudaMemcpyAsync(H.val.data(), D.val, D.nnz * sizeof(double), cudaMemcpyDeviceToHost, s));
    AMG_CUDA(cudaStreamSynchronize(s));
}

// Lanes per row for the tail kernel's plain-load rows: about a quarter of the
// mean row length, a power of two in [1, 32].
static int tail_vw(const DevCsr& D) {
    const double avg = D.nrows ? (double)D.nnz / (double)D.nrows : 1.0;
    int vw = 1;
    while (vw < 32 && 2.0 * vw <= avg / 4.0) vw *= 2;
    return vw;
}

constexpr int64_t kTailMaxNnz = 4 << 20;

// Phases of the tail kernel: levels ls..L-2 down (pre-sweep + residual,
// restriction), the dense coarsest solve, levels L-2..ls up (prolongation +
// correction, post-sweep).  Only with one pre- and one post-sweep.
static void build_tail(amg_handle* h) {
    const int nl = (int)h->lev.size();
    h->tail_ls = 0;
    if (!h->prm.use_tail || h->prm.npre != 1 || h->prm.npost != 1 || nl < 3 ||
        h->prm.precision == AMG_PRECISION_BF16)
        return;
    int ls = 0;
    for (int l = 1; l < nl - 1; ++l)
        if (h->lev[l].A.nnz <= kTailMaxNnz) { ls = l; break; }
    if (ls == 0) return;
    const bool f32 = h->prm.precision == AMG_PRECISION_FP32;
    for (int pass = 0; pass < (f32 ? 2 : 1); ++pass) {
        const bool p32 = pass == 1;
        std::vector<TailPhase> ph;
        auto V = [&](double* a, float* b) -> void* { return p32 ? (void*)b : (void*)a; };
        for (int l = ls; l < nl - 1; ++l) {
            Level& v = h->lev[l];
            Level& c = h->lev[l + 1];
            TailPhase pre = {};
            pre.op = TAIL_PRE; pre.n = v.A.nrows; pre.vw = tail_vw(v.A);
            pre.ptr = v.A.ptr; pre.col = v.A.col; pre.val = p32 ? (const void*)v.A.vald32 : (const void*)v.A.vald;
            pre.d = p32 ? (const void*)v.d32 : (const void*)v.d; pre.f = V(v.f, v.f32);
            pre.out1 = V(v.x, v.x32); pre.out2 = V(v.t, v.t32);
            ph.push_back(pre);
            TailPhase rs = {};
            rs.op = TAIL_SPMV; rs.n = v.R.nrows; rs.vw = tail_vw(v.R);
            rs.ptr = v.R.ptr; rs.col = v.R.col; rs.val = p32 ? (const void*)v.R.val32 : (const void*)v.R.val;
            rs.xin = V(v.t, v.t32); rs.out1 = V(c.f, c.f32);
            ph.push_back(rs);
        }
        Level& cl = h->lev[nl - 1];
        TailPhase co = {};
        co.op = TAIL_COARSE; co.n = h->nc; co.ncols = h->nc; co.inv = h->cinv;
        co.f = V(cl.f, cl.f32); co.out1 = V(cl.x, cl.x32);
        ph.push_back(co);
        for (int l = nl - 2; l >= ls; --l) {
            Level& v = h->lev[l];
            Level& c = h->lev[l + 1];
            TailPhase pr = {};
            pr.op = TAIL_PROLONG; pr.n = v.P.nrows; pr.vw = tail_vw(v.P);
            pr.ptr = v.P.ptr; pr.col = v.P.col; pr.val = p32 ? (const void*)v.P.val32 : (const void*)v.P.val;
            pr.xin = (l + 1 == nl - 1) ? V(c.x, c.x32) : V(c.y, c.y32);
            pr.out1 = V(v.x, v.x32);
            ph.push_back(pr);
            TailPhase po = {};
            po.op = TAIL_POST; po.n = v.A.nrows; po.vw = tail_vw(v.A);
            po.ptr = v.A.ptr; po.col = v.A.col; po.val = p32 ? (const void*)v.A.val32 : (const void*)v.A.val;
            po.d = p32 ? (const void*)v.d32 : (const void*)v.d; po.f = V(v.f, v.f32);
            po.xin = V(v.x, v.x32); po.out1 = V(v.y, v.y32);
            ph.push_back(po);
        }
        TailPlan& plan = p32 ? h->tail32 : h->tail64;
        plan.nph = (int)ph.size();
        plan.phases = halloc<TailPhase>(h, ph.size());
        AMG_CUDA(cudaMemcpyAsync(plan.phases, ph.data(), ph.size() * sizeof(TailPhase), cudaMemcpyHostToDevice, h->stream));
    }
    h->tail_ls = ls;
}

// Level vectors of every level and the tail plan (both set-up paths).
static void finish_hierarchy(amg_handle* h);

static std::vector<int32_t> download_ptr(const DevCsr& D, cudaStream_t s) {
    std::vector<int32_t> p(D.nrows + 1);
    AMG_CUDA(cudaMemcpyAsync(p.data(), D.ptr, (D.nrows + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    AMG_CUDA(cudaStreamSynchronize(s));
    return p;
}

// The fused restriction operator of a level.  With one pre-sweep from zero
// the first half of Algorithm 2 on level l -- x = d f, t = f - A x,
// f_{l+1} = R t -- is one linear map of f: f_{l+1} = M f with
// M = R (I - A D) = R - (R A) D, and x = d f can wait for the prolongation
// (x = d f + P x_{l+1}).  M replaces the pre-sweep's product, the round trip
// of t and the product with R by one product, where that moves fewer bytes:
// nnz(M) < nnz(A) + nnz(P) + 7n/3 (12 bytes per nonzero against the 28 bytes
// per row that the separate steps move in addition).  R A is formed only
// when its size bound sum_i nnz(A_i) nnz(P_i) is at most 12 times that and
// at most 2^28 (the rows of R overlap heavily on coarse levels, so the bound
// overestimates nnz(R A) 2-13 times on 3D stencils; the cap keeps the dense
// coarse levels of strongly varying coefficients from costing a huge
// product).  The float32 V-cycle keeps the separate steps on the finest
// level, where M's longer rows cost their gathers more than M saves, and the
// bfloat16-stored one everywhere (no gain there, and M's entries rounded to
// bfloat16 cost an iteration); both measured on 150^3 Poisson.
static void build_fused_restriction(amg_handle* h, Level& L, int level, const std::vector<int32_t>& aptr,
                                    const std::vector<int32_t>& pptr) {
    const bool f32 = h->prm.precision != AMG_PRECISION_FP64;
    if (!h->prm.fused_restriction || h->prm.npre != 1 || h->prm.use_tail || (f32 && level == 0) ||
        h->prm.precision == AMG_PRECISION_BF16)
        return;
    const int64_t n = L.A.nrows;
    double bound = 0.0;
    for (int64_t i = 0; i < n; ++i)
        bound += (double)(aptr[i + 1] - aptr[i]) * (double)(pptr[i + 1] - pptr[i]);
    const double keep = (double)L.A.nnz + (double)L.P.nnz + 7.0 * (double)n / 3.0;
    if (bound > 12.0 * keep || bound > (double)(1 << 28)) return;
    DevCsr M;
    device_spgemm(L.R, L.A, M, h->stream);
    if ((double)M.nnz >= keep) {
        dev_free_async(M.ptr, h->stream);
        dev_free_async(M.col, h->stream);
        dev_free_async(M.val, h->stream);
        return;
    }
    track(h, M);
    dev_fused_restriction(L.R, L.d, M, h->stream);
    schedule(h, download_ptr(M, h->stream), M, kRowsPerBlock, !f32);
    if (f32) make_f32(h, M);
    L.M = M;
}

// Row pointers of a device matrix on the host (for the launch schedules).

// float32 / bfloat16 copies of a level's matrix values, scaled values and
// smoother diagonal (mixed-precision V-cycles), from the device copies.
static void make_level_f32(amg_handle* h, Level& L, int64_t n) {
    make_f32(h, L.A);
    if (h->prm.precision == AMG_PRECISION_BF16) {
        L.A.vald16 = halloc<uint16_t>(h, L.A.nnz + kPad);
        AMG_CUDA(cudaMemsetAsync(L.A.vald16, 0, (L.A.nnz + kPad) * sizeof(uint16_t), h->stream));
        launch_copy_to_bf16(L.A.vald, L.A.vald16, L.A.nnz, h->stream);
    } else {
        L.A.vald32 = halloc<float>(h, L.A.nnz + kPad);
        AMG_CUDA(cudaMemsetAsync(L.A.vald32, 0, (L.A.nnz + kPad) * sizeof(float), h->stream));
        launch_copy_to_f32(L.A.vald, L.A.vald32, L.A.nnz, h->stream);
    }
    L.d32 = halloc<float>(h, n + kPad);
    AMG_CUDA(cudaMemsetAsync(L.d32, 0, (n + kPad) * sizeof(float), h->stream));
    launch_copy_to_f32(L.d, L.d32, n, h->stream);
}

// Algorithm 1 on the GPU: the level matrices never leave the device; the host
// reads back only row pointers (for the launch schedules), the aggregate
// count and damping factor of each level, and the coarsest matrix (for its
// dense inverse).  Same stop rule and the same hierarchy, bit for bit, as the
// host set-up below.
static void build_hierarchy_dev(amg_handle* h, const HostCsr& A0) {
    const amg_params& prm = h->prm;
    const bool f32 = prm.precision != AMG_PRECISION_FP64;
    cudaStream_t s = h->stream;
    h->lev.clear();
    h->lev.reserve(AMG_MAX_LEVELS + 1);
    h->lev.emplace_back();
    upload(h, A0, h->lev[0].A, kRowsPerBlock);
    std::vector<int32_t> aptr = A0.ptr;  // row pointers of the current level's A
    for (int l = 0;; ++l) {
        Level& L = h->lev[l];
        const int64_t n = L.A.nrows;
        double* dg = dev_alloc_async<double>(n, s);
        uint8_t* strong = nullptr;
        auto release = [&]() {
            if (dg) dev_free_async(dg, s);
            if (strong) dev_free_async(strong, s);
            dg = nullptr;
            strong = nullptr;
        };
        try {
            dev_diagonal(L.A, dg, s);
            L.d = halloc<double>(h, n + kPad);
            AMG_CUDA(cudaMemsetAsync(L.d, 0, (n + kPad) * sizeof(double), s));
            dev_smoother_diag(L.A, dg, prm, L.d, s);
            L.A.vald = halloc<double>(h, L.A.nnz + kPad);
            AMG_CUDA(cudaMemsetAsync(L.A.vald, 0, (L.A.nnz + kPad) * sizeof(double), s));
            dev_scale_columns(L.A, L.d, L.A.vald, s);
            bool coarsest = n <= prm.coarse_enough || l + 1 >= prm.max_levels || l + 1 >= AMG_MAX_LEVELS;
            if (!coarsest) {
                double eps = prm.strength_eps;
                if (prm.strength_halving)
                    for (int q = 0; q < l; ++q) eps *= 0.5;
                strong = dev_alloc_async<uint8_t>(L.A.nnz > 0 ? L.A.nnz : 1, s);
                L.agg_dev = halloc<int32_t>(h, n);
                L.nagg = dev_aggregate(L.A, dg, eps, L.agg_dev, strong, s);
                if ((double)L.nagg >= 0.95 * (double)n) {
                    L.nagg = 0;
                    L.agg_dev = nullptr;  // freed with the handle
                    if (n > prm.max_coarse_dense)
                        fail(AMG_ERR_COARSENING_STALLED,
                             "aggregation stalled on level " + std::to_string(l) + " with " +
                                 std::to_string(n) + " rows");
                    coarsest = true;
                } else {
                    dev_prolongation(L.A, dg, strong, L.agg_dev, L.nagg, L.P, L.omega_p, s);
                    track(h, L.P);
                    release();
                    dev_transpose(L.P, L.R, s);
                    track(h, L.R);
                    const std::vector<int32_t> pptr = download_ptr(L.P, s);
                    schedule(h, pptr, L.P, 2 * kRowsPerBlock);
                    schedule(h, download_ptr(L.R, s), L.R, 2 * kRowsPerBlock);
                    DevCsr AP, Ac;
                    device_spgemm(L.A, L.P, AP, s);
                    auto free_ap = [&]() {
                        dev_free_async(AP.ptr, s);
                        dev_free_async(AP.col, s);
                        dev_free_async(AP.val, s);
                    };
                    try {
                        device_spgemm(L.R, AP, Ac, s);
                    } catch (...) {
                        free_ap();
                        throw;
                    }
                    free_ap();
                    track(h, Ac);
                    std::vector<int32_t> cptr = download_ptr(Ac, s);
                    schedule(h, cptr, Ac, kRowsPerBlock);
                    if (f32) { make_f32(h, L.P); make_f32(h, L.R); }
                    build_fused_restriction(h, L, l, aptr, pptr);
                    aptr = std::move(cptr);
                    h->lev.emplace_back();
                    h->lev.back().A = Ac;
                }
            }
            release();
            if (f32) make_level_f32(h, h->lev[l], n);
            if (coarsest) {
                Level& C = h->lev[l];
                if (n > prm.max_coarse_dense)
                    fail(AMG_ERR_TOO_LARGE, "coarsest level has " + std::to_string(n) +
                                                " rows, above max_coarse_dense");
                HostCsr H;
                download(C.A, H, s);
                std::vector<double> inv;
                host_dense_inverse(H, inv);
                h->nc = (int32_t)n;
                h->cinv = halloc<double>(h, inv.size());
                AMG_CUDA(cudaMemcpyAsync(h->cinv, inv.data(), inv.size() * sizeof(double), cudaMemcpyHostToDevice, s));
                break;
            }
        } catch (...) {
            release();
            throw;
        }
    }
    finish_hierarchy(h);
}

// ------------------------------------------------------------- setup
// Algorithm 1.  Stop rule: a level with at most coarse_enough rows, the
// max_levels-th level, or a level whose aggregation keeps >= 95% of the rows
// is the coarsest; a stall on a level larger than max_coarse_dense is an
// error, and so is a coarsest level larger than max_coarse_dense.
void build_hierarchy(amg_handle* h, HostCsr A) {
    if (h->prm.device_setup) {
        build_hierarchy_dev(h, A);
        return;
    }
    const amg_params& prm = h->prm;
    const bool f32 = prm.precision != AMG_PRECISION_FP64;  // float32 V-cycle (values fp32 or bf16)
    h->lev.clear();
    h->lev.reserve(AMG_MAX_LEVELS + 1);  // references to levels stay valid below
    h->lev.emplace_back();
    upload(h, A, h->lev[0].A, kRowsPerBlock);
    for (int l = 0;; ++l) {
        Level& L = h->lev[l];
        const int64_t n = A.nrows;
        const std::vector<double> dg = host_diagonal(A);
        host_smoother_diag(A, dg, prm, L.dhost);
        L.d = halloc<double>(h, n + kPad);
        AMG_CUDA(cudaMemsetAsync(L.d, 0, (n + kPad) * sizeof(double), h->stream));
        AMG_CUDA(cudaMemcpyAsync(L.d, L.dhost.data(), n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        {   // values scaled by the smoother diagonal, for the fused first pre-sweep
            std::vector<double> vd(A.nnz());
            parallel_rows(A.nrows, A.nnz(), [&](int, int64_t lo, int64_t hi) {
                for (int64_t k = A.ptr[lo]; k < A.ptr[hi]; ++k) vd[k] = A.val[k] * L.dhost[A.col[k]];
            });
            L.A.vald = halloc<double>(h, A.nnz() + kPad);
            AMG_CUDA(cudaMemsetAsync(L.A.vald, 0, (A.nnz() + kPad) * sizeof(double), h->stream));
            AMG_CUDA(cudaMemcpyAsync(L.A.vald, vd.data(), A.nnz() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        }
        bool coarsest = n <= prm.coarse_enough || l + 1 >= prm.max_levels || l + 1 >= AMG_MAX_LEVELS;
        if (!coarsest) {
            double eps = prm.strength_eps;
            if (prm.strength_halving)
                for (int q = 0; q < l; ++q) eps *= 0.5;
            L.nagg = host_aggregate(A, dg, eps, L.agg);
            if ((double)L.nagg >= 0.95 * (double)n) {
                L.agg.clear();
                L.nagg = 0;
                if (n > prm.max_coarse_dense)
                    fail(AMG_ERR_COARSENING_STALLED,
                         "aggregation stalled on level " + std::to_string(l) + " with " +
                             std::to_string(n) + " rows");
                coarsest = true;
            } else {
                HostCsr P, R;
                host_prolongation(A, dg, eps, L.agg, L.nagg, P, L.omega_p);
                host_transpose(P, R);
                upload(h, P, L.P, 2 * kRowsPerBlock);
                upload(h, R, L.R, 2 * kRowsPerBlock);
                DevCsr AP, Ac;
                device_spgemm(L.A, L.P, AP, h->stream);
                auto free_ap = [&]() {
                    dev_free_async(AP.ptr, h->stream);
                    dev_free_async(AP.col, h->stream);
                    dev_free_async(AP.val, h->stream);
                };
                try {
                    device_spgemm(L.R, AP, Ac, h->stream);
                } catch (...) {
                    free_ap();
                    throw;
                }
                free_ap();
                track(h, Ac);
                HostCsr next;
                download(Ac, next, h->stream);
                schedule(h, next.ptr, Ac, kRowsPerBlock);
                if (f32) { make_f32(h, L.P); make_f32(h, L.R); }
                build_fused_restriction(h, L, l, A.ptr, P.ptr);
                h->lev.emplace_back();
                h->lev.back().A = Ac;
                A = std::move(next);
            }
        }
        if (f32) {
            make_f32(h, L.A);
            if (prm.precision == AMG_PRECISION_BF16) {
                L.A.vald16 = halloc<uint16_t>(h, L.A.nnz + kPad);
                AMG_CUDA(cudaMemsetAsync(L.A.vald16, 0, (L.A.nnz + kPad) * sizeof(uint16_t), h->stream));
                launch_copy_to_bf16(L.A.vald, L.A.vald16, L.A.nnz, h->stream);
            } else {
                L.A.vald32 = halloc<float>(h, L.A.nnz + kPad);
                AMG_CUDA(cudaMemsetAsync(L.A.vald32, 0, (L.A.nnz + kPad) * sizeof(float), h->stream));
                launch_copy_to_f32(L.A.vald, L.A.vald32, L.A.nnz, h->stream);
            }
            L.d32 = halloc<float>(h, n + kPad);
            std::vector<float> d32(L.dhost.begin(), L.dhost.end());
            d32.resize(n + kPad, 0.0f);
            AMG_CUDA(cudaMemcpyAsync(L.d32, d32.data(), (n + kPad) * sizeof(float), cudaMemcpyHostToDevice, h->stream));
        }
        if (coarsest) {
            if (n > prm.max_coarse_dense)
                fail(AMG_ERR_TOO_LARGE, "coarsest level has " + std::to_string(n) +
                                            " rows, above max_coarse_dense");
            std::vector<double> inv;
            host_dense_inverse(A, inv);
            h->nc = (int32_t)n;
            h->cinv = halloc<double>(h, inv.size());
            AMG_CUDA(cudaMemcpyAsync(h->cinv, inv.data(), inv.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
            break;
        }
    }
    finish_hierarchy(h);
}

static void finish_hierarchy(amg_handle* h) {
    const bool f32 = h->prm.precision != AMG_PRECISION_FP64;
    // level vectors
    const int nl = (int)h->lev.size();
    for (int l = 0; l < nl; ++l) {
        Level& L = h->lev[l];
        const int64_t n = L.A.nrows;
        const bool last = l == nl - 1;
        if (nl == 1) break;
        // padded: the streaming kernels copy 16-byte-aligned row slices
        auto v64 = [&]() { double* p = halloc<double>(h, n + kPad);
                           AMG_CUDA(cudaMemsetAsync(p, 0, (n + kPad) * sizeof(double), h->stream)); return p; };
        auto v32 = [&]() { float* p = halloc<float>(h, n + kPad);
                           AMG_CUDA(cudaMemsetAsync(p, 0, (n + kPad) * sizeof(float), h->stream)); return p; };
        if (l > 0) L.f = v64();
        L.x = v64();
        if (!last) { L.y = v64(); L.t = v64(); }
        if (f32) {
            if (l > 0) L.f32 = v32();
            L.x32 = v32();
            if (!last) { L.y32 = v32(); L.t32 = v32(); }
        }
    }
    AMG_CUDA(cudaStreamSynchronize(h->stream));
    build_tail(h);
}

// ------------------------------------------------------------ issuing
void Issue::pre(int kc) {
    cur = kc;
    ++launches;
    if (!profile) return;
    while (pool->size() < pool_used + 2) {
        cudaEvent_t e;
        AMG_CUDA(cudaEventCreate(&e));
        pool->push_back(e);
    }
    cudaEvent_t a = (*pool)[pool_used++], b = (*pool)[pool_used++];
    AMG_CUDA(cudaEventRecord(a, s));
    events->push_back({kc, {a, b}});
}

void Issue::post() {
    if (!profile) return;
    AMG_CUDA(cudaEventRecord(events->back().second.second, s));
}

static const int* flag_ptr(amg_handle* h, size_t off) {
    return reinterpret_cast<const int*>(reinterpret_cast<const char*>(h->st) + off);
}

// One V-cycle, z = M r (Algorithm 2 body with zero initial guess on every
// level).  `rz`, if given, reduces r.z (fused into the last kernel).
static void issue_vcycle64(amg_handle* h, Issue& I, const double* r, double* z, const int* skip,
                           const Reduce* rz) {
    std::vector<Level>& L = h->lev;
    const int nl = (int)L.size();
    const int npre = h->prm.npre, npost = h->prm.npost;
    cudaStream_t s = I.s;
    std::vector<double*> cur(nl, nullptr);
    const int ls = h->tail_ls;  // levels >= ls run in the tail kernel
    const int down_end = ls ? ls : nl - 1;
    for (int l = 0; l < down_end; ++l) {
        Level& v = L[l];
        const int64_t n = v.A.nrows;
        const double* f = (l == 0) ? r : v.f;
        const int kcp = l == 0 ? AMG_KC_PRESMOOTH_L0 : AMG_KC_VCYCLE_COARSER;
        const int kcr = l == 0 ? AMG_KC_RESTRICT_L0 : AMG_KC_VCYCLE_COARSER;
        if (npre == 0) {
            I.pre(kcp); launch_fill(v.x, 0.0, n, s); I.post();
            I.pre(kcr); launch_spmv(v.R, f, L[l + 1].f, skip, s); I.post();
            cur[l] = v.x;
            continue;
        }
        if (npre == 1 && v.M.nrows > 0) {  // f_{l+1} = M f (pre-sweep, residual and restriction)
            I.pre(kcr); launch_spmv(v.M, f, L[l + 1].f, skip, s); I.post();
            cur[l] = v.x;  // x = d f is formed by the prolongation
            continue;
        }
        if (npre == 1) {
            I.pre(kcp); launch_presmooth_residual(v.A, v.d, f, v.x, v.t, skip, s); I.post();
            cur[l] = v.x;
        } else {
            I.pre(kcp); launch_scale(v.d, f, v.x, n, skip, s); I.post();
            double* a = v.x;
            for (int k = 1; k < npre; ++k) {
                double* b = (a == v.x) ? v.y : v.x;
                I.pre(kcp); launch_smooth(v.A, v.d, f, a, b, nullptr, nullptr, skip, s); I.post();
                a = b;
            }
            I.pre(kcp); launch_residual_plain(v.A, f, a, v.t, skip, s); I.post();
            cur[l] = a;
        }
        I.pre(kcr); launch_spmv(v.R, v.t, L[l + 1].f, skip, s); I.post();
    }
    if (nl == 1) {
        I.pre(AMG_KC_COARSE_SOLVE); launch_coarse_solve(h->cinv, h->nc, r, z, skip, s); I.post();
        if (rz) { I.pre(AMG_KC_OTHER); launch_dot2(*rz, r, z, nullptr, nullptr, h->n, skip, s); I.post(); }
        return;
    }
    std::vector<double*> out(nl, nullptr);
    if (ls) {
        I.pre(AMG_KC_VCYCLE_COARSER); launch_tail(h->tail64, false, skip, s); I.post();
        out[ls] = L[ls].y;
    } else {
        Level& c = L[nl - 1];
        I.pre(AMG_KC_COARSE_SOLVE); launch_coarse_solve(h->cinv, h->nc, c.f, c.x, skip, s); I.post();
        out[nl - 1] = c.x;
    }
    for (int l = (ls ? ls : nl - 1) - 1; l >= 0; --l) {
        Level& v = L[l];
        const double* f = (l == 0) ? r : v.f;
        const int kc = l == 0 ? AMG_KC_PROLONG_L0 : AMG_KC_VCYCLE_COARSER;
        const int kcs = l == 0 ? AMG_KC_POSTSMOOTH_L0 : AMG_KC_VCYCLE_COARSER;
        double* a = cur[l];
        if (npre == 1 && v.M.nrows > 0) {  // x = d f + P x_{l+1}
            I.pre(kc); launch_prolong_pre(v.P, v.d, f, out[l + 1], a, skip, s); I.post();
        } else {
            I.pre(kc); launch_prolong_add(v.P, out[l + 1], a, skip, s); I.post();
        }
        if (npost == 0) {
            if (l == 0) {
                I.pre(AMG_KC_OTHER);
                AMG_CUDA(cudaMemcpyAsync(z, a, v.A.nrows * sizeof(double), cudaMemcpyDeviceToDevice, s));
                I.post();
                if (rz) { I.pre(AMG_KC_OTHER); launch_dot2(*rz, r, z, nullptr, nullptr, h->n, skip, s); I.post(); }
            }
            out[l] = a;
            continue;
        }
        for (int k = 0; k < npost; ++k) {
            const bool last = k == npost - 1;
            double* b = (last && l == 0) ? z : ((a == v.x) ? v.y : v.x);
            const Reduce* red = (last && l == 0) ? rz : nullptr;
            I.pre(kcs); launch_smooth(v.A, v.d, f, a, b, red ? r : nullptr, red, skip, s); I.post();
            a = b;
        }
        out[l] = a;
    }
}

// float32 V-cycle (one pre- and one post-sweep); the finest level reads r and
// writes z in float64, and r.z is reduced in float64.
// r32, if given, is r rounded to float32 (written by the kernel that produced
// r): the finest level then reads it instead of converting r's entries at
// every use -- seven gathers per entry on a 7-point stencil, each conversion
// from float64 an instruction of GB300's narrow float64 pipe.  The result is
// the same either way (the kernels round r to float32 before using it).
static void issue_vcycle32(amg_handle* h, Issue& I, const double* r, const float* r32, double* z,
                           const int* skip, const Reduce* rz) {
    std::vector<Level>& L = h->lev;
    const int nl = (int)L.size();
    cudaStream_t s = I.s;
    if (nl == 1) { issue_vcycle64(h, I, r, z, skip, rz); return; }
    const int ls = h->tail_ls;
    for (int l = 0; l < (ls ? ls : nl - 1); ++l) {
        Level& v = L[l];
        const int kcp = l == 0 ? AMG_KC_PRESMOOTH_L0 : AMG_KC_VCYCLE_COARSER;
        const int kcr = l == 0 ? AMG_KC_RESTRICT_L0 : AMG_KC_VCYCLE_COARSER;
        if (v.M.nrows > 0) {  // f_{l+1} = M f (pre-sweep, residual and restriction; levels >= 1)
            I.pre(kcr); launch_spmv_f32(v.M, v.f32, L[l + 1].f32, skip, s); I.post();
            continue;
        }
        I.pre(kcp);
        launch_presmooth_residual_f32(v.A, v.d32, l == 0 ? r32 : v.f32, (l == 0 && !r32) ? r : nullptr,
                                      v.x32, v.t32, skip, s);
        I.post();
        I.pre(kcr); launch_spmv_f32(v.R, v.t32, L[l + 1].f32, skip, s); I.post();
    }
    const float* below = nullptr;
    if (ls) {
        I.pre(AMG_KC_VCYCLE_COARSER); launch_tail(h->tail32, true, skip, s); I.post();
        below = L[ls].y32;
    } else {
        Level& c = L[nl - 1];
        I.pre(AMG_KC_COARSE_SOLVE); launch_coarse_solve_f32(h->cinv, h->nc, c.f32, c.x32, skip, s); I.post();
        below = c.x32;
    }
    for (int l = (ls ? ls : nl - 1) - 1; l >= 0; --l) {
        Level& v = L[l];
        const int kc = l == 0 ? AMG_KC_PROLONG_L0 : AMG_KC_VCYCLE_COARSER;
        const int kcs = l == 0 ? AMG_KC_POSTSMOOTH_L0 : AMG_KC_VCYCLE_COARSER;
        if (v.M.nrows > 0) {  // x = d f + P x_{l+1}
            I.pre(kc); launch_prolong_pre_f32(v.P, v.d32, v.f32, below, v.x32, skip, s); I.post();
        } else {
            I.pre(kc); launch_prolong_add_f32(v.P, below, v.x32, skip, s); I.post();
        }
        I.pre(kcs);
        launch_smooth_f32(v.A, v.d32, l == 0 ? r32 : v.f32, (l == 0 && !r32) ? r : nullptr, v.x32,
                          l == 0 ? nullptr : v.y32, l == 0 ? z : nullptr,
                          (l == 0 && rz) ? r : nullptr, l == 0 ? rz : nullptr, skip, s);
        I.post();
        below = v.y32;
    }
}

static void issue_vcycle(amg_handle* h, Issue& I, const double* r, const float* r32, double* z,
                         const int* skip, const Reduce* rz) {
    if (h->prm.precision != AMG_PRECISION_FP64) issue_vcycle32(h, I, r, r32, z, skip, rz);
    else issue_vcycle64(h, I, r, z, skip, rz);
}

static Reduce base_reduce(amg_handle* h) {
    Reduce r;
    r.partial = h->partial;
    r.stride = h->stride;
    r.counter = h->counter;
    r.st = h->st;
    return r;
}

static Reduce with(Reduce r, int fin) {
    r.fin = fin;
    return r;
}

// CG (Saad Alg. 9.1, preconditioned): init forms r = f - A x and the norms;
// each pass of the body is z = M r (with r.z), p = z + beta p, q = A p (with
// p.q), x += alpha p, r -= alpha q (with r.r and the loop test).  The x update
// of a pass is applied by the next pass's p update, which reads that p
// anyway, and the last one after the loop (k_cg_xfinal).
static void cg_init(amg_handle* h, Issue& I, const double* f, double* x, const Reduce& b) {
    const DevCsr& A = h->lev[0].A;
    I.pre(AMG_KC_OTHER); launch_residual(A, f, x, h->r, nullptr, with(b, FIN_INIT), nullptr, I.s, h->vin32); I.post();
    I.pre(AMG_KC_OTHER); launch_fill(h->p, 0.0, h->n, I.s); I.post();
}

static void cg_body(amg_handle* h, Issue& I, double* x, const Reduce& b) {
    const DevCsr& A = h->lev[0].A;
    const int* halt = flag_ptr(h, offsetof(KState, halt));
    const Reduce rz = with(b, FIN_CG_RHO);
    issue_vcycle(h, I, h->r, h->vin32, h->z, halt, &rz);
    I.pre(AMG_KC_KRYLOV_UPDATE); launch_cg_pupdate(h->st, h->z, h->p, x, h->n, I.s); I.post();
    I.pre(AMG_KC_SPMV_DOT); launch_spmv_dot(A, h->p, nullptr, h->q, with(b, FIN_CG_ALPHA), halt, I.s); I.post();
    I.pre(AMG_KC_KRYLOV_UPDATE); launch_cg_update(with(b, FIN_CG_RES), h->q, h->r, h->n, I.s, h->vin32); I.post();
}

// BiCGStab (van der Vorst; right-preconditioned, Saad Alg. 7.7).
static void bi_init(amg_handle* h, Issue& I, const double* f, double* x, const Reduce& b) {
    const DevCsr& A = h->lev[0].A;
    I.pre(AMG_KC_OTHER); launch_residual(A, f, x, h->r, h->rh, with(b, FIN_BI_INIT), nullptr, I.s); I.post();
    I.pre(AMG_KC_OTHER); launch_fill(h->p, 0.0, h->n, I.s); I.post();
    I.pre(AMG_KC_OTHER); launch_fill(h->v, 0.0, h->n, I.s); I.post();
}

static void bi_body(amg_handle* h, Issue& I, double* x, const Reduce& b) {
    const DevCsr& A = h->lev[0].A;
    const int* halt = flag_ptr(h, offsetof(KState, halt));
    const int* skip2 = flag_ptr(h, offsetof(KState, skip2));
    I.pre(AMG_KC_KRYLOV_UPDATE); launch_bi_pupdate(h->st, h->r, h->v, h->p, h->n, I.s, h->vin32); I.post();
    issue_vcycle(h, I, h->p, h->vin32, h->ph, halt, nullptr);
    I.pre(AMG_KC_SPMV_DOT); launch_spmv_dot(A, h->ph, h->rh, h->v, with(b, FIN_BI_ALPHA), halt, I.s); I.post();
    I.pre(AMG_KC_KRYLOV_UPDATE); launch_bi_s(with(b, FIN_BI_HALF), h->r, h->v, h->sv, h->n, I.s, h->vin32); I.post();
    issue_vcycle(h, I, h->sv, h->vin32, h->sh, skip2, nullptr);
    I.pre(AMG_KC_SPMV_DOT); launch_spmv_dot2(A, h->sh, h->sv, h->tv, with(b, FIN_BI_OMEGA), skip2, I.s); I.post();
    I.pre(AMG_KC_KRYLOV_UPDATE);
    launch_bi_update(with(b, FIN_BI_RES), h->rh, h->ph, h->sh, h->sv, h->tv, x, h->r, h->n, I.s);
    I.post();
}

static void issue_init(amg_handle* h, Issue& I, const double* f, double* x, const Reduce& b) {
    if (h->prm.solver == AMG_SOLVER_BICGSTAB) bi_init(h, I, f, x, b);
    else cg_init(h, I, f, x, b);
}

static void issue_body(amg_handle* h, Issue& I, double* x, const Reduce& b) {
    if (h->prm.solver == AMG_SOLVER_BICGSTAB) bi_body(h, I, x, b);
    else cg_body(h, I, x, b);
}

static void issue_post(amg_handle* h, Issue& I, const double* f, double* x, const Reduce& b) {
    if (h->prm.solver != AMG_SOLVER_BICGSTAB) {
        I.pre(AMG_KC_KRYLOV_UPDATE); launch_cg_xfinal(h->st, h->p, x, h->n, I.s); I.post();
    }
    I.pre(AMG_KC_OTHER);
    launch_residual(h->lev[0].A, f, x, h->r, nullptr, with(b, FIN_TRUE), nullptr, I.s);
    I.post();
}

// --------------------------------------------------------------- graphs
static void destroy_graph(CachedGraph& g) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.graph) cudaGraphDestroy(g.graph);
    g.exec = nullptr;
    g.graph = nullptr;
}

void destroy_graphs(amg_handle* h) {
    for (CachedGraph& g : h->graphs) destroy_graph(g);
    h->graphs.clear();
}

// Capture [state upload] -> init -> while(cond){ body } -> true residual ->
// [state download] for one (f, x) pair.  The while-node's condition is set
// on the device by the kernels that finish each iteration.
static CachedGraph capture(amg_handle* h, const double* f, double* x) {
    CachedGraph g;
    g.f = f;
    g.x = x;
    cudaStream_t cs = h->cap;
    AMG_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    bool capturing = true, capturing2 = false;
    try {
        cudaStreamCaptureStatus cst;
        cudaGraph_t capg = nullptr;
        const cudaGraphNode_t* deps = nullptr;
        const cudaGraphEdgeData* edata = nullptr;
        size_t ndeps = 0;
        AMG_CUDA(cudaStreamGetCaptureInfo(cs, &cst, nullptr, &capg, &deps, &edata, &ndeps));
        cudaGraphConditionalHandle hc;
        AMG_CUDA(cudaGraphConditionalHandleCreate(&hc, capg, 0, cudaGraphCondAssignDefault));
        Reduce b = base_reduce(h);
        b.set_cond = 1;
        b.cond_handle = (unsigned long long)hc;
        AMG_CUDA(cudaMemcpyAsync(h->st, h->st_in, sizeof(KState), cudaMemcpyHostToDevice, cs));
        Issue I;
        I.s = cs;
        issue_init(h, I, f, x, b);
        g.init_launches = I.launches;

        AMG_CUDA(cudaStreamGetCaptureInfo(cs, &cst, nullptr, &capg, &deps, &edata, &ndeps));
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = hc;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t cnode;
        AMG_CUDA(cudaGraphAddNode(&cnode, capg, deps, edata, ndeps, &cp));
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        AMG_CUDA(cudaStreamUpdateCaptureDependencies(cs, &cnode, nullptr, 1,
                                                     cudaStreamSetCaptureDependencies));
        AMG_CUDA(cudaStreamBeginCaptureToGraph(h->cap2, body, nullptr, nullptr, 0,
                                               cudaStreamCaptureModeThreadLocal));
        capturing2 = true;
        Issue I2;
        I2.s = h->cap2;
        issue_body(h, I2, x, b);
        g.body_launches = I2.launches;
        cudaGraph_t tmp = nullptr;
        capturing2 = false;
        AMG_CUDA(cudaStreamEndCapture(h->cap2, &tmp));

        Issue I3;
        I3.s = cs;
        issue_post(h, I3, f, x, b);
        g.post_launches = I3.launches;
        AMG_CUDA(cudaMemcpyAsync(h->st_out, h->st, sizeof(KState), cudaMemcpyDeviceToHost, cs));
        enqueue_dev_err_copy(h->err_host, cs);
        capturing = false;
        AMG_CUDA(cudaStreamEndCapture(cs, &g.graph));
        AMG_CUDA(cudaGraphInstantiate(&g.exec, g.graph, 0));
    } catch (...) {
        cudaGraph_t tmp = nullptr;
        if (capturing2) cudaStreamEndCapture(h->cap2, &tmp);
        if (tmp) cudaGraphDestroy(tmp);
        tmp = nullptr;
        if (capturing) cudaStreamEndCapture(cs, &tmp);
        if (tmp) cudaGraphDestroy(tmp);
        destroy_graph(g);
        cudaGetLastError();
        throw;
    }
    return g;
}

static CachedGraph& graph_for(amg_handle* h, const double* f, double* x) {
    for (CachedGraph& g : h->graphs)
        if (g.f == f && g.x == x) return g;
    if (h->graphs.size() >= 4) {
        destroy_graph(h->graphs.front());
        h->graphs.erase(h->graphs.begin());
    }
    h->graphs.push_back(capture(h, f, x));
    return h->graphs.back();
}

// ----------------------------------------------------------------- solve
// One attempt: (graph | host loop) -> st_out.  Returns launches issued.
static int64_t attempt(amg_handle* h, const double* f, double* x, bool use_graph, Issue* prof) {
    if (use_graph) {
        CachedGraph* gp = nullptr;
        try {
            gp = &graph_for(h, f, x);
        } catch (const Error& e) {
            // the graph could not be built (e.g. conditional nodes refused):
            // run the same kernels from the host from now on
            h->graph_unsupported = true;
            destroy_graphs(h);
            return attempt(h, f, x, false, prof);
        }
        CachedGraph& g = *gp;
        const int it0 = h->st_in->it;
        ++h->last_graph_attempts;
        AMG_CUDA(cudaGraphLaunch(g.exec, h->stream));
        AMG_CUDA(cudaStreamSynchronize(h->stream));
        const int64_t iters = std::max(0, h->st_out->it - it0);
        return g.init_launches + iters * g.body_launches + g.post_launches;
    }
    Issue local;
    Issue& I = prof ? *prof : local;
    I.s = h->stream;
    ++h->last_host_attempts;
    const int64_t l0 = I.launches;
    Reduce b = base_reduce(h);
    AMG_CUDA(cudaMemcpyAsync(h->st, h->st_in, sizeof(KState), cudaMemcpyHostToDevice, h->stream));
    issue_init(h, I, f, x, b);
    AMG_CUDA(cudaMemcpyAsync(h->st_out, h->st, sizeof(KState), cudaMemcpyDeviceToHost, h->stream));
    AMG_CUDA(cudaStreamSynchronize(h->stream));
    int guard = 0;
    while (h->st_out->cond && guard++ <= h->st_in->maxiter + 1) {
        issue_body(h, I, x, b);
        AMG_CUDA(cudaMemcpyAsync(h->st_out, h->st, sizeof(KState), cudaMemcpyDeviceToHost, h->stream));
        AMG_CUDA(cudaStreamSynchronize(h->stream));
    }
    issue_post(h, I, f, x, b);
    AMG_CUDA(cudaMemcpyAsync(h->st_out, h->st, sizeof(KState), cudaMemcpyDeviceToHost, h->stream));
    enqueue_dev_err_copy(h->err_host, h->stream);
    AMG_CUDA(cudaStreamSynchronize(h->stream));
    return I.launches - l0;
}

amg_status run_solve(amg_handle* h, const double* f, double* x, double rtol, int maxiter,
                     int* iters, double* relres, Issue* prof) {
    if (!f || !x) fail(AMG_ERR_INVALID_ARG, "f and x must be device pointers");
    if (!(rtol >= 0.0) || maxiter < 0) fail(AMG_ERR_INVALID_ARG, "rtol must be >= 0 and maxiter >= 0");
    if (f == x) fail(AMG_ERR_INVALID_ARG, "f and x must be distinct buffers");
    std::memset(h->st_in, 0, sizeof(KState));
    h->st_in->rtol = rtol;
    h->st_in->maxiter = maxiter;
    bool use_graph = h->prm.use_graph && !h->graph_unsupported && !prof;
    int64_t launches = 0;
    h->last_graph_attempts = h->last_host_attempts = 0;
    amg_status status = AMG_OK;
    for (int attempt_no = 0; attempt_no < 64; ++attempt_no) {
        *h->err_host = 0;
        launches += attempt(h, f, x, use_graph && !h->graph_unsupported, prof);
        if (*h->err_host) {
            read_and_clear_dev_err();
            fail(AMG_ERR_CUDA, "a device pipeline wait timed out; results are invalid");
        }
        const KState& o = *h->st_out;
        if (!std::isfinite(o.nf) || !std::isfinite(o.relres)) {
            // nothing to iterate on: non-finite data in f or in the initial guess
            if (iters) *iters = o.it;
            if (relres) *relres = o.relres;
            h->last_launches = launches;
            if (o.it == 0) fail(AMG_ERR_INVALID_ARG, "f or the initial guess contains non-finite values");
            return AMG_ERR_BREAKDOWN;
        }
        if (o.zero_rhs) {
            AMG_CUDA(cudaMemsetAsync(x, 0, h->n * sizeof(double), h->stream));
            AMG_CUDA(cudaStreamSynchronize(h->stream));
            if (iters) *iters = 0;
            if (relres) *relres = 0.0;
            h->last_launches = launches;
            return AMG_OK;
        }
        if (o.status == AMG_ERR_BREAKDOWN) { status = AMG_ERR_BREAKDOWN; break; }
        if (o.relres <= rtol) { status = AMG_OK; break; }
        if (o.it >= maxiter) { status = AMG_ERR_NOT_CONVERGED; break; }
        // the recurrence met rtol but the true residual did not: restart
        h->st_in->it = o.it;
        status = AMG_ERR_NOT_CONVERGED;
    }
    if (iters) *iters = h->st_out->it;
    if (relres) *relres = h->st_out->relres;
    h->last_launches = launches;
    return status;
}

void run_vcycle(amg_handle* h, const double* r, double* z) {
    Issue I;
    I.s = h->stream;
    // the V-cycle streams row slices of its input: take it from a padded buffer
    AMG_CUDA(cudaMemcpyAsync(h->r, r, h->n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    issue_vcycle(h, I, h->r, nullptr, z, nullptr, nullptr);
    AMG_CUDA(cudaStreamSynchronize(h->stream));
}

}  // namespace amg
