// capi.cu -- the extern "C" entry points of include/amg.h.  Every entry
// point catches internal errors and returns a status; the message of the
// last failure is kept per thread.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <string>

#include "amg_internal.h"
#include "batch.h"
#include "handle.h"
#include "host_parallel.h"

namespace amg {

static thread_local std::string g_last_error;

// the calling thread's message of amg_last_error (the server reports its
// requests' errors to the thread that waits for them)
void set_last_error(const std::string& msg) { g_last_error = msg; }

void fail(amg_status st, const std::string& msg) { throw Error{st, msg}; }

void cuda_check(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return;
    cudaGetLastError();  // clear a non-sticky error
    const amg_status st = (e == cudaErrorMemoryAllocation) ? AMG_ERR_OOM : AMG_ERR_CUDA;
    fail(st, std::string(what) + ": " + cudaGetErrorString(e));
}

template <typename T>
T* dev_alloc(size_t count) {
    void* p = nullptr;
    const cudaError_t e = cudaMalloc(&p, count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        fail(e == cudaErrorMemoryAllocation ? AMG_ERR_OOM : AMG_ERR_CUDA,
             "cudaMalloc of " + std::to_string(count * sizeof(T)) + " bytes: " + cudaGetErrorString(e));
    }
    return static_cast<T*>(p);
}
template int32_t* dev_alloc<int32_t>(size_t);
template double* dev_alloc<double>(size_t);
template float* dev_alloc<float>(size_t);
template uint16_t* dev_alloc<uint16_t>(size_t);
template unsigned int* dev_alloc<unsigned int>(size_t);
template KState* dev_alloc<KState>(size_t);
template TailPhase* dev_alloc<TailPhase>(size_t);
template unsigned char* dev_alloc<unsigned char>(size_t);
template int64_t* dev_alloc<int64_t>(size_t);
template BSys* dev_alloc<BSys>(size_t);
template BResult* dev_alloc<BResult>(size_t);

void dev_free(void* p) {
    if (p) cudaFree(p);
}

void* dev_alloc_async_bytes(size_t bytes, cudaStream_t s) {
    void* p = nullptr;
    const cudaError_t e = cudaMallocAsync(&p, bytes > 0 ? bytes : 1, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        fail(e == cudaErrorMemoryAllocation ? AMG_ERR_OOM : AMG_ERR_CUDA,
             "cudaMallocAsync of " + std::to_string(bytes) + " bytes: " + cudaGetErrorString(e));
    }
    return p;
}

void dev_free_async(void* p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

void build_hierarchy(amg_handle* h, HostCsr A);
amg_status spmv_dot_noalloc(const amg_csr* A, const double* x, double* y, double* dot, void* stream);
void build_batch(amg_batch* b, const amg_csr* systems);

static void free_batch(amg_batch* b) {
    if (!b) return;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (void* p : b->allocs) cudaFree(p);
    if (b->res_host) cudaFreeHost(b->res_host);
    delete b;
}

// Run the batch with the current schedule; fills res_host.  Returns the
// worst status over the systems.
static amg_status run_batch(amg_batch* b, const double* f, double* x, double rtol, int maxiter) {
    launch_batch_cg(b->sys, b->order_mode == 0 ? b->order_by_size : b->order_input, b->nsys, b->row_off_dev,
                    b->queue, f, x, rtol, maxiter, b->prm.precision == AMG_PRECISION_FP32, b->res,
                    b->threads, b->ctas_per_sm, b->stream);
    AMG_CUDA(cudaMemcpyAsync(b->res_host, b->res, b->nsys * sizeof(BResult), cudaMemcpyDeviceToHost, b->stream));
    AMG_CUDA(cudaStreamSynchronize(b->stream));
    int worst = AMG_OK;
    for (int k = 0; k < b->nsys; ++k) {
        const int st = b->res_host[k].status;
        if (st == AMG_ERR_INVALID_ARG) worst = AMG_ERR_INVALID_ARG;
        else if (st == AMG_ERR_BREAKDOWN && worst != AMG_ERR_INVALID_ARG) worst = AMG_ERR_BREAKDOWN;
        else if (st == AMG_ERR_NOT_CONVERGED && worst == AMG_OK) worst = AMG_ERR_NOT_CONVERGED;
    }
    return (amg_status)worst;
}
amg_status run_solve(amg_handle* h, const double* f, double* x, double rtol, int maxiter,
                     int* iters, double* relres, Issue* prof);
void run_vcycle(amg_handle* h, const double* r, double* z);
void destroy_graphs(amg_handle* h);

template <typename F>
static amg_status guarded(F&& body) {
    try {
        g_last_error.clear();
        return body();
    } catch (const Error& e) {
        g_last_error = e.msg;
        return e.status;
    } catch (const std::bad_alloc&) {
        g_last_error = "host allocation failed";
        return AMG_ERR_OOM;
    } catch (const std::exception& e) {
        g_last_error = e.what();
        return AMG_ERR_INVALID_ARG;
    }
}

static void free_handle(amg_handle* h) {
    if (!h) return;
    cudaSetDevice(h->device);
    cudaStreamSynchronize(h->stream);
    destroy_graphs(h);
    for (void* p : h->dev_allocs) cudaFreeAsync(p, h->stream);  // no device-wide synchronisation
    cudaStreamSynchronize(h->stream);
    if (h->st_in) cudaFreeHost(h->st_in);
    if (h->st_out) cudaFreeHost(h->st_out);
    if (h->err_host) cudaFreeHost(h->err_host);
    if (h->cap) cudaStreamDestroy(h->cap);
    if (h->cap2) cudaStreamDestroy(h->cap2);
    for (cudaEvent_t e : h->event_pool) cudaEventDestroy(e);
    delete h;
}

static void check_params(const amg_params& p) {
    if (!(p.strength_eps >= 0.0)) fail(AMG_ERR_INVALID_ARG, "strength_eps must be >= 0");
    if (p.smoother != AMG_SMOOTHER_JACOBI && p.smoother != AMG_SMOOTHER_SPAI0)
        fail(AMG_ERR_INVALID_ARG, "unknown smoother");
    if (p.npre < 0 || p.npre > 16 || p.npost < 0 || p.npost > 16)
        fail(AMG_ERR_INVALID_ARG, "npre and npost must be in [0, 16]");
    if (p.coarse_enough < 1) fail(AMG_ERR_INVALID_ARG, "coarse_enough must be >= 1");
    if (p.max_levels < 1 || p.max_levels > AMG_MAX_LEVELS)
        fail(AMG_ERR_INVALID_ARG, "max_levels must be in [1, AMG_MAX_LEVELS]");
    if (p.max_coarse_dense < 1 || p.max_coarse_dense > 16384)
        fail(AMG_ERR_INVALID_ARG, "max_coarse_dense must be in [1, 16384]");
    if (p.solver != AMG_SOLVER_CG && p.solver != AMG_SOLVER_BICGSTAB)
        fail(AMG_ERR_INVALID_ARG, "unknown solver");
    if (p.precision != AMG_PRECISION_FP64 && p.precision != AMG_PRECISION_FP32 &&
        p.precision != AMG_PRECISION_BF16)
        fail(AMG_ERR_INVALID_ARG, "unknown precision");
    if (p.precision != AMG_PRECISION_FP64 && (p.npre != 1 || p.npost != 1))
        fail(AMG_ERR_INVALID_ARG, "the float32 V-cycle supports npre = npost = 1");
}

static const amg::Level& level_of(const amg_handle* h, int level) {
    if (!h) fail(AMG_ERR_INVALID_ARG, "null handle");
    if (level < 0 || level >= (int)h->lev.size()) fail(AMG_ERR_INVALID_ARG, "level out of range");
    return h->lev[level];
}

}  // namespace amg

using namespace amg;

extern "C" {

amg_status amg_params_default(amg_params* p) {
    if (!p) return AMG_ERR_INVALID_ARG;
    std::memset(p, 0, sizeof(*p));
    p->strength_eps = 0.08;
    p->strength_halving = 1;
    p->smoother = AMG_SMOOTHER_JACOBI;
    p->jacobi_omega = 0.72;
    p->npre = 1;
    p->npost = 1;
    p->coarse_enough = 500;
    p->max_levels = 25;
    p->max_coarse_dense = 4096;
    p->solver = AMG_SOLVER_CG;
    p->precision = AMG_PRECISION_FP64;
    p->use_graph = 1;
    p->use_stream = 1;
    p->use_pdl = 0;
    p->use_tail = 0;
    p->device_setup = 1;
    p->fused_restriction = 1;
    return AMG_OK;
}

const char* amg_last_error(void) { return g_last_error.c_str(); }

amg_status amg_setup(const amg_csr* A, const amg_params* prm, void* stream, amg_handle** out) {
    return guarded([&]() -> amg_status {
        if (!out) fail(AMG_ERR_INVALID_ARG, "out is null");
        *out = nullptr;
        if (!A || !A->row_ptr || !A->col || !A->val) fail(AMG_ERR_INVALID_ARG, "null matrix");
        if (A->n < 1) fail(AMG_ERR_INVALID_ARG, "n must be >= 1");
        if (A->n >= (1LL << 31) - 1 || A->nnz < 0 || A->nnz >= (1LL << 31) - 1)
            fail(AMG_ERR_TOO_LARGE, "n and nnz must be below 2^31");
        amg_params p;
        if (prm) p = *prm;
        else amg_params_default(&p);
        check_params(p);
        HostCsr H;
        H.nrows = H.ncols = A->n;
        H.ptr.resize(A->n + 1);
        auto fetch = [&](void* dst, const void* src, size_t bytes) {
            if (A->on_device) {
                AMG_CUDA(cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost));
                return;
            }
            // host input: copied in parallel chunks (a large matrix is
            // hundreds of MB)
            const int64_t C = row_chunks((int64_t)(bytes / 8), (int64_t)(bytes / 8));
            parallel_for(C, [&](int64_t c) {
                const size_t lo = bytes * c / C, hi = bytes * (c + 1) / C;
                std::memcpy(static_cast<char*>(dst) + lo, static_cast<const char*>(src) + lo, hi - lo);
            });
        };
        fetch(H.ptr.data(), A->row_ptr, (A->n + 1) * sizeof(int32_t));
        if (H.ptr[A->n] != A->nnz) fail(AMG_ERR_INVALID_ARG, "row_ptr[n] != nnz");
        H.col.resize(A->nnz);
        H.val.resize(A->nnz);
        fetch(H.col.data(), A->col, A->nnz * sizeof(int32_t));
        fetch(H.val.data(), A->val, A->nnz * sizeof(double));
        host_validate(H);

        amg_handle* h = new amg_handle();
        try {
            h->prm = p;
            h->stream = static_cast<cudaStream_t>(stream);
            AMG_CUDA(cudaGetDevice(&h->device));
            h->n = A->n;
            AMG_CUDA(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
            AMG_CUDA(cudaStreamCreateWithFlags(&h->cap2, cudaStreamNonBlocking));
            build_hierarchy(h, std::move(H));
            auto vec = [&](double*& v) {  // padded: see kPad
                v = dev_alloc_async<double>(h->n + kPad, h->stream);
                h->dev_allocs.push_back(v);
                h->dev_bytes += (h->n + kPad) * 8;
                AMG_CUDA(cudaMemsetAsync(v, 0, (h->n + kPad) * sizeof(double), h->stream));
            };
            for (double** v : {&h->r, &h->z, &h->p, &h->q, &h->rh, &h->v, &h->ph, &h->sv, &h->sh,
                               &h->tv, &h->fbuf, &h->xbuf})
                vec(*v);
            if (h->prm.precision != AMG_PRECISION_FP64 && h->lev.size() > 1) {
                h->vin32 = dev_alloc_async<float>(h->n + kPad, h->stream);
                h->dev_allocs.push_back(h->vin32);
                h->dev_bytes += (h->n + kPad) * 4;
                AMG_CUDA(cudaMemsetAsync(h->vin32, 0, (h->n + kPad) * sizeof(float), h->stream));
            }
            h->st = dev_alloc_async<KState>(1, h->stream);
            h->dev_allocs.push_back(h->st);
            AMG_CUDA(cudaMemsetAsync(h->st, 0, sizeof(KState), h->stream));
            AMG_CUDA(cudaMallocHost(&h->st_in, sizeof(KState)));
            AMG_CUDA(cudaMallocHost(&h->st_out, sizeof(KState)));
            AMG_CUDA(cudaMallocHost(&h->err_host, sizeof(int)));
            *h->err_host = 0;
            std::memset(h->st_in, 0, sizeof(KState));
            std::memset(h->st_out, 0, sizeof(KState));
            h->stride = std::max(std::max<int>(h->lev[0].A.nblk, vec_grid(h->n)),
                                 stream_grid(std::max(1, h->lev[0].A.ntiles), kStreamCtasMax));
            h->dev_bytes += 2 * (int64_t)h->stride * 8 + 512;
            h->partial = dev_alloc_async<double>(2 * (size_t)h->stride, h->stream);
            h->dev_allocs.push_back(h->partial);
            h->counter = dev_alloc_async<unsigned int>(1, h->stream);
            h->dev_allocs.push_back(h->counter);
            AMG_CUDA(cudaMemsetAsync(h->counter, 0, sizeof(unsigned int), h->stream));
            // the set-up's own work only: other streams may be solving meanwhile
            AMG_CUDA(cudaStreamSynchronize(h->stream));
            AMG_CUDA(cudaStreamSynchronize(nullptr));
        } catch (...) {
            free_handle(h);
            throw;
        }
        *out = h;
        return AMG_OK;
    });
}

amg_status amg_free(amg_handle* h) {
    return guarded([&]() -> amg_status {
        free_handle(h);
        return AMG_OK;
    });
}

amg_status amg_solve(amg_handle* h, const double* f, double* x, double rtol, int maxiter,
                     int* iters, double* relres) {
    return guarded([&]() -> amg_status {
        if (!h) fail(AMG_ERR_INVALID_ARG, "null handle");
        AMG_CUDA(cudaSetDevice(h->device));
        set_stream_options(h->prm.use_pdl != 0);
        return run_solve(h, f, x, rtol, maxiter, iters, relres, nullptr);
    });
}

amg_status amg_solve_host(amg_handle* h, const double* f_host, double* x_host, double rtol,
                          int maxiter, int* iters, double* relres) {
    return guarded([&]() -> amg_status {
        if (!h || !f_host || !x_host) fail(AMG_ERR_INVALID_ARG, "null argument");
        AMG_CUDA(cudaSetDevice(h->device));
        set_stream_options(h->prm.use_pdl != 0);
        const size_t bytes = h->n * sizeof(double);
        AMG_CUDA(cudaMemcpyAsync(h->fbuf, f_host, bytes, cudaMemcpyHostToDevice, h->stream));
        AMG_CUDA(cudaMemcpyAsync(h->xbuf, x_host, bytes, cudaMemcpyHostToDevice, h->stream));
        amg_status st = run_solve(h, h->fbuf, h->xbuf, rtol, maxiter, iters, relres, nullptr);
        AMG_CUDA(cudaMemcpyAsync(x_host, h->xbuf, bytes, cudaMemcpyDeviceToHost, h->stream));
        AMG_CUDA(cudaStreamSynchronize(h->stream));
        return st;
    });
}

amg_status amg_solve_profile(amg_handle* h, const double* f, double* x, double rtol, int maxiter,
                             int* iters, double* relres, double* ms, int* launches) {
    return guarded([&]() -> amg_status {
        if (!h) fail(AMG_ERR_INVALID_ARG, "null handle");
        AMG_CUDA(cudaSetDevice(h->device));
        set_stream_options(h->prm.use_pdl != 0);
        std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> events;
        Issue I;
        I.s = h->stream;
        I.profile = true;
        I.events = &events;
        I.pool = &h->event_pool;
        amg_status st = run_solve(h, f, x, rtol, maxiter, iters, relres, &I);
        AMG_CUDA(cudaStreamSynchronize(h->stream));
        double acc[AMG_KC_COUNT] = {0};
        int cnt[AMG_KC_COUNT] = {0};
        for (auto& e : events) {
            float t = 0.f;
            AMG_CUDA(cudaEventElapsedTime(&t, e.second.first, e.second.second));
            acc[e.first] += t;
            cnt[e.first] += 1;
        }
        for (int k = 0; k < AMG_KC_COUNT; ++k) {
            if (ms) ms[k] = acc[k];
            if (launches) launches[k] = cnt[k];
        }
        return st;
    });
}

amg_status amg_check_wait_limit(double* seconds) {
    return guarded([&]() -> amg_status {
        const int err = check_wait_limit(seconds);
        if (err & 4) fail(AMG_ERR_CUDA, "a device pipeline wait timed out (bounded-wait check)");
        fail(AMG_ERR_CUDA, "the bounded-wait check kernel did not record its timeout");
    });
}

amg_status amg_last_launch_count(const amg_handle* h, int64_t* launches) {
    if (!h || !launches) return AMG_ERR_INVALID_ARG;
    *launches = h->last_launches;
    return AMG_OK;
}

amg_status amg_last_solve_mode(const amg_handle* h, int* graph_attempts, int* host_attempts) {
    if (!h) return AMG_ERR_INVALID_ARG;
    if (graph_attempts) *graph_attempts = h->last_graph_attempts;
    if (host_attempts) *host_attempts = h->last_host_attempts;
    return AMG_OK;
}

amg_status amg_hierarchy_info(const amg_handle* h, int* levels, int64_t* rows, int64_t* nnz_a,
                              int64_t* nnz_p) {
    return guarded([&]() -> amg_status {
        if (!h) fail(AMG_ERR_INVALID_ARG, "null handle");
        if (levels) *levels = (int)h->lev.size();
        for (size_t l = 0; l < h->lev.size(); ++l) {
            if (rows) rows[l] = h->lev[l].A.nrows;
            if (nnz_a) nnz_a[l] = h->lev[l].A.nnz;
            if (nnz_p) nnz_p[l] = (l + 1 < h->lev.size()) ? h->lev[l].P.nnz : 0;
        }
        return AMG_OK;
    });
}

amg_status amg_fused_restriction_nnz(const amg_handle* h, int level, int64_t* nnz) {
    return guarded([&]() -> amg_status {
        const Level& L = level_of(h, level);
        if (!nnz) fail(AMG_ERR_INVALID_ARG, "null output");
        *nnz = L.M.nrows > 0 ? L.M.nnz : 0;
        return AMG_OK;
    });
}

amg_status amg_hierarchy_bytes(const amg_handle* h, double* bytes_per_iteration) {
    return guarded([&]() -> amg_status {
        if (!h || !bytes_per_iteration) fail(AMG_ERR_INVALID_ARG, "null argument");
        std::vector<LevelSizes> sz(h->lev.size());
        for (size_t l = 0; l < h->lev.size(); ++l)
            sz[l] = {h->lev[l].A.nrows, h->lev[l].A.nnz, l + 1 < h->lev.size() ? h->lev[l].P.nnz : 0,
                     h->lev[l].M.nrows > 0 ? h->lev[l].M.nnz : 0};
        *bytes_per_iteration = krylov_iteration_bytes(sz, h->prm.precision, h->prm.solver, true);
        return AMG_OK;
    });
}

amg_status amg_get_level_matrix(const amg_handle* h, int level, int which, int32_t* row_ptr,
                                int32_t* col, double* val) {
    return guarded([&]() -> amg_status {
        const Level& L = level_of(h, level);
        if (which < 0 || which > 3) fail(AMG_ERR_INVALID_ARG, "which must be 0 (A), 1 (P), 2 (R) or 3 (M)");
        if (which > 0 && level + 1 >= (int)h->lev.size())
            fail(AMG_ERR_INVALID_ARG, "the coarsest level has no P, R or M");
        if (which == 3 && L.M.nrows == 0) fail(AMG_ERR_INVALID_ARG, "this level has no fused restriction operator");
        if (!row_ptr || !col || !val) fail(AMG_ERR_INVALID_ARG, "null output");
        AMG_CUDA(cudaSetDevice(h->device));
        const DevCsr& D = which == 0 ? L.A : which == 1 ? L.P : which == 2 ? L.R : L.M;
        AMG_CUDA(cudaMemcpy(row_ptr, D.ptr, (D.nrows + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost));
        AMG_CUDA(cudaMemcpy(col, D.col, D.nnz * sizeof(int32_t), cudaMemcpyDeviceToHost));
        AMG_CUDA(cudaMemcpy(val, D.val, D.nnz * sizeof(double), cudaMemcpyDeviceToHost));
        return AMG_OK;
    });
}

amg_status amg_get_aggregates(const amg_handle* h, int level, int32_t* agg) {
    return guarded([&]() -> amg_status {
        const Level& L = level_of(h, level);
        if (level + 1 >= (int)h->lev.size()) fail(AMG_ERR_INVALID_ARG, "the coarsest level has no aggregates");
        if (!agg) fail(AMG_ERR_INVALID_ARG, "null output");
        if (L.agg_dev) {
            AMG_CUDA(cudaMemcpyAsync(agg, L.agg_dev, L.A.nrows * sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
            AMG_CUDA(cudaStreamSynchronize(h->stream));
        } else {
            std::memcpy(agg, L.agg.data(), L.agg.size() * sizeof(int32_t));
        }
        return AMG_OK;
    });
}

amg_status amg_get_smoother_diag(const amg_handle* h, int level, double* d) {
    return guarded([&]() -> amg_status {
        const Level& L = level_of(h, level);
        if (!d) fail(AMG_ERR_INVALID_ARG, "null output");
        if (L.dhost.empty()) {
            AMG_CUDA(cudaMemcpyAsync(d, L.d, L.A.nrows * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
            AMG_CUDA(cudaStreamSynchronize(h->stream));
        } else {
            std::memcpy(d, L.dhost.data(), L.dhost.size() * sizeof(double));
        }
        return AMG_OK;
    });
}

amg_status amg_apply_precond(amg_handle* h, const double* r, double* z) {
    return guarded([&]() -> amg_status {
        if (!h || !r || !z || r == z) fail(AMG_ERR_INVALID_ARG, "bad arguments");
        AMG_CUDA(cudaSetDevice(h->device));
        set_stream_options(h->prm.use_pdl != 0);
        run_vcycle(h, r, z);
        return AMG_OK;
    });
}

amg_status amg_level_spmv(amg_handle* h, int level, int which, const double* x, double* y) {
    return guarded([&]() -> amg_status {
        const Level& L = level_of(h, level);
        if (which < 0 || which > 2) fail(AMG_ERR_INVALID_ARG, "which must be 0 (A), 1 (P) or 2 (R)");
        if (which > 0 && level + 1 >= (int)h->lev.size())
            fail(AMG_ERR_INVALID_ARG, "the coarsest level has no P or R");
        if (!x || !y || x == y) fail(AMG_ERR_INVALID_ARG, "bad vectors");
        AMG_CUDA(cudaSetDevice(h->device));
        const DevCsr& D = which == 0 ? L.A : which == 1 ? L.P : L.R;
        set_stream_options(h->prm.use_pdl != 0);
        launch_spmv(D, x, y, nullptr, h->stream);
        AMG_CUDA(cudaStreamSynchronize(h->stream));
        return AMG_OK;
    });
}

amg_status amg_spmv_dot(const amg_csr* A, const double* x, double* y, double* dot, void* stream) {
    return guarded([&]() -> amg_status {
        if (!A || !A->on_device || !A->row_ptr || !A->col || !A->val || !x || !y || !dot || x == y)
            fail(AMG_ERR_INVALID_ARG, "bad arguments (the matrix must be on the device)");
        if (A->n < 1 || A->n >= (1LL << 31) - 1 || A->nnz < 0 || A->nnz >= (1LL << 31) - 1)
            fail(AMG_ERR_INVALID_ARG, "n must be in [1, 2^31) and nnz in [0, 2^31)");
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        const int32_t n = (int32_t)A->n;
        const double avg = (double)A->nnz / (double)n;
        int rpb = kRowsPerBlock;
        while (rpb > 1 && rpb * avg > kTileNnz) rpb >>= 1;
        const int nb = (int)((n + rpb - 1) / rpb);
        // scratch: two arrays of nb partial sums, the block counter, the error word
        const size_t bytes = 2 * (size_t)nb * sizeof(double) + 2 * sizeof(unsigned int);
        void* scratch = nullptr;
        AMG_CUDA(cudaMallocAsync(&scratch, bytes, s));
        amg_status result = AMG_OK;
        try {
            double* partial = static_cast<double*>(scratch);
            unsigned int* counter = reinterpret_cast<unsigned int*>(partial + 2 * (size_t)nb);
            int* err = reinterpret_cast<int*>(counter + 1);
            AMG_CUDA(cudaMemsetAsync(counter, 0, 2 * sizeof(unsigned int), s));
            launch_validate_csr(n, A->nnz, A->row_ptr, err, s);
            int herr = 0;
            AMG_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
            AMG_CUDA(cudaStreamSynchronize(s));
            if (herr) fail(AMG_ERR_INVALID_ARG, "row_ptr is not a valid CSR row pointer");
            Reduce red;
            red.partial = partial;
            red.stride = nb;
            red.counter = counter;
            red.out = dot;
            red.fin = FIN_NONE;
            launch_spmv_dot_uniform(n, n, A->row_ptr, A->col, A->val, x, y, rpb, red, err, s);
            AMG_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
            AMG_CUDA(cudaStreamSynchronize(s));
            if (herr) fail(AMG_ERR_INVALID_ARG, "column index out of range");
        } catch (const Error& e) {
            cudaFreeAsync(scratch, s);
            throw;
        }
        AMG_CUDA(cudaFreeAsync(scratch, s));
        AMG_CUDA(cudaStreamSynchronize(s));
        return result;
    });
}

amg_status amg_batch_setup(int nsys, const amg_csr* systems, const amg_params* prm, void* stream,
                           amg_batch** out) {
    return guarded([&]() -> amg_status {
        if (!out) fail(AMG_ERR_INVALID_ARG, "out is null");
        *out = nullptr;
        if (nsys < 1 || !systems) fail(AMG_ERR_INVALID_ARG, "nsys must be >= 1 and systems non-null");
        amg_params p;
        if (prm) p = *prm;
        else amg_params_default(&p);
        check_params(p);
        if (p.npre != 1 || p.npost != 1 || p.solver != AMG_SOLVER_CG)
            fail(AMG_ERR_INVALID_ARG, "the batched solve supports CG with one pre- and one post-sweep");
        if (p.precision == AMG_PRECISION_BF16)
            fail(AMG_ERR_INVALID_ARG, "the batched solve supports the FP64 and FP32 V-cycles");
        amg_batch* b = new amg_batch();
        try {
            b->prm = p;
            b->nsys = nsys;
            b->stream = static_cast<cudaStream_t>(stream);
            AMG_CUDA(cudaGetDevice(&b->device));
            build_batch(b, systems);
        } catch (...) {
            free_batch(b);
            throw;
        }
        *out = b;
        return AMG_OK;
    });
}

amg_status amg_batch_solve(amg_batch* b, const double* f, double* x, double rtol, int maxiter, int* iters,
                           double* relres, int* status) {
    return guarded([&]() -> amg_status {
        if (!b || !f || !x || f == x) fail(AMG_ERR_INVALID_ARG, "bad arguments");
        if (!(rtol >= 0.0) || maxiter < 0) fail(AMG_ERR_INVALID_ARG, "rtol must be >= 0 and maxiter >= 0");
        AMG_CUDA(cudaSetDevice(b->device));
        const amg_status st = run_batch(b, f, x, rtol, maxiter);
        for (int k = 0; k < b->nsys; ++k) {
            if (iters) iters[k] = b->res_host[k].iters;
            if (relres) relres[k] = b->res_host[k].relres;
            if (status) status[k] = b->res_host[k].status;
        }
        return st;
    });
}

amg_status amg_batch_tune(amg_batch* b, const double* f, double* x, double rtol, int maxiter, int* threads,
                          int* ctas_per_sm) {
    return guarded([&]() -> amg_status {
        if (!b || !f || !x || f == x) fail(AMG_ERR_INVALID_ARG, "bad arguments");
        AMG_CUDA(cudaSetDevice(b->device));
        const int cand[][2] = {{128, 4}, {256, 2}, {256, 4}, {512, 1}, {512, 2}, {1024, 1}};
        cudaEvent_t e0, e1;
        AMG_CUDA(cudaEventCreate(&e0));
        AMG_CUDA(cudaEventCreate(&e1));
        float best = 1e30f;
        int bt = b->threads, bc = b->ctas_per_sm, bo = b->order_mode;
        try {
            const int maxt = batch_max_threads(b->prm.precision == AMG_PRECISION_FP32);
            for (int order = 0; order < 2; ++order)
                for (const auto& c : cand) {
                    if (c[0] > maxt) continue;
                    b->threads = c[0];
                    b->ctas_per_sm = c[1];
                    b->order_mode = order;
                    AMG_CUDA(cudaMemsetAsync(x, 0, b->total_rows * sizeof(double), b->stream));
                    AMG_CUDA(cudaEventRecord(e0, b->stream));
                    run_batch(b, f, x, rtol, maxiter);
                    AMG_CUDA(cudaEventRecord(e1, b->stream));
                    AMG_CUDA(cudaEventSynchronize(e1));
                    float ms = 0.f;
                    AMG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                    if (ms < best) { best = ms; bt = c[0]; bc = c[1]; bo = order; }
                }
        } catch (...) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            throw;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        b->threads = bt;
        b->ctas_per_sm = bc;
        b->order_mode = bo;
        b->tuned = 1;
        if (threads) *threads = bt;
        if (ctas_per_sm) *ctas_per_sm = bc;
        AMG_CUDA(cudaMemsetAsync(x, 0, b->total_rows * sizeof(double), b->stream));
        run_batch(b, f, x, rtol, maxiter);  // leave x solved with the chosen schedule
        return AMG_OK;
    });
}

amg_status amg_batch_info(const amg_batch* b, int64_t* total_rows, int64_t* row_off, int* levels) {
    return guarded([&]() -> amg_status {
        if (!b) fail(AMG_ERR_INVALID_ARG, "null batch");
        if (total_rows) *total_rows = b->total_rows;
        for (int k = 0; k <= b->nsys; ++k) {
            if (row_off) row_off[k] = b->row_off[k];
            if (levels && k < b->nsys) levels[k] = b->levels[k];
        }
        return AMG_OK;
    });
}

amg_status amg_batch_bytes(const amg_batch* b, double* bytes_per_iteration) {
    return guarded([&]() -> amg_status {
        if (!b || !bytes_per_iteration) fail(AMG_ERR_INVALID_ARG, "null argument");
        for (int k = 0; k < b->nsys; ++k) bytes_per_iteration[k] = b->iter_bytes[k];
        return AMG_OK;
    });
}

amg_status amg_batch_free(amg_batch* b) {
    return guarded([&]() -> amg_status {
        free_batch(b);
        return AMG_OK;
    });
}

amg_status amg_spmv_dot_noalloc(const amg_csr* A, const double* x, double* y, double* dot,
                                void* stream) {
    return guarded([&]() -> amg_status { return spmv_dot_noalloc(A, x, y, dot, stream); });
}

}  // extern "C"
