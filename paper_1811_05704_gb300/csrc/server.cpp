// server.cpp -- a solve server with continuous batching.
//
// The paper notes that the setup depends only on the matrix, so a hierarchy
// can serve many right-hand sides (Sec. 3, design principles).  The server
// keeps hierarchies resident on the device under caller-chosen keys and
// serves a stream of requests, each a new matrix with a right-hand side or a
// key of a resident hierarchy with a new right-hand side.  Requests wait in a
// FIFO queue; whenever a slot is free, a worker admits the first queued
// request (looking a few entries ahead) whose device memory fits the HBM
// budget, evicting idle resident hierarchies (least recently used) to make
// room.  Each slot is a host thread with its own CUDA stream, so the set-ups
// and solves of the admitted requests run concurrently and their kernels
// overlap on the GPU; a request that arrives while others run is admitted as
// soon as a slot and the memory free up.  Every solve is deterministic (fixed
// launch shapes, fixed-order reductions), so a result is the same alone and
// in the mix.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>

#include "amg_internal.h"
#include "handle.h"
#include "host_parallel.h"

namespace amg {

namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
    int64_t id = 0;
    int64_t key = -1;
    bool has_matrix = false;
    HostCsr A;
    std::vector<double> f, x;
    amg_params prm{};  // set-up and solver parameters of a new hierarchy
    double rtol = 1e-8;
    int maxiter = 500;
    int64_t estimate = 0;  // device bytes if a hierarchy must be built
    // results
    int iters = 0;
    double relres = 0.0;
    amg_status status = AMG_OK;
    std::string error;
    double t_submit = 0.0, t_admit = 0.0, t_done = 0.0;
    bool done = false;
};

}  // namespace

void set_last_error(const std::string& msg);

namespace {

struct Resident {
    amg_handle* h = nullptr;
    int64_t bytes = 0;
    bool busy = false;
    double last_used = 0.0;
};

}  // namespace

}  // namespace amg

struct amg_server {
    amg_server_params sp{};
    amg_params prm{};
    int device = 0;
    std::mutex m;
    std::condition_variable cv_work;   // queue changed, slot or memory freed
    std::condition_variable cv_done;   // a request finished
    std::deque<amg::Request*> queue;
    std::map<int64_t, std::unique_ptr<amg::Request>> requests;
    std::map<int64_t, amg::Resident> resident;
    std::vector<int64_t> building;     // keys whose hierarchy a worker is building
    int64_t next_id = 1;
    int64_t in_use = 0;        // bytes charged: resident hierarchies + hierarchies being built
    int64_t peak = 0;
    int64_t completed = 0;
    int64_t evictions = 0;
    double solve_bytes = 0.0;  // algorithmic bytes of the finished solves
    int running = 0;
    std::atomic<int> setups{0};  // set-ups running now (their host steps share the cores)
    bool stop = false;
    std::vector<std::thread> workers;
};

namespace amg {

namespace {

constexpr int kLookahead = 16;

// Device bytes a new hierarchy of this matrix will hold (measured about 64
// bytes per nonzero on 3D stencils with every level, the smoother-scaled
// values and the Krylov vectors), plus the coarsest inverse.
int64_t estimate_bytes(const HostCsr& A) { return 72 * A.nnz() + 64 * A.nrows + (8 << 20); }

void finish_locked(amg_server* s, Request* r, amg_status st, const std::string& err) {
    r->status = st;
    r->error = err;
    r->done = true;
    r->t_done = now_s();
    s->completed++;
    s->cv_done.notify_all();
}

// Under the lock: pick the next admissible request.  Requests that reuse a
// resident hierarchy need no memory and may pass others; requests that need
// a new hierarchy are admitted in arrival order (once one does not fit, none
// behind it is built before it), so a large matrix is not starved by small
// ones.  Evicted hierarchies go to `evict` and are freed by the caller after
// unlocking.
Request* pick(amg_server* s, bool& reuse, amg_handle*& h, std::vector<amg_handle*>& evict) {
    int look = std::min<int>(kLookahead, (int)s->queue.size());
    bool blocked = false;
    for (int i = 0; i < look; ++i) {
        Request* r = s->queue[i];
        auto it = (r->key >= 0) ? s->resident.find(r->key) : s->resident.end();
        if (it != s->resident.end()) {
            if (it->second.busy) continue;  // one solve at a time per hierarchy
            it->second.busy = true;
            reuse = true;
            h = it->second.h;
            s->queue.erase(s->queue.begin() + i);
            return r;
        }
        if (r->key >= 0 && std::find(s->building.begin(), s->building.end(), r->key) != s->building.end())
            continue;  // an earlier request is building this key's hierarchy
        if (!r->has_matrix) {
            s->queue.erase(s->queue.begin() + i);
            finish_locked(s, r, AMG_ERR_INVALID_ARG, "no resident hierarchy for this key and no matrix given");
            --i;
            --look;
            continue;
        }
        if (blocked) continue;
        int64_t idle = 0;
        for (auto& kv : s->resident)
            if (!kv.second.busy) idle += kv.second.bytes;
        // too big for the whole budget: run it once nothing else holds memory
        const bool fits = s->in_use - idle + r->estimate <= s->sp.hbm_budget || s->running == 0;
        if (!fits) {
            blocked = true;
            continue;
        }
        // admission: evict idle hierarchies, least recently used first
        while (s->in_use + r->estimate > s->sp.hbm_budget) {
            auto victim = s->resident.end();
            for (auto q = s->resident.begin(); q != s->resident.end(); ++q)
                if (!q->second.busy && (victim == s->resident.end() || q->second.last_used < victim->second.last_used))
                    victim = q;
            if (victim == s->resident.end()) break;
            s->in_use -= victim->second.bytes;
            evict.push_back(victim->second.h);
            s->resident.erase(victim);
            s->evictions++;
        }
        s->in_use += r->estimate;
        s->peak = std::max(s->peak, s->in_use);
        reuse = false;
        h = nullptr;
        if (r->key >= 0) s->building.push_back(r->key);
        s->queue.erase(s->queue.begin() + i);
        return r;
    }
    return nullptr;
}

void worker(amg_server* s) {
    cudaSetDevice(s->device);
    cudaStream_t st = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    for (;;) {
        Request* r = nullptr;
        bool reuse = false;
        amg_handle* h = nullptr;
        std::vector<amg_handle*> evict;
        {
            std::unique_lock<std::mutex> lk(s->m);
            for (;;) {
                if (s->stop && s->queue.empty()) {
                    lk.unlock();
                    if (st) cudaStreamDestroy(st);
                    return;
                }
                r = pick(s, reuse, h, evict);
                if (r || !evict.empty()) break;
                s->cv_work.wait(lk);
            }
            if (r) {
                s->running++;
                r->t_admit = now_s();
            }
        }
        for (amg_handle* e : evict) amg_free(e);
        if (!r) continue;
        amg_status status = AMG_OK;
        std::string err;
        if (!reuse) {
            amg_csr c;
            c.n = r->A.nrows;
            c.nnz = r->A.nnz();
            c.row_ptr = r->A.ptr.data();
            c.col = r->A.col.data();
            c.val = r->A.val.data();
            c.on_device = 0;
            // the host steps of this set-up use its share of the cores among
            // the set-ups running now (all of them when it runs alone)
            const int sharing = ++s->setups;
            const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
            t_thread_cap = std::max(1u, hw / (unsigned)sharing);
            status = amg_setup(&c, &r->prm, st, &h);
            if (status == AMG_ERR_OOM) {
                // the charge underestimated this hierarchy or other memory is
                // in use: free every idle resident hierarchy and try once more
                std::vector<amg_handle*> idle;
                {
                    std::lock_guard<std::mutex> lk(s->m);
                    for (auto q = s->resident.begin(); q != s->resident.end();) {
                        if (q->second.busy) { ++q; continue; }
                        s->in_use -= q->second.bytes;
                        idle.push_back(q->second.h);
                        q = s->resident.erase(q);
                        s->evictions++;
                    }
                }
                for (amg_handle* e : idle) amg_free(e);
                if (!idle.empty()) status = amg_setup(&c, &r->prm, st, &h);
            }
            --s->setups;
            if (status != AMG_OK) err = amg_last_error();
        } else {
            h->stream = st;  // run on this slot's stream
        }
        if (status == AMG_OK && (int64_t)r->f.size() != h->n) {
            status = AMG_ERR_INVALID_ARG;
            err = "right-hand side length differs from the matrix size";
        }
        if (status == AMG_OK) {
            r->x.assign(r->f.size(), 0.0);
            status = amg_solve_host(h, r->f.data(), r->x.data(), r->rtol, r->maxiter, &r->iters, &r->relres);
            if (status == AMG_ERR_NOT_CONVERGED) err = "the solve did not reach rtol within maxiter";
            else if (status == AMG_ERR_BREAKDOWN) err = "the Krylov recurrence broke down";
            else if (status != AMG_OK) err = amg_last_error();
        }
        // a hierarchy whose solve hit a device error is not kept
        const bool keep = h && status != AMG_ERR_CUDA && status != AMG_ERR_OOM;
        double bytes = 0.0;
        if (h && (status == AMG_OK || status == AMG_ERR_NOT_CONVERGED) && amg_hierarchy_bytes(h, &bytes) == AMG_OK)
            bytes *= r->iters;
        amg_handle* to_free = nullptr;
        {
            std::lock_guard<std::mutex> lk(s->m);
            s->solve_bytes += bytes;
            if (reuse) {
                auto it = s->resident.find(r->key);
                if (keep) {
                    it->second.busy = false;
                    it->second.last_used = now_s();
                } else {
                    s->in_use -= it->second.bytes;
                    s->resident.erase(it);
                    to_free = h;
                }
            } else {
                auto b = std::find(s->building.begin(), s->building.end(), r->key);
                if (b != s->building.end()) s->building.erase(b);
                s->in_use -= r->estimate;
                if (keep && r->key >= 0) {  // keep resident for later right-hand sides
                    Resident R;
                    R.h = h;
                    R.bytes = h->dev_bytes;
                    R.last_used = now_s();
                    s->resident[r->key] = R;
                    s->in_use += R.bytes;
                    s->peak = std::max(s->peak, s->in_use);
                } else {
                    to_free = h;
                }
            }
            // drop the copies of the inputs; the result stays until collected
            decltype(r->A.ptr)().swap(r->A.ptr);
            std::vector<int32_t>().swap(r->A.col);
            std::vector<double>().swap(r->A.val);
            std::vector<double>().swap(r->f);
            s->running--;
            finish_locked(s, r, status, err);
            s->cv_work.notify_all();
        }
        if (to_free) amg_free(to_free);
    }
}

}  // namespace

}  // namespace amg

using namespace amg;

extern "C" {

amg_status amg_server_create(const amg_server_params* sp, const amg_params* prm, amg_server** out) {
    if (!out) return AMG_ERR_INVALID_ARG;
    *out = nullptr;
    amg_server* s = new amg_server();
    if (sp) s->sp = *sp;
    if (s->sp.slots < 1) s->sp.slots = 4;
    if (s->sp.slots > 64) s->sp.slots = 64;
    if (prm) s->prm = *prm;
    else amg_params_default(&s->prm);
    if (cudaGetDevice(&s->device) != cudaSuccess) { delete s; return AMG_ERR_CUDA; }
    if (s->sp.hbm_budget <= 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) { cudaGetLastError(); delete s; return AMG_ERR_CUDA; }
        s->sp.hbm_budget = (int64_t)(0.8 * (double)fr);
    }
    for (int k = 0; k < s->sp.slots; ++k) s->workers.emplace_back(worker, s);
    *out = s;
    return AMG_OK;
}

amg_status amg_server_submit(amg_server* s, int64_t key, const amg_csr* A, const double* f_host, int64_t n,
                             const amg_params* prm, double rtol, int maxiter, int64_t* id) {
    if (!s || !f_host || n < 1 || !id || !(rtol >= 0.0) || maxiter < 0) return AMG_ERR_INVALID_ARG;
    auto r = std::make_unique<Request>();
    r->key = key;
    r->prm = prm ? *prm : s->prm;
    r->rtol = rtol;
    r->maxiter = maxiter;
    r->f.assign(f_host, f_host + n);
    if (A) {
        if (A->on_device || !A->row_ptr || !A->col || !A->val || A->n != n || A->nnz < 0) return AMG_ERR_INVALID_ARG;
        r->has_matrix = true;
        r->A.nrows = r->A.ncols = A->n;
        r->A.ptr.assign(A->row_ptr, A->row_ptr + A->n + 1);
        r->A.col.assign(A->col, A->col + A->nnz);
        r->A.val.assign(A->val, A->val + A->nnz);
        r->estimate = estimate_bytes(r->A);
    }
    std::lock_guard<std::mutex> lk(s->m);
    r->id = s->next_id++;
    r->t_submit = now_s();
    *id = r->id;
    s->queue.push_back(r.get());
    s->requests[r->id] = std::move(r);
    s->cv_work.notify_all();
    return AMG_OK;
}

amg_status amg_server_wait(amg_server* s, int64_t id, double* x_host, int* iters, double* relres,
                           double* latency_s, double* queue_s) {
    if (!s) return AMG_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->m);
    auto it = s->requests.find(id);
    if (it == s->requests.end()) return AMG_ERR_INVALID_ARG;
    Request* r = it->second.get();
    s->cv_done.wait(lk, [&] { return r->done; });
    if (x_host && !r->x.empty()) std::memcpy(x_host, r->x.data(), r->x.size() * sizeof(double));
    if (iters) *iters = r->iters;
    if (relres) *relres = r->relres;
    if (latency_s) *latency_s = r->t_done - r->t_submit;
    if (queue_s) *queue_s = (r->t_admit > 0 ? r->t_admit : r->t_done) - r->t_submit;
    const amg_status st = r->status;
    if (st != AMG_OK) set_last_error(r->error);
    s->requests.erase(it);
    return st;
}

amg_status amg_server_stats(amg_server* s, int64_t* completed, int* resident_count, int64_t* resident_bytes,
                            int64_t* peak_bytes, int64_t* evictions) {
    if (!s) return AMG_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->m);
    int64_t rb = 0;
    for (auto& kv : s->resident) rb += kv.second.bytes;
    if (completed) *completed = s->completed;
    if (resident_count) *resident_count = (int)s->resident.size();
    if (resident_bytes) *resident_bytes = rb;
    if (peak_bytes) *peak_bytes = s->peak;
    if (evictions) *evictions = s->evictions;
    return AMG_OK;
}

amg_status amg_server_solve_bytes(amg_server* s, double* bytes) {
    if (!s || !bytes) return AMG_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->m);
    *bytes = s->solve_bytes;
    return AMG_OK;
}

amg_status amg_server_destroy(amg_server* s) {
    if (!s) return AMG_OK;
    {
        std::lock_guard<std::mutex> lk(s->m);
        s->stop = true;
        s->cv_work.notify_all();
    }
    for (auto& t : s->workers) t.join();
    for (auto& kv : s->resident) {
        kv.second.h->stream = nullptr;  // its slot's stream went with the worker
        amg_free(kv.second.h);
    }
    delete s;
    return AMG_OK;
}

}  // extern "C"
