// host_parallel.h -- small host thread helpers for the set-up.
//
// Work is split into a fixed number of contiguous chunks that depends only on
// the problem size, so per-chunk results (partial maxima, row lists) are
// combined in chunk order and every result is independent of the thread
// count and of scheduling.
#pragma once

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <exception>
#include <mutex>
#include <thread>
#include <vector>

namespace amg {

// Cap on the threads of one parallel step for the calling thread (0: none).
// A server worker sets it to its share of the cores, so that several
// set-ups running at once do not oversubscribe the host.
inline thread_local unsigned t_thread_cap = 0;

// Host threads for one parallel step (at most 16, and at most the calling
// thread's cap).
inline unsigned host_threads() {
    const unsigned hw = std::thread::hardware_concurrency();
    unsigned n = std::max(1u, std::min(16u, hw ? hw : 1u));
    if (t_thread_cap) n = std::min(n, t_thread_cap);
    return n;
}

// Run fn(i) for i in [0, n) on host_threads() threads; rethrows the first
// exception after all workers finished.  Parallel steps inside fn run on the
// calling worker alone (the workers' thread cap is 1), so nested parallelism
// -- the per-system set-ups of the batched form -- does not oversubscribe the
// host.
template <class F>
void parallel_for(int64_t n, F&& fn) {
    const unsigned nt = (unsigned)std::min<int64_t>(host_threads(), std::max<int64_t>(n, 1));
    std::atomic<int64_t> next{0};
    std::exception_ptr err;
    std::mutex m;
    auto worker = [&]() {
        const unsigned saved = t_thread_cap;
        if (nt > 1) t_thread_cap = 1;
        for (;;) {
            const int64_t i = next++;
            if (i >= n) break;
            try {
                fn(i);
            } catch (...) {
                std::lock_guard<std::mutex> g(m);
                if (!err) err = std::current_exception();
            }
        }
        t_thread_cap = saved;
    };
    std::vector<std::thread> pool;
    for (unsigned t = 1; t < nt; ++t) pool.emplace_back(worker);
    worker();
    for (auto& t : pool) t.join();
    if (err) std::rethrow_exception(err);
}

// fn(s, t, T) for steps s = 0 .. nsteps-1 on a team of T threads (t = 0 ..
// T-1); a step starts on every thread only after every thread finished the
// previous one (a spinning barrier), and before(s) runs on thread 0 alone
// between step s-1 and step s.  The team is created once, so many short steps
// (the pivot steps of a dense factorisation) do not pay a thread start each.
template <class B, class F>
void parallel_steps(int64_t nsteps, B&& before, F&& fn) {
    const unsigned T = host_threads();
    std::atomic<unsigned> arrived{0};
    std::atomic<int64_t> started{0};  // steps whose before() ran (monotone)
    std::atomic<int64_t> done{0};     // steps every thread finished (monotone)
    std::atomic<bool> failed{false};
    std::exception_ptr err;
    std::mutex m;
    auto record = [&]() {
        std::lock_guard<std::mutex> g(m);
        if (!err) err = std::current_exception();
        failed.store(true);
    };
    auto body = [&](unsigned t) {
        for (int64_t s = 0; s < nsteps; ++s) {
            if (t == 0) {
                if (!failed.load()) {
                    try {
                        before(s);
                    } catch (...) {
                        record();
                    }
                }
                started.store(s + 1, std::memory_order_release);
            } else {
                while (started.load(std::memory_order_acquire) < s + 1) std::this_thread::yield();
            }
            if (!failed.load()) {
                try {
                    fn(s, t, T);
                } catch (...) {
                    record();
                }
            }
            // barrier: the last thread to arrive resets the count, then
            // publishes the step as done
            if (arrived.fetch_add(1, std::memory_order_acq_rel) + 1 == T) {
                arrived.store(0, std::memory_order_relaxed);
                done.store(s + 1, std::memory_order_release);
            } else {
                while (done.load(std::memory_order_acquire) < s + 1) std::this_thread::yield();
            }
        }
    };
    std::vector<std::thread> pool;
    for (unsigned t = 1; t < T; ++t) pool.emplace_back(body, t);
    body(0);
    for (auto& th : pool) th.join();
    if (err) std::rethrow_exception(err);
}

// Number of chunks for n rows holding `work` nonzeros: one per 65,536 rows
// or per 262,144 nonzeros, whichever gives more (coarse levels have few rows
// of many nonzeros), at most 64 and at most n; small matrices (and the many
// small systems of the batched set-up, which already run one system per
// thread) stay on the calling thread.
inline int row_chunks(int64_t n, int64_t work = 0) {
    const int64_t c = std::max<int64_t>(n / 65536, work / 262144);
    return (int)std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(64, c), n));
}

// fn(c, lo, hi) for the chunks c of [0, n): chunk c is
// [n c / C, n (c + 1) / C) with C = row_chunks(n, work).
template <class F>
void parallel_rows(int64_t n, int64_t work, F&& fn) {
    const int C = row_chunks(n, work);
    if (C == 1) {
        fn(0, (int64_t)0, n);
        return;
    }
    parallel_for(C, [&](int64_t c) { fn((int)c, n * c / C, n * (c + 1) / C); });
}
template <class F>
void parallel_rows(int64_t n, F&& fn) {
    parallel_rows(n, (int64_t)0, fn);
}

}  // namespace amg
