// handle.h -- the solver handle: a device-resident AMG hierarchy, the Krylov
// work vectors, the device-side Krylov state and the cached CUDA graphs.
#pragma once

#include <cuda_runtime.h>

#include <memory>
#include <vector>

#include "amg_internal.h"

namespace amg {

struct Level {
    DevCsr A, P, R;             // P, R unused on the coarsest level
    // fused restriction operator M = R (I - A D) (one pre-sweep from zero,
    // the residual and the restriction as one product), where it moves
    // fewer bytes than the three steps; M.nrows == 0 if not used
    DevCsr M;
    double* d = nullptr;        // smoother diagonal
    float* d32 = nullptr;
    // level vectors: f rhs (unused on level 0), x pre-smoothed / corrected
    // iterate, y post-smoothed output, t residual
    double *f = nullptr, *x = nullptr, *y = nullptr, *t = nullptr;
    float *f32 = nullptr, *x32 = nullptr, *y32 = nullptr, *t32 = nullptr;
    std::vector<int32_t> agg;   // host copy of the aggregates (non-coarsest, host set-up)
    int32_t* agg_dev = nullptr; // device aggregates (non-coarsest, device set-up)
    std::vector<double> dhost;  // host copy of the smoother diagonal (host set-up)
    int64_t nagg = 0;
    double omega_p = 0.0;
};

// What issued kernels are tagged with and how they are recorded.
struct Issue {
    cudaStream_t s = nullptr;
    int64_t launches = 0;
    bool profile = false;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>>* events = nullptr;
    std::vector<cudaEvent_t>* pool = nullptr;
    size_t pool_used = 0;
    int cur = 0;
    void pre(int kc);
    void post();
};

struct CachedGraph {
    const double* f = nullptr;
    double* x = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    int64_t init_launches = 0, body_launches = 0, post_launches = 0;
};

}  // namespace amg

struct amg_handle {
    amg_params prm{};
    cudaStream_t stream = nullptr;    // caller's stream
    cudaStream_t cap = nullptr;       // internal streams used for graph capture
    cudaStream_t cap2 = nullptr;
    int device = 0;
    int64_t n = 0;
    std::vector<amg::Level> lev;
    double* cinv = nullptr;           // dense inverse of the coarsest matrix
    int32_t nc = 0;
    int tail_ls = 0;                  // first level run by the tail kernel (0: none)
    amg::TailPlan tail64, tail32;
    // Krylov vectors (length n)
    double *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *rh = nullptr, *v = nullptr,
           *ph = nullptr, *sv = nullptr, *sh = nullptr, *tv = nullptr, *fbuf = nullptr,
           *xbuf = nullptr;
    // float32 V-cycles: the preconditioner's input rounded to float32, written
    // by the kernel that produces the input (r for CG, p and s for BiCGStab);
    // null for a float64 V-cycle or a one-level hierarchy
    float* vin32 = nullptr;
    amg::KState* st = nullptr;        // device
    amg::KState* st_in = nullptr;     // pinned host
    amg::KState* st_out = nullptr;    // pinned host
    int* err_host = nullptr;          // pinned host copy of the device error word
    double* partial = nullptr;
    int stride = 0;
    unsigned int* counter = nullptr;
    std::vector<void*> dev_allocs;
    int64_t dev_bytes = 0;            // bytes of device memory held (for admission control)
    std::vector<amg::CachedGraph> graphs;
    bool graph_unsupported = false;
    int64_t last_launches = 0;
    // attempts of the last solve (first run and restarts) launched as one
    // graph, and launched kernel by kernel from the host
    int last_graph_attempts = 0, last_host_attempts = 0;
    std::vector<cudaEvent_t> event_pool;
};
