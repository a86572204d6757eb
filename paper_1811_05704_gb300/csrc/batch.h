// batch.h -- many independent systems solved by one persistent kernel.
//
// Each system has its own hierarchy (Algorithm 1 per system) packed into
// shared arenas; a CTA takes a system from a device work queue and runs the
// whole preconditioned CG loop for it (Algorithm 2 as the preconditioner),
// with block-level barriers between steps, then takes the next system.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "amg_internal.h"

namespace amg {

constexpr int kBatchMaxLev = 12;

// One level of one system (device pointers into the arenas).  Values and
// level vectors are of the V-cycle type (float or double); the coarsest level
// uses only f and x.
struct BLevel {
    int n;       // rows of this level
    int nc;      // rows of the next level
    const int32_t* Aptr;
    const int32_t* Acol;
    const void* Aval;   // a_ij
    const void* Avald;  // a_ij d_j (first pre-sweep)
    const void* d;      // smoother diagonal
    const int32_t* Pptr;
    const int32_t* Pcol;
    const void* Pval;
    const int32_t* Rptr;
    const int32_t* Rcol;
    const void* Rval;
    void* f;
    void* x;
    void* y;
    void* t;
};

struct BSys {
    int n;     // rows of the finest level
    int nlev;  // levels
    int nc;    // rows of the coarsest level
    int pad;
    const int32_t* ptr;  // finest matrix in float64, for the Krylov product
    const int32_t* col;
    const double* val;
    const double* inv;   // dense inverse of the coarsest matrix (nc x nc, row-major)
    double* r;
    double* z;
    double* p;
    double* q;
    BLevel lev[kBatchMaxLev];
};

struct BResult {
    int iters;
    int status;
    double relres;
};

// Kernel launch (batch.cu): solve systems order[0..nsys) with the given
// schedule (threads per CTA, CTAs per SM).  f and x are the concatenated
// right-hand sides and solutions; offsets per system in row_off.
void launch_batch_cg(const BSys* sys, const int* order, int nsys, const int64_t* row_off,
                     unsigned int* queue, const double* f, double* x, double rtol, int maxiter,
                     bool vcycle_f32, BResult* res, int threads, int ctas_per_sm, cudaStream_t s);

int batch_max_threads(bool vcycle_f32);

}  // namespace amg

struct amg_batch {
    amg_params prm{};
    cudaStream_t stream = nullptr;
    int device = 0;
    int nsys = 0;
    int64_t total_rows = 0;
    std::vector<int64_t> row_off;     // nsys + 1
    std::vector<int> levels;          // per system
    std::vector<int64_t> nnz_fine;    // per system
    std::vector<double> iter_bytes;   // per system: algorithmic bytes of one CG iteration
    amg::BSys* sys = nullptr;         // device descriptors
    int64_t* row_off_dev = nullptr;
    int* order_by_size = nullptr;     // device: largest system first
    int* order_input = nullptr;       // device: input order
    unsigned int* queue = nullptr;
    amg::BResult* res = nullptr;      // device
    amg::BResult* res_host = nullptr; // pinned
    std::vector<void*> allocs;
    // schedule (autotuned by amg_batch_tune)
    int threads = 512;
    int ctas_per_sm = 2;
    int order_mode = 0;  // 0: largest first, 1: input order
    int tuned = 0;
};
