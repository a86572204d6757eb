// batch_host.cpp -- setup of many independent systems (one hierarchy each).
//
// The per-system graph work (strength, aggregation, smoothed prolongation,
// R = P^T, coarsest inverse) runs on a pool of host threads.  The Galerkin
// products run on the GPU, one sparse product per level for all systems that
// still coarsen: their matrices are concatenated block-diagonally, and a
// row-wise product of block-diagonal matrices is the block-diagonal matrix of
// the per-system products, entry for entry (the same inner-index order), so
// every system gets exactly the hierarchy it would get alone.  The result is
// packed into two device arenas: the constant hierarchy data and the
// zero-initialised work vectors.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <exception>
#include <mutex>
#include <thread>

#include "batch.h"
#include "host_parallel.h"

namespace amg {

namespace {

struct HSys {
    std::vector<HostCsr> A, P, R;
    std::vector<std::vector<double>> d;
    std::vector<double> inv;
    int nc = 0;
};

// One level of the setup of one system (the stop rule and steps of
// Algorithm 1, as in the single-system setup).  Returns true if the system
// coarsens further (P and R appended), false if level l is its coarsest.
bool level_step(HSys& S, int l, const amg_params& prm) {
    const HostCsr& A = S.A[l];
    const int64_t n = A.nrows;
    const std::vector<double> dg = host_diagonal(A);
    S.d.emplace_back();
    host_smoother_diag(A, dg, prm, S.d.back());
    bool coarsest = n <= prm.coarse_enough || l + 1 >= prm.max_levels || l + 1 >= kBatchMaxLev;
    if (!coarsest) {
        double eps = prm.strength_eps;
        if (prm.strength_halving)
            for (int q = 0; q < l; ++q) eps *= 0.5;
        std::vector<int32_t> agg;
        const int64_t nagg = host_aggregate(A, dg, eps, agg);
        if ((double)nagg >= 0.95 * (double)n) {
            if (n > prm.max_coarse_dense)
                fail(AMG_ERR_COARSENING_STALLED, "aggregation stalled on a system with " + std::to_string(n) + " rows");
            coarsest = true;
        } else {
            HostCsr P, R;
            double omega = 0.0;
            host_prolongation(A, dg, eps, agg, nagg, P, omega);
            host_transpose(P, R);
            S.P.push_back(std::move(P));
            S.R.push_back(std::move(R));
            return true;
        }
    }
    if (n > prm.max_coarse_dense) fail(AMG_ERR_TOO_LARGE, "a coarsest level exceeds max_coarse_dense");
    host_dense_inverse(A, S.inv);
    S.nc = (int)n;
    return false;
}

// Block-diagonal concatenation: row block k of the result is M[k] with its
// columns shifted by col_off[k].
HostCsr concat(const std::vector<const HostCsr*>& M, const std::vector<int64_t>& col_off, int64_t ncols) {
    HostCsr C;
    int64_t rows = 0, nnz = 0;
    for (auto* m : M) { rows += m->nrows; nnz += m->nnz(); }
    if (nnz >= (1LL << 31) - 1) fail(AMG_ERR_TOO_LARGE, "batched level has more than 2^31 nonzeros");
    C.nrows = rows;
    C.ncols = ncols;
    C.ptr.reserve(rows + 1);
    C.col.reserve(nnz);
    C.val.reserve(nnz);
    C.ptr.push_back(0);
    for (size_t k = 0; k < M.size(); ++k) {
        const HostCsr& m = *M[k];
        for (int64_t i = 0; i < m.nrows; ++i) {
            for (int32_t q = m.ptr[i]; q < m.ptr[i + 1]; ++q) {
                C.col.push_back((int32_t)(m.col[q] + col_off[k]));
                C.val.push_back(m.val[q]);
            }
            C.ptr.push_back((int32_t)C.col.size());
        }
    }
    return C;
}

DevCsr upload_tmp(const HostCsr& H) {
    DevCsr D;
    D.nrows = (int32_t)H.nrows;
    D.ncols = (int32_t)H.ncols;
    D.nnz = H.nnz();
    D.ptr = dev_alloc<int32_t>(H.nrows + 1);
    D.col = dev_alloc<int32_t>(D.nnz > 0 ? D.nnz : 1);
    D.val = dev_alloc<double>(D.nnz > 0 ? D.nnz : 1);
    AMG_CUDA(cudaMemcpy(D.ptr, H.ptr.data(), (H.nrows + 1) * sizeof(int32_t), cudaMemcpyHostToDevice));
    if (D.nnz) {
        AMG_CUDA(cudaMemcpy(D.col, H.col.data(), D.nnz * sizeof(int32_t), cudaMemcpyHostToDevice));
        AMG_CUDA(cudaMemcpy(D.val, H.val.data(), D.nnz * sizeof(double), cudaMemcpyHostToDevice));
    }
    return D;
}

void free_tmp(DevCsr& D) {
    dev_free(D.ptr);
    dev_free(D.col);
    dev_free(D.val);
    D.ptr = nullptr;
    D.col = nullptr;
    D.val = nullptr;
}

// the outputs of device_spgemm (stream-ordered allocations)
void free_product(DevCsr& D, cudaStream_t s) {
    dev_free_async(D.ptr, s);
    dev_free_async(D.col, s);
    dev_free_async(D.val, s);
    D.ptr = nullptr;
    D.col = nullptr;
    D.val = nullptr;
}

// Galerkin products of level l for the systems in `act` (one GPU product
// pair for all of them); appends A_{l+1} to each.
void galerkin_batch(std::vector<HSys>& sys, const std::vector<int>& act, int l, cudaStream_t s) {
    std::vector<const HostCsr*> As, Ps, Rs;
    std::vector<int64_t> foff, coff;
    int64_t nf = 0, nc = 0;
    for (int k : act) {
        As.push_back(&sys[k].A[l]);
        Ps.push_back(&sys[k].P[l]);
        Rs.push_back(&sys[k].R[l]);
        foff.push_back(nf);
        coff.push_back(nc);
        nf += sys[k].A[l].nrows;
        nc += sys[k].P[l].ncols;
    }
    DevCsr dA = upload_tmp(concat(As, foff, nf));
    DevCsr dP = upload_tmp(concat(Ps, coff, nc));
    DevCsr dR = upload_tmp(concat(Rs, foff, nf));
    DevCsr AP, Ac;
    try {
        device_spgemm(dA, dP, AP, s);
        device_spgemm(dR, AP, Ac, s);
    } catch (...) {
        free_tmp(dA); free_tmp(dP); free_tmp(dR); free_product(AP, s); free_product(Ac, s);
        throw;
    }
    free_tmp(dA); free_tmp(dP); free_tmp(dR); free_product(AP, s);
    std::vector<int32_t> ptr(Ac.nrows + 1), col(Ac.nnz);
    std::vector<double> val(Ac.nnz);
    AMG_CUDA(cudaMemcpy(ptr.data(), Ac.ptr, (Ac.nrows + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost));
    AMG_CUDA(cudaMemcpy(col.data(), Ac.col, Ac.nnz * sizeof(int32_t), cudaMemcpyDeviceToHost));
    AMG_CUDA(cudaMemcpy(val.data(), Ac.val, Ac.nnz * sizeof(double), cudaMemcpyDeviceToHost));
    free_product(Ac, s);
    AMG_CUDA(cudaStreamSynchronize(s));
    for (size_t q = 0; q < act.size(); ++q) {  // split the block diagonal
        const int64_t r0 = coff[q], rn = sys[act[q]].P[l].ncols;
        HostCsr C;
        C.nrows = C.ncols = rn;
        C.ptr.resize(rn + 1);
        const int32_t base = ptr[r0];
        for (int64_t i = 0; i <= rn; ++i) C.ptr[i] = ptr[r0 + i] - base;
        C.col.resize(C.ptr[rn]);
        C.val.resize(C.ptr[rn]);
        for (int32_t k = 0; k < C.ptr[rn]; ++k) {
            C.col[k] = col[base + k] - (int32_t)r0;
            C.val[k] = val[base + k];
        }
        sys[act[q]].A.push_back(std::move(C));
    }
}

constexpr size_t kNone = ~(size_t)0;

struct Arena {  // constant data, built on the host then uploaded once
    std::vector<unsigned char> buf;
    size_t add(const void* p, size_t bytes) {
        const size_t off = (buf.size() + 255) & ~(size_t)255;
        buf.resize(off + bytes + 16);  // + slack: no two arrays share a tail
        if (bytes) std::memcpy(buf.data() + off, p, bytes);
        return off;
    }
};

struct Reserve {  // zero-initialised work vectors
    size_t size = 0;
    size_t add(size_t bytes) {
        const size_t off = (size + 255) & ~(size_t)255;
        size = off + bytes + 16;
        return off;
    }
};

struct LOff {
    size_t Aptr = kNone, Acol = kNone, Aval = kNone, Avald = kNone, d = kNone;
    size_t Pptr = kNone, Pcol = kNone, Pval = kNone, Rptr = kNone, Rcol = kNone, Rval = kNone;
    size_t f = kNone, x = kNone, y = kNone, t = kNone;  // work arena
};

struct SOff {
    size_t ptr = kNone, col = kNone, val = kNone, inv = kNone;
    size_t r = kNone, z = kNone, p = kNone, q = kNone;  // work arena
    LOff lev[kBatchMaxLev];
};

template <typename T>
size_t add_vals(Arena& a, const std::vector<double>& v) {
    std::vector<T> w(v.begin(), v.end());
    return a.add(w.data(), w.size() * sizeof(T));
}

}  // namespace

void build_batch(amg_batch* b, const amg_csr* systems) {
    const amg_params& prm = b->prm;
    const int ns = b->nsys;
    const bool f32 = prm.precision == AMG_PRECISION_FP32;
    const size_t tb = f32 ? sizeof(float) : sizeof(double);
    std::vector<HSys> sys(ns);

    // inputs (host or device arrays of each system)
    for (int k = 0; k < ns; ++k) {
        const amg_csr& c = systems[k];
        if (!c.row_ptr || !c.col || !c.val || c.n < 1 || c.nnz < 0 || c.n >= (1LL << 31) - 1 ||
            c.nnz >= (1LL << 31) - 1)
            fail(AMG_ERR_INVALID_ARG, "system " + std::to_string(k) + ": bad matrix");
        HostCsr H;
        H.nrows = H.ncols = c.n;
        H.ptr.resize(c.n + 1);
        auto fetch = [&](void* dst, const void* src, size_t bytes) {
            if (c.on_device) AMG_CUDA(cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost));
            else std::memcpy(dst, src, bytes);
        };
        fetch(H.ptr.data(), c.row_ptr, (c.n + 1) * sizeof(int32_t));
        if (H.ptr[c.n] != c.nnz) fail(AMG_ERR_INVALID_ARG, "system " + std::to_string(k) + ": row_ptr[n] != nnz");
        H.col.resize(c.nnz);
        H.val.resize(c.nnz);
        fetch(H.col.data(), c.col, c.nnz * sizeof(int32_t));
        fetch(H.val.data(), c.val, c.nnz * sizeof(double));
        sys[k].A.push_back(std::move(H));
    }
    parallel_for(ns, [&](int k) { host_validate(sys[k].A[0]); });

    // Algorithm 1, level by level for all systems
    std::vector<int> act(ns);
    for (int k = 0; k < ns; ++k) act[k] = k;
    for (int l = 0; !act.empty(); ++l) {
        std::vector<char> more(ns, 0);
        parallel_for((int)act.size(), [&](int q) { more[act[q]] = level_step(sys[act[q]], l, prm) ? 1 : 0; });
        std::vector<int> next;
        for (int k : act)
            if (more[k]) next.push_back(k);
        if (!next.empty()) galerkin_batch(sys, next, l, b->stream);
        act.swap(next);
    }

    // pack
    Arena data;
    Reserve work;
    std::vector<SOff> off(ns);
    b->row_off.assign(ns + 1, 0);
    b->levels.resize(ns);
    b->nnz_fine.resize(ns);
    b->iter_bytes.resize(ns);
    for (int k = 0; k < ns; ++k) {
        HSys& S = sys[k];
        SOff& o = off[k];
        const int L = (int)S.A.size();
        const HostCsr& A0 = S.A[0];
        {
            std::vector<LevelSizes> sz(L);
            for (int l = 0; l < L; ++l)
                sz[l] = {S.A[l].nrows, S.A[l].nnz(), l + 1 < L ? S.P[l].nnz() : 0};
            b->iter_bytes[k] = krylov_iteration_bytes(sz, prm.precision, AMG_SOLVER_CG, false);
        }
        b->row_off[k + 1] = b->row_off[k] + A0.nrows;
        b->levels[k] = L;
        b->nnz_fine[k] = A0.nnz();
        o.ptr = data.add(A0.ptr.data(), A0.ptr.size() * 4);
        o.col = data.add(A0.col.data(), A0.col.size() * 4);
        o.val = data.add(A0.val.data(), A0.val.size() * 8);
        o.inv = data.add(S.inv.data(), S.inv.size() * 8);
        for (size_t* v : {&o.r, &o.z, &o.p, &o.q}) *v = work.add(A0.nrows * 8);
        for (int l = 0; l < L && L > 1; ++l) {
            LOff& lo = o.lev[l];
            const HostCsr& A = S.A[l];
            const int64_t n = A.nrows;
            if (l == L - 1) {  // coarsest: f, x only
                lo.f = work.add(n * tb);
                lo.x = work.add(n * tb);
                continue;
            }
            lo.Aptr = (l == 0) ? o.ptr : data.add(A.ptr.data(), A.ptr.size() * 4);
            lo.Acol = (l == 0) ? o.col : data.add(A.col.data(), A.col.size() * 4);
            std::vector<double> vd(A.nnz());
            for (int64_t q = 0; q < A.nnz(); ++q) vd[q] = A.val[q] * S.d[l][A.col[q]];
            lo.Aval = f32 ? add_vals<float>(data, A.val) : data.add(A.val.data(), A.val.size() * 8);
            lo.Avald = f32 ? add_vals<float>(data, vd) : data.add(vd.data(), vd.size() * 8);
            lo.d = f32 ? add_vals<float>(data, S.d[l]) : data.add(S.d[l].data(), S.d[l].size() * 8);
            const HostCsr& P = S.P[l];
            const HostCsr& R = S.R[l];
            lo.Pptr = data.add(P.ptr.data(), P.ptr.size() * 4);
            lo.Pcol = data.add(P.col.data(), P.col.size() * 4);
            lo.Pval = f32 ? add_vals<float>(data, P.val) : data.add(P.val.data(), P.val.size() * 8);
            lo.Rptr = data.add(R.ptr.data(), R.ptr.size() * 4);
            lo.Rcol = data.add(R.col.data(), R.col.size() * 4);
            lo.Rval = f32 ? add_vals<float>(data, R.val) : data.add(R.val.data(), R.val.size() * 8);
            if (l > 0) lo.f = work.add(n * tb);
            lo.x = work.add(n * tb);
            lo.y = work.add(n * tb);
            lo.t = work.add(n * tb);
        }
    }
    b->total_rows = b->row_off[ns];

    unsigned char* dbase = dev_alloc<unsigned char>(data.buf.size());
    b->allocs.push_back(dbase);
    AMG_CUDA(cudaMemcpy(dbase, data.buf.data(), data.buf.size(), cudaMemcpyHostToDevice));
    unsigned char* wbase = dev_alloc<unsigned char>(work.size);
    b->allocs.push_back(wbase);
    AMG_CUDA(cudaMemset(wbase, 0, work.size));
    auto D = [&](size_t o) -> void* { return o == kNone ? nullptr : (void*)(dbase + o); };
    auto W = [&](size_t o) -> void* { return o == kNone ? nullptr : (void*)(wbase + o); };

    std::vector<BSys> hs(ns);
    for (int k = 0; k < ns; ++k) {
        const SOff& o = off[k];
        BSys& s = hs[k];
        std::memset(&s, 0, sizeof(BSys));
        const int L = b->levels[k];
        s.n = (int)sys[k].A[0].nrows;
        s.nlev = L;
        s.nc = sys[k].nc;
        s.ptr = (const int32_t*)D(o.ptr);
        s.col = (const int32_t*)D(o.col);
        s.val = (const double*)D(o.val);
        s.inv = (const double*)D(o.inv);
        s.r = (double*)W(o.r);
        s.z = (double*)W(o.z);
        s.p = (double*)W(o.p);
        s.q = (double*)W(o.q);
        for (int l = 0; l < L && L > 1; ++l) {
            const LOff& lo = o.lev[l];
            BLevel& v = s.lev[l];
            v.n = (int)sys[k].A[l].nrows;
            v.nc = (l + 1 < L) ? (int)sys[k].A[l + 1].nrows : 0;
            v.Aptr = (const int32_t*)D(lo.Aptr);
            v.Acol = (const int32_t*)D(lo.Acol);
            v.Aval = D(lo.Aval);
            v.Avald = D(lo.Avald);
            v.d = D(lo.d);
            v.Pptr = (const int32_t*)D(lo.Pptr);
            v.Pcol = (const int32_t*)D(lo.Pcol);
            v.Pval = D(lo.Pval);
            v.Rptr = (const int32_t*)D(lo.Rptr);
            v.Rcol = (const int32_t*)D(lo.Rcol);
            v.Rval = D(lo.Rval);
            v.f = W(lo.f);
            v.x = W(lo.x);
            v.y = W(lo.y);
            v.t = W(lo.t);
        }
    }
    b->sys = dev_alloc<BSys>(ns);
    b->allocs.push_back(b->sys);
    AMG_CUDA(cudaMemcpy(b->sys, hs.data(), ns * sizeof(BSys), cudaMemcpyHostToDevice));
    b->row_off_dev = dev_alloc<int64_t>(ns + 1);
    b->allocs.push_back(b->row_off_dev);
    AMG_CUDA(cudaMemcpy(b->row_off_dev, b->row_off.data(), (ns + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
    std::vector<int> ord(ns);
    for (int k = 0; k < ns; ++k) ord[k] = k;
    b->order_input = dev_alloc<int>(ns);
    b->allocs.push_back(b->order_input);
    AMG_CUDA(cudaMemcpy(b->order_input, ord.data(), ns * sizeof(int), cudaMemcpyHostToDevice));
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int c) {
        return b->nnz_fine[a] * b->levels[a] > b->nnz_fine[c] * b->levels[c];
    });
    b->order_by_size = dev_alloc<int>(ns);
    b->allocs.push_back(b->order_by_size);
    AMG_CUDA(cudaMemcpy(b->order_by_size, ord.data(), ns * sizeof(int), cudaMemcpyHostToDevice));
    b->queue = dev_alloc<unsigned int>(1);
    b->allocs.push_back(b->queue);
    b->res = dev_alloc<BResult>(ns);
    b->allocs.push_back(b->res);
    AMG_CUDA(cudaMallocHost(&b->res_host, ns * sizeof(BResult)));
}

}  // namespace amg
