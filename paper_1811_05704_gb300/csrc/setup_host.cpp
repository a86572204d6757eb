// setup_host.cpp -- host part of the smoothed-aggregation setup.
//
// The paper builds the whole hierarchy on the CPU (Sec. 3, design principles:
// the setup is "intrinsically serial", the hierarchy is then moved into the
// backend).  This library keeps the serial graph work here -- strength of
// connection, aggregation, the smoothed prolongation and R = P^T -- and runs
// the Galerkin product R A P on the GPU (spgemm.cu).
//
// Floating-point decisions (strength test, pass-2 argmax) and the prolongation
// values are evaluated in a fixed order with no FMA contraction (the file is
// built with -ffp-contract=off), so that the aggregates and P are reproducible
// bit for bit from the level matrix.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "amg_internal.h"
#include "host_parallel.h"

namespace amg {

void host_validate(const HostCsr& A) {
    if (A.nrows < 1) fail(AMG_ERR_INVALID_ARG, "matrix has no rows");
    if ((int64_t)A.ptr.size() != A.nrows + 1) fail(AMG_ERR_INVALID_ARG, "row_ptr size");
    if (A.ptr[0] != 0) fail(AMG_ERR_INVALID_ARG, "row_ptr[0] != 0");
    // row_ptr first (the rows below index col and val through it)
    for (int64_t i = 0; i < A.nrows; ++i)
        if (A.ptr[i + 1] < A.ptr[i]) fail(AMG_ERR_INVALID_ARG, "row_ptr not monotone at row " + std::to_string(i));
    if ((int64_t)A.ptr[A.nrows] > (int64_t)A.col.size() || (int64_t)A.ptr[A.nrows] > (int64_t)A.val.size())
        fail(AMG_ERR_INVALID_ARG, "row_ptr[n] exceeds the column and value arrays");
    // the first bad row of each chunk; the lowest over the chunks is reported
    std::vector<int64_t> bad(row_chunks(A.nrows, A.ptr[A.nrows]), -1);
    std::vector<int> why(bad.size(), 0);
    parallel_rows(A.nrows, A.ptr[A.nrows], [&](int c, int64_t lo, int64_t hi) {
        for (int64_t i = lo; i < hi && bad[c] < 0; ++i)
            for (int32_t k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
                int w = 0;
                if (A.col[k] < 0 || A.col[k] >= A.ncols) w = 1;
                else if (k > A.ptr[i] && A.col[k] <= A.col[k - 1]) w = 2;
                else if (!std::isfinite(A.val[k])) w = 3;
                if (w) { bad[c] = i; why[c] = w; break; }
            }
    });
    for (size_t c = 0; c < bad.size(); ++c) {
        if (bad[c] < 0) continue;
        const std::string row = std::to_string(bad[c]);
        if (why[c] == 1) fail(AMG_ERR_INVALID_ARG, "column index out of range in row " + row);
        if (why[c] == 2) fail(AMG_ERR_INVALID_ARG, "columns not strictly ascending in row " + row);
        fail(AMG_ERR_INVALID_ARG, "non-finite value in row " + row);
    }
}

std::vector<double> host_diagonal(const HostCsr& A) {
    std::vector<double> dg(A.nrows, 0.0);
    parallel_rows(A.nrows, A.nnz(), [&](int, int64_t lo, int64_t hi) {
        for (int64_t i = lo; i < hi; ++i) {
            const int32_t* b = A.col.data() + A.ptr[i];
            const int32_t* e = A.col.data() + A.ptr[i + 1];
            const int32_t* it = std::lower_bound(b, e, (int32_t)i);
            if (it != e && *it == i) dg[i] = A.val[it - A.col.data()];
        }
    });
    for (int64_t i = 0; i < A.nrows; ++i)
        if (dg[i] == 0.0) fail(AMG_ERR_INVALID_ARG, "zero or missing diagonal in row " + std::to_string(i));
    return dg;
}

namespace {

// Strength of connection (Vanek, Mandel and Brezina 1996, the smoothed
// aggregation the paper cites in Sec. 3): j != i is strong for i iff
// a_ij^2 > eps^2 |a_ii a_jj|, decided from row i.
std::vector<uint8_t> strong_mask(const HostCsr& A, const std::vector<double>& dg, double eps) {
    const double e2 = eps * eps;
    std::vector<uint8_t> s(A.nnz(), 0);
    parallel_rows(A.nrows, A.nnz(), [&](int, int64_t lo, int64_t hi) {
        for (int64_t i = lo; i < hi; ++i)
            for (int32_t k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
                const int32_t j = A.col[k];
                const double a = A.val[k];
                s[k] = (j != i) && (a * a > e2 * std::fabs(dg[i] * dg[j]));
            }
    });
    return s;
}

}  // namespace

// Plain aggregation in four passes: (0) nodes without strong neighbours are
// singletons; (1) in row order, a free node whose strong neighbours are all
// free seeds an aggregate with them; (2) every node still free joins, as
// assigned after pass 1, the aggregate of its strong neighbour with the
// largest |a_ij| / sqrt(|a_ii a_jj|), the lowest j on ties; (3) any node still
// free seeds an aggregate with its free strong neighbours.  Ids are given in
// creation order.
int64_t host_aggregate(const HostCsr& A, const std::vector<double>& dg, double eps,
                       std::vector<int32_t>& agg) {
    const int64_t n = A.nrows;
    const std::vector<uint8_t> s = strong_mask(A, dg, eps);
    agg.assign(n, -1);
    int32_t next = 0;

    std::vector<int32_t> degree(n, 0);
    parallel_rows(n, A.nnz(), [&](int, int64_t lo, int64_t hi) {
        for (int64_t i = lo; i < hi; ++i)
            for (int32_t k = A.ptr[i]; k < A.ptr[i + 1]; ++k) degree[i] += s[k];
    });

    for (int64_t i = 0; i < n; ++i)
        if (degree[i] == 0) agg[i] = next++;

    for (int64_t i = 0; i < n; ++i) {
        if (agg[i] != -1) continue;
        bool free_nbhd = true;
        for (int32_t k = A.ptr[i]; k < A.ptr[i + 1]; ++k)
            if (s[k] && agg[A.col[k]] != -1) { free_nbhd = false; break; }
        if (!free_nbhd) continue;
        agg[i] = next;
        for (int32_t k = A.ptr[i]; k < A.ptr[i + 1]; ++k)
            if (s[k]) agg[A.col[k]] = next;
        ++next;
    }

    // pass 2 reads only the assignment after pass 1: rows are independent
    const std::vector<int32_t> after1(agg);
    parallel_rows(n, A.nnz(), [&](int, int64_t lo, int64_t hi) {
        for (int64_t i = lo; i < hi; ++i) {
            if (after1[i] != -1) continue;
            int32_t pick = -1;
            double best = -1.0;
            for (int32_t k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
                if (!s[k]) continue;
                const int32_t j = A.col[k];
                if (after1[j] == -1) continue;
                const double c = std::fabs(A.val[k]) / std::sqrt(std::fabs(dg[i] * dg[j]));
                if (c > best) { best = c; pick = after1[j]; }
            }
            if (pick != -1) agg[i] = pick;
        }
    });

    for (int64_t i = 0; i < n; ++i) {
        if (agg[i] != -1) continue;
        agg[i] = next;
        for (int32_t k = A.ptr[i]; k < A.ptr[i + 1]; ++k)
            if (s[k] && agg[A.col[k]] == -1) agg[A.col[k]] = next;
        ++next;
    }
    return next;
}

// Smoothed prolongation P = (I - omega D_F^{-1} A_F) P_t.
//   P_t(i, agg(i)) = t_i = 1/sqrt(|agg(i)|).
//   A_F: diagonal and strong entries; weak entries of a row are summed in
//   column order and subtracted from the diagonal (aF_ii = a_ii - sum_weak).
//   omega = (4/3) / rho, rho = max_i (sum over the row of A_F, in column
//   order, of |aF_ij|) / |aF_ii|.
//   P_ij = [j == agg(i)] t_i - (omega / aF_ii) * s_ij, where s_ij sums
//   aF_ik t_k over the row of A_F in column order for the k with agg(k) = j.
// The pattern of row i is {agg(i)} union {agg(k): k in the row of A_F},
// sorted; entries that evaluate to zero are kept.
// Rows of at most this many nonzeros search their few coarse columns
// linearly; longer rows (dense coarse levels) group them by sorting.
constexpr int32_t kShortRow = 32;

void host_prolongation(const HostCsr& A, const std::vector<double>& dg, double eps,
                       const std::vector<int32_t>& agg, int64_t nagg, HostCsr& P,
                       double& omega) {
    const int64_t n = A.nrows;
    const std::vector<uint8_t> s = strong_mask(A, dg, eps);

    std::vector<int64_t> size(nagg, 0);
    for (int64_t i = 0; i < n; ++i) size[agg[i]]++;
    std::vector<double> t(n), dF(n);
    const int C = row_chunks(n, A.nnz());
    std::vector<double> rho_c(C, 0.0);  // per-chunk maxima; a max is order-independent
    parallel_rows(n, A.nnz(), [&](int c, int64_t lo, int64_t hi) {
        for (int64_t i = lo; i < hi; ++i) {
            t[i] = 1.0 / std::sqrt((double)size[agg[i]]);
            double weak = 0.0;
            for (int32_t k = A.ptr[i]; k < A.ptr[i + 1]; ++k)
                if (A.col[k] != i && !s[k]) weak += A.val[k];
            dF[i] = dg[i] - weak;
        }
        double rmax = 0.0;  // written once per chunk (no false sharing between threads)
        for (int64_t i = lo; i < hi; ++i) {
            double row = 0.0;
            for (int32_t k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
                if (A.col[k] == i) row += std::fabs(dF[i]);
                else if (s[k]) row += std::fabs(A.val[k]);
            }
            rmax = std::max(rmax, row / std::fabs(dF[i]));
        }
        rho_c[c] = rmax;
    });
    double rho = 0.0;
    for (double r : rho_c) rho = std::max(rho, r);
    omega = (4.0 / 3.0) / rho;

    // rows of P per chunk, then concatenated in chunk order
    std::vector<std::vector<int32_t>> ccol(C);
    std::vector<std::vector<double>> cval(C);
    P.nrows = n;
    P.ncols = nagg;
    P.ptr.assign(n + 1, 0);
    parallel_rows(n, A.nnz(), [&](int c, int64_t lo, int64_t hi) {
        std::vector<std::pair<int32_t, double>> row;  // (coarse column, s_ij), few entries
        std::vector<std::pair<int32_t, int32_t>> byc;   // long rows: (coarse column, k), stably sorted
        // thread-local output, moved into place at the end (the vector
        // objects of neighbouring chunks share cache lines)
        std::vector<int32_t> oc;
        std::vector<double> ov;
        oc.reserve(A.ptr[hi] - A.ptr[lo] + (hi - lo));
        ov.reserve(A.ptr[hi] - A.ptr[lo] + (hi - lo));
        for (int64_t i = lo; i < hi; ++i) {
            row.clear();
            if (A.ptr[i + 1] - A.ptr[i] <= kShortRow) {
                row.emplace_back(agg[i], 0.0);
                for (int32_t k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
                    const int32_t j = A.col[k];
                    if (j != i && !s[k]) continue;
                    const double a = (j == i) ? dF[i] : A.val[k];
                    const int32_t cc = agg[j];
                    auto it = std::find_if(row.begin(), row.end(),
                                           [cc](const std::pair<int32_t, double>& e) { return e.first == cc; });
                    if (it == row.end()) it = row.emplace(row.end(), cc, 0.0);
                    it->second += a * t[j];
                }
            } else {
                // long rows: group the kept entries by coarse column with a
                // stable sort, so that each column's terms are still added in
                // ascending k (the same sums as above, without a search per
                // entry)
                byc.clear();
                for (int32_t k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
                    const int32_t j = A.col[k];
                    if (j != i && !s[k]) continue;
                    byc.emplace_back(agg[j], k);
                }
                std::stable_sort(byc.begin(), byc.end(),
                                 [](const std::pair<int32_t, int32_t>& a, const std::pair<int32_t, int32_t>& b) {
                                     return a.first < b.first;
                                 });
                bool own = false;
                for (size_t q = 0; q < byc.size();) {
                    const int32_t cc = byc[q].first;
                    double sum = 0.0;
                    for (; q < byc.size() && byc[q].first == cc; ++q) {
                        const int32_t k = byc[q].second, j = A.col[k];
                        const double a = (j == i) ? dF[i] : A.val[k];
                        sum += a * t[j];
                    }
                    row.emplace_back(cc, sum);
                    own = own || cc == agg[i];
                }
                if (!own) row.emplace_back(agg[i], 0.0);
            }
            std::sort(row.begin(), row.end());
            const double w = omega / dF[i];
            for (const auto& e : row) {
                const double base = (e.first == agg[i]) ? t[i] : 0.0;
                oc.push_back(e.first);
                ov.push_back(base - w * e.second);
            }
            P.ptr[i + 1] = (int32_t)(row.size());  // row length; prefix-summed below
        }
        ccol[c] = std::move(oc);
        cval[c] = std::move(ov);
    });
    for (int64_t i = 0; i < n; ++i) P.ptr[i + 1] += P.ptr[i];
    P.col.resize(P.ptr[n]);
    P.val.resize(P.ptr[n]);
    parallel_for(C, [&](int64_t c) {
        const int64_t lo = n * c / C;
        std::copy(ccol[c].begin(), ccol[c].end(), P.col.begin() + P.ptr[lo]);
        std::copy(cval[c].begin(), cval[c].end(), P.val.begin() + P.ptr[lo]);
    });
}

// R = P^T (Sec. 2), columns ascending.  A counting sort over chunks of rows
// of P: each chunk counts its entries per column, the counts are laid out
// column by column in chunk order, and each chunk scatters its entries, so
// the entries of a column stay in row order (the result is the serial
// transpose's).
void host_transpose(const HostCsr& P, HostCsr& R) {
    R.nrows = P.ncols;
    R.ncols = P.nrows;
    R.ptr.assign(R.nrows + 1, 0);
    R.col.resize(P.nnz());
    R.val.resize(P.nnz());
    const int64_t nc = R.nrows, n = P.nrows;
    // one chunk of rows per thread (at most 16), none for small matrices
    const int C = row_chunks(n, P.nnz()) == 1 ? 1 : (int)host_threads();
    if (C == 1) {
        for (int64_t k = 0; k < P.nnz(); ++k) R.ptr[P.col[k] + 1]++;
        for (int64_t c = 0; c < nc; ++c) R.ptr[c + 1] += R.ptr[c];
        std::vector<int32_t> pos(R.ptr.begin(), R.ptr.end() - 1);
        for (int64_t i = 0; i < n; ++i)
            for (int32_t k = P.ptr[i]; k < P.ptr[i + 1]; ++k) {
                const int32_t dst = pos[P.col[k]]++;
                R.col[dst] = (int32_t)i;
                R.val[dst] = P.val[k];
            }
        return;
    }
    // cnt[c][j]: entries of chunk c in column j, then their first slot
    std::vector<std::vector<int32_t>> cnt(C);
    parallel_for(C, [&](int64_t c) {
        cnt[c].assign(nc, 0);
        int32_t* my = cnt[c].data();
        for (int32_t k = P.ptr[n * c / C]; k < P.ptr[n * (c + 1) / C]; ++k) my[P.col[k]]++;
    });
    for (int64_t j = 0; j < nc; ++j) {
        int32_t at = R.ptr[j];
        for (int c = 0; c < C; ++c) {
            const int32_t k = cnt[c][j];
            cnt[c][j] = at;
            at += k;
        }
        R.ptr[j + 1] = at;
    }
    parallel_for(C, [&](int64_t c) {
        int32_t* pos = cnt[c].data();
        for (int64_t i = n * c / C; i < n * (c + 1) / C; ++i)
            for (int32_t k = P.ptr[i]; k < P.ptr[i + 1]; ++k) {
                const int32_t dst = pos[P.col[k]]++;
                R.col[dst] = (int32_t)i;
                R.val[dst] = P.val[k];
            }
    });
}

// Smoother diagonal (Sec. 3, relaxation): damped Jacobi omega / a_ii, or
// SPAI-0, the diagonal minimising ||I - D A||_F: a_ii / sum_j a_ij^2.
void host_smoother_diag(const HostCsr& A, const std::vector<double>& dg, const amg_params& prm,
                        std::vector<double>& d) {
    d.resize(A.nrows);
    parallel_rows(A.nrows, A.nnz(), [&](int, int64_t lo, int64_t hi) {
        for (int64_t i = lo; i < hi; ++i) {
            if (prm.smoother == AMG_SMOOTHER_SPAI0) {
                double s2 = 0.0;
                for (int32_t k = A.ptr[i]; k < A.ptr[i + 1]; ++k) s2 += A.val[k] * A.val[k];
                d[i] = dg[i] / s2;
            } else {
                d[i] = prm.jacobi_omega / dg[i];
            }
        }
    });
}

// Coarsest direct solver (Algorithm 1, last step): LU with partial pivoting
// (largest magnitude, lowest row on ties), then the explicit inverse, so that
// the solve on the GPU is one matrix-vector product.  Large matrices run on
// a team of host threads: the rows below a pivot are updated in parallel
// (each entry still receives its updates in pivot order), and the columns of
// the inverse are independent solves; the result does not depend on the
// thread count.
void host_dense_inverse(const HostCsr& A, std::vector<double>& inv) {
    const int64_t n = A.nrows;
    std::vector<double> a(n * n, 0.0);
    for (int64_t i = 0; i < n; ++i)
        for (int32_t k = A.ptr[i]; k < A.ptr[i + 1]; ++k) a[i * n + A.col[k]] = A.val[k];
    std::vector<int64_t> perm(n);
    for (int64_t i = 0; i < n; ++i) perm[i] = i;
    auto pivot = [&](int64_t c) {
        int64_t p = c;
        for (int64_t i = c + 1; i < n; ++i)
            if (std::fabs(a[i * n + c]) > std::fabs(a[p * n + c])) p = i;
        if (a[p * n + c] == 0.0) fail(AMG_ERR_INVALID_ARG, "coarsest level matrix is singular");
        if (p != c) {
            std::swap_ranges(a.begin() + c * n, a.begin() + c * n + n, a.begin() + p * n);
            std::swap(perm[c], perm[p]);
        }
    };
    auto eliminate = [&](int64_t c, int64_t i) {
        const double l = a[i * n + c] / a[c * n + c];
        a[i * n + c] = l;
        if (l != 0.0)
            for (int64_t j = c + 1; j < n; ++j) a[i * n + j] -= l * a[c * n + j];
    };
    const bool team = n >= 256 && host_threads() > 1;
    if (team) {
        parallel_steps(n, pivot, [&](int64_t c, unsigned t, unsigned T) {
            for (int64_t i = c + 1 + t; i < n; i += T) eliminate(c, i);
        });
    } else {
        for (int64_t c = 0; c < n; ++c) {
            pivot(c);
            for (int64_t i = c + 1; i < n; ++i) eliminate(c, i);
        }
    }
    inv.assign(n * n, 0.0);
    // column e of A^{-1}: solve A x = e_e with the factors
    auto column = [&](int64_t e, std::vector<double>& y) {
        for (int64_t i = 0; i < n; ++i) {
            double v = (perm[i] == e) ? 1.0 : 0.0;
            for (int64_t j = 0; j < i; ++j) v -= a[i * n + j] * y[j];
            y[i] = v;
        }
        for (int64_t i = n - 1; i >= 0; --i) {
            double v = y[i];
            for (int64_t j = i + 1; j < n; ++j) v -= a[i * n + j] * y[j];
            y[i] = v / a[i * n + i];
        }
        for (int64_t i = 0; i < n; ++i) inv[i * n + e] = y[i];
    };
    if (team) {
        const int64_t C = std::min<int64_t>(n, 64);
        parallel_for(C, [&](int64_t c) {
            std::vector<double> y(n);
            for (int64_t e = n * c / C; e < n * (c + 1) / C; ++e) column(e, y);
        });
    } else {
        std::vector<double> y(n);
        for (int64_t e = 0; e < n; ++e) column(e, y);
    }
}

// Greedy row blocks for the SpMV kernel: consecutive rows while the block
// stays within rows_cap rows and nnz_cap nonzeros (a longer single row gets a
// block of its own and is processed in several shared-memory tiles).
std::vector<int32_t> host_row_blocks(const std::vector<int32_t>& ptr, int rows_cap, int nnz_cap) {
    const int64_t n = (int64_t)ptr.size() - 1;
    std::vector<int32_t> blk;
    blk.reserve(n / 8 + 2);
    blk.push_back(0);
    int64_t start = 0;
    while (start < n) {
        int64_t end = start + 1;
        while (end < n && end - start < rows_cap && ptr[end + 1] - ptr[start] <= nnz_cap) ++end;
        blk.push_back((int32_t)end);
        start = end;
    }
    return blk;
}

// Tiles of the streaming engine: `vw` lanes share a row (a power of two
// about a sixth of the mean row length, so each lane handles a handful of
// nonzeros; a twelfth with long-row tiles of twice the nonzeros); a tile
// holds at most nnz_cap nonzeros and rows_cap rows, where
// rows_cap is one consumer pass (256/vw rows), or two passes when the rows are
// short enough for two passes to fit in nnz_cap, capped by rows_cap_max.  Returned as flattened (first row, first nonzero) pairs,
// one per tile plus the end; empty if a single row exceeds nnz_cap.
std::vector<int32_t> host_tiles(const std::vector<int32_t>& ptr, int nnz_cap, int rows_cap_max,
                                int& vw, int& rows_cap) {
    const int64_t n = (int64_t)ptr.size() - 1;
    int64_t longest = 0;
    for (int64_t i = 0; i < n; ++i) longest = std::max<int64_t>(longest, ptr[i + 1] - ptr[i]);
    if (longest > nnz_cap || n == 0) return {};
    const double avg = (double)ptr[n] / (double)n;
    vw = 1;
    const double per_lane = 6.0 * (double)nnz_cap / (double)kTileNnz;  // nonzeros a lane aims for
    while (vw < 32 && 2.0 * vw <= avg / per_lane) vw *= 2;
    // a second consumer pass only when two passes of rows still fit the tile
    const int pass = kRowsPerBlock / vw;
    rows_cap = std::min(rows_cap_max, (2.0 * pass * avg <= (double)nnz_cap) ? 2 * pass : pass);
    const std::vector<int32_t> rows = host_row_blocks(ptr, rows_cap, nnz_cap);
    std::vector<int32_t> out;
    out.reserve(2 * rows.size());
    for (int32_t r : rows) {
        out.push_back(r);
        out.push_back(ptr[r]);
    }
    return out;
}

double krylov_iteration_bytes(const std::vector<LevelSizes>& lev, int precision, int solver, bool cg_x_deferred) {
    if (lev.empty()) return 0.0;
    const double e = precision == AMG_PRECISION_BF16 ? 6.0 : precision == AMG_PRECISION_FP32 ? 8.0 : 12.0;
    const double v = precision == AMG_PRECISION_FP64 ? 8.0 : 4.0;
    const size_t L = lev.size();
    double vc = 0.0;  // one V-cycle
    for (size_t l = 0; l + 1 < L; ++l) {
        const double n = (double)lev[l].n, z = (double)lev[l].nnz, zp = (double)lev[l].nnz_p;
        const double nc = (double)lev[l + 1].n, zm = (double)lev[l].nnz_m;
        if (zm > 0) {
            vc += e * zm + 4 * nc + v * n + v * nc;      // f_{l+1} = M f: f gathered, f_{l+1} written
            vc += e * zp + 4 * n + v * nc + 3 * v * n;   // x = d f + P x_{l+1}: d, f read, x written
        } else {
            vc += e * z + 4 * n + 4 * v * n;             // pre-sweep + residual: d, f read; x, t written
            vc += e * zp + 4 * nc + v * n + v * nc;      // restriction: t gathered, f_{l+1} written
            vc += e * zp + 4 * n + v * nc + 2 * v * n;   // prolongation + correction
        }
        vc += e * z + 4 * n + 4 * v * n;                 // post-sweep: x gathered, d, f read, y written
    }
    const double nL = (double)lev[L - 1].n;
    vc += 8 * nL * nL + 2 * v * nL;                  // dense coarsest solve (float64 inverse)
    const double n0 = (double)lev[0].n, z0 = (double)lev[0].nnz;
    const double spmv = 12 * z0 + 4 * n0 + 16 * n0;  // q = A p with a dot product
    if (solver == AMG_SOLVER_BICGSTAB)
        return 2 * vc + 2 * spmv + 136 * n0;         // p, s, x, r updates and the extra dots
    if (cg_x_deferred)
        return vc + spmv + 64 * n0;                  // r update with ||r||; x += alpha p with p = z + beta p
    return vc + spmv + 72 * n0;                      // x, r update with ||r||; p = z + beta p
}

}  // namespace amg
