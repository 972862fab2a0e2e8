// Smoothed-aggregation algebraic multigrid: host-side setup.
//
// The paper solves eq. (lin_syst) directly; on the GPU the tangent systems of
// the 2D/3D meshes have condition numbers of 1e6..1e7, where one-level
// (block-)Jacobi Krylov needs thousands of iterations.  This hierarchy turns
// each solve into tens of iterations.  It is built once per mesh from K_elast
// (fixed), with the rigid-body modes of the mesh as near-null space:
//   * strength-filtered node (or aggregate) graph, greedy aggregation;
//   * tentative prolongator from a QR of the near-null space per aggregate;
//   * prolongator smoothing P = (I - omega D^-1 A) P0, omega = 4/(3 rho(D^-1 A));
//   * Galerkin coarse operator A_c = P^T A P;
//   * until at most AMG_COARSE_MAX DOFs remain, inverted densely.
// Prescribed DOFs are decoupled (identity rows) and have zero near-null rows,
// so the coarse spaces never see them.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include <numeric>
#include <string>
#include <vector>

#include "amg.h"

namespace ep {
namespace {

struct Csr {
    int64_t n = 0, m = 0;   // rows, cols
    std::vector<int64_t> rp;
    std::vector<int32_t> ci;
    std::vector<double> v;
};

Csr transpose(const Csr& A) {
    Csr T;
    T.n = A.m;
    T.m = A.n;
    T.rp.assign(T.n + 1, 0);
    for (int32_t c : A.ci) T.rp[c + 1]++;
    for (int64_t i = 0; i < T.n; ++i) T.rp[i + 1] += T.rp[i];
    T.ci.resize(A.ci.size());
    T.v.resize(A.v.size());
    std::vector<int64_t> fill(T.rp.begin(), T.rp.end() - 1);
    for (int64_t i = 0; i < A.n; ++i)
        for (int64_t k = A.rp[i]; k < A.rp[i + 1]; ++k) {
            const int64_t pos = fill[A.ci[k]]++;
            T.ci[pos] = (int32_t)i;
            T.v[pos] = A.v[k];
        }
    return T;
}

// C = A * B (Gustavson, dense accumulator per row; rows in parallel)
Csr spgemm(const Csr& A, const Csr& B) {
    Csr C;
    C.n = A.n;
    C.m = B.m;
    std::vector<std::vector<int32_t>> rows_c(A.n);
    std::vector<std::vector<double>> rows_v(A.n);
#pragma omp parallel
    {
        std::vector<double> acc(B.m, 0.0);
        std::vector<int32_t> mark(B.m, -1);
        std::vector<int32_t> cols;
#pragma omp for schedule(dynamic, 256)
        for (int64_t i = 0; i < A.n; ++i) {
            cols.clear();
            for (int64_t ka = A.rp[i]; ka < A.rp[i + 1]; ++ka) {
                const int32_t k = A.ci[ka];
                const double a = A.v[ka];
                for (int64_t kb = B.rp[k]; kb < B.rp[k + 1]; ++kb) {
                    const int32_t j = B.ci[kb];
                    if (mark[j] != (int32_t)i) {
                        mark[j] = (int32_t)i;
                        acc[j] = 0.0;
                        cols.push_back(j);
                    }
                    acc[j] += a * B.v[kb];
                }
            }
            std::sort(cols.begin(), cols.end());
            rows_c[i] = cols;
            rows_v[i].resize(cols.size());
            for (size_t t = 0; t < cols.size(); ++t) rows_v[i][t] = acc[cols[t]];
        }
    }
    C.rp.assign(C.n + 1, 0);
    for (int64_t i = 0; i < C.n; ++i) C.rp[i + 1] = C.rp[i] + (int64_t)rows_c[i].size();
    C.ci.resize(C.rp[C.n]);
    C.v.resize(C.rp[C.n]);
    for (int64_t i = 0; i < C.n; ++i) {
        std::copy(rows_c[i].begin(), rows_c[i].end(), C.ci.begin() + C.rp[i]);
        std::copy(rows_v[i].begin(), rows_v[i].end(), C.v.begin() + C.rp[i]);
    }
    return C;
}

void spmv(const Csr& A, const std::vector<double>& x, std::vector<double>& y) {
    y.assign(A.n, 0.0);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < A.n; ++i) {
        double s = 0.0;
        for (int64_t k = A.rp[i]; k < A.rp[i + 1]; ++k) s += A.v[k] * x[A.ci[k]];
        y[i] = s;
    }
}

// Invert a small dense row-major matrix in place (Gauss-Jordan, partial pivoting).
bool invert_dense(std::vector<double>& M, int n) {
    std::vector<double> I((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) I[(size_t)i * n + i] = 1.0;
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(M[(size_t)r * n + c]) > std::fabs(M[(size_t)piv * n + c])) piv = r;
        if (M[(size_t)piv * n + c] == 0.0) return false;
        if (piv != c)
            for (int k = 0; k < n; ++k) {
                std::swap(M[(size_t)piv * n + k], M[(size_t)c * n + k]);
                std::swap(I[(size_t)piv * n + k], I[(size_t)c * n + k]);
            }
        const double d = 1.0 / M[(size_t)c * n + c];
        for (int k = 0; k < n; ++k) {
            M[(size_t)c * n + k] *= d;
            I[(size_t)c * n + k] *= d;
        }
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            const double f = M[(size_t)r * n + c];
            if (f == 0.0) continue;
            for (int k = 0; k < n; ++k) {
                M[(size_t)r * n + k] -= f * M[(size_t)c * n + k];
                I[(size_t)r * n + k] -= f * I[(size_t)c * n + k];
            }
        }
    }
    M.swap(I);
    return true;
}

// Largest eigenvalue estimate of D^-1 A (D = bs x bs diagonal blocks) by power iteration.
double lambda_max(const Csr& A, int bs, const std::vector<double>& dinv, int iters = 20) {
    std::vector<double> x(A.n), y;
    for (int64_t i = 0; i < A.n; ++i) x[i] = 1.0 + 0.1 * std::sin(0.7 * (double)i);
    double lam = 1.0;
    for (int it = 0; it < iters; ++it) {
        double nx = 0.0;
        for (double v : x) nx += v * v;
        nx = std::sqrt(nx);
        if (nx == 0.0) return 1.0;
        for (double& v : x) v /= nx;
        spmv(A, x, y);
        std::vector<double> z(A.n, 0.0);
        const int64_t nb = A.n / bs;
        for (int64_t b = 0; b < nb; ++b)
            for (int r = 0; r < bs; ++r) {
                double s = 0.0;
                for (int c = 0; c < bs; ++c) s += dinv[((size_t)b * bs + r) * bs + c] * y[b * bs + c];
                z[b * bs + r] = s;
            }
        double nz = 0.0;
        for (double v : z) nz += v * v;
        lam = std::sqrt(nz);   // ||D^-1 A x|| with ||x|| = 1
        x.swap(z);
    }
    return lam;
}

// Inverses of the bs x bs diagonal blocks of A (identity where singular).
std::vector<double> block_diag_inv(const Csr& A, int bs) {
    const int64_t nb = A.n / bs;
    std::vector<double> out((size_t)nb * bs * bs, 0.0);
#pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < nb; ++b) {
        std::vector<double> M((size_t)bs * bs, 0.0);
        for (int r = 0; r < bs; ++r) {
            const int64_t i = b * bs + r;
            for (int64_t k = A.rp[i]; k < A.rp[i + 1]; ++k) {
                const int64_t j = A.ci[k];
                if (j >= b * bs && j < (b + 1) * bs) M[(size_t)r * bs + (j - b * bs)] = A.v[k];
            }
        }
        if (!invert_dense(M, bs)) {
            std::fill(M.begin(), M.end(), 0.0);
            for (int r = 0; r < bs; ++r) M[(size_t)r * bs + r] = 1.0;
        }
        std::copy(M.begin(), M.end(), out.begin() + (size_t)b * bs * bs);
    }
    return out;
}

// Block-CSR copy of a scalar CSR with row blocks rb and column blocks cb (dense blocks).
HostBsr to_bsr(const Csr& A, int rb, int cb) {
    HostBsr B;
    B.rb = rb;
    B.cb = cb;
    B.n_rows = A.n / rb;
    B.n_cols = A.m / cb;
    B.row_ptr.assign(B.n_rows + 1, 0);
    std::vector<std::vector<int32_t>> cols(B.n_rows);
    for (int64_t I = 0; I < B.n_rows; ++I) {
        for (int r = 0; r < rb; ++r) {
            const int64_t i = I * rb + r;
            for (int64_t k = A.rp[i]; k < A.rp[i + 1]; ++k) cols[I].push_back(A.ci[k] / cb);
        }
        std::sort(cols[I].begin(), cols[I].end());
        cols[I].erase(std::unique(cols[I].begin(), cols[I].end()), cols[I].end());
        B.row_ptr[I + 1] = B.row_ptr[I] + (int32_t)cols[I].size();
    }
    B.col_idx.resize(B.row_ptr[B.n_rows]);
    B.vals.assign((size_t)B.col_idx.size() * rb * cb, 0.0);
    for (int64_t I = 0; I < B.n_rows; ++I) {
        std::copy(cols[I].begin(), cols[I].end(), B.col_idx.begin() + B.row_ptr[I]);
        for (int r = 0; r < rb; ++r) {
            const int64_t i = I * rb + r;
            for (int64_t k = A.rp[i]; k < A.rp[i + 1]; ++k) {
                const int32_t J = A.ci[k] / cb, c = A.ci[k] % cb;
                const int32_t* beg = B.col_idx.data() + B.row_ptr[I];
                const int32_t* end = B.col_idx.data() + B.row_ptr[I + 1];
                const int64_t pos = std::lower_bound(beg, end, J) - B.col_idx.data();
                B.vals[(size_t)pos * rb * cb + (size_t)r * cb + c] = A.v[k];
            }
        }
    }
    return B;
}

// Greedy aggregation of the strength graph of A (blocks of size bs).
std::vector<int32_t> aggregate(const Csr& A, int bs, double theta, int64_t& n_agg) {
    const int64_t nb = A.n / bs;
    // block norms and strength graph
    std::vector<double> dn(nb, 0.0);
    std::vector<std::vector<std::pair<int32_t, double>>> nb_norm(nb);
    for (int64_t I = 0; I < nb; ++I) {
        std::vector<std::pair<int32_t, double>> acc;
        for (int r = 0; r < bs; ++r) {
            const int64_t i = I * bs + r;
            for (int64_t k = A.rp[i]; k < A.rp[i + 1]; ++k) acc.emplace_back(A.ci[k] / bs, A.v[k] * A.v[k]);
        }
        std::sort(acc.begin(), acc.end(), [](auto& a, auto& b) { return a.first < b.first; });
        for (size_t t = 0; t < acc.size();) {
            size_t u = t;
            double s = 0.0;
            while (u < acc.size() && acc[u].first == acc[t].first) s += acc[u++].second;
            nb_norm[I].emplace_back(acc[t].first, std::sqrt(s));
            if (acc[t].first == I) dn[I] = std::sqrt(s);
            t = u;
        }
    }
    std::vector<std::vector<int32_t>> strong(nb);
    for (int64_t I = 0; I < nb; ++I)
        for (auto& [J, v] : nb_norm[I])
            if (J != I && v > theta * std::sqrt(dn[I] * dn[J])) strong[I].push_back(J);
    // structurally decoupled nodes (only their own diagonal block: prescribed nodes, dead coarse DOFs)
    // belong to no aggregate and get zero prolongator rows
    std::vector<char> decoupled(nb, 0);
    for (int64_t I = 0; I < nb; ++I) decoupled[I] = (nb_norm[I].size() == 1 && nb_norm[I][0].first == I);
    std::vector<int32_t> agg(nb, -1);
    n_agg = 0;
    // phase 1: root nodes whose strong neighbourhood is free
    for (int64_t I = 0; I < nb; ++I) {
        if (decoupled[I] || agg[I] >= 0 || strong[I].empty()) continue;
        bool free_nb = true;
        for (int32_t J : strong[I])
            if (agg[J] >= 0) { free_nb = false; break; }
        if (!free_nb) continue;
        agg[I] = (int32_t)n_agg;
        for (int32_t J : strong[I]) agg[J] = (int32_t)n_agg;
        ++n_agg;
    }
    // phase 2: attach to the aggregate of the strongest aggregated neighbour
    std::vector<int32_t> agg2 = agg;
    for (int64_t I = 0; I < nb; ++I) {
        if (decoupled[I] || agg[I] >= 0) continue;
        double best = -1.0;
        for (auto& [J, v] : nb_norm[I])
            if (J != I && agg[J] >= 0 && v > best) { best = v; agg2[I] = agg[J]; }
    }
    agg = agg2;
    // phase 3: leftovers (not decoupled) form their own aggregates
    for (int64_t I = 0; I < nb; ++I) {
        if (decoupled[I] || agg[I] >= 0) continue;
        agg[I] = (int32_t)n_agg;
        for (int32_t J : strong[I])
            if (agg[J] < 0 && !decoupled[J]) agg[J] = (int32_t)n_agg;
        ++n_agg;
    }
    return agg;
}

}  // namespace

bool amg_invert_dense(std::vector<double>& M, int n) { return invert_dense(M, n); }

bool amg_setup_host(const AmgInput& in, AmgHierarchy& H, std::string& err) {
    const int d = in.dim;
    const int k = d == 2 ? 3 : 6;     // rigid-body modes
    H = AmgHierarchy{};
    H.nnzb0 = in.row_ptr[in.n_nodes];
    // level-0 scalar matrix with prescribed DOFs decoupled
    Csr A;
    A.n = A.m = in.n_nodes * d;
    A.rp.assign(A.n + 1, 0);
    {
        std::vector<std::vector<std::pair<int32_t, double>>> rows(A.n);
        for (int64_t I = 0; I < in.n_nodes; ++I)
            for (int32_t b = in.row_ptr[I]; b < in.row_ptr[I + 1]; ++b) {
                const int64_t J = in.col_idx[b];
                for (int r = 0; r < d; ++r)
                    for (int c = 0; c < d; ++c) {
                        const int64_t i = I * d + r, j = J * d + c;
                        const double v = in.vals[(size_t)b * d * d + r * d + c];
                        if (in.free_dof[i] && in.free_dof[j]) rows[i].emplace_back((int32_t)j, v);
                    }
            }
        for (int64_t i = 0; i < A.n; ++i)
            if (!in.free_dof[i]) rows[i].emplace_back((int32_t)i, 1.0);
        for (int64_t i = 0; i < A.n; ++i) {
            std::sort(rows[i].begin(), rows[i].end());
            A.rp[i + 1] = A.rp[i] + (int64_t)rows[i].size();
        }
        A.ci.resize(A.rp[A.n]);
        A.v.resize(A.rp[A.n]);
        for (int64_t i = 0; i < A.n; ++i)
            for (size_t t = 0; t < rows[i].size(); ++t) {
                A.ci[A.rp[i] + t] = rows[i][t].first;
                A.v[A.rp[i] + t] = rows[i][t].second;
            }
    }
    // near-null space: rigid-body modes about the centroid, zero on prescribed DOFs
    std::vector<double> B((size_t)A.n * k, 0.0);
    {
        double cen[3] = {0, 0, 0};
        for (int64_t I = 0; I < in.n_nodes; ++I)
            for (int c = 0; c < d; ++c) cen[c] += in.coords[I * d + c];
        for (int c = 0; c < d; ++c) cen[c] /= (double)in.n_nodes;
        for (int64_t I = 0; I < in.n_nodes; ++I) {
            const double x = in.coords[I * d] - cen[0], y = in.coords[I * d + 1] - cen[1];
            const double z = d == 3 ? in.coords[I * d + 2] - cen[2] : 0.0;
            for (int c = 0; c < d; ++c) {
                const int64_t i = I * d + c;
                if (!in.free_dof[i]) continue;
                double* row = &B[(size_t)i * k];
                row[c] = 1.0;
                if (d == 2) row[2] = (c == 0) ? -y : x;
                else {
                    // rotations about z, x, y
                    row[3] = (c == 0) ? -y : (c == 1 ? x : 0.0);
                    row[4] = (c == 1) ? -z : (c == 2 ? y : 0.0);
                    row[5] = (c == 0) ? z : (c == 2 ? -x : 0.0);
                }
            }
        }
    }
    int bs = d;
    for (int level = 0;; ++level) {
        AmgLevel L;
        L.bs = bs;
        L.n = A.n;
        bool coarsest = A.n <= AMG_COARSE_MAX || level >= AMG_MAX_LEVELS - 1;
        if (!coarsest && level > 0 && A.n > (int64_t)(0.8 * (double)H.levels.back().n)) {
            // coarsening stalled: stop here if the level is small enough to invert densely
            if (A.n > 4 * AMG_COARSE_MAX) {
                err = "AMG: coarsening stalled at " + std::to_string(A.n) + " DOFs";
                return false;
            }
            coarsest = true;
        }
        if (!coarsest) {
            L.dinv = block_diag_inv(A, bs);
            L.lambda = lambda_max(A, bs, L.dinv);
        }
        if (level > 0) {
            L.A = to_bsr(A, bs, bs);
            L.diag.assign(L.A.n_rows, 0);
            for (int64_t I = 0; I < L.A.n_rows; ++I) {
                const int32_t* b = L.A.col_idx.data() + L.A.row_ptr[I];
                const int32_t* e = L.A.col_idx.data() + L.A.row_ptr[I + 1];
                const int32_t* it = std::lower_bound(b, e, (int32_t)I);
                if (it == e || *it != I) {
                    err = "AMG: coarse operator without a diagonal block";
                    return false;
                }
                L.diag[I] = (int32_t)(it - L.A.col_idx.data());
            }
        }
        if (coarsest) {
            std::vector<double> M((size_t)A.n * A.n, 0.0);
            for (int64_t i = 0; i < A.n; ++i)
                for (int64_t t = A.rp[i]; t < A.rp[i + 1]; ++t) M[(size_t)i * A.n + A.ci[t]] = A.v[t];
            if (!invert_dense(M, (int)A.n)) {
                err = "AMG: singular coarsest matrix";
                return false;
            }
            L.dense_inv = std::move(M);
            H.levels.push_back(std::move(L));
            break;
        }
        // aggregation and tentative prolongator
        int64_t n_agg = 0;
        const std::vector<int32_t> agg = aggregate(A, bs, level == 0 ? 0.02 : 0.0, n_agg);
        const int64_t nb = A.n / bs;
        if (std::getenv("EP_AMG_DEBUG"))
            std::fprintf(stderr, "[amg] level %d: %lld block rows, nnz %lld, %lld aggregates\n", level, (long long)nb,
                         (long long)A.rp[A.n], (long long)n_agg);
        std::vector<std::vector<int32_t>> members(n_agg);
        for (int64_t I = 0; I < nb; ++I)
            if (agg[I] >= 0) members[agg[I]].push_back((int32_t)I);
        Csr P0;
        P0.n = A.n;
        P0.m = n_agg * k;
        std::vector<std::vector<std::pair<int32_t, double>>> prow(A.n);
        std::vector<double> Bc((size_t)n_agg * k * k, 0.0);
        for (int64_t a = 0; a < n_agg; ++a) {
            std::vector<int64_t> dofs;
            for (int32_t I : members[a])
                for (int c = 0; c < bs; ++c) dofs.push_back((int64_t)I * bs + c);
            const size_t m = dofs.size();
            std::vector<double> Q(m * k);
            for (size_t t = 0; t < m; ++t)
                for (int j = 0; j < k; ++j) Q[t * k + j] = B[(size_t)dofs[t] * k + j];
            std::vector<double> R((size_t)k * k, 0.0);
            // modified Gram-Schmidt with drop tolerance
            for (int j = 0; j < k; ++j) {
                double n0 = 0.0;
                for (size_t t = 0; t < m; ++t) n0 += Q[t * k + j] * Q[t * k + j];
                n0 = std::sqrt(n0);
                for (int i = 0; i < j; ++i) {
                    double s = 0.0;
                    for (size_t t = 0; t < m; ++t) s += Q[t * k + i] * Q[t * k + j];
                    R[(size_t)i * k + j] = s;
                    for (size_t t = 0; t < m; ++t) Q[t * k + j] -= s * Q[t * k + i];
                }
                double nj = 0.0;
                for (size_t t = 0; t < m; ++t) nj += Q[t * k + j] * Q[t * k + j];
                nj = std::sqrt(nj);
                if (nj <= 1e-10 * std::max(n0, 1e-300)) {
                    for (size_t t = 0; t < m; ++t) Q[t * k + j] = 0.0;
                    R[(size_t)j * k + j] = 0.0;
                } else {
                    for (size_t t = 0; t < m; ++t) Q[t * k + j] /= nj;
                    R[(size_t)j * k + j] = nj;
                }
            }
            if (std::getenv("EP_AMG_DEBUG")) {
                int dropped = 0;
                for (int j = 0; j < k; ++j) dropped += (R[(size_t)j * k + j] == 0.0);
                if (dropped) std::fprintf(stderr, "[amg]   aggregate %lld: %zu dofs, %d of %d modes dropped\n", (long long)a, m, dropped, k);
            }
            for (size_t t = 0; t < m; ++t)
                for (int j = 0; j < k; ++j)
                    if (Q[t * k + j] != 0.0) prow[dofs[t]].emplace_back((int32_t)(a * k + j), Q[t * k + j]);
            std::copy(R.begin(), R.end(), Bc.begin() + (size_t)a * k * k);
        }
        P0.rp.assign(P0.n + 1, 0);
        for (int64_t i = 0; i < P0.n; ++i) P0.rp[i + 1] = P0.rp[i] + (int64_t)prow[i].size();
        P0.ci.resize(P0.rp[P0.n]);
        P0.v.resize(P0.rp[P0.n]);
        for (int64_t i = 0; i < P0.n; ++i)
            for (size_t t = 0; t < prow[i].size(); ++t) {
                P0.ci[P0.rp[i] + t] = prow[i][t].first;
                P0.v[P0.rp[i] + t] = prow[i][t].second;
            }
        // prolongator smoothing with point Jacobi
        std::vector<double> dpt(A.n, 1.0);
        for (int64_t i = 0; i < A.n; ++i)
            for (int64_t t = A.rp[i]; t < A.rp[i + 1]; ++t)
                if (A.ci[t] == i && A.v[t] != 0.0) dpt[i] = A.v[t];
        std::vector<double> dinv_pt(A.n);
        for (int64_t i = 0; i < A.n; ++i) dinv_pt[i] = 1.0 / dpt[i];
        const double lam_pt = lambda_max(A, 1, dinv_pt);
        const double omega = 4.0 / (3.0 * lam_pt);
        Csr AP0 = spgemm(A, P0);
        Csr P;   // P = P0 - omega D^-1 A P0 (same pattern as AP0 plus P0)
        {
            P.n = P0.n;
            P.m = P0.m;
            P.rp.assign(P.n + 1, 0);
            std::vector<std::vector<std::pair<int32_t, double>>> rows(P.n);
#pragma omp parallel for schedule(dynamic, 256)
            for (int64_t i = 0; i < P.n; ++i) {
                std::vector<std::pair<int32_t, double>> r;
                int64_t a = P0.rp[i], b = AP0.rp[i];
                const double f = omega * dinv_pt[i];
                while (a < P0.rp[i + 1] || b < AP0.rp[i + 1]) {
                    const int32_t ca = a < P0.rp[i + 1] ? P0.ci[a] : INT32_MAX;
                    const int32_t cb2 = b < AP0.rp[i + 1] ? AP0.ci[b] : INT32_MAX;
                    if (ca == cb2) { r.emplace_back(ca, P0.v[a] - f * AP0.v[b]); ++a; ++b; }
                    else if (ca < cb2) { r.emplace_back(ca, P0.v[a]); ++a; }
                    else { r.emplace_back(cb2, -f * AP0.v[b]); ++b; }
                }
                rows[i] = std::move(r);
            }
            for (int64_t i = 0; i < P.n; ++i) P.rp[i + 1] = P.rp[i] + (int64_t)rows[i].size();
            P.ci.resize(P.rp[P.n]);
            P.v.resize(P.rp[P.n]);
            for (int64_t i = 0; i < P.n; ++i)
                for (size_t t = 0; t < rows[i].size(); ++t) {
                    P.ci[P.rp[i] + t] = rows[i][t].first;
                    P.v[P.rp[i] + t] = rows[i][t].second;
                }
        }
        Csr PT = transpose(P);
        Csr AP = spgemm(A, P);
        Csr Ac = spgemm(PT, AP);
        // coarse DOFs of dropped near-null columns have empty rows: make them identity
        {
            std::vector<std::vector<std::pair<int32_t, double>>> extra;
            bool any = false;
            for (int64_t i = 0; i < Ac.n; ++i) {
                bool has = false;
                for (int64_t t = Ac.rp[i]; t < Ac.rp[i + 1]; ++t)
                    if (Ac.ci[t] == i && Ac.v[t] != 0.0) has = true;
                if (!has) { any = true; break; }
            }
            if (any) {
                Csr F;
                F.n = F.m = Ac.n;
                F.rp.assign(F.n + 1, 0);
                std::vector<std::vector<std::pair<int32_t, double>>> rows(F.n);
                for (int64_t i = 0; i < Ac.n; ++i) {
                    bool has = false;
                    for (int64_t t = Ac.rp[i]; t < Ac.rp[i + 1]; ++t) {
                        if (Ac.ci[t] == i) {
                            if (Ac.v[t] == 0.0) continue;
                            has = true;
                        }
                        rows[i].emplace_back(Ac.ci[t], Ac.v[t]);
                    }
                    if (!has) {
                        rows[i].clear();
                        rows[i].emplace_back((int32_t)i, 1.0);
                    }
                    std::sort(rows[i].begin(), rows[i].end());
                    F.rp[i + 1] = F.rp[i] + (int64_t)rows[i].size();
                }
                F.ci.resize(F.rp[F.n]);
                F.v.resize(F.rp[F.n]);
                for (int64_t i = 0; i < F.n; ++i)
                    for (size_t t = 0; t < rows[i].size(); ++t) {
                        F.ci[F.rp[i] + t] = rows[i][t].first;
                        F.v[F.rp[i] + t] = rows[i][t].second;
                    }
                Ac = std::move(F);
            }
        }
        L.P = to_bsr(P, bs, k);
        L.R = to_bsr(PT, k, bs);
        L.T = to_bsr(AP, bs, k);
        for (int64_t I = 0; I < L.T.n_rows; ++I)
            L.max_t_row = std::max<int>(L.max_t_row, L.T.row_ptr[I + 1] - L.T.row_ptr[I]);
        {
            const HostBsr nextA = to_bsr(Ac, k, k);
            for (int64_t I = 0; I < nextA.n_rows; ++I)
                L.max_next_row = std::max<int>(L.max_next_row, nextA.row_ptr[I + 1] - nextA.row_ptr[I]);
        }
        H.levels.push_back(std::move(L));
        A = std::move(Ac);
        B = std::move(Bc);
        bs = k;
    }
    return true;
}

}  // namespace ep
