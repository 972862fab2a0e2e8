// Symbolic analysis of the sparse direct solver (host): nested-dissection ordering, the separator
// tree of fronts, their node lists and the maps of the numeric phase.  See direct.h.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include "direct.h"

namespace ep {

namespace {

struct TreeNode {
    std::vector<int32_t> piv;    // pivot nodes
    std::vector<int> kids;       // tree-node ids of the children
};

struct Dissector {
    int dim;
    int64_t n;
    const int32_t* rp;
    const int32_t* ci;
    const double* X;
    int leaf;
    std::vector<int8_t> side;    // 1 left half, 2 right half, 0 outside the set being split
    std::vector<TreeNode> T;

    // Splits node set S (consumed); appends the tree roots of S to roots.
    void split(std::vector<int32_t>& S, std::vector<int>& roots) {
        if (S.empty()) return;
        if ((int64_t)S.size() <= leaf) {
            std::sort(S.begin(), S.end());
            T.push_back(TreeNode{std::move(S), {}});
            roots.push_back((int)T.size() - 1);
            return;
        }
        // longest extent of the set's coordinates
        int axis = 0;
        double best = -1.0;
        for (int a = 0; a < dim; ++a) {
            double lo = INFINITY, hi = -INFINITY;
            for (int32_t v : S) {
                lo = std::min(lo, X[(int64_t)v * dim + a]);
                hi = std::max(hi, X[(int64_t)v * dim + a]);
            }
            if (hi - lo > best) { best = hi - lo; axis = a; }
        }
        std::sort(S.begin(), S.end(), [&](int32_t a, int32_t b) {
            const double xa = X[(int64_t)a * dim + axis], xb = X[(int64_t)b * dim + axis];
            return xa < xb || (xa == xb && a < b);
        });
        const size_t mid = S.size() / 2;
        const double cut = X[(int64_t)S[mid] * dim + axis];
        // left = coordinate below the median value (or up to it when nothing lies below); a set
        // whose nodes share the coordinate is halved by index
        size_t nl = std::lower_bound(S.begin(), S.end(), cut, [&](int32_t v, double c) {
                        return X[(int64_t)v * dim + axis] < c;
                    }) - S.begin();
        if (nl == 0)
            nl = std::upper_bound(S.begin(), S.end(), cut, [&](double c, int32_t v) {
                     return c < X[(int64_t)v * dim + axis];
                 }) - S.begin();
        if (nl == 0 || nl == S.size()) nl = mid;
        for (size_t i = 0; i < S.size(); ++i) side[S[i]] = i < nl ? 1 : 2;
        // one-sided vertex separators: nodes of a half adjacent to the other half
        std::vector<int32_t> sepL, sepR;
        for (size_t i = 0; i < S.size(); ++i) {
            const int32_t v = S[i];
            const int8_t other = side[v] == 1 ? 2 : 1;
            for (int32_t k = rp[v]; k < rp[v + 1]; ++k)
                if (side[ci[k]] == other) {
                    (side[v] == 1 ? sepL : sepR).push_back(v);
                    break;
                }
        }
        const bool from_left = sepL.size() < sepR.size();
        std::vector<int32_t>& sep = from_left ? sepL : sepR;
        std::vector<int32_t> A, B;
        A.reserve(nl);
        B.reserve(S.size() - nl);
        {
            std::vector<int32_t> sorted_sep(sep);
            std::sort(sorted_sep.begin(), sorted_sep.end());
            for (size_t i = 0; i < S.size(); ++i) {
                const int32_t v = S[i];
                const bool in_sep = ((i < nl) == from_left) && std::binary_search(sorted_sep.begin(), sorted_sep.end(), v);
                if (in_sep) continue;
                (i < nl ? A : B).push_back(v);
            }
        }
        for (int32_t v : S) side[v] = 0;
        std::vector<int32_t>().swap(S);
        std::vector<int> kids;
        split(A, kids);
        split(B, kids);
        if (sep.empty()) {   // the halves are not connected: independent subtrees
            roots.insert(roots.end(), kids.begin(), kids.end());
            return;
        }
        std::sort(sep.begin(), sep.end());
        T.push_back(TreeNode{std::move(sep), std::move(kids)});
        roots.push_back((int)T.size() - 1);
    }
};

}  // namespace

bool direct_analyse(int dim, int64_t n_nodes, const int32_t* row_ptr, const int32_t* col_idx, const double* coords,
                    int leaf, DirectPlan& P, std::string& err) {
    P = DirectPlan{};
    if (n_nodes <= 0 || (dim != 2 && dim != 3) || leaf < 1) {
        err = "direct solver: empty pattern or bad dimension";
        return false;
    }
    const int64_t nnzb = row_ptr[n_nodes];
    for (int64_t v = 0; v < n_nodes; ++v)
        if (row_ptr[v + 1] < row_ptr[v]) {
            err = "direct solver: malformed row pointers";
            return false;
        }
    for (int64_t k = 0; k < nnzb; ++k)
        if (col_idx[k] < 0 || col_idx[k] >= n_nodes) {
            err = "direct solver: column index out of range";
            return false;
        }
    P.dim = dim;
    P.n_nodes = n_nodes;
    P.nnzb = nnzb;

    // 1. nested dissection
    Dissector nd{dim, n_nodes, row_ptr, col_idx, coords, leaf, std::vector<int8_t>(n_nodes, 0), {}};
    std::vector<int> roots;
    {
        std::vector<int32_t> all(n_nodes);
        for (int64_t v = 0; v < n_nodes; ++v) all[v] = (int32_t)v;
        nd.split(all, roots);
    }
    const int nt = (int)nd.T.size();
    (void)roots;
    // The dissection's creation order (every separator after the sets it splits) is the
    // elimination order.  The assembly tree is the elimination tree of the fronts: the parent of a
    // front is the front whose pivot is the first node of its update set.  Update sets follow from
    // it children first: the later nodes coupled to a pivot or in a child's update set; that is
    // the filled matrix's structure of the pivots' columns (no front carries a structural zero from
    // a separator it does not touch, as a dissection of disconnected parts would give).
    std::vector<int32_t> owner(n_nodes, -1), cpos(n_nodes, -1), last_c(nt);
    {
        int32_t p = 0;
        for (int t = 0; t < nt; ++t) {
            for (int32_t v : nd.T[t].piv) {
                owner[v] = t;
                cpos[v] = p++;
            }
            last_c[t] = p - 1;
        }
        if (p != n_nodes) {
            err = "direct solver: the dissection lost nodes";
            return false;
        }
    }
    std::vector<std::vector<int32_t>> upd(nt);
    std::vector<std::vector<int>> kids(nt);
    std::vector<int> tparent(nt, -1);
    {
        std::vector<int32_t> stamp(n_nodes, -1);
        for (int t = 0; t < nt; ++t) {
            std::vector<int32_t>& U = upd[t];
            auto take = [&](int32_t w) {
                if (cpos[w] > last_c[t] && stamp[w] != t) {
                    stamp[w] = t;
                    U.push_back(w);
                }
            };
            for (int32_t v : nd.T[t].piv)
                for (int32_t k = row_ptr[v]; k < row_ptr[v + 1]; ++k) take(col_idx[k]);
            for (int c : kids[t])
                for (int32_t w : upd[c]) take(w);
            if (!U.empty()) {
                const int32_t first = *std::min_element(U.begin(), U.end(),
                                                        [&](int32_t a, int32_t b) { return cpos[a] < cpos[b]; });
                tparent[t] = owner[first];
                kids[owner[first]].push_back(t);
            }
        }
    }
    // depths (a parent is created after its children: a reverse sweep visits parents first)
    std::vector<int> depth(nt, 0);
    for (int t = nt - 1; t >= 0; --t)
        if (tparent[t] >= 0) depth[t] = depth[tparent[t]] + 1;
    int max_depth = 0;
    for (int t = 0; t < nt; ++t) max_depth = std::max(max_depth, depth[t]);
    // processing order: deepest level first, creation order within a level (children before
    // parents; fronts of one level are independent)
    std::vector<int> order;
    order.reserve(nt);
    P.level_ptr.assign(1, 0);
    {
        std::vector<std::vector<int>> by_depth(max_depth + 1);
        for (int t = 0; t < nt; ++t) by_depth[depth[t]].push_back(t);
        for (int d = max_depth; d >= 0; --d) {
            order.insert(order.end(), by_depth[d].begin(), by_depth[d].end());
            P.level_ptr.push_back((int32_t)order.size());
        }
    }
    std::vector<int> fid(nt);
    for (int i = 0; i < nt; ++i) fid[order[i]] = i;
    P.n_fronts = nt;
    P.parent.assign(nt, -1);
    P.npiv.assign(nt, 0);
    P.nupd.assign(nt, 0);
    P.child_ptr.assign(nt + 1, 0);
    P.child_rank.assign(nt, 0);
    for (int i = 0; i < nt; ++i) {
        const int t = order[i];
        P.parent[i] = tparent[t] >= 0 ? fid[tparent[t]] : -1;
        P.npiv[i] = (int32_t)nd.T[t].piv.size();
        P.nupd[i] = (int32_t)upd[t].size();
        P.child_ptr[i + 1] = P.child_ptr[i] + (int32_t)kids[t].size();
    }
    P.children.resize(P.child_ptr[nt]);
    for (int i = 0; i < nt; ++i) {
        const std::vector<int>& kt = kids[order[i]];
        for (size_t k = 0; k < kt.size(); ++k) {
            P.children[P.child_ptr[i] + k] = fid[kt[k]];
            P.child_rank[fid[kt[k]]] = (int32_t)k;
        }
    }
    // elimination positions in processing order; update sets sorted by them
    P.pos.assign(n_nodes, -1);
    {
        int32_t p = 0;
        for (int i = 0; i < nt; ++i)
            for (int32_t v : nd.T[order[i]].piv) P.pos[v] = p++;
    }
    for (int t = 0; t < nt; ++t)
        std::sort(upd[t].begin(), upd[t].end(), [&](int32_t a, int32_t b) { return P.pos[a] < P.pos[b]; });

    // 3. node lists, sizes, offsets
    P.node_off.assign(nt + 1, 0);
    P.f_off.assign(nt + 1, 0);
    P.v_off.assign(nt + 1, 0);
    for (int i = 0; i < nt; ++i) {
        P.node_off[i + 1] = P.node_off[i] + P.npiv[i] + P.nupd[i];
        const int64_t m = (int64_t)(P.npiv[i] + P.nupd[i]) * dim;
        P.f_off[i + 1] = P.f_off[i] + ((m * m + 3) / 4) * 4;
        P.v_off[i + 1] = P.v_off[i] + (int64_t)P.nupd[i] * dim;
        // partial LU: pivot t scales the r = m - t - 1 entries below it and updates the r x r rest
        for (int64_t t = 0; t < (int64_t)P.npiv[i] * dim; ++t) {
            const double r = (double)(m - t - 1);
            P.flops += r + 2.0 * r * r;
        }
    }
    P.nodes.resize(P.node_off[nt]);
    P.umap.assign(P.node_off[nt], -1);
    for (int i = 0; i < nt; ++i) {
        int64_t o = P.node_off[i];
        for (int32_t v : nd.T[order[i]].piv) P.nodes[o++] = v;
        for (int32_t w : upd[order[i]]) P.nodes[o++] = w;
    }
    std::vector<std::vector<int32_t>>().swap(upd);
    // 4. extend-add maps: positions of a child's update set in its parent's list
    std::vector<int32_t> loc(n_nodes, -1);
    for (int p = 0; p < nt; ++p) {
        const int64_t o = P.node_off[p], len = P.node_off[p + 1] - o;
        for (int64_t a = 0; a < len; ++a) loc[P.nodes[o + a]] = (int32_t)a;
        for (int32_t k = P.child_ptr[p]; k < P.child_ptr[p + 1]; ++k) {
            const int c = P.children[k];
            for (int64_t a = P.npiv[c]; a < P.npiv[c] + P.nupd[c]; ++a) {
                const int32_t w = P.nodes[P.node_off[c] + a];
                if (loc[w] < 0) {
                    err = "direct solver: an update set is not inside its parent's front";
                    return false;
                }
                P.umap[P.node_off[c] + a] = loc[w];
            }
        }
        for (int64_t a = 0; a < len; ++a) loc[P.nodes[o + a]] = -1;
    }
    // 5. blocks: block (i, j) belongs to the front of whichever of i, j is eliminated first
    P.blk_front.assign(nnzb, -1);
    P.blk_row.assign(nnzb, -1);
    P.blk_col.assign(nnzb, -1);
    for (int s = 0; s < nt; ++s) {
        const int64_t o = P.node_off[s], len = P.node_off[s + 1] - o;
        for (int64_t a = 0; a < len; ++a) loc[P.nodes[o + a]] = (int32_t)a;
        for (int64_t a = 0; a < P.npiv[s]; ++a) {
            const int32_t v = P.nodes[o + a];
            for (int32_t k = row_ptr[v]; k < row_ptr[v + 1]; ++k) {
                const int32_t w = col_idx[k];
                if (P.pos[w] < P.pos[v]) continue;
                if (loc[w] < 0) {
                    err = "direct solver: a coupled node is missing from a front";
                    return false;
                }
                P.blk_front[k] = s;
                P.blk_row[k] = loc[v];
                P.blk_col[k] = loc[w];
                if (w == v) continue;
                // the transposed block (w, v)
                const int32_t* b = col_idx + row_ptr[w];
                const int32_t* e = col_idx + row_ptr[w + 1];
                const int32_t* f = std::lower_bound(b, e, v);
                if (f == e || *f != v) {
                    err = "direct solver: the pattern is not structurally symmetric";
                    return false;
                }
                const int64_t kt = f - col_idx;
                P.blk_front[kt] = s;
                P.blk_row[kt] = loc[w];
                P.blk_col[kt] = loc[v];
            }
        }
        for (int64_t a = 0; a < len; ++a) loc[P.nodes[o + a]] = -1;
    }
    for (int64_t k = 0; k < nnzb; ++k)
        if (P.blk_front[k] < 0) {
            err = "direct solver: a block was assigned to no front";
            return false;
        }
    // 6. per-level extents
    const int nl = (int)P.level_ptr.size() - 1;
    P.lvl_kmax.assign(nl, 0);
    P.lvl_mmax.assign(nl, 0);
    P.lvl_umax.assign(nl, 0);
    P.lvl_maxkids.assign(nl, 0);
    for (int l = 0; l < nl; ++l)
        for (int s = P.level_ptr[l]; s < P.level_ptr[l + 1]; ++s) {
            P.lvl_kmax[l] = std::max(P.lvl_kmax[l], P.npiv[s] * dim);
            P.lvl_mmax[l] = std::max(P.lvl_mmax[l], (P.npiv[s] + P.nupd[s]) * dim);
            P.lvl_umax[l] = std::max(P.lvl_umax[l], P.nupd[s] * dim);
            P.lvl_maxkids[l] = std::max(P.lvl_maxkids[l], P.child_ptr[s + 1] - P.child_ptr[s]);
        }
    return true;
}

}  // namespace ep
