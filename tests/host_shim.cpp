// C wrappers around the library's host-side builders, compiled by tests/test_host_code.py (no GPU):
// the block-CSR pattern with its element-to-slot map, and the reference-element tables.
#include <algorithm>
#include <cstdint>
#include <string>
#include <vector>

#include "../paper_1805_04155_gb300/csrc/ep_internal.h"

extern "C" {

// 1 on success (outputs filled, *nnzb set), 0 when the builder rejects the mesh, -1 when cap is too small.
int shim_build_pattern(int64_t n_nodes, int64_t n_elem, int n_p, const int32_t* elem, int32_t* row_ptr, int64_t cap,
                       int32_t* col_idx, int32_t* slots, int64_t* nnzb) {
    std::vector<int32_t> rp, ci, sl;
    std::string err;
    if (!ep::build_pattern(n_nodes, n_elem, n_p, elem, rp, ci, sl, err)) return 0;
    *nnzb = (int64_t)ci.size();
    if ((int64_t)ci.size() > cap) return -1;
    std::copy(rp.begin(), rp.end(), row_ptr);
    std::copy(ci.begin(), ci.end(), col_idx);
    std::copy(sl.begin(), sl.end(), slots);
    return 1;
}

// Element colouring: color_ptr [n_elem + 1] (first n_colors + 1 entries used), color_elems [n_elem];
// returns n_colors, or 0 when the builder rejects the mesh.
int shim_color_elements(int64_t n_nodes, int64_t n_elem, int n_p, const int32_t* elem, int32_t* color_ptr,
                        int32_t* color_elems) {
    std::vector<int32_t> cp, ce;
    std::string err;
    if (!ep::color_elements(n_nodes, n_elem, n_p, elem, cp, ce, err)) return 0;
    std::copy(cp.begin(), cp.end(), color_ptr);
    std::copy(ce.begin(), ce.end(), color_elems);
    return (int)cp.size() - 1;
}

// dhat [n_q][n_p][dim] and wq [n_q]; returns n_q, or -1 when a buffer is too small.
int shim_reference_tables(int family, int dim, double* dhat, int64_t cap_dhat, double* wq, int64_t cap_wq) {
    std::vector<double> d, w;
    ep::reference_tables(family, dim, d, w);
    if ((int64_t)d.size() > cap_dhat || (int64_t)w.size() > cap_wq) return -1;
    std::copy(d.begin(), d.end(), dhat);
    std::copy(w.begin(), w.end(), wq);
    return (int)w.size();
}

}  // extern "C"

// -- AMG host setup -------------------------------------------------------------------------------
#include "../paper_1805_04155_gb300/csrc/amg.h"

extern "C" {

// Runs the smoothed-aggregation setup; returns a heap hierarchy (free with shim_amg_free) or null.
void* shim_amg_setup(int dim, int64_t n_nodes, const int32_t* row_ptr, const int32_t* col_idx, const double* vals,
                     const uint8_t* free_dof, const double* coords) {
    ep::AmgInput in{dim, n_nodes, row_ptr, col_idx, vals, free_dof, coords};
    auto* H = new ep::AmgHierarchy();
    std::string err;
    if (!ep::amg_setup_host(in, *H, err)) {
        delete H;
        return nullptr;
    }
    return H;
}

void shim_amg_free(void* h) { delete static_cast<ep::AmgHierarchy*>(h); }

int shim_amg_levels(void* h) { return (int)static_cast<ep::AmgHierarchy*>(h)->levels.size(); }

// bs, n, lambda of level l
void shim_amg_level(void* h, int l, int* bs, int64_t* n, double* lambda) {
    const ep::AmgLevel& L = static_cast<ep::AmgHierarchy*>(h)->levels[l];
    *bs = L.bs;
    *n = L.n;
    *lambda = L.lambda;
}

static const ep::HostBsr& pick(void* h, int l, int which) {
    const ep::AmgLevel& L = static_cast<ep::AmgHierarchy*>(h)->levels[l];
    return which == 0 ? L.A : (which == 1 ? L.P : L.R);
}

// shape of matrix `which` (0 A, 1 P, 2 R) of level l: block rows, block columns, block shape, blocks
void shim_amg_mat_shape(void* h, int l, int which, int64_t* n_rows, int64_t* n_cols, int* rb, int* cb, int64_t* nnzb) {
    const ep::HostBsr& M = pick(h, l, which);
    *n_rows = M.n_rows;
    *n_cols = M.n_cols;
    *rb = M.rb;
    *cb = M.cb;
    *nnzb = M.row_ptr.empty() ? 0 : M.row_ptr.back();
}

void shim_amg_mat_copy(void* h, int l, int which, int32_t* row_ptr, int32_t* col_idx, double* vals) {
    const ep::HostBsr& M = pick(h, l, which);
    std::copy(M.row_ptr.begin(), M.row_ptr.end(), row_ptr);
    std::copy(M.col_idx.begin(), M.col_idx.end(), col_idx);
    std::copy(M.vals.begin(), M.vals.end(), vals);
}

// sizes of the block-diagonal inverses and of the coarsest dense inverse of level l
void shim_amg_inv_sizes(void* h, int l, int64_t* n_dinv, int64_t* n_dense) {
    const ep::AmgLevel& L = static_cast<ep::AmgHierarchy*>(h)->levels[l];
    *n_dinv = (int64_t)L.dinv.size();
    *n_dense = (int64_t)L.dense_inv.size();
}

void shim_amg_inv_copy(void* h, int l, double* dinv, double* dense) {
    const ep::AmgLevel& L = static_cast<ep::AmgHierarchy*>(h)->levels[l];
    std::copy(L.dinv.begin(), L.dinv.end(), dinv);
    std::copy(L.dense_inv.begin(), L.dense_inv.end(), dense);
}

}  // extern "C"

// -- sparse LU: symbolic analysis ----------------------------------------------------------------
#include "../paper_1805_04155_gb300/csrc/direct.h"

extern "C" {

// Analyses the pattern; a heap plan (free with shim_direct_free) or null.
void* shim_direct_analyse(int dim, int64_t n_nodes, const int32_t* row_ptr, const int32_t* col_idx,
                          const double* coords, int leaf) {
    auto* P = new ep::DirectPlan();
    std::string err;
    if (!ep::direct_analyse(dim, n_nodes, row_ptr, col_idx, coords, leaf, *P, err)) {
        delete P;
        return nullptr;
    }
    return P;
}

void shim_direct_free(void* h) { delete static_cast<ep::DirectPlan*>(h); }

// n_fronts, n_levels, length of the node lists, front values, update-vector values
void shim_direct_sizes(void* h, int64_t* out) {
    const ep::DirectPlan& P = *static_cast<ep::DirectPlan*>(h);
    out[0] = P.n_fronts;
    out[1] = (int64_t)P.level_ptr.size() - 1;
    out[2] = (int64_t)P.nodes.size();
    out[3] = P.factor_vals();
    out[4] = P.v_off.back();
}

void shim_direct_copy(void* h, int32_t* level_ptr, int32_t* parent, int32_t* npiv, int32_t* nupd, int64_t* node_off,
                      int32_t* nodes, int32_t* umap, int32_t* blk_front, int32_t* blk_row, int32_t* blk_col,
                      int32_t* pos, double* flops) {
    const ep::DirectPlan& P = *static_cast<ep::DirectPlan*>(h);
    std::copy(P.level_ptr.begin(), P.level_ptr.end(), level_ptr);
    std::copy(P.parent.begin(), P.parent.end(), parent);
    std::copy(P.npiv.begin(), P.npiv.end(), npiv);
    std::copy(P.nupd.begin(), P.nupd.end(), nupd);
    std::copy(P.node_off.begin(), P.node_off.end(), node_off);
    std::copy(P.nodes.begin(), P.nodes.end(), nodes);
    std::copy(P.umap.begin(), P.umap.end(), umap);
    std::copy(P.blk_front.begin(), P.blk_front.end(), blk_front);
    std::copy(P.blk_row.begin(), P.blk_row.end(), blk_row);
    std::copy(P.blk_col.begin(), P.blk_col.end(), blk_col);
    std::copy(P.pos.begin(), P.pos.end(), pos);
    *flops = P.flops;
}

}  // extern "C"
