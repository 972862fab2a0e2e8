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
