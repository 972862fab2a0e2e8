// Block-CSR pattern of the stiffness matrix and the element-to-slot map.
//
// The sparsity of K is fixed by the mesh (Section 6.3: K_elast = B^T D B and
// Section 7: K_tangent share one pattern).  Rows and columns are nodes; each
// stored block is the dim x dim coupling of two nodes that share an element.
// The slot map gives, for every element and local node pair (p, q), the index
// of block (node_p, node_q), so each Newton iteration scatters into fixed
// positions without searching.
#include <algorithm>
#include <string>
#include <vector>

#include "ep_internal.h"

namespace ep {

bool build_pattern(int64_t n_nodes, int64_t n_elem, int n_p, const int32_t* elem, std::vector<int32_t>& row_ptr,
                   std::vector<int32_t>& col_idx, std::vector<int32_t>& slots, std::string& err) {
    for (int64_t i = 0; i < n_elem * n_p; ++i) {
        if (elem[i] < 0 || elem[i] >= n_nodes) {
            err = "element " + std::to_string(i / n_p) + " references node " + std::to_string(elem[i]) +
                  " outside [0, " + std::to_string(n_nodes) + ")";
            return false;
        }
    }
    // node -> elements incidence
    std::vector<int64_t> inc_ptr(n_nodes + 1, 0);
    for (int64_t i = 0; i < n_elem * n_p; ++i) inc_ptr[elem[i] + 1]++;
    for (int64_t n = 0; n < n_nodes; ++n) inc_ptr[n + 1] += inc_ptr[n];
    std::vector<int32_t> inc(inc_ptr[n_nodes]);
    {
        std::vector<int64_t> fill(inc_ptr.begin(), inc_ptr.end() - 1);
        for (int64_t e = 0; e < n_elem; ++e)
            for (int p = 0; p < n_p; ++p) inc[fill[elem[e * n_p + p]]++] = (int32_t)e;
    }
    // rows: sorted unique neighbours of each node
    std::vector<int32_t> counts(n_nodes, 0);
    row_ptr.assign(n_nodes + 1, 0);
    // first pass: count (with a scratch buffer per node)
    std::vector<int32_t> buf;
    for (int64_t n = 0; n < n_nodes; ++n) {
        buf.clear();
        for (int64_t k = inc_ptr[n]; k < inc_ptr[n + 1]; ++k) {
            const int64_t e = inc[k];
            for (int p = 0; p < n_p; ++p) buf.push_back(elem[e * n_p + p]);
        }
        std::sort(buf.begin(), buf.end());
        buf.erase(std::unique(buf.begin(), buf.end()), buf.end());
        counts[n] = (int32_t)buf.size();
    }
    int64_t total = 0;
    for (int64_t n = 0; n < n_nodes; ++n) {
        row_ptr[n] = (int32_t)total;
        total += counts[n];
        if (total > INT32_MAX) {
            err = "stiffness pattern exceeds 2^31 blocks";
            return false;
        }
    }
    row_ptr[n_nodes] = (int32_t)total;
    col_idx.assign(total, 0);
    for (int64_t n = 0; n < n_nodes; ++n) {
        buf.clear();
        for (int64_t k = inc_ptr[n]; k < inc_ptr[n + 1]; ++k) {
            const int64_t e = inc[k];
            for (int p = 0; p < n_p; ++p) buf.push_back(elem[e * n_p + p]);
        }
        std::sort(buf.begin(), buf.end());
        buf.erase(std::unique(buf.begin(), buf.end()), buf.end());
        std::copy(buf.begin(), buf.end(), col_idx.begin() + row_ptr[n]);
    }
    // slot map
    slots.assign((size_t)n_elem * n_p * n_p, 0);
    for (int64_t e = 0; e < n_elem; ++e) {
        for (int p = 0; p < n_p; ++p) {
            const int32_t r = elem[e * n_p + p];
            const int32_t* beg = col_idx.data() + row_ptr[r];
            const int32_t* end = col_idx.data() + row_ptr[r + 1];
            for (int q = 0; q < n_p; ++q) {
                const int32_t c = elem[e * n_p + q];
                const int32_t* it = std::lower_bound(beg, end, c);
                slots[(size_t)e * n_p * n_p + p * n_p + q] = (int32_t)(it - col_idx.data());
            }
        }
    }
    return true;
}

}  // namespace ep
