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

// Element colouring for the deterministic assembly: elements of one colour share no node, so
// within a colour every F entry and every K block receives at most one contribution and plain
// read-modify-write stores replace atomics.  Greedy, in element order (the smallest colour not
// used by an already coloured element sharing a node).  color_ptr [n_colors + 1] and color_elems
// [n_elem] list the elements of each colour in increasing order.
bool color_elements(int64_t n_nodes, int64_t n_elem, int n_p, const int32_t* elem, std::vector<int32_t>& color_ptr,
                    std::vector<int32_t>& color_elems, std::string& err) {
    for (int64_t i = 0; i < n_elem * n_p; ++i)
        if (elem[i] < 0 || elem[i] >= n_nodes) {
            err = "colouring: node index out of range";
            return false;
        }
    std::vector<int64_t> inc_ptr(n_nodes + 1, 0);
    for (int64_t i = 0; i < n_elem * n_p; ++i) inc_ptr[elem[i] + 1]++;
    for (int64_t n = 0; n < n_nodes; ++n) inc_ptr[n + 1] += inc_ptr[n];
    std::vector<int32_t> inc(inc_ptr[n_nodes]);
    {
        std::vector<int64_t> fill(inc_ptr.begin(), inc_ptr.end() - 1);
        for (int64_t e = 0; e < n_elem; ++e)
            for (int p = 0; p < n_p; ++p) inc[fill[elem[e * n_p + p]]++] = (int32_t)e;
    }
    std::vector<int32_t> color(n_elem, -1);
    std::vector<int64_t> stamp;   // stamp[c] == e: colour c is used by a neighbour of e
    int n_colors = 0;
    for (int64_t e = 0; e < n_elem; ++e) {
        for (int p = 0; p < n_p; ++p) {
            const int32_t v = elem[e * n_p + p];
            for (int64_t k = inc_ptr[v]; k < inc_ptr[v + 1]; ++k) {
                const int32_t c = color[inc[k]];
                if (c >= 0) stamp[c] = e;
            }
        }
        int c = 0;
        while (c < n_colors && stamp[c] == e) ++c;
        if (c == n_colors) {
            ++n_colors;
            stamp.push_back(-1);
        }
        color[e] = c;
    }
    color_ptr.assign(n_colors + 1, 0);
    for (int64_t e = 0; e < n_elem; ++e) color_ptr[color[e] + 1]++;
    for (int c = 0; c < n_colors; ++c) color_ptr[c + 1] += color_ptr[c];
    color_elems.resize(n_elem);
    std::vector<int32_t> fill(color_ptr.begin(), color_ptr.end() - 1);
    for (int64_t e = 0; e < n_elem; ++e) color_elems[fill[color[e]]++] = (int32_t)e;
    return true;
}

}  // namespace ep
