// Sparse direct LU of the block-CSR tangent: multifrontal factorisation in nested-dissection order
// with static pivoting (FP64 fronts, or FP32 ones), used as the preconditioner of an FP64 GMRES (the
// outer iteration refines what the perturbed pivots and the factors' rounding leave).
//
// The paper solves every linearised system (eq. (lin_syst)) with a direct solver.  Near the limit
// load of a nonassociated Drucker-Prager body the tangent acquires eigenvalues with negative real
// parts (local plastic-flow modes, Section 2.3); Krylov methods with a multigrid preconditioner
// stall there, a factorisation does not.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "ep_internal.h"

namespace ep {

// Symbolic analysis on the host.  The node graph (the block-CSR pattern) is ordered by nested
// dissection: recursive coordinate bisection of the node set at the median along its longest
// extent, with the smaller one-sided vertex separator (nodes of one half adjacent to the other)
// eliminated after both halves.  Each separator, and each node set at the leaves, is a front: its
// pivot nodes followed by its update set (the later nodes coupled to a pivot or in a child's update
// set: the filled matrix's structure of the pivots' columns), in elimination order.  The fronts
// form the elimination tree (a front's parent holds the first node of its update set) and are
// numbered in processing order, the deepest level first, so every child precedes its parent.
struct DirectPlan {
    int dim = 0;
    int64_t n_nodes = 0, nnzb = 0;
    int n_fronts = 0;
    std::vector<int32_t> level_ptr;        // level l (deepest first) = fronts [level_ptr[l], level_ptr[l + 1])
    std::vector<int32_t> parent;           // [n_fronts] parent front, -1 for a root
    std::vector<int32_t> child_ptr;        // [n_fronts + 1] children of front s: children[child_ptr[s] ..)
    std::vector<int32_t> children;
    std::vector<int32_t> child_rank;       // [n_fronts] position among its parent's children
    std::vector<int32_t> npiv, nupd;       // [n_fronts] pivot nodes, update-set nodes
    std::vector<int64_t> node_off;         // [n_fronts + 1] offsets into nodes / umap
    std::vector<int32_t> nodes;            // front node lists: pivots, then update set
    std::vector<int32_t> umap;             // at the update-set positions of front s: the node's index in its
                                           // parent's list (-1 at pivot positions and for roots)
    std::vector<int64_t> f_off;            // [n_fronts + 1] offsets of the dense fronts (values, multiple of 4)
    std::vector<int64_t> v_off;            // [n_fronts + 1] offsets of the update vectors of the solve
    std::vector<int32_t> blk_front, blk_row, blk_col;   // [nnzb] front of every block, local node row / column
    std::vector<int32_t> pos;              // [n_nodes] elimination position of every node
    std::vector<int32_t> lvl_kmax, lvl_mmax, lvl_umax, lvl_maxkids;   // per level: largest pivot count,
                                           // front order, update order (scalar rows), number of children
    double flops = 0.0;                    // factorisation flops (partial LU of every front)
    int64_t factor_vals() const { return f_off.empty() ? 0 : f_off.back(); }
};

// Builds the plan; false (err set) on an empty or malformed pattern.  leaf: largest node set
// factored as one front.
bool direct_analyse(int dim, int64_t n_nodes, const int32_t* row_ptr, const int32_t* col_idx, const double* coords,
                    int leaf, DirectPlan& P, std::string& err);

// Device state of the factorisation (owned by a context).
struct DirectDev {
    DirectPlan plan;
    bool ready = false;        // plan analysed and device memory allocated
    bool refused = false;      // analysis or allocation refused (too large): not tried again
    std::string why;           // reason of a refusal
    int32_t *blk_front = nullptr, *blk_row = nullptr, *blk_col = nullptr;
    int32_t *nodes = nullptr, *umap = nullptr, *npiv = nullptr, *nupd = nullptr, *child_ptr = nullptr,
            *children = nullptr, *parent = nullptr, *child_rank = nullptr;
    int64_t *node_off = nullptr, *f_off = nullptr, *v_off = nullptr;
    int fp64 = 1;              // front precision: 1 FP64, 0 FP32 (set before direct_setup)
    void* F = nullptr;         // fronts (FP64 or FP32)
    void* vupd = nullptr;      // update vectors of the forward solve (front precision)
    void* y = nullptr;         // [n_nodes * dim] forward-solve values at the pivots (front precision)
    float* anorm = nullptr;    // device scalar: largest |diagonal entry| on free DOFs
    unsigned int* n_perturbed = nullptr;   // device counter of perturbed pivots (static pivoting)
    int64_t bytes = 0;         // device memory held
    int n_factor = 0;          // factorisations (accumulates)
    int n_solve = 0;           // solves (accumulates)
    int launches = 0;          // kernels launched (accumulates)
    // profile = 1: CUDA events around every factorisation and solve (the host waits for each), their
    // summed durations
    int profile = 0;
    double factor_ms = 0.0, solve_ms = 0.0;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    double solve_bytes = 0.0;  // bytes of the fronts one solve reads (L and U parts)
    std::vector<void*> allocs;
};

// Allocates the device side of an analysed plan (D.plan); false with D.why on failure (too large:
// the fronts must fit in max_bytes, the solve's working vector in shared memory).
bool direct_setup(DirectDev& D, int64_t max_bytes);
void direct_free(DirectDev& D);
// Factorises A (FP64 or FP32 values; Dirichlet rows and columns replaced by the identity) into D.
cudaError_t direct_factor(DirectDev& D, const BsrT<double>& A, cudaStream_t s);
cudaError_t direct_factor(DirectDev& D, const BsrT<float>& A, cudaStream_t s);
// x = (LU)^-1 b on the free DOFs (x = 0 on the others).  rec (may be null): the kernels return at
// once when rec->done is set (iterations enqueued after a Krylov solve converged).
cudaError_t direct_solve(DirectDev& D, const double* b, double* x, const uint8_t* free_dof, const KrylovRec* rec,
                         cudaStream_t s);
cudaError_t direct_solve(DirectDev& D, const float* b, float* x, const uint8_t* free_dof, const KrylovRec* rec,
                         cudaStream_t s);

}  // namespace ep
