// Smoothed-aggregation AMG preconditioner: host setup (amg_host.cpp) and the
// device V-cycle (amg.cu).
#pragma once

#include <stdint.h>

#include <string>
#include <vector>

#include "ep_internal.h"

namespace ep {

constexpr int AMG_COARSE_MAX = 1200;   // DOFs of the coarsest level (inverted densely)
constexpr int AMG_MAX_LEVELS = 10;
constexpr int AMG_CHEB_DEGREE = 2;     // Chebyshev smoothing steps before and after the coarse correction

struct HostBsr {
    int rb = 0, cb = 0;                // block shape
    int64_t n_rows = 0, n_cols = 0;    // block rows / block columns
    std::vector<int32_t> row_ptr, col_idx;
    std::vector<double> vals;          // [nnzb][rb][cb]
};

struct AmgLevel {
    int bs = 0;                        // DOFs per block row of A at this level
    int64_t n = 0;                     // DOFs at this level
    HostBsr A;                         // operator (levels >= 1; level 0 is the live tangent)
    std::vector<double> dinv;          // inverses of the bs x bs diagonal blocks
    double lambda = 1.0;               // spectral radius estimate of D^-1 A
    HostBsr P, R;                      // prolongation from the next level and its transpose
    std::vector<double> dense_inv;     // coarsest level only
};

struct AmgHierarchy {
    std::vector<AmgLevel> levels;
};

struct AmgInput {
    int dim;
    int64_t n_nodes;
    const int32_t* row_ptr;            // block-CSR of K_elast (node blocks dim x dim)
    const int32_t* col_idx;
    const double* vals;
    const uint8_t* free_dof;
    const double* coords;              // [n_nodes][dim]
};

bool amg_setup_host(const AmgInput& in, AmgHierarchy& H, std::string& err);

// Device side
struct DevBsr {
    int rb = 0, cb = 0;
    int64_t n_rows = 0, n_cols = 0;
    int32_t *row_ptr = nullptr, *col_idx = nullptr;
    double* vals = nullptr;
};

struct AmgDevLevel {
    int bs = 0;
    int64_t n = 0;
    DevBsr A, P, R;
    double* dinv = nullptr;
    double lambda = 1.0;
    double* dense_inv = nullptr;
    double *b = nullptr, *x = nullptr, *x2 = nullptr, *d = nullptr, *r = nullptr;   // work vectors
};

struct AmgDev {
    int n_levels = 0;
    AmgDevLevel lv[AMG_MAX_LEVELS];
    double* lambda0 = nullptr;         // device scalar: spectral radius estimate for the live level-0 matrix
    double* pw = nullptr;              // power-iteration work [2][n0]
    double* pw_part = nullptr;
    int nparts = 0;
    std::vector<void*> allocs;
    int launches = 0;
};

cudaError_t amg_upload(const AmgHierarchy& H, AmgDev& D, int num_sms);
void amg_free(AmgDev& D);
// Refresh level-0 data for a new tangent: spectral radius of minv * A0 by power iteration.
cudaError_t amg_refresh(AmgDev& D, const BsrDev& A0, const double* minv0, cudaStream_t s);
// One V-cycle: out = M^-1 in (level 0 uses A0 and its block-Jacobi inverse minv0).
// rec (may be null): the calling solver's record; every launch exits at once once rec->done is set.
cudaError_t amg_apply(AmgDev& D, const BsrDev& A0, const double* minv0, const double* in, double* out,
                      const KrylovRec* rec, cudaStream_t s);

}  // namespace ep
