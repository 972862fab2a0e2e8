// Smoothed-aggregation AMG preconditioner: host setup (amg_host.cpp) and the
// device V-cycle with on-device Galerkin refresh (amg.cu).
#pragma once

#include <stdint.h>

#include <string>
#include <vector>

#include "ep_internal.h"

namespace ep {

constexpr int AMG_COARSE_MAX = 600;    // DOFs of the coarsest level (inverted densely on the host)
constexpr int AMG_MAX_LEVELS = 10;
constexpr int AMG_CHEB_DEGREE = 3;     // largest number of Chebyshev smoothing steps on either side of the coarse correction

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
    std::vector<int32_t> diag;         // block index of each row's diagonal block in A (levels >= 1)
    std::vector<double> dinv;          // inverses of the bs x bs diagonal blocks
    double lambda = 1.0;               // spectral radius estimate of D^-1 A
    HostBsr P, R;                      // prolongation from the next level and its transpose
    HostBsr T;                         // pattern of A P (values unused): the first Galerkin factor
    int max_t_row = 0;                 // longest block row of T
    int max_next_row = 0;              // longest block row of the next level's A
    std::vector<double> dense_inv;     // coarsest level only
};

struct AmgHierarchy {
    std::vector<AmgLevel> levels;
    int64_t nnzb0 = 0;                 // blocks of the level-0 (tangent) pattern
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
// In-place inverse of a dense row-major n x n matrix (partial pivoting); false if singular.
bool amg_invert_dense(std::vector<double>& M, int n);

// Device side.  The whole V-cycle is single precision (level 0 on an FP32 copy
// of the tangent): the preconditioner's precision does not limit the accuracy
// of the FP64 Krylov iteration it serves.
struct DevPat {
    int rb = 0, cb = 0;
    int g = 8;                         // lanes per block row in the row kernels (from the average row length)
    int64_t n_rows = 0, n_cols = 0;
    int32_t *row_ptr = nullptr, *col_idx = nullptr;
};

struct AmgDevLevel {
    int bs = 0;
    int64_t n = 0;
    DevPat A, P, R, T;                 // patterns (A for levels >= 1; P, R, T towards the next level)
    float *Avals = nullptr, *Pvals = nullptr, *Rvals = nullptr, *Tvals = nullptr;
    int32_t* diag = nullptr;           // diagonal block index per row of A (levels >= 1)
    float* dinv = nullptr;             // levels >= 1
    float* dense_inv = nullptr;        // coarsest level
    float* dense_work = nullptr;       // coarsest level: [n][2n] Gauss-Jordan work
    int max_t_row = 0, max_next_row = 0;
    float *b = nullptr, *x = nullptr, *x2 = nullptr, *d = nullptr, *r = nullptr;   // work vectors (all levels)
    // FP64 coarse correction (precise mode, allocated on first use): the operator, its block
    // inverses, the product A P of the Galerkin refresh, the coarsest dense inverse and work vectors;
    // level 0 uses x64 (iterate) and r64 (residual) only
    double *Avals64 = nullptr, *dinv64 = nullptr, *Tvals64 = nullptr, *dense_inv64 = nullptr;
    double *b64 = nullptr, *x64 = nullptr, *x2_64 = nullptr, *d64 = nullptr, *r64 = nullptr;
    int64_t a_vals = 0, t_vals = 0;    // value counts of A (levels >= 1) and of A P
};

struct AmgDev {
    int n_levels = 0;
    AmgDevLevel lv[AMG_MAX_LEVELS];
    double* lam = nullptr;             // device [AMG_MAX_LEVELS]: spectral radius estimates per level
    float* coef = nullptr;             // device [AMG_MAX_LEVELS][AMG_CHEB_DEGREE][3]: Chebyshev coefficients
    float* K32 = nullptr;              // FP64 path: FP32 copy of the live level-0 matrix values [nnzb0][dim][dim]
    float* minv32 = nullptr;           // FP64 path: FP32 copy of its block-Jacobi inverse [n_nodes][dim][dim]
    const float* K0 = nullptr;         // level-0 values of the V-cycle (K32, or the mixed path's FP32 tangent)
    const float* minv0 = nullptr;      // their block-Jacobi inverse
    int64_t nnzb0 = 0;
    int g0 = 4;                        // lanes per block row of the level-0 matrix
    int deg_pre0 = 2, deg_post0 = 2;   // Chebyshev steps on level 0 before / after the coarse correction
    int deg_c = 2;                     // ... on the coarse levels (both sides)
    double* pw = nullptr;              // power-iteration work [2][n0] (FP64)
    float* pwf = nullptr;              // power-iteration work [2][n1] (FP32)
    float* pw0 = nullptr;              // level-0 eigenvector estimate, kept between refreshes [n0]
    bool pw0_valid = false;
    double* pw_part = nullptr;
    int nparts = 0;
    std::vector<void*> allocs;
    int launches = 0;
    // precise mode: levels >= 1, their Galerkin operators, the coarsest inverse and the level-0
    // residuals in FP64, the level-0 smoothing in FP32 on the residual equation (see amg_apply)
    int precise = 0;
    int deterministic = 0;             // 1: Galerkin products summed in a fixed order (no shared atomics)
    bool precise_ready = false;        // FP64 arrays allocated
    bool precise_valid = false;        // the FP64 coarse operators follow the last Galerkin refresh
    double* pwd = nullptr;             // FP64 power-iteration work [2][n1]
    // instrumentation (profile = 1): CUDA events around the level-0 pre-smoothing sweep of the
    // V-cycles of a chunk of Krylov iterations, as many as ev holds
    int profile = 0;
    cudaEvent_t ev[64] = {};
    int nev = 0;
    double smooth0_ms = 0.0;           // summed duration of the timed level-0 Chebyshev launches
    int smooth0_n = 0;                 // their number
};

// Instrumentation: add the first n_valid timed sweeps (V-cycles that did work) to smooth0_ms /
// smooth0_n and restart the event list.  Call after the stream has been synchronised.
void amg_profile_collect(AmgDev& D, int n_valid);

cudaError_t amg_upload(const AmgHierarchy& H, AmgDev& D, int num_sms);
void amg_free(AmgDev& D);
// New level-0 matrix A0 (with block-Jacobi inverse minv0): spectral estimate of level 0 and, when
// galerkin != 0, coarse operators R A P recomputed from A0 down the hierarchy (with their block
// inverses, spectral estimates and the coarsest dense inverse).  The FP64 overload first rounds A0
// and minv0 to FP32 copies; the FP32 overload (mixed path) uses the given arrays, which must stay
// valid until the next refresh.
// In precise mode (D.precise != 0) the FP64 overload builds the coarse operators in FP64 from A0's
// FP64 values.
cudaError_t amg_refresh(AmgDev& D, const BsrDev& A0, const double* minv0, int galerkin, cudaStream_t s);
cudaError_t amg_refresh(AmgDev& D, const BsrF& A0, const float* minv0, int galerkin, cudaStream_t s);
// One V-cycle: out = M^-1 in (level 0 uses the operator of the last refresh; A0 gives its pattern
// and free-DOF mask).  The FP64 overload in precise mode: FP32 pre-smoothing from zero, the FP64
// residual with A0's FP64 values, the FP64 coarse correction, the FP64 residual again, FP32
// smoothing of the correction equation from zero, and the sum in FP64; a refresh in precise mode
// must precede it.
// rec (may be null): the calling solver's record; every launch exits at once once rec->done is set.
cudaError_t amg_apply(AmgDev& D, const BsrDev& A0, const double* in, double* out, const KrylovRec* rec,
                      cudaStream_t s);
cudaError_t amg_apply(AmgDev& D, const BsrF& A0, const float* in, float* out, const KrylovRec* rec,
                      cudaStream_t s);

}  // namespace ep
