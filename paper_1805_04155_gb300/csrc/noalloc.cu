// ep_linear_solve_noalloc: the preconditioned Krylov solve of ep_linear_solve
// for callers that cannot allocate device memory, e.g. code running while
// another runtime owns the device's memory pool, or a phase that must not
// call cudaMalloc at all.  The caller passes the matrix, the right-hand side
// and the solution buffer; every other buffer the solver needs (its Krylov
// vectors, the preconditioner blocks, the partial sums of its deterministic
// reductions and its per-iteration scalars) lives in one file-scope device
// array of fixed size, which every GPU that loads this library holds until
// the process exits.  Calls share that array, so calls that overlap on the
// GPU (two streams, or two host threads) race; each call re-initialises
// everything it reads before use.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "ep_internal.h"

namespace ep {
namespace {

constexpr int64_t NOALLOC_MAX_DOF = EP_NOALLOC_MAX_DOF;
constexpr int NOALLOC_MAX_IT = EP_NOALLOC_MAX_ITERATIONS;
constexpr int NOALLOC_MAX_PARTS = 512;
// vectors: x is the caller's; r, z, p, q, rhat, v, s, t, phat, shat = 10 vectors
constexpr int64_t NV = 10;
constexpr int64_t OFF_MINV = NV * NOALLOC_MAX_DOF;                   // minv: <= 3 doubles per DOF
constexpr int64_t OFF_PART = OFF_MINV + 3 * NOALLOC_MAX_DOF;
constexpr int64_t OFF_HIST = OFF_PART + 8 * NOALLOC_MAX_PARTS;
constexpr int64_t OFF_REC = OFF_HIST + 3 * (NOALLOC_MAX_IT + 2);
constexpr int64_t SCRATCH_DOUBLES = OFF_REC + 8;

static __device__ __align__(256) double g_scratch[SCRATCH_DOUBLES];

std::mutex g_mu;
double* g_scratch_addr[64] = {nullptr};   // device address of g_scratch, per device id

}  // namespace
}  // namespace ep

using namespace ep;

#define g_err (ep::thread_error())

extern "C" ep_status ep_linear_solve_noalloc(int32_t dim, int64_t n_nodes, const int32_t* row_ptr,
                                             const int32_t* col_idx, const int32_t* diag_slot, const double* vals,
                                             const uint8_t* free_dof, const double* b, double* x, int32_t method,
                                             int32_t precond, double rtol, int32_t maxit, int32_t* iterations,
                                             double* rel_resid, void* cuda_stream) {
    if ((dim != 2 && dim != 3) || n_nodes <= 0 || !row_ptr || !col_idx || !diag_slot || !vals || !free_dof || !b ||
        !x) {
        g_err = "ep_linear_solve_noalloc: bad dimension, size or null pointer";
        return EP_ERR_INVALID_ARG;
    }
    if (n_nodes * dim > NOALLOC_MAX_DOF) {
        g_err = "ep_linear_solve_noalloc: " + std::to_string(n_nodes * dim) + " DOFs exceed the fixed workspace limit of " +
                std::to_string(NOALLOC_MAX_DOF) + " (EP_NOALLOC_MAX_DOF)";
        return EP_ERR_INVALID_ARG;
    }
    if (maxit < 1 || maxit > NOALLOC_MAX_IT) {
        g_err = "ep_linear_solve_noalloc: maxit must be in [1, " + std::to_string(NOALLOC_MAX_IT) + "]";
        return EP_ERR_INVALID_ARG;
    }
    if ((method != 1 && method != 2) || (precond != 0 && precond != 1) || !(rtol > 0.0)) {
        g_err = "ep_linear_solve_noalloc: method must be 1 (CG) or 2 (BiCGStab), precond 0 or 1, rtol > 0";
        return EP_ERR_INVALID_ARG;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        g_err = "ep_linear_solve_noalloc: no current CUDA device";
        return EP_ERR_CUDA;
    }
    double* base = nullptr;
    {
        // once per device, with that device current: the host-side symbol is only a stand-in, the
        // kernels need its device address
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_scratch_addr[dev]) {
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
            if (e != cudaSuccess) {
                g_err = std::string("ep_linear_solve_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e);
                return EP_ERR_CUDA;
            }
            g_scratch_addr[dev] = static_cast<double*>(p);
        }
        base = g_scratch_addr[dev];
    }
    int num_sms = 152;
    cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);

    KrylovWork w{};
    w.n = n_nodes * dim;
    w.block = 512;
    w.grid = std::min(2 * num_sms, NOALLOC_MAX_PARTS);
    w.nparts = w.grid;
    w.hist_len = NOALLOC_MAX_IT + 2;
    w.gm_m = 0;
    double** vecs[NV] = {&w.d.r, &w.d.z, &w.d.p, &w.d.q, &w.d.rhat, &w.d.v, &w.d.s, &w.d.t, &w.d.phat, &w.d.shat};
    for (int64_t i = 0; i < NV; ++i) *vecs[i] = base + i * NOALLOC_MAX_DOF;
    w.d.x = x;
    w.d.minv = base + OFF_MINV;
    w.part = base + OFF_PART;
    w.hist = base + OFF_HIST;
    w.rec = reinterpret_cast<KrylovRec*>(base + OFF_REC);
    KrylovRec rec_host{};
    w.rec_host = &rec_host;          // pageable host copy: no pinned allocation
    w.amg = nullptr;
    w.use_amg = 0;
    w.profile = 0;

    BsrDev A;
    A.n_rows = n_nodes;
    A.dim = dim;
    A.row_ptr = row_ptr;
    A.col_idx = col_idx;
    A.diag_slot = diag_slot;
    A.vals = vals;
    A.free_dof = free_dof;
    // the record must start clean: the previous call's contents stay in the array
    if (cudaMemsetAsync(w.rec, 0, sizeof(KrylovRec), s) != cudaSuccess) {
        g_err = "ep_linear_solve_noalloc: cudaMemsetAsync failed";
        return EP_ERR_CUDA;
    }
    cudaError_t e = krylov_precond(A, w, precond, s);
    int its = 0, st = EP_OK;
    double rel = 0.0;
    if (e == cudaSuccess) e = krylov_solve(A, w, b, method, rtol, maxit, s, &its, &rel, &st);
    if (e != cudaSuccess) {
        g_err = std::string("ep_linear_solve_noalloc: ") + cudaGetErrorString(e);
        return EP_ERR_CUDA;
    }
    if (iterations) *iterations = its;
    if (rel_resid) *rel_resid = rel;
    if (st != EP_OK) g_err = "ep_linear_solve_noalloc: no convergence within maxit, or breakdown";
    return (ep_status)st;
}

