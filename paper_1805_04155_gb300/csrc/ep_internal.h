// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/ep.h"

namespace ep {

// ---------------------------------------------------------------------------
// Element types: (family, dim) -> compile-time sizes.
// ---------------------------------------------------------------------------
enum ElemId { P1_2D = 0, P2_2D, Q1_2D, Q2_2D, P1_3D, P2_3D, Q1_3D, Q2_3D, N_ELEM_IDS };

inline int elem_id(int family, int dim) { return (dim == 2 ? 0 : 4) + family; }

template <int ID> struct Elem;
#define EP_ELEM(ID_, DIM_, NP_, NQ_, EPC_)                                   \
    template <> struct Elem<ID_> {                                           \
        static constexpr int ID = ID_, DIM = DIM_, NP = NP_, NQ = NQ_;       \
        static constexpr int NS = (DIM_ == 2 ? 3 : 6);  /* strain rows */    \
        static constexpr int NA = (DIM_ == 2 ? 4 : 6);  /* active components */ \
        static constexpr int EPC = EPC_;                /* elements per CTA */ \
    };
EP_ELEM(P1_2D, 2, 3, 1, 128)
EP_ELEM(P2_2D, 2, 6, 7, 32)
EP_ELEM(Q1_2D, 2, 4, 4, 64)
EP_ELEM(Q2_2D, 2, 8, 9, 16)
EP_ELEM(P1_3D, 3, 4, 1, 64)
EP_ELEM(P2_3D, 3, 10, 11, 4)
EP_ELEM(Q1_3D, 3, 8, 8, 8)
EP_ELEM(Q2_3D, 3, 20, 27, 1)
#undef EP_ELEM

inline int elem_np(int id) { static const int v[] = {3, 6, 4, 8, 4, 10, 8, 20}; return v[id]; }
inline int elem_nq(int id) { static const int v[] = {1, 7, 4, 9, 1, 11, 8, 27}; return v[id]; }

// ---------------------------------------------------------------------------
// Material constants as the kernels use them.
// ---------------------------------------------------------------------------
struct MatConst {
    int model;
    double K, G;        // bulk and shear moduli
    double Y, H;        // von Mises yield value and hardening modulus
    double eta, c, eta_bar, Hc;   // Drucker-Prager
    // reciprocals computed once on the host (FP64 divisions are costly on the device)
    double inv_vm;      // 1 / (2G + H)
    double inv_den_s;   // 1 / (G + K eta eta_bar + Hc)
    double inv_den_a;   // 1 / (K eta eta_bar + Hc), 0 when that is 0
    double inv_3K;      // 1 / (3K)
};

// ---------------------------------------------------------------------------
// Device-side views passed to kernels.
// ---------------------------------------------------------------------------
struct MeshDev {
    int64_t n_nodes, n_elem, n_int;
    const int32_t* elem_nodes;  // [n_elem][n_p]
    const int32_t* slots;       // [n_elem][n_p*n_p], block index of node pair (p, q)
    const double* dphi;         // [n_int][n_p][dim], physical basis gradients
    const double* wgt;          // [n_int]
    const MatConst* mat_table;  // material constants, >= 1 entry
    const int32_t* elem_mat;    // [n_elem] index into mat_table (null: every element uses entry 0)
};

// The material of element e.
__host__ __device__ inline const MatConst& elem_material(const MeshDev& m, int64_t e) {
    return m.mat_table[m.elem_mat ? m.elem_mat[e] : 0];
}

struct StateDev {
    double* ep;       // [n_comp][n_int]
    double* hard;     // [n_int] or [n_comp][n_int]
    double* sig;      // [n_comp][n_int]
    uint8_t* flag;    // [n_int]
};

enum AsmMode { ASM_FULL = 0, ASM_DELTA = 1 };

// Launchers defined per element type (asm_<type>.cu).
struct AsmArgs {
    MeshDev mesh;
    MatConst mat;
    StateDev state;
    const double* u;           // [n_dof]
    double* F;                 // [n_dof], accumulated (caller zeroes)
    double* Kvals;             // [nnzb][dim][dim], accumulated (caller initialises)
    float* Kvals32;            // non-null: the tangent is formed in FP32 and accumulated here instead of Kvals
    int mode;                  // AsmMode
    int want_K;                // 0: F only
    int elastic_only;          // 1: D = C everywhere (K_elast assembly), u/state ignored
    unsigned long long* n_plastic;  // device counter (may be null)
    int* err_flag;             // device error word (return-map failures)
    // split mode with want_K: every slot a plastic element adds to is marked 1 here (may be null)
    uint8_t* dirty;
    unsigned long long* n_plastic_elem;   // device counter of elements with a plastic point (may be null)
    // deterministic form: the launch covers the list_n elements elem_list[0 .. list_n) (one colour:
    // no two share a node) and adds into F and K with plain stores; null = elements 0 .. n_elem
    // in order, FP64/FP32 atomics
    const int32_t* elem_list;
    int64_t list_n;
    int tile;                  // assembly schedule: 1 the element type's tile of elements per CTA, 2 half of it
};
cudaError_t launch_assemble(int elem_id, const AsmArgs& a, cudaStream_t s);

// Split-mode reset of eq. (K-split): Kt[b] = Kel[b] for every block b marked in dirty (blocks of d2
// values), and the marks cleared.
cudaError_t launch_reset_dirty(uint8_t* dirty, int64_t nnzb, int d2, const double* Kel, double* Kt, int grid,
                               cudaStream_t s);
cudaError_t launch_reset_dirty(uint8_t* dirty, int64_t nnzb, int d2, const float* Kel, float* Kt, int grid,
                               cudaStream_t s);

struct CommitArgs {
    MeshDev mesh;
    MatConst mat;
    StateDev state;            // updated in place
    const double* u;
    unsigned long long* n_plastic;
    int* err_flag;
};
cudaError_t launch_commit(int elem_id, const CommitArgs& a, cudaStream_t s);

struct GeomArgs {
    int64_t n_elem, n_int;
    const double* coords;      // [n_nodes][dim]
    const int32_t* elem_nodes;
    const double* dhat;        // [n_q][n_p][dim] reference gradients
    const double* wq;          // [n_q]
    double* dphi;
    double* wgt;
    int* bad_count;            // number of points with det J <= 0
};
cudaError_t launch_geometry(int elem_id, const GeomArgs& a, cudaStream_t s);

cudaError_t launch_constitutive(int dim, const MatConst& m, int64_t n, const double* E, const double* ep_prev,
                                const double* hard_prev, double* S, double* DS, uint8_t* flag, double* ep_new,
                                double* hard_new, cudaStream_t s);

// Message of the last failed context-free call (ep_create, ep_linear_solve_noalloc) on this thread.
std::string& thread_error();

// Host-side reference tables (elements_host.cpp): gradients [n_q][n_p][dim], weights [n_q].
void reference_tables(int family, int dim, std::vector<double>& dhat, std::vector<double>& wq);

// Host-side pattern construction (pattern_host.cpp).
// Builds the node-pair pattern (row_ptr [n_nodes+1], col_idx) and the slot map
// slots [n_elem][n_p*n_p] (block index of each node pair).  Returns false on
// invalid node indices.
bool build_pattern(int64_t n_nodes, int64_t n_elem, int n_p, const int32_t* elem, std::vector<int32_t>& row_ptr,
                   std::vector<int32_t>& col_idx, std::vector<int32_t>& slots, std::string& err);

// Element colouring (pattern_host.cpp): elements of one colour share no node.  color_ptr
// [n_colors + 1], color_elems [n_elem] (the elements of colour c are color_elems[color_ptr[c] ..
// color_ptr[c + 1]), in increasing order).  Returns false on invalid node indices.
bool color_elements(int64_t n_nodes, int64_t n_elem, int n_p, const int32_t* elem, std::vector<int32_t>& color_ptr,
                    std::vector<int32_t>& color_elems, std::string& err);

// ---------------------------------------------------------------------------
// Krylov solver on the block-CSR matrix (krylov.cu).
// ---------------------------------------------------------------------------
template <class T>
struct BsrT {
    int64_t n_rows;            // node rows
    int dim;
    const int32_t* row_ptr;
    const int32_t* col_idx;
    const int32_t* diag_slot;  // [n_rows] block index of the diagonal block
    const T* vals;             // [nnzb][dim][dim]
    const uint8_t* free_dof;   // [n_rows*dim], 1 = free
    const int32_t* perm = nullptr;   // SpMV row order (rows grouped by length, a permutation of
                                     // 0..n_rows-1), or null for the natural order
};
using BsrDev = BsrT<double>;   // the FP64 tangent
using BsrF = BsrT<float>;      // the FP32 tangent of the mixed path

// Per-solve scalar record, written by the device, read by the host.
struct KrylovRec {
    int its;          // iterations done
    int done;         // 1 converged, 2 breakdown, 3 iteration cap
    double rr0;       // ||r_0||^2
    double rr;        // ||r||^2 of the last iterate
    int why;          // which test ended the solve (diagnostics): 1 converged, 2 non-finite, 3 rho = 0,
                      // 4 (rhat, v) = 0, 5 omega = 0, 6 iteration cap
    int pad;
};

struct AmgDev;
struct DirectDev;

// Solver vectors of one precision.
template <class T>
struct KVecs {
    T *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *rhat = nullptr, *v = nullptr,
      *s = nullptr, *t = nullptr, *phat = nullptr, *shat = nullptr;
    T* minv = nullptr;       // preconditioner: [n_rows][dim][dim]
    T* V = nullptr;          // GMRES basis [GM_M + 1][n]
};

struct KrylovWork {
    int64_t n;               // vector length (n_rows*dim)
    int nparts;              // partial-sum slots per reduction
    int grid, block;         // launch shape of the vector/SpMV kernels
    KVecs<double> d;         // FP64 solver (allocated by krylov_alloc)
    KVecs<float> f;          // FP32 solver of the mixed path (allocated by krylov_alloc_f32 on first use)
    double* part;            // [max(8, GM_M + 2)][nparts] partial sums
    double* gm;              // GMRES small arrays: H [(GM_M+1) x GM_M], cs, sn, g [GM_M+1]
    double* hist;            // [3][maxit+2] rho, alpha, omega per iteration
    int hist_len;
    KrylovRec* rec;          // device
    KrylovRec* rec_host;     // pinned host mirror
    AmgDev* amg;             // AMG hierarchy (precond 2), owned by the context; null if not built
    int use_amg;             // set by krylov_precond: 1 when the current preconditioner is the AMG V-cycle
    DirectDev* direct = nullptr;   // sparse LU (precond 3), owned by the context; null if not set up
    int use_direct = 0;      // set by krylov_precond: 1 when the current preconditioner is the sparse LU
    int gm_m;                // GMRES restart length (<= GM_M)
    int galerkin;            // 1: recompute the AMG coarse operators from the current matrix in krylov_precond
    int last_its;            // iterations of the previous solve: sizes the first chunk of launches of the next
    int stall_guard;         // 1: an FP32-basis GMRES stops when a restart cycle does not halve the residual
    int stall_guard64;       // 1: an FP64 GMRES stops when a restart cycle after the first gains less than 10%
    // instrumentation
    int profile;             // 1: CUDA events around every SpMV launch
    int verbose;             // 2: per-cycle host enqueue / wait times on stderr
    // CUDA graphs of GMRES iterations (graphs = 1, profile = 0): iteration j of a restart cycle (the
    // preconditioner, the SpMV, the orthogonalisation and the Givens/norm kernels, about 30 launches
    // with the V-cycle) is captured once per solver configuration and replayed with one
    // cudaGraphLaunch; the per-solve scalars the captured kernels read (tolerance, iteration base
    // and cap) live in gdyn on the device
    int graphs = 0;
    double* gdyn = nullptr;            // device [3]: rtol^2, iterations before this cycle, cap
    // GMRES with the sparse LU keeps z_j = M^-1 v_j of the cycle ([z_cap][n], allocated on first
    // use) and updates x += Z y: no preconditioner solve at the end of a cycle
    void* Z = nullptr;
    int z_cap = 0, z_bytes = 0;
    cudaStream_t cap_stream = nullptr; // private stream the captures are made on
    std::vector<cudaGraphExec_t> gexec;
    std::vector<int> gexec_launches;   // kernels inside each graph
    long long gkey = -1;               // configuration the cached graphs were captured for
    const void* gkey_ptr = nullptr;
    int graph_launches = 0;            // graph launches (accumulates)
    int launches;            // kernels launched by the solver (accumulates)
    int spmv_n;              // SpMV launches that did work (profile = 1)
    double spmv_ms;          // their summed duration
    cudaEvent_t ev[2 * 32];
};

constexpr int GM_M = 128;    // largest GMRES restart length (buffers); the run-time length is KrylovWork::gm_m
cudaError_t krylov_alloc(KrylovWork& w, int64_t n_rows, int dim, int maxit_cap, int num_sms);
cudaError_t krylov_alloc_f32(KrylovWork& w, int64_t n_rows, int dim);
void krylov_free(KrylovWork& w);
// Preconditioner of A (kind 0 Jacobi, 1 block Jacobi, 2 AMG with block-Jacobi smoothing, 3 the sparse
// LU of w.direct, which must be set up) in A's precision.
cudaError_t krylov_precond(const BsrDev& A, KrylovWork& w, int kind, cudaStream_t s);
cudaError_t krylov_precond(const BsrF& A, KrylovWork& w, int kind, cudaStream_t s);
// The sparse LU's current factors (of an earlier matrix) as the preconditioner of the next solve,
// without refactoring; false if none have been computed.
bool krylov_keep_direct(KrylovWork& w);
// Solves A x = b on the free DOFs; x starts at zero.  method 1 CG, 2 BiCGStab, 3 GMRES(m).
// The FP64 overload works on w.d, the FP32 overload on w.f (solution in w.f.x).
// Returns cudaSuccess; *status receives EP_OK / EP_ERR_KRYLOV / EP_ERR_NAN.
cudaError_t krylov_solve(const BsrDev& A, KrylovWork& w, const double* b, int method, double rtol, int maxit,
                         cudaStream_t s, int* its, double* relres, int* status);
cudaError_t krylov_solve(const BsrF& A, KrylovWork& w, const float* b, int method, double rtol, int maxit,
                         cudaStream_t s, int* its, double* relres, int* status);
// GMRES with the FP64 operator and an FP32 basis (w.f's V, z and preconditioner; solution w.d.x):
// the operator keeps FP64 accuracy (no cancellation error on the soft modes) while the
// orthogonalisation and the preconditioner move FP32 vectors.  Needs krylov_precond(A) first.
cudaError_t krylov_solve_fp32_basis(const BsrDev& A, KrylovWork& w, const double* b, double rtol, int maxit,
                                    cudaStream_t s, int* its, double* relres, int* status);

// Small vector kernels (krylov.cu).
// r = (zeta f_unit - F) on the free DOFs (and its FP32 copy r32 when non-null); out3 = (||r||^2, ||f||^2, ||F||^2).
cudaError_t vec_residual(const double* f_unit, double zeta, const double* F, const uint8_t* free_dof, double* r,
                         float* r32, int64_t n, double* part, int nparts, double* out3, cudaStream_t s);
cudaError_t vec_axpy_f32(double* y, const float* x, int64_t n, cudaStream_t s);   // y += x
// Residual norms per DOF chunk (see k_chunk_norms): out = [r^2 | f^2 | F^2][nc].
cudaError_t vec_chunk_norms(const double* f_unit, double zeta, const double* F, const uint8_t* free_dof,
                            const double* r, const int64_t* chunks, int64_t nc, double* out, cudaStream_t s);
cudaError_t vec_cvt_f32(const double* x, float* y, int64_t n, cudaStream_t s);    // y = (float) x
cudaError_t vec_cvt_f64(const float* x, double* y, int64_t n, cudaStream_t s);    // y = (double) x
cudaError_t vec_axpy(double* y, double a, const double* x, int64_t n, cudaStream_t s);
cudaError_t vec_set_dirichlet(double* u, const double* uD_unit, double zeta, const uint8_t* free_dof, int64_t n,
                              cudaStream_t s);
cudaError_t vec_extrapolate(double* u, const double* u_prev, double ratio, int64_t n, cudaStream_t s);
cudaError_t vec_mask_copy(double* dst, const double* src, const uint8_t* free_dof, int64_t n, cudaStream_t s);

// ---------------------------------------------------------------------------
// Learned warm start (warm_start.cu): node features, targets and the start correction.
// node_prob: [n_nodes] problem of each node, or null (one problem).
// ---------------------------------------------------------------------------
// cnt[node] += points of the adjacent elements (flag null) or their plastic points (flag != 0);
// the caller zeroes cnt.
cudaError_t ws_node_counts(const int32_t* elem, int64_t n_elem, int n_p, int n_q, const uint8_t* flag, int32_t* cnt,
                           cudaStream_t s);
// pf = cnt_pl / cnt_ip per node (0 where cnt_ip = 0).
cudaError_t ws_fraction(const int32_t* cnt_pl, const int32_t* cnt_ip, int64_t n_nodes, float* pf, cudaStream_t s);
// scale [2][n_prob]: s_p = RMS of (u1 - u2) over the DOFs [prob_dof[p], prob_dof[p+1]) and 1/s_p (0 if s_p = 0).
cudaError_t ws_scale(const double* u1, const double* u2, const int64_t* prob_dof, int n_prob, double* scale,
                     cudaStream_t s);
// X [n_nodes][16]: the network inputs of step k (u1, u2, u3 = u_{k-1}, u_{k-2}, u_{k-3}; pf1, pf2 the
// plastic fractions after k-1, k-2; prox1 the yield proximity after k-1; stat [n_nodes][5]).
cudaError_t ws_features(const double* u1, const double* u2, const double* u3, const int32_t* node_prob,
                        const double* scale, int n_prob, int dim, int64_t n_nodes, double r_k, double r_k1,
                        const float* pf1, const float* pf2, const float* prox1, const float* stat, float* X,
                        cudaStream_t s);
// prox [n_nodes]: the largest yield proximity of the committed state over the points of the adjacent
// elements (sig [n_comp][n_int], hard [n_int] or [n_comp][n_int]).
cudaError_t ws_proximity(const MeshDev& mesh, const double* sig, const double* hard, int n_p, int n_q, int dim,
                         float* prox, cudaStream_t s);
// Y[:, 0..dim) <- its projection, per problem and component, onto the span of X[:, c], X[:, 3 + c].
cudaError_t ws_project(const float* X, float* Y, const uint8_t* free_dof, const int64_t* prob_dof, int n_prob,
                       int dim, cudaStream_t s);
// u += s_p * Y[node][c] on free DOFs.
cudaError_t ws_apply(double* u, const float* Y, const int32_t* node_prob, const double* scale, int n_prob,
                     const uint8_t* free_dof, int dim, int64_t n_dof, cudaStream_t s);
// T [n_nodes][4]: ((u_k - (u1 + ratio (u1 - u2))) / s_p on free DOFs, 0 elsewhere; pf_k).
cudaError_t ws_targets(const double* uk, const double* u1, const double* u2, double ratio, const int32_t* node_prob,
                       const double* scale, int n_prob, const uint8_t* free_dof, const float* pf_k, int dim,
                       int64_t n_nodes, float* T, cudaStream_t s);
// u = u_alt on the DOFs of every problem p with take_alt[p] != 0.
cudaError_t ws_select(double* u, const double* u_alt, const int32_t* node_prob, const uint8_t* take_alt, int dim,
                      int64_t n_dof, cudaStream_t s);
// The network (opaque ep_mlp_* handle): Y [n][4] = net(X [n][16]) on stream s.
cudaError_t mlp_forward_on(void* mlp, const float* X, int64_t n, float* Y, cudaStream_t s);
// Waits for the network's own stream (its parameters may still be being written by a training step).
cudaError_t mlp_sync(void* mlp);

}  // namespace ep
