// C-ABI entry points and the Newton / load-path driver (Section 4, ALG-NEWTON).
//
// Each Newton iteration on the device: assemble F(u) and K(u) (fused kernel,
// Section 7), residual r = f_k - F on the free DOFs with its norms, Krylov
// solve of K dr = r (eq. (lin_syst)), update u += du.  After convergence the
// state is committed (Sections 2.2, 2.3).  The only per-iteration device-to-
// host traffic is the three residual norms and the Krylov record.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "amg.h"
#include "direct.h"
#include "ep_internal.h"

namespace ep {

cudaError_t launch_assemble_0(const AsmArgs&, cudaStream_t);
cudaError_t launch_assemble_1(const AsmArgs&, cudaStream_t);
cudaError_t launch_assemble_2(const AsmArgs&, cudaStream_t);
cudaError_t launch_assemble_3(const AsmArgs&, cudaStream_t);
cudaError_t launch_assemble_4(const AsmArgs&, cudaStream_t);
cudaError_t launch_assemble_5(const AsmArgs&, cudaStream_t);
cudaError_t launch_assemble_6(const AsmArgs&, cudaStream_t);
cudaError_t launch_assemble_7(const AsmArgs&, cudaStream_t);
cudaError_t launch_commit_0(const CommitArgs&, cudaStream_t);
cudaError_t launch_commit_1(const CommitArgs&, cudaStream_t);
cudaError_t launch_commit_2(const CommitArgs&, cudaStream_t);
cudaError_t launch_commit_3(const CommitArgs&, cudaStream_t);
cudaError_t launch_commit_4(const CommitArgs&, cudaStream_t);
cudaError_t launch_commit_5(const CommitArgs&, cudaStream_t);
cudaError_t launch_commit_6(const CommitArgs&, cudaStream_t);
cudaError_t launch_commit_7(const CommitArgs&, cudaStream_t);
cudaError_t launch_geometry_0(const GeomArgs&, cudaStream_t);
cudaError_t launch_geometry_1(const GeomArgs&, cudaStream_t);
cudaError_t launch_geometry_2(const GeomArgs&, cudaStream_t);
cudaError_t launch_geometry_3(const GeomArgs&, cudaStream_t);
cudaError_t launch_geometry_4(const GeomArgs&, cudaStream_t);
cudaError_t launch_geometry_5(const GeomArgs&, cudaStream_t);
cudaError_t launch_geometry_6(const GeomArgs&, cudaStream_t);
cudaError_t launch_geometry_7(const GeomArgs&, cudaStream_t);

cudaError_t launch_assemble(int id, const AsmArgs& a, cudaStream_t s) {
    switch (id) {
        case 0: return launch_assemble_0(a, s);
        case 1: return launch_assemble_1(a, s);
        case 2: return launch_assemble_2(a, s);
        case 3: return launch_assemble_3(a, s);
        case 4: return launch_assemble_4(a, s);
        case 5: return launch_assemble_5(a, s);
        case 6: return launch_assemble_6(a, s);
        case 7: return launch_assemble_7(a, s);
    }
    return cudaErrorInvalidValue;
}
cudaError_t launch_commit(int id, const CommitArgs& a, cudaStream_t s) {
    switch (id) {
        case 0: return launch_commit_0(a, s);
        case 1: return launch_commit_1(a, s);
        case 2: return launch_commit_2(a, s);
        case 3: return launch_commit_3(a, s);
        case 4: return launch_commit_4(a, s);
        case 5: return launch_commit_5(a, s);
        case 6: return launch_commit_6(a, s);
        case 7: return launch_commit_7(a, s);
    }
    return cudaErrorInvalidValue;
}
cudaError_t launch_geometry(int id, const GeomArgs& a, cudaStream_t s) {
    switch (id) {
        case 0: return launch_geometry_0(a, s);
        case 1: return launch_geometry_1(a, s);
        case 2: return launch_geometry_2(a, s);
        case 3: return launch_geometry_3(a, s);
        case 4: return launch_geometry_4(a, s);
        case 5: return launch_geometry_5(a, s);
        case 6: return launch_geometry_6(a, s);
        case 7: return launch_geometry_7(a, s);
    }
    return cudaErrorInvalidValue;
}

// Material constants: K, G from E, nu; Drucker-Prager eta, c, eta_bar from
// (c0, phi, psi) by the 3D or plane-strain formulas of Section 8.3.
bool make_matconst(const ep_material& m, int dim, MatConst& out, std::string& err) {
    if (!(m.E > 0.0) || !(m.nu > -1.0 && m.nu < 0.5)) {
        err = "material: need E > 0 and -1 < nu < 0.5";
        return false;
    }
    if (m.model < 0 || m.model > 3) {
        err = "material: unknown model";
        return false;
    }
    out = MatConst{};
    out.model = m.model;
    out.K = m.E / (3.0 * (1.0 - 2.0 * m.nu));
    out.G = m.E / (2.0 * (1.0 + m.nu));
    out.Y = m.Y;
    out.H = m.H;
    if ((m.model == 1 || m.model == 2) && (!(m.Y > 0.0) || !(m.H >= 0.0))) {
        err = "material: von Mises needs Y > 0 and H >= 0";
        return false;
    }
    if (m.model == 3) {
        if (!(m.c0 >= 0.0) || !(m.phi >= 0.0 && m.phi < 1.5707963267948966) || !(m.psi >= 0.0 && m.psi < 1.5707963267948966) ||
            !(m.Hc >= 0.0)) {
            err = "material: Drucker-Prager needs c0 >= 0, 0 <= phi, psi < pi/2, Hc >= 0";
            return false;
        }
        if (dim == 3) {
            const double sp = std::sin(m.phi), ss = std::sin(m.psi);
            out.eta = 6.0 * sp / (std::sqrt(3.0) * (3.0 + sp));
            out.c = m.c0 * 6.0 * std::cos(m.phi) / (std::sqrt(3.0) * (3.0 + sp));
            out.eta_bar = 6.0 * ss / (std::sqrt(3.0) * (3.0 + ss));
        } else {
            const double tp = std::tan(m.phi), ts = std::tan(m.psi);
            const double qp = std::sqrt(9.0 + 12.0 * tp * tp), qs = std::sqrt(9.0 + 12.0 * ts * ts);
            out.eta = 3.0 * tp / qp;
            out.c = 3.0 * m.c0 / qp;
            out.eta_bar = 3.0 * ts / qs;
        }
        out.Hc = m.Hc;
    }
    out.inv_vm = 1.0 / (2.0 * out.G + out.H);
    const double den_a = out.K * out.eta * out.eta_bar + out.Hc;
    out.inv_den_s = 1.0 / (out.G + den_a);
    out.inv_den_a = den_a != 0.0 ? 1.0 / den_a : 0.0;
    out.inv_3K = 1.0 / (3.0 * out.K);
    return true;
}

// Smallest relative tolerance asked of the FP32 inner Krylov solve of the mixed path.
constexpr double MIXED_ETA_MIN = 1e-5;
// A Newton iteration on the FP32 tangent that reduces the FP64 residual by less than this factor
// ends the FP32 phase: the rest of the load path uses the FP64 tangent and solve.  Near a limit
// load the tangent is so ill-conditioned that its FP32 rounding (relative 2^-24 per entry) moves
// the soft modes by O(1), and Newton on it stalls.
constexpr double MIXED_STALL_RATIO = 0.5;
// Newton on an FP32 tangent contracts linearly, by about kappa * 2^-24 per iteration (kappa the
// tangent's condition number), where Newton on the FP64 tangent contracts by about its Krylov
// tolerance eta.  When an FP32 iteration of the mixed path reduced the FP64 residual by less than
// 1 / (MIXED_RHO_FACTOR * eta), the FP32 tangent limits Newton: the step continues, from the same
// iterate (re-assembled), with the FP64 tangent.
constexpr double MIXED_RHO_FACTOR = 10.0;

// Learned warm start: the history the node features need, and recorded training rows.
struct WsState {
    void* mlp = nullptr;            // attached network (warm_start = 2), not owned
    bool ready = false;             // buffers allocated, history tracked at every commit
    int hist = 0;                   // converged steps since the history started
    double* u3 = nullptr;           // u_{k-3}
    double zeta3 = 0.0;             // zeta_{k-3}
    int32_t *cnt_ip = nullptr, *cnt_pl = nullptr, *node_prob = nullptr;
    int64_t* prob_dof = nullptr;    // device [n_prob + 1]
    float *pf1 = nullptr, *pf2 = nullptr, *pfk = nullptr;   // plastic fractions after k-1, k-2, k
    float* prox1 = nullptr;         // yield proximity after step k-1
    float* stat = nullptr;          // [n_nodes][5] static inputs
    double* uL = nullptr;           // the learned start of the last step that computed one
    bool uL_valid = false;
    double* scale = nullptr;        // [2][n_prob]: s_p, 1/s_p
    float *X = nullptr, *Y = nullptr;   // inputs / outputs of one step when not recording
    double* u_ex = nullptr;         // the plain extrapolated start
    uint8_t* take_ex = nullptr;     // device [n_prob]: the problem keeps the plain extrapolation
    std::vector<uint8_t> h_take;
    float *rec_X = nullptr, *rec_T = nullptr;   // recorded rows [rec_cap][16], [rec_cap][4]
    int64_t rec_cap = 0, rec_n = 0;
};

struct Ctx {
    std::string err;
    int device = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 152;
    int dim = 0, family = 0, eid = 0, n_p = 0, n_q = 0, n_comp = 0;
    int64_t n_nodes = 0, n_elem = 0, n_int = 0, n_dof = 0, nnzb = 0, hard_len = 0;
    MatConst mat{};                 // material of entry 0 (the model and the symmetry test)
    MatConst* mat_table = nullptr;  // device [n_mat]
    int32_t* elem_mat = nullptr;    // device [n_elem] or null (one material)
    int n_mat = 1;
    // batch of independent problems: problem p owns DOFs [prob_dof[p], prob_dof[p + 1])
    int n_prob = 1;
    std::vector<int64_t> prob_dof;
    std::vector<int64_t> chunk_prob, chunk_beg, chunk_end;   // residual-norm chunks (host copy)
    int64_t* d_chunks = nullptr;    // device [3][n_chunks]: problem, begin, end
    double* d_chunk_norms = nullptr;   // device [3][n_chunks]
    std::vector<double> h_chunk_norms;
    // mesh and pattern
    double* coords = nullptr;
    int32_t *elem = nullptr, *slots = nullptr, *row_ptr = nullptr, *col_idx = nullptr, *diag_slot = nullptr;
    int32_t* spmv_perm = nullptr;   // SpMV row order: rows grouped by their number of blocks
    double *dphi = nullptr, *wgt = nullptr;
    double *Kel = nullptr, *Kt = nullptr;
    // mixed path (allocated on first use): FP32 tangent, FP32 K_elast, FP32 right-hand side
    float *K32 = nullptr, *Kel32 = nullptr, *r32 = nullptr;
    // state
    double *ep = nullptr, *hard = nullptr, *sig = nullptr;
    uint8_t* flag = nullptr;
    // vectors
    double *u = nullptr, *u_prev = nullptr, *u_it = nullptr, *F = nullptr, *r = nullptr;
    double *f_unit = nullptr, *uD_unit = nullptr;
    uint8_t* free_dof = nullptr;
    // scalars
    unsigned long long* counter = nullptr;
    int* err_flag = nullptr;
    double* norms = nullptr;        // device [3]
    double* norms_host = nullptr;   // pinned [3]
    unsigned long long* counter_host = nullptr;
    int* err_host = nullptr;
    KrylovWork kw{};
    bool K_valid = false;      // Kt holds the tangent of the last assembly
    bool K32_valid = false;    // K32 holds the tangent of the last assembly
    // split form (eq. (K-split)): Kt (K32) equals K_elast (Kel32) outside the blocks marked in dirty64
    // (dirty32); a split assembly resets just those blocks before adding the new plastic terms
    uint8_t *dirty64 = nullptr, *dirty32 = nullptr;
    // deterministic form (ep_opts.deterministic): element colours, one assembly launch per colour
    int deterministic = 0;
    int asm_tile = 1;                   // assembly schedule (ep_opts.asm_tile)
    // Eisenstat-Walker forcing terms of the inexact Newton iteration: the first iteration of a step
    // and the cap, FP64 path and mixed path (tuning knobs EP_NEWTON_ETA0, EP_NEWTON_ETA_MAX set
    // both).  Measured on the 256x256 P2 column, FP64: (1e-3, 1e-2) 0.307 s, (1e-2, 1e-2) 0.288 s,
    // (3e-2, 3e-2) 0.275 s per load path, 17 Newton iterations each (the final iterations take the
    // floor 0.5 tol ||f|| / ||r|| anyway); mixed: (3e-2, 3e-2) 0.333 s and 23 Newton iterations
    // against 0.322 s and 17 with (1e-3, 1e-2) -- its FP32 phase hands over to FP64 by comparing
    // an iteration's contraction with the forcing term, so a looser term keeps it longer on the
    // FP32 tangent.
    double eta0 = 3e-2, eta_max = 3e-2, eta0_mixed = 1e-3, eta_max_mixed = 1e-2;
    std::vector<int32_t> h_color_ptr;   // [n_colors + 1]
    int32_t* color_elems = nullptr;     // device [n_elem]
    bool split_base64 = false, split_base32 = false;   // the statement above holds
    int reset_grid = 0;
    int n_committed = 0;
    double zeta_last = 0.0, zeta_prev = 0.0;
    cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    int launches = 0;          // kernels launched (instrumentation)
    int profile = 0;
    int verbose = 0;           // EP_VERBOSE=1: one line per Newton iteration on stderr
    // host copies kept for the AMG setup
    std::vector<int32_t> h_row_ptr, h_col_idx;
    std::vector<double> h_coords;
    std::vector<uint8_t> h_free;
    AmgDev amg;
    // sparse LU (precond 3): set up on first use; direct_mode = the Newton loop solves with it for
    // the rest of the load path (switched on when a GMRES solve with the V-cycle stalled)
    DirectDev direct;
    bool direct_mode = false;
    double direct_setup_ms = 0.0;
    bool amg_built = false;
    bool amg_elastic = true;     // the AMG coarse operators currently come from K_elast
    int64_t amg_np = -1;         // plastic points of the tangent the coarse operators were last built from
    bool mixed_fallback = false; // the mixed path has switched to FP64 for the rest of the load path
    double amg_setup_ms = 0.0;
    WsState ws;
    std::vector<float> h_node_static;   // [n_nodes][5] static warm-start inputs (host, built at creation)
    std::vector<int32_t> h_node_prob;   // [n_nodes] problem of each node (batches only)
    std::vector<void*> allocs;
};

static ep_status cuda_fail(Ctx* c, cudaError_t e, const char* where) {
    if (c) c->err = std::string(where) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? EP_ERR_OOM : EP_ERR_CUDA;
}

#define CK(call)                                                    \
    do {                                                            \
        cudaError_t _e = (call);                                    \
        if (_e != cudaSuccess) return cuda_fail(c, _e, #call);      \
    } while (0)

template <class T>
static cudaError_t dalloc(Ctx* c, T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
    if (e == cudaSuccess) c->allocs.push_back((void*)*p);
    return e;
}

static MeshDev mesh_dev(const Ctx* c) {
    MeshDev m;
    m.n_nodes = c->n_nodes;
    m.n_elem = c->n_elem;
    m.n_int = c->n_int;
    m.elem_nodes = c->elem;
    m.slots = c->slots;
    m.dphi = c->dphi;
    m.wgt = c->wgt;
    m.mat_table = c->mat_table;
    m.elem_mat = c->elem_mat;
    return m;
}

static StateDev state_dev(const Ctx* c) { return StateDev{c->ep, c->hard, c->sig, c->flag}; }

template <class T>
static BsrT<T> bsr_dev(const Ctx* c, const T* vals) {
    BsrT<T> b;
    b.n_rows = c->n_nodes;
    b.dim = c->dim;
    b.row_ptr = c->row_ptr;
    b.col_idx = c->col_idx;
    b.diag_slot = c->diag_slot;
    b.vals = vals;
    b.free_dof = c->free_dof;
    b.perm = c->spmv_perm;
    return b;
}

// Buffers of the mixed path, on first use: K32, r32, the FP32 solver vectors, and K_elast rounded
// once to FP32 (the split path's starting matrix).
static ep_status ensure_mixed(Ctx* c) {
    if (c->K32) return EP_OK;
    const int64_t nk = c->nnzb * c->dim * c->dim;
    CK(dalloc(c, &c->K32, nk));
    CK(dalloc(c, &c->Kel32, nk));
    CK(dalloc(c, &c->dirty32, c->nnzb));
    c->split_base32 = false;
    CK(dalloc(c, &c->r32, c->n_dof));
    CK(krylov_alloc_f32(c->kw, c->n_nodes, c->dim));
    CK(vec_cvt_f32(c->Kel, c->Kel32, nk, c->stream));
    c->launches += 1;
    return EP_OK;
}

// Assemble F and K at u_dev with the committed state.  split: K = K_elast + plastic deltas.
// mixed: the tangent is formed in FP32 into K32 (F, strains and return mapping stay FP64).
static ep_status assemble(Ctx* c, const double* u_dev, bool split, bool want_K, bool mixed) {
    cudaStream_t s = c->stream;
    CK(cudaMemsetAsync(c->F, 0, sizeof(double) * c->n_dof, s));
    CK(cudaMemsetAsync(c->counter, 0, 2 * sizeof(unsigned long long), s));
    if (mixed) {
        ep_status st = ensure_mixed(c);
        if (st != EP_OK) return st;
    }
    const size_t nk = (size_t)c->nnzb * c->dim * c->dim;
    const int d2 = c->dim * c->dim;
    uint8_t* dirty = mixed ? c->dirty32 : c->dirty64;
    bool& base = mixed ? c->split_base32 : c->split_base64;
    if (want_K && split) {
        // eq. (K-split): K = K_elast + sum over plastic elements.  The blocks the last split assembly
        // moved away from K_elast get K_elast's values back (only those: an elastic tangent costs
        // nothing here); the first split assembly after a full one copies K_elast whole.
        if (!base) {
            if (mixed) CK(cudaMemcpyAsync(c->K32, c->Kel32, sizeof(float) * nk, cudaMemcpyDeviceToDevice, s));
            else CK(cudaMemcpyAsync(c->Kt, c->Kel, sizeof(double) * nk, cudaMemcpyDeviceToDevice, s));
            CK(cudaMemsetAsync(dirty, 0, c->nnzb, s));
        } else {
            if (mixed) CK(launch_reset_dirty(dirty, c->nnzb, d2, c->Kel32, c->K32, c->reset_grid, s));
            else CK(launch_reset_dirty(dirty, c->nnzb, d2, c->Kel, c->Kt, c->reset_grid, s));
            c->launches += 1;
        }
        base = true;
    } else if (want_K) {
        if (mixed) CK(cudaMemsetAsync(c->K32, 0, sizeof(float) * nk, s));
        else CK(cudaMemsetAsync(c->Kt, 0, sizeof(double) * nk, s));
        base = false;
    }
    AsmArgs a{};
    a.mesh = mesh_dev(c);
    a.mat = c->mat;
    a.state = state_dev(c);
    a.u = u_dev;
    a.F = c->F;
    a.Kvals = c->Kt;
    a.Kvals32 = mixed ? c->K32 : nullptr;
    a.mode = split ? ASM_DELTA : ASM_FULL;
    a.want_K = want_K ? 1 : 0;
    a.elastic_only = 0;
    a.n_plastic = c->counter;
    a.err_flag = c->err_flag;
    a.dirty = (want_K && split) ? dirty : nullptr;
    a.tile = c->asm_tile;
    a.n_plastic_elem = want_K ? c->counter + 1 : nullptr;
    if (c->profile) CK(cudaEventRecord(c->ev[4], s));
    if (c->deterministic) {
        // one launch per colour, in colour order: no two elements of a launch share a node, so F and
        // K receive plain adds in a fixed order (bit-reproducible)
        const int nc = (int)c->h_color_ptr.size() - 1;
        for (int col = 0; col < nc; ++col) {
            a.elem_list = c->color_elems + c->h_color_ptr[col];
            a.list_n = c->h_color_ptr[col + 1] - c->h_color_ptr[col];
            CK(launch_assemble(c->eid, a, s));
        }
        c->launches += nc;
    } else {
        CK(launch_assemble(c->eid, a, s));
        c->launches += 1;
    }
    if (c->profile) CK(cudaEventRecord(c->ev[5], s));
    c->K_valid = want_K && !mixed;
    c->K32_valid = want_K && mixed;
    return EP_OK;
}

// A load path starts with the V-cycle's coarse correction in FP32 (EP_AMG_PRECISE=1: in FP64) and
// the preconditioner the options name; the Newton loop switches to the sparse LU (or, where that
// cannot be set up, to the precise V-cycle) when an FP64 GMRES solve stalls with the FP32 V-cycle.
static void precise_default(Ctx* c) {
    const char* v = std::getenv("EP_AMG_PRECISE");
    const int want = (v && std::atoi(v) == 1) ? 1 : 0;
    if (c->amg.precise && !want) c->amg_elastic = false;   // the FP32 coarse operators are stale
    c->amg.precise = want;
    c->direct_mode = false;
}

static ep_status read_flags(Ctx* c, unsigned long long* n_plastic, bool* rm_err) {
    CK(cudaMemcpyAsync(c->counter_host, c->counter, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(c->err_host, c->err_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (n_plastic) *n_plastic = *c->counter_host;
    if (rm_err) *rm_err = *c->err_host != 0;
    return EP_OK;
}

static ep_status commit(Ctx* c, const double* u_dev, unsigned long long* n_plastic) {
    CK(cudaMemsetAsync(c->counter, 0, sizeof(unsigned long long), c->stream));
    CommitArgs a{};
    a.mesh = mesh_dev(c);
    a.mat = c->mat;
    a.state = state_dev(c);
    a.u = u_dev;
    a.n_plastic = c->counter;
    a.err_flag = c->err_flag;
    CK(launch_commit(c->eid, a, c->stream));
    c->launches += 1;
    bool rm_err = false;
    ep_status st = read_flags(c, n_plastic, &rm_err);
    if (st != EP_OK) return st;
    if (rm_err) {
        c->err = "return mapping: apex reached with K*eta*eta_bar + Hc = 0 (no admissible stress)";
        return EP_ERR_RETURN_MAP;
    }
    return EP_OK;
}

static int krylov_method(const Ctx* c, const ep_opts& o) {
    if (o.krylov >= 1 && o.krylov <= 3) return o.krylov;
    const bool sym = c->mat.model != 3 || (c->mat.eta == c->mat.eta_bar && c->mat.Hc == 0.0);
    return sym ? 1 : 3;
}

}  // namespace ep

using namespace ep;

// message of the last failed context-free call on this thread (no context exists then)
namespace ep {
std::string& thread_error() {
    static thread_local std::string msg;
    return msg;
}
}  // namespace ep
#define g_create_err (ep::thread_error())

extern "C" {

void ep_default_opts(ep_opts* o) {
    if (!o) return;
    o->precision = EP_FP64;
    o->newton_rtol = 1e-10;
    o->newton_maxit = 25;
    o->krylov = 0;
    o->krylov_rtol = 0.0;
    o->krylov_maxit = 20000;
    o->precond = 2;
    o->split_elastic_cache = 1;
    o->warm_start = 1;
    o->profile = 0;
    o->deterministic = 0;
    o->asm_tile = 1;
    o->krylov_graphs = 1;
    o->direct_fallback = 1;
}

const char* ep_status_str(int32_t s) {
    switch (s) {
        case EP_OK: return "ok";
        case EP_ERR_INVALID_ARG: return "invalid argument";
        case EP_ERR_CUDA: return "CUDA error";
        case EP_ERR_OOM: return "out of device memory";
        case EP_ERR_BAD_ELEMENT: return "element with det J <= 0";
        case EP_ERR_RETURN_MAP: return "return mapping failed (no admissible stress)";
        case EP_ERR_NEWTON_NO_CONVERGENCE: return "Newton did not converge";
        case EP_ERR_KRYLOV: return "Krylov solver failed";
        case EP_ERR_NAN: return "NaN or Inf in a residual";
        case EP_ERR_STATE: return "call out of order";
    }
    return "unknown status";
}

const char* ep_last_error(const void* ctx) {
    if (!ctx) return g_create_err.c_str();
    return static_cast<const Ctx*>(ctx)->err.c_str();
}

ep_status ep_destroy(void* ctx) {
    if (!ctx) return EP_OK;
    Ctx* c = static_cast<Ctx*>(ctx);
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (void* p : c->allocs) cudaFree(p);
    if (c->ws.rec_X) cudaFree(c->ws.rec_X);
    if (c->ws.rec_T) cudaFree(c->ws.rec_T);
    krylov_free(c->kw);
    if (c->norms_host) cudaFreeHost(c->norms_host);
    if (c->counter_host) cudaFreeHost(c->counter_host);
    if (c->err_host) cudaFreeHost(c->err_host);
    for (auto& e : c->ev)
        if (e) cudaEventDestroy(e);
    amg_free(c->amg);
    direct_free(c->direct);
    cudaSetDevice(prev);
    delete c;
    return EP_OK;
}

}  // extern "C"

namespace ep {
// Creation shared by ep_create (one problem) and ep_create_batch (problems concatenated into one
// mesh): n_mat materials of one model, elem_mat (host, [n_elem], or null) the material of each
// element, prob_node (host, [n_prob + 1], or null) the node range of each problem.
static ep_status create_impl(void** out, const ep_mesh* mesh, const ep_material* mats, int32_t n_mat,
                             const int32_t* elem_mat, const int64_t* prob_node, int32_t n_prob, const ep_bc* bc,
                             int32_t device, void* cuda_stream) {
    if (!out) return EP_ERR_INVALID_ARG;
    *out = nullptr;
    if (!mesh || !mats || n_mat < 1 || !bc || !mesh->coords || !mesh->elem_nodes || !bc->dirichlet_mask)
        return EP_ERR_INVALID_ARG;
    if ((mesh->dim != 2 && mesh->dim != 3) || mesh->elem < 0 || mesh->elem > 3 || mesh->n_nodes <= 0 ||
        mesh->n_elem <= 0 || mesh->n_nodes > INT32_MAX)
        return EP_ERR_INVALID_ARG;
    Ctx* c = new Ctx();
    auto fail = [&](ep_status st) {
        g_create_err = c->err;
        ep_destroy(c);
        return st;
    };
    c->device = device;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    if (const char* v = std::getenv("EP_VERBOSE")) c->verbose = std::atoi(v);
    if (const char* v = std::getenv("EP_NEWTON_ETA0"))
        c->eta0 = c->eta0_mixed = std::max(1e-12, std::min(0.5, std::atof(v)));
    if (const char* v = std::getenv("EP_NEWTON_ETA_MAX"))
        c->eta_max = c->eta_max_mixed = std::max(1e-12, std::min(0.5, std::atof(v)));
    if (cudaSetDevice(device) != cudaSuccess) {
        c->err = "cudaSetDevice failed";
        return fail(EP_ERR_CUDA);
    }
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    c->dim = mesh->dim;
    c->family = mesh->elem;
    c->eid = elem_id(c->family, c->dim);
    c->n_p = elem_np(c->eid);
    c->n_q = elem_nq(c->eid);
    c->n_comp = c->dim == 2 ? 4 : 6;
    c->n_nodes = mesh->n_nodes;
    c->n_elem = mesh->n_elem;
    c->n_int = c->n_elem * c->n_q;
    c->n_dof = c->n_nodes * c->dim;
    std::vector<MatConst> mtab(n_mat);
    for (int i = 0; i < n_mat; ++i) {
        if (!make_matconst(mats[i], c->dim, mtab[i], c->err)) return fail(EP_ERR_INVALID_ARG);
        if (mtab[i].model != mtab[0].model) {
            c->err = "batch: every problem must use the same material model";
            return fail(EP_ERR_INVALID_ARG);
        }
    }
    c->mat = mtab[0];
    c->n_mat = n_mat;
    if (elem_mat)
        for (int64_t e = 0; e < c->n_elem; ++e)
            if (elem_mat[e] < 0 || elem_mat[e] >= n_mat) {
                c->err = "batch: element material index out of range";
                return fail(EP_ERR_INVALID_ARG);
            }
    c->hard_len = (c->mat.model == 1) ? c->n_int * c->n_comp : c->n_int;
    {
        // static inputs of the warm-start network per node: the material of (any) element holding
        // it, and its prescribed components
        std::vector<int32_t> node_mat(c->n_nodes, 0);
        if (elem_mat)
            for (int64_t e = 0; e < c->n_elem; ++e)
                for (int a = 0; a < elem_np(c->eid); ++a) {
                    const int32_t v = mesh->elem_nodes[e * elem_np(c->eid) + a];
                    if (v >= 0 && v < c->n_nodes) node_mat[v] = elem_mat[e];
                }
        c->h_node_static.assign((size_t)c->n_nodes * 5, 0.f);
        for (int64_t n = 0; n < c->n_nodes; ++n) {
            const ep_material& m = mats[node_mat[n]];
            const bool dp = m.model == EP_DP, el = m.model == EP_ELASTIC;
            int fixed = 0;
            for (int k = 0; k < c->dim; ++k) fixed += bc->dirichlet_mask[n * c->dim + k] ? 1 : 0;
            float* f = &c->h_node_static[(size_t)n * 5];
            f[0] = (float)m.nu;
            f[1] = el ? 0.f : (float)((dp ? m.c0 : m.Y) / m.E * 1e3);
            f[2] = el ? 0.f : (float)((dp ? m.Hc : m.H) / m.E * 10.0);
            f[3] = dp ? 1.f : 0.f;
            f[4] = (float)((double)fixed / c->dim);
        }
        if (prob_node && n_prob > 1) {
            c->h_node_prob.assign(c->n_nodes, 0);
            for (int p = 0; p < n_prob; ++p)
                for (int64_t n = prob_node[p]; n < prob_node[p + 1] && n < c->n_nodes; ++n) c->h_node_prob[n] = p;
        }
    }
    // problems and their residual-norm chunks (64 Ki DOFs each)
    c->n_prob = std::max(1, n_prob);
    c->prob_dof.assign(c->n_prob + 1, 0);
    for (int p = 0; p <= c->n_prob; ++p) c->prob_dof[p] = prob_node ? prob_node[p] * c->dim : (p ? c->n_dof : 0);
    for (int p = 0; p < c->n_prob; ++p)
        for (int64_t b = c->prob_dof[p]; b < c->prob_dof[p + 1]; b += 65536) {
            c->chunk_prob.push_back(p);
            c->chunk_beg.push_back(b);
            c->chunk_end.push_back(std::min(c->prob_dof[p + 1], b + (int64_t)65536));
        }

    // pattern and slot map (host)
    std::vector<int32_t> row_ptr, col_idx, slots;
    if (!build_pattern(c->n_nodes, c->n_elem, c->n_p, mesh->elem_nodes, row_ptr, col_idx, slots, c->err))
        return fail(EP_ERR_INVALID_ARG);
    c->nnzb = (int64_t)col_idx.size();
    std::vector<int32_t> color_elems;
    if (!color_elements(c->n_nodes, c->n_elem, c->n_p, mesh->elem_nodes, c->h_color_ptr, color_elems, c->err))
        return fail(EP_ERR_INVALID_ARG);
    std::vector<int32_t> diag(c->n_nodes);
    for (int64_t n = 0; n < c->n_nodes; ++n) {
        const int32_t* b = col_idx.data() + row_ptr[n];
        const int32_t* e = col_idx.data() + row_ptr[n + 1];
        const int32_t* it = std::lower_bound(b, e, (int32_t)n);
        if (it == e || *it != n) {
            c->err = "node " + std::to_string(n) + " belongs to no element";
            return fail(EP_ERR_INVALID_ARG);
        }
        diag[n] = (int32_t)(it - col_idx.data());
    }
    std::vector<double> dhat, wq;
    reference_tables(c->family, c->dim, dhat, wq);

    const int d = c->dim;
    cudaStream_t s = c->stream;
#define CKF(call)                                                   \
    do {                                                            \
        cudaError_t _e = (call);                                    \
        if (_e != cudaSuccess) return fail(cuda_fail(c, _e, #call)); \
    } while (0)
    double *d_dhat = nullptr, *d_wq = nullptr;
    int* bad = nullptr;
    CKF(dalloc(c, &c->coords, c->n_nodes * d));
    CKF(dalloc(c, &c->elem, c->n_elem * c->n_p));
    CKF(dalloc(c, &c->slots, c->n_elem * c->n_p * c->n_p));
    CKF(dalloc(c, &c->row_ptr, c->n_nodes + 1));
    CKF(dalloc(c, &c->col_idx, c->nnzb));
    CKF(dalloc(c, &c->diag_slot, c->n_nodes));
    CKF(dalloc(c, &c->spmv_perm, c->n_nodes));
    CKF(dalloc(c, &c->dphi, c->n_int * c->n_p * d));
    CKF(dalloc(c, &c->wgt, c->n_int));
    CKF(dalloc(c, &c->Kel, c->nnzb * d * d));
    CKF(dalloc(c, &c->Kt, c->nnzb * d * d));
    CKF(dalloc(c, &c->dirty64, c->nnzb));
    CKF(dalloc(c, &c->color_elems, c->n_elem));
    c->reset_grid = c->num_sms * 8;
    CKF(dalloc(c, &c->ep, c->n_int * c->n_comp));
    CKF(dalloc(c, &c->hard, c->hard_len));
    CKF(dalloc(c, &c->sig, c->n_int * c->n_comp));
    CKF(dalloc(c, &c->flag, c->n_int));
    CKF(dalloc(c, &c->u, c->n_dof));
    CKF(dalloc(c, &c->u_prev, c->n_dof));
    CKF(dalloc(c, &c->u_it, c->n_dof));
    CKF(dalloc(c, &c->F, c->n_dof));
    CKF(dalloc(c, &c->r, c->n_dof));
    CKF(dalloc(c, &c->f_unit, c->n_dof));
    CKF(dalloc(c, &c->uD_unit, c->n_dof));
    CKF(dalloc(c, &c->free_dof, c->n_dof));
    CKF(dalloc(c, &c->mat_table, n_mat));
    if (elem_mat) CKF(dalloc(c, &c->elem_mat, c->n_elem));
    if (c->n_prob > 1) {
        const int64_t nc = (int64_t)c->chunk_prob.size();
        CKF(dalloc(c, &c->d_chunks, 3 * nc));
        CKF(dalloc(c, &c->d_chunk_norms, 3 * nc));
        c->h_chunk_norms.resize(3 * nc);
    }
    CKF(dalloc(c, &c->counter, 2));   // plastic points, plastic elements of the last assembly
    CKF(dalloc(c, &c->err_flag, 1));
    CKF(dalloc(c, &c->norms, 3));
    CKF(dalloc(c, &d_dhat, dhat.size()));
    CKF(dalloc(c, &d_wq, wq.size()));
    CKF(dalloc(c, &bad, 1));
    CKF(cudaMallocHost(&c->norms_host, 3 * sizeof(double)));
    CKF(cudaMallocHost(&c->counter_host, 2 * sizeof(unsigned long long)));
    CKF(cudaMallocHost(&c->err_host, sizeof(int)));
    for (auto& e : c->ev) CKF(cudaEventCreate(&e));
    CKF(krylov_alloc(c->kw, c->n_nodes, d, 20000, c->num_sms));

    std::vector<uint8_t> freem(c->n_dof);
    for (int64_t i = 0; i < c->n_dof; ++i) freem[i] = bc->dirichlet_mask[i] ? 0 : 1;
    CKF(cudaMemcpyAsync(c->mat_table, mtab.data(), sizeof(MatConst) * n_mat, cudaMemcpyHostToDevice, s));
    if (elem_mat)
        CKF(cudaMemcpyAsync(c->elem_mat, elem_mat, sizeof(int32_t) * c->n_elem, cudaMemcpyHostToDevice, s));
    if (c->n_prob > 1) {
        const int64_t nc = (int64_t)c->chunk_prob.size();
        std::vector<int64_t> ch(3 * nc);
        for (int64_t i = 0; i < nc; ++i) {
            ch[i] = c->chunk_prob[i];
            ch[nc + i] = c->chunk_beg[i];
            ch[2 * nc + i] = c->chunk_end[i];
        }
        CKF(cudaMemcpyAsync(c->d_chunks, ch.data(), sizeof(int64_t) * ch.size(), cudaMemcpyHostToDevice, s));
        CKF(cudaStreamSynchronize(s));   // ch is a host temporary
    }
    CKF(cudaMemcpyAsync(c->coords, mesh->coords, sizeof(double) * c->n_nodes * d, cudaMemcpyHostToDevice, s));
    CKF(cudaMemcpyAsync(c->elem, mesh->elem_nodes, sizeof(int32_t) * c->n_elem * c->n_p, cudaMemcpyHostToDevice, s));
    CKF(cudaMemcpyAsync(c->slots, slots.data(), sizeof(int32_t) * slots.size(), cudaMemcpyHostToDevice, s));
    CKF(cudaMemcpyAsync(c->color_elems, color_elems.data(), sizeof(int32_t) * color_elems.size(),
                        cudaMemcpyHostToDevice, s));
    CKF(cudaMemcpyAsync(c->row_ptr, row_ptr.data(), sizeof(int32_t) * row_ptr.size(), cudaMemcpyHostToDevice, s));
    CKF(cudaMemcpyAsync(c->col_idx, col_idx.data(), sizeof(int32_t) * col_idx.size(), cudaMemcpyHostToDevice, s));
    CKF(cudaMemcpyAsync(c->diag_slot, diag.data(), sizeof(int32_t) * diag.size(), cudaMemcpyHostToDevice, s));
    // SpMV row order: rows sorted by their number of blocks (stable, so rows of one length keep the
    // mesh order and their neighbours' x entries stay close)
    std::vector<int32_t> perm(c->n_nodes);
    for (int64_t n = 0; n < c->n_nodes; ++n) perm[n] = (int32_t)n;
    std::stable_sort(perm.begin(), perm.end(), [&](int32_t a, int32_t b) {
        return row_ptr[a + 1] - row_ptr[a] < row_ptr[b + 1] - row_ptr[b];
    });
    CKF(cudaMemcpyAsync(c->spmv_perm, perm.data(), sizeof(int32_t) * perm.size(), cudaMemcpyHostToDevice, s));
    CKF(cudaMemcpyAsync(d_dhat, dhat.data(), sizeof(double) * dhat.size(), cudaMemcpyHostToDevice, s));
    CKF(cudaMemcpyAsync(d_wq, wq.data(), sizeof(double) * wq.size(), cudaMemcpyHostToDevice, s));
    CKF(cudaMemcpyAsync(c->free_dof, freem.data(), c->n_dof, cudaMemcpyHostToDevice, s));
    if (bc->f_ext_unit)
        CKF(cudaMemcpyAsync(c->f_unit, bc->f_ext_unit, sizeof(double) * c->n_dof, cudaMemcpyHostToDevice, s));
    else
        CKF(cudaMemsetAsync(c->f_unit, 0, sizeof(double) * c->n_dof, s));
    if (bc->u_D_unit)
        CKF(cudaMemcpyAsync(c->uD_unit, bc->u_D_unit, sizeof(double) * c->n_dof, cudaMemcpyHostToDevice, s));
    else
        CKF(cudaMemsetAsync(c->uD_unit, 0, sizeof(double) * c->n_dof, s));
    CKF(cudaMemsetAsync(c->ep, 0, sizeof(double) * c->n_int * c->n_comp, s));
    CKF(cudaMemsetAsync(c->hard, 0, sizeof(double) * c->hard_len, s));
    CKF(cudaMemsetAsync(c->sig, 0, sizeof(double) * c->n_int * c->n_comp, s));
    CKF(cudaMemsetAsync(c->flag, 0, c->n_int, s));
    CKF(cudaMemsetAsync(c->u, 0, sizeof(double) * c->n_dof, s));
    CKF(cudaMemsetAsync(c->u_prev, 0, sizeof(double) * c->n_dof, s));
    CKF(cudaMemsetAsync(c->err_flag, 0, sizeof(int), s));
    CKF(cudaMemsetAsync(bad, 0, sizeof(int), s));

    // geometry (Section 6.1) -- cached per point
    GeomArgs g{};
    g.n_elem = c->n_elem;
    g.n_int = c->n_int;
    g.coords = c->coords;
    g.elem_nodes = c->elem;
    g.dhat = d_dhat;
    g.wq = d_wq;
    g.dphi = c->dphi;
    g.wgt = c->wgt;
    g.bad_count = bad;
    CKF(launch_geometry(c->eid, g, s));
    int bad_host = 0;
    CKF(cudaMemcpyAsync(&bad_host, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    CKF(cudaStreamSynchronize(s));
    if (bad_host) {
        c->err = std::to_string(bad_host) + " integration points with det J <= 0";
        return fail(EP_ERR_BAD_ELEMENT);
    }
    // K_elast (Section 6.3)
    CKF(cudaMemsetAsync(c->Kel, 0, sizeof(double) * c->nnzb * d * d, s));
    AsmArgs a{};
    a.mesh = mesh_dev(c);
    a.mat = c->mat;
    a.state = state_dev(c);
    a.u = c->u;
    a.F = c->F;
    a.Kvals = c->Kel;
    a.mode = ASM_FULL;
    a.want_K = 1;
    a.elastic_only = 1;
    // coloured (one launch per colour, plain adds): K_elast is bit-reproducible, so the split
    // tangent and the AMG hierarchy built from it are too
    for (size_t col = 0; col + 1 < c->h_color_ptr.size(); ++col) {
        a.elem_list = c->color_elems + c->h_color_ptr[col];
        a.list_n = c->h_color_ptr[col + 1] - c->h_color_ptr[col];
        CKF(launch_assemble(c->eid, a, s));
    }
    CKF(cudaStreamSynchronize(s));
#undef CKF
    c->h_row_ptr = std::move(row_ptr);
    c->h_col_idx = std::move(col_idx);
    c->h_coords.assign(mesh->coords, mesh->coords + c->n_nodes * d);
    c->h_free = std::move(freem);
    *out = c;
    return EP_OK;
}
}  // namespace ep

extern "C" {

ep_status ep_create(void** out, const ep_mesh* mesh, const ep_material* mat, const ep_bc* bc, int32_t device,
                    void* cuda_stream) {
    return create_impl(out, mesh, mat, 1, nullptr, nullptr, 1, bc, device, cuda_stream);
}

ep_status ep_create_batch(void** out, int32_t n_problems, const ep_mesh* meshes, const ep_material* mats,
                          const ep_bc* bcs, int32_t device, void* cuda_stream) {
    if (!out) return EP_ERR_INVALID_ARG;
    *out = nullptr;
    if (n_problems < 1 || !meshes || !mats || !bcs) return EP_ERR_INVALID_ARG;
    const int dim = meshes[0].dim, fam = meshes[0].elem;
    if ((dim != 2 && dim != 3) || fam < 0 || fam > 3) return EP_ERR_INVALID_ARG;
    const int n_p = elem_np(elem_id(fam, dim));
    int64_t nn = 0, ne = 0;
    std::vector<int64_t> node_off(n_problems + 1, 0);
    for (int p = 0; p < n_problems; ++p) {
        const ep_mesh& m = meshes[p];
        if (m.dim != dim || m.elem != fam || m.n_nodes <= 0 || m.n_elem <= 0 || !m.coords || !m.elem_nodes ||
            !bcs[p].dirichlet_mask) {
            g_create_err = "ep_create_batch: problem " + std::to_string(p) + " has a different element type or no data";
            return EP_ERR_INVALID_ARG;
        }
        nn += m.n_nodes;
        ne += m.n_elem;
        node_off[p + 1] = nn;
    }
    if (nn > INT32_MAX) return EP_ERR_INVALID_ARG;
    std::vector<double> coords((size_t)nn * dim), uD((size_t)nn * dim, 0.0), fe((size_t)nn * dim, 0.0);
    std::vector<int32_t> elem((size_t)ne * n_p), emat(ne);
    std::vector<uint8_t> mask((size_t)nn * dim);
    int64_t eo = 0;
    for (int p = 0; p < n_problems; ++p) {
        const ep_mesh& m = meshes[p];
        const int64_t no = node_off[p];
        std::copy(m.coords, m.coords + m.n_nodes * dim, coords.begin() + no * dim);
        std::copy(bcs[p].dirichlet_mask, bcs[p].dirichlet_mask + m.n_nodes * dim, mask.begin() + no * dim);
        if (bcs[p].u_D_unit) std::copy(bcs[p].u_D_unit, bcs[p].u_D_unit + m.n_nodes * dim, uD.begin() + no * dim);
        if (bcs[p].f_ext_unit)
            std::copy(bcs[p].f_ext_unit, bcs[p].f_ext_unit + m.n_nodes * dim, fe.begin() + no * dim);
        for (int64_t i = 0; i < m.n_elem * n_p; ++i) {
            const int32_t v = m.elem_nodes[i];
            if (v < 0 || v >= m.n_nodes) {
                g_create_err = "ep_create_batch: problem " + std::to_string(p) + " has a node index out of range";
                return EP_ERR_INVALID_ARG;
            }
            elem[(size_t)(eo * n_p + i)] = (int32_t)(v + no);
        }
        std::fill(emat.begin() + eo, emat.begin() + eo + m.n_elem, p);
        eo += m.n_elem;
    }
    const ep_mesh all{dim, fam, nn, ne, coords.data(), elem.data()};
    const ep_bc bc{mask.data(), uD.data(), fe.data()};
    return create_impl(out, &all, mats, n_problems, emat.data(), node_off.data(), n_problems, &bc, device, cuda_stream);
}

// Build the AMG hierarchy from K_elast on first use of preconditioner 2.
static ep_status ensure_amg(Ctx* c) {
    if (c->amg_built) return EP_OK;
    const auto t0 = std::chrono::steady_clock::now();
    std::vector<double> kel((size_t)c->nnzb * c->dim * c->dim);
    CK(cudaMemcpyAsync(kel.data(), c->Kel, sizeof(double) * kel.size(), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    AmgInput in{c->dim, c->n_nodes, c->h_row_ptr.data(), c->h_col_idx.data(), kel.data(), c->h_free.data(),
                c->h_coords.data()};
    AmgHierarchy H;
    if (!amg_setup_host(in, H, c->err)) return EP_ERR_STATE;
    CK(amg_upload(H, c->amg, c->num_sms));
    c->kw.amg = &c->amg;
    c->amg_built = true;
    precise_default(c);
    c->amg_setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (c->verbose) {
        std::fprintf(stderr, "[ep] AMG: %zu levels, setup %.1f ms, sizes", H.levels.size(), c->amg_setup_ms);
        for (auto& L : H.levels) std::fprintf(stderr, " %lld", (long long)L.n);
        std::fprintf(stderr, "\n");
    }
    return EP_OK;
}

// nodes factored together at the leaves of the nested dissection (256x256 P2 column: 41.6 GFLOP per
// factorisation with 16, 43.8 with 32, 50.7 with 64)
constexpr int DIRECT_LEAF = 16;
// Relative tolerance of the Newton systems solved with the sparse LU (one to three GMRES iterations
// with FP64 fronts).  Near a limit load the tangent is nearly singular: the oracle's FP64 direct
// solves follow the homogeneous branch, while GMRES stopped at 1e-10 left O(1) errors in the Newton
// step along the soft modes and the iteration diverged (measured, 256x256 column at 0.98 t_lim).
constexpr double DIRECT_ETA = 1e-13;
// GMRES iterations a solve with the previous iteration's factors may take before they are refreshed
constexpr int DIRECT_REUSE_MAXIT = 12;

// The sparse LU's symbolic analysis (host) and device memory, on first use; false (reason in
// c->direct.why) when the factors would not fit in 60% of the free device memory (or in
// EP_DIRECT_MAX_MB MiB).
static bool ensure_direct(Ctx* c) {
    if (c->direct.ready) return true;
    if (c->direct.refused) return false;
    const auto t0 = std::chrono::steady_clock::now();
    std::string err;
    if (!direct_analyse(c->dim, c->n_nodes, c->h_row_ptr.data(), c->h_col_idx.data(), c->h_coords.data(), DIRECT_LEAF,
                        c->direct.plan, err)) {
        c->direct.refused = true;
        c->direct.why = err;
        return false;
    }
    // fronts in FP64 (EP_DIRECT_FP32=1: FP32, 1/30 of the factorisation time, but GMRES then needs
    // tens of iterations on a nearly singular tangent where FP64 fronts need one to three)
    const char* f32 = std::getenv("EP_DIRECT_FP32");
    c->direct.fp64 = (f32 && std::atoi(f32) == 1) ? 0 : 1;
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) fr = 0;
    int64_t cap = (int64_t)(0.6 * (double)fr);
    if (const char* mb = std::getenv("EP_DIRECT_MAX_MB")) cap = std::min<int64_t>(cap, (int64_t)std::atoll(mb) << 20);
    if (!direct_setup(c->direct, cap)) return false;
    c->kw.direct = &c->direct;
    c->direct_setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (c->verbose) {
        const DirectPlan& P = c->direct.plan;
        int mmax = 0;
        for (int v : P.lvl_mmax) mmax = std::max(mmax, v);
        std::fprintf(stderr, "[ep] sparse LU: %d fronts on %zu levels, largest front %d, %s factors %.1f MiB, %.2f GFLOP, "
                     "setup %.1f ms\n", P.n_fronts, P.level_ptr.size() - 1, mmax, c->direct.fp64 ? "FP64" : "FP32",
                     (double)P.factor_vals() * (c->direct.fp64 ? 8.0 : 4.0) / 1048576.0, P.flops * 1e-9, c->direct_setup_ms);
    }
    return true;
}

ep_status ep_get_info(const void* ctx, ep_info* info) {
    if (!ctx || !info) return EP_ERR_INVALID_ARG;
    const Ctx* c = static_cast<const Ctx*>(ctx);
    info->n_nodes = c->n_nodes;
    info->n_elem = c->n_elem;
    info->n_int = c->n_int;
    info->nnz_blocks = c->nnzb;
    info->dim = c->dim;
    info->n_p = c->n_p;
    info->n_q = c->n_q;
    info->n_comp = c->n_comp;
    return EP_OK;
}

static ep_status field_ptr(Ctx* c, int32_t field, void** p, size_t* bytes, bool writing) {
    const size_t d2 = (size_t)c->dim * c->dim;
    switch (field) {
        case EP_U: *p = c->u; *bytes = sizeof(double) * c->n_dof; return EP_OK;
        case EP_STRESS: *p = c->sig; *bytes = sizeof(double) * c->n_int * c->n_comp; return EP_OK;
        case EP_PLASTIC_STRAIN: *p = c->ep; *bytes = sizeof(double) * c->n_int * c->n_comp; return EP_OK;
        case EP_HARDENING: *p = c->hard; *bytes = sizeof(double) * c->hard_len; return EP_OK;
        case EP_PLASTIC_FLAG: *p = c->flag; *bytes = c->n_int; return EP_OK;
    }
    if (writing) return EP_ERR_INVALID_ARG;
    switch (field) {
        case EP_F_INT: *p = c->F; *bytes = sizeof(double) * c->n_dof; return EP_OK;
        case EP_K_ROW_PTR: *p = c->row_ptr; *bytes = sizeof(int32_t) * (c->n_nodes + 1); return EP_OK;
        case EP_K_COL_IDX: *p = c->col_idx; *bytes = sizeof(int32_t) * c->nnzb; return EP_OK;
        case EP_K_VALUES: *p = c->Kt; *bytes = sizeof(double) * c->nnzb * d2; return EP_OK;
        case EP_K_ELASTIC: *p = c->Kel; *bytes = sizeof(double) * c->nnzb * d2; return EP_OK;
        case EP_WEIGHT: *p = c->wgt; *bytes = sizeof(double) * c->n_int; return EP_OK;
        case EP_DPHI: *p = c->dphi; *bytes = sizeof(double) * c->n_int * c->n_p * c->dim; return EP_OK;
        case EP_SOLUTION: *p = c->kw.d.x; *bytes = sizeof(double) * c->n_dof; return EP_OK;
        case EP_K_VALUES_F32:
            if (!c->K32) return EP_ERR_STATE;
            *p = c->K32; *bytes = sizeof(float) * c->nnzb * d2; return EP_OK;
        case EP_WS_X:
            if (!c->ws.rec_X) return EP_ERR_STATE;
            *p = c->ws.rec_X; *bytes = sizeof(float) * c->ws.rec_n * EP_WS_N_IN; return EP_OK;
        case EP_WS_T:
            if (!c->ws.rec_T) return EP_ERR_STATE;
            *p = c->ws.rec_T; *bytes = sizeof(float) * c->ws.rec_n * EP_WS_N_OUT; return EP_OK;
        case EP_WS_START:
            if (!c->ws.uL_valid) return EP_ERR_STATE;
            *p = c->ws.uL; *bytes = sizeof(double) * c->n_dof; return EP_OK;
    }
    return EP_ERR_INVALID_ARG;
}

ep_status ep_get(void* ctx, int32_t field, void* dst, size_t bytes, int32_t dst_is_device) {
    if (!ctx || !dst) return EP_ERR_INVALID_ARG;
    Ctx* c = static_cast<Ctx*>(ctx);
    void* src = nullptr;
    size_t want = 0;
    const ep_status fs = field_ptr(c, field, &src, &want, false);
    if (fs != EP_OK) {
        c->err = fs == EP_ERR_STATE ? "ep_get: the field does not exist yet (no mixed-precision assembly, or no recording)"
                                    : "ep_get: unknown field";
        return fs;
    }
    if (bytes != want) {
        c->err = "ep_get: size mismatch (expected " + std::to_string(want) + " bytes)";
        return EP_ERR_INVALID_ARG;
    }
    cudaSetDevice(c->device);
    CK(cudaMemcpyAsync(dst, src, bytes, dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return EP_OK;
}

ep_status ep_set(void* ctx, int32_t field, const void* src, size_t bytes, int32_t src_is_device) {
    if (!ctx || !src) return EP_ERR_INVALID_ARG;
    Ctx* c = static_cast<Ctx*>(ctx);
    void* dst = nullptr;
    size_t want = 0;
    if (field_ptr(c, field, &dst, &want, true) != EP_OK) {
        c->err = "ep_set: field is not writable";
        return EP_ERR_INVALID_ARG;
    }
    if (bytes != want) {
        c->err = "ep_set: size mismatch (expected " + std::to_string(want) + " bytes)";
        return EP_ERR_INVALID_ARG;
    }
    cudaSetDevice(c->device);
    CK(cudaMemcpyAsync(dst, src, bytes, src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (field == EP_U) {
        c->n_committed = 0;      // no extrapolation history across a reset
        c->ws.hist = 0;
        c->mixed_fallback = false;
        precise_default(c);
    }
    return EP_OK;
}

ep_status ep_reset(void* ctx) {
    if (!ctx) return EP_ERR_INVALID_ARG;
    Ctx* c = static_cast<Ctx*>(ctx);
    cudaSetDevice(c->device);
    cudaStream_t s = c->stream;
    CK(cudaMemsetAsync(c->u, 0, sizeof(double) * c->n_dof, s));
    CK(cudaMemsetAsync(c->u_prev, 0, sizeof(double) * c->n_dof, s));
    CK(cudaMemsetAsync(c->ep, 0, sizeof(double) * c->n_int * c->n_comp, s));
    CK(cudaMemsetAsync(c->hard, 0, sizeof(double) * c->hard_len, s));
    CK(cudaMemsetAsync(c->sig, 0, sizeof(double) * c->n_int * c->n_comp, s));
    CK(cudaMemsetAsync(c->flag, 0, c->n_int, s));
    CK(cudaMemsetAsync(c->err_flag, 0, sizeof(int), s));
    c->n_committed = 0;
    c->zeta_last = c->zeta_prev = 0.0;
    c->ws.hist = 0;
    c->ws.uL_valid = false;
    c->mixed_fallback = false;
    precise_default(c);
    return EP_OK;
}

static ep_status load_u(Ctx* c, const double* u, int32_t u_is_device) {
    CK(cudaMemcpyAsync(c->u_it, u, sizeof(double) * c->n_dof,
                       u_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
    return EP_OK;
}

ep_status ep_assemble_prec(void* ctx, const double* u, int32_t u_is_device, int32_t split, int32_t precision,
                           int64_t* n_plastic) {
    if (!ctx || !u || (precision != EP_FP64 && precision != EP_MIXED)) return EP_ERR_INVALID_ARG;
    Ctx* c = static_cast<Ctx*>(ctx);
    cudaSetDevice(c->device);
    ep_status st = load_u(c, u, u_is_device);
    if (st != EP_OK) return st;
    CK(cudaMemsetAsync(c->err_flag, 0, sizeof(int), c->stream));
    st = assemble(c, c->u_it, split != 0, true, precision == EP_MIXED);
    if (st != EP_OK) return st;
    unsigned long long np = 0;
    bool rm_err = false;
    st = read_flags(c, &np, &rm_err);
    if (st != EP_OK) return st;
    if (n_plastic) *n_plastic = (int64_t)np;
    if (rm_err) {
        c->err = "return mapping: apex reached with K*eta*eta_bar + Hc = 0";
        return EP_ERR_RETURN_MAP;
    }
    return EP_OK;
}

ep_status ep_assemble(void* ctx, const double* u, int32_t u_is_device, int32_t split, int64_t* n_plastic) {
    return ep_assemble_prec(ctx, u, u_is_device, split, EP_FP64, n_plastic);
}

ep_status ep_commit(void* ctx, const double* u, int32_t u_is_device) {
    if (!ctx || !u) return EP_ERR_INVALID_ARG;
    Ctx* c = static_cast<Ctx*>(ctx);
    cudaSetDevice(c->device);
    ep_status st = load_u(c, u, u_is_device);
    if (st != EP_OK) return st;
    CK(cudaMemsetAsync(c->err_flag, 0, sizeof(int), c->stream));
    st = commit(c, c->u_it, nullptr);
    if (st != EP_OK) return st;
    CK(cudaMemcpyAsync(c->u, c->u_it, sizeof(double) * c->n_dof, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->n_committed = 0;
    return EP_OK;
}

ep_status ep_linear_solve(void* ctx, const double* b, int32_t b_is_device, const ep_opts* opts, int32_t* iterations,
                          double* rel_resid) {
    if (!ctx || !b || !opts) return EP_ERR_INVALID_ARG;
    Ctx* c = static_cast<Ctx*>(ctx);
    const bool mixed = opts->precision == EP_MIXED;
    if (opts->precision != EP_FP64 && !mixed) return EP_ERR_INVALID_ARG;
    if (mixed ? !c->K32_valid : !c->K_valid) {
        c->err = mixed ? "ep_linear_solve: no FP32 matrix (call ep_assemble_prec with EP_MIXED first)"
                       : "ep_linear_solve: no assembled matrix (call ep_assemble first)";
        return EP_ERR_STATE;
    }
    if (!(opts->krylov_rtol > 0.0) || opts->krylov_maxit <= 0) {
        c->err = "ep_linear_solve: need krylov_rtol > 0 and krylov_maxit > 0";
        return EP_ERR_INVALID_ARG;
    }
    cudaSetDevice(c->device);
    c->deterministic = opts->deterministic ? 1 : 0;
    c->amg.deterministic = c->deterministic;
    c->kw.graphs = opts->krylov_graphs ? 1 : 0;
    if (opts->precond < 0 || opts->precond > 3) {
        c->err = "precond must be 0, 1, 2 or 3";
        return EP_ERR_INVALID_ARG;
    }
    if (opts->precond == 2) {
        ep_status st = ensure_amg(c);
        if (st != EP_OK) return st;
    }
    if (opts->precond == 3 && !ensure_direct(c)) {
        c->err = c->direct.why;
        return EP_ERR_STATE;
    }
    // the sparse LU is nonsymmetric in rounding: it preconditions GMRES
    const int lmethod = opts->precond == 3 ? 3 : krylov_method(c, *opts);
    CK(cudaMemcpyAsync(c->r, b, sizeof(double) * c->n_dof, b_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                       c->stream));
    c->kw.galerkin = 1;
    c->amg_elastic = false;
    int its = 0, status = 0;
    double rel = 0.0;
    if (mixed) {
        const BsrF A = bsr_dev(c, (const float*)c->K32);
        CK(vec_cvt_f32(c->r, c->r32, c->n_dof, c->stream));
        CK(krylov_precond(A, c->kw, opts->precond, c->stream));
        CK(krylov_solve(A, c->kw, c->r32, lmethod, opts->krylov_rtol, opts->krylov_maxit, c->stream, &its, &rel,
                        &status));
        CK(vec_cvt_f64(c->kw.f.x, c->kw.d.x, c->n_dof, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    } else {
        const BsrDev A = bsr_dev(c, (const double*)c->Kt);
        CK(krylov_precond(A, c->kw, opts->precond, c->stream));
        CK(krylov_solve(A, c->kw, c->r, lmethod, opts->krylov_rtol, opts->krylov_maxit, c->stream, &its, &rel,
                        &status));
    }
    if (iterations) *iterations = its;
    if (rel_resid) *rel_resid = rel;
    if (status != EP_OK) c->err = "Krylov: no convergence within the iteration cap, or breakdown";
    return (ep_status)status;
}

// Buffers and history of the learned warm start (first ep_ws_record / ep_ws_attach).  The history
// starts here: the plastic fractions of the current state, no converged step yet.
static ep_status ws_setup(Ctx* c) {
    WsState& w = c->ws;
    cudaStream_t s = c->stream;
    if (!w.ready) {
        CK(dalloc(c, &w.u3, c->n_dof));
        CK(dalloc(c, &w.cnt_ip, c->n_nodes));
        CK(dalloc(c, &w.cnt_pl, c->n_nodes));
        if (!c->h_node_prob.empty()) CK(dalloc(c, &w.node_prob, c->n_nodes));
        CK(dalloc(c, &w.prob_dof, c->n_prob + 1));
        CK(dalloc(c, &w.pf1, c->n_nodes));
        CK(dalloc(c, &w.pf2, c->n_nodes));
        CK(dalloc(c, &w.pfk, c->n_nodes));
        CK(dalloc(c, &w.stat, c->n_nodes * 5));
        CK(dalloc(c, &w.prox1, c->n_nodes));
        CK(dalloc(c, &w.uL, c->n_dof));
        CK(dalloc(c, &w.scale, 2 * c->n_prob));
        CK(dalloc(c, &w.X, c->n_nodes * EP_WS_N_IN));
        CK(dalloc(c, &w.Y, c->n_nodes * EP_WS_N_OUT));
        CK(dalloc(c, &w.u_ex, c->n_dof));
        CK(dalloc(c, &w.take_ex, c->n_prob));
        w.h_take.assign(c->n_prob, 0);
        if (w.node_prob)
            CK(cudaMemcpyAsync(w.node_prob, c->h_node_prob.data(), sizeof(int32_t) * c->n_nodes, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(w.prob_dof, c->prob_dof.data(), sizeof(int64_t) * (c->n_prob + 1), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(w.stat, c->h_node_static.data(), sizeof(float) * c->n_nodes * 5, cudaMemcpyHostToDevice, s));
        CK(cudaMemsetAsync(w.cnt_ip, 0, sizeof(int32_t) * c->n_nodes, s));
        CK(ws_node_counts(c->elem, c->n_elem, c->n_p, c->n_q, nullptr, w.cnt_ip, s));
        c->launches += 1;
        w.ready = true;
    }
    CK(cudaMemsetAsync(w.cnt_pl, 0, sizeof(int32_t) * c->n_nodes, s));
    CK(ws_node_counts(c->elem, c->n_elem, c->n_p, c->n_q, c->flag, w.cnt_pl, s));
    CK(ws_fraction(w.cnt_pl, w.cnt_ip, c->n_nodes, w.pf1, s));
    CK(cudaMemcpyAsync(w.pf2, w.pf1, sizeof(float) * c->n_nodes, cudaMemcpyDeviceToDevice, s));
    CK(ws_proximity(mesh_dev(c), c->sig, c->hard, c->n_p, c->n_q, c->dim, w.prox1, s));
    CK(cudaStreamSynchronize(s));
    w.hist = 0;
    return EP_OK;
}

// Residual norm ||(zeta f - F(u))_free|| of every problem at a candidate start (an F-only assembly
// with the committed state), and the largest relative residual over the problems (the Newton
// test's measure).  A return-mapping failure or a non-finite norm reads as +inf.
static ep_status start_residuals(Ctx* c, const double* u, double z, std::vector<double>& rn, double* rel_max) {
    cudaStream_t s = c->stream;
    CK(cudaMemsetAsync(c->err_flag, 0, sizeof(int), s));
    ep_status st = assemble(c, u, true, false, false);
    if (st != EP_OK) return st;
    CK(vec_residual(c->f_unit, z, c->F, c->free_dof, c->r, nullptr, c->n_dof, c->kw.part, c->kw.nparts, c->norms, s));
    c->launches += 1;
    rn.assign(c->n_prob, 0.0);
    const int64_t nchunk = (int64_t)c->chunk_prob.size();
    if (c->n_prob > 1) {
        CK(vec_chunk_norms(c->f_unit, z, c->F, c->free_dof, c->r, c->d_chunks, nchunk, c->d_chunk_norms, s));
        CK(cudaMemcpyAsync(c->h_chunk_norms.data(), c->d_chunk_norms, sizeof(double) * 3 * nchunk,
                           cudaMemcpyDeviceToHost, s));
        c->launches += 1;
    }
    CK(cudaMemcpyAsync(c->norms_host, c->norms, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(c->err_host, c->err_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    std::vector<double> sc(c->n_prob, 0.0);
    if (c->n_prob > 1) {
        std::vector<double> pf(c->n_prob, 0.0), pF(c->n_prob, 0.0);
        for (int64_t i = 0; i < nchunk; ++i) {
            rn[c->chunk_prob[i]] += c->h_chunk_norms[i];
            pf[c->chunk_prob[i]] += c->h_chunk_norms[nchunk + i];
            pF[c->chunk_prob[i]] += c->h_chunk_norms[2 * nchunk + i];
        }
        for (int p = 0; p < c->n_prob; ++p) sc[p] = std::max(std::sqrt(pf[p]), std::sqrt(pF[p]));
    } else {
        rn[0] = c->norms_host[0];
        sc[0] = std::max(std::sqrt(c->norms_host[1]), std::sqrt(c->norms_host[2]));
    }
    *rel_max = 0.0;
    for (int p = 0; p < c->n_prob; ++p) {
        double& v = rn[p];
        v = std::sqrt(v);
        if (*c->err_host || !std::isfinite(v)) v = HUGE_VAL;
        *rel_max = std::max(*rel_max, sc[p] > 0.0 ? v / sc[p] : v);
    }
    CK(cudaMemsetAsync(c->err_flag, 0, sizeof(int), s));
    return EP_OK;
}

ep_status ep_ws_record(void* ctx, int64_t max_rows) {
    if (!ctx || max_rows < 0) return EP_ERR_INVALID_ARG;
    Ctx* c = static_cast<Ctx*>(ctx);
    cudaSetDevice(c->device);
    CK(cudaStreamSynchronize(c->stream));
    if (c->ws.rec_X) cudaFree(c->ws.rec_X);
    if (c->ws.rec_T) cudaFree(c->ws.rec_T);
    c->ws.rec_X = c->ws.rec_T = nullptr;
    c->ws.rec_cap = c->ws.rec_n = 0;
    if (max_rows == 0) return EP_OK;
    CK(cudaMalloc((void**)&c->ws.rec_X, sizeof(float) * max_rows * EP_WS_N_IN));
    CK(cudaMalloc((void**)&c->ws.rec_T, sizeof(float) * max_rows * EP_WS_N_OUT));
    c->ws.rec_cap = max_rows;
    return ws_setup(c);
}

ep_status ep_ws_samples(void* ctx, const float** X, const float** T, int64_t* n_rows) {
    if (!ctx || !X || !T || !n_rows) return EP_ERR_INVALID_ARG;
    Ctx* c = static_cast<Ctx*>(ctx);
    *X = c->ws.rec_X;
    *T = c->ws.rec_T;
    *n_rows = c->ws.rec_n;
    return EP_OK;
}

ep_status ep_ws_attach(void* ctx, void* mlp) {
    if (!ctx) return EP_ERR_INVALID_ARG;
    Ctx* c = static_cast<Ctx*>(ctx);
    cudaSetDevice(c->device);
    c->ws.mlp = mlp;
    if (!mlp || c->ws.ready) return EP_OK;
    return ws_setup(c);
}

ep_status ep_solve_load_path(void* ctx, int32_t n_steps, const double* zeta, const ep_opts* opts,
                             ep_step_report* reports) {
    if (!ctx || n_steps < 0 || (n_steps > 0 && !zeta)) return EP_ERR_INVALID_ARG;
    Ctx* c = static_cast<Ctx*>(ctx);
    ep_opts o;
    if (opts) o = *opts;
    else ep_default_opts(&o);
    if (o.precision != EP_FP64 && o.precision != EP_MIXED) {
        c->err = "precision must be EP_FP64 or EP_MIXED";
        return EP_ERR_INVALID_ARG;
    }
    if (o.warm_start < 0 || o.warm_start > 2) {
        c->err = "warm_start must be 0, 1 or 2";
        return EP_ERR_INVALID_ARG;
    }
    if (o.warm_start == 2 && !c->ws.mlp) {
        c->err = "warm_start = 2 needs a network (ep_ws_attach)";
        return EP_ERR_INVALID_ARG;
    }
    const bool mixed = o.precision == EP_MIXED;
    if (!(o.newton_rtol > 0.0) || o.newton_maxit < 1 || o.krylov_maxit < 1) return EP_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    cudaStream_t s = c->stream;
    if (o.precond < 0 || o.precond > 3) {
        c->err = "precond must be 0, 1, 2 or 3";
        return EP_ERR_INVALID_ARG;
    }
    if (o.precond == 2) {
        ep_status st = ensure_amg(c);
        if (st != EP_OK) return st;
    }
    if (o.precond == 3 && !ensure_direct(c)) {
        c->err = c->direct.why;
        return EP_ERR_STATE;
    }
    const int method = o.precond == 3 ? 3 : krylov_method(c, o);
    const bool split = o.split_elastic_cache != 0;
    const BsrDev A = bsr_dev(c, (const double*)c->Kt);
    if (mixed) {
        ep_status st = ensure_mixed(c);
        if (st != EP_OK) return st;
    }
    const BsrF Af = bsr_dev(c, (const float*)c->K32);
    c->profile = o.profile;
    c->kw.profile = o.profile;
    c->amg.profile = o.profile;
    c->deterministic = o.deterministic ? 1 : 0;
    c->amg.deterministic = c->deterministic;
    if (o.asm_tile != 1 && o.asm_tile != 2) {
        c->err = "asm_tile must be 1 or 2";
        return EP_ERR_INVALID_ARG;
    }
    c->asm_tile = o.asm_tile;
    c->kw.graphs = o.krylov_graphs ? 1 : 0;
    c->kw.verbose = c->verbose;
    for (int k = 0; k < n_steps; ++k) {
        const auto t_step0 = std::chrono::steady_clock::now();
        ep_step_report rep{};
        float t_asm = 0.f, t_sol = 0.f;
        c->launches = 0;
        c->kw.launches = 0;
        c->amg.launches = 0;
        c->direct.launches = 0;
        c->direct.profile = o.profile;
        const int dfac0 = c->direct.n_factor, dsol0 = c->direct.n_solve;
        const double dfms0 = c->direct.factor_ms, dsms0 = c->direct.solve_ms;
        c->kw.spmv_n = 0;
        c->kw.spmv_ms = 0.0;
        c->amg.smooth0_ms = 0.0;
        c->amg.smooth0_n = 0;
        double t_asm_kernel = 0.0;
        const double z = zeta[k];
        ep_status st = EP_OK;
        double rel = 0.0;
        int it = 0;
        bool converged = false;
        // Inputs of the warm-start network for this step (learned start, or recording): three
        // converged steps since the history started and a load that keeps its direction.
        WsState& ws = c->ws;
        const bool ws_learn = o.warm_start == 2 && ws.mlp;
        const bool ws_rec = ws.rec_cap - ws.rec_n >= c->n_nodes;
        bool ws_feat = false;
        double ws_ratio = 0.0;
        float* ws_X = ws.X;
        if (ws.ready && (ws_learn || ws_rec) && ws.hist >= 3 && c->zeta_last != c->zeta_prev) {
            ws_ratio = (z - c->zeta_last) / (c->zeta_last - c->zeta_prev);
            if (ws_ratio > 0.0) {
                const double r_k1 =
                    c->zeta_prev != ws.zeta3 ? (c->zeta_last - c->zeta_prev) / (c->zeta_prev - ws.zeta3) : 0.0;
                if (ws_rec) ws_X = ws.rec_X + ws.rec_n * EP_WS_N_IN;
                CK(ws_scale(c->u, c->u_prev, ws.prob_dof, c->n_prob, ws.scale, s));
                CK(ws_features(c->u, c->u_prev, ws.u3, ws.node_prob, ws.scale, c->n_prob, c->dim, c->n_nodes, ws_ratio,
                               r_k1, ws.pf1, ws.pf2, ws.prox1, ws.stat, ws_X, s));
                c->launches += 2;
                ws_feat = true;
            }
        }
        // Start iterate: the last converged u with the new Dirichlet values, plus (warm_start >= 1)
        // the linear extrapolation of the last two steps while the load keeps its direction, plus
        // (warm_start = 2) the network's correction where it lowers the residual.  A step that
        // does not converge from the extrapolated start (a predictor past a change of the plastic
        // regime) is retried once from the unextrapolated one.
        bool redo_step = false;   // the attempt runs again (the path switched to the sparse LU in it)
        for (int attempt = 0; attempt < 2; ++attempt) {
        bool extrapolated = false;
        rep.start = 0;
        rep.n_learned = 0;
        CK(cudaMemcpyAsync(c->u_it, c->u, sizeof(double) * c->n_dof, cudaMemcpyDeviceToDevice, s));
        if (attempt == 0 && o.warm_start >= 1 && c->n_committed >= 2 && c->zeta_last != c->zeta_prev) {
            const double ratio = (z - c->zeta_last) / (c->zeta_last - c->zeta_prev);
            if (ratio > 0.0) {
                CK(vec_extrapolate(c->u_it, c->u_prev, ratio, c->n_dof, s));
                c->launches += 1;
                extrapolated = true;
            }
        }
        CK(vec_set_dirichlet(c->u_it, c->uD_unit, z, c->free_dof, c->n_dof, s));
        c->launches += 1;
        if (extrapolated) rep.start = 1;
        std::vector<double> r_ex;
        double rel_ex = HUGE_VAL;
        if (extrapolated && ws_learn && ws_feat) {
            st = start_residuals(c, c->u_it, z, r_ex, &rel_ex);
            if (st != EP_OK) return st;
            rep.n_assemble += 1;
        }
        if (extrapolated && ws_learn && ws_feat && rel_ex > o.newton_rtol) {
            // learned start: u_ex + s * P(y) on free DOFs, P the projection of the per-node prediction
            // onto the span of the last two increments (per problem and component); each problem
            // keeps whichever start has the smaller residual.  (An extrapolated start that already
            // meets the tolerance, as in a linear-elastic stretch of the path, is kept as it is.)
            CK(cudaMemcpyAsync(ws.u_ex, c->u_it, sizeof(double) * c->n_dof, cudaMemcpyDeviceToDevice, s));
            CK(mlp_sync(ws.mlp));
            CK(mlp_forward_on(ws.mlp, ws_X, c->n_nodes, ws.Y, s));
            CK(ws_project(ws_X, ws.Y, c->free_dof, ws.prob_dof, c->n_prob, c->dim, s));
            CK(ws_apply(c->u_it, ws.Y, ws.node_prob, ws.scale, c->n_prob, c->free_dof, c->dim, c->n_dof, s));
            CK(cudaMemcpyAsync(ws.uL, c->u_it, sizeof(double) * c->n_dof, cudaMemcpyDeviceToDevice, s));
            ws.uL_valid = true;
            c->launches += 3;
            std::vector<double> r_L;
            double rel_L = 0.0;
            st = start_residuals(c, c->u_it, z, r_L, &rel_L);
            if (st != EP_OK) return st;
            rep.n_assemble += 1;
            bool any_ex = false, any_L = false;
            for (int p = 0; p < c->n_prob; ++p) {
                ws.h_take[p] = r_L[p] <= r_ex[p] ? 0 : 1;
                any_ex = any_ex || ws.h_take[p];
                any_L = any_L || !ws.h_take[p];
            }
            if (any_ex) {
                CK(cudaMemcpyAsync(ws.take_ex, ws.h_take.data(), c->n_prob, cudaMemcpyHostToDevice, s));
                CK(ws_select(c->u_it, ws.u_ex, ws.node_prob, ws.take_ex, c->dim, c->n_dof, s));
                CK(cudaStreamSynchronize(s));   // h_take is read by the copy
                c->launches += 1;
            }
            if (any_L) rep.start = 2;
            for (int p = 0; p < c->n_prob; ++p) rep.n_learned += ws.h_take[p] ? 0 : 1;
        }
        CK(cudaMemsetAsync(c->err_flag, 0, sizeof(int), s));
        st = EP_OK;
        rel = 0.0;
        it = 0;
        converged = false;
        double rnorm_prev = -1.0, rel_best = 1e300;
        double rel_prev = -1.0;  // largest per-problem relative residual before the last solve
        bool use32 = false;      // this iteration's tangent and solve in FP32
        bool fp64_step = false;  // the rest of this step in FP64 (an FP32 iteration contracted poorly)
        double eta_prev = 1.0;   // Krylov tolerance of the last solve
        // The last solve aimed at the Newton tolerance itself and Newton contracted well: the iterate
        // is expected to converge, so F is evaluated alone first and the tangent only if it does not.
        bool f_first = false;
        double last_ratio = 1.0;  // ||r|| / ||r_prev|| of this iteration (1: first iteration)
        int fact_it = -1;         // Newton iteration of this attempt whose tangent the sparse LU holds
        for (;;) {
            use32 = mixed && !c->mixed_fallback && !fp64_step && !c->direct_mode;
            CK(cudaEventRecord(c->ev[0], s));
            st = assemble(c, c->u_it, split, !f_first, use32);
            if (st != EP_OK) break;
            CK(cudaEventRecord(c->ev[1], s));
            CK(vec_residual(c->f_unit, z, c->F, c->free_dof, c->r, use32 ? c->r32 : nullptr, c->n_dof, c->kw.part,
                            c->kw.nparts, c->norms, s));
            c->launches += 2;
            rep.n_assemble += 1;
            const int64_t nchunk = (int64_t)c->chunk_prob.size();
            if (c->n_prob > 1) {
                CK(vec_chunk_norms(c->f_unit, z, c->F, c->free_dof, c->r, c->d_chunks, nchunk, c->d_chunk_norms, s));
                CK(cudaMemcpyAsync(c->h_chunk_norms.data(), c->d_chunk_norms, sizeof(double) * 3 * nchunk,
                                   cudaMemcpyDeviceToHost, s));
                c->launches += 1;
            }
            CK(cudaMemcpyAsync(c->norms_host, c->norms, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
            CK(cudaMemcpyAsync(c->err_host, c->err_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
            CK(cudaMemcpyAsync(c->counter_host, c->counter, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]));
            t_asm += ms;
            if (c->profile) {
                CK(cudaEventElapsedTime(&ms, c->ev[4], c->ev[5]));
                t_asm_kernel += ms;
            }
            rep.n_plastic_assembled += (int64_t)c->counter_host[0];
            if (!f_first) rep.n_plastic_elem_assembled += (int64_t)c->counter_host[1];
            if (*c->err_host) {
                c->err = "return mapping: apex reached with K*eta*eta_bar + Hc = 0 (no admissible stress)";
                st = EP_ERR_RETURN_MAP;
                break;
            }
            const double rnorm = std::sqrt(c->norms_host[0]);
            const double scale = std::max(std::sqrt(c->norms_host[1]), std::sqrt(c->norms_host[2]));
            if (!std::isfinite(rnorm) || !std::isfinite(scale)) {
                c->err = "non-finite residual norm";
                st = EP_ERR_NAN;
                break;
            }
            rel = scale > 0.0 ? rnorm / scale : rnorm;
            if (c->n_prob > 1) {
                // a batch converges when every problem does, each relative to its own load and forces
                std::vector<double> pr(c->n_prob, 0.0), pf(c->n_prob, 0.0), pF(c->n_prob, 0.0);
                for (int64_t i = 0; i < nchunk; ++i) {
                    const int64_t p = c->chunk_prob[i];
                    pr[p] += c->h_chunk_norms[i];
                    pf[p] += c->h_chunk_norms[nchunk + i];
                    pF[p] += c->h_chunk_norms[2 * nchunk + i];
                }
                rel = 0.0;
                for (int p = 0; p < c->n_prob; ++p) {
                    const double sc = std::max(std::sqrt(pf[p]), std::sqrt(pF[p]));
                    const double rp = std::sqrt(pr[p]);
                    rel = std::max(rel, sc > 0.0 ? rp / sc : rp);
                }
            }
            if (rel <= o.newton_rtol || rnorm == 0.0) {
                converged = true;
                break;
            }
            if (f_first) {   // not converged after all: the same iterate again, with the tangent
                f_first = false;
                continue;
            }
            if (it >= o.newton_maxit) {
                st = EP_ERR_NEWTON_NO_CONVERGENCE;
                c->err = "Newton: no convergence in " + std::to_string(o.newton_maxit) + " iterations";
                break;
            }
            // from an extrapolated start, a residual that keeps growing (10x above the best after 5
            // iterations) ends the attempt early
            rel_best = std::min(rel_best, rel);
            if (extrapolated && it >= 5 && rel > 10.0 * rel_best) {
                st = EP_ERR_NEWTON_NO_CONVERGENCE;
                c->err = "Newton: diverging from the extrapolated start";
                break;
            }
            // forcing term
            double eta;
            if (o.krylov_rtol > 0.0) eta = o.krylov_rtol;
            else {
                const double eta_min = 0.5 * o.newton_rtol * scale / rnorm;
                // the mixed path's FP32 iterations keep the tighter terms (see eta0_mixed); its
                // FP64-tangent iterations take the FP64 path's
                const bool t32 = mixed && !c->mixed_fallback && !fp64_step;
                const double e0 = t32 ? c->eta0_mixed : c->eta0, emax = t32 ? c->eta_max_mixed : c->eta_max;
                const double eta_ew = (rnorm_prev < 0.0) ? e0 : 0.9 * (rnorm / rnorm_prev) * (rnorm / rnorm_prev);
                eta = std::min(emax, std::max(eta_ew, eta_min));
                eta = std::max(eta, 1e-14);
            }
            // FP32 phase of the mixed path: if the last FP32 Newton step barely reduced the FP64
            // residual, the FP32 tangent is too coarse here; this and later steps use FP64, starting
            // with an FP64 assembly at the same iterate (this iteration's tangent is FP32)
            // (this iteration's tangent is FP32: on a switch the same iterate is re-assembled in FP64)
            if (use32 && rnorm_prev > 0.0 && rnorm > MIXED_STALL_RATIO * rnorm_prev) {
                c->mixed_fallback = true;
                if (c->verbose) std::fprintf(stderr, "[ep] step %d: FP32 tangent stalled, FP64 from here\n", k);
                continue;
            }
            // a batch converges when its worst problem does: an FP32 iteration that leaves the worst
            // relative residual above half its previous value (a small problem at FP32 rounding
            // level while the batch's norm, dominated by the large ones, still contracts) finishes
            // the step in FP64
            if (use32 && c->n_prob > 1 && rel_prev > 0.0 && rel > MIXED_STALL_RATIO * rel_prev) {
                fp64_step = true;
                if (c->verbose > 1)
                    std::fprintf(stderr, "[ep] step %d: worst problem %.2e after %.2e on the FP32 tangent, FP64 tangent\n",
                                 k, rel, rel_prev);
                continue;
            }
            if (use32 && rnorm_prev > 0.0 && rnorm > MIXED_RHO_FACTOR * eta_prev * rnorm_prev) {
                fp64_step = true;
                if (c->verbose > 1)
                    std::fprintf(stderr, "[ep] step %d: FP32 contraction %.2e vs tolerance %.2e, FP64 tangent\n", k,
                                 rnorm / rnorm_prev, eta_prev);
                continue;
            }
            // with no plastic point the tangent is K_elast, symmetric: CG suffices even for a
            // nonassociated model
            // the preconditioner of this solve: the sparse LU once the path has switched to it (with
            // GMRES: its factors are not symmetric in rounding)
            const int pk = c->direct_mode ? 3 : o.precond;
            const int m_it = pk == 3 ? 3 : (o.krylov == 0 && *c->counter_host == 0) ? 1 : method;
            // the mixed path's FP64-tangent iterations solve with GMRES on the FP64 operator and an
            // FP32 basis (orthogonalisation, preconditioner and basis in FP32)
            const bool basis32 = mixed && !use32 && m_it == 3 && !c->amg.precise && !c->direct_mode;
            // an FP32 inner solve cannot go much below FP32 rounding; Newton (FP64 residual) refines further
            if (use32 || basis32) eta = std::max(eta, MIXED_ETA_MIN);
            // this solve aims at the final tolerance (its forcing term is the floor eta_min) after a
            // strongly contracting iteration: expect convergence at the next iterate
            f_first = o.krylov_rtol <= 0.0 && eta * rnorm <= 0.5000001 * o.newton_rtol * scale &&
                      rnorm_prev > 0.0 && rnorm < 0.1 * rnorm_prev;
            last_ratio = rnorm_prev > 0.0 ? rnorm / rnorm_prev : 1.0;
            rnorm_prev = rnorm;
            rel_prev = rel;
            eta_prev = eta;
            CK(cudaEventRecord(c->ev[2], s));
            // Coarse operators: rebuilt (Galerkin, from the current tangent) at the first Newton
            // iteration of a step and whenever the plastic set changed by more than 5% of the points
            // since the last rebuild; otherwise the last ones are reused (a preconditioner need not
            // follow the tangent exactly; level 0 always is the current tangent).  An elastic
            // tangent is K_elast, whose coarse operators are kept from the setup.
            const int64_t np_now = (int64_t)*c->counter_host;
            const bool tangent_elastic = split && np_now == 0;
            if (tangent_elastic) c->kw.galerkin = c->amg_elastic ? 0 : 1;
            else c->kw.galerkin = (c->amg_elastic || it == 0 || std::llabs(np_now - c->amg_np) * 20 > c->n_int) ? 1 : 0;
            if (c->deterministic && it == 0) {
                // a step's preconditioner depends on nothing before the step: coarse operators from
                // this tangent, spectral estimate from the fixed start vector
                c->kw.galerkin = 1;
                c->amg.pw0_valid = false;
            }
            if (c->kw.galerkin) {
                c->amg_elastic = tangent_elastic;
                c->amg_np = np_now;
            }
            int kits = 0, kst = 0;
            double krel = 0.0;
            const bool direct_before = c->direct_mode;
            // The FP64 solve: the sparse LU once the path has switched to it (to DIRECT_ETA: near a
            // limit load the tangent is nearly singular, and a loose forcing term leaves large errors
            // along its soft modes, from which the semismooth iteration diverges), else the options'
            // preconditioner; a GMRES solve that stalls with the V-cycle switches the path to the
            // sparse LU, or where that cannot be set up to the precise V-cycle.
            auto solve64 = [&](int& its_out, double& rel_out, int& st_out) -> ep_status {
                // inside Newton a solve that needs far more than the usual count is not worth
                // finishing: its partial progress is taken as an inexact step
                const int maxit64 = std::min(o.krylov_maxit, std::max(2000, 20 * c->kw.last_its));
                const double eta_d = o.krylov_rtol > 0.0 ? eta : std::min(eta, DIRECT_ETA);
                if (c->direct_mode || pk == 3) {
                    c->kw.stall_guard64 = 1;   // a solve at the rounding floor of the FP64 residual stops
                    // Deep in Newton's quadratic phase the tangent barely moves between iterations: the
                    // previous iteration's factors precondition this system (the operator is the
                    // current tangent, so the Newton step is the same); a solve that misses the
                    // tolerance within DIRECT_REUSE_MAXIT iterations is refactored and done again.
                    // (Oracle tangents of the 0.98 t_lim column, 64x64 cells, GMRES to 1e-10: the
                    // previous LU needs 3 iterations against 2 at residual 7e-10, 7 against 2 at 3e-6,
                    // and fails at 2e-4.)
                    if (fact_it == it - 1 && rel <= 1e-6 && last_ratio <= 1e-2 && krylov_keep_direct(c->kw)) {
                        CK(krylov_solve(A, c->kw, c->r, 3, eta_d, DIRECT_REUSE_MAXIT, s, &its_out, &rel_out, &st_out));
                        if (st_out == EP_OK) {
                            c->kw.stall_guard64 = 0;
                            return EP_OK;
                        }
                        if (c->verbose)
                            std::fprintf(stderr, "[ep] step %d: previous factors missed (rel %.3e after %d), refactoring\n",
                                         k, rel_out, its_out);
                    }
                    int k2 = 0;
                    CK(krylov_precond(A, c->kw, 3, s));
                    fact_it = it;
                    CK(krylov_solve(A, c->kw, c->r, 3, eta_d, maxit64, s, &k2, &rel_out, &st_out));
                    its_out += k2;
                    c->kw.stall_guard64 = 0;
                    return EP_OK;
                }
                const bool can_switch = pk == 2 && c->amg_built && !c->amg.precise && m_it == 3;
                c->kw.stall_guard64 = can_switch ? 1 : 0;
                CK(krylov_precond(A, c->kw, pk, s));
                CK(krylov_solve(A, c->kw, c->r, m_it, eta, maxit64, s, &its_out, &rel_out, &st_out));
                c->kw.stall_guard64 = 0;
                if (st_out == EP_ERR_KRYLOV && can_switch) {
                    // the V-cycle cannot resolve this tangent's soft modes (a limit load is near:
                    // eigenvalues with negative real parts, around which restarted GMRES stalls)
                    int k2 = 0;
                    if (o.direct_fallback && ensure_direct(c)) {
                        c->direct_mode = true;
                        if (c->verbose)
                            std::fprintf(stderr, "[ep] step %d: V-cycle GMRES stalled (rel %.3e after %d), sparse LU from here\n",
                                         k, rel_out, its_out);
                        // after earlier V-cycle iterations of this step the step starts again (see
                        // below): nothing to solve at this iterate
                        if (it == 0) {
                            c->kw.stall_guard64 = 1;
                            CK(krylov_precond(A, c->kw, 3, s));
                            fact_it = it;
                            CK(krylov_solve(A, c->kw, c->r, 3, eta_d, maxit64, s, &k2, &rel_out, &st_out));
                            c->kw.stall_guard64 = 0;
                        }
                    } else {
                        c->amg.precise = 1;
                        c->kw.galerkin = 1;
                        c->amg_np = np_now;
                        c->amg_elastic = false;
                        if (c->verbose)
                            std::fprintf(stderr, "[ep] step %d: FP32 V-cycle stalled (rel %.3e after %d), precise V-cycle from here%s%s\n",
                                         k, rel_out, its_out, o.direct_fallback ? " (" : "",
                                         o.direct_fallback ? (c->direct.why + ")").c_str() : "");
                        CK(krylov_precond(A, c->kw, pk, s));
                        CK(krylov_solve(A, c->kw, c->r, m_it, eta, maxit64, s, &k2, &rel_out, &st_out));
                        rep.precise = 1;
                    }
                    its_out += k2;
                }
                return EP_OK;
            };
            // inside Newton a stagnating FP32-basis solve is cut short (the FP64 path takes over)
            c->kw.stall_guard = 1;
            if (use32) {
                rep.newton_its_fp32 += 1;
                // an FP32 solve that needs far more iterations than usual is stagnating on rounding
                const int maxit32 = std::min(o.krylov_maxit, std::max(300, 4 * c->kw.last_its));
                CK(krylov_precond(Af, c->kw, pk, s));
                CK(krylov_solve(Af, c->kw, c->r32, m_it, eta, maxit32, s, &kits, &krel, &kst));
            } else if (basis32) {
                const int maxit32 = std::min(o.krylov_maxit, std::max(300, 4 * c->kw.last_its));
                CK(krylov_precond(A, c->kw, pk, s));
                CK(krylov_solve_fp32_basis(A, c->kw, c->r, eta, maxit32, s, &kits, &krel, &kst));
                if (kst != EP_OK && !(krel < 0.5)) {   // no progress with the FP32 basis: the FP64 solve
                    int k2 = 0;
                    st = solve64(k2, krel, kst);
                    if (st != EP_OK) return st;
                    kits += k2;
                }
                if (kst != EP_OK && krel < 0.5) kst = EP_OK;   // partial progress: an inexact Newton step
            } else {
                st = solve64(kits, krel, kst);
                if (st != EP_OK) return st;
            }
            if (c->direct_mode || pk == 3) {
                rep.direct = 1;
                if (c->verbose) {
                    unsigned int npert = 0;
                    cudaMemcpy(&npert, c->direct.n_perturbed, sizeof(npert), cudaMemcpyDeviceToHost);
                    std::fprintf(stderr, "[ep] step %d: sparse LU, %u perturbed pivots\n", k, npert);
                }
            }
            if (c->amg.precise) rep.precise = 1;
            c->kw.stall_guard = 0;
            CK(cudaEventRecord(c->ev[3], s));
            rep.krylov_its += kits;
            if (c->verbose)
                std::fprintf(stderr, "[ep] step %d zeta %.6g newton %d rel %.3e eta %.2e krylov(%s) its %d rel %.3e done %d why %d\n",
                             k, z, it, rel, eta, m_it == 1 ? "cg" : (m_it == 2 ? "bicgstab" : "gmres"), kits, krel, c->kw.rec_host->done,
                             c->kw.rec_host->why);
            if (c->verbose > 1 && kst != EP_OK) {
                std::vector<double> h(3 * c->kw.hist_len);
                cudaMemcpy(h.data(), c->kw.hist, sizeof(double) * h.size(), cudaMemcpyDeviceToHost);
                const int n = std::min(kits + 1, c->kw.hist_len);
                for (int j = std::max(0, n - 6); j < n; ++j)
                    std::fprintf(stderr, "[ep]   it %d rho %.6e alpha %.6e omega %.6e\n", j, h[j], h[c->kw.hist_len + j],
                                 h[2 * c->kw.hist_len + j]);
            }
            if (!direct_before && c->direct_mode && it > 0) {
                // switched to the sparse LU after iterations with the V-cycle: the step starts again
                // from its start iterate, every Newton step now solved accurately.  (Near the limit
                // load the tangent has unstable modes: the non-homogeneous error a loose solve leaves
                // in the iterate grows, and Newton can settle on another solution branch.)
                CK(cudaEventSynchronize(c->ev[3]));
                CK(cudaEventElapsedTime(&ms, c->ev[2], c->ev[3]));
                t_sol += ms;
                redo_step = true;
                if (c->verbose) std::fprintf(stderr, "[ep] step %d: again from the start iterate with the sparse LU\n", k);
                break;
            }
            if (kst == EP_ERR_NAN) {
                st = EP_ERR_NAN;
                c->err = "Krylov: non-finite residual";
                break;
            }
            if (kst != EP_OK && use32) {
                // the FP32 inner solve stagnated: FP32 is too coarse for this tangent; keep the step if
                // it made progress, and continue the load path in FP64
                c->mixed_fallback = true;
                if (c->verbose) std::fprintf(stderr, "[ep] step %d: FP32 solve stagnated, FP64 from here\n", k);
                if (!(krel < 0.5)) continue;   // no progress: redo this iteration in FP64
                kst = EP_OK;
            }
            if (kst != EP_OK && !(krel < 0.5)) {
                // accept a partially converged solve as an inexact Newton step; fail only if it made no progress
                st = EP_ERR_KRYLOV;
                c->err = "Krylov: no progress (relative residual " + std::to_string(krel) + ")";
                break;
            }
            if (use32) CK(vec_axpy_f32(c->u_it, c->kw.f.x, c->n_dof, s));
            else CK(vec_axpy(c->u_it, 1.0, c->kw.d.x, c->n_dof, s));
            c->launches += 1;
            CK(cudaEventSynchronize(c->ev[3]));
            CK(cudaEventElapsedTime(&ms, c->ev[2], c->ev[3]));
            t_sol += ms;
            ++it;
        }
        if (redo_step) {
            redo_step = false;
            --attempt;
            continue;
        }
        if (converged || !extrapolated ||
            (st != EP_ERR_NEWTON_NO_CONVERGENCE && st != EP_ERR_KRYLOV && st != EP_ERR_NAN))
            break;
        if (c->verbose) std::fprintf(stderr, "[ep] step %d: retrying from the last converged state\n", k);
        }   // attempt
        rep.newton_its = it;
        rep.rel_resid = rel;
        rep.t_assemble_ms = t_asm;
        rep.t_solve_ms = t_sol;
        if (converged) {
            unsigned long long np = 0;
            st = commit(c, c->u_it, &np);
            rep.n_plastic = (int64_t)np;
            if (st == EP_OK && ws.ready) {
                // warm-start history: plastic fractions after step k, the recorded targets, then
                // u_{k-3} <- u_{k-2} <- u_{k-1} <- u_k
                CK(cudaMemsetAsync(ws.cnt_pl, 0, sizeof(int32_t) * c->n_nodes, s));
                CK(ws_node_counts(c->elem, c->n_elem, c->n_p, c->n_q, c->flag, ws.cnt_pl, s));
                CK(ws_fraction(ws.cnt_pl, ws.cnt_ip, c->n_nodes, ws.pfk, s));
                CK(ws_proximity(mesh_dev(c), c->sig, c->hard, c->n_p, c->n_q, c->dim, ws.prox1, s));
                c->launches += 3;
                if (ws_feat && ws_rec) {
                    CK(ws_targets(c->u_it, c->u, c->u_prev, ws_ratio, ws.node_prob, ws.scale, c->n_prob, c->free_dof,
                                  ws.pfk, c->dim, c->n_nodes, ws.rec_T + ws.rec_n * EP_WS_N_OUT, s));
                    c->launches += 1;
                    ws.rec_n += c->n_nodes;
                }
                float* pf = ws.pf2;
                ws.pf2 = ws.pf1;
                ws.pf1 = ws.pfk;
                ws.pfk = pf;
                double* u3 = ws.u3;
                ws.u3 = c->u_prev;
                c->u_prev = c->u;
                c->u = c->u_it;
                c->u_it = u3;
                ws.zeta3 = c->zeta_prev;
                ws.hist++;
                c->zeta_prev = c->zeta_last;
                c->zeta_last = z;
                c->n_committed++;
            } else if (st == EP_OK) {
                std::swap(c->u_prev, c->u);     // u_prev <- u_{k-1}
                std::swap(c->u, c->u_it);       // u <- u_k
                c->zeta_prev = c->zeta_last;
                c->zeta_last = z;
                c->n_committed++;
            }
        }
        CK(cudaStreamSynchronize(s));
        rep.t_step_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_step0).count();
        rep.status = st;
        rep.launches = c->launches + c->kw.launches + c->amg.launches + c->direct.launches;
        rep.n_direct_factor = c->direct.n_factor - dfac0;
        rep.n_direct_solve = c->direct.n_solve - dsol0;
        rep.t_direct_factor_ms = c->direct.factor_ms - dfms0;
        rep.t_direct_solve_ms = c->direct.solve_ms - dsms0;
        rep.direct_factor_flop = c->direct.ready ? c->direct.plan.flops : 0.0;
        rep.direct_solve_bytes = c->direct.ready ? c->direct.solve_bytes : 0.0;
        rep.n_spmv = c->kw.spmv_n;
        rep.t_spmv_kernel_ms = c->kw.spmv_ms;
        rep.n_smooth0 = c->amg.smooth0_n;
        rep.t_smooth0_kernel_ms = c->amg.smooth0_ms;
        rep.t_assemble_kernel_ms = t_asm_kernel;
        if (reports) reports[k] = rep;
        if (st != EP_OK) return st;
    }
    return EP_OK;
}

ep_status ep_constitutive(const ep_material* mat, int32_t dim, int64_t n, const double* E, const double* ep_prev,
                          const double* hard_prev, double* S, double* DS, uint8_t* flag, double* ep_new,
                          double* hard_new, void* cuda_stream) {
    if (!mat || (dim != 2 && dim != 3) || n < 0) return EP_ERR_INVALID_ARG;
    if (n == 0) return EP_OK;
    if (!E || !ep_prev || !hard_prev || !S || !DS || !flag || !ep_new || !hard_new) return EP_ERR_INVALID_ARG;
    MatConst m;
    std::string err;
    if (!make_matconst(*mat, dim, m, err)) return EP_ERR_INVALID_ARG;
    cudaError_t e = launch_constitutive(dim, m, n, E, ep_prev, hard_prev, S, DS, flag, ep_new, hard_new,
                                        static_cast<cudaStream_t>(cuda_stream));
    return e == cudaSuccess ? EP_OK : EP_ERR_CUDA;
}

}  // extern "C"
