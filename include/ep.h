/*
 * ep.h -- C ABI of the GB300 elastoplastic hot path.
 *
 * The library solves the incremental elastoplastic problem (P_k) of Section 1
 * (eq. (eqn)) by the finite element method of Section 3 and the semismooth
 * Newton method ALG-NEWTON of Section 4.  Every Newton iteration evaluates the
 * stress-strain operator T_k and its consistent tangent T_k^o at all
 * integration points (Sections 2.2, 2.3), assembles the internal forces F and
 * the tangent stiffness K = B^T W D_p B (Section 7, eq. (K-split); Section 9,
 * eq. (K-split_Petr)) into a block-CSR pattern fixed by the mesh, and solves
 * eq. (lin_syst) on the free DOFs with a preconditioned Krylov method.
 *
 * Conventions (Section 5):
 *   - DOF index = dim*node + component (the ordering of U(:)).
 *   - Integration point index = element*n_q + q.
 *   - Voigt order, 3D: (11,22,33,12,23,13); stresses stress-type, strains
 *     and plastic strains strain-type (engineering shear).
 *   - Plane strain (dim = 2) stores n_comp = 4 components per point in the
 *     order (11,22,12,33); 3D stores n_comp = 6.
 *   - Per-point fields are structure-of-arrays: [n_comp][n_int].
 *
 * Memory and errors:
 *   - Inputs passed to ep_create are host arrays, copied during the call; the
 *     caller keeps ownership.  The library owns every device buffer of a
 *     context and frees them in ep_destroy.
 *   - Every function returns an ep_status and never aborts or traps.  The
 *     message of the last failure of a context is available from
 *     ep_last_error.  A load step that fails leaves the state at the last
 *     converged step.
 *   - All device work of a context runs on the CUDA stream given to
 *     ep_create; one context must not be used from two host threads at once.
 */
#ifndef EP_H
#define EP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    EP_OK = 0,
    EP_ERR_INVALID_ARG = 1,          /* bad pointer, size, enum value or node index */
    EP_ERR_CUDA = 2,                 /* a CUDA runtime call failed; see ep_last_error */
    EP_ERR_OOM = 3,                  /* device allocation failed */
    EP_ERR_BAD_ELEMENT = 4,          /* det J <= 0 at an integration point (Section 6.1) */
    EP_ERR_RETURN_MAP = 5,           /* Drucker-Prager apex with K*eta*eta_bar + Hc = 0: no admissible stress */
    EP_ERR_NEWTON_NO_CONVERGENCE = 6,/* newton_maxit reached */
    EP_ERR_KRYLOV = 7,               /* Krylov iteration cap or breakdown */
    EP_ERR_NAN = 8,                  /* NaN/Inf in a residual norm */
    EP_ERR_STATE = 9                 /* call out of order (e.g. no assembled matrix) */
} ep_status;

/* Element families of the Appendix (3D) and their plane analogues (2D). */
typedef enum { EP_P1 = 0, EP_P2 = 1, EP_Q1 = 2, EP_Q2 = 3 } ep_elem;

/* Constitutive models (Sections 2.2, 2.3 and their extensions). */
typedef enum {
    EP_ELASTIC = 0,   /* T = C eps (eq. (elastic_operator)) */
    EP_VM_KIN = 1,    /* von Mises, linear kinematic hardening a = H (eqs. (T_kinematic), (DT_kinematic)) */
    EP_VM_ISO = 2,    /* von Mises, linear isotropic hardening: |s| <= Y + H*alpha */
    EP_DP = 3         /* Drucker-Prager; nonassociated (psi != phi) and cohesion hardening Hc optional */
} ep_model;

/*
 * Arithmetic of a solve.  EP_FP64: every step in FP64.  EP_MIXED: strains, the
 * return mapping (yield test and plastic multiplier), the internal forces F,
 * the Newton residual and its norms and the update of u stay FP64; the
 * tangent D_p is rounded to FP32 per point and the local element matrices,
 * their assembly into K and the inner Krylov solve (vectors, SpMV,
 * preconditioner) run in FP32.  Newton on the FP64 residual is the outer
 * refinement, so the load path still reaches newton_rtol; the inner relative
 * tolerance is not taken below 1e-5.  Newton on an FP32 tangent contracts
 * only linearly (by about cond(K) * 2^-24 per iteration): once an FP32
 * iteration reduces the FP64 residual by less than 1/(10 eta) (eta its Krylov
 * tolerance), the same iterate is re-assembled and the step continues with the
 * FP64 tangent, solved by GMRES on the FP64 operator with an FP32 Krylov basis
 * and preconditioner (CG, for symmetric tangents, in FP64).  When a Newton
 * iteration on the FP32 tangent reduces
 * the FP64 residual by less than half (an ill-conditioned tangent, e.g. near a
 * limit load), that load step and the rest of the path continue in FP64
 * (until EP_U is set again).
 */
typedef enum { EP_FP64 = 0, EP_MIXED = 1 } ep_precision;

/* Mesh (Section 6: ELEM and COORD).  Host pointers, copied by ep_create. */
typedef struct {
    int32_t dim;                 /* 2 (plane strain) or 3 */
    int32_t elem;                /* ep_elem */
    int64_t n_nodes;
    int64_t n_elem;
    const double* coords;        /* [n_nodes][dim] */
    const int32_t* elem_nodes;   /* [n_elem][n_p], 0-based, reference node order of the Appendix */
} ep_mesh;

/* Material (Sections 2.2, 2.3, 8.3).  K = E/(3(1-2nu)), G = E/(2(1+nu)). */
typedef struct {
    int32_t model;               /* ep_model */
    double E, nu;
    double Y, H;                 /* von Mises: yield value (Frobenius norm of the deviator) and hardening modulus */
    double c0, phi, psi, Hc;     /* Drucker-Prager: cohesion, friction and dilatancy angles [rad], cohesion hardening */
} ep_material;

/* Boundary conditions and loads (Section 4: u_D, f).  Host pointers, copied. */
typedef struct {
    const uint8_t* dirichlet_mask;  /* [n_nodes*dim], 1 = prescribed DOF (complement of Q, Section 5) */
    const double* u_D_unit;         /* [n_nodes*dim], prescribed values at zeta = 1 (NULL = zero) */
    const double* f_ext_unit;       /* [n_nodes*dim], external load vector at zeta = 1 (NULL = zero) */
} ep_bc;

typedef struct {
    int32_t precision;           /* ep_precision */
    double newton_rtol;          /* ||(f - F)_free|| <= rtol * max(||f_free||, ||F||) */
    int32_t newton_maxit;
    int32_t krylov;              /* 0 auto (CG if the tangent is symmetric, else GMRES), 1 CG, 2 BiCGStab, 3 GMRES(30) */
    double krylov_rtol;          /* > 0: fixed relative tolerance; 0: adaptive forcing term */
    int32_t krylov_maxit;
    int32_t precond;             /* 0 Jacobi, 1 block Jacobi (dim x dim node blocks), 2 smoothed-aggregation AMG
                                    (built from K_elast on first use; Chebyshev/block-Jacobi smoothing),
                                    3 sparse LU of the tangent (multifrontal, nested-dissection order, FP64
                                    factors with static pivoting, refactored at every Newton iteration; with
                                    GMRES, which refines to the FP64 tolerance).  The paper solves eq.
                                    (lin_syst) directly; 3 is its counterpart here.  Set up on first use:
                                    EP_ERR_STATE if the factors would not fit in 60% of the free device memory
                                    or a front exceeds the solve's shared-memory limit (order 24 000) */
    int32_t split_elastic_cache; /* 1: K = K_elast + sum over plastic points (eq. (K-split)); 0: K = B^T D B */
    int32_t warm_start;          /* 0: last converged u; 1: linear extrapolation of the last two steps;
                                    2: the extrapolation corrected by the attached warm-start network
                                    (ep_ws_attach), judged per problem against the plain extrapolation */
    int32_t profile;             /* 1: time the assembly and SpMV kernels with CUDA events (fills t_*_kernel_ms) */
    int32_t deterministic;       /* 1: bit-reproducible runs.  Elements are coloured at ep_create (no two elements
                                    of a colour share a node) and the assembly runs one launch per colour with
                                    plain adds into F and K instead of atomics; the AMG Galerkin products sum in
                                    a fixed order; the preconditioner's spectral estimate and coarse operators are
                                    rebuilt from the tangent at the first Newton iteration of every load step, so
                                    a step depends only on its start state (a run resumed with ep_set from a saved
                                    state repeats the uninterrupted run bit for bit when warm_start = 0).  The
                                    setting stays with the context: later ep_assemble / ep_commit calls follow
                                    the last ep_solve_load_path or ep_linear_solve that passed it (n_steps = 0
                                    sets it without solving). */
    int32_t asm_tile;            /* assembly schedule: 1 the element type's tile of elements per CTA (default),
                                    2 half of it (half the shared memory per CTA, more CTAs per SM) */
    int32_t krylov_graphs;       /* 1 (default): the GMRES iterations are captured once per solver configuration
                                    as CUDA graphs and replayed (one launch per iteration instead of about 30);
                                    0: direct launches.  Either way the same kernels run in the same order.
                                    profile = 1 always launches directly (events around the kernels). */
    int32_t direct_fallback;     /* 1 (default): with precond = 2, when a GMRES solve stalls with the V-cycle
                                    (near a limit load the nonassociated tangent has eigenvalues with negative
                                    real parts, Section 2.3), the rest of the load path is solved with the
                                    sparse LU (precond 3), or, where its factors do not fit, with the precise
                                    V-cycle; 0: always the precise V-cycle */
} ep_opts;

typedef struct {
    int32_t newton_its;
    int32_t krylov_its;          /* summed over the step's linear solves */
    int64_t n_plastic;           /* plastic integration points after the step */
    double rel_resid;
    double t_assemble_ms, t_solve_ms, t_step_ms;
    int32_t status;              /* ep_status of the step */
    int32_t launches;            /* kernels of this library launched during the step */
    int32_t n_assemble;          /* assembly kernel launches */
    int32_t n_spmv;              /* SpMV kernel launches that did work (profile = 1) */
    double t_assemble_kernel_ms; /* summed duration of the assembly kernel launches (profile = 1) */
    double t_spmv_kernel_ms;     /* summed duration of those SpMV launches (profile = 1) */
    int64_t n_plastic_assembled; /* plastic points summed over the step's assemblies (local-tangent work done) */
    int32_t newton_its_fp32;     /* EP_MIXED: Newton iterations of the step that used the FP32 tangent and solve */
    int32_t start;               /* Newton start used: 0 last converged u, 1 extrapolated, 2 learned (for at
                                    least one problem of a batch) */
    int32_t n_learned;           /* warm_start = 2: problems that kept the learned start */
    int32_t n_smooth0;           /* AMG level-0 Chebyshev launches timed (profile = 1; a sample: the pre-smoothing
                                    sweeps of the first V-cycles of every chunk of Krylov iterations) */
    double t_smooth0_kernel_ms;  /* their summed duration (profile = 1) */
    int64_t n_plastic_elem_assembled;   /* elements with a plastic point, summed over the step's assemblies that
                                           formed a tangent (their blocks are the ones the split form rewrites) */
    int32_t precise;             /* 1: the step's preconditioner used the precise V-cycle (FP64 coarse correction;
                                    switched on for the rest of the path when GMRES stalled with the FP32 one) */
    int32_t direct;              /* 1: the step solved with the sparse LU (precond 3, or switched to it for the
                                    rest of the path when GMRES stalled with the V-cycle) */
    int32_t n_direct_factor;     /* sparse-LU factorisations of the step */
    int32_t n_direct_solve;      /* sparse-LU solves (preconditioner applications) of the step */
    double t_direct_factor_ms;   /* their summed durations (profile = 1) */
    double t_direct_solve_ms;
    double direct_factor_flop;   /* FLOP of one factorisation (partial LU of every front) */
    double direct_solve_bytes;   /* bytes of the factors one solve reads */
} ep_step_report;

/* Fields readable with ep_get / writable with ep_set. */
typedef enum {
    EP_U = 0,                /* double [n_nodes*dim], displacements u_k */
    EP_STRESS = 1,           /* double [n_comp][n_int], committed stress sigma_k */
    EP_PLASTIC_STRAIN = 2,   /* double [n_comp][n_int], committed eps^p_k (strain-type) */
    EP_HARDENING = 3,        /* double [n_int] (alpha) or [n_comp][n_int] (back stress, EP_VM_KIN) */
    EP_PLASTIC_FLAG = 4,     /* uint8 [n_int]: 0 elastic, 1 plastic (DP: 1 smooth, 2 apex) */
    EP_F_INT = 5,            /* double [n_nodes*dim], internal forces F of the last assembly (read only) */
    EP_K_ROW_PTR = 6,        /* int32 [n_nodes+1], block-CSR row pointers (read only) */
    EP_K_COL_IDX = 7,        /* int32 [nnz_blocks], block column (node) indices (read only) */
    EP_K_VALUES = 8,         /* double [nnz_blocks][dim][dim], K of the last assembly, row-major blocks (read only) */
    EP_K_ELASTIC = 9,        /* double [nnz_blocks][dim][dim], K_elast (read only) */
    EP_WEIGHT = 10,          /* double [n_int], |det J| w_q (Section 6.3, WEIGHT) (read only) */
    EP_DPHI = 11,            /* double [n_int][n_p][dim], physical basis gradients (Section 6.1, DPhi) (read only) */
    EP_SOLUTION = 12,        /* double [n_nodes*dim], x of the last ep_linear_solve (read only) */
    EP_K_VALUES_F32 = 13,    /* float [nnz_blocks][dim][dim], K of the last EP_MIXED assembly (read only;
                                EP_ERR_STATE before the first one) */
    EP_WS_X = 14,            /* float [n_rows][16], recorded warm-start inputs (read only; EP_ERR_STATE when
                                not recording; n_rows from ep_ws_samples) */
    EP_WS_T = 15,            /* float [n_rows][4], recorded warm-start targets (read only, as EP_WS_X) */
    EP_WS_START = 16         /* double [n_nodes*dim], the learned start u_ex + s P(y) of the last step that
                                computed one, before the per-problem choice (read only; EP_ERR_STATE before) */
} ep_field;

/* Sizes of a context: n_int, n_comp, nnz_blocks, n_p, n_q. */
typedef struct {
    int64_t n_nodes, n_elem, n_int, nnz_blocks;
    int32_t dim, n_p, n_q, n_comp;
} ep_info;

/* Fill *opts with defaults (FP64, rtol 1e-10, adaptive Krylov, AMG, split on, no profiling). */
void ep_default_opts(ep_opts* opts);

/*
 * Create a context: copy the mesh, material, BCs and loads to the device on
 * `cuda_stream` (a cudaStream_t; NULL = legacy default stream) of `device`,
 * build the block-CSR pattern of K and the element-to-slot map, compute the
 * per-point geometry (Section 6.1: J, det J, J^-1, DPhi, WEIGHT) and assemble
 * K_elast = B^T D_elast B (Section 6.3).  The state starts virgin (u = 0,
 * eps^p = 0, hardening 0).  Errors: EP_ERR_INVALID_ARG for bad sizes/indices,
 * EP_ERR_BAD_ELEMENT if det J <= 0 anywhere, EP_ERR_OOM, EP_ERR_CUDA.  On error
 * *out is NULL.
 */
ep_status ep_create(void** out, const ep_mesh* mesh, const ep_material* mat, const ep_bc* bc,
                    int32_t device, void* cuda_stream);

/*
 * A batch of independent problems in one context (the batched form of the
 * hot path): n_problems meshes of one element type and dimension, with their
 * own materials (one model for all; parameters may differ) and boundary
 * conditions, are concatenated into one mesh (problem p's nodes and elements
 * follow problem p-1's; fields of ep_get / ep_set are concatenated in that
 * order).  Every assembly, Krylov solve and commit covers all problems in the
 * same launches; ep_solve_load_path applies the same load factors to all and
 * a step converges when every problem's own relative residual reaches
 * newton_rtol.  Host arrays are copied; errors as ep_create.
 */
ep_status ep_create_batch(void** out, int32_t n_problems, const ep_mesh* meshes, const ep_material* mats,
                          const ep_bc* bcs, int32_t device, void* cuda_stream);

ep_status ep_destroy(void* ctx);

ep_status ep_get_info(const void* ctx, ep_info* info);

/*
 * Solve load steps k = 1..n_steps with load factors zeta[k] (host array):
 * f_k = zeta_k f_ext_unit, u_{D,k} = zeta_k u_D_unit, ALG-NEWTON (Section 4) to
 * opts->newton_rtol, then commit eps^p_k and the hardening variable (Sections
 * 2.1, 2.2, 2.3).  `reports` is a caller-allocated host array [n_steps] (may be
 * NULL).  Stops at the first failing step and returns its status; earlier
 * steps stay committed.  Continues from the context's current state, so
 * consecutive calls continue one load path.
 */
ep_status ep_solve_load_path(void* ctx, int32_t n_steps, const double* zeta, const ep_opts* opts,
                             ep_step_report* reports);

/*
 * Return the context to the virgin state it had after ep_create (the state
 * before the first load step of a path, Section 4): u = 0, eps^p = 0,
 * hardening variables 0, stresses 0, plastic flags 0, and no load-path
 * history (the next step starts like the first one, without extrapolation).
 * Device memsets on the context's stream, no host transfer and no
 * synchronisation; the mesh, K_elast and the preconditioner's setup are kept.
 */
ep_status ep_reset(void* ctx);

/*
 * Copy a field (ep_field) to `dst` (host, or device when dst_is_device != 0).
 * `bytes` must equal the field's size.  Synchronises the context's stream.
 */
ep_status ep_get(void* ctx, int32_t field, void* dst, size_t bytes, int32_t dst_is_device);

/*
 * Overwrite a state field (EP_U, EP_PLASTIC_STRAIN, EP_HARDENING, EP_STRESS,
 * EP_PLASTIC_FLAG) from `src` (host or device).  Used to resume from a saved
 * state and to evaluate K and F at a given iterate.
 */
ep_status ep_set(void* ctx, int32_t field, const void* src, size_t bytes, int32_t src_is_device);

/*
 * One evaluation of the hot path at displacement u (host or device array
 * [n_nodes*dim]) with the committed state as eps^p_{k-1}: strains (Section
 * 6.2), return mapping (Sections 2.2, 2.3), internal forces F = B^T (W S) and
 * the tangent K (Section 7).  split != 0 uses K = K_elast + B^T (D_t - D_e) B
 * over plastic points only (eq. (K-split)); split == 0 sums B^T D_t B over all
 * points (eq. (K-split_Petr)).  Results stay on the device (EP_F_INT,
 * EP_K_VALUES); *n_plastic (may be NULL) receives the number of plastic points.
 */
ep_status ep_assemble(void* ctx, const double* u, int32_t u_is_device, int32_t split, int64_t* n_plastic);

/*
 * ep_assemble with the tangent's precision chosen (ep_precision): EP_FP64 is
 * ep_assemble; EP_MIXED computes strains, return mapping and F in FP64 as
 * ep_assemble does and forms the tangent in FP32 into EP_K_VALUES_F32 (the
 * split path starts from K_elast rounded to FP32).
 */
ep_status ep_assemble_prec(void* ctx, const double* u, int32_t u_is_device, int32_t split, int32_t precision,
                           int64_t* n_plastic);

/*
 * Commit the state at displacement u (host or device): evaluate the return
 * mapping at every point and store sigma_k, eps^p_k, the hardening variable
 * and the plastic flags (Sections 2.2, 2.3, the T_other updates) as the new
 * committed state; u becomes EP_U.
 */
ep_status ep_commit(void* ctx, const double* u, int32_t u_is_device);

/*
 * Solve K x = b on the free DOFs with the matrix of the last ep_assemble
 * (eq. (lin_syst)); b is a host or device array [n_nodes*dim] (prescribed
 * entries ignored), x is kept as EP_SOLUTION (zero on prescribed DOFs).  Uses
 * opts->krylov, krylov_rtol (must be > 0 here), krylov_maxit, precond and
 * precision: EP_MIXED solves with the FP32 matrix of the last EP_MIXED
 * assembly in FP32 arithmetic (b rounded to FP32, x returned as double).
 * *iterations and *rel_resid (may be NULL) receive the iteration count and
 * the final ||b - K x|| / ||b|| on the free DOFs.
 */
ep_status ep_linear_solve(void* ctx, const double* b, int32_t b_is_device, const ep_opts* opts,
                          int32_t* iterations, double* rel_resid);

/*
 * Stand-alone return mapping on device arrays (Sections 2.2, 2.3): for n
 * points with strains E [n_strain][n] (n_strain = 3 in 2D: e11,e22,2e12;
 * 6 in 3D), previous plastic strain ep_prev [n_comp][n] and hardening
 * hard_prev ([n] or [n_comp][n] for EP_VM_KIN), write the stress S
 * [n_comp][n], the tangent DS [n_strain][n_strain][n] (row = stress, column =
 * strain component), the flag [n], and the trial state ep_new, hard_new
 * (same shapes as the inputs).  Runs on `cuda_stream`; does not synchronise.
 * EP_ERR_RETURN_MAP is reported only through flag value 255 at failing points.
 */
ep_status ep_constitutive(const ep_material* mat, int32_t dim, int64_t n, const double* E,
                          const double* ep_prev, const double* hard_prev, double* S, double* DS,
                          uint8_t* flag, double* ep_new, double* hard_new, void* cuda_stream);

/*
 * Workspace-free variant of ep_linear_solve, for callers that cannot allocate
 * device memory: code that runs while another runtime owns the device's
 * memory pool, or a phase in which no cudaMalloc may be issued.  The paper
 * has no counterpart: this is an interface for such callers, not a step of
 * the method.  The caller passes every array (device pointers): the
 * block-CSR matrix of K (node blocks dim x dim, row-major blocks, as returned
 * by EP_K_ROW_PTR / EP_K_COL_IDX / EP_K_VALUES), diag_slot [n_nodes] (index
 * of each row's diagonal block), the free-DOF mask, b and the output x
 * [n_nodes*dim] (zero on prescribed DOFs on return).  method: 1 CG, 2
 * BiCGStab; precond: 0 Jacobi, 1 block Jacobi.  The solver's own buffers live
 * in one fixed device array inside the library (about 3.7 MB), held by every
 * GPU that loads the library until the process exits; it limits the system
 * to EP_NOALLOC_MAX_DOF DOFs and maxit to EP_NOALLOC_MAX_ITERATIONS, and
 * larger requests fail with EP_ERR_INVALID_ARG (message in
 * ep_last_error(NULL)).  The first call on a device looks up that array's
 * device address (with the device current), so make it before any stream
 * capture.  All calls share the array: calls that overlap on the GPU race.
 * Issues no cudaMalloc/cudaFree and no allocating library call; runs on
 * cuda_stream and returns after synchronising it.
 */
#define EP_NOALLOC_MAX_DOF 32768
#define EP_NOALLOC_MAX_ITERATIONS 10000
ep_status ep_linear_solve_noalloc(int32_t dim, int64_t n_nodes, const int32_t* row_ptr, const int32_t* col_idx,
                                  const int32_t* diag_slot, const double* vals, const uint8_t* free_dof,
                                  const double* b, double* x, int32_t method, int32_t precond, double rtol,
                                  int32_t maxit, int32_t* iterations, double* rel_resid, void* cuda_stream);

/*
 * Learned warm start (a per-node network that corrects the extrapolated
 * Newton start).  The paper starts Newton at step k from the prescribed
 * values u_{D,k} (ALG-NEWTON, Section 4); warm_start = 1 extrapolates the
 * last two converged steps, u_ex = u_{k-1} + r_k (u_{k-1} - u_{k-2}) with
 * r_k = (zeta_k - zeta_{k-1}) / (zeta_{k-1} - zeta_{k-2}).  warm_start = 2
 * adds s * P(y) on free DOFs, where s is the problem's RMS of
 * u_{k-1} - u_{k-2}, y [node][0..dim) the output of a network
 *     16 -> 128 (ReLU) -> 128 (ReLU) -> 4,
 * (weights rounded to bfloat16; biases, activations and sums in FP32), and P
 * the least-squares projection of y, per problem and displacement component,
 * onto the span of the scaled last two increments over the free DOFs (FP64
 * normal equations; the last increment alone when they are singular).  The 16
 * inputs of a node: u_{k-1} - u_{k-2} and u_{k-2} - u_{k-3} divided by s (3
 * each, zero-padded in 2D), r_k, r_{k-1}, the fraction of plastic points of
 * the adjacent elements after step k-1 and its change since step k-2, the
 * largest yield proximity of those points after step k-1 (von Mises
 * |dev s - beta| / (Y + H alpha), Drucker-Prager (|dev s|/sqrt(2) + eta p) /
 * (c + Hc alpha), clamped at 0), then nu, yield strain x 1e3 (Y/E; c0/E for
 * Drucker-Prager), hardening ratio x 10 (H/E; Hc/E), 1 for Drucker-Prager, the
 * fraction of the node's prescribed components.  Output 3 is a logit of the
 * node's plastic fraction after step k (trained, reported, not used by the
 * start).  The learned start
 * needs three converged steps since ep_ws_attach / ep_ws_record and a load
 * that keeps its direction; each problem of a batch keeps the plain
 * extrapolation when that has the smaller residual (the network is not run
 * when the extrapolated start already meets the Newton tolerance), and a step
 * that fails to converge from either is retried from the last converged u.
 *
 * Parameters: one float32 vector of EP_WS_N_PARAMS entries, W1 [128][16],
 * b1 [128], W2 [128][128], b2 [128], W3 [4][128], b3 [4] (y = W x + b).
 * Training loss over n rows (targets t [n][4]):
 *     (1/n) sum [ sum_{c<3} (y_c - t_c)^2 + 0.1 * (max(y_3,0) - y_3 t_3 + log(1 + exp(-|y_3|))) ];
 * Adam (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) on FP32 master
 * parameters, the bfloat16 copy refreshed after every step.
 *
 * Errors: EP_ERR_INVALID_ARG for a null handle or array, n_rows < 0 (forward;
 * 0 is an empty call) or <= 0 (grad, train), lr <= 0, and warm_start = 2
 * without an attached network; EP_ERR_OOM / EP_ERR_CUDA for device failures
 * (ep_mlp_create's message in ep_last_error(NULL)).  The network's buffers
 * (parameters, Adam moments, per-CTA gradient partials) are owned by its
 * handle; the context's recording buffers by the context.
 */
#define EP_WS_N_IN 16
#define EP_WS_WIDTH 128
#define EP_WS_N_OUT 4
#define EP_WS_N_PARAMS 19204
/* A network on `device`, parameters copied from host `params`; kernels run on cuda_stream.
 * Several contexts may read one network at once (forward passes); training it while a context
 * solves with it is the caller's race to avoid (a context waits for the network's stream before
 * each forward pass, so a training step enqueued earlier is complete by then). */
ep_status ep_mlp_create(void** out, const float* params, int32_t device, void* cuda_stream);
ep_status ep_mlp_destroy(void* mlp);
/* Current FP32 master parameters into host dst [EP_WS_N_PARAMS]. */
ep_status ep_mlp_get_params(void* mlp, float* dst);
/* Y [n][4] = network(X [n][16]); device pointers; returns when the outputs are written. */
ep_status ep_mlp_forward(void* mlp, const float* X, int64_t n_rows, float* Y);
/* Loss and its gradient (host loss, host grad [EP_WS_N_PARAMS]) over n rows of device X, T; no update. */
ep_status ep_mlp_grad(void* mlp, const float* X, const float* T, int64_t n_rows, double* loss, float* grad);
/* One Adam step with learning rate lr on the n rows of device X [n][16], T [n][4]; *loss (host, may
 * be NULL) receives the loss before the step. */
ep_status ep_mlp_train_step(void* mlp, const float* X, const float* T, int64_t n_rows, float lr, double* loss);
/* Record training rows during ep_solve_load_path: after every converged step with features (three
 * earlier converged steps, a load keeping its direction), n_nodes rows of inputs and targets
 * (t_c = (u_k - u_ex)_c / s on free DOFs, 0 on prescribed ones; t_3 the node's plastic fraction after
 * step k) are appended while max_rows allows.  max_rows = 0 frees the buffers.  Starts the history
 * the features need (as does ep_ws_attach). */
ep_status ep_ws_record(void* ctx, int64_t max_rows);
/* The recorded rows: device pointers X [n][16], T [n][4] owned by the context, valid until the next
 * ep_ws_record or ep_destroy. */
ep_status ep_ws_samples(void* ctx, const float** X, const float** T, int64_t* n_rows);
/* Use `mlp` (not owned; NULL detaches) for warm_start = 2. */
ep_status ep_ws_attach(void* ctx, void* mlp);

/* Human-readable name of a status code. */
const char* ep_status_str(int32_t status);
/* Message of the last failure of `ctx`; with ctx == NULL, the message of the
 * last failed ep_create, ep_create_batch, ep_mlp_create or ep_linear_solve_noalloc
 * on the calling thread. */
const char* ep_last_error(const void* ctx);

#ifdef __cplusplus
}
#endif

#endif /* EP_H */
