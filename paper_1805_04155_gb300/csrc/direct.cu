// Numeric phase of the sparse direct solver (see direct.h): multifrontal LU with static pivoting in
// FP64 or FP32 fronts, processed level by level over the elimination tree (every front of a level in
// one launch), and the forward / backward solves that mirror it.
//
// Front s is a dense m x m row-major matrix (m = (pivots + update nodes) * dim) whose first k rows
// and columns are its pivots.  Its partial factorisation runs in panels of 32 pivots: the 32 x 32
// diagonal block is factored in shared memory by one warp, the panel's column below it becomes
// L21 = A21 U11^-1 and its row to the right U12 = L11^-1 A12, and the trailing matrix takes the
// rank-32 update A22 -= L21 U12.  After the k pivots the trailing (m - k)^2 block is the Schur
// complement, added into the parent front (extend-add, one launch per child rank so that no two
// launches of a level write one parent entry at once: no atomics, the same result every run).
#include <algorithm>
#include <cfloat>

#include "direct.h"

namespace ep {

namespace {

constexpr int DNB = 32;     // pivots per panel
constexpr int PANEL_THREADS = 64;    // threads per CTA of the panel solves
// threads per front in the solves of a level: enough for the rows of its largest front (a thread per
// row of a block update), 64 .. 512
inline int solve_threads(int mmax) { return std::max(64, std::min(512, ((mmax + 63) / 64) * 64)); }

// static pivoting: a pivot below this times max |a_ii| in magnitude is replaced by +- that value
template <class TF> __device__ __forceinline__ TF pivot_tiny();
template <> __device__ __forceinline__ float pivot_tiny<float>() { return 1e-6f; }
template <> __device__ __forceinline__ double pivot_tiny<double>() { return 1e-10; }
template <class TF> __device__ __forceinline__ TF tiny_floor();
template <> __device__ __forceinline__ float tiny_floor<float>() { return FLT_MIN; }
template <> __device__ __forceinline__ double tiny_floor<double>() { return DBL_MIN; }

template <class TF>
struct FrontArgs {
    TF* F;
    const int64_t* f_off;
    const int32_t* npiv;
    const int32_t* nupd;
    const int64_t* node_off;
    const int32_t* nodes;
    const int32_t* umap;
    const int32_t* parent;
    const int32_t* child_rank;
    const int32_t* child_ptr;
    const int32_t* children;
    const int64_t* v_off;
    int dim;
};

// Blocks into the fronts (Dirichlet rows and columns: identity); the largest |a_ii| on free DOFs
// into anorm (non-negative floats order like their bit patterns)
template <class T, class TF>
__global__ void __launch_bounds__(256) k_df_scatter(FrontArgs<TF> a, const T* __restrict__ vals, int64_t nnzb,
                                                    const int32_t* __restrict__ blk_front,
                                                    const int32_t* __restrict__ blk_row,
                                                    const int32_t* __restrict__ blk_col,
                                                    const uint8_t* __restrict__ free_dof, float* anorm) {
    const int dim = a.dim, d2 = dim * dim;
    float amax = 0.f;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nnzb * d2; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = t / d2;
        const int e = (int)(t - b * d2), r = e / dim, c = e - r * dim;
        const int s = blk_front[b], lr = blk_row[b], lc = blk_col[b];
        const int64_t m = (int64_t)(a.npiv[s] + a.nupd[s]) * dim;
        const int64_t di = (int64_t)a.nodes[a.node_off[s] + lr] * dim + r;
        const int64_t dj = (int64_t)a.nodes[a.node_off[s] + lc] * dim + c;
        TF v;
        if (free_dof[di] && free_dof[dj]) {
            v = (TF)vals[t];
            if (di == dj) amax = fmaxf(amax, fabsf((float)v));
        } else {
            v = di == dj ? TF(1) : TF(0);
        }
        a.F[a.f_off[s] + (int64_t)(lr * dim + r) * m + lc * dim + c] = v;
    }
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if ((threadIdx.x & 31) == 0 && amax > 0.f) atomicMax(reinterpret_cast<unsigned int*>(anorm), __float_as_uint(amax));
}

template <class TF>
__device__ __forceinline__ bool front_dims(const FrontArgs<TF>& a, int s, int p0, int& k, int& m, int& nb) {
    k = a.npiv[s] * a.dim;
    if (p0 >= k) return false;
    m = (a.npiv[s] + a.nupd[s]) * a.dim;
    nb = min(DNB, k - p0);
    return true;
}

// LU without row exchanges of the nb x nb diagonal block at (p0, p0) of every front of the level
// that still has pivots there; one warp per front, the block in shared memory, lane j updating
// column j.  (Holding the columns in registers and broadcasting the multipliers by shuffles was
// slower: 70 against 51 us per launch at the top front, FP64.)
template <class TF>
__global__ void __launch_bounds__(32) k_df_diag(FrontArgs<TF> a, int s0, int p0, const float* anorm,
                                                unsigned int* n_perturbed) {
    const int s = s0 + blockIdx.x;
    int k, m, nb;
    if (!front_dims(a, s, p0, k, m, nb)) return;
    __shared__ TF A[DNB][DNB + 1];
    TF* Fs = a.F + a.f_off[s];
    const int lane = threadIdx.x;
    for (int i = 0; i < nb; ++i)
        if (lane < nb) A[i][lane] = Fs[(int64_t)(p0 + i) * m + p0 + lane];
    __syncwarp();
    const TF tiny = max(pivot_tiny<TF>() * (TF)*anorm, tiny_floor<TF>());
    unsigned int pert = 0;
    for (int t = 0; t < nb; ++t) {
        TF d = A[t][t];
        if (fabs(d) < tiny) {
            d = d < TF(0) ? -tiny : tiny;
            ++pert;
        }
        __syncwarp();
        if (lane == t) A[t][t] = d;
        if (lane > t && lane < nb) A[lane][t] = A[lane][t] / d;
        __syncwarp();
        if (lane > t && lane < nb) {
            const TF u = A[t][lane];
            for (int i = t + 1; i < nb; ++i) A[i][lane] -= A[i][t] * u;
        }
        __syncwarp();
    }
    for (int i = 0; i < nb; ++i)
        if (lane < nb) Fs[(int64_t)(p0 + i) * m + p0 + lane] = A[i][lane];
    if (lane == 0 && pert) atomicAdd(n_perturbed, pert);
}

// L21 = A21 U11^-1 (one row below the block per work item) and U12 = L11^-1 A12 (one column right
// of it per item); each thread solves its item's 32 values in place in its own column of shared
// memory (xs[j][thread]: no bank conflicts, no register arrays)
template <class TF>
__global__ void __launch_bounds__(64) k_df_panel(FrontArgs<TF> a, int s0, int p0) {
    const int s = s0 + blockIdx.y;
    int k, m, nb;
    if (!front_dims(a, s, p0, k, m, nb)) return;
    __shared__ TF D[DNB][DNB + 1];
    __shared__ TF dinv[DNB];
    extern __shared__ __align__(16) unsigned char sh_raw[];
    TF* xs = reinterpret_cast<TF*>(sh_raw);   // [DNB][blockDim.x]
    const int nt = blockDim.x, tid = threadIdx.x;
    TF* Fs = a.F + a.f_off[s];
    for (int e = tid; e < DNB * DNB; e += nt) {
        const int i = e / DNB, j = e % DNB;
        D[i][j] = (i < nb && j < nb) ? Fs[(int64_t)(p0 + i) * m + p0 + j] : TF(0);
    }
    __syncthreads();
    if (tid < DNB) dinv[tid] = tid < nb ? TF(1) / D[tid][tid] : TF(0);
    __syncthreads();
    const int q0 = p0 + nb, rest = m - q0;
    for (int item = blockIdx.x * nt + tid; item < 2 * rest; item += gridDim.x * nt) {
        const bool is_row = item < rest;
        // a row of A21 (stride 1) or a column of A12 (stride m)
        TF* v = is_row ? Fs + (int64_t)(q0 + item) * m + p0 : Fs + (int64_t)p0 * m + q0 + (item - rest);
        const int64_t st = is_row ? 1 : m;
        for (int j = 0; j < nb; ++j) xs[j * nt + tid] = v[j * st];
        if (is_row) {
            // x U11 = a: forward in j
            for (int j = 0; j < nb; ++j) {
                TF t = xs[j * nt + tid];
                for (int q = 0; q < j; ++q) t -= xs[q * nt + tid] * D[q][j];
                xs[j * nt + tid] = t * dinv[j];
            }
        } else {
            // L11 y = a, unit lower: forward in j
            for (int j = 0; j < nb; ++j) {
                TF t = xs[j * nt + tid];
                for (int q = 0; q < j; ++q) t -= D[j][q] * xs[q * nt + tid];
                xs[j * nt + tid] = t;
            }
        }
        for (int j = 0; j < nb; ++j) v[j * st] = xs[j * nt + tid];
    }
}

// A22 -= L21 U12 on the trailing part of every front of the level; DT x DT tile per CTA of 256
// threads, R x R entries per thread (DT = 16 R: 64 for large fronts, 32 for levels of small ones)
template <class TF, int R>
__global__ void __launch_bounds__(256) k_df_update(FrontArgs<TF> a, int s0, int p0, int tiles) {
    constexpr int DT = 16 * R;
    const int s = s0 + blockIdx.y;
    int k, m, nb;
    if (!front_dims(a, s, p0, k, m, nb)) return;
    const int q0 = p0 + nb;
    const int i0 = q0 + (int)(blockIdx.x / tiles) * DT, j0 = q0 + (int)(blockIdx.x % tiles) * DT;
    if (i0 >= m || j0 >= m) return;
    __shared__ __align__(16) TF Ls[DNB][DT + 4];   // Ls[t][i] = L21[i0 + i][t]
    __shared__ __align__(16) TF Us[DNB][DT + 4];   // Us[t][j] = U12[t][j0 + j]
    TF* Fs = a.F + a.f_off[s];
    for (int e = threadIdx.x; e < DT * DNB; e += blockDim.x) {
        const int i = e / DNB, t = e % DNB;
        Ls[t][i] = (i0 + i < m && t < nb) ? Fs[(int64_t)(i0 + i) * m + p0 + t] : TF(0);
    }
    for (int e = threadIdx.x; e < DT * DNB; e += blockDim.x) {
        const int t = e / DT, j = e % DT;
        Us[t][j] = (j0 + j < m && t < nb) ? Fs[(int64_t)(p0 + t) * m + j0 + j] : TF(0);
    }
    __syncthreads();
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    TF acc[R][R];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < R; ++c) acc[r][c] = TF(0);
#pragma unroll 8
    for (int t = 0; t < DNB; ++t) {
        TF lv[R], uv[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            lv[r] = Ls[t][ty * R + r];
            uv[r] = Us[t][tx * R + r];
        }
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int c = 0; c < R; ++c) acc[r][c] = fma(lv[r], uv[c], acc[r][c]);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = i0 + ty * R + r;
        if (i >= m) continue;
        TF* row = Fs + (int64_t)i * m;
#pragma unroll
        for (int c = 0; c < R; ++c) {
            const int j = j0 + tx * R + c;
            if (j < m) row[j] -= acc[r][c];
        }
    }
}

// Schur complements of the level's fronts of child rank `rank` into their parents
template <class TF>
__global__ void __launch_bounds__(256) k_df_extend(FrontArgs<TF> a, int s0, int rank) {
    const int s = s0 + blockIdx.y;
    const int p = a.parent[s];
    if (p < 0 || a.child_rank[s] != rank) return;
    const int dim = a.dim;
    const int k = a.npiv[s] * dim, u = a.nupd[s] * dim, m = k + u;
    const int64_t mp = (int64_t)(a.npiv[p] + a.nupd[p]) * dim;
    const TF* Fs = a.F + a.f_off[s];
    TF* Fp = a.F + a.f_off[p];
    const int32_t* um = a.umap + a.node_off[s] + a.npiv[s];
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)u * u;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int ia = (int)(t / u), ib = (int)(t - (int64_t)ia * u);
        const int64_t pa = (int64_t)um[ia / dim] * dim + ia % dim, pb = (int64_t)um[ib / dim] * dim + ib % dim;
        Fp[pa * mp + pb] += Fs[(int64_t)(k + ia) * m + k + ib];
    }
}

// Forward solve of one level: per front, w = (b at the pivots, 0) plus the children's update
// vectors; L11 y = w_E (unit lower, by 32-row blocks); the update vector w_U - L21 y goes to the
// parent, y to Y.
template <class TV, class TF>
__global__ void __launch_bounds__(512) k_ds_fwd(FrontArgs<TF> a, int s0, const TV* __restrict__ b,
                                                const uint8_t* __restrict__ free_dof, TF* __restrict__ Y,
                                                TF* __restrict__ vupd, const KrylovRec* rec) {
    if (rec && rec->done) return;
    extern __shared__ __align__(16) unsigned char sh_raw[];
    TF (*T)[DNB + 1] = reinterpret_cast<TF (*)[DNB + 1]>(sh_raw);
    TF* w = reinterpret_cast<TF*>(sh_raw) + DNB * (DNB + 1);
    const int s = s0 + blockIdx.x, dim = a.dim;
    const int k = a.npiv[s] * dim, m = (a.npiv[s] + a.nupd[s]) * dim;
    const int32_t* nd = a.nodes + a.node_off[s];
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        TF v = TF(0);
        if (i < k) {
            const int64_t g = (int64_t)nd[i / dim] * dim + i % dim;
            v = free_dof[g] ? (TF)b[g] : TF(0);
        }
        w[i] = v;
    }
    __syncthreads();
    for (int ci = a.child_ptr[s]; ci < a.child_ptr[s + 1]; ++ci) {
        const int c = a.children[ci];
        const int uc = a.nupd[c] * dim;
        const int32_t* um = a.umap + a.node_off[c] + a.npiv[c];
        const TF* vc = vupd + a.v_off[c];
        for (int i = threadIdx.x; i < uc; i += blockDim.x) w[um[i / dim] * dim + i % dim] += vc[i];
        __syncthreads();
    }
    const TF* Fs = a.F + a.f_off[s];
    for (int blk = 0; blk < k; blk += DNB) {
        const int nbk = min(DNB, k - blk);
        for (int e = threadIdx.x; e < DNB * DNB; e += blockDim.x) {
            const int i = e / DNB, j = e % DNB;
            T[i][j] = (i < nbk && j < nbk) ? Fs[(int64_t)(blk + i) * m + blk + j] : TF(0);
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            TF val = lane < nbk ? w[blk + lane] : TF(0);
            for (int t = 0; t < nbk; ++t) {
                const TF yt = __shfl_sync(0xffffffffu, val, t);
                if (lane > t) val -= T[lane][t] * yt;
            }
            if (lane < nbk) w[blk + lane] = val;
        }
        __syncthreads();
        // rows below the block: w_i -= L[i, blk..] y_blk, a thread per row (its 32 loads in flight
        // together; a warp per row would walk the rows one after another)
        for (int i = blk + nbk + threadIdx.x; i < m; i += blockDim.x) {
            const TF* row = Fs + (int64_t)i * m + blk;
            TF acc = TF(0);
            for (int t = 0; t < nbk; ++t) acc = fma(row[t], w[blk + t], acc);
            w[i] -= acc;
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        if (i < k) Y[(int64_t)nd[i / dim] * dim + i % dim] = w[i];
        else vupd[a.v_off[s] + (i - k)] = w[i];
    }
}

// Backward solve of one level: per front, t = y_E - U12 x_U (x_U: the ancestors' solution, already
// in x), then U11 x_E = t by 32-row blocks from the last; x_E into x (0 on fixed DOFs).
template <class TV, class TF>
__global__ void __launch_bounds__(512) k_ds_bwd(FrontArgs<TF> a, int s0, TV* __restrict__ x,
                                                const uint8_t* __restrict__ free_dof, const TF* __restrict__ Y,
                                                const KrylovRec* rec) {
    if (rec && rec->done) return;
    extern __shared__ __align__(16) unsigned char sh_raw[];
    TF (*T)[DNB + 1] = reinterpret_cast<TF (*)[DNB + 1]>(sh_raw);
    TF* t = reinterpret_cast<TF*>(sh_raw) + DNB * (DNB + 1);
    const int s = s0 + blockIdx.x, dim = a.dim;
    const int k = a.npiv[s] * dim, m = (a.npiv[s] + a.nupd[s]) * dim, u = m - k;
    TF* xu = t + k;
    const int32_t* nd = a.nodes + a.node_off[s];
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const int64_t g = (int64_t)nd[i / dim] * dim + i % dim;
        t[i] = i < k ? Y[g] : (TF)x[g];
    }
    __syncthreads();
    const TF* Fs = a.F + a.f_off[s];
    if (u > 0) {
        // t -= U12 x_U: a warp per row, its lanes reading consecutive entries
        const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
        for (int i = threadIdx.x >> 5; i < k; i += nw) {
            const TF* row = Fs + (int64_t)i * m + k;
            TF acc = TF(0);
            for (int j = lane; j < u; j += 32) acc = fma(row[j], xu[j], acc);
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) t[i] -= acc;
        }
    }
    __syncthreads();
    for (int blk = ((k - 1) / DNB) * DNB; blk >= 0 && k > 0; blk -= DNB) {
        const int nbk = min(DNB, k - blk);
        for (int e = threadIdx.x; e < DNB * DNB; e += blockDim.x) {
            const int i = e / DNB, j = e % DNB;
            T[i][j] = (i < nbk && j < nbk) ? Fs[(int64_t)(blk + i) * m + blk + j] : (i == j ? TF(1) : TF(0));
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            TF val = lane < nbk ? t[blk + lane] : TF(0);
            const TF dl = TF(1) / T[lane][lane];
            for (int q = nbk - 1; q >= 0; --q) {
                const TF xq = __shfl_sync(0xffffffffu, val * dl, q);
                if (lane == q) val = xq;
                else if (lane < q) val -= T[lane][q] * xq;
            }
            if (lane < nbk) t[blk + lane] = val;
        }
        __syncthreads();
        // rows above the block: t_i -= U[i, blk..] x_blk, a thread per row
        for (int i = threadIdx.x; i < blk; i += blockDim.x) {
            const TF* row = Fs + (int64_t)i * m + blk;
            TF acc = TF(0);
            for (int q = 0; q < nbk; ++q) acc = fma(row[q], t[blk + q], acc);
            t[i] -= acc;
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        const int64_t g = (int64_t)nd[i / dim] * dim + i % dim;
        x[g] = free_dof[g] ? (TV)t[i] : TV(0);
    }
}

template <class TF>
FrontArgs<TF> front_args(DirectDev& D) {
    FrontArgs<TF> a;
    a.F = static_cast<TF*>(D.F);
    a.f_off = D.f_off;
    a.npiv = D.npiv;
    a.nupd = D.nupd;
    a.node_off = D.node_off;
    a.nodes = D.nodes;
    a.umap = D.umap;
    a.parent = D.parent;
    a.child_rank = D.child_rank;
    a.child_ptr = D.child_ptr;
    a.children = D.children;
    a.v_off = D.v_off;
    a.dim = D.plan.dim;
    return a;
}

// shared memory of the solve kernels for fronts of order m
template <class TF>
size_t solve_smem(int m) { return sizeof(TF) * ((size_t)DNB * (DNB + 1) + (size_t)m); }

constexpr int MAX_GRID_Y = 65535;

// profile = 1: event before the work
cudaError_t prof_begin(DirectDev& D, cudaStream_t s) {
    if (!D.profile) return cudaSuccess;
    for (auto& ev : D.ev)
        if (!ev) {
            cudaError_t e = cudaEventCreate(&ev);
            if (e != cudaSuccess) return e;
        }
    return cudaEventRecord(D.ev[0], s);
}

// profile = 1: event after the work, waited for; its duration added to *ms
cudaError_t prof_end(DirectDev& D, cudaStream_t s, double* ms) {
    if (!D.profile) return cudaSuccess;
    cudaError_t e = cudaEventRecord(D.ev[1], s);
    if (e == cudaSuccess) e = cudaEventSynchronize(D.ev[1]);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, D.ev[0], D.ev[1]);
    if (e == cudaSuccess) *ms += t;
    return e;
}

template <class T, class TF>
cudaError_t factor_t(DirectDev& D, const BsrT<T>& A, cudaStream_t s) {
    const DirectPlan& P = D.plan;
    cudaError_t e = prof_begin(D, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(D.F, 0, sizeof(TF) * (size_t)P.factor_vals(), s);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(D.anorm, 0, sizeof(float), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(D.n_perturbed, 0, sizeof(unsigned int), s)) != cudaSuccess) return e;
    const FrontArgs<TF> a = front_args<TF>(D);
    {
        const int64_t work = P.nnzb * P.dim * P.dim;
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, 4096));
        k_df_scatter<T, TF><<<grid, 256, 0, s>>>(a, A.vals, P.nnzb, D.blk_front, D.blk_row, D.blk_col, A.free_dof,
                                                 D.anorm);
        D.launches += 1;
    }
    const int nl = (int)P.level_ptr.size() - 1;
    for (int l = 0; l < nl; ++l) {
        const int kmax = P.lvl_kmax[l], mmax = P.lvl_mmax[l];
        for (int c0 = P.level_ptr[l]; c0 < P.level_ptr[l + 1]; c0 += MAX_GRID_Y) {
            const int nf = std::min(MAX_GRID_Y, P.level_ptr[l + 1] - c0);
            for (int p0 = 0; p0 < kmax; p0 += DNB) {
                k_df_diag<TF><<<nf, 32, 0, s>>>(a, c0, p0, D.anorm, D.n_perturbed);
                const int rest = mmax - p0 - 1;   // the largest trailing order of the level (at least)
                if (rest > 0) {
                    // 64 threads per CTA: the top levels' few fronts spread their panel over more SMs
                    const int gx = std::max(1, std::min((2 * rest + PANEL_THREADS - 1) / PANEL_THREADS, 256));
                    k_df_panel<TF><<<dim3(gx, nf), PANEL_THREADS, sizeof(TF) * DNB * PANEL_THREADS, s>>>(a, c0, p0);
                    if (mmax <= 160) {   // small fronts: 32 x 32 tiles (less of a tile outside the front)
                        const int tiles = (rest + 31) / 32;
                        k_df_update<TF, 2><<<dim3(tiles * tiles, nf), 256, 0, s>>>(a, c0, p0, tiles);
                    } else {
                        const int tiles = (rest + 63) / 64;
                        k_df_update<TF, 4><<<dim3(tiles * tiles, nf), 256, 0, s>>>(a, c0, p0, tiles);
                    }
                    D.launches += 2;
                }
                D.launches += 1;
            }
        }
        if (l + 1 < nl) {
            // extend-add into the next level, one child rank at a time
            const int ranks = P.lvl_maxkids[l + 1];
            const int64_t umax = P.lvl_umax[l];
            const int gx = (int)std::max<int64_t>(1, std::min<int64_t>((umax * umax + 255) / 256, 1024));
            for (int r = 0; r < ranks; ++r)
                for (int c0 = P.level_ptr[l]; c0 < P.level_ptr[l + 1]; c0 += MAX_GRID_Y) {
                    const int nf = std::min(MAX_GRID_Y, P.level_ptr[l + 1] - c0);
                    k_df_extend<TF><<<dim3(gx, nf), 256, 0, s>>>(a, c0, r);
                    D.launches += 1;
                }
        }
    }
    D.n_factor += 1;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return prof_end(D, s, &D.factor_ms);
}

template <class TV, class TF>
cudaError_t solve_t(DirectDev& D, const TV* b, TV* x, const uint8_t* free_dof, const KrylovRec* rec, cudaStream_t s) {
    const DirectPlan& P = D.plan;
    const FrontArgs<TF> a = front_args<TF>(D);
    TF* Y = static_cast<TF*>(D.y);
    TF* vupd = static_cast<TF*>(D.vupd);
    const int nl = (int)P.level_ptr.size() - 1;
    cudaError_t e = prof_begin(D, s);
    if (e != cudaSuccess) return e;
    for (int l = 0; l < nl; ++l)
        for (int c0 = P.level_ptr[l]; c0 < P.level_ptr[l + 1]; c0 += MAX_GRID_Y) {
            const int nf = std::min(MAX_GRID_Y, P.level_ptr[l + 1] - c0);
            k_ds_fwd<TV, TF><<<nf, solve_threads(P.lvl_mmax[l]), solve_smem<TF>(P.lvl_mmax[l]), s>>>(a, c0, b, free_dof, Y,
                                                                                                      vupd, rec);
            D.launches += 1;
        }
    for (int l = nl - 1; l >= 0; --l)
        for (int c0 = P.level_ptr[l]; c0 < P.level_ptr[l + 1]; c0 += MAX_GRID_Y) {
            const int nf = std::min(MAX_GRID_Y, P.level_ptr[l + 1] - c0);
            k_ds_bwd<TV, TF><<<nf, solve_threads(P.lvl_mmax[l]), solve_smem<TF>(P.lvl_mmax[l]), s>>>(a, c0, x, free_dof, Y,
                                                                                                      rec);
            D.launches += 1;
        }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return prof_end(D, s, &D.solve_ms);
}

template <class T>
cudaError_t upload(DirectDev& D, T** dst, const std::vector<T>& src) {
    const size_t n = std::max<size_t>(1, src.size());
    cudaError_t e = cudaMalloc((void**)dst, n * sizeof(T));
    if (e != cudaSuccess) return e;
    D.allocs.push_back((void*)*dst);
    D.bytes += (int64_t)(n * sizeof(T));
    if (!src.empty()) e = cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
    return e;
}

cudaError_t alloc_bytes(DirectDev& D, void** dst, size_t bytes) {
    bytes = std::max<size_t>(16, bytes);
    cudaError_t e = cudaMalloc(dst, bytes);
    if (e != cudaSuccess) return e;
    D.allocs.push_back(*dst);
    D.bytes += (int64_t)bytes;
    return cudaSuccess;
}

template <class TF>
cudaError_t set_smem(int smem) {
    cudaError_t e = cudaFuncSetAttribute(k_df_panel<TF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(sizeof(TF) * DNB * PANEL_THREADS));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_ds_fwd<double, TF>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_ds_fwd<float, TF>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_ds_bwd<double, TF>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_ds_bwd<float, TF>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    return e;
}

}  // namespace

// largest front order the solve kernels take (their working vector lives in shared memory)
constexpr int DIRECT_MAX_FRONT_64 = 24000, DIRECT_MAX_FRONT_32 = 48000;

bool direct_setup(DirectDev& D, int64_t max_bytes) {
    const DirectPlan& P = D.plan;
    const size_t vb = D.fp64 ? sizeof(double) : sizeof(float);
    int mmax = 0;
    for (int v : P.lvl_mmax) mmax = std::max(mmax, v);
    const int max_front = D.fp64 ? DIRECT_MAX_FRONT_64 : DIRECT_MAX_FRONT_32;
    const int64_t need = (int64_t)vb * (P.factor_vals() + P.v_off.back() + P.n_nodes * P.dim) +
                         (int64_t)sizeof(int32_t) * (3 * P.nnzb + 2 * (int64_t)P.nodes.size() + 8 * (int64_t)P.n_fronts);
    if (mmax > max_front) {
        D.refused = true;
        D.why = "direct solver: largest front of order " + std::to_string(mmax) + " exceeds " +
                std::to_string(max_front);
        return false;
    }
    if (need > max_bytes) {
        D.refused = true;
        D.why = "direct solver: the factors need " + std::to_string(need >> 20) + " MiB, more than the " +
                std::to_string(max_bytes >> 20) + " MiB allowed";
        return false;
    }
    cudaError_t e = cudaSuccess;
    auto ok = [&](cudaError_t r) { if (e == cudaSuccess) e = r; return e == cudaSuccess; };
    ok(upload(D, &D.blk_front, P.blk_front));
    ok(upload(D, &D.blk_row, P.blk_row));
    ok(upload(D, &D.blk_col, P.blk_col));
    ok(upload(D, &D.nodes, P.nodes));
    ok(upload(D, &D.umap, P.umap));
    ok(upload(D, &D.npiv, P.npiv));
    ok(upload(D, &D.nupd, P.nupd));
    ok(upload(D, &D.child_ptr, P.child_ptr));
    ok(upload(D, &D.children, P.children));
    ok(upload(D, &D.parent, P.parent));
    ok(upload(D, &D.child_rank, P.child_rank));
    ok(upload(D, &D.node_off, P.node_off));
    ok(upload(D, &D.f_off, P.f_off));
    ok(upload(D, &D.v_off, P.v_off));
    ok(alloc_bytes(D, &D.F, vb * (size_t)P.factor_vals()));
    ok(alloc_bytes(D, &D.vupd, vb * (size_t)P.v_off.back()));
    ok(alloc_bytes(D, &D.y, vb * (size_t)(P.n_nodes * P.dim)));
    ok(alloc_bytes(D, (void**)&D.anorm, sizeof(float)));
    ok(alloc_bytes(D, (void**)&D.n_perturbed, sizeof(unsigned int)));
    ok(D.fp64 ? set_smem<double>((int)solve_smem<double>(mmax)) : set_smem<float>((int)solve_smem<float>(mmax)));
    if (e != cudaSuccess) {
        D.refused = true;
        D.why = std::string("direct solver setup: ") + cudaGetErrorString(e);
        direct_free(D);
        cudaGetLastError();
        return false;
    }
    // a solve reads every front's pivot rows and columns (L11, U11, L21, U12), not its Schur block
    D.solve_bytes = 0.0;
    for (int f = 0; f < P.n_fronts; ++f) {
        const double m = (double)(P.npiv[f] + P.nupd[f]) * P.dim, u = (double)P.nupd[f] * P.dim;
        D.solve_bytes += (double)vb * (m * m - u * u);
    }
    D.ready = true;
    return true;
}

void direct_free(DirectDev& D) {
    for (auto& ev : D.ev)
        if (ev) {
            cudaEventDestroy(ev);
            ev = nullptr;
        }
    for (void* p : D.allocs) cudaFree(p);
    D.allocs.clear();
    D.ready = false;
    D.bytes = 0;
}

cudaError_t direct_factor(DirectDev& D, const BsrT<double>& A, cudaStream_t s) {
    if (!D.ready) return cudaErrorInvalidValue;
    return D.fp64 ? factor_t<double, double>(D, A, s) : factor_t<double, float>(D, A, s);
}
cudaError_t direct_factor(DirectDev& D, const BsrT<float>& A, cudaStream_t s) {
    if (!D.ready) return cudaErrorInvalidValue;
    return D.fp64 ? factor_t<float, double>(D, A, s) : factor_t<float, float>(D, A, s);
}
cudaError_t direct_solve(DirectDev& D, const double* b, double* x, const uint8_t* free_dof, const KrylovRec* rec,
                         cudaStream_t s) {
    if (!D.ready) return cudaErrorInvalidValue;
    return D.fp64 ? solve_t<double, double>(D, b, x, free_dof, rec, s) : solve_t<double, float>(D, b, x, free_dof, rec, s);
}
cudaError_t direct_solve(DirectDev& D, const float* b, float* x, const uint8_t* free_dof, const KrylovRec* rec,
                         cudaStream_t s) {
    if (!D.ready) return cudaErrorInvalidValue;
    return D.fp64 ? solve_t<float, double>(D, b, x, free_dof, rec, s) : solve_t<float, float>(D, b, x, free_dof, rec, s);
}

}  // namespace ep
