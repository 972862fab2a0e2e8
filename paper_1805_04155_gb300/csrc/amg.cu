// Smoothed-aggregation AMG preconditioner: device V-cycle.
//
// Level 0 is the live tangent K (masked to the free DOFs) with its block-
// Jacobi inverse; levels >= 1 are the Galerkin operators built once from
// K_elast.  Smoother: Chebyshev polynomial of degree AMG_CHEB_DEGREE in
// D^-1 A on [beta/30, beta], beta = 1.1 * rho(D^-1 A); the same polynomial
// before and after the coarse correction keeps the V-cycle symmetric for
// symmetric A.  The coarsest level is applied as a dense inverse.  Every
// block-row product uses G lanes per row reading consecutive blocks.
#include <algorithm>
#include <cmath>

#include "amg.h"

namespace ep {

constexpr int AB = 256;   // threads per CTA

struct MatView {
    int64_t n_rows;
    const int32_t* row_ptr;
    const int32_t* col_idx;
    const double* vals;
    const uint8_t* mask;   // per DOF (level 0) or null
};

static MatView view(const DevBsr& M) { return MatView{M.n_rows, M.row_ptr, M.col_idx, M.vals, nullptr}; }
static MatView view(const BsrDev& A) { return MatView{A.n_rows, A.row_ptr, A.col_idx, A.vals, A.free_dof}; }

// acc = (M x)_row for a group of G lanes (every lane of the group gets the sum)
template <int RB, int CB, int G>
__device__ __forceinline__ void group_row(const MatView& M, int64_t row, bool active, int lg,
                                          const double* __restrict__ x, double (&acc)[RB]) {
#pragma unroll
    for (int r = 0; r < RB; ++r) acc[r] = 0.0;
    if (active) {
        const int beg = M.row_ptr[row], end = M.row_ptr[row + 1];
        for (int k = beg + lg; k < end; k += G) {
            const int64_t col = M.col_idx[k];
            const double* blk = M.vals + (int64_t)k * (RB * CB);
            double xc[CB];
#pragma unroll
            for (int c = 0; c < CB; ++c) xc[c] = x[col * CB + c];
#pragma unroll
            for (int r = 0; r < RB; ++r)
#pragma unroll
                for (int c = 0; c < CB; ++c) acc[r] += blk[r * CB + c] * xc[c];
        }
    }
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1)
#pragma unroll
        for (int r = 0; r < RB; ++r) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], off);
}

#define ROW_LOOP_BEGIN(NROWS)                                                            \
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;                 \
    const int lane = threadIdx.x & 31;                                                   \
    const int64_t warp = gtid >> 5;                                                      \
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;                       \
    constexpr int GPW = 32 / G;                                                          \
    const int lg = lane % G;                                                             \
    for (int64_t rbase = warp * GPW; rbase < (NROWS); rbase += nwarps * GPW) {           \
        const int64_t row = rbase + lane / G;                                            \
        const bool active = row < (NROWS);

#define ROW_LOOP_END }

struct ChebCoef {
    double inv_theta, c1, c2;
};

__device__ __forceinline__ ChebCoef cheb_coef(double lambda, int step) {
    const double beta = 1.1 * lambda, alpha = beta / 30.0;
    const double theta = 0.5 * (beta + alpha), delta = 0.5 * (beta - alpha);
    const double sigma = theta / delta;
    double rho_prev = 1.0 / sigma, rho = rho_prev;
    for (int k = 1; k <= step; ++k) {
        rho_prev = rho;
        rho = 1.0 / (2.0 * sigma - rho_prev);
    }
    ChebCoef c;
    c.inv_theta = 1.0 / theta;
    c.c1 = rho * rho_prev;
    c.c2 = 2.0 * rho / delta;
    return c;
}

// One Chebyshev update: r = b - A x_in (or b when x_in is zero), d = c1 d + c2 D^-1 r (step 0: D^-1 r / theta),
// x_out = x_in + d.
template <int RB, int G>
__global__ void __launch_bounds__(AB) k_cheb(MatView A, const double* __restrict__ dinv, const double* __restrict__ b,
                                              const double* __restrict__ x_in, double* __restrict__ x_out,
                                              double* __restrict__ d, const double* lam, double lam_host, int step,
                                              const KrylovRec* rec) {
    if (rec && rec->done) return;
    const ChebCoef cf = cheb_coef(lam ? *lam : lam_host, step);
    ROW_LOOP_BEGIN(A.n_rows)
    double acc[RB];
    if (x_in) group_row<RB, RB, G>(A, row, active, lg, x_in, acc);
    else {
#pragma unroll
        for (int r = 0; r < RB; ++r) acc[r] = 0.0;
    }
    if (active && lg == 0) {
        double res[RB];
#pragma unroll
        for (int r = 0; r < RB; ++r) {
            const int64_t i = row * RB + r;
            const bool fr = A.mask ? A.mask[i] != 0 : true;
            res[r] = fr ? b[i] - acc[r] : 0.0;
        }
        const double* m = dinv + row * (RB * RB);
#pragma unroll
        for (int r = 0; r < RB; ++r) {
            double s = 0.0;
#pragma unroll
            for (int c = 0; c < RB; ++c) s += m[r * RB + c] * res[c];
            const int64_t i = row * RB + r;
            const double dn = (step == 0) ? cf.inv_theta * s : cf.c1 * d[i] + cf.c2 * s;
            d[i] = dn;
            x_out[i] = (x_in ? x_in[i] : 0.0) + dn;
        }
    }
    ROW_LOOP_END
}

// r = b - A x (masked)
template <int RB, int G>
__global__ void __launch_bounds__(AB) k_resid(MatView A, const double* __restrict__ b, const double* __restrict__ x,
                                               double* __restrict__ r, const KrylovRec* rec) {
    if (rec && rec->done) return;
    ROW_LOOP_BEGIN(A.n_rows)
    double acc[RB];
    group_row<RB, RB, G>(A, row, active, lg, x, acc);
    if (active && lg == 0) {
#pragma unroll
        for (int q = 0; q < RB; ++q) {
            const int64_t i = row * RB + q;
            const bool fr = A.mask ? A.mask[i] != 0 : true;
            r[i] = fr ? b[i] - acc[q] : 0.0;
        }
    }
    ROW_LOOP_END
}

// y = M x (add = 0) or y += M x (add = 1)
template <int RB, int CB, int G>
__global__ void __launch_bounds__(AB) k_mv(MatView M, const double* __restrict__ x, double* __restrict__ y, int add,
                                            const KrylovRec* rec) {
    if (rec && rec->done) return;
    ROW_LOOP_BEGIN(M.n_rows)
    double acc[RB];
    group_row<RB, CB, G>(M, row, active, lg, x, acc);
    if (active && lg == 0) {
#pragma unroll
        for (int q = 0; q < RB; ++q) {
            const int64_t i = row * RB + q;
            y[i] = add ? y[i] + acc[q] : acc[q];
        }
    }
    ROW_LOOP_END
}

// x = Ainv b, dense (coarsest level); one warp per row
__global__ void __launch_bounds__(AB) k_dense(const double* __restrict__ Ainv, int64_t n, const double* __restrict__ b,
                                               double* __restrict__ x, const KrylovRec* rec) {
    if (rec && rec->done) return;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= n) return;
    double s = 0.0;
    for (int64_t j = lane; j < n; j += 32) s += Ainv[warp * n + j] * b[j];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) x[warp] = s;
}

// ---------------------------------------------------------------------------
// power iteration for rho(D^-1 A) of the live level-0 matrix
// ---------------------------------------------------------------------------
template <int RB, int G>
__global__ void __launch_bounds__(AB) k_pw_apply(MatView A, const double* __restrict__ dinv,
                                                  const double* __restrict__ x, double* __restrict__ y, double* part) {
    __shared__ double sh[AB / 32];
    double s2 = 0.0;
    ROW_LOOP_BEGIN(A.n_rows)
    double acc[RB];
    group_row<RB, RB, G>(A, row, active, lg, x, acc);
    if (active && lg == 0) {
        const double* m = dinv + row * (RB * RB);
#pragma unroll
        for (int r = 0; r < RB; ++r) {
            double s = 0.0;
#pragma unroll
            for (int c = 0; c < RB; ++c) {
                const bool fr = A.mask ? A.mask[row * RB + c] != 0 : true;
                s += m[r * RB + c] * (fr ? acc[c] : 0.0);
            }
            y[row * RB + r] = s;
            s2 += s * s;
        }
    }
    ROW_LOOP_END
    // CTA sum
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, off);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s2;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < AB / 32; ++w) t += sh[w];
        part[blockIdx.x] = t;
    }
}

// lambda = ||y|| (x had unit norm); x = y / ||y||
__global__ void __launch_bounds__(AB) k_pw_norm(const double* part, int nparts, double* y, double* x, int64_t n,
                                                 double* lam) {
    __shared__ double tot;
    if (threadIdx.x < 32) {
        double v = 0.0;
        for (int i = threadIdx.x; i < nparts; i += 32) v += part[i];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (threadIdx.x == 0) tot = v;
    }
    __syncthreads();
    const double nrm = sqrt(tot);
    if (blockIdx.x == 0 && threadIdx.x == 0) *lam = nrm;
    const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = y[i] * inv;
}

__global__ void k_pw_init(double* x, int64_t n, const uint8_t* mask) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long z = (unsigned long long)i * 0x9E3779B97F4A7C15ull + 12345ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        const double v = (double)(z >> 11) * (1.0 / 9007199254740992.0) + 0.5;
        x[i] = (mask && !mask[i]) ? 0.0 : v / sqrt((double)n);
    }
}

// ---------------------------------------------------------------------------
// Dispatch over block shapes
// ---------------------------------------------------------------------------
static unsigned rows_grid(int64_t n_rows, int G) {
    const int64_t groups_per_cta = AB / G;
    int64_t g = (n_rows + groups_per_cta - 1) / groups_per_cta;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 16));
}

template <int RB, int G>
static void cheb_t(const MatView& A, const double* dinv, const double* b, const double* xi, double* xo, double* d,
                   const double* lam, double lamh, int step, const KrylovRec* rec, cudaStream_t s) {
    k_cheb<RB, G><<<rows_grid(A.n_rows, G), AB, 0, s>>>(A, dinv, b, xi, xo, d, lam, lamh, step, rec);
}
static void cheb(int bs, const MatView& A, const double* dinv, const double* b, const double* xi, double* xo,
                 double* d, const double* lam, double lamh, int step, const KrylovRec* rec, cudaStream_t s) {
    switch (bs) {
        case 2: cheb_t<2, 4>(A, dinv, b, xi, xo, d, lam, lamh, step, rec, s); break;
        case 3: cheb_t<3, 8>(A, dinv, b, xi, xo, d, lam, lamh, step, rec, s); break;
        case 6: cheb_t<6, 8>(A, dinv, b, xi, xo, d, lam, lamh, step, rec, s); break;
    }
}
static void resid(int bs, const MatView& A, const double* b, const double* x, double* r, const KrylovRec* rec,
                  cudaStream_t s) {
    switch (bs) {
        case 2: k_resid<2, 4><<<rows_grid(A.n_rows, 4), AB, 0, s>>>(A, b, x, r, rec); break;
        case 3: k_resid<3, 8><<<rows_grid(A.n_rows, 8), AB, 0, s>>>(A, b, x, r, rec); break;
        case 6: k_resid<6, 8><<<rows_grid(A.n_rows, 8), AB, 0, s>>>(A, b, x, r, rec); break;
    }
}
static void mv(const DevBsr& M, const double* x, double* y, int add, const KrylovRec* rec, cudaStream_t s) {
    const MatView v = view(M);
    const int key = M.rb * 10 + M.cb;
    switch (key) {
        case 23: k_mv<2, 3, 4><<<rows_grid(M.n_rows, 4), AB, 0, s>>>(v, x, y, add, rec); break;
        case 32: k_mv<3, 2, 8><<<rows_grid(M.n_rows, 8), AB, 0, s>>>(v, x, y, add, rec); break;
        case 33: k_mv<3, 3, 8><<<rows_grid(M.n_rows, 8), AB, 0, s>>>(v, x, y, add, rec); break;
        case 36: k_mv<3, 6, 8><<<rows_grid(M.n_rows, 8), AB, 0, s>>>(v, x, y, add, rec); break;
        case 63: k_mv<6, 3, 8><<<rows_grid(M.n_rows, 8), AB, 0, s>>>(v, x, y, add, rec); break;
        case 66: k_mv<6, 6, 8><<<rows_grid(M.n_rows, 8), AB, 0, s>>>(v, x, y, add, rec); break;
    }
}

template <class T>
static cudaError_t up(AmgDev& D, T** dst, const std::vector<T>& src) {
    *dst = nullptr;
    cudaError_t e = cudaMalloc((void**)dst, sizeof(T) * std::max<size_t>(1, src.size()));
    if (e != cudaSuccess) return e;
    D.allocs.push_back(*dst);
    if (!src.empty()) e = cudaMemcpy(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice);
    return e;
}

static cudaError_t up_bsr(AmgDev& D, DevBsr& d, const HostBsr& h) {
    d.rb = h.rb;
    d.cb = h.cb;
    d.n_rows = h.n_rows;
    d.n_cols = h.n_cols;
    cudaError_t e;
    if ((e = up(D, &d.row_ptr, h.row_ptr)) != cudaSuccess) return e;
    if ((e = up(D, &d.col_idx, h.col_idx)) != cudaSuccess) return e;
    return up(D, &d.vals, h.vals);
}

static cudaError_t dvec(AmgDev& D, double** p, int64_t n) {
    cudaError_t e = cudaMalloc((void**)p, sizeof(double) * std::max<int64_t>(1, n));
    if (e == cudaSuccess) D.allocs.push_back(*p);
    return e;
}

cudaError_t amg_upload(const AmgHierarchy& H, AmgDev& D, int num_sms) {
    D.n_levels = (int)H.levels.size();
    cudaError_t e;
    for (int l = 0; l < D.n_levels; ++l) {
        const AmgLevel& L = H.levels[l];
        AmgDevLevel& d = D.lv[l];
        d.bs = L.bs;
        d.n = L.n;
        d.lambda = L.lambda;
        if (l > 0 && (e = up_bsr(D, d.A, L.A)) != cudaSuccess) return e;
        if (!L.dinv.empty() && (e = up(D, &d.dinv, L.dinv)) != cudaSuccess) return e;
        if (!L.P.vals.empty()) {
            if ((e = up_bsr(D, d.P, L.P)) != cudaSuccess) return e;
            if ((e = up_bsr(D, d.R, L.R)) != cudaSuccess) return e;
        }
        if (!L.dense_inv.empty() && (e = up(D, &d.dense_inv, L.dense_inv)) != cudaSuccess) return e;
        double** vecs[] = {&d.b, &d.x, &d.x2, &d.d, &d.r};
        for (double** v : vecs)
            if ((e = dvec(D, v, L.n)) != cudaSuccess) return e;
    }
    D.nparts = 2 * (num_sms > 0 ? num_sms : 152);
    if ((e = dvec(D, &D.lambda0, 1)) != cudaSuccess) return e;
    if ((e = dvec(D, &D.pw, 2 * H.levels[0].n)) != cudaSuccess) return e;
    if ((e = dvec(D, &D.pw_part, D.nparts)) != cudaSuccess) return e;
    return cudaMemcpy(D.lambda0, &H.levels[0].lambda, sizeof(double), cudaMemcpyHostToDevice);
}

void amg_free(AmgDev& D) {
    for (void* p : D.allocs) cudaFree(p);
    D = AmgDev{};
}

cudaError_t amg_refresh(AmgDev& D, const BsrDev& A0, const double* minv0, cudaStream_t s) {
    const MatView A = view(A0);
    const int64_t n = A0.n_rows * A0.dim;
    double* x = D.pw;
    double* y = D.pw + n;
    k_pw_init<<<256, 256, 0, s>>>(x, n, A0.free_dof);
    D.launches += 1;
    for (int it = 0; it < 12; ++it) {
        if (A0.dim == 2) k_pw_apply<2, 4><<<D.nparts, AB, 0, s>>>(A, minv0, x, y, D.pw_part);
        else k_pw_apply<3, 8><<<D.nparts, AB, 0, s>>>(A, minv0, x, y, D.pw_part);
        k_pw_norm<<<256, AB, 0, s>>>(D.pw_part, D.nparts, y, x, n, D.lambda0);
        D.launches += 2;
    }
    return cudaGetLastError();
}

cudaError_t amg_apply(AmgDev& D, const BsrDev& A0, const double* minv0, const double* in, double* out,
                      const KrylovRec* rec, cudaStream_t s) {
    const int L = D.n_levels;
    // descending leg
    const double* b = in;
    for (int l = 0; l < L - 1; ++l) {
        AmgDevLevel& lv = D.lv[l];
        const MatView A = (l == 0) ? view(A0) : view(lv.A);
        const double* dinv = (l == 0) ? minv0 : lv.dinv;
        const double* lam = (l == 0) ? D.lambda0 : nullptr;
        double* xa = (l == 0) ? lv.x2 : lv.x2;
        double* xb = (l == 0) ? out : lv.x;
        // pre-smoothing from zero: step 0 -> xa, step 1 -> xb
        cheb(lv.bs, A, dinv, b, nullptr, xa, lv.d, lam, lv.lambda, 0, rec, s);
        cheb(lv.bs, A, dinv, b, xa, xb, lv.d, lam, lv.lambda, 1, rec, s);
        resid(lv.bs, A, b, xb, lv.r, rec, s);
        mv(lv.R, lv.r, D.lv[l + 1].b, 0, rec, s);
        D.launches += 4;
        b = D.lv[l + 1].b;
    }
    // coarsest
    {
        AmgDevLevel& c = D.lv[L - 1];
        double* xc = (L == 1) ? out : c.x;
        const unsigned g = (unsigned)((c.n * 32 + AB - 1) / AB);
        k_dense<<<g, AB, 0, s>>>(c.dense_inv, c.n, b, xc, rec);
        D.launches += 1;
    }
    // ascending leg
    for (int l = L - 2; l >= 0; --l) {
        AmgDevLevel& lv = D.lv[l];
        const MatView A = (l == 0) ? view(A0) : view(lv.A);
        const double* dinv = (l == 0) ? minv0 : lv.dinv;
        const double* lam = (l == 0) ? D.lambda0 : nullptr;
        const double* bl = (l == 0) ? in : lv.b;
        double* xb = (l == 0) ? out : lv.x;     // current iterate
        double* xa = lv.x2;
        mv(lv.P, D.lv[l + 1].x, xb, 1, rec, s);
        // post-smoothing: xb -> xa -> xb
        cheb(lv.bs, A, dinv, bl, xb, xa, lv.d, lam, lv.lambda, 0, rec, s);
        cheb(lv.bs, A, dinv, bl, xa, xb, lv.d, lam, lv.lambda, 1, rec, s);
        D.launches += 3;
    }
    return cudaGetLastError();
}

}  // namespace ep
