// Smoothed-aggregation AMG preconditioner: device V-cycle and Galerkin refresh.
//
// Level 0 is the live tangent K (masked to the free DOFs) with its
// block-Jacobi inverse, in FP32: a rounded copy for the FP64 path, the FP32
// tangent itself for the mixed path.  Levels >= 1 are single precision and, after every
// change of K, are rebuilt as Galerkin products A_{l+1} = R (A_l P) on the
// device with the fixed patterns computed at setup, so the coarse spaces see
// the plastic tangent's soft modes, not K_elast's.  Smoother: Chebyshev
// polynomial of degree AMG_CHEB_DEGREE in D^-1 A on [beta/30, beta],
// beta = 1.1 rho(D^-1 A) (rho by power iteration per level and per refresh);
// the same polynomial before and after the coarse correction keeps the cycle
// symmetric for symmetric A.  The coarsest level is a dense inverse, computed
// on the host after each refresh.  Every block-row product uses G lanes per
// row reading consecutive blocks.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "amg.h"
#include "pdl.cuh"

namespace ep {

constexpr int AB = 256;   // threads per CTA

template <class T>
struct Mat {
    int64_t n_rows;
    const int32_t* row_ptr;
    const int32_t* col_idx;
    const T* vals;
    const uint8_t* mask;   // per DOF (level 0) or null
};

// acc = (M x)_row for a group of G lanes (every lane of the group gets the sum)
template <int RB, int CB, int G, class TM, class TX, class TA>
__device__ __forceinline__ void group_row(const Mat<TM>& M, int64_t row, bool active, int lg, const TX* __restrict__ x,
                                          TA (&acc)[RB]) {
#pragma unroll
    for (int r = 0; r < RB; ++r) acc[r] = TA(0);
    if (active) {
        const int beg = M.row_ptr[row], end = M.row_ptr[row + 1];
        // two blocks per lane per step: two independent index -> gather chains in flight
        auto block = [&](int k) {
            const int64_t col = M.col_idx[k];
            const TM* blk = M.vals + (int64_t)k * (RB * CB);
            TA xc[CB];
#pragma unroll
            for (int c = 0; c < CB; ++c) xc[c] = (TA)x[col * CB + c];
            TM bv[RB * CB];
            if constexpr (RB * CB == 4 && sizeof(TM) == 4) {   // one 16-byte load per 2x2 FP32 block
                const float4 v = *reinterpret_cast<const float4*>(blk);
                bv[0] = v.x; bv[1] = v.y; bv[2] = v.z; bv[3] = v.w;
            } else {
#pragma unroll
                for (int e = 0; e < RB * CB; ++e) bv[e] = blk[e];
            }
#pragma unroll
            for (int r = 0; r < RB; ++r)
#pragma unroll
                for (int c = 0; c < CB; ++c) acc[r] += (TA)bv[r * CB + c] * xc[c];
        };
        int k = beg + lg;
        for (; k + G < end; k += 2 * G) {
            block(k);
            block(k + G);
        }
        if (k < end) block(k);
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
    const double beta = 1.15 * lambda, alpha = beta / 30.0;
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

// Chebyshev coefficients of every level and step, from the spectral estimates (one thread):
// coef[(l * AMG_CHEB_DEGREE + step) * 3 + {0,1,2}] = (1/theta, c1, c2)
__global__ void k_cheb_setup(const double* lam, int n_levels, float* coef) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    for (int l = 0; l < n_levels; ++l)
        for (int st = 0; st < AMG_CHEB_DEGREE; ++st) {
            const ChebCoef c = cheb_coef(lam[l], st);
            float* o = coef + (l * AMG_CHEB_DEGREE + st) * 3;
            o[0] = (float)c.inv_theta;
            o[1] = (float)c.c1;
            o[2] = (float)c.c2;
        }
}

// One Chebyshev update in precision T: r = b - A x_in (or b when x_in is null),
// d = c1 d + c2 D^-1 r (step 0: D^-1 r / theta), x_out = x_in + d.  cf = (1/theta, c1, c2).
template <int RB, int G, class T>
__global__ void __launch_bounds__(AB) k_cheb(Mat<T> A, const T* __restrict__ dinv, const T* __restrict__ b,
                                              const T* __restrict__ x_in, T* __restrict__ x_out, T* __restrict__ d,
                                              const float* __restrict__ coef, int step, const KrylovRec* rec) {
    pdl_enter();
    if (rec && rec->done) return;
    struct { T inv_theta, c1, c2; } cf = {(T)coef[0], (T)coef[1], (T)coef[2]};
    ROW_LOOP_BEGIN(A.n_rows)
    T acc[RB];
    if (x_in) group_row<RB, RB, G, T, T, T>(A, row, active, lg, x_in, acc);
    else {
#pragma unroll
        for (int r = 0; r < RB; ++r) acc[r] = T(0);
    }
    if (active && lg == 0) {
        T res[RB];
#pragma unroll
        for (int r = 0; r < RB; ++r) {
            const int64_t i = row * RB + r;
            const bool fr = A.mask ? A.mask[i] != 0 : true;
            res[r] = fr ? b[i] - acc[r] : T(0);
        }
        const T* m = dinv + row * (RB * RB);
#pragma unroll
        for (int r = 0; r < RB; ++r) {
            T s = T(0);
#pragma unroll
            for (int c = 0; c < RB; ++c) s += m[r * RB + c] * res[c];
            const int64_t i = row * RB + r;
            const T dn = (step == 0) ? cf.inv_theta * s : cf.c1 * d[i] + cf.c2 * s;
            d[i] = dn;
            x_out[i] = (x_in ? x_in[i] : T(0)) + dn;
        }
    }
    ROW_LOOP_END
}

// r = b - A x (masked)
template <int RB, int G, class T>
__global__ void __launch_bounds__(AB) k_resid(Mat<T> A, const T* __restrict__ b, const T* __restrict__ x,
                                               T* __restrict__ r, const KrylovRec* rec) {
    pdl_enter();
    if (rec && rec->done) return;
    ROW_LOOP_BEGIN(A.n_rows)
    T acc[RB];
    group_row<RB, RB, G, T, T, T>(A, row, active, lg, x, acc);
    if (active && lg == 0) {
#pragma unroll
        for (int q = 0; q < RB; ++q) {
            const int64_t i = row * RB + q;
            const bool fr = A.mask ? A.mask[i] != 0 : true;
            r[i] = fr ? b[i] - acc[q] : T(0);
        }
    }
    ROW_LOOP_END
}

// y = M x (add = 0) or y += M x (add = 1); FP32 matrix, accumulation in TACC
template <int RB, int CB, int G, class TX, class TY, class TACC = float>
__global__ void __launch_bounds__(AB) k_mv(Mat<float> M, const TX* __restrict__ x, TY* __restrict__ y, int add,
                                            const KrylovRec* rec) {
    pdl_enter();
    if (rec && rec->done) return;
    ROW_LOOP_BEGIN(M.n_rows)
    TACC acc[RB];
    group_row<RB, CB, G, float, TX, TACC>(M, row, active, lg, x, acc);
    if (active && lg == 0) {
#pragma unroll
        for (int q = 0; q < RB; ++q) {
            const int64_t i = row * RB + q;
            y[i] = add ? y[i] + (TY)acc[q] : (TY)acc[q];
        }
    }
    ROW_LOOP_END
}

// x = Ainv b, dense FP32 (coarsest level); one warp per row
__global__ void __launch_bounds__(AB) k_dense(const float* __restrict__ Ainv, int64_t n, const float* __restrict__ b,
                                               float* __restrict__ x, const KrylovRec* rec) {
    pdl_enter();
    if (rec && rec->done) return;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= n) return;
    float s = 0.f;
    for (int64_t j = lane; j < n; j += 32) s += Ainv[warp * n + j] * b[j];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) x[warp] = s;
}

// x = Ainv b, dense FP64 (coarsest level of the precise mode); one warp per row
__global__ void __launch_bounds__(AB) k_dense64(const double* __restrict__ Ainv, int64_t n,
                                                 const double* __restrict__ b, double* __restrict__ x,
                                                 const KrylovRec* rec) {
    pdl_enter();
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

// r = b - A x (masked) with FP64 A, b, r and an FP32 iterate x (the precise mode's level-0 residual
// after the FP32 pre-smoothing)
template <int RB, int G>
__global__ void __launch_bounds__(AB) k_resid_mx(Mat<double> A, const double* __restrict__ b,
                                                  const float* __restrict__ x, double* __restrict__ r,
                                                  const KrylovRec* rec) {
    pdl_enter();
    if (rec && rec->done) return;
    ROW_LOOP_BEGIN(A.n_rows)
    double acc[RB];
    group_row<RB, RB, G, double, float, double>(A, row, active, lg, x, acc);
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

// out = x + e (FP64 iterate plus the FP32 correction)
__global__ void k_add_mx(const double* __restrict__ x, const float* __restrict__ e, double* __restrict__ out, int64_t n,
                         const KrylovRec* rec) {
    pdl_enter();
    if (rec && rec->done) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = x[i] + (double)e[i];
}

// ---------------------------------------------------------------------------
// Galerkin products with fixed patterns: T = A P, A_next = R T.  One warp per
// output block row; the row is accumulated in shared memory (FP32), each lane
// taking one block of the left factor at a time.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int find_col(const int32_t* cols, int len, int c) {
    int lo = 0, hi = len;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (cols[mid] < c) lo = mid + 1;
        else hi = mid;
    }
    return (lo < len && cols[lo] == c) ? lo : -1;
}

template <int RA, int CA, int CP, class TA, class TO>
__global__ void __launch_bounds__(AB) k_rap_ap(Mat<TA> A, Mat<float> P, DevPat T, TO* __restrict__ Tvals,
                                                int max_row, int det) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    TO* sm = reinterpret_cast<TO*>(sm_raw);
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    TO* acc = sm + (size_t)wib * max_row * (RA * CP);
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < A.n_rows; i += nwarps) {
        const int tb = T.row_ptr[i], tlen = T.row_ptr[i + 1] - tb;
        const int32_t* tcols = T.col_idx + tb;
        for (int e = lane; e < tlen * RA * CP; e += 32) acc[e] = TO(0);
        __syncwarp();
        // default: lanes take the row's blocks in turn and add with shared-memory atomics; det: every
        // lane walks the whole row in order and adds only to the output blocks it owns (pos mod 32),
        // so each sum has a fixed order
        const int k0 = det ? A.row_ptr[i] : A.row_ptr[i] + lane, kstep = det ? 1 : 32;
        for (int k = k0; k < A.row_ptr[i + 1]; k += kstep) {
            const int64_t j = A.col_idx[k];
            TO a[RA * CA];
#pragma unroll
            for (int e = 0; e < RA * CA; ++e) a[e] = (TO)A.vals[(int64_t)k * (RA * CA) + e];
            for (int kp = P.row_ptr[j]; kp < P.row_ptr[j + 1]; ++kp) {
                const int pos = find_col(tcols, tlen, P.col_idx[kp]);
                if (pos < 0 || (det && (pos & 31) != lane)) continue;
                const float* p = P.vals + (int64_t)kp * (CA * CP);
                TO* dst = acc + pos * (RA * CP);
#pragma unroll
                for (int r = 0; r < RA; ++r)
#pragma unroll
                    for (int c = 0; c < CP; ++c) {
                        TO s = TO(0);
#pragma unroll
                        for (int m = 0; m < CA; ++m) s += a[r * CA + m] * (TO)p[m * CP + c];
                        if (det) dst[r * CP + c] += s;
                        else atomicAdd(dst + r * CP + c, s);
                    }
            }
        }
        __syncwarp();
        for (int e = lane; e < tlen * RA * CP; e += 32) Tvals[(int64_t)tb * (RA * CP) + e] = acc[e];
        __syncwarp();
    }
}

template <int RR, int CR, int CT, class TO>
__global__ void __launch_bounds__(AB) k_rap_rt(Mat<float> R, Mat<TO> T, DevPat An, TO* __restrict__ Anvals,
                                                int max_row, int det) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    TO* sm = reinterpret_cast<TO*>(sm_raw);
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    TO* acc = sm + (size_t)wib * max_row * (RR * CT);
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t a = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; a < R.n_rows; a += nwarps) {
        const int ab = An.row_ptr[a], alen = An.row_ptr[a + 1] - ab;
        const int32_t* acols = An.col_idx + ab;
        for (int e = lane; e < alen * RR * CT; e += 32) acc[e] = TO(0);
        __syncwarp();
        const int k0 = det ? R.row_ptr[a] : R.row_ptr[a] + lane, kstep = det ? 1 : 32;
        for (int k = k0; k < R.row_ptr[a + 1]; k += kstep) {
            const int64_t i = R.col_idx[k];
            TO rb[RR * CR];
#pragma unroll
            for (int e = 0; e < RR * CR; ++e) rb[e] = (TO)R.vals[(int64_t)k * (RR * CR) + e];
            for (int kt = T.row_ptr[i]; kt < T.row_ptr[i + 1]; ++kt) {
                const int pos = find_col(acols, alen, T.col_idx[kt]);
                if (pos < 0 || (det && (pos & 31) != lane)) continue;
                const TO* t = T.vals + (int64_t)kt * (CR * CT);
                TO* dst = acc + pos * (RR * CT);
#pragma unroll
                for (int r = 0; r < RR; ++r)
#pragma unroll
                    for (int c = 0; c < CT; ++c) {
                        TO s = TO(0);
#pragma unroll
                        for (int m = 0; m < CR; ++m) s += rb[r * CR + m] * t[m * CT + c];
                        if (det) dst[r * CT + c] += s;
                        else atomicAdd(dst + r * CT + c, s);
                    }
            }
        }
        __syncwarp();
        for (int e = lane; e < alen * RR * CT; e += 32) Anvals[(int64_t)ab * (RR * CT) + e] = acc[e];
        __syncwarp();
    }
}

// inverses of the BS x BS diagonal blocks (Gauss-Jordan with partial pivoting; identity if singular)
template <int BS, class T>
__global__ void k_blockinv(DevPat A, const T* __restrict__ Avals, const int32_t* __restrict__ diag,
                           T* __restrict__ dinv) {
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= A.n_rows) return;
    T m[BS][BS], inv[BS][BS];
    const int64_t dk = diag[row];
    if (dk < A.row_ptr[row] || dk >= A.row_ptr[row + 1]) {
        // a row without its diagonal block (the host setup rejects such operators): identity, no read
#pragma unroll
        for (int r = 0; r < BS; ++r)
#pragma unroll
            for (int c = 0; c < BS; ++c) dinv[row * (BS * BS) + r * BS + c] = (r == c) ? T(1) : T(0);
        return;
    }
    const T* src = Avals + dk * (BS * BS);
#pragma unroll
    for (int r = 0; r < BS; ++r)
#pragma unroll
        for (int c = 0; c < BS; ++c) {
            m[r][c] = src[r * BS + c];
            inv[r][c] = (r == c) ? T(1) : T(0);
        }
    bool ok = true;
#pragma unroll
    for (int c = 0; c < BS; ++c) {
        int piv = c;
        T best = fabs(m[c][c]);
#pragma unroll
        for (int r = c + 1; r < BS; ++r)
            if (fabs(m[r][c]) > best) { best = fabs(m[r][c]); piv = r; }
        if (!(best > T(0))) { ok = false; break; }
        if (piv != c) {
#pragma unroll
            for (int k = 0; k < BS; ++k) {
                T t = m[c][k]; m[c][k] = m[piv][k]; m[piv][k] = t;
                t = inv[c][k]; inv[c][k] = inv[piv][k]; inv[piv][k] = t;
            }
        }
        const T dd = T(1) / m[c][c];
#pragma unroll
        for (int k = 0; k < BS; ++k) { m[c][k] *= dd; inv[c][k] *= dd; }
#pragma unroll
        for (int r = 0; r < BS; ++r) {
            if (r == c) continue;
            const T f = m[r][c];
#pragma unroll
            for (int k = 0; k < BS; ++k) { m[r][k] -= f * m[c][k]; inv[r][k] -= f * inv[c][k]; }
        }
    }
    T* dst = dinv + row * (BS * BS);
#pragma unroll
    for (int r = 0; r < BS; ++r)
#pragma unroll
        for (int c = 0; c < BS; ++c) dst[r * BS + c] = ok ? inv[r][c] : (r == c ? T(1) : T(0));
}

// ---------------------------------------------------------------------------
// power iteration for rho(D^-1 A) (level 0 in FP64, coarse levels in FP32)
// ---------------------------------------------------------------------------
template <int RB, int G, class T>
__global__ void __launch_bounds__(AB) k_pw_apply(Mat<T> A, const T* __restrict__ dinv, const T* __restrict__ x,
                                                  T* __restrict__ y, double* part) {
    __shared__ double sh[AB / 32];
    double s2 = 0.0;
    ROW_LOOP_BEGIN(A.n_rows)
    T acc[RB];
    group_row<RB, RB, G, T, T, T>(A, row, active, lg, x, acc);
    if (active && lg == 0) {
        const T* m = dinv + row * (RB * RB);
#pragma unroll
        for (int r = 0; r < RB; ++r) {
            T s = T(0);
#pragma unroll
            for (int c = 0; c < RB; ++c) {
                const bool fr = A.mask ? A.mask[row * RB + c] != 0 : true;
                s += m[r * RB + c] * (fr ? acc[c] : T(0));
            }
            y[row * RB + r] = s;
            s2 += (double)s * (double)s;
        }
    }
    ROW_LOOP_END
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

// Start vector of the power iteration: positive pseudo-random entries (splitmix64 of the index),
// zero on prescribed DOFs.
template <class T>
__device__ __forceinline__ T pw_start(int64_t i, int64_t n, const uint8_t* mask) {
    unsigned long long z = (unsigned long long)i * 0x9E3779B97F4A7C15ull + 12345ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const double v = (double)(z >> 11) * (1.0 / 9007199254740992.0) + 0.5;
    return (mask && !mask[i]) ? T(0) : (T)(v / sqrt((double)n));
}

// lambda = ||y|| (x had unit norm); x = y / ||y||, or the start vector again if ||y|| is zero or
// not finite (so a warm-started iteration recovers from a bad tangent)
template <class T>
__global__ void __launch_bounds__(AB) k_pw_norm(const double* part, int nparts, T* y, T* x, int64_t n, double* lam,
                                                 const uint8_t* mask) {
    __shared__ double tot;
    if (threadIdx.x < 32) {
        double v = 0.0;
        for (int i = threadIdx.x; i < nparts; i += 32) v += part[i];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (threadIdx.x == 0) tot = v;
    }
    __shared__ double s_inv;
    if (threadIdx.x == 0) {
        const double nrm = sqrt(tot);
        if (blockIdx.x == 0) *lam = (nrm > 0.0 && isfinite(nrm)) ? nrm : 1.0;
        s_inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
    }
    __syncthreads();
    const T inv = (T)s_inv;
    const bool ok = s_inv > 0.0 && isfinite(s_inv);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = ok ? y[i] * inv : pw_start<T>(i, n, mask);
}

template <class T>
__global__ void k_pw_init(T* x, int64_t n, const uint8_t* mask) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = pw_start<T>(i, n, mask);
}

// ---------------------------------------------------------------------------
// Dispatch helpers
// ---------------------------------------------------------------------------
// SMs of the device (set at upload).  Row kernels use at most one resident wave of CTAs
// (RES_CTAS of AB threads per SM at <= 40 registers) and loop over the rows: every extra wave
// costs CTA launch and drain time on these short kernels.
static int g_num_sms = 152;
constexpr int RES_CTAS = 6;

static unsigned rows_grid(int64_t n_rows, int G, int res_ctas = RES_CTAS) {
    const int64_t groups_per_cta = AB / G;
    int64_t g = (n_rows + groups_per_cta - 1) / groups_per_cta;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, (int64_t)g_num_sms * res_ctas));
}

// CTAs of AB threads one SM holds for a kernel (its registers and shared memory), asked once
template <class K>
static int resident_ctas(K kern) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, AB, 0) != cudaSuccess || n < 1) n = RES_CTAS;
    return n;
}

template <class T>
static Mat<float> mat0f(const BsrT<T>& A, const float* v) { return Mat<float>{A.n_rows, A.row_ptr, A.col_idx, v, A.free_dof}; }

template <class TI, class TO>
__global__ void k_cvt(const TI* __restrict__ in, TO* __restrict__ out, int64_t n, const KrylovRec* rec) {
    pdl_enter();
    if (rec && rec->done) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (TO)in[i];
}

static unsigned cvt_grid(int64_t n) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)g_num_sms * RES_CTAS));
}
static Mat<float> matf(const DevPat& p, const float* v) { return Mat<float>{p.n_rows, p.row_ptr, p.col_idx, v, nullptr}; }

// Lanes per block row (G): about two blocks per lane, and enough lanes in total to keep the SMs
// busy on short levels (few rows: up to a warp per row, but no more lanes than blocks).
static int lanes_for(int64_t n_rows, double avg_blocks) {
    auto floor2 = [](double v) { int g = 1; while (2 * g <= v) g *= 2; return g; };
    auto ceil2 = [](double v) { int g = 1; while (g < v) g *= 2; return g; };
    int g = std::max(2, std::min(32, floor2(avg_blocks / 2.0)));
    if (n_rows * g < 32768) g = std::max(g, std::min({32, ceil2(32768.0 / std::max<int64_t>(1, n_rows)), ceil2(avg_blocks)}));
    return g;
}

#define EP_G_SWITCH(G, CALL)                  \
    switch (G) {                              \
        case 2: { constexpr int GG = 2; CALL; } break;   \
        case 4: { constexpr int GG = 4; CALL; } break;   \
        case 8: { constexpr int GG = 8; CALL; } break;   \
        case 16: { constexpr int GG = 16; CALL; } break; \
        default: { constexpr int GG = 32; CALL; } break; \
    }

template <class T>
static void cheb(int bs, int g, const Mat<T>& A, const T* dinv, const T* b, const T* xi, T* xo, T* d,
                 const float* coef_l, int step, const KrylovRec* rec, cudaStream_t s) {
    const float* cf = coef_l + step * 3;
#define EP_CHEB(RB) EP_G_SWITCH(g, { static const int occ = resident_ctas(k_cheb<RB, GG, T>);                       \
                                     launch_pdl(k_cheb<RB, GG, T>, dim3(rows_grid(A.n_rows, GG, occ)), dim3(AB), 0, s, \
                                                A, dinv, b, xi, xo, d, cf, step, rec); })
    switch (bs) {
        case 2: EP_CHEB(2) break;
        case 3: EP_CHEB(3) break;
        case 6: EP_CHEB(6) break;
    }
#undef EP_CHEB
}
template <class T>
static void resid(int bs, int g, const Mat<T>& A, const T* b, const T* x, T* r, const KrylovRec* rec, cudaStream_t s) {
#define EP_RESID(RB) EP_G_SWITCH(g, { static const int occ = resident_ctas(k_resid<RB, GG, T>);                     \
                                      launch_pdl(k_resid<RB, GG, T>, dim3(rows_grid(A.n_rows, GG, occ)), dim3(AB), 0, \
                                                 s, A, b, x, r, rec); })
    switch (bs) {
        case 2: EP_RESID(2) break;
        case 3: EP_RESID(3) break;
        case 6: EP_RESID(6) break;
    }
#undef EP_RESID
}
static void resid_mx(int bs, int g, const Mat<double>& A, const double* b, const float* x, double* r,
                     const KrylovRec* rec, cudaStream_t s) {
#define EP_RMX(RB) EP_G_SWITCH(g, { static const int occ = resident_ctas(k_resid_mx<RB, GG>);                      \
                                    launch_pdl(k_resid_mx<RB, GG>, dim3(rows_grid(A.n_rows, GG, occ)), dim3(AB), 0, s, \
                                               A, b, x, r, rec); })
    switch (bs) {
        case 2: EP_RMX(2) break;
        case 3: EP_RMX(3) break;
        case 6: EP_RMX(6) break;
    }
#undef EP_RMX
}
template <class TX, class TY, class TACC = float>
static void mv(const DevPat& p, const float* v, const TX* x, TY* y, int add, const KrylovRec* rec, cudaStream_t s) {
    const Mat<float> M = matf(p, v);
#define EP_MV(RB, CB) EP_G_SWITCH(p.g, { static const int occ = resident_ctas(k_mv<RB, CB, GG, TX, TY, TACC>);      \
                                         launch_pdl(k_mv<RB, CB, GG, TX, TY, TACC>, dim3(rows_grid(M.n_rows, GG, occ)), \
                                                    dim3(AB), 0, s, M, x, y, add, rec); })
    switch (p.rb * 10 + p.cb) {
        case 23: EP_MV(2, 3) break;
        case 32: EP_MV(3, 2) break;
        case 33: EP_MV(3, 3) break;
        case 36: EP_MV(3, 6) break;
        case 63: EP_MV(6, 3) break;
        case 66: EP_MV(6, 6) break;
    }
#undef EP_MV
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

static cudaError_t up_pat(AmgDev& D, DevPat& d, const HostBsr& h) {
    d.rb = h.rb;
    d.cb = h.cb;
    d.n_rows = h.n_rows;
    d.n_cols = h.n_cols;
    d.g = lanes_for(h.n_rows, h.n_rows ? (double)h.col_idx.size() / h.n_rows : 1.0);
    cudaError_t e;
    if ((e = up(D, &d.row_ptr, h.row_ptr)) != cudaSuccess) return e;
    return up(D, &d.col_idx, h.col_idx);
}

static cudaError_t up_f(AmgDev& D, float** dst, const std::vector<double>& src, size_t n) {
    std::vector<float> f(std::max<size_t>(n, 1), 0.f);
    for (size_t i = 0; i < src.size() && i < f.size(); ++i) f[i] = (float)src[i];
    return up(D, dst, f);
}

template <class T>
static cudaError_t dvec(AmgDev& D, T** p, int64_t n) {
    cudaError_t e = cudaMalloc((void**)p, sizeof(T) * std::max<int64_t>(1, n));
    if (e == cudaSuccess) D.allocs.push_back(*p);
    return e;
}

cudaError_t amg_upload(const AmgHierarchy& H, AmgDev& D, int num_sms) {
    if (num_sms > 0) g_num_sms = num_sms;
    // smoothing steps (1 .. AMG_CHEB_DEGREE): level-0 pre, level-0 post, coarse levels; EP_AMG_SMOOTH="pre,post,coarse"
    if (const char* sm = std::getenv("EP_AMG_SMOOTH")) {
        int a = 2, b = 2, c = 2;
        if (std::sscanf(sm, "%d,%d,%d", &a, &b, &c) == 3) {
            D.deg_pre0 = std::max(1, std::min(AMG_CHEB_DEGREE, a));
            D.deg_post0 = std::max(1, std::min(AMG_CHEB_DEGREE, b));
            D.deg_c = std::max(1, std::min(AMG_CHEB_DEGREE, c));
        }
    }
    D.n_levels = (int)H.levels.size();
    cudaError_t e;
    for (auto& ev : D.ev)
        if ((e = cudaEventCreate(&ev)) != cudaSuccess) return e;
    std::vector<double> lam(AMG_MAX_LEVELS, 1.0);
    for (int l = 0; l < D.n_levels; ++l) {
        const AmgLevel& L = H.levels[l];
        AmgDevLevel& d = D.lv[l];
        d.bs = L.bs;
        d.n = L.n;
        d.max_t_row = L.max_t_row;
        d.max_next_row = L.max_next_row;
        lam[l] = L.lambda;
        if (l > 0) {
            if ((e = up_pat(D, d.A, L.A)) != cudaSuccess) return e;
            if ((e = up_f(D, &d.Avals, L.A.vals, L.A.vals.size())) != cudaSuccess) return e;
            d.a_vals = (int64_t)L.A.vals.size();
            if ((e = up(D, &d.diag, L.diag)) != cudaSuccess) return e;
            // one bs x bs block per row of A on every coarse level (the coarsest too, unused there)
            if ((e = up_f(D, &d.dinv, L.dinv, (size_t)L.A.n_rows * L.bs * L.bs)) != cudaSuccess) return e;
            float** fv[] = {&d.b, &d.x, &d.x2, &d.d, &d.r};
            for (float** v : fv)
                if ((e = dvec(D, v, L.n)) != cudaSuccess) return e;
        } else {
            float** fv[] = {&d.b, &d.x, &d.x2, &d.d, &d.r};
            for (float** v : fv)
                if ((e = dvec(D, v, L.n)) != cudaSuccess) return e;
        }
        if (!L.P.vals.empty()) {
            if ((e = up_pat(D, d.P, L.P)) != cudaSuccess) return e;
            if ((e = up_f(D, &d.Pvals, L.P.vals, L.P.vals.size())) != cudaSuccess) return e;
            if ((e = up_pat(D, d.R, L.R)) != cudaSuccess) return e;
            if ((e = up_f(D, &d.Rvals, L.R.vals, L.R.vals.size())) != cudaSuccess) return e;
            if ((e = up_pat(D, d.T, L.T)) != cudaSuccess) return e;
            d.t_vals = (int64_t)L.T.col_idx.size() * L.T.rb * L.T.cb;
            if ((e = dvec(D, &d.Tvals, d.t_vals)) != cudaSuccess) return e;
        }
        if (!L.dense_inv.empty() && (e = up_f(D, &d.dense_inv, L.dense_inv, L.dense_inv.size())) != cudaSuccess)
            return e;
    }
    // one partial per CTA of the power iteration's SpMV, whose grid is one resident wave of AB-thread
    // CTAs (RES_CTAS per SM): fewer CTAs left it latency-bound (53 us against 18 us for a Chebyshev step)
    D.nparts = RES_CTAS * (num_sms > 0 ? num_sms : 152);
    D.nnzb0 = H.nnzb0;
    {
        const int64_t rows0 = H.levels[0].n / H.levels[0].bs;
        D.g0 = lanes_for(rows0, rows0 ? (double)H.nnzb0 / rows0 : 1.0);
    }
    if ((e = dvec(D, &D.lam, AMG_MAX_LEVELS)) != cudaSuccess) return e;
    if ((e = dvec(D, &D.coef, AMG_MAX_LEVELS * AMG_CHEB_DEGREE * 3)) != cudaSuccess) return e;
    if ((e = dvec(D, &D.pw, 2)) != cudaSuccess) return e;
    if ((e = dvec(D, &D.pwf, 2 * H.levels[0].n)) != cudaSuccess) return e;
    if ((e = dvec(D, &D.pw0, H.levels[0].n)) != cudaSuccess) return e;
    if ((e = dvec(D, &D.pw_part, D.nparts)) != cudaSuccess) return e;
    if ((e = cudaMemcpy(D.lam, lam.data(), sizeof(double) * AMG_MAX_LEVELS, cudaMemcpyHostToDevice)) != cudaSuccess)
        return e;
    k_cheb_setup<<<1, 1>>>(D.lam, D.n_levels, D.coef);
    return cudaDeviceSynchronize();
}

void amg_free(AmgDev& D) {
    for (void* p : D.allocs) cudaFree(p);
    for (auto& ev : D.ev)
        if (ev) cudaEventDestroy(ev);
    D = AmgDev{};
}

template <class T>
// Power iteration for rho(D^-1 A): `its` steps from x (a fresh pseudo-random vector when init).
// The estimate approaches rho from below; the Chebyshev interval adds a safety margin, and a
// warm start from the previous refresh's vector keeps the level-0 estimate converged although
// the top eigenvalues of a batch of similar problems are clustered.
static void power(AmgDev& D, int bs, const Mat<T>& A, const T* dinv, T* x, T* y, int64_t n, const uint8_t* mask,
                  double* lam, cudaStream_t s, bool init = true, int its = 12) {
    if (init) k_pw_init<T><<<256, 256, 0, s>>>(x, n, mask);
    for (int it = 0; it < its; ++it) {
        switch (bs) {
            case 2: k_pw_apply<2, 4, T><<<D.nparts, AB, 0, s>>>(A, dinv, x, y, D.pw_part); break;
            case 3: k_pw_apply<3, 8, T><<<D.nparts, AB, 0, s>>>(A, dinv, x, y, D.pw_part); break;
            case 6: k_pw_apply<6, 8, T><<<D.nparts, AB, 0, s>>>(A, dinv, x, y, D.pw_part); break;
        }
        k_pw_norm<T><<<256, AB, 0, s>>>(D.pw_part, D.nparts, y, x, n, lam, mask);
    }
    D.launches += 2 * its + (init ? 1 : 0);
}

// Galerkin refresh of level l + 1: T = A_l P_l, A_{l+1} = R_l T, and the block inverses of A_{l+1}
// (not on the coarsest level), accumulated and stored in TO (float, or double in precise mode).
template <class TA, class TO>
static cudaError_t rap_level(AmgDev& D, int l, const Mat<TA>& A, cudaStream_t s) {
    AmgDevLevel& L = D.lv[l];
    AmgDevLevel& N = D.lv[l + 1];
    constexpr bool F64 = sizeof(TO) == 8;
    TO* Tv = F64 ? (TO*)L.Tvals64 : (TO*)L.Tvals;
    TO* Nv = F64 ? (TO*)N.Avals64 : (TO*)N.Avals;
    TO* Nd = F64 ? (TO*)N.dinv64 : (TO*)N.dinv;
    const int bs = L.bs, k = N.bs;
    // one warp per output row; as many warps per CTA as 160 KB of shared accumulators allow
    const size_t per_ap = (size_t)std::max(1, L.max_t_row) * bs * k * sizeof(TO);
    const size_t per_rt = (size_t)std::max(1, L.max_next_row) * k * k * sizeof(TO);
    const size_t budget = 160 * 1024;
    if (per_ap > budget || per_rt > budget) return cudaErrorInvalidConfiguration;
    const int w_ap = (int)std::min<size_t>(AB / 32, budget / per_ap);
    const int w_rt = (int)std::min<size_t>(AB / 32, budget / per_rt);
    const size_t sm_ap = per_ap * w_ap, sm_rt = per_rt * w_rt;
    const unsigned g_ap = (unsigned)std::max<int64_t>(1, std::min<int64_t>((A.n_rows + w_ap - 1) / w_ap, 152 * 64));
    const unsigned g_rt = (unsigned)std::max<int64_t>(1, std::min<int64_t>((L.R.n_rows + w_rt - 1) / w_rt, 152 * 64));
    const Mat<float> P = matf(L.P, L.Pvals);
    const Mat<float> R = matf(L.R, L.Rvals);
    const Mat<TO> Tm{L.T.n_rows, L.T.row_ptr, L.T.col_idx, Tv, nullptr};
    cudaError_t e = cudaSuccess;
#define EP_AP(RA, CP)                                                                                        \
    {                                                                                                         \
        auto kern = k_rap_ap<RA, RA, CP, TA, TO>;                                                             \
        if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_ap)) !=       \
            cudaSuccess)                                                                                      \
            return e;                                                                                         \
        kern<<<g_ap, 32 * w_ap, sm_ap, s>>>(A, P, L.T, Tv, L.max_t_row, D.deterministic);                                       \
    }
#define EP_RT(RR, CR)                                                                                        \
    {                                                                                                         \
        auto kern = k_rap_rt<RR, CR, RR, TO>;                                                                 \
        if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_rt)) !=       \
            cudaSuccess)                                                                                      \
            return e;                                                                                         \
        kern<<<g_rt, 32 * w_rt, sm_rt, s>>>(R, Tm, N.A, Nv, L.max_next_row, D.deterministic);                                   \
    }
    switch (bs * 10 + k) {
        case 23: EP_AP(2, 3) EP_RT(3, 2) break;
        case 36: EP_AP(3, 6) EP_RT(6, 3) break;
        case 33: EP_AP(3, 3) EP_RT(3, 3) break;
        case 66: EP_AP(6, 6) EP_RT(6, 6) break;
        default: return cudaErrorInvalidValue;
    }
#undef EP_AP
#undef EP_RT
    if (l + 1 < D.n_levels - 1) {   // block inverses feed the smoother; the coarsest level is inverted densely
        const unsigned gb = (unsigned)((N.A.n_rows + 127) / 128);
        if (k == 3) k_blockinv<3, TO><<<gb, 128, 0, s>>>(N.A, Nv, N.diag, Nd);
        else k_blockinv<6, TO><<<gb, 128, 0, s>>>(N.A, Nv, N.diag, Nd);
        D.launches += 1;
    }
    D.launches += 2;
    return cudaGetLastError();
}

// Dense inverse of the coarsest operator (values TV on the device) on the host, stored as TI.
template <class TV, class TI>
static cudaError_t coarsest_inverse(AmgDevLevel& C, const TV* vals, TI* inv_dev, cudaStream_t s) {
    const int64_t nb = C.A.n_rows, bs = C.bs, n = C.n;
    std::vector<int32_t> rp(nb + 1), ci;
    std::vector<TV> v;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(rp.data(), C.A.row_ptr, sizeof(int32_t) * (nb + 1), cudaMemcpyDeviceToHost, s)) !=
        cudaSuccess)
        return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    ci.resize(rp[nb]);
    v.resize((size_t)rp[nb] * bs * bs);
    if ((e = cudaMemcpyAsync(ci.data(), C.A.col_idx, sizeof(int32_t) * ci.size(), cudaMemcpyDeviceToHost, s)) !=
        cudaSuccess)
        return e;
    if ((e = cudaMemcpyAsync(v.data(), vals, sizeof(TV) * v.size(), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    std::vector<double> dense((size_t)n * n, 0.0);
    for (int64_t I = 0; I < nb; ++I)
        for (int32_t b = rp[I]; b < rp[I + 1]; ++b)
            for (int r = 0; r < bs; ++r)
                for (int c = 0; c < bs; ++c)
                    dense[(size_t)(I * bs + r) * n + (size_t)ci[b] * bs + c] = (double)v[((size_t)b * bs + r) * bs + c];
    if (!amg_invert_dense(dense, (int)n)) return cudaErrorInvalidValue;
    std::vector<TI> inv(dense.begin(), dense.end());
    if ((e = cudaMemcpyAsync(inv_dev, inv.data(), sizeof(TI) * inv.size(), cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return e;
    return cudaStreamSynchronize(s);
}

// FP64 arrays of the precise mode, on first use.
static cudaError_t ensure_precise(AmgDev& D) {
    if (D.precise_ready) return cudaSuccess;
    cudaError_t e;
    for (int l = 0; l < D.n_levels; ++l) {
        AmgDevLevel& v = D.lv[l];
        if (l == 0) {
            if ((e = dvec(D, &v.x64, v.n)) != cudaSuccess) return e;
            if ((e = dvec(D, &v.r64, v.n)) != cudaSuccess) return e;
        } else {
            double** dv[] = {&v.b64, &v.x64, &v.x2_64, &v.d64, &v.r64};
            for (double** q : dv)
                if ((e = dvec(D, q, v.n)) != cudaSuccess) return e;
            if ((e = dvec(D, &v.Avals64, v.a_vals)) != cudaSuccess) return e;
            if ((e = dvec(D, &v.dinv64, v.A.n_rows * v.bs * v.bs)) != cudaSuccess) return e;
        }
        if (l + 1 < D.n_levels && (e = dvec(D, &v.Tvals64, v.t_vals)) != cudaSuccess) return e;
        if (l == D.n_levels - 1 && (e = dvec(D, &v.dense_inv64, v.n * v.n)) != cudaSuccess) return e;
    }
    if ((e = dvec(D, &D.pwd, 2 * (D.n_levels > 1 ? D.lv[1].n : 1))) != cudaSuccess) return e;
    D.precise_ready = true;
    return cudaSuccess;
}

// Common part of the refresh: level 0 is (A0's pattern, D.K0, D.minv0).  K64 (may be null): A0's
// FP64 values, from which the precise mode builds FP64 coarse operators.
template <class T>
static cudaError_t refresh_core(AmgDev& D, const BsrT<T>& A0, const double* K64, int galerkin, cudaStream_t s) {
    const int L = D.n_levels;
    const int d0 = A0.dim;
    const int64_t n0 = A0.n_rows * d0;
    const Mat<float> M0 = mat0f(A0, D.K0);
    power<float>(D, d0, M0, D.minv0, D.pw0, D.pwf, n0, A0.free_dof, D.lam + 0, s, !D.pw0_valid, 16);
    D.pw0_valid = true;
    const bool precise = D.precise && K64 && L >= 2;
    if (precise && !D.precise_valid) galerkin = 1;   // the FP64 coarse operators do not exist yet
    if (!galerkin || L < 2) {
        k_cheb_setup<<<1, 1, 0, s>>>(D.lam, L, D.coef);
        D.launches += 1;
        return cudaGetLastError();
    }
    cudaError_t e;
    if (precise) {
        if ((e = ensure_precise(D)) != cudaSuccess) return e;
        const Mat<double> M0d{A0.n_rows, A0.row_ptr, A0.col_idx, K64, A0.free_dof};
        for (int l = 0; l + 1 < L; ++l) {
            if (l == 0) e = rap_level<double, double>(D, 0, M0d, s);
            else {
                const Mat<double> Al{D.lv[l].A.n_rows, D.lv[l].A.row_ptr, D.lv[l].A.col_idx, D.lv[l].Avals64, nullptr};
                e = rap_level<double, double>(D, l, Al, s);
            }
            if (e != cudaSuccess) return e;
            AmgDevLevel& N = D.lv[l + 1];
            if (l + 1 < L - 1) {
                const Mat<double> An{N.A.n_rows, N.A.row_ptr, N.A.col_idx, N.Avals64, nullptr};
                power<double>(D, N.bs, An, N.dinv64, D.pwd, D.pwd + N.n, N.n, nullptr, D.lam + l + 1, s);
            }
        }
        k_cheb_setup<<<1, 1, 0, s>>>(D.lam, L, D.coef);
        D.launches += 1;
        AmgDevLevel& C = D.lv[L - 1];
        if ((e = coarsest_inverse<double, double>(C, C.Avals64, C.dense_inv64, s)) != cudaSuccess) return e;
        D.precise_valid = true;
        return cudaSuccess;
    }
    for (int l = 0; l + 1 < L; ++l) {
        if (l == 0) e = rap_level<float, float>(D, 0, M0, s);
        else e = rap_level<float, float>(D, l, matf(D.lv[l].A, D.lv[l].Avals), s);
        if (e != cudaSuccess) return e;
        AmgDevLevel& N = D.lv[l + 1];
        if (l + 1 < L - 1)
            power<float>(D, N.bs, matf(N.A, N.Avals), N.dinv, D.pwf, D.pwf + N.n, N.n, nullptr, D.lam + l + 1, s);
    }
    k_cheb_setup<<<1, 1, 0, s>>>(D.lam, L, D.coef);
    D.launches += 1;
    D.precise_valid = false;   // the FP64 coarse operators (if any) no longer follow the tangent
    AmgDevLevel& C = D.lv[L - 1];
    return coarsest_inverse<float, float>(C, C.Avals, C.dense_inv, s);
}

cudaError_t amg_refresh(AmgDev& D, const BsrDev& A0, const double* minv0, int galerkin, cudaStream_t s) {
    const int d0 = A0.dim;
    const int64_t n0 = A0.n_rows * d0;
    cudaError_t e;
    if (!D.K32) {   // FP32 copies of the live matrix and of its block-Jacobi inverse, on first FP64 use
        if ((e = dvec(D, &D.K32, D.nnzb0 * d0 * d0)) != cudaSuccess) return e;
        if ((e = dvec(D, &D.minv32, n0 * d0)) != cudaSuccess) return e;
    }
    k_cvt<double, float><<<cvt_grid(D.nnzb0 * d0 * d0), 256, 0, s>>>(A0.vals, D.K32, D.nnzb0 * d0 * d0, nullptr);
    k_cvt<double, float><<<cvt_grid(n0 * d0), 256, 0, s>>>(minv0, D.minv32, n0 * d0, nullptr);
    D.launches += 2;
    D.K0 = D.K32;
    D.minv0 = D.minv32;
    return refresh_core(D, A0, A0.vals, galerkin, s);
}

cudaError_t amg_refresh(AmgDev& D, const BsrF& A0, const float* minv0, int galerkin, cudaStream_t s) {
    D.K0 = A0.vals;
    D.minv0 = minv0;
    return refresh_core(D, A0, (const double*)nullptr, galerkin, s);
}

// 1-level hierarchy: out = Ainv in, FP32 inverse applied to FP64 vectors
__global__ void __launch_bounds__(AB) k_dense_d(const float* __restrict__ Ainv, int64_t n, const double* __restrict__ b,
                                                 double* __restrict__ x, const KrylovRec* rec) {
    pdl_enter();
    if (rec && rec->done) return;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= n) return;
    double s = 0.0;
    for (int64_t j = lane; j < n; j += 32) s += (double)Ainv[warp * n + j] * b[j];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) x[warp] = s;
}

// The V-cycle on FP32 vectors: x0 = M^-1 b0 (b0 and x0 distinct; level-0 work vectors x2, d, r).
// Chebyshev smoothing of A x = b by `deg` steps (1 .. AMG_CHEB_DEGREE) ending in `fin`, with `scr` as the
// other buffer.  From zero (start == nullptr) the first step needs no matrix product.  Returns the
// buffer the first step reads from (the pre-smoothing "work" buffer for the caller).
template <class T>
static void smooth(int bs, int g, const Mat<T>& A, const T* dinv, const T* b, const T* start, T* fin, T* scr, T* d,
                   const float* coef_l, int deg, const KrylovRec* rec, cudaStream_t s, int& launches) {
    const T* cur = start;
    for (int st = 0; st < deg; ++st) {
        T* nxt = ((deg - st) % 2 == 1) ? fin : scr;
        if (nxt == cur) nxt = (nxt == fin) ? scr : fin;
        cheb<T>(bs, g, A, dinv, b, cur, nxt, d, coef_l, st, rec, s);
        cur = nxt;
        ++launches;
    }
}

// The V-cycle on FP32 vectors: x0 = M^-1 b0 (b0 and x0 distinct; level-0 work vectors x2, d, r).
// Level l's pre-smoothed, coarse-corrected iterate lives in the buffer from which its post-smoothing
// ends in the level's result (x0 on level 0, lv[l].x below): the result buffer itself for an even
// number of post-smoothing steps, the scratch buffer x2 for an odd one.
template <class T>
static cudaError_t vcycle(AmgDev& D, const BsrT<T>& A0, const float* b0, float* x0, const KrylovRec* rec,
                          cudaStream_t s) {
    const int L = D.n_levels;
    AmgDevLevel& l0 = D.lv[0];
    const Mat<float> M0 = mat0f(A0, D.K0);
    const int bs0 = A0.dim;
    const float* cf0 = D.coef;
    auto work_of = [](int dpost, float* fin, float* scr) { return dpost % 2 == 0 ? fin : scr; };
    // level 0: pre-smoothing from zero, residual, restriction
    float* w0 = work_of(D.deg_post0, x0, l0.x2);
    const bool ev_ok = D.profile && D.ev[0] && D.nev + 2 <= (int)(sizeof(D.ev) / sizeof(D.ev[0]));
    if (ev_ok) cudaEventRecord(D.ev[D.nev++], s);
    smooth<float>(bs0, D.g0, M0, D.minv0, b0, nullptr, w0, w0 == x0 ? l0.x2 : x0, l0.d, cf0, D.deg_pre0, rec, s,
                  D.launches);
    if (ev_ok) cudaEventRecord(D.ev[D.nev++], s);
    resid<float>(bs0, D.g0, M0, b0, w0, l0.r, rec, s);
    mv<float, float>(l0.R, l0.Rvals, l0.r, D.lv[1].b, 0, rec, s);
    D.launches += 2;
    // coarse levels (FP32), descending
    for (int l = 1; l < L - 1; ++l) {
        AmgDevLevel& v = D.lv[l];
        const Mat<float> A = matf(v.A, v.Avals);
        float* w = work_of(D.deg_c, v.x, v.x2);
        smooth<float>(v.bs, v.A.g, A, v.dinv, v.b, nullptr, w, w == v.x ? v.x2 : v.x, v.d,
                      D.coef + l * AMG_CHEB_DEGREE * 3, D.deg_c, rec, s, D.launches);
        resid<float>(v.bs, v.A.g, A, v.b, w, v.r, rec, s);
        mv<float, float>(v.R, v.Rvals, v.r, D.lv[l + 1].b, 0, rec, s);
        D.launches += 2;
    }
    {
        AmgDevLevel& c = D.lv[L - 1];
        const unsigned g = (unsigned)((c.n * 32 + AB - 1) / AB);
        launch_pdl(k_dense, dim3(g), dim3(AB), 0, s, c.dense_inv, c.n, c.b, c.x, rec);
        D.launches += 1;
    }
    // ascending: coarse correction into the work buffer, post-smoothing into the result
    for (int l = L - 2; l >= 1; --l) {
        AmgDevLevel& v = D.lv[l];
        const Mat<float> A = matf(v.A, v.Avals);
        float* w = work_of(D.deg_c, v.x, v.x2);
        mv<float, float>(v.P, v.Pvals, D.lv[l + 1].x, w, 1, rec, s);
        smooth<float>(v.bs, v.A.g, A, v.dinv, v.b, w, v.x, v.x2, v.d, D.coef + l * AMG_CHEB_DEGREE * 3, D.deg_c, rec,
                      s, D.launches);
        D.launches += 1;
    }
    mv<float, float>(l0.P, l0.Pvals, D.lv[1].x, w0, 1, rec, s);
    smooth<float>(bs0, D.g0, M0, D.minv0, b0, w0, x0, l0.x2, l0.d, cf0, D.deg_post0, rec, s, D.launches);
    D.launches += 1;
    return cudaGetLastError();
}

void amg_profile_collect(AmgDev& D, int n_valid) {
    for (int q = 0; q < D.nev / 2 && q < n_valid; ++q) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, D.ev[2 * q], D.ev[2 * q + 1]) == cudaSuccess) {
            D.smooth0_ms += ms;
            D.smooth0_n += D.deg_pre0;
        }
    }
    D.nev = 0;
}

// Precise V-cycle, x = M^-1 b with FP64 b, x: near a limit load the tangent's softest modes sit at
// FP32 rounding level relative to its largest entries (eigenvalue ratios of 1e-8 and below), so
// FP32 coarse operators and FP32 residuals misplace them and GMRES stalls.  Here only the level-0
// smoothing runs in FP32, and always on an equation whose right-hand side is an FP64 residual:
//   x1 = S(b) (FP32, from zero);  r = b - K x1 (FP64);  x2 = x1 + P C^-1 R r (FP64 coarse levels);
//   r2 = b - K x2 (FP64);  x = x2 + S(r2) (FP32 smoothing from zero, FP64 sum).
static cudaError_t vcycle_precise(AmgDev& D, const BsrDev& A0, const double* b, double* x, const KrylovRec* rec,
                                  cudaStream_t s) {
    const int L = D.n_levels;
    AmgDevLevel& l0 = D.lv[0];
    const Mat<float> M0 = mat0f(A0, D.K0);
    const Mat<double> K64{A0.n_rows, A0.row_ptr, A0.col_idx, A0.vals, A0.free_dof};
    const int bs0 = A0.dim;
    const float* cf0 = D.coef;
    const int64_t n0 = l0.n;
    auto work_of = [](int dpost, auto* fin, auto* scr) { return dpost % 2 == 0 ? fin : scr; };
    // level 0: FP32 pre-smoothing from zero, FP64 residual, restriction (FP64 sums)
    launch_pdl(k_cvt<double, float>, dim3(cvt_grid(n0)), dim3(256), 0, s, b, l0.b, n0, rec);
    const bool ev_ok = D.profile && D.ev[0] && D.nev + 2 <= (int)(sizeof(D.ev) / sizeof(D.ev[0]));
    if (ev_ok) cudaEventRecord(D.ev[D.nev++], s);
    smooth<float>(bs0, D.g0, M0, D.minv0, l0.b, nullptr, l0.x, l0.x2, l0.d, cf0, D.deg_pre0, rec, s, D.launches);
    if (ev_ok) cudaEventRecord(D.ev[D.nev++], s);
    resid_mx(bs0, D.g0, K64, b, l0.x, l0.r64, rec, s);
    mv<double, double, double>(l0.R, l0.Rvals, l0.r64, D.lv[1].b64, 0, rec, s);
    D.launches += 3;
    // coarse levels (FP64), descending
    for (int l = 1; l < L - 1; ++l) {
        AmgDevLevel& v = D.lv[l];
        const Mat<double> A{v.A.n_rows, v.A.row_ptr, v.A.col_idx, v.Avals64, nullptr};
        double* w = work_of(D.deg_c, v.x64, v.x2_64);
        smooth<double>(v.bs, v.A.g, A, v.dinv64, v.b64, nullptr, w, w == v.x64 ? v.x2_64 : v.x64, v.d64,
                       D.coef + l * AMG_CHEB_DEGREE * 3, D.deg_c, rec, s, D.launches);
        resid<double>(v.bs, v.A.g, A, v.b64, w, v.r64, rec, s);
        mv<double, double, double>(v.R, v.Rvals, v.r64, D.lv[l + 1].b64, 0, rec, s);
        D.launches += 2;
    }
    {
        AmgDevLevel& c = D.lv[L - 1];
        const unsigned g = (unsigned)((c.n * 32 + AB - 1) / AB);
        launch_pdl(k_dense64, dim3(g), dim3(AB), 0, s, c.dense_inv64, c.n, c.b64, c.x64, rec);
        D.launches += 1;
    }
    // ascending
    for (int l = L - 2; l >= 1; --l) {
        AmgDevLevel& v = D.lv[l];
        const Mat<double> A{v.A.n_rows, v.A.row_ptr, v.A.col_idx, v.Avals64, nullptr};
        double* w = work_of(D.deg_c, v.x64, v.x2_64);
        mv<double, double, double>(v.P, v.Pvals, D.lv[l + 1].x64, w, 1, rec, s);
        smooth<double>(v.bs, v.A.g, A, v.dinv64, v.b64, w, v.x64, v.x2_64, v.d64, D.coef + l * AMG_CHEB_DEGREE * 3,
                       D.deg_c, rec, s, D.launches);
        D.launches += 1;
    }
    // level 0: x2 = x1 + P e (FP64), r2 = b - K x2 (FP64), FP32 smoothing of the correction, sum
    launch_pdl(k_cvt<float, double>, dim3(cvt_grid(n0)), dim3(256), 0, s, l0.x, l0.x64, n0, rec);
    mv<double, double, double>(l0.P, l0.Pvals, D.lv[1].x64, l0.x64, 1, rec, s);
    resid<double>(bs0, D.g0, K64, b, l0.x64, l0.r64, rec, s);
    launch_pdl(k_cvt<double, float>, dim3(cvt_grid(n0)), dim3(256), 0, s, l0.r64, l0.r, n0, rec);
    smooth<float>(bs0, D.g0, M0, D.minv0, l0.r, nullptr, l0.x, l0.x2, l0.d, cf0, D.deg_post0, rec, s, D.launches);
    launch_pdl(k_add_mx, dim3(cvt_grid(n0)), dim3(256), 0, s, (const double*)l0.x64, (const float*)l0.x, x, n0, rec);
    D.launches += 5;
    return cudaGetLastError();
}

cudaError_t amg_apply(AmgDev& D, const BsrDev& A0, const double* in, double* out, const KrylovRec* rec,
                      cudaStream_t s) {
    AmgDevLevel& l0 = D.lv[0];
    if (D.precise && D.precise_valid && D.n_levels > 1) return vcycle_precise(D, A0, in, out, rec, s);
    if (D.n_levels == 1) {
        const unsigned g = (unsigned)((l0.n * 32 + AB - 1) / AB);
        launch_pdl(k_dense_d, dim3(g), dim3(AB), 0, s, l0.dense_inv, l0.n, in, out, rec);
        D.launches += 1;
        return cudaGetLastError();
    }
    launch_pdl(k_cvt<double, float>, dim3(cvt_grid(l0.n)), dim3(256), 0, s, in, l0.b, l0.n, rec);
    cudaError_t e = vcycle(D, A0, l0.b, l0.x, rec, s);
    launch_pdl(k_cvt<float, double>, dim3(cvt_grid(l0.n)), dim3(256), 0, s, l0.x, out, l0.n, rec);
    D.launches += 2;
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t amg_apply(AmgDev& D, const BsrF& A0, const float* in, float* out, const KrylovRec* rec,
                      cudaStream_t s) {
    AmgDevLevel& l0 = D.lv[0];
    if (D.n_levels == 1) {
        const unsigned g = (unsigned)((l0.n * 32 + AB - 1) / AB);
        launch_pdl(k_dense, dim3(g), dim3(AB), 0, s, l0.dense_inv, l0.n, in, out, rec);
        D.launches += 1;
        return cudaGetLastError();
    }
    return vcycle(D, A0, in, out, rec, s);
}

}  // namespace ep
