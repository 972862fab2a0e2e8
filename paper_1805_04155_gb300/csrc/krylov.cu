// Preconditioned Krylov solve of eq. (lin_syst) (Section 4) on the block-CSR
// tangent, restricted to the free DOFs (the K(Q,Q) of Section 5), plus the
// small vector kernels of the Newton loop.
//
// The paper solves this system with MATLAB's sparse direct solver; here it is
// a hand-written PCG (symmetric tangents: elastic, von Mises, associated
// Drucker-Prager), BiCGStab or right-preconditioned GMRES(m) (nonassociated
// Drucker-Prager), preconditioned by point Jacobi, by the inverse dim x dim
// diagonal node blocks, or by the AMG V-cycle of amg.cu.
//
// Every solver is templated on the vector type T: double for the FP64 path,
// float for the inner solve of the mixed path (the Newton residual, computed
// in FP64 by the assembly, is the outer refinement).  Scalars (rho, alpha,
// omega, the GMRES Hessenberg matrix and rotations) are FP64 in both.
//
// Every reduction is deterministic: each CTA writes one partial sum (warp sums
// in T, the CTA's warp partials in FP64), and every consumer CTA re-reduces
// all partials in the same fixed order, so all CTAs (and all runs) agree bit
// for bit and no extra finalising launch is needed.  Iteration scalars are
// kept per iteration in a device array so that no kernel reads a value another
// CTA of the same launch may be writing.  Kernels exit at once when the device
// record says the solve has finished, so the host may enqueue iterations in
// chunks and poll rarely.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>

#include "amg.h"
#include "direct.h"
#include "ep_internal.h"
#include "pdl.cuh"

namespace ep {

constexpr int VB = 512;   // threads per CTA of vector and SpMV kernels
enum { P_RZ = 0, P_RR = 1, P_PQ = 2, P_TS = 3, P_TT = 4, P_N = 8 };

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// Sum over the CTA (warp sums in T, then the warps' partials in FP64); result valid in thread 0.
template <class T>
__device__ __forceinline__ double block_sum(T v, double* sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[wid] = (double)v;
    __syncthreads();
    double r = 0.0;
    if (wid == 0) {
        r = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
        r = warp_sum(r);
    }
    return r;
}

// Sum of the n partials of one warp-lane stripe (lane, lane + 32, ...), loaded 8 at a time so the
// L2 latencies overlap; the same order in every warp.
__device__ __forceinline__ double lane_partials(const double* __restrict__ part, int n, int lane) {
    double v = 0.0;
    for (int i0 = 0; i0 < n; i0 += 256) {
        double t[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int i = i0 + q * 32 + lane;
            t[q] = i < n ? part[i] : 0.0;
        }
        v += ((t[0] + t[1]) + (t[2] + t[3])) + ((t[4] + t[5]) + (t[6] + t[7]));
    }
    return v;
}

// Sum of n partials in a fixed order; identical in every thread of every CTA.
__device__ __forceinline__ double sum_partials(const double* part, int n, double* sh) {
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = lane_partials(part, n, threadIdx.x);
        v = warp_sum(v);
        if (threadIdx.x == 0) sh[0] = v;
    }
    __syncthreads();
    const double r = sh[0];
    __syncthreads();
    return r;
}

// Broadcast a scalar computed by thread 0 (one division per CTA, not per thread).
#define EP_CTA_SCALAR(name, expr)                 \
    __shared__ double s_##name;                   \
    if (threadIdx.x == 0) s_##name = (expr);      \
    __syncthreads();                              \
    const double name = s_##name;

// ---------------------------------------------------------------------------
// y = P A x (P = free-DOF mask), optional partial of dot(dv, y).
// G lanes share one block row; lanes read consecutive blocks (coalesced).
// ---------------------------------------------------------------------------
template <int D, int G, class TA, class TX, class TY>
__global__ void __launch_bounds__(VB) k_spmv(BsrT<TA> A, const TX* __restrict__ x, TY* __restrict__ y,
                                              const TY* __restrict__ dv, double* part, const KrylovRec* rec) {
    pdl_enter();
    __shared__ double sh[32];
    if (rec && rec->done) return;
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const int64_t warp = gtid >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    constexpr int GPW = 32 / G;
    const int lg = lane % G;
    TA dot = TA(0);
    for (int64_t rbase = warp * GPW; rbase < A.n_rows; rbase += nwarps * GPW) {
        // the G-lane groups of a warp take consecutive entries of the row order: with rows grouped
        // by length they run the same number of block steps (no lanes idle on short rows)
        const int64_t idx = rbase + lane / G;
        const int64_t row = idx < A.n_rows ? (A.perm ? (int64_t)A.perm[idx] : idx) : A.n_rows;
        TA acc[D];
#pragma unroll
        for (int r = 0; r < D; ++r) acc[r] = TA(0);
        if (row < A.n_rows) {
            const int beg = A.row_ptr[row], end = A.row_ptr[row + 1];
            auto block = [&](int k) {
                const int64_t col = A.col_idx[k];
                const TA* blk = A.vals + (int64_t)k * (D * D);
                TA bv[D * D];
                if constexpr (D == 2 && sizeof(TA) == 4) {   // one 16-byte load per 2x2 FP32 block
                    const float4 v = *reinterpret_cast<const float4*>(blk);
                    bv[0] = v.x; bv[1] = v.y; bv[2] = v.z; bv[3] = v.w;
                } else {
#pragma unroll
                    for (int e = 0; e < D * D; ++e) bv[e] = blk[e];
                }
                TA xc[D];
#pragma unroll
                for (int c = 0; c < D; ++c) xc[c] = (TA)x[col * D + c];
#pragma unroll
                for (int r = 0; r < D; ++r)
#pragma unroll
                    for (int c = 0; c < D; ++c) acc[r] += bv[r * D + c] * xc[c];
            };
            // two blocks per lane per step: two independent index -> gather chains in flight
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
            for (int r = 0; r < D; ++r) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], off);
        if (row < A.n_rows && lg == 0) {
#pragma unroll
            for (int r = 0; r < D; ++r) {
                const int64_t dof = row * D + r;
                const TA val = A.free_dof[dof] ? acc[r] : TA(0);
                y[dof] = (TY)val;
                if (dv) dot += (TA)dv[dof] * val;
            }
        }
    }
    if (part) {
        const double s = block_sum(dot, sh);
        if (threadIdx.x == 0) part[blockIdx.x] = s;
    }
}

// z = M^-1 r for one node block (minv row-major [D][D])
template <int D, class T>
__device__ __forceinline__ void apply_minv(const T* __restrict__ minv, const T* __restrict__ r, T* __restrict__ z,
                                           int64_t node) {
    const T* m = minv + node * (D * D);
    T rv[D];
#pragma unroll
    for (int c = 0; c < D; ++c) rv[c] = r[node * D + c];
#pragma unroll
    for (int i = 0; i < D; ++i) {
        T s = T(0);
#pragma unroll
        for (int c = 0; c < D; ++c) s += m[i * D + c] * rv[c];
        z[node * D + i] = s;
    }
}

// ---------------------------------------------------------------------------
// Preconditioner: kind 0 point Jacobi, 1 block Jacobi.  Prescribed DOFs get
// identity rows/columns.  A zero or non-finite pivot also gets identity.
// ---------------------------------------------------------------------------
template <int D, class T>
__global__ void k_precond(BsrT<T> A, T* minv, int kind) {
    const int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= A.n_rows) return;
    const T* blk = A.vals + (int64_t)A.diag_slot[node] * (D * D);
    T m[D][D];
    bool fr[D];
#pragma unroll
    for (int r = 0; r < D; ++r) fr[r] = A.free_dof[node * D + r] != 0;
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
        for (int c = 0; c < D; ++c) {
            T v = blk[r * D + c];
            if (!fr[r] || !fr[c] || (kind == 0 && r != c)) v = (r == c) ? T(1) : T(0);
            m[r][c] = v;
        }
    T inv[D][D];
    T det;
    if (D == 2) {
        det = m[0][0] * m[1][1] - m[0][1] * m[1][0];
        const T id = T(1) / det;
        inv[0][0] = m[1][1] * id;  inv[0][1] = -m[0][1] * id;
        inv[1][0] = -m[1][0] * id; inv[1][1] = m[0][0] * id;
    } else {
        const T c00 = m[1][1] * m[2][2] - m[1][2] * m[2][1];
        const T c01 = m[1][2] * m[2][0] - m[1][0] * m[2][2];
        const T c02 = m[1][0] * m[2][1] - m[1][1] * m[2][0];
        det = m[0][0] * c00 + m[0][1] * c01 + m[0][2] * c02;
        const T id = T(1) / det;
        inv[0][0] = c00 * id;
        inv[0][1] = (m[0][2] * m[2][1] - m[0][1] * m[2][2]) * id;
        inv[0][2] = (m[0][1] * m[1][2] - m[0][2] * m[1][1]) * id;
        inv[1][0] = c01 * id;
        inv[1][1] = (m[0][0] * m[2][2] - m[0][2] * m[2][0]) * id;
        inv[1][2] = (m[0][2] * m[1][0] - m[0][0] * m[1][2]) * id;
        inv[2][0] = c02 * id;
        inv[2][1] = (m[0][1] * m[2][0] - m[0][0] * m[2][1]) * id;
        inv[2][2] = (m[0][0] * m[1][1] - m[0][1] * m[1][0]) * id;
    }
    const bool ok = isfinite(det) && det != T(0);
    T* out = minv + node * (D * D);
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
        for (int c = 0; c < D; ++c) out[r * D + c] = ok ? inv[r][c] : (r == c ? T(1) : T(0));
}

// ---------------------------------------------------------------------------
// CG and BiCGStab kernels.  `it` is the iteration index supplied by the host.
// ---------------------------------------------------------------------------
template <class T>
struct KArgs {
    int64_t n_rows;
    const uint8_t* free_dof;
    const T* minv;
    T *x, *r, *z, *p, *q, *rhat, *v, *s, *t, *phat, *shat;
    double* part;       // [P_N][nparts]
    int nparts;
    double* h_rho;      // [hist_len]
    double* h_alpha;
    double* h_omega;
    KrylovRec* rec;
    double rtol2;
    int maxit;
    int cold;           // 1 on the first start of a solve (fixes rr0), 0 on restarts
    int amg;            // 1: the preconditioner is applied by separate V-cycle launches
};

#define PART(k) (a.part + (int64_t)(k) * a.nparts)

// Shadow residual of BiCGStab: a fixed pseudo-random vector on the free DOFs
// (splitmix64 of the DOF index and a restart counter, mapped to [-1, 1]).
// r0 itself is a poor choice here: for a traction load it lives on a few
// boundary DOFs, and (rhat, r) then cancels to zero long before convergence.
__device__ __forceinline__ double shadow_value(int64_t i, int seed) {
    unsigned long long z = (unsigned long long)i + 0x9E3779B97F4A7C15ull * (unsigned long long)(seed + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

// init: r = P (b - A x) (warm) or x = 0, r = P b (cold); z = M^-1 r (CG) or
// rhat = shadow, p = v = 0 (BiCGStab); partials (rhat or z).r and r.r.
// For the warm start q must hold A x.
template <int D, class T>
__global__ void __launch_bounds__(VB) k_init(KArgs<T> a, const T* __restrict__ b, int bicg, int warm, int seed) {
    pdl_enter();
    __shared__ double sh[32];
    T s1 = T(0), s2 = T(0);
    for (int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; node < a.n_rows;
         node += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const int64_t i = node * D + c;
            const bool fr = a.free_dof[i] != 0;
            const T ri = fr ? (warm ? b[i] - a.q[i] : b[i]) : T(0);
            a.r[i] = ri;
            if (!warm) a.x[i] = T(0);
            a.p[i] = T(0);
            if (bicg) { a.rhat[i] = fr ? (T)shadow_value(i, seed) : T(0); a.v[i] = T(0); }
        }
        if (!bicg && !a.amg) apply_minv<D>(a.minv, a.r, a.z, node);
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const int64_t i = node * D + c;
            if (bicg) s1 += a.rhat[i] * a.r[i];
            else if (!a.amg) s1 += a.z[i] * a.r[i];
            s2 += a.r[i] * a.r[i];
        }
    }
    const double b1 = block_sum(s1, sh);
    const double b2 = block_sum(s2, sh);
    if (threadIdx.x == 0) {
        if (bicg || !a.amg) PART(P_RZ)[blockIdx.x] = b1;
        PART(P_RR)[blockIdx.x] = b2;
        if (blockIdx.x == 0) { a.rec->its = 0; a.rec->done = 0; a.rec->rr = 0.0; a.rec->why = 0; }
    }
}

// Convergence test at the start of iteration `it`; returns true if the CTA must stop.
template <class T>
__device__ __forceinline__ bool check_done(const KArgs<T>& a, int it, double rz, double rr) {
    const bool first = (it == 0 && a.cold);
    const double rr0 = first ? rr : a.rec->rr0;
    int done = 0, why = 0;
    if (!isfinite(rr) || !isfinite(rz)) { done = 2; why = 2; }
    else if (rr <= a.rtol2 * rr0) { done = 1; why = 1; }
    else if (rz == 0.0) { done = 2; why = 3; }
    else if (it >= a.maxit) { done = 3; why = 6; }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (first) a.rec->rr0 = rr;
        a.rec->rr = rr;
        a.rec->its = it;
        if (done) { a.rec->done = done; a.rec->why = why; }
    }
    return done != 0;
}

// CG: p = z + beta p
template <int D, class T>
__global__ void __launch_bounds__(VB) k_cg_p(KArgs<T> a, int it) {
    pdl_enter();
    __shared__ double sh[32];
    if (a.rec->done) return;
    const double rz = sum_partials(PART(P_RZ), a.nparts, sh);
    const double rr = sum_partials(PART(P_RR), a.nparts, sh);
    if (check_done(a, it, rz, rr)) return;
    EP_CTA_SCALAR(beta, (it == 0) ? 0.0 : rz / a.h_rho[it - 1])
    if (blockIdx.x == 0 && threadIdx.x == 0) a.h_rho[it] = rz;
    const T bt = (T)beta;
    const int64_t n = a.n_rows * D;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a.p[i] = a.z[i] + bt * a.p[i];
}

// CG: alpha = rho / (p.q); x += alpha p; r -= alpha q; z = M^-1 r; partials r.z, r.r
template <int D, class T>
__global__ void __launch_bounds__(VB) k_cg_update(KArgs<T> a, int it) {
    pdl_enter();
    __shared__ double sh[32];
    if (a.rec->done) return;
    const double pq = sum_partials(PART(P_PQ), a.nparts, sh);
    EP_CTA_SCALAR(alpha, a.h_rho[it] / pq)
    const T al = (T)alpha;
    T s1 = T(0), s2 = T(0);
    for (int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; node < a.n_rows;
         node += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const int64_t i = node * D + c;
            a.x[i] += al * a.p[i];
            a.r[i] -= al * a.q[i];
        }
        if (!a.amg) apply_minv<D>(a.minv, a.r, a.z, node);
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const int64_t i = node * D + c;
            if (!a.amg) s1 += a.r[i] * a.z[i];
            s2 += a.r[i] * a.r[i];
        }
    }
    const double b1 = block_sum(s1, sh);
    const double b2 = block_sum(s2, sh);
    if (threadIdx.x == 0) {
        if (!a.amg) PART(P_RZ)[blockIdx.x] = b1;
        PART(P_RR)[blockIdx.x] = b2;
    }
}

// partial of (x, y) into PART(slot), skipped once the solve is done
template <class T>
__global__ void __launch_bounds__(VB) k_dot(KArgs<T> a, const T* __restrict__ x, const T* __restrict__ y, int64_t n,
                                             int slot) {
    pdl_enter();
    __shared__ double sh[32];
    if (a.rec->done) return;
    T s1 = T(0);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s1 += x[i] * y[i];
    const double b1 = block_sum(s1, sh);
    if (threadIdx.x == 0) PART(slot)[blockIdx.x] = b1;
}

// BiCGStab: p = r + beta (p - omega v); phat = M^-1 p
template <int D, class T>
__global__ void __launch_bounds__(VB) k_bicg_p(KArgs<T> a, int it) {
    pdl_enter();
    __shared__ double sh[32];
    if (a.rec->done) return;
    const double rho = sum_partials(PART(P_RZ), a.nparts, sh);
    const double rr = sum_partials(PART(P_RR), a.nparts, sh);
    if (check_done(a, it, rho, rr)) return;
    double om = 0.0;
    if (it > 0) {
        om = a.h_omega[it - 1];
        if (om == 0.0) {   // t = 0 in the last step: breakdown (convergence was tested above)
            if (blockIdx.x == 0 && threadIdx.x == 0) { a.rec->done = 2; a.rec->why = 5; }
            return;
        }
    }
    EP_CTA_SCALAR(beta, it > 0 ? (rho / a.h_rho[it - 1]) * (a.h_alpha[it - 1] / om) : 0.0)
    if (blockIdx.x == 0 && threadIdx.x == 0) a.h_rho[it] = rho;
    const T bt = (T)beta, omt = (T)om;
    for (int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; node < a.n_rows;
         node += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const int64_t i = node * D + c;
            a.p[i] = a.r[i] + bt * (a.p[i] - omt * a.v[i]);
        }
        if (!a.amg) apply_minv<D>(a.minv, a.p, a.phat, node);
    }
}

// BiCGStab: alpha = rho / (rhat.v); s = r - alpha v; shat = M^-1 s
template <int D, class T>
__global__ void __launch_bounds__(VB) k_bicg_s(KArgs<T> a, int it) {
    pdl_enter();
    __shared__ double sh[32];
    if (a.rec->done) return;
    const double rv = sum_partials(PART(P_PQ), a.nparts, sh);
    if (rv == 0.0 || !isfinite(rv)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) { a.rec->done = 2; a.rec->why = 4; }
        return;
    }
    EP_CTA_SCALAR(alpha, a.h_rho[it] / rv)
    if (blockIdx.x == 0 && threadIdx.x == 0) a.h_alpha[it] = alpha;
    const T al = (T)alpha;
    for (int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; node < a.n_rows;
         node += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const int64_t i = node * D + c;
            a.s[i] = a.r[i] - al * a.v[i];
        }
        if (!a.amg) apply_minv<D>(a.minv, a.s, a.shat, node);
    }
}

// BiCGStab: omega = (t.s)/(t.t); x += alpha phat + omega shat; r = s - omega t; partials rhat.r, r.r
template <int D, class T>
__global__ void __launch_bounds__(VB) k_bicg_x(KArgs<T> a, int it) {
    pdl_enter();
    __shared__ double sh[32];
    if (a.rec->done) return;
    const double ts = sum_partials(PART(P_TS), a.nparts, sh);
    const double tt = sum_partials(PART(P_TT), a.nparts, sh);
    EP_CTA_SCALAR(om, (tt > 0.0) ? ts / tt : 0.0)
    if (blockIdx.x == 0 && threadIdx.x == 0) a.h_omega[it] = om;
    const T al = (T)a.h_alpha[it], omt = (T)om;
    T s1 = T(0), s2 = T(0);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n_rows * D;
         i += (int64_t)gridDim.x * blockDim.x) {
        a.x[i] += al * a.phat[i] + omt * a.shat[i];
        const T ri = a.s[i] - omt * a.t[i];
        a.r[i] = ri;
        s1 += a.rhat[i] * ri;
        s2 += ri * ri;
    }
    const double b1 = block_sum(s1, sh);
    const double b2 = block_sum(s2, sh);
    if (threadIdx.x == 0) {
        PART(P_RZ)[blockIdx.x] = b1;
        PART(P_RR)[blockIdx.x] = b2;
    }
}

// Two dot partials (t.s and t.t) after the second SpMV of BiCGStab.
template <class T>
__global__ void __launch_bounds__(VB) k_dot2(KArgs<T> a, int64_t n) {
    pdl_enter();
    __shared__ double sh[32];
    if (a.rec->done) return;
    T s1 = T(0), s2 = T(0);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const T ti = a.t[i];
        s1 += ti * a.s[i];
        s2 += ti * ti;
    }
    const double b1 = block_sum(s1, sh);
    const double b2 = block_sum(s2, sh);
    if (threadIdx.x == 0) {
        PART(P_TS)[blockIdx.x] = b1;
        PART(P_TT)[blockIdx.x] = b2;
    }
}

// ---------------------------------------------------------------------------
// Host side: buffers
// ---------------------------------------------------------------------------
template <class T>
static cudaError_t alloc_vecs(KVecs<T>& v, int64_t n, int64_t n_rows, int dim) {
    const size_t vb = sizeof(T) * (size_t)std::max<int64_t>(n, 1);
    T** vecs[] = {&v.x, &v.r, &v.z, &v.p, &v.q, &v.rhat, &v.v, &v.s, &v.t, &v.phat, &v.shat};
    for (T** p : vecs) {
        cudaError_t e = cudaMalloc(p, vb);
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaMalloc(&v.minv, sizeof(T) * (size_t)std::max<int64_t>(n_rows, 1) * dim * dim);
    if (e != cudaSuccess) return e;
    return cudaMalloc(&v.V, vb * (GM_M + 1));
}

template <class T>
static void free_vecs(KVecs<T>& v) {
    T* vecs[] = {v.x, v.r, v.z, v.p, v.q, v.rhat, v.v, v.s, v.t, v.phat, v.shat, v.minv, v.V};
    for (T* p : vecs)
        if (p) cudaFree(p);
    v = KVecs<T>{};
}

cudaError_t krylov_alloc(KrylovWork& w, int64_t n_rows, int dim, int maxit_cap, int num_sms) {
    w = KrylovWork{};
    w.n = n_rows * dim;
    w.block = VB;
    // one resident wave of 512-thread CTAs (<= 42 registers: 3 per SM); the SpMV and the vector kernels
    // are latency-bound gathers and streams, and a third CTA per SM adds the bytes in flight they need
    w.grid = 3 * (num_sms > 0 ? num_sms : 152);
    w.nparts = w.grid;
    w.hist_len = maxit_cap + 2;
    w.gm_m = 30;
    if (const char* m = std::getenv("EP_GMRES_M")) w.gm_m = std::atoi(m);
    cudaError_t e = alloc_vecs(w.d, w.n, n_rows, dim);
    if (e != cudaSuccess) return e;
    if ((e = cudaMalloc(&w.part, sizeof(double) * std::max<int>((int)P_N, GM_M + 2) * w.nparts)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&w.gm, sizeof(double) * ((GM_M + 1) * GM_M + 3 * (GM_M + 1)))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&w.hist, sizeof(double) * 3 * w.hist_len)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&w.rec, sizeof(KrylovRec))) != cudaSuccess) return e;
    if ((e = cudaMallocHost(&w.rec_host, sizeof(KrylovRec))) != cudaSuccess) return e;
    for (auto& ev : w.ev)
        if ((e = cudaEventCreate(&ev)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&w.gdyn, sizeof(double) * 3)) != cudaSuccess) return e;
    if ((e = cudaStreamCreateWithFlags(&w.cap_stream, cudaStreamNonBlocking)) != cudaSuccess) return e;
    w.graphs = 1;
    return cudaSuccess;
}

// Destroys the cached iteration graphs.
static void drop_graphs(KrylovWork& w) {
    for (auto& g : w.gexec)
        if (g) cudaGraphExecDestroy(g);
    w.gexec.clear();
    w.gexec_launches.clear();
    w.gkey = -1;
    w.gkey_ptr = nullptr;
}

cudaError_t krylov_alloc_f32(KrylovWork& w, int64_t n_rows, int dim) {
    if (w.f.x) return cudaSuccess;
    return alloc_vecs(w.f, w.n, n_rows, dim);
}

void krylov_free(KrylovWork& w) {
    free_vecs(w.d);
    free_vecs(w.f);
    double* arrs[] = {w.part, w.hist, w.gm};
    for (double* v : arrs)
        if (v) cudaFree(v);
    if (w.rec) cudaFree(w.rec);
    if (w.rec_host) cudaFreeHost(w.rec_host);
    for (auto& ev : w.ev)
        if (ev) cudaEventDestroy(ev);
    drop_graphs(w);
    if (w.gdyn) cudaFree(w.gdyn);
    if (w.Z) cudaFree(w.Z);
    if (w.cap_stream) cudaStreamDestroy(w.cap_stream);
    w = KrylovWork{};
}

template <class T> static KVecs<T>& vecs_of(KrylovWork& w);
template <> KVecs<double>& vecs_of<double>(KrylovWork& w) { return w.d; }
template <> KVecs<float>& vecs_of<float>(KrylovWork& w) { return w.f; }

template <class T>
static cudaError_t precond_t(const BsrT<T>& A, KrylovWork& w, int kind, cudaStream_t s) {
    const unsigned g = (unsigned)((A.n_rows + 255) / 256);
    if (g == 0) return cudaSuccess;
    const int bj = (kind == 0) ? 0 : 1;    // the AMG smoother uses the block-Jacobi inverse
    T* minv = vecs_of<T>(w).minv;
    if (A.dim == 2) k_precond<2, T><<<g, 256, 0, s>>>(A, minv, bj);
    else k_precond<3, T><<<g, 256, 0, s>>>(A, minv, bj);
    w.launches += 1;
    w.use_amg = (kind == 2 && w.amg) ? 1 : 0;
    w.use_direct = 0;
    if (w.use_amg) {
        cudaError_t e = amg_refresh(*w.amg, A, minv, w.galerkin, s);
        if (e != cudaSuccess) return e;
    }
    if (kind == 3) {
        if (!w.direct || !w.direct->ready) return cudaErrorInvalidValue;
        cudaError_t e = direct_factor(*w.direct, A, s);
        if (e != cudaSuccess) return e;
        w.use_direct = 1;
    }
    return cudaGetLastError();
}

cudaError_t krylov_precond(const BsrDev& A, KrylovWork& w, int kind, cudaStream_t s) { return precond_t(A, w, kind, s); }
cudaError_t krylov_precond(const BsrF& A, KrylovWork& w, int kind, cudaStream_t s) { return precond_t(A, w, kind, s); }

bool krylov_keep_direct(KrylovWork& w) {
    if (!w.direct || !w.direct->ready || w.direct->n_factor == 0) return false;
    w.use_direct = 1;
    w.use_amg = 0;
    return true;
}

// y = P A x with A's values TA (accumulation in TA), x and y of their own types
template <int D, class TA, class TX, class TY>
static void launch_spmv(const BsrT<TA>& A, const TX* x, TY* y, const TY* dv, double* part, const KrylovRec* rec,
                        int grid, cudaStream_t s) {
    // FP64: 2 lanes per 2x2-block row (fewer idle lanes and cross-lane FP64 adds on the FP64 pipe)
    if (D == 2 && sizeof(TA) == 8) launch_pdl(k_spmv<2, 2, TA, TX, TY>, dim3(grid), dim3(VB), 0, s, A, x, y, dv, part, rec);
    else if (D == 2) launch_pdl(k_spmv<2, 4, TA, TX, TY>, dim3(grid), dim3(VB), 0, s, A, x, y, dv, part, rec);
    else launch_pdl(k_spmv<3, 8, TA, TX, TY>, dim3(grid), dim3(VB), 0, s, A, x, y, dv, part, rec);
}

// AMG V-cycle out = M^-1 in, in the solver's precision
static cudaError_t amg_apply_t(KrylovWork& w, const BsrDev& A, const double* in, double* out, const KrylovRec* rec,
                               cudaStream_t s) {
    return amg_apply(*w.amg, A, in, out, rec, s);
}
static cudaError_t amg_apply_t(KrylovWork& w, const BsrF& A, const float* in, float* out, const KrylovRec* rec,
                               cudaStream_t s) {
    return amg_apply(*w.amg, A, in, out, rec, s);
}
// FP64 operator, FP32 vectors (the V-cycle's level 0 is the refresh's FP32 copy; A gives the pattern)
static cudaError_t amg_apply_t(KrylovWork& w, const BsrDev& A, const float* in, float* out, const KrylovRec* rec,
                               cudaStream_t s) {
    const BsrF pat{A.n_rows, A.dim, A.row_ptr, A.col_idx, A.diag_slot, nullptr, A.free_dof};
    return amg_apply(*w.amg, pat, in, out, rec, s);
}
// out = M^-1 in with the current operator preconditioner: the sparse LU (precond 3) or the V-cycle
template <class TA, class TV>
static cudaError_t prec_apply_t(KrylovWork& w, const BsrT<TA>& A, const TV* in, TV* out, const KrylovRec* rec,
                                cudaStream_t s) {
    if (w.use_direct) return direct_solve(*w.direct, in, out, A.free_dof, rec, s);
    return amg_apply_t(w, A, in, out, rec, s);
}

template <int D, class T>
static cudaError_t solve_t(const BsrT<T>& A, KrylovWork& w, const T* b, int method, double rtol, int maxit,
                           cudaStream_t s, int* its, double* relres, int* status) {
    KVecs<T>& vv = vecs_of<T>(w);
    KArgs<T> a;
    a.n_rows = A.n_rows;
    a.free_dof = A.free_dof;
    a.minv = vv.minv;
    a.x = vv.x; a.r = vv.r; a.z = vv.z; a.p = vv.p; a.q = vv.q; a.rhat = vv.rhat; a.v = vv.v; a.s = vv.s; a.t = vv.t;
    a.phat = vv.phat; a.shat = vv.shat;
    a.part = w.part;
    a.nparts = w.nparts;
    if (maxit > w.hist_len - 2) maxit = w.hist_len - 2;
    a.h_rho = w.hist;
    a.h_alpha = w.hist + w.hist_len;
    a.h_omega = w.hist + 2 * w.hist_len;
    a.rec = w.rec;
    a.rtol2 = rtol * rtol;
    a.maxit = maxit;
    a.amg = ((w.use_amg && w.amg) || (w.use_direct && w.direct)) ? 1 : 0;   // an operator preconditioner
    const int grid = w.grid;
    const bool bicg = (method == 2);
    // Iterations enqueued between two polls of the device record: the first chunk covers the
    // previous solve's count (consecutive Newton systems need similar counts), later ones are
    // short, so few launches run after convergence (each costs a few microseconds even when its
    // CTAs exit at once) and few polls stall the GPU.
    int chunk = std::max(4, std::min(64, w.last_its + 2));
    const int max_restarts = bicg ? 8 : 0;
    // FP32: the recursively updated residual can drift from b - A x by O(u32) times the largest
    // intermediate residual; a solve that reports convergence is restarted once from its x, which
    // recomputes the true residual (and continues only if that one misses the tolerance)
    int n_verify = sizeof(T) == 4 ? 1 : 0;
    int total_its = 0;
    for (int restart = 0;; ++restart) {
    a.cold = (restart == 0);
    a.maxit = maxit - total_its;
    if (restart > 0) {   // warm restart from the current x after a breakdown
        launch_spmv<D, T, T, T>(A, vv.x, vv.q, nullptr, nullptr, nullptr, grid, s);
        w.launches += 1;
    }
    launch_pdl(k_init<D, T>, dim3(grid), dim3(VB), 0, s, a, b, bicg ? 1 : 0, restart > 0 ? 1 : 0, restart);
    w.launches += 1;
    if (a.amg && !bicg) {   // z = M^-1 r0, then (r, z)
        prec_apply_t(w, A, vv.r, vv.z, w.rec, s);
        launch_pdl(k_dot<T>, dim3(grid), dim3(VB), 0, s, a, vv.r, vv.z, w.n, P_RZ);
        w.launches += 1;
    }
    int it = 0;
    for (;;) {
        const int first = it;
        const int stop = std::min(it + chunk, a.maxit + 1);
        int nev = 0;
        if (a.amg && w.use_amg) w.amg->nev = 0;
        for (; it < stop; ++it) {
            // profiling events: as many iterations of the chunk as the event array holds
            const bool ev_ok = w.profile && nev + (bicg ? 4 : 2) <= (int)(sizeof(w.ev) / sizeof(w.ev[0]));
            if (!bicg) {
                launch_pdl(k_cg_p<D, T>, dim3(grid), dim3(VB), 0, s, a, it);
                if (ev_ok) cudaEventRecord(w.ev[nev++], s);
                launch_spmv<D, T, T, T>(A, vv.p, vv.q, vv.p, a.part + (int64_t)P_PQ * a.nparts, w.rec, grid, s);
                if (ev_ok) cudaEventRecord(w.ev[nev++], s);
                launch_pdl(k_cg_update<D, T>, dim3(grid), dim3(VB), 0, s, a, it);
                w.launches += 3;
                if (a.amg) {
                    prec_apply_t(w, A, vv.r, vv.z, w.rec, s);
                    launch_pdl(k_dot<T>, dim3(grid), dim3(VB), 0, s, a, vv.r, vv.z, w.n, P_RZ);
                    w.launches += 1;
                }
            } else {
                launch_pdl(k_bicg_p<D, T>, dim3(grid), dim3(VB), 0, s, a, it);
                if (a.amg) prec_apply_t(w, A, vv.p, vv.phat, w.rec, s);
                if (ev_ok) cudaEventRecord(w.ev[nev++], s);
                launch_spmv<D, T, T, T>(A, vv.phat, vv.v, vv.rhat, a.part + (int64_t)P_PQ * a.nparts, w.rec, grid, s);
                if (ev_ok) cudaEventRecord(w.ev[nev++], s);
                launch_pdl(k_bicg_s<D, T>, dim3(grid), dim3(VB), 0, s, a, it);
                if (a.amg) prec_apply_t(w, A, vv.s, vv.shat, w.rec, s);
                if (ev_ok) cudaEventRecord(w.ev[nev++], s);
                launch_spmv<D, T, T, T>(A, vv.shat, vv.t, nullptr, nullptr, w.rec, grid, s);
                if (ev_ok) cudaEventRecord(w.ev[nev++], s);
                launch_pdl(k_dot2<T>, dim3(grid), dim3(VB), 0, s, a, w.n);
                launch_pdl(k_bicg_x<D, T>, dim3(grid), dim3(VB), 0, s, a, it);
                w.launches += 6;
            }
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        e = cudaMemcpyAsync(w.rec_host, w.rec, sizeof(KrylovRec), cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return e;
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return e;
        if (w.profile) {
            // SpMVs of iterations before the converged one did work; later ones exited at once
            const int done_at = w.rec_host->done ? w.rec_host->its : it;
            const int per = bicg ? 2 : 1;
            if (a.amg && w.use_amg) amg_profile_collect(*w.amg, per * std::max(0, done_at - first));
            for (int j = 0; j < nev / 2; ++j) {
                if (first + j / per >= done_at) break;
                float ms = 0.f;
                if (cudaEventElapsedTime(&ms, w.ev[2 * j], w.ev[2 * j + 1]) == cudaSuccess) {
                    w.spmv_ms += ms;
                    w.spmv_n += 1;
                }
            }
        }
        if (w.rec_host->done || it > a.maxit) break;
        chunk = 6;
    }
    total_its += w.rec_host->its;
    if (w.rec_host->done == 2 && restart < max_restarts && std::isfinite(w.rec_host->rr) && total_its < maxit) continue;
    if (w.rec_host->done == 1 && n_verify > 0 && w.rec_host->its > 0 && total_its < maxit) {
        --n_verify;
        continue;
    }
    break;
    }
    const KrylovRec& r = *w.rec_host;
    *its = total_its;
    w.last_its = total_its;
    *relres = (r.rr0 > 0.0) ? sqrt(r.rr / r.rr0) : 0.0;
    if (r.done == 1) *status = EP_OK;
    else if (!std::isfinite(r.rr)) *status = EP_ERR_NAN;
    else if (r.done == 2 && r.rr <= rtol * rtol * r.rr0) *status = EP_OK;
    else *status = EP_ERR_KRYLOV;
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
// GMRES(m), right preconditioned: x = x0 + M^-1 V y.  The Hessenberg matrix,
// the Givens rotations and the residual estimate live in device memory (FP64)
// and are updated by thread 0 of CTA 0; every CTA recomputes the reductions it
// needs from the partial sums, so no launch reads a value written in that
// launch.
// ---------------------------------------------------------------------------
template <class TX, class TV>
struct GArgs {          // TX: solution and residual; TV: Krylov basis and preconditioned vectors
    int64_t n_rows;
    const uint8_t* free_dof;
    const TV* minv;
    TX* x;
    TX* r;              // r0 of the cycle
    TX* q;              // A x for warm restarts
    TV* z;              // M^-1 v_j
    TV* V;              // [m+1][n]
    double* H;          // [m+1][m], H[i*m + j]
    double* cs;
    double* sn;
    double* g;          // [m+1]
    double* part;       // [m+2][nparts]
    int nparts;
    KrylovRec* rec;
    double rtol2;
    int cold;
    int m;              // restart length
    const double* dyn = nullptr;   // graph replay: device (rtol^2, iteration base, cap) read instead of rtol2
                                   // and the arguments of k_gm_norm (null: direct launches)
};

#define GPART(k) (a.part + (int64_t)(k) * a.nparts)

// r = P(b - q) (warm) or P b with x = 0 (cold); partial ||r||^2 -> GPART(0)
template <int D, class TX, class TV>
__global__ void __launch_bounds__(VB) k_gm_init(GArgs<TX, TV> a, const TX* __restrict__ b, int warm) {
    pdl_enter();
    __shared__ double sh[32];
    TX s1 = TX(0);
    const int64_t n = a.n_rows * D;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const TX ri = a.free_dof[i] ? (warm ? b[i] - a.q[i] : b[i]) : TX(0);
        a.r[i] = ri;
        if (!warm) a.x[i] = TX(0);
        s1 += ri * ri;
    }
    const double b1 = block_sum(s1, sh);
    if (threadIdx.x == 0) {
        GPART(0)[blockIdx.x] = b1;
        if (blockIdx.x == 0) { a.rec->done = 0; a.rec->why = 0; }
    }
}

// beta = ||r||, v_0 = r / beta, g = (beta, 0, ...); convergence test of the cycle start
template <int D, class TX, class TV>
__global__ void __launch_bounds__(VB) k_gm_start(GArgs<TX, TV> a) {
    pdl_enter();
    __shared__ double sh[32];
    const double rr = sum_partials(GPART(0), a.nparts, sh);
    const double rr0 = a.cold ? rr : a.rec->rr0;
    __shared__ double s_b[2];
    if (threadIdx.x == 0) { s_b[0] = sqrt(rr); s_b[1] = 1.0 / s_b[0]; }
    __syncthreads();
    const double beta = s_b[0];
    const bool conv = !(rr > a.rtol2 * rr0);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (a.cold) a.rec->rr0 = rr;
        a.rec->rr = rr;
        a.rec->its = 0;
        a.g[0] = beta;
        for (int i = 1; i <= a.m; ++i) a.g[i] = 0.0;
        if (!isfinite(rr)) { a.rec->done = 2; a.rec->why = 2; }
        else if (conv) { a.rec->done = 1; a.rec->why = 1; }
    }
    if (conv || !isfinite(rr)) return;
    const TX ib = (TX)s_b[1];
    const int64_t n = a.n_rows * D;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a.V[i] = (TV)(a.r[i] * ib);
}

// z = M^-1 v_j
template <int D, class TX, class TV>
__global__ void __launch_bounds__(VB) k_gm_prec(GArgs<TX, TV> a, int j) {
    pdl_enter();
    if (a.rec->done) return;
    const TV* v = a.V + (int64_t)j * a.n_rows * D;
    for (int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; node < a.n_rows;
         node += (int64_t)gridDim.x * blockDim.x)
        apply_minv<D>(a.minv, v, a.z, node);
}

// Sum of MJ per-lane values over a warp by recursive halving: at each of the first log2(MJ) levels
// a lane keeps half of its slots and adds its partner's copies of them, then the remaining levels
// sum within lane groups.  On return lane (s << (5 - log2 MJ)) holds slot s's total.  FP64 adds
// per lane: MJ - 1 + 5 - log2 MJ instead of 5 MJ for MJ separate butterflies (an FP64 warp add
// occupies this GPU's FP64 pipe for 16 cycles).
template <int MJ, class T>
__device__ __forceinline__ T warp_multi_sum(const T (&v)[MJ], int lane) {
    T cur[MJ];
#pragma unroll
    for (int q = 0; q < MJ; ++q) cur[q] = v[q];
    int off = 16;
#pragma unroll
    for (int width = MJ; width > 1; width /= 2, off >>= 1) {
        const int half = width / 2;
        const bool up = (lane & off) != 0;
#pragma unroll
        for (int q = 0; q < half; ++q) {
            const T keep = up ? cur[q + half] : cur[q];
            const T send = up ? cur[q] : cur[q + half];
            cur[q] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
    }
    for (; off > 0; off >>= 1) cur[0] += __shfl_xor_sync(0xffffffffu, cur[0], off);
    return cur[0];
}

// The same partials from one launch (grid <= nparts; slots of absent CTAs are zeroed): v_0..v_j
// are taken MJ at a time, each thread keeping its MJ products in registers (w re-read per group,
// from L2), each group reduced over the warp by warp_multi_sum and over the CTA's warps in FP64.
template <int D, class TX, class TV, int MJ>
__global__ void __launch_bounds__(VB) k_gm_dots1(GArgs<TX, TV> a, int j) {
    pdl_enter();
    constexpr int LG = (MJ == 2 ? 1 : MJ == 4 ? 2 : MJ == 8 ? 3 : MJ == 16 ? 4 : 5);
    __shared__ double sh[MJ][VB / 32];
    if (a.rec->done) return;
    const int64_t n = a.n_rows * D;
    const TV* w = a.V + (int64_t)(j + 1) * n;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int i0 = 0; i0 <= j; i0 += MJ) {
        TV acc[MJ];
#pragma unroll
        for (int i = 0; i < MJ; ++i) acc[i] = TV(0);
        for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
            const TV wk = w[k];
            const TV* vk = a.V + (int64_t)i0 * n + k;
#pragma unroll
            for (int i = 0; i < MJ; ++i)
                if (i0 + i <= j) acc[i] += wk * vk[(int64_t)i * n];
        }
        const TV r = warp_multi_sum<MJ>(acc, lane);
        if ((lane & ((32 >> LG) - 1)) == 0) sh[lane >> (5 - LG)][wid] = (double)r;
        __syncthreads();
        if ((int)threadIdx.x < MJ && i0 + (int)threadIdx.x <= j) {
            double t = 0.0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sh[threadIdx.x][q];
            double* slot = GPART(i0 + threadIdx.x);
            slot[blockIdx.x] = t;
            for (int q = blockIdx.x + gridDim.x; q < a.nparts; q += gridDim.x) slot[q] = 0.0;
        }
        __syncthreads();
    }
}

// w -= sum_i h_i v_i; partial ||w||^2 -> GPART(GM_M + 1); CTA 0 stores H[:, j]
template <int D, class TX, class TV>
__global__ void __launch_bounds__(VB) k_gm_orth(GArgs<TX, TV> a, int j) {
    pdl_enter();
    __shared__ double sh[32];
    __shared__ TV h[GM_M];
    if (a.rec->done) return;
    {
        // h_i, i = 0..j: warp q reduces slots q, q + 16, ... (each in the fixed order of lane_partials)
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int i = wid; i <= j; i += nw) {
            const double v = warp_sum(lane_partials(GPART(i), a.nparts, lane));
            if (lane == 0) {
                h[i] = (TV)v;
                if (blockIdx.x == 0) a.H[i * GM_M + j] = v;
            }
        }
        __syncthreads();
    }
    const int64_t n = a.n_rows * D;
    TV* w = a.V + (int64_t)(j + 1) * n;
    TV s1 = TV(0);
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        // two interleaved sums: half the dependent FMA chain
        TV c0 = TV(0), c1 = TV(0);
        int i = 0;
        for (; i + 1 <= j; i += 2) {
            c0 += h[i] * a.V[(int64_t)i * n + k];
            c1 += h[i + 1] * a.V[(int64_t)(i + 1) * n + k];
        }
        if (i <= j) c0 += h[i] * a.V[(int64_t)i * n + k];
        const TV wk = w[k] - (c0 + c1);
        w[k] = wk;
        s1 += wk * wk;
    }
    const double b1 = block_sum(s1, sh);
    if (threadIdx.x == 0) GPART(GM_M + 1)[blockIdx.x] = b1;
}

// h_{j+1,j} = ||w||, v_{j+1} = w / h; CTA 0: Givens update and convergence test
template <int D, class TX, class TV>
__global__ void __launch_bounds__(VB) k_gm_norm(GArgs<TX, TV> a, int j, int it_base, int maxit) {
    pdl_enter();
    __shared__ double sh[32];
    if (a.rec->done) return;
    double rtol2 = a.rtol2;
    if (a.dyn) {
        rtol2 = a.dyn[0];
        it_base = (int)a.dyn[1];
        maxit = (int)a.dyn[2];
    }
    __shared__ double s_h[2];
    {
        const double hh = sum_partials(GPART(GM_M + 1), a.nparts, sh);
        if (threadIdx.x == 0) { s_h[0] = sqrt(hh); s_h[1] = s_h[0] > 0.0 ? 1.0 / s_h[0] : 0.0; }
        __syncthreads();
    }
    const double hn = s_h[0];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double* H = a.H;
        // apply the previous rotations to column j, held in a local array (not a chain of
        // dependent global-memory round trips)
        double col[GM_M + 1];
        for (int i = 0; i <= j; ++i) col[i] = H[i * GM_M + j];
        col[j + 1] = hn;
        for (int i = 0; i < j; ++i) {
            const double t1 = col[i], t2 = col[i + 1];
            col[i] = a.cs[i] * t1 + a.sn[i] * t2;
            col[i + 1] = -a.sn[i] * t1 + a.cs[i] * t2;
        }
        for (int i = 0; i < j; ++i) H[i * GM_M + j] = col[i];
        const double h0 = col[j], h1 = col[j + 1];
        const double den = hypot(h0, h1);
        const double c = den > 0.0 ? h0 / den : 1.0, s = den > 0.0 ? h1 / den : 0.0;
        a.cs[j] = c;
        a.sn[j] = s;
        H[j * GM_M + j] = den;
        H[(j + 1) * GM_M + j] = 0.0;
        a.g[j + 1] = -s * a.g[j];
        a.g[j] = c * a.g[j];
        const double res2 = a.g[j + 1] * a.g[j + 1];
        a.rec->rr = res2;
        a.rec->its = j + 1;
        if (!isfinite(res2) || den == 0.0) { a.rec->done = 2; a.rec->why = isfinite(res2) ? 4 : 2; }
        else if (res2 <= rtol2 * a.rec->rr0 || hn == 0.0) { a.rec->done = 1; a.rec->why = 1; }
        else if (it_base + j + 1 >= maxit) { a.rec->done = 3; a.rec->why = 6; }
        else if (j + 1 == a.m) { a.rec->done = 4; }   // end of the cycle: update and restart
    }
    if (hn == 0.0 || !isfinite(hn)) return;
    const TV ih = (TV)s_h[1];
    const int64_t n = a.n_rows * D;
    TV* w = a.V + (int64_t)(j + 1) * n;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        w[k] *= ih;
}

// y = R^-1 g (k x k upper triangle) into shared memory, by thread 0 of every CTA
template <class TX, class TV>
__device__ __forceinline__ void gm_solve_y(const GArgs<TX, TV>& a, int k, TV* y) {
    __shared__ double yd[GM_M];
    if (threadIdx.x == 0) {
        for (int i = k - 1; i >= 0; --i) {
            double s = a.g[i];
            for (int l = i + 1; l < k; ++l) s -= a.H[i * GM_M + l] * yd[l];
            yd[i] = s / a.H[i * GM_M + i];
            y[i] = (TV)yd[i];
        }
    }
    __syncthreads();
}

// x += M^-1 (V_k y), y = R^-1 g (k = its of the cycle); every CTA solves the small triangle itself
template <int D, class TX, class TV>
__global__ void __launch_bounds__(VB) k_gm_update(GArgs<TX, TV> a, int k) {
    pdl_enter();
    __shared__ TV y[GM_M];
    gm_solve_y(a, k, y);
    const int64_t n = a.n_rows * D;
    for (int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; node < a.n_rows;
         node += (int64_t)gridDim.x * blockDim.x) {
        TV u[D];
#pragma unroll
        for (int c = 0; c < D; ++c) {
            TV s = TV(0);
            for (int i = 0; i < k; ++i) s += y[i] * a.V[(int64_t)i * n + node * D + c];
            u[c] = s;
        }
        const TV* m = a.minv + node * (D * D);
#pragma unroll
        for (int r = 0; r < D; ++r) {
            TV s = TV(0);
#pragma unroll
            for (int c = 0; c < D; ++c) s += m[r * D + c] * u[c];
            a.x[node * D + r] += (TX)s;
        }
    }
}

// u = V_k y (y = R^-1 g solved redundantly by every CTA)
template <int D, class TX, class TV>
__global__ void __launch_bounds__(VB) k_gm_combine(GArgs<TX, TV> a, int k, TV* __restrict__ u) {
    pdl_enter();
    __shared__ TV y[GM_M];
    gm_solve_y(a, k, y);
    const int64_t n = a.n_rows * D;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        TV s = TV(0);
        for (int i = 0; i < k; ++i) s += y[i] * a.V[(int64_t)i * n + t];
        u[t] = s;
    }
}

// x += Z_k y (Z: the cycle's preconditioned vectors z_j = M^-1 v_j; y = R^-1 g solved by every CTA)
template <int D, class TX, class TV>
__global__ void __launch_bounds__(VB) k_gm_zupdate(GArgs<TX, TV> a, int k, const TV* __restrict__ Z) {
    pdl_enter();
    __shared__ TV y[GM_M];
    gm_solve_y(a, k, y);
    const int64_t n = a.n_rows * D;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        TV s = TV(0);
        for (int i = 0; i < k; ++i) s += y[i] * Z[(int64_t)i * n + t];
        a.x[t] += (TX)s;
    }
}

// x += z (z of the basis precision)
template <class TX, class TV>
__global__ void k_axpy_plain(TX* __restrict__ x, const TV* __restrict__ z, int64_t n) {
    pdl_enter();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] += (TX)z[i];
}

// per-chunk scalars of the replayed iteration graphs
__global__ void k_gdyn_set(double* dyn, double rtol2, int it_base, int maxit) {
    pdl_enter();
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        dyn[0] = rtol2;
        dyn[1] = (double)it_base;
        dyn[2] = (double)maxit;
    }
}

// TA: operator values; TX: solution and residual; TV: basis (TA = TX = TV for the FP64 and FP32
// solvers; TA = TX = double, TV = float for the FP32-basis solve with the FP64 operator)
template <int D, class TA, class TX, class TV>
static cudaError_t solve_gmres_t(const BsrT<TA>& A, KrylovWork& w, const TX* b, double rtol, int maxit,
                                 cudaStream_t s, int* its, double* relres, int* status) {
    KVecs<TX>& vx = vecs_of<TX>(w);
    KVecs<TV>& vv = vecs_of<TV>(w);
    GArgs<TX, TV> a;
    a.n_rows = A.n_rows;
    a.free_dof = A.free_dof;
    a.minv = vv.minv;
    a.x = vx.x;
    a.r = vx.r;
    a.q = vx.q;
    a.z = vv.z;
    a.V = vv.V;
    a.H = w.gm;
    a.cs = w.gm + (GM_M + 1) * GM_M;
    a.sn = a.cs + (GM_M + 1);
    a.g = a.sn + (GM_M + 1);
    a.part = w.part;
    a.nparts = w.nparts;
    a.rec = w.rec;
    a.rtol2 = rtol * rtol;
    a.m = std::max(2, std::min(GM_M, w.gm_m > 0 ? w.gm_m : 30));
    const int grid = w.grid;
    const bool use_amg = w.use_amg && w.amg;
    const bool use_direct = w.use_direct && w.direct;
    const bool use_op = use_amg || use_direct;   // an operator preconditioner (z = M^-1 v by its own kernels)
    int total = 0;
    // sparse LU: z_j kept in Z (allocated on first use, reallocated for a longer restart)
    TV* Zb = nullptr;
    if (use_direct) {
        if (!w.Z || w.z_cap < a.m || w.z_bytes != (int)sizeof(TV)) {
            if (w.Z) cudaFree(w.Z);
            w.Z = nullptr;
            cudaError_t e = cudaMalloc(&w.Z, sizeof(TV) * (size_t)a.m * (size_t)w.n);
            if (e != cudaSuccess) return e;
            w.z_cap = a.m;
            w.z_bytes = (int)sizeof(TV);
            drop_graphs(w);   // captured iterations name the old buffer
        }
        Zb = static_cast<TV*>(w.Z);
    }
    // the launches of iteration j of a cycle (direct, or into a capture)
    auto issue = [&](const GArgs<TX, TV>& ga, int j, cudaStream_t st, int& nev) {
        TV* zj = use_direct ? Zb + (int64_t)j * w.n : ga.z;
        if (use_op) prec_apply_t(w, A, ga.V + (int64_t)j * w.n, zj, w.rec, st);
        else launch_pdl(k_gm_prec<D, TX, TV>, dim3(grid), dim3(VB), 0, st, ga, j);
        const bool ev_ok = w.profile && nev + 2 <= (int)(sizeof(w.ev) / sizeof(w.ev[0]));
        if (ev_ok) cudaEventRecord(w.ev[nev++], st);
        launch_spmv<D, TA, TV, TV>(A, zj, ga.V + (int64_t)(j + 1) * w.n, nullptr, nullptr, w.rec, grid, st);
        if (ev_ok) cudaEventRecord(w.ev[nev++], st);
        // one resident wave (FP32: 61 registers, 2 CTAs per SM); FP64: one CTA per SM, fewer
        // cross-lane FP64 adds
        launch_pdl(k_gm_dots1<D, TX, TV, sizeof(TV) == 8 ? 4 : 8>,
                   dim3(std::max(1, sizeof(TV) == 8 ? grid / 3 : 2 * grid / 3)), dim3(VB), 0, st, ga, j);
        launch_pdl(k_gm_orth<D, TX, TV>, dim3(grid), dim3(VB), 0, st, ga, j);
        launch_pdl(k_gm_norm<D, TX, TV>, dim3(grid), dim3(VB), 0, st, ga, j, total, maxit);
        w.launches += 5;
    };
    const bool use_graphs = w.graphs && !w.profile && w.cap_stream;
    if (use_graphs) {
        // graphs are valid for one operator, solver precision, preconditioner and restart length
        const long long key = ((long long)a.m << 32) | ((long long)D << 24) | ((long long)sizeof(TA) << 16) |
                              ((long long)sizeof(TX) << 12) | ((long long)sizeof(TV) << 8) |
                              (use_amg ? 2 : 0) | (use_amg && w.amg->precise ? 1 : 0) | (use_direct ? 4 : 0);
        if (key != w.gkey || (const void*)A.vals != w.gkey_ptr) {
            drop_graphs(w);
            w.gkey = key;
            w.gkey_ptr = (const void*)A.vals;
        }
        if ((int)w.gexec.size() < a.m) {
            w.gexec.resize(a.m, nullptr);
            w.gexec_launches.resize(a.m, 0);
        }
    }
    KrylovRec last{};
    double rr_prev_end = 0.0;   // residual estimate ||r||^2 at the end of the previous cycle
    // FP32 basis: re-check a converged estimate once (see solve_t).  Sparse LU: a tight solve restarts
    // once from its x, so that the FP64 residual b - A x, not the Arnoldi estimate, ends it.  (Its
    // update is x += Z y with the stored z_j = M^-1 v_j, consistent with the Arnoldi relation; the
    // first form, x += M^-1 (V y), carried the rounding of an FP32 solve of the combination: 5e-7
    // instead of 1e-13.)
    int n_verify = (sizeof(TV) == 4 || (use_direct && rtol < 1e-5)) ? 1 : 0;
    for (int cycle = 0;; ++cycle) {
        a.cold = (cycle == 0);
        if (cycle > 0) {
            launch_spmv<D, TA, TX, TX>(A, vx.x, vx.q, nullptr, nullptr, nullptr, grid, s);
            w.launches += 1;
        }
        launch_pdl(k_gm_init<D, TX, TV>, dim3(grid), dim3(VB), 0, s, a, b, cycle > 0 ? 1 : 0);
        launch_pdl(k_gm_start<D, TX, TV>, dim3(grid), dim3(VB), 0, s, a);
        w.launches += 2;
        // the cycle's iterations in chunks, polling the device record between chunks (the first
        // chunk covers the previous solve's count, see solve_t)
        int chunk = std::max(4, std::min(a.m, w.last_its + 2 - total));
        double t_enq = 0.0, t_wait = 0.0;
        for (int j0 = 0; j0 < a.m; j0 += chunk, chunk = 6) {
            const auto t0 = std::chrono::steady_clock::now();
            const int j1 = std::min(a.m, j0 + chunk);
            int nev = 0;
            if (use_amg) w.amg->nev = 0;
            if (use_graphs) {
                launch_pdl(k_gdyn_set, dim3(1), dim3(32), 0, s, w.gdyn, a.rtol2, total, maxit);
                w.launches += 1;
                for (int j = j0; j < j1; ++j) {
                    if (!w.gexec[j]) {
                        // capture iteration j once on the private stream (nothing runs during a capture)
                        GArgs<TX, TV> ac = a;
                        ac.dyn = w.gdyn;
                        const int l_save = w.launches, la_save = use_amg ? w.amg->launches : 0;
                        const int ld_save = use_direct ? w.direct->launches : 0;
                        cudaGraph_t g = nullptr;
                        cudaError_t e = cudaStreamBeginCapture(w.cap_stream, cudaStreamCaptureModeThreadLocal);
                        if (e != cudaSuccess) return e;
                        issue(ac, j, w.cap_stream, nev);
                        e = cudaStreamEndCapture(w.cap_stream, &g);
                        if (e != cudaSuccess) return e;
                        e = cudaGraphInstantiate(&w.gexec[j], g, 0);
                        cudaGraphDestroy(g);
                        if (e != cudaSuccess) return e;
                        w.gexec_launches[j] = (w.launches - l_save) + (use_amg ? w.amg->launches - la_save : 0) +
                                              (use_direct ? w.direct->launches - ld_save : 0);
                        w.launches = l_save;
                        if (use_amg) w.amg->launches = la_save;
                        if (use_direct) w.direct->launches = ld_save;
                    }
                    cudaError_t e = cudaGraphLaunch(w.gexec[j], s);
                    if (e != cudaSuccess) return e;
                    w.launches += w.gexec_launches[j];
                    w.graph_launches += 1;
                }
            } else {
                for (int j = j0; j < j1; ++j) issue(a, j, s, nev);
            }
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return e;
            if ((e = cudaMemcpyAsync(w.rec_host, w.rec, sizeof(KrylovRec), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
                return e;
            const auto t1 = std::chrono::steady_clock::now();
            if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
            t_enq += std::chrono::duration<double, std::milli>(t1 - t0).count();
            t_wait += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t1).count();
            last = *w.rec_host;
            // sparse-LU solves that did work (replayed graphs included)
            if (use_direct) w.direct->n_solve += std::max(0, std::min(j1, last.its) - j0);
            if (w.profile) {
                if (use_amg) amg_profile_collect(*w.amg, std::max(0, std::min(j1, last.its) - j0));
                for (int q = 0; q < nev / 2 && j0 + q < last.its; ++q) {
                    float ms = 0.f;
                    if (cudaEventElapsedTime(&ms, w.ev[2 * q], w.ev[2 * q + 1]) == cudaSuccess) {
                        w.spmv_ms += ms;
                        w.spmv_n += 1;
                    }
                }
            }
            if (last.done) break;
        }
        if (w.verbose > 1)
            std::fprintf(stderr, "[ep]   gmres cycle %d: its %d, host enqueue %.3f ms, wait %.3f ms\n", cycle,
                         last.its, t_enq, t_wait);
        if (last.its > 0) {
            if (use_direct) {
                launch_pdl(k_gm_zupdate<D, TX, TV>, dim3(grid), dim3(VB), 0, s, a, last.its, (const TV*)Zb);
                w.launches += 1;
            } else if (use_op) {
                launch_pdl(k_gm_combine<D, TX, TV>, dim3(grid), dim3(VB), 0, s, a, last.its, vv.q);
                prec_apply_t(w, A, vv.q, vv.z, nullptr, s);
                launch_pdl(k_axpy_plain<TX, TV>, dim3(grid), dim3(VB), 0, s, vx.x, vv.z, w.n);
                w.launches += 2;
            } else {
                launch_pdl(k_gm_update<D, TX, TV>, dim3(grid), dim3(VB), 0, s, a, last.its);
                w.launches += 1;
            }
        }
        total += last.its;
        if (last.done == 1 && n_verify > 0 && last.its > 0) {   // a new cycle recomputes b - A x
            --n_verify;
            continue;
        }
        if (last.done != 4) break;           // converged, breakdown, non-finite or cap
        // an FP32-basis solve whose restart cycle did not halve the residual has reached what its
        // rounding allows on this matrix: stop (the caller treats it as an inexact or failed solve)
        if (sizeof(TV) == 4 && w.stall_guard && last.rr > 0.25 * (cycle == 0 ? last.rr0 : rr_prev_end)) break;
        // an FP64 solve whose preconditioner no longer resolves the matrix: stop early (the caller
        // switches to the precise V-cycle)
        if (sizeof(TV) == 8 && w.stall_guard64 && cycle >= 1 && last.rr > 0.81 * rr_prev_end) break;
        rr_prev_end = last.rr;
    }
    *its = total;
    w.last_its = total;
    *relres = last.rr0 > 0.0 ? sqrt(last.rr / last.rr0) : 0.0;
    if (last.done == 1) *status = EP_OK;
    else if (!std::isfinite(last.rr)) *status = EP_ERR_NAN;
    else if (last.rr <= rtol * rtol * last.rr0) *status = EP_OK;
    else *status = EP_ERR_KRYLOV;
    return cudaStreamSynchronize(s);
}

template <class T>
static cudaError_t solve_any(const BsrT<T>& A, KrylovWork& w, const T* b, int method, double rtol, int maxit,
                             cudaStream_t s, int* its, double* relres, int* status) {
    if (method == 3) {
        if (A.dim == 2) return solve_gmres_t<2, T, T, T>(A, w, b, rtol, maxit, s, its, relres, status);
        return solve_gmres_t<3, T, T, T>(A, w, b, rtol, maxit, s, its, relres, status);
    }
    if (A.dim == 2) return solve_t<2, T>(A, w, b, method, rtol, maxit, s, its, relres, status);
    return solve_t<3, T>(A, w, b, method, rtol, maxit, s, its, relres, status);
}

cudaError_t krylov_solve(const BsrDev& A, KrylovWork& w, const double* b, int method, double rtol, int maxit,
                         cudaStream_t s, int* its, double* relres, int* status) {
    return solve_any(A, w, b, method, rtol, maxit, s, its, relres, status);
}
cudaError_t krylov_solve(const BsrF& A, KrylovWork& w, const float* b, int method, double rtol, int maxit,
                         cudaStream_t s, int* its, double* relres, int* status) {
    if (!w.f.x) return cudaErrorInvalidValue;
    return solve_any(A, w, b, method, rtol, maxit, s, its, relres, status);
}

cudaError_t krylov_solve_fp32_basis(const BsrDev& A, KrylovWork& w, const double* b, double rtol, int maxit,
                                    cudaStream_t s, int* its, double* relres, int* status) {
    if (!w.f.x) return cudaErrorInvalidValue;
    // the basis-precision preconditioner: the FP64 block-Jacobi inverse rounded to FP32
    cudaError_t e = vec_cvt_f32(w.d.minv, w.f.minv, A.n_rows * A.dim * A.dim, s);
    if (e != cudaSuccess) return e;
    w.launches += 1;
    if (A.dim == 2) return solve_gmres_t<2, double, double, float>(A, w, b, rtol, maxit, s, its, relres, status);
    return solve_gmres_t<3, double, double, float>(A, w, b, rtol, maxit, s, its, relres, status);
}

// ---------------------------------------------------------------------------
// Newton-loop vector kernels
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(VB) k_residual(const double* __restrict__ f_unit, double zeta,
                                                  const double* __restrict__ F, const uint8_t* __restrict__ free_dof,
                                                  double* __restrict__ r, float* __restrict__ r32, int64_t n,
                                                  double* part, int nparts) {
    __shared__ double sh[32];
    double s_r = 0.0, s_f = 0.0, s_F = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double fi = f_unit ? zeta * f_unit[i] : 0.0;
        const double Fi = F[i];
        const bool fr = free_dof[i] != 0;
        const double ri = fr ? fi - Fi : 0.0;
        r[i] = ri;
        if (r32) r32[i] = (float)ri;
        s_r += ri * ri;
        s_f += fr ? fi * fi : 0.0;
        s_F += Fi * Fi;
    }
    const double a = block_sum(s_r, sh);
    const double b = block_sum(s_f, sh);
    const double c = block_sum(s_F, sh);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = a;
        part[nparts + blockIdx.x] = b;
        part[2 * nparts + blockIdx.x] = c;
    }
}

// Per-chunk sums of r^2, (zeta f)^2 on free DOFs and F^2 over DOF chunks [beg, end) (one CTA per
// chunk; chunks never straddle two problems of a batch).  chunks = [problem | begin | end][nc].
__global__ void __launch_bounds__(VB) k_chunk_norms(const double* __restrict__ f_unit, double zeta,
                                                     const double* __restrict__ F, const uint8_t* __restrict__ free_dof,
                                                     const double* __restrict__ r, const int64_t* __restrict__ chunks,
                                                     int64_t nc, double* __restrict__ out) {
    __shared__ double sh[32];
    const int64_t c = blockIdx.x;
    const int64_t beg = chunks[nc + c], end = chunks[2 * nc + c];
    double s_r = 0.0, s_f = 0.0, s_F = 0.0;
    for (int64_t i = beg + threadIdx.x; i < end; i += blockDim.x) {
        const double fi = f_unit ? zeta * f_unit[i] : 0.0;
        s_r += r[i] * r[i];
        s_f += free_dof[i] ? fi * fi : 0.0;
        s_F += F[i] * F[i];
    }
    const double a = block_sum(s_r, sh);
    const double b = block_sum(s_f, sh);
    const double d = block_sum(s_F, sh);
    if (threadIdx.x == 0) {
        out[c] = a;
        out[nc + c] = b;
        out[2 * nc + c] = d;
    }
}

cudaError_t vec_chunk_norms(const double* f_unit, double zeta, const double* F, const uint8_t* free_dof,
                            const double* r, const int64_t* chunks, int64_t nc, double* out, cudaStream_t s) {
    if (nc <= 0) return cudaSuccess;
    k_chunk_norms<<<(unsigned)nc, VB, 0, s>>>(f_unit, zeta, F, free_dof, r, chunks, nc, out);
    return cudaGetLastError();
}

__global__ void k_finalize3(const double* part, int nparts, double* out3) {
    __shared__ double sh[32];
    for (int k = 0; k < 3; ++k) {
        const double v = sum_partials(part + (int64_t)k * nparts, nparts, sh);
        if (threadIdx.x == 0) out3[k] = v;
    }
}

cudaError_t vec_residual(const double* f_unit, double zeta, const double* F, const uint8_t* free_dof, double* r,
                         float* r32, int64_t n, double* part, int nparts, double* out3, cudaStream_t s) {
    k_residual<<<nparts, VB, 0, s>>>(f_unit, zeta, F, free_dof, r, r32, n, part, nparts);
    k_finalize3<<<1, 32, 0, s>>>(part, nparts, out3);
    return cudaGetLastError();
}

__global__ void k_axpy(double* y, double a, const double* x, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] += a * x[i];
}

__global__ void k_set_dirichlet(double* u, const double* uD, double zeta, const uint8_t* free_dof, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (!free_dof[i]) u[i] = uD ? zeta * uD[i] : 0.0;
}

__global__ void k_extrapolate(double* u, const double* u_prev, double ratio, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        u[i] += ratio * (u[i] - u_prev[i]);
}

__global__ void k_axpy_f32(double* __restrict__ y, const float* __restrict__ x, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] += (double)x[i];
}

template <class TI, class TO>
__global__ void k_convert(const TI* __restrict__ x, TO* __restrict__ y, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = (TO)x[i];
}

__global__ void k_mask_copy(double* dst, const double* src, const uint8_t* free_dof, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = free_dof[i] ? src[i] : 0.0;
}

static unsigned vgrid(int64_t n) {
    int64_t g = (n + VB - 1) / VB;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, 4096));
}

cudaError_t vec_axpy(double* y, double a, const double* x, int64_t n, cudaStream_t s) {
    k_axpy<<<vgrid(n), VB, 0, s>>>(y, a, x, n);
    return cudaGetLastError();
}
cudaError_t vec_set_dirichlet(double* u, const double* uD_unit, double zeta, const uint8_t* free_dof, int64_t n,
                              cudaStream_t s) {
    k_set_dirichlet<<<vgrid(n), VB, 0, s>>>(u, uD_unit, zeta, free_dof, n);
    return cudaGetLastError();
}
cudaError_t vec_extrapolate(double* u, const double* u_prev, double ratio, int64_t n, cudaStream_t s) {
    k_extrapolate<<<vgrid(n), VB, 0, s>>>(u, u_prev, ratio, n);
    return cudaGetLastError();
}
cudaError_t vec_axpy_f32(double* y, const float* x, int64_t n, cudaStream_t s) {
    k_axpy_f32<<<vgrid(n), VB, 0, s>>>(y, x, n);
    return cudaGetLastError();
}
cudaError_t vec_cvt_f32(const double* x, float* y, int64_t n, cudaStream_t s) {
    k_convert<double, float><<<vgrid(n), VB, 0, s>>>(x, y, n);
    return cudaGetLastError();
}
cudaError_t vec_cvt_f64(const float* x, double* y, int64_t n, cudaStream_t s) {
    k_convert<float, double><<<vgrid(n), VB, 0, s>>>(x, y, n);
    return cudaGetLastError();
}
cudaError_t vec_mask_copy(double* dst, const double* src, const uint8_t* free_dof, int64_t n, cudaStream_t s) {
    k_mask_copy<<<vgrid(n), VB, 0, s>>>(dst, src, free_dof, n);
    return cudaGetLastError();
}

}  // namespace ep
