// Fused hot-path kernels, templated on the element type and the material model.
//
//  k_geometry : per point J = sum_p dPhi^_p (x) x_p, det J, J^-1, physical
//               gradients DPhi and WEIGHT = |det J| w_q (Section 6.1, eqs.
//               (Jacobian), (Jacobian2), (basis_derivative); Section 6.3).
//               Run once per mesh; the results are cached in HBM.
//  k_assemble : per Newton iteration.  One CTA owns EPC consecutive elements:
//               (0) stage the elements' displacements, gradients and weights
//                   in shared memory (contiguous, coalesced copies);
//               (1a) one thread per point: strain eps = sum_p G_p u_p
//                   (eq. (local_strain-displ)), return mapping (Section 2),
//                   w*sigma and w*D (D = T^o, or T^o - C in split mode) to
//                   shared memory;
//               (1b) one thread per (point, node): H_p = (w D) G_p;
//               (2a) one thread per (element, node): F_p = sum_q G_p^T (w sigma)_q,
//                   scattered with FP64 atomics (Section 7, F = B^T(W S));
//               (2b) one thread per (element, node pair): K_pq = sum_q G_p^T H_q,
//                   scattered into the fixed block-CSR slots through the
//                   element-to-slot map (Section 7: K_tangent; eq. (K-split)
//                   adds only plastic points to the cached K_elast).
//  k_commit   : after Newton has converged, the return mapping once more at
//               every point; the trial internal variables become the state of
//               step k (Sections 2.2, 2.3, eq. (T_other)).
#pragma once

#include <algorithm>

#include "constitutive.cuh"

namespace ep {

constexpr int ASM_THREADS = 256;

// TILE: 1 = the element type's tile of EPC elements per CTA; 2 = half that tile (half the shared
// memory per CTA, so more CTAs per SM) -- the two assembly schedules the autotuner chooses from.
template <int ID, class KT, int TILE = 1>
struct AsmShape {
    using ET = Elem<ID>;
    static constexpr int D = ET::DIM, NP = ET::NP, NQ = ET::NQ, NS = ET::NS, NA = ET::NA;
    static constexpr int EPC = (ET::EPC / TILE) > 0 ? ET::EPC / TILE : 1;
    static constexpr int NIP = EPC * NQ;
    static constexpr bool F32 = sizeof(KT) == 4;
    // FP64 region: displacements, gradients, weights, w*sigma
    static constexpr int OFF_U = 0;
    static constexpr int OFF_G = OFF_U + EPC * NP * D;
    static constexpr int OFF_W = OFF_G + NIP * NP * D;
    static constexpr int OFF_WS = OFF_W + NIP;
    static constexpr int N_DBL = OFF_WS + NIP * NS;
    // tangent region (KT): w*D, H, and an FP32 copy of the gradients when KT is float
    static constexpr int OFF_D = 0;
    static constexpr int OFF_H = OFF_D + NIP * NS * NS;
    static constexpr int OFF_GK = OFF_H + NIP * NP * NS * D;
    static constexpr int N_KT = OFF_GK + (F32 ? NIP * NP * D : 0);
    static constexpr size_t BYTES_KT = (sizeof(KT) * N_KT + 7) / 8 * 8;
    static constexpr size_t SMEM = sizeof(double) * N_DBL + BYTES_KT + sizeof(int) * (EPC * NP + 2 * EPC + NIP);
};

// Load the stored state of one point into active components.
// Stored layout: 3D (11,22,33,12,23,13); plane strain (11,22,12,33).
template <int NA>
__device__ __forceinline__ int stored_row(int a) {
    // active (11,22,33,12) -> stored (11,22,12,33) in plane strain
    return NA == 4 ? (a == 2 ? 3 : (a == 3 ? 2 : a)) : a;
}

template <int NA, int MODEL>
__device__ __forceinline__ void load_state(const StateDev& st, int64_t n_int, int64_t ip, PointIn<NA>& in) {
#pragma unroll
    for (int a = 0; a < NA; ++a) in.ep[a] = st.ep[(int64_t)stored_row<NA>(a) * n_int + ip];
    in.alpha = 0.0;
#pragma unroll
    for (int a = 0; a < NA; ++a) in.beta[a] = 0.0;
    if (MODEL == 2 || MODEL == 3) in.alpha = st.hard[ip];
    if (MODEL == 1) {
#pragma unroll
        for (int a = 0; a < NA; ++a) in.beta[a] = st.hard[(int64_t)stored_row<NA>(a) * n_int + ip];
    }
}

// eps (active, strain-type) from gradients g[p][D] and displacements u[p][D]
template <int D, int NP, int NA>
__device__ __forceinline__ void strain_at(const double* __restrict__ g, const double* __restrict__ u, double (&eps)[NA]) {
#pragma unroll
    for (int a = 0; a < NA; ++a) eps[a] = 0.0;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const double* gp = g + p * D;
        const double* up = u + p * D;
        if (D == 2) {
            eps[0] += gp[0] * up[0];
            eps[1] += gp[1] * up[1];
            eps[3] += gp[1] * up[0] + gp[0] * up[1];
        } else {
            eps[0] += gp[0] * up[0];
            eps[1] += gp[1] * up[1];
            eps[2] += gp[2] * up[2];
            eps[3] += gp[1] * up[0] + gp[0] * up[1];
            eps[4] += gp[2] * up[1] + gp[1] * up[2];
            eps[5] += gp[2] * up[0] + gp[0] * up[2];
        }
    }
}

// ---------------------------------------------------------------------------
// KT is the value type of the tangent: double (the FP64 path) or float (the
// mixed path: strains, return mapping and F stay FP64, and the FP64 tangent
// coefficients are rounded once to FP32 before D, H and the K blocks are
// formed and scattered with FP32 atomics).
template <int ID, int MODEL, bool DELTA, bool WANT_F, class KT, int TILE>
__global__ void __launch_bounds__(ASM_THREADS) k_assemble(AsmArgs a) {
    using S = AsmShape<ID, KT, TILE>;
    constexpr int D = S::D, NP = S::NP, NQ = S::NQ, NS = S::NS, NA = S::NA, EPC = S::EPC;
    constexpr bool SYM = (MODEL != 3);
    constexpr int NB = SYM ? NP * (NP + 1) / 2 : NP * NP;
    extern __shared__ __align__(16) double smem[];
    double* s_u = smem + S::OFF_U;     // [EPC][NP][D]
    double* s_g = smem + S::OFF_G;     // [NIP][NP][D]
    double* s_w = smem + S::OFF_W;     // [NIP]
    double* s_ws = smem + S::OFF_WS;   // [NIP][NS]      (w * sigma)
    KT* s_kt = reinterpret_cast<KT*>(smem + S::N_DBL);
    KT* s_D = s_kt + S::OFF_D;         // [NIP][NS][NS]  (w * D)
    KT* s_H = s_kt + S::OFF_H;         // [NIP][NP][NS][D]
    const KT* s_gk = S::F32 ? s_kt + S::OFF_GK : reinterpret_cast<const KT*>(s_g);   // gradients in KT
    int* s_node = reinterpret_cast<int*>(reinterpret_cast<char*>(s_kt) + S::BYTES_KT);   // [EPC][NP]
    int* s_eplast = s_node + EPC * NP;                        // [EPC]
    int* s_ipflag = s_eplast + EPC;                           // [NIP]
    int* s_eid = s_ipflag + S::NIP;                           // [EPC] global element ids
    KT* Kout = S::F32 ? reinterpret_cast<KT*>(a.Kvals32) : reinterpret_cast<KT*>(a.Kvals);

    const int tid = threadIdx.x;
    const int64_t n_int = a.mesh.n_int;
    const bool listed = a.elem_list != nullptr;   // deterministic form: one colour, plain stores
    const int64_t n_elem = listed ? a.list_n : a.mesh.n_elem;
    const int64_t n_tiles = (n_elem + EPC - 1) / EPC;
    // persistent: the CTAs of one resident wave take the (problem, element-tile) items of the
    // concatenated element array in turn (a batch of problems is one such array)
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t e0 = tile * EPC;
    const int ne = (int)min((int64_t)EPC, n_elem - e0);
    const int nip = ne * NQ;
    const int64_t ip0 = e0 * NQ;

    // (0) stage connectivity, gradients, weights and displacements
    for (int i = tid; i < EPC; i += ASM_THREADS) {
        s_eplast[i] = 0;
        s_eid[i] = listed ? (i < ne ? a.elem_list[e0 + i] : 0) : (int)(e0 + i);
    }
    if (listed) __syncthreads();
    if (!listed) {
        for (int i = tid; i < ne * NP; i += ASM_THREADS) s_node[i] = a.mesh.elem_nodes[e0 * NP + i];
        const double* src = a.mesh.dphi + ip0 * (NP * D);
        for (int i = tid; i < nip * NP * D; i += ASM_THREADS) {
            const double g = src[i];
            s_g[i] = g;
            if (S::F32) const_cast<KT*>(s_gk)[i] = (KT)g;
        }
        for (int i = tid; i < nip; i += ASM_THREADS) s_w[i] = a.mesh.wgt[ip0 + i];
    } else {
        // elements of one colour: each element's connectivity, gradients and weights are contiguous
        for (int i = tid; i < ne * NP; i += ASM_THREADS)
            s_node[i] = a.mesh.elem_nodes[(int64_t)s_eid[i / NP] * NP + i % NP];
        constexpr int PER = NQ * NP * D;
        for (int i = tid; i < nip * NP * D; i += ASM_THREADS) {
            const double g = a.mesh.dphi[(int64_t)s_eid[i / PER] * PER + i % PER];
            s_g[i] = g;
            if (S::F32) const_cast<KT*>(s_gk)[i] = (KT)g;
        }
        for (int i = tid; i < nip; i += ASM_THREADS) s_w[i] = a.mesh.wgt[(int64_t)s_eid[i / NQ] * NQ + i % NQ];
    }
    __syncthreads();
    if (MODEL != 0 || WANT_F) {
        for (int i = tid; i < ne * NP * D; i += ASM_THREADS) {
            const int c = i % D, ep = i / D;
            s_u[i] = a.u[(int64_t)s_node[ep] * D + c];
        }
    }
    __syncthreads();

    // (1a) one thread per integration point
    unsigned my_plastic = 0;
    for (int j = tid; j < nip; j += ASM_THREADS) {
        const int e = j / NQ;
        const int64_t ip = (int64_t)s_eid[e] * NQ + j % NQ;
        const double w = s_w[j];
        const MatConst& mat = elem_material(a.mesh, s_eid[e]);
        PointOut<NA> o;
        if (MODEL == 0 && !WANT_F) {
            PointIn<NA> in;
#pragma unroll
            for (int c = 0; c < NA; ++c) { in.eps[c] = 0.0; in.ep[c] = 0.0; in.beta[c] = 0.0; }
            in.alpha = 0.0;
            return_map<NA, 0>(mat, in, o);
        } else {
            PointIn<NA> in;
            strain_at<D, NP, NA>(s_g + j * NP * D, s_u + e * NP * D, in.eps);
            load_state<NA, MODEL>(a.state, n_int, ip, in);
            return_map<NA, MODEL>(mat, in, o);
            if (o.err && a.err_flag) atomicOr(a.err_flag, 1);
        }
        const int plastic = (o.flag != 0);
        my_plastic += plastic;
        s_ipflag[j] = plastic;
        if (plastic) s_eplast[e] = 1;
        if (WANT_F) {
#pragma unroll
            for (int r = 0; r < NS; ++r) s_ws[j * NS + r] = w * o.sig[row_active<NS>(r)];
        }
        // split mode: an elastic point adds nothing (D - C = 0), its tangent is not formed
        if (DELTA && !plastic) continue;
        if (DELTA) { o.cV -= mat.K; o.cD -= 2.0 * mat.G; }
        if (S::F32) {
            // the tangent from FP64 coefficients rounded once to FP32
            PointTan<NA, KT> t;
            tangent_coeffs(o, (KT)w, t);
#pragma unroll
            for (int r = 0; r < NS; ++r)
#pragma unroll
                for (int c = 0; c < NS; ++c) s_D[(j * NS + r) * NS + c] = tangent_entry_t<NS, NA>(t, r, c);
        } else {
#pragma unroll
            for (int r = 0; r < NS; ++r)
#pragma unroll
                for (int c = 0; c < NS; ++c) s_D[(j * NS + r) * NS + c] = (KT)(w * tangent_entry<NS, NA>(o, r, c));
        }
    }
    if (a.n_plastic) {
        // warp-aggregated count
        unsigned v = my_plastic;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if ((tid & 31) == 0 && v) atomicAdd(a.n_plastic, (unsigned long long)v);
    }
    __syncthreads();
    if (a.n_plastic_elem && tid < 32) {
        unsigned v = 0;
        for (int e = tid; e < ne; e += 32) v += s_eplast[e] ? 1u : 0u;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if (tid == 0 && v) atomicAdd(a.n_plastic_elem, (unsigned long long)v);
    }

    // (1b) H_p = (w D) G_p, one thread per (point, node)
    if (a.want_K) {
        for (int t = tid; t < nip * NP; t += ASM_THREADS) {
            const int j = t / NP, p = t % NP;
            KT* H = s_H + (j * NP + p) * NS * D;
            if (DELTA && !s_ipflag[j]) {
#pragma unroll
                for (int i = 0; i < NS * D; ++i) H[i] = KT(0);
                continue;
            }
            const KT* g = s_gk + (j * NP + p) * D;
            const KT* Dm = s_D + j * NS * NS;
#pragma unroll
            for (int r = 0; r < NS; ++r) {
                const KT* dr = Dm + r * NS;
                if (D == 2) {
                    H[r * 2 + 0] = dr[0] * g[0] + dr[2] * g[1];
                    H[r * 2 + 1] = dr[1] * g[1] + dr[2] * g[0];
                } else {
                    H[r * 3 + 0] = dr[0] * g[0] + dr[3] * g[1] + dr[5] * g[2];
                    H[r * 3 + 1] = dr[1] * g[1] + dr[3] * g[0] + dr[4] * g[2];
                    H[r * 3 + 2] = dr[2] * g[2] + dr[4] * g[1] + dr[5] * g[0];
                }
            }
        }
    }
    __syncthreads();

    // (2a) internal forces (FP64), one thread per (element, node)
    if (WANT_F) {
        for (int t = tid; t < ne * NP; t += ASM_THREADS) {
            const int e = t / NP, p = t % NP;
            double f[D];
#pragma unroll
            for (int c = 0; c < D; ++c) f[c] = 0.0;
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const int j = e * NQ + q;
                const double* g = s_g + (j * NP + p) * D;
                const double* ws = s_ws + j * NS;
                if (D == 2) {
                    f[0] += g[0] * ws[0] + g[1] * ws[2];
                    f[1] += g[1] * ws[1] + g[0] * ws[2];
                } else {
                    f[0] += g[0] * ws[0] + g[1] * ws[3] + g[2] * ws[5];
                    f[1] += g[1] * ws[1] + g[0] * ws[3] + g[2] * ws[4];
                    f[2] += g[2] * ws[2] + g[1] * ws[4] + g[0] * ws[5];
                }
            }
            const int64_t node = s_node[t];
            if (listed) {   // one colour: this element is the node's only contributor in the launch
#pragma unroll
                for (int c = 0; c < D; ++c) a.F[node * D + c] += f[c];
            } else {
#pragma unroll
                for (int c = 0; c < D; ++c) atomicAdd(a.F + node * D + c, f[c]);
            }
        }
    }
    // (2b) element blocks K_pq, one thread per (element, node pair)
    for (int t = tid; t < (a.want_K ? ne * NB : 0); t += ASM_THREADS) {
        const int e = t / NB, b = t % NB;
        if (DELTA && !s_eplast[e]) continue;
        int p, q;
        if (SYM) {
            // b -> (p, q), p <= q, row-wise enumeration
            p = 0;
            int rem = b;
            while (rem >= NP - p) { rem -= NP - p; ++p; }
            q = p + rem;
        } else {
            p = b / NP;
            q = b % NP;
        }
        KT k[D][D];
#pragma unroll
        for (int r = 0; r < D; ++r)
#pragma unroll
            for (int c = 0; c < D; ++c) k[r][c] = KT(0);
#pragma unroll
        for (int qq = 0; qq < NQ; ++qq) {
            const int j = e * NQ + qq;
            const KT* g = s_gk + (j * NP + p) * D;
            const KT* H = s_H + (j * NP + q) * NS * D;
#pragma unroll
            for (int c = 0; c < D; ++c) {
                if (D == 2) {
                    k[0][c] += g[0] * H[0 * 2 + c] + g[1] * H[2 * 2 + c];
                    k[1][c] += g[1] * H[1 * 2 + c] + g[0] * H[2 * 2 + c];
                } else {
                    k[0][c] += g[0] * H[0 * 3 + c] + g[1] * H[3 * 3 + c] + g[2] * H[5 * 3 + c];
                    k[1][c] += g[1] * H[1 * 3 + c] + g[0] * H[3 * 3 + c] + g[2] * H[4 * 3 + c];
                    k[2][c] += g[2] * H[2 * 3 + c] + g[1] * H[4 * 3 + c] + g[0] * H[5 * 3 + c];
                }
            }
        }
        const int64_t eg = s_eid[e];
        const int64_t slot = a.mesh.slots[eg * (NP * NP) + p * NP + q];
        KT* dst = Kout + slot * (D * D);
        // split mode: these slots now differ from K_elast; the next split assembly resets them
        if (DELTA && a.dirty) a.dirty[slot] = 1;
        if (listed) {   // one colour: no other element of the launch owns this node pair
#pragma unroll
            for (int r = 0; r < D; ++r)
#pragma unroll
                for (int c = 0; c < D; ++c) dst[r * D + c] += k[r][c];
        } else {
#pragma unroll
            for (int r = 0; r < D; ++r)
#pragma unroll
                for (int c = 0; c < D; ++c) atomicAdd(dst + r * D + c, k[r][c]);
        }
        if (SYM && p != q) {
            const int64_t slot2 = a.mesh.slots[eg * (NP * NP) + q * NP + p];
            if (DELTA && a.dirty) a.dirty[slot2] = 1;
            KT* dst2 = Kout + slot2 * (D * D);
            if (listed) {
#pragma unroll
                for (int r = 0; r < D; ++r)
#pragma unroll
                    for (int c = 0; c < D; ++c) dst2[c * D + r] += k[r][c];
            } else {
#pragma unroll
                for (int r = 0; r < D; ++r)
#pragma unroll
                    for (int c = 0; c < D; ++c) atomicAdd(dst2 + c * D + r, k[r][c]);
            }
        }
    }
    __syncthreads();   // the next tile reuses the shared buffers
    }   // tile
}

// ---------------------------------------------------------------------------
template <int ID, int MODEL>
__global__ void __launch_bounds__(256) k_commit(CommitArgs a) {
    using ET = Elem<ID>;
    constexpr int D = ET::DIM, NP = ET::NP, NQ = ET::NQ, NA = ET::NA;
    const int64_t n_int = a.mesh.n_int;
    const int64_t ip = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned plastic = 0;
    if (ip < n_int) {
        const int64_t e = ip / NQ;
        double u[NP * D];
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            const int64_t node = a.mesh.elem_nodes[e * NP + p];
#pragma unroll
            for (int c = 0; c < D; ++c) u[p * D + c] = a.u[node * D + c];
        }
        double g[NP * D];
        const double* src = a.mesh.dphi + ip * (NP * D);
#pragma unroll
        for (int i = 0; i < NP * D; ++i) g[i] = src[i];
        PointIn<NA> in;
        strain_at<D, NP, NA>(g, u, in.eps);
        load_state<NA, MODEL>(a.state, n_int, ip, in);
        PointOut<NA> o;
        return_map<NA, MODEL>(elem_material(a.mesh, e), in, o);
        if (o.err && a.err_flag) atomicOr(a.err_flag, 1);
#pragma unroll
        for (int c = 0; c < NA; ++c) {
            const int64_t row = (int64_t)stored_row<NA>(c) * n_int + ip;
            a.state.ep[row] = o.ep[c];
            a.state.sig[row] = o.sig[c];
            if (MODEL == 1) a.state.hard[row] = o.beta[c];
        }
        if (MODEL == 2 || MODEL == 3) a.state.hard[ip] = o.alpha;
        a.state.flag[ip] = (uint8_t)(o.err ? 255 : o.flag);
        plastic = (o.flag != 0);
    }
    if (a.n_plastic) {
        unsigned v = plastic;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if ((threadIdx.x & 31) == 0 && v) atomicAdd(a.n_plastic, (unsigned long long)v);
    }
}

// ---------------------------------------------------------------------------
template <int ID>
__global__ void __launch_bounds__(256) k_geometry(GeomArgs a) {
    using ET = Elem<ID>;
    constexpr int D = ET::DIM, NP = ET::NP, NQ = ET::NQ;
    const int64_t ip = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (ip >= a.n_int) return;
    const int64_t e = ip / NQ;
    const int q = (int)(ip % NQ);
    const double* dh = a.dhat + (int64_t)q * NP * D;   // [p][i]
    double J[D][D];
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) J[i][j] = 0.0;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const int64_t node = a.elem_nodes[e * NP + p];
#pragma unroll
        for (int j = 0; j < D; ++j) {
            const double x = a.coords[node * D + j];
#pragma unroll
            for (int i = 0; i < D; ++i) J[i][j] += dh[p * D + i] * x;
        }
    }
    double det, Ji[D][D];
    if (D == 2) {
        det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        const double id = 1.0 / det;
        Ji[0][0] = J[1][1] * id;  Ji[0][1] = -J[0][1] * id;
        Ji[1][0] = -J[1][0] * id; Ji[1][1] = J[0][0] * id;
    } else {
        const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
        const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
        const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
        det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
        const double id = 1.0 / det;
        Ji[0][0] = c00 * id;
        Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * id;
        Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * id;
        Ji[1][0] = c01 * id;
        Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * id;
        Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * id;
        Ji[2][0] = c02 * id;
        Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * id;
        Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * id;
    }
    if (!(det > 0.0)) atomicAdd(a.bad_count, 1);
    double* dst = a.dphi + ip * (NP * D);
#pragma unroll
    for (int p = 0; p < NP; ++p)
#pragma unroll
        for (int i = 0; i < D; ++i) {
            double s = 0.0;
#pragma unroll
            for (int j = 0; j < D; ++j) s += Ji[i][j] * dh[p * D + j];
            dst[p * D + i] = s;
        }
    a.wgt[ip] = fabs(det) * a.wq[q];
}

// ---------------------------------------------------------------------------
// Split-mode reset (eq. (K-split)): blocks moved away from K_elast by the last split assembly get
// K_elast's values back; one thread per block, the mark cleared as it is read.
template <class T>
__global__ void __launch_bounds__(256) k_reset_dirty(uint8_t* __restrict__ dirty, int64_t nnzb, int d2,
                                                     const T* __restrict__ Kel, T* __restrict__ Kt) {
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nnzb; b += (int64_t)gridDim.x * blockDim.x) {
        if (!dirty[b]) continue;
        dirty[b] = 0;
        for (int i = 0; i < d2; ++i) Kt[b * d2 + i] = Kel[b * d2 + i];
    }
}

// ---------------------------------------------------------------------------
// Launchers for one element type.
// ---------------------------------------------------------------------------
template <int ID, int MODEL, bool DELTA, bool WANT_F, class KT, int TILE = 1>
cudaError_t launch_asm_t(const AsmArgs& a, cudaStream_t s) {
    using S = AsmShape<ID, KT, TILE>;
    auto kern = k_assemble<ID, MODEL, DELTA, WANT_F, KT, TILE>;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const int64_t n = a.elem_list ? a.list_n : a.mesh.n_elem;
    const int64_t tiles = (n + S::EPC - 1) / S::EPC;
    if (tiles == 0) return cudaSuccess;
    // one resident wave of CTAs (persistent over the tiles)
    static int wave = 0;
    if (wave == 0) {
        int occ = 0, sms = 0, dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, ASM_THREADS, S::SMEM) != cudaSuccess || occ < 1)
            occ = 1;
        wave = std::max(1, sms) * occ;
    }
    const int64_t grid = std::min<int64_t>(tiles, wave);
    kern<<<(unsigned)grid, ASM_THREADS, S::SMEM, s>>>(a);
    return cudaGetLastError();
}

template <int ID, int MODEL, class KT>
cudaError_t launch_asm_model(const AsmArgs& a, cudaStream_t s) {
    if (a.tile == 2)
        return a.mode == ASM_DELTA ? launch_asm_t<ID, MODEL, true, true, KT, 2>(a, s)
                                   : launch_asm_t<ID, MODEL, false, true, KT, 2>(a, s);
    return a.mode == ASM_DELTA ? launch_asm_t<ID, MODEL, true, true, KT>(a, s)
                               : launch_asm_t<ID, MODEL, false, true, KT>(a, s);
}

template <int ID, class KT>
cudaError_t launch_assemble_kt(const AsmArgs& a, cudaStream_t s) {
    switch (a.mat.model) {
        case 0: return launch_asm_model<ID, 0, KT>(a, s);
        case 1: return launch_asm_model<ID, 1, KT>(a, s);
        case 2: return launch_asm_model<ID, 2, KT>(a, s);
        case 3: return launch_asm_model<ID, 3, KT>(a, s);
    }
    return cudaErrorInvalidValue;
}

template <int ID>
cudaError_t launch_assemble_elem(const AsmArgs& a, cudaStream_t s) {
    if (a.elastic_only) return launch_asm_t<ID, 0, false, false, double>(a, s);
    if (a.Kvals32) return launch_assemble_kt<ID, float>(a, s);
    return launch_assemble_kt<ID, double>(a, s);
}

template <int ID>
cudaError_t launch_commit_elem(const CommitArgs& a, cudaStream_t s) {
    const int64_t grid = (a.mesh.n_int + 255) / 256;
    if (grid == 0) return cudaSuccess;
    switch (a.mat.model) {
        case 0: k_commit<ID, 0><<<(unsigned)grid, 256, 0, s>>>(a); break;
        case 1: k_commit<ID, 1><<<(unsigned)grid, 256, 0, s>>>(a); break;
        case 2: k_commit<ID, 2><<<(unsigned)grid, 256, 0, s>>>(a); break;
        case 3: k_commit<ID, 3><<<(unsigned)grid, 256, 0, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int ID>
cudaError_t launch_geometry_elem(const GeomArgs& a, cudaStream_t s) {
    const int64_t grid = (a.n_int + 255) / 256;
    if (grid == 0) return cudaSuccess;
    k_geometry<ID><<<(unsigned)grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace ep

// One translation unit per element type: asm_<type>.cu defines EP_TU_ELEM.
#define EP_DEFINE_ELEM_LAUNCHERS(ID)                                                                   \
    namespace ep {                                                                                     \
    cudaError_t launch_assemble_##ID(const AsmArgs& a, cudaStream_t s) { return launch_assemble_elem<ID>(a, s); } \
    cudaError_t launch_commit_##ID(const CommitArgs& a, cudaStream_t s) { return launch_commit_elem<ID>(a, s); }   \
    cudaError_t launch_geometry_##ID(const GeomArgs& a, cudaStream_t s) { return launch_geometry_elem<ID>(a, s); } \
    }
