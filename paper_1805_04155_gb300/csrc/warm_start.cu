// Learned warm start of the Newton iteration: the per-node network and the node features it reads.
//
// The network maps the 16 inputs of a node to 4 outputs through two hidden
// layers of 128 ReLU units (16 -> 128 -> 128 -> 4).  Weights are held as
// bfloat16 (rounded from FP32 master copies after every optimiser step);
// biases, activations and every sum are FP32.  The inputs are the node's last
// two displacement increments divided by the problem's RMS increment, the
// load-increment ratios, the plastic fraction of the adjacent integration
// points and material / boundary scalars; the outputs correct the extrapolated
// start (ALG-NEWTON's initial iterate, Section 4) and predict the node's
// plastic fraction.
//
// Kernels:
//   k_mlp<false>  forward pass of tiles of 64 rows (inference)
//   k_mlp<true>   forward + backward of the same tiles; every CTA keeps its
//                 weight-gradient partial sums in registers over its tiles and
//                 writes them once (deterministic, no atomics)
//   k_mlp_update  sums the CTA partials in a fixed order, then an Adam step
//                 (or only returns the gradient)
// One CTA of 256 threads per SM (149 KB of shared memory: the tile's inputs,
// both hidden activations and FP32 copies of the bfloat16 weights); each
// thread computes a 4 x 8 tile of the 128-wide layers, 12 shared loads per 32
// FMA.  The network is small next to a Newton iteration (about 1.9e4 FMA per
// row forward), so its layers run as FP32 FMA loops over shared memory rather
// than tensor-core tiles.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

#include "ep_internal.h"

namespace ep {
namespace {

constexpr int NIN = EP_WS_N_IN, NW = EP_WS_WIDTH, NOUT = EP_WS_N_OUT;
constexpr int OFF_W1 = 0;
constexpr int OFF_B1 = OFF_W1 + NW * NIN;
constexpr int OFF_W2 = OFF_B1 + NW;
constexpr int OFF_B2 = OFF_W2 + NW * NW;
constexpr int OFF_W3 = OFF_B2 + NW;
constexpr int OFF_B3 = OFF_W3 + NOUT * NW;
constexpr int NPAR = OFF_B3 + NOUT;
static_assert(NPAR == EP_WS_N_PARAMS, "parameter layout");
static_assert(NIN == 16 && NW == 128 && NOUT == 4, "the thread mapping below assumes 16 -> 128 -> 128 -> 4");

constexpr int TR = 64;          // rows per tile
constexpr int NT = 256;         // threads per CTA: 8 warps
constexpr int LX = NIN + 1;     // padded row strides in shared memory: odd strides put the 16 column
constexpr int LH = NW + 1;      // groups of a warp (consecutive rows or columns) in distinct banks
constexpr int LW1 = NIN + 1;
constexpr int LW = NW + 1;
constexpr int LY = NOUT + 1;
constexpr float LAMBDA_PL = 0.1f;
constexpr float ADAM_B1 = 0.9f, ADAM_B2 = 0.999f, ADAM_EPS = 1e-8f;

// Weights are kept in shared memory as FP32 copies of their bfloat16 values (exact), so the inner
// loops are one load per operand and no conversions.
struct MlpSmem {
    double red[NT / 32];
    float X[TR * LX];
    float H1[TR * LH];
    float H2[TR * LH];
    float Y[TR * LY];           // outputs, then their loss gradients
    float b1[NW], b2[NW], b3[NOUT];
    float W1[NW * LW1], W2[NW * LW], W3[NOUT * LW];
};

// Thread mapping: cg = t % 16, rg = t / 16 (two row groups per warp: loads indexed by rg are broadcasts,
// loads indexed by cg hit 16 distinct banks through the odd strides).
//   activations (r, j) of the 128-wide layers: r = rg + 16 a (a < 4), j = cg + 16 b (b < 8): 4 x 8 tile
//   dW2 (j, i): j = cg + 16 b (b < 8), i = rg + 16 a (a < 8); dW1 (j, i): j = cg + 16 b, i = rg
//   layer 3 and dY (r, o): r = t / 4, o = t % 4; dW3 entry e = t + 256 q (q < 2): o = e / 128, i = e % 128
template <bool TRAIN>
__global__ void __launch_bounds__(NT, 1)
    k_mlp(const float* __restrict__ X, const float* __restrict__ T, int64_t n, float inv_n, const float* __restrict__ p,
          const __nv_bfloat16* __restrict__ pb, float* __restrict__ Y, float* __restrict__ gpart,
          double* __restrict__ lpart) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    MlpSmem& S = *reinterpret_cast<MlpSmem*>(smem_raw);
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int cg = t & 15, rg = t >> 4;
    for (int i = t; i < NW * NIN; i += NT) S.W1[(i / NIN) * LW1 + i % NIN] = __bfloat162float(pb[OFF_W1 + i]);
    for (int i = t; i < NW * NW; i += NT) S.W2[(i / NW) * LW + i % NW] = __bfloat162float(pb[OFF_W2 + i]);
    for (int i = t; i < NOUT * NW; i += NT) S.W3[(i / NW) * LW + i % NW] = __bfloat162float(pb[OFF_W3 + i]);
    if (t < NW) {
        S.b1[t] = p[OFF_B1 + t];
        S.b2[t] = p[OFF_B2 + t];
    }
    if (t < NOUT) S.b3[t] = p[OFF_B3 + t];

    float g2[8][8], g1[8], g3[2], gb1[8], gb2[8];
    float gb3 = 0.f;
    double lsum = 0.0;
    if (TRAIN) {
#pragma unroll
        for (int b = 0; b < 8; ++b) {
#pragma unroll
            for (int a = 0; a < 8; ++a) g2[b][a] = 0.f;
            g1[b] = gb1[b] = gb2[b] = 0.f;
        }
        g3[0] = g3[1] = 0.f;
    }

    const int64_t n_tiles = (n + TR - 1) / TR;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int64_t row0 = tile * TR;
        __syncthreads();   // weights loaded; the previous tile is done with the buffers
        for (int i = t; i < TR * NIN; i += NT) {
            const int r = i / NIN, c = i % NIN;
            const int64_t row = row0 + r;
            S.X[r * LX + c] = row < n ? X[row * NIN + c] : 0.f;
        }
        __syncthreads();
        // layer 1: H1 = relu(X W1^T + b1)
        {
            float acc[4][8];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
#pragma unroll 4
            for (int i = 0; i < NIN; ++i) {
                float xv[4], wv[8];
#pragma unroll
                for (int a = 0; a < 4; ++a) xv[a] = S.X[(rg + 16 * a) * LX + i];
#pragma unroll
                for (int b = 0; b < 8; ++b) wv[b] = S.W1[(cg + 16 * b) * LW1 + i];
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(wv[b], xv[a], acc[a][b]);
            }
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 8; ++b) {
                    const int j = cg + 16 * b;
                    S.H1[(rg + 16 * a) * LH + j] = fmaxf(acc[a][b] + S.b1[j], 0.f);
                }
        }
        __syncthreads();
        // layer 2: H2 = relu(H1 W2^T + b2)
        {
            float acc[4][8];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
#pragma unroll 2
            for (int i = 0; i < NW; ++i) {
                float hv[4], wv[8];
#pragma unroll
                for (int a = 0; a < 4; ++a) hv[a] = S.H1[(rg + 16 * a) * LH + i];
#pragma unroll
                for (int b = 0; b < 8; ++b) wv[b] = S.W2[(cg + 16 * b) * LW + i];
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(wv[b], hv[a], acc[a][b]);
            }
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 8; ++b) {
                    const int j = cg + 16 * b;
                    S.H2[(rg + 16 * a) * LH + j] = fmaxf(acc[a][b] + S.b2[j], 0.f);
                }
        }
        __syncthreads();
        // layer 3: Y = H2 W3^T + b3, one output per thread; in training, the loss and dL/dY
        {
            const int r = t >> 2, o = t & 3;
            float acc = 0.f;
#pragma unroll 8
            for (int i = 0; i < NW; ++i) acc = fmaf(S.W3[o * LW + i], S.H2[r * LH + i], acc);
            const float y = acc + S.b3[o];
            const int64_t row = row0 + r;
            if (!TRAIN) {
                if (row < n) Y[row * NOUT + o] = y;
            } else {
                float dy = 0.f;
                if (row < n) {
                    const float tv = T[row * NOUT + o];
                    if (o < 3) {
                        const float d = y - tv;
                        lsum += (double)d * (double)d;
                        dy = 2.f * d * inv_n;
                    } else {
                        lsum += (double)LAMBDA_PL * (double)(fmaxf(y, 0.f) - y * tv + log1pf(expf(-fabsf(y))));
                        dy = LAMBDA_PL * (1.f / (1.f + expf(-y)) - tv) * inv_n;
                    }
                }
                S.Y[r * LY + o] = dy;
            }
        }
        if (!TRAIN) continue;
        __syncthreads();
        // dW3 += dY^T H2, db3 += sum dY
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int e = t + NT * q, o = e >> 7, i = e & (NW - 1);
            float acc = 0.f;
            for (int r = 0; r < TR; ++r) acc = fmaf(S.Y[r * LY + o], S.H2[r * LH + i], acc);
            g3[q] += acc;
        }
        if (t < NOUT) {
            float acc = 0.f;
            for (int r = 0; r < TR; ++r) acc += S.Y[r * LY + t];
            gb3 += acc;
        }
        __syncthreads();
        // dH2 = (dY W3) * [H2 > 0], in place of H2 (each thread reads and writes only its own entries)
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int r = rg + 16 * a;
            float dy[NOUT];
#pragma unroll
            for (int o = 0; o < NOUT; ++o) dy[o] = S.Y[r * LY + o];
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                const int i = cg + 16 * b;
                float v = 0.f;
#pragma unroll
                for (int o = 0; o < NOUT; ++o) v = fmaf(dy[o], S.W3[o * LW + i], v);
                const float h = S.H2[r * LH + i];
                S.H2[r * LH + i] = h > 0.f ? v : 0.f;
            }
        }
        __syncthreads();
        // dW2 += dH2^T H1 (rg = 0 threads also sum db2 over the rows)
        for (int r = 0; r < TR; ++r) {
            float dh[8], hv[8];
#pragma unroll
            for (int b = 0; b < 8; ++b) dh[b] = S.H2[r * LH + cg + 16 * b];
#pragma unroll
            for (int a = 0; a < 8; ++a) hv[a] = S.H1[r * LH + rg + 16 * a];
#pragma unroll
            for (int b = 0; b < 8; ++b)
#pragma unroll
                for (int a = 0; a < 8; ++a) g2[b][a] = fmaf(dh[b], hv[a], g2[b][a]);
            if (rg == 0) {
#pragma unroll
                for (int b = 0; b < 8; ++b) gb2[b] += dh[b];
            }
        }
        __syncthreads();
        // dH1 = (dH2 W2) * [H1 > 0], in place of H1
        {
            float acc[4][8];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
#pragma unroll 2
            for (int j = 0; j < NW; ++j) {
                float dv[4], wv[8];
#pragma unroll
                for (int a = 0; a < 4; ++a) dv[a] = S.H2[(rg + 16 * a) * LH + j];
#pragma unroll
                for (int b = 0; b < 8; ++b) wv[b] = S.W2[j * LW + cg + 16 * b];
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(dv[a], wv[b], acc[a][b]);
            }
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 8; ++b) {
                    const int idx = (rg + 16 * a) * LH + cg + 16 * b;
                    S.H1[idx] = S.H1[idx] > 0.f ? acc[a][b] : 0.f;
                }
        }
        __syncthreads();
        // dW1 += dH1^T X (rg = 0 threads also sum db1)
        for (int r = 0; r < TR; ++r) {
            const float xv = S.X[r * LX + rg];
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                const float dh = S.H1[r * LH + cg + 16 * b];
                g1[b] = fmaf(dh, xv, g1[b]);
                if (rg == 0) gb1[b] += dh;
            }
        }
    }
    if (!TRAIN) return;
    float* gp = gpart + (size_t)blockIdx.x * NPAR;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const int j = cg + 16 * b;
        gp[OFF_W1 + j * NIN + rg] = g1[b];
#pragma unroll
        for (int a = 0; a < 8; ++a) gp[OFF_W2 + j * NW + rg + 16 * a] = g2[b][a];
        if (rg == 0) {
            gp[OFF_B1 + j] = gb1[b];
            gp[OFF_B2 + j] = gb2[b];
        }
    }
    gp[OFF_W3 + t] = g3[0];
    gp[OFF_W3 + t + NT] = g3[1];
    if (t < NOUT) gp[OFF_B3 + t] = gb3;
    // the CTA's loss: warp sums, then thread 0
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, off);
    if (lane == 0) S.red[w] = lsum;
    __syncthreads();
    if (t == 0) {
        double l = 0.0;
        for (int i = 0; i < NT / 32; ++i) l += S.red[i];
        lpart[blockIdx.x] = l / (double)n;   // the loss is the mean over the rows
    }
}

// Gradient = sum of the CTA partials (fixed order); then, with ADAM, one Adam step on the FP32 master
// parameters and their bfloat16 copy.  c1, c2 = 1 / (1 - beta^t) (bias corrections).
template <bool ADAM>
__global__ void k_mlp_update(const float* __restrict__ gpart, int nb, const double* __restrict__ lpart, float* p,
                             __nv_bfloat16* pb, float* m, float* v, float lr, float c1, float c2,
                             float* __restrict__ grad_out, double* __restrict__ loss_out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        double l = 0.0;
        for (int b = 0; b < nb; ++b) l += lpart[b];
        *loss_out = l;
    }
    if (i >= NPAR) return;
    float g = 0.f;
    for (int b = 0; b < nb; ++b) g += gpart[(size_t)b * NPAR + i];
    if (grad_out) grad_out[i] = g;
    if (ADAM) {
        const float mi = ADAM_B1 * m[i] + (1.f - ADAM_B1) * g;
        const float vi = ADAM_B2 * v[i] + (1.f - ADAM_B2) * g * g;
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr * (mi * c1) / (sqrtf(vi * c2) + ADAM_EPS);
        p[i] = pi;
        pb[i] = __float2bfloat16_rn(pi);
    }
}

__global__ void k_mlp_round(const float* __restrict__ p, __nv_bfloat16* __restrict__ pb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < NPAR) pb[i] = __float2bfloat16_rn(p[i]);
}

constexpr int UB = 256;   // threads of the update / feature kernels
inline unsigned ublocks(int64_t n) { return (unsigned)((n + UB - 1) / UB); }

struct Mlp {
    int device = 0;
    cudaStream_t stream = nullptr;
    int nb = 0;                    // CTAs of the training kernel (one per SM)
    float *p = nullptr, *m = nullptr, *v = nullptr, *gpart = nullptr, *grad = nullptr;
    __nv_bfloat16* pb = nullptr;
    double *lpart = nullptr, *loss = nullptr;
    int64_t step = 0;              // Adam steps taken
    std::string err;
};

// The kernels' shared-memory opt-in (idempotent; contexts on several host threads may race here harmlessly).
cudaError_t mlp_attr() {
    const int bytes = (int)sizeof(MlpSmem);
    cudaError_t e = cudaFuncSetAttribute(k_mlp<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_mlp<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    return e;
}

void mlp_free(Mlp* q) {
    for (void* a : {(void*)q->p, (void*)q->m, (void*)q->v, (void*)q->gpart, (void*)q->grad, (void*)q->pb,
                    (void*)q->lpart, (void*)q->loss})
        if (a) cudaFree(a);
}

// forward + backward over n rows, then the update kernel (ADAM or gradient only)
cudaError_t mlp_train_pass(Mlp* q, const float* X, const float* T, int64_t n, bool adam, float lr) {
    cudaError_t e = mlp_attr();
    if (e != cudaSuccess) return e;
    const float inv_n = 1.0f / (float)n;
    k_mlp<true><<<q->nb, NT, sizeof(MlpSmem), q->stream>>>(X, T, n, inv_n, q->p, q->pb, nullptr, q->gpart, q->lpart);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    float c1 = 1.f, c2 = 1.f;
    if (adam) {
        q->step += 1;
        c1 = (float)(1.0 / (1.0 - std::pow((double)ADAM_B1, (double)q->step)));
        c2 = (float)(1.0 / (1.0 - std::pow((double)ADAM_B2, (double)q->step)));
        k_mlp_update<true><<<ublocks(NPAR), UB, 0, q->stream>>>(q->gpart, q->nb, q->lpart, q->p, q->pb, q->m, q->v,
                                                                 lr, c1, c2, q->grad, q->loss);
    } else {
        k_mlp_update<false><<<ublocks(NPAR), UB, 0, q->stream>>>(q->gpart, q->nb, q->lpart, q->p, q->pb, q->m,
                                                                  q->v, lr, c1, c2, q->grad, q->loss);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Node features
// ---------------------------------------------------------------------------------------------
__global__ void k_ws_counts(const int32_t* __restrict__ elem, int64_t n_elem, int n_p, int n_q,
                            const uint8_t* __restrict__ flag, int32_t* cnt) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_elem; e += (int64_t)gridDim.x * blockDim.x) {
        int c = n_q;
        if (flag) {
            c = 0;
            for (int q = 0; q < n_q; ++q) c += flag[e * n_q + q] != 0;
        }
        if (c == 0) continue;
        for (int a = 0; a < n_p; ++a) atomicAdd(&cnt[elem[e * n_p + a]], c);
    }
}

// Yield proximity of the committed state (Sections 2.2, 2.3): per point, the ratio of the yield
// function's stress part to its current limit (von Mises |dev s - beta| / (Y + H alpha), Drucker-
// Prager (|dev s| / sqrt(2) + eta p) / (c + Hc alpha)), clamped at 0; per element the largest, and
// per node the largest over its elements (atomicMax on the bits of a non-negative float).
__global__ void k_ws_prox(MeshDev mesh, const double* __restrict__ sig, const double* __restrict__ hard, int n_p,
                          int n_q, int dim, int* prox_bits) {
    const int nc = dim == 2 ? 4 : 6;
    const int64_t n_int = mesh.n_int;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < mesh.n_elem;
         e += (int64_t)gridDim.x * blockDim.x) {
        const MatConst& m = elem_material(mesh, e);
        if (m.model == 0) continue;
        double qmax = 0.0;
        for (int q = 0; q < n_q; ++q) {
            const int64_t ip = e * n_q + q;
            double v[6];
            for (int k = 0; k < nc; ++k) v[k] = sig[k * n_int + ip];
            if (m.model == 1)
                for (int k = 0; k < nc; ++k) v[k] -= hard[k * n_int + ip];
            // (11, 22, 33) and the shear entries of the stored layout
            double s11, s22, s33, sh2;
            if (dim == 2) {
                s11 = v[0]; s22 = v[1]; s33 = v[3];
                sh2 = v[2] * v[2];
            } else {
                s11 = v[0]; s22 = v[1]; s33 = v[2];
                sh2 = v[3] * v[3] + v[4] * v[4] + v[5] * v[5];
            }
            // the back stress is deviatoric: subtracting it leaves the mean stress unchanged
            const double mean = (s11 + s22 + s33) / 3.0;
            const double d1 = s11 - mean, d2 = s22 - mean, d3 = s33 - mean;
            const double nrm = sqrt(d1 * d1 + d2 * d2 + d3 * d3 + 2.0 * sh2);
            double r;
            if (m.model == 1) r = nrm / m.Y;
            else if (m.model == 2) r = nrm / (m.Y + m.H * hard[ip]);
            else r = (nrm * 0.70710678118654752440 + m.eta * mean) / (m.c + m.Hc * hard[ip]);
            qmax = fmax(qmax, r);
        }
        const float qf = (float)qmax;
        if (!(qf > 0.f)) continue;
        const int bits = __float_as_int(qf);
        for (int a = 0; a < n_p; ++a) atomicMax(&prox_bits[mesh.elem_nodes[e * n_p + a]], bits);
    }
}

__global__ void k_ws_fraction(const int32_t* __restrict__ cnt_pl, const int32_t* __restrict__ cnt_ip, int64_t n,
                              float* __restrict__ pf) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        pf[i] = cnt_ip[i] > 0 ? (float)cnt_pl[i] / (float)cnt_ip[i] : 0.f;
}

// one CTA per problem: sum of squares of u1 - u2 over its DOFs (fixed-order reduction)
constexpr int SB = 1024;
__global__ void __launch_bounds__(SB) k_ws_scale(const double* __restrict__ u1, const double* __restrict__ u2,
                                                 const int64_t* __restrict__ prob_dof, int n_prob,
                                                 double* __restrict__ scale) {
    __shared__ double red[SB / 32];
    const int p = blockIdx.x;
    const int64_t b = prob_dof[p], e = prob_dof[p + 1];
    double acc = 0.0;
    for (int64_t i = b + threadIdx.x; i < e; i += SB) {
        const double d = u1[i] - u2[i];
        acc = fma(d, d, acc);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double sum = 0.0;
        for (int i = 0; i < SB / 32; ++i) sum += red[i];
        const int64_t nd = e - b;
        const double sv = nd > 0 ? sqrt(sum / (double)nd) : 0.0;
        scale[p] = sv;
        scale[n_prob + p] = sv > 0.0 ? 1.0 / sv : 0.0;
    }
}

__global__ void k_ws_features(const double* __restrict__ u1, const double* __restrict__ u2,
                              const double* __restrict__ u3, const int32_t* __restrict__ node_prob,
                              const double* __restrict__ scale, int n_prob, int dim, int64_t n_nodes, float r_k,
                              float r_k1, const float* __restrict__ pf1, const float* __restrict__ pf2,
                              const float* __restrict__ prox1, const float* __restrict__ stat,
                              float* __restrict__ X) {
    for (int64_t nd = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; nd < n_nodes;
         nd += (int64_t)gridDim.x * blockDim.x) {
        const int p = node_prob ? node_prob[nd] : 0;
        const double inv_s = scale[n_prob + p];
        float* x = X + nd * NIN;
        for (int c = 0; c < 3; ++c) {
            float a = 0.f, b = 0.f;
            if (c < dim) {
                const int64_t i = nd * dim + c;
                a = (float)((u1[i] - u2[i]) * inv_s);
                b = (float)((u2[i] - u3[i]) * inv_s);
            }
            x[c] = a;
            x[3 + c] = b;
        }
        x[6] = r_k;
        x[7] = r_k1;
        x[8] = pf1[nd];
        x[9] = pf1[nd] - pf2[nd];
        x[10] = prox1[nd];
        for (int c = 0; c < 5; ++c) x[11 + c] = stat[nd * 5 + c];
    }
}

// P(Y): one CTA per problem; per displacement component c the least-squares fit of Y[:, c] over the
// problem's free DOFs by a x1 + b x2 (x1, x2 = the scaled last two increments X[:, c], X[:, 3 + c]),
// from the 2x2 normal equations (FP64 sums, fixed-order reduction); singular (det <= 1e-12 S11 S22):
// x1 alone; x1 = 0: nothing.  Y[:, c] is replaced by the fit (0 on prescribed DOFs).
constexpr int PB = 512;
__global__ void __launch_bounds__(PB) k_ws_project(const float* __restrict__ X, float* __restrict__ Y,
                                                   const uint8_t* __restrict__ free_dof,
                                                   const int64_t* __restrict__ prob_dof, int dim) {
    __shared__ double red[PB / 32][15];
    __shared__ double coef[3][2];
    const int p = blockIdx.x;
    const int64_t n0 = prob_dof[p] / dim, n1 = prob_dof[p + 1] / dim;
    double acc[15];
#pragma unroll
    for (int k = 0; k < 15; ++k) acc[k] = 0.0;
    for (int64_t nd = n0 + threadIdx.x; nd < n1; nd += PB) {
        for (int c = 0; c < dim; ++c) {
            if (!free_dof[nd * dim + c]) continue;
            const double x1 = X[nd * NIN + c], x2 = X[nd * NIN + 3 + c], y = Y[nd * NOUT + c];
            acc[5 * c + 0] = fma(x1, x1, acc[5 * c + 0]);
            acc[5 * c + 1] = fma(x1, x2, acc[5 * c + 1]);
            acc[5 * c + 2] = fma(x2, x2, acc[5 * c + 2]);
            acc[5 * c + 3] = fma(x1, y, acc[5 * c + 3]);
            acc[5 * c + 4] = fma(x2, y, acc[5 * c + 4]);
        }
    }
#pragma unroll
    for (int k = 0; k < 15; ++k) {
        double v = acc[k];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        const int c = threadIdx.x;
        double S[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        for (int w = 0; w < PB / 32; ++w)
            for (int k = 0; k < 5; ++k) S[k] += red[w][5 * c + k];
        const double s11 = S[0], s12 = S[1], s22 = S[2], b1 = S[3], b2 = S[4];
        const double det = s11 * s22 - s12 * s12;
        double a = 0.0, b = 0.0;
        if (det > 1e-12 * s11 * s22 && det > 0.0) {
            a = (s22 * b1 - s12 * b2) / det;
            b = (s11 * b2 - s12 * b1) / det;
        } else if (s11 > 0.0) {
            a = b1 / s11;
        }
        coef[c][0] = a;
        coef[c][1] = b;
    }
    __syncthreads();
    for (int64_t nd = n0 + threadIdx.x; nd < n1; nd += PB)
        for (int c = 0; c < dim; ++c) {
            const double x1 = X[nd * NIN + c], x2 = X[nd * NIN + 3 + c];
            Y[nd * NOUT + c] = free_dof[nd * dim + c] ? (float)(coef[c][0] * x1 + coef[c][1] * x2) : 0.f;
        }
}

__global__ void k_ws_apply(double* __restrict__ u, const float* __restrict__ Y, const int32_t* __restrict__ node_prob,
                           const double* __restrict__ scale, const uint8_t* __restrict__ free_dof, int dim,
                           int64_t n_dof) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_dof; i += (int64_t)gridDim.x * blockDim.x) {
        if (!free_dof[i]) continue;
        const int64_t nd = i / dim;
        const int c = (int)(i - nd * dim);
        const int p = node_prob ? node_prob[nd] : 0;
        u[i] += scale[p] * (double)Y[nd * NOUT + c];
    }
}

__global__ void k_ws_targets(const double* __restrict__ uk, const double* __restrict__ u1,
                             const double* __restrict__ u2, double ratio, const int32_t* __restrict__ node_prob,
                             const double* __restrict__ scale, int n_prob, const uint8_t* __restrict__ free_dof,
                             const float* __restrict__ pf_k, int dim, int64_t n_nodes, float* __restrict__ T) {
    for (int64_t nd = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; nd < n_nodes;
         nd += (int64_t)gridDim.x * blockDim.x) {
        const int p = node_prob ? node_prob[nd] : 0;
        const double inv_s = scale[n_prob + p];
        for (int c = 0; c < 3; ++c) {
            float v = 0.f;
            if (c < dim) {
                const int64_t i = nd * dim + c;
                if (free_dof[i]) v = (float)((uk[i] - (u1[i] + ratio * (u1[i] - u2[i]))) * inv_s);
            }
            T[nd * NOUT + c] = v;
        }
        T[nd * NOUT + 3] = pf_k[nd];
    }
}

__global__ void k_ws_select(double* __restrict__ u, const double* __restrict__ u_alt,
                            const int32_t* __restrict__ node_prob, const uint8_t* __restrict__ take_alt, int dim,
                            int64_t n_dof) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_dof; i += (int64_t)gridDim.x * blockDim.x) {
        const int p = node_prob ? node_prob[i / dim] : 0;
        if (take_alt[p]) u[i] = u_alt[i];
    }
}

inline unsigned fgrid(int64_t n) {
    const int64_t b = (n + UB - 1) / UB;
    return (unsigned)(b < 1 ? 1 : (b > 65535 ? 65535 : b));
}

}  // namespace

cudaError_t ws_node_counts(const int32_t* elem, int64_t n_elem, int n_p, int n_q, const uint8_t* flag, int32_t* cnt,
                           cudaStream_t s) {
    k_ws_counts<<<fgrid(n_elem), UB, 0, s>>>(elem, n_elem, n_p, n_q, flag, cnt);
    return cudaGetLastError();
}
cudaError_t ws_fraction(const int32_t* cnt_pl, const int32_t* cnt_ip, int64_t n_nodes, float* pf, cudaStream_t s) {
    k_ws_fraction<<<fgrid(n_nodes), UB, 0, s>>>(cnt_pl, cnt_ip, n_nodes, pf);
    return cudaGetLastError();
}
cudaError_t ws_scale(const double* u1, const double* u2, const int64_t* prob_dof, int n_prob, double* scale,
                     cudaStream_t s) {
    k_ws_scale<<<n_prob, SB, 0, s>>>(u1, u2, prob_dof, n_prob, scale);
    return cudaGetLastError();
}
cudaError_t ws_features(const double* u1, const double* u2, const double* u3, const int32_t* node_prob,
                        const double* scale, int n_prob, int dim, int64_t n_nodes, double r_k, double r_k1,
                        const float* pf1, const float* pf2, const float* prox1, const float* stat, float* X,
                        cudaStream_t s) {
    k_ws_features<<<fgrid(n_nodes), UB, 0, s>>>(u1, u2, u3, node_prob, scale, n_prob, dim, n_nodes, (float)r_k,
                                                (float)r_k1, pf1, pf2, prox1, stat, X);
    return cudaGetLastError();
}
cudaError_t ws_proximity(const MeshDev& mesh, const double* sig, const double* hard, int n_p, int n_q, int dim,
                         float* prox, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(prox, 0, sizeof(float) * mesh.n_nodes, s);
    if (e != cudaSuccess) return e;
    k_ws_prox<<<fgrid(mesh.n_elem), UB, 0, s>>>(mesh, sig, hard, n_p, n_q, dim, reinterpret_cast<int*>(prox));
    return cudaGetLastError();
}
cudaError_t ws_project(const float* X, float* Y, const uint8_t* free_dof, const int64_t* prob_dof, int n_prob,
                       int dim, cudaStream_t s) {
    k_ws_project<<<n_prob, PB, 0, s>>>(X, Y, free_dof, prob_dof, dim);
    return cudaGetLastError();
}
cudaError_t ws_apply(double* u, const float* Y, const int32_t* node_prob, const double* scale, int n_prob,
                     const uint8_t* free_dof, int dim, int64_t n_dof, cudaStream_t s) {
    (void)n_prob;
    k_ws_apply<<<fgrid(n_dof), UB, 0, s>>>(u, Y, node_prob, scale, free_dof, dim, n_dof);
    return cudaGetLastError();
}
cudaError_t ws_targets(const double* uk, const double* u1, const double* u2, double ratio, const int32_t* node_prob,
                       const double* scale, int n_prob, const uint8_t* free_dof, const float* pf_k, int dim,
                       int64_t n_nodes, float* T, cudaStream_t s) {
    k_ws_targets<<<fgrid(n_nodes), UB, 0, s>>>(uk, u1, u2, ratio, node_prob, scale, n_prob, free_dof, pf_k, dim,
                                               n_nodes, T);
    return cudaGetLastError();
}
cudaError_t ws_select(double* u, const double* u_alt, const int32_t* node_prob, const uint8_t* take_alt, int dim,
                      int64_t n_dof, cudaStream_t s) {
    k_ws_select<<<fgrid(n_dof), UB, 0, s>>>(u, u_alt, node_prob, take_alt, dim, n_dof);
    return cudaGetLastError();
}

cudaError_t mlp_forward_on(void* mlp, const float* X, int64_t n, float* Y, cudaStream_t s) {
    Mlp* q = static_cast<Mlp*>(mlp);
    if (n <= 0) return cudaSuccess;
    cudaError_t e = mlp_attr();
    if (e != cudaSuccess) return e;
    const int64_t tiles = (n + TR - 1) / TR;
    const int grid = (int)(tiles < 2 * q->nb ? tiles : 2 * q->nb);
    k_mlp<false><<<grid, NT, sizeof(MlpSmem), s>>>(X, nullptr, n, 0.f, q->p, q->pb, Y, nullptr, nullptr);
    return cudaGetLastError();
}

cudaError_t mlp_sync(void* mlp) { return cudaStreamSynchronize(static_cast<Mlp*>(mlp)->stream); }

}  // namespace ep

using namespace ep;

extern "C" {

ep_status ep_mlp_create(void** out, const float* params, int32_t device, void* cuda_stream) {
    if (!out) return EP_ERR_INVALID_ARG;
    *out = nullptr;
    if (!params) {
        thread_error() = "ep_mlp_create: params is null";
        return EP_ERR_INVALID_ARG;
    }
    if (cudaSetDevice(device) != cudaSuccess) {
        thread_error() = "ep_mlp_create: cudaSetDevice failed";
        return EP_ERR_CUDA;
    }
    Mlp* q = new Mlp();
    q->device = device;
    q->stream = static_cast<cudaStream_t>(cuda_stream);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    q->nb = sms > 0 ? sms : 1;
    cudaError_t e = cudaSuccess;
    auto al = [&](auto** ptr, size_t count) {
        if (e == cudaSuccess) e = cudaMalloc((void**)ptr, count * sizeof(**ptr));
    };
    al(&q->p, NPAR);
    al(&q->m, NPAR);
    al(&q->v, NPAR);
    al(&q->grad, NPAR);
    al(&q->pb, NPAR);
    al(&q->gpart, (size_t)q->nb * NPAR);
    al(&q->lpart, (size_t)q->nb);
    al(&q->loss, 1);
    if (e == cudaSuccess) e = cudaMemcpyAsync(q->p, params, sizeof(float) * NPAR, cudaMemcpyHostToDevice, q->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(q->m, 0, sizeof(float) * NPAR, q->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(q->v, 0, sizeof(float) * NPAR, q->stream);
    if (e == cudaSuccess) {
        k_mlp_round<<<ublocks(NPAR), UB, 0, q->stream>>>(q->p, q->pb);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(q->stream);
    if (e != cudaSuccess) {
        thread_error() = std::string("ep_mlp_create: ") + cudaGetErrorString(e);
        mlp_free(q);
        delete q;
        return e == cudaErrorMemoryAllocation ? EP_ERR_OOM : EP_ERR_CUDA;
    }
    *out = q;
    return EP_OK;
}

ep_status ep_mlp_destroy(void* mlp) {
    if (!mlp) return EP_OK;
    Mlp* q = static_cast<Mlp*>(mlp);
    cudaSetDevice(q->device);
    cudaStreamSynchronize(q->stream);
    mlp_free(q);
    delete q;
    return EP_OK;
}

ep_status ep_mlp_get_params(void* mlp, float* dst) {
    if (!mlp || !dst) return EP_ERR_INVALID_ARG;
    Mlp* q = static_cast<Mlp*>(mlp);
    cudaSetDevice(q->device);
    cudaError_t e = cudaMemcpyAsync(dst, q->p, sizeof(float) * NPAR, cudaMemcpyDeviceToHost, q->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(q->stream);
    return e == cudaSuccess ? EP_OK : EP_ERR_CUDA;
}

ep_status ep_mlp_forward(void* mlp, const float* X, int64_t n_rows, float* Y) {
    if (!mlp || n_rows < 0) return EP_ERR_INVALID_ARG;
    if (n_rows == 0) return EP_OK;
    if (!X || !Y) return EP_ERR_INVALID_ARG;
    Mlp* q = static_cast<Mlp*>(mlp);
    cudaSetDevice(q->device);
    cudaError_t e = mlp_forward_on(q, X, n_rows, Y, q->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(q->stream);
    return e == cudaSuccess ? EP_OK : EP_ERR_CUDA;
}

ep_status ep_mlp_grad(void* mlp, const float* X, const float* T, int64_t n_rows, double* loss, float* grad) {
    if (!mlp || n_rows <= 0 || !X || !T || !loss || !grad) return EP_ERR_INVALID_ARG;
    Mlp* q = static_cast<Mlp*>(mlp);
    cudaSetDevice(q->device);
    cudaError_t e = mlp_train_pass(q, X, T, n_rows, false, 0.f);
    if (e == cudaSuccess) e = cudaMemcpyAsync(grad, q->grad, sizeof(float) * NPAR, cudaMemcpyDeviceToHost, q->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(loss, q->loss, sizeof(double), cudaMemcpyDeviceToHost, q->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(q->stream);
    return e == cudaSuccess ? EP_OK : EP_ERR_CUDA;
}

ep_status ep_mlp_train_step(void* mlp, const float* X, const float* T, int64_t n_rows, float lr, double* loss) {
    if (!mlp || n_rows <= 0 || !X || !T || !(lr > 0.f)) return EP_ERR_INVALID_ARG;
    Mlp* q = static_cast<Mlp*>(mlp);
    cudaSetDevice(q->device);
    cudaError_t e = mlp_train_pass(q, X, T, n_rows, true, lr);
    if (e == cudaSuccess && loss) {
        e = cudaMemcpyAsync(loss, q->loss, sizeof(double), cudaMemcpyDeviceToHost, q->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(q->stream);
    }
    return e == cudaSuccess ? EP_OK : EP_ERR_CUDA;
}

}  // extern "C"
