// Stand-alone return mapping over arrays of points (ep_constitutive): the same
// device code as the fused assembly kernel (Sections 2.2, 2.3), exposed so the
// operator T_k, its tangent T_k^o and the internal-variable updates can be
// checked point by point.
#include "assemble.cuh"

namespace ep {

template <int DIM, int MODEL>
__global__ void __launch_bounds__(256) k_constitutive(MatConst m, int64_t n, const double* __restrict__ E,
                                                       const double* __restrict__ ep_prev,
                                                       const double* __restrict__ hard_prev, double* __restrict__ S,
                                                       double* __restrict__ DS, uint8_t* __restrict__ flag,
                                                       double* __restrict__ ep_new, double* __restrict__ hard_new) {
    constexpr int NA = DIM == 2 ? 4 : 6, NS = DIM == 2 ? 3 : 6;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    PointIn<NA> in;
#pragma unroll
    for (int a = 0; a < NA; ++a) in.eps[a] = 0.0;
#pragma unroll
    for (int r = 0; r < NS; ++r) in.eps[row_active<NS>(r)] = E[(int64_t)r * n + i];
    StateDev st{const_cast<double*>(ep_prev), const_cast<double*>(hard_prev), nullptr, nullptr};
    load_state<NA, MODEL>(st, n, i, in);
    PointOut<NA> o;
    return_map<NA, MODEL>(m, in, o);
#pragma unroll
    for (int a = 0; a < NA; ++a) {
        const int64_t row = (int64_t)stored_row<NA>(a) * n + i;
        S[row] = o.sig[a];
        ep_new[row] = o.ep[a];
        if (MODEL == 1) hard_new[row] = o.beta[a];
    }
    if (MODEL != 1) hard_new[i] = (MODEL == 0) ? hard_prev[i] : o.alpha;
#pragma unroll
    for (int r = 0; r < NS; ++r)
#pragma unroll
        for (int c = 0; c < NS; ++c) DS[((int64_t)r * NS + c) * n + i] = tangent_entry<NS, NA>(o, r, c);
    flag[i] = (uint8_t)(o.err ? 255 : o.flag);
}

cudaError_t launch_constitutive(int dim, const MatConst& m, int64_t n, const double* E, const double* ep_prev,
                                const double* hard_prev, double* S, double* DS, uint8_t* flag, double* ep_new,
                                double* hard_new, cudaStream_t s) {
    const unsigned g = (unsigned)((n + 255) / 256);
#define EP_LC(D_, M_) k_constitutive<D_, M_><<<g, 256, 0, s>>>(m, n, E, ep_prev, hard_prev, S, DS, flag, ep_new, hard_new)
    if (dim == 2) {
        switch (m.model) {
            case 0: EP_LC(2, 0); break;
            case 1: EP_LC(2, 1); break;
            case 2: EP_LC(2, 2); break;
            case 3: EP_LC(2, 3); break;
        }
    } else {
        switch (m.model) {
            case 0: EP_LC(3, 0); break;
            case 1: EP_LC(3, 1); break;
            case 2: EP_LC(3, 2); break;
            case 3: EP_LC(3, 3); break;
        }
    }
#undef EP_LC
    return cudaGetLastError();
}

cudaError_t launch_reset_dirty(uint8_t* dirty, int64_t nnzb, int d2, const double* Kel, double* Kt, int grid,
                               cudaStream_t s) {
    k_reset_dirty<double><<<grid, 256, 0, s>>>(dirty, nnzb, d2, Kel, Kt);
    return cudaGetLastError();
}

cudaError_t launch_reset_dirty(uint8_t* dirty, int64_t nnzb, int d2, const float* Kel, float* Kt, int grid,
                               cudaStream_t s) {
    k_reset_dirty<float><<<grid, 256, 0, s>>>(dirty, nnzb, d2, Kel, Kt);
    return cudaGetLastError();
}

}  // namespace ep
