// Return mappings of the elastoplastic models, one integration point per call.
//
// Implements the closed-form operators T_k and T_k^o of Section 2:
//   * von Mises with linear kinematic hardening (Section 2.2, eqs. (T_kinematic),
//     (DT_kinematic), (T_other));
//   * von Mises with linear isotropic hardening, |s| <= Y + H alpha (the same
//     radial return with a scalar internal variable);
//   * Drucker-Prager (Section 2.3: elastic, smooth and apex returns), with a
//     plastic potential of slope eta_bar and cohesion c + Hc alpha.
// The trial mean stress is K tr(eps_tr); the point is plastic when the trial
// yield function is > 0 and returns to the apex when CRIT2 > 0 (Section 7.2).
//
// Components are "active" Voigt entries: 3D (11,22,33,12,23,13); plane strain
// (11,22,33,12) with eps33 = 0 imposed on the total strain.  Stress-type
// vectors carry tensor shear components, strain-type vectors engineering
// shear.  The tangent is written as
//     D = cV I(x)I + cD DEV + cN n(x)n + cNI n(x)I + cIN I(x)n
// (n = unit trial deviator, stress-type) and evaluated on the NS strain rows
// (3D: all six; plane strain: 11, 22, 12).
#pragma once

#include "ep_internal.h"

namespace ep {

template <int NA>
struct PointIn {
    double eps[NA];     // total strain (strain-type)
    double ep[NA];      // eps^p_{k-1} (strain-type)
    double alpha;       // isotropic hardening variable
    double beta[NA];    // back stress (stress-type), kinematic model only
};

template <int NA>
struct PointOut {
    double sig[NA];
    double ep[NA];
    double alpha;
    double beta[NA];
    double cV, cD, cN, cNI, cIN;   // tangent coefficients (see above)
    double n[NA];                  // unit trial deviator (stress-type)
    int flag;                      // 0 elastic, 1 plastic/smooth, 2 apex
    bool err;
};

__device__ __forceinline__ double dev_norm_sq_normal_shear(double a0, double a1, double a2, double shear_sq) {
    return a0 * a0 + a1 * a1 + a2 * a2 + 2.0 * shear_sq;
}

// MODEL: 0 elastic, 1 VM kinematic, 2 VM isotropic, 3 Drucker-Prager
template <int NA, int MODEL>
__device__ __forceinline__ void return_map(const MatConst& m, const PointIn<NA>& in, PointOut<NA>& out) {
    constexpr int NSH = NA - 3;   // shear components
    const double K = m.K, G = m.G;
    double et[NA];
#pragma unroll
    for (int a = 0; a < NA; ++a) et[a] = in.eps[a] - in.ep[a];
    const double tr = et[0] + et[1] + et[2];
    const double p_tr = K * tr;
    // deviatoric strain, tensor components
    double ed[NA];
    ed[0] = et[0] - tr * (1.0 / 3.0);
    ed[1] = et[1] - tr * (1.0 / 3.0);
    ed[2] = et[2] - tr * (1.0 / 3.0);
#pragma unroll
    for (int a = 3; a < NA; ++a) ed[a] = 0.5 * et[a];
    // trial stress
#pragma unroll
    for (int a = 0; a < 3; ++a) out.sig[a] = 2.0 * G * ed[a] + p_tr;
#pragma unroll
    for (int a = 3; a < NA; ++a) out.sig[a] = 2.0 * G * ed[a];
#pragma unroll
    for (int a = 0; a < NA; ++a) { out.ep[a] = in.ep[a]; out.beta[a] = in.beta[a]; out.n[a] = 0.0; }
    out.alpha = in.alpha;
    out.cV = K; out.cD = 2.0 * G; out.cN = 0.0; out.cNI = 0.0; out.cIN = 0.0;
    out.flag = 0;
    out.err = false;
    if (MODEL == 0) return;

    if (MODEL == 1 || MODEL == 2) {
        // s_tr = 2G dev(eps_tr) - beta (kinematic) ; |s_tr| Frobenius
        double sd[NA];
#pragma unroll
        for (int a = 0; a < NA; ++a) sd[a] = 2.0 * G * ed[a] - (MODEL == 1 ? in.beta[a] : 0.0);
        double sh = 0.0;
#pragma unroll
        for (int a = 3; a < NA; ++a) sh += sd[a] * sd[a];
        // |s_tr| and 1/|s_tr| from one reciprocal square root (no FP64 division)
        const double nsq = dev_norm_sq_normal_shear(sd[0], sd[1], sd[2], sh);
        const double inv = nsq > 0.0 ? rsqrt(nsq) : 0.0;
        const double nrm = nsq * inv;
        const double Yk = (MODEL == 1) ? m.Y : m.Y + m.H * in.alpha;
        const double crit = nrm - Yk;
        if (crit > 0.0) {
            const double lam = crit * m.inv_vm;   // crit / (2G + H)
#pragma unroll
            for (int a = 0; a < NA; ++a) {
                const double na = sd[a] * inv;
                out.n[a] = na;
                out.sig[a] -= 2.0 * G * lam * na;
                out.ep[a] += lam * na * (a < 3 ? 1.0 : 2.0);
                if (MODEL == 1) out.beta[a] += m.H * lam * na;
            }
            if (MODEL == 2) out.alpha += lam;
            const double c4 = 4.0 * G * G;
            if (MODEL == 1) {
                // C - c DEV + c (Y/|s|) (DEV - n(x)n),  c = 4G^2/(2G+a)
                const double c = c4 * m.inv_vm;
                const double cy = c * m.Y * inv;
                out.cD = 2.0 * G - c + cy;
                out.cN = -cy;
            } else {
                // C - 4G^2/(2G+H) n(x)n - 4G^2 lam/|s| (DEV - n(x)n)
                const double cl = c4 * lam * inv;
                out.cD = 2.0 * G - cl;
                out.cN = -c4 * m.inv_vm + cl;
            }
            out.flag = 1;
        }
        (void)NSH;
        return;
    }

    // Drucker-Prager
    double sh = 0.0;
#pragma unroll
    for (int a = 3; a < NA; ++a) sh += ed[a] * ed[a];
    // |dev eps_tr| and its reciprocal from one reciprocal square root (no FP64 division)
    const double nsq = dev_norm_sq_normal_shear(ed[0], ed[1], ed[2], sh);
    const double inv = nsq > 0.0 ? rsqrt(nsq) : 0.0;
    const double normE = nsq * inv;
    const double rho = 2.0 * G * normE;
    const double ck = m.c + m.Hc * in.alpha;
    const double denom_a = K * m.eta * m.eta_bar + m.Hc;
    const double rs2 = 0.70710678118654752440;   // 1/sqrt(2)
    const double crit1 = rho * rs2 + m.eta * p_tr - ck;
    // denom_a * rho / (sqrt(2) G) = sqrt(2) denom_a normE
    const double crit2 = m.eta * p_tr - ck - denom_a * normE * 1.41421356237309504880;
    if (!(crit1 > 0.0)) return;
    if (!(crit2 > 0.0)) {
        // return to the smooth portion of the cone
        const double lam = crit1 * m.inv_den_s;   // crit1 / (G + K eta eta_bar + Hc)
        const double s2G = 1.41421356237309504880 * G;   // sqrt(2) G
        const double Kb = K * m.eta_bar;
#pragma unroll
        for (int a = 0; a < NA; ++a) {
            const double na = ed[a] * inv;
            out.n[a] = na;
            const double Mbar = s2G * na + (a < 3 ? Kb : 0.0);
            out.sig[a] -= lam * Mbar;
            out.ep[a] += lam * (na * rs2 + (a < 3 ? m.eta_bar * (1.0 / 3.0) : 0.0)) * (a < 3 ? 1.0 : 2.0);
        }
        out.alpha += lam;
        // C - c1 (DEV - n(x)n) - Mbar(x)M / denom_s,  c1 = 2 sqrt(2) G^2 lam / rho = sqrt(2) G lam / |dev eps_tr|
        const double c1 = s2G * lam * inv;
        const double id = m.inv_den_s;
        out.cV = K - K * K * m.eta * m.eta_bar * id;
        out.cD = 2.0 * G - c1;
        out.cN = c1 - 2.0 * G * G * id;
        out.cNI = -s2G * K * m.eta * id;
        out.cIN = -s2G * K * m.eta_bar * id;
        out.flag = 1;
        return;
    }
    // return to the apex
    out.flag = 2;
    if (denom_a == 0.0) {
        out.err = true;
        return;
    }
    const double lam = (m.eta * p_tr - ck) * m.inv_den_a;
    const double p = p_tr - K * m.eta_bar * lam;
#pragma unroll
    for (int a = 0; a < NA; ++a) {
        out.sig[a] = (a < 3) ? p : 0.0;
        out.ep[a] = in.eps[a] - ((a < 3) ? p * m.inv_3K : 0.0);
    }
    out.alpha += lam;
    out.cV = K * m.Hc * m.inv_den_a;
    out.cD = 0.0;
}

// Strain rows -> active index: 3D identity; plane strain (11,22,12) -> (0,1,3).
template <int NS>
__device__ __forceinline__ constexpr int row_active(int r) { return NS == 3 ? (r == 2 ? 3 : r) : r; }

// D entry (row r, column s over the NS strain rows).
template <int NS, int NA>
__device__ __forceinline__ double tangent_entry(const PointOut<NA>& o, int r, int s) {
    const int ar = row_active<NS>(r), as = row_active<NS>(s);
    const double Ir = ar < 3 ? 1.0 : 0.0, Is = as < 3 ? 1.0 : 0.0;
    double dev = 0.0;
    if (ar < 3 && as < 3) dev = (ar == as ? 1.0 : 0.0) - 1.0 / 3.0;
    else if (ar == as) dev = 0.5;
    return o.cV * Ir * Is + o.cD * dev + o.cN * o.n[ar] * o.n[as] + o.cNI * o.n[ar] * Is + o.cIN * Ir * o.n[as];
}

// The tangent's coefficients, scaled by the point weight w, and the unit deviator,
// rounded to precision T (the mixed path forms D, H and K in FP32 from these).
template <int NA, class T>
struct PointTan {
    T cV, cD, cN, cNI, cIN;
    T n[NA];
};

template <int NA, class T>
__device__ __forceinline__ void tangent_coeffs(const PointOut<NA>& o, T w, PointTan<NA, T>& t) {
    t.cV = w * (T)o.cV;
    t.cD = w * (T)o.cD;
    t.cN = w * (T)o.cN;
    t.cNI = w * (T)o.cNI;
    t.cIN = w * (T)o.cIN;
#pragma unroll
    for (int a = 0; a < NA; ++a) t.n[a] = (T)o.n[a];
}

// w * D entry (row r, column s over the NS strain rows) from rounded coefficients.
template <int NS, int NA, class T>
__device__ __forceinline__ T tangent_entry_t(const PointTan<NA, T>& t, int r, int s) {
    const int ar = row_active<NS>(r), as = row_active<NS>(s);
    const T Ir = ar < 3 ? T(1) : T(0), Is = as < 3 ? T(1) : T(0);
    T dev = T(0);
    if (ar < 3 && as < 3) dev = (ar == as ? T(1) : T(0)) - T(1) / T(3);
    else if (ar == as) dev = T(0.5);
    return t.cV * Ir * Is + t.cD * dev + t.cN * t.n[ar] * t.n[as] + t.cNI * t.n[ar] * Is + t.cIN * Ir * t.n[as];
}

}  // namespace ep
