"""Constitutive operators T_k, T_k^o and internal-variable updates (plain numpy, FP64).

Test infrastructure: part of the CPU oracle; never used by the product path.

Voigt conventions of Section 5: stresses (s11,s22,s33,s12,s23,s13), strains
(e11,e22,e33,2e12,2e23,2e13).  IOTA, VOL and DEV are the vector I, the matrix
I (x) I and the deviatoric projector that maps a strain-type vector to a
stress-type one (Section 6.3).  All functions work on arrays [6][n] and return
the stress S [6][n], the tangent DS [6][6][n] (row = stress component, column =
strain component), the plastic flag, and the trial internal variables that
become the new state once the step has converged.

Models:
  * von Mises, linear kinematic hardening (Section 2.2, eqs. (T_kinematic),
    (DT_kinematic), (T_other)); a = 0 gives perfect plasticity.
  * von Mises, linear isotropic hardening: yield |s| <= Y + H*alpha with
    alpha incremented by the plastic multiplier; the same radial return with
    a scalar internal variable (extension; reduces to the kinematic formulas
    on a virgin state with H = a).
  * Drucker-Prager (Section 2.3): elastic / smooth / apex cases, here with a
    plastic potential of slope eta_bar (nonassociated when eta_bar != eta)
    and linear cohesion hardening c + Hc*alpha (extension; eta_bar = eta and
    Hc = 0 give the paper's perfect-plastic formulas).  p_tr is the mean
    trial stress K tr(e_tr): the trace I:sigma in Section 2.3's notation list
    is read as I:sigma/3, which is what the yield function and Section 7.2's
    listing use.  Apex when CRIT2 > 0, plastic when CRIT1 > 0 (Section 7.2).
"""
from __future__ import annotations

import math

import numpy as np

IOTA = np.array([1.0, 1.0, 1.0, 0.0, 0.0, 0.0])
VOL = np.outer(IOTA, IOTA)
DEV = np.diag([1.0, 1.0, 1.0, 0.5, 0.5, 0.5]) - VOL / 3.0
SHEAR2 = np.array([1.0, 1.0, 1.0, 2.0, 2.0, 2.0])   # stress-type -> strain-type factor

ERR_RETURN_MAP = 1


def moduli(E: float, nu: float):
    """Bulk and shear moduli of the isotropic Hooke law (Section 2, eq. (elastic_law))."""
    return E / (3.0 * (1.0 - 2.0 * nu)), E / (2.0 * (1.0 + nu))


def dp_parameters(c0: float, phi: float, psi: float, dim: int):
    """(eta, c, eta_bar) from cohesion and friction/dilatancy angles (Section 8.3).

    3D: eta = 6 sin(phi)/(sqrt(3)(3+sin(phi))), c = c0 6 cos(phi)/(sqrt(3)(3+sin(phi)));
    plane strain: eta = 3 tan(phi)/sqrt(9+12 tan^2 phi), c = 3 c0/sqrt(9+12 tan^2 phi).
    eta_bar is the same map applied to the dilatancy angle.
    """
    if dim == 3:
        def f(a):
            return 6.0 * math.sin(a) / (math.sqrt(3.0) * (3.0 + math.sin(a)))
        c = c0 * 6.0 * math.cos(phi) / (math.sqrt(3.0) * (3.0 + math.sin(phi)))
    else:
        def f(a):
            return 3.0 * math.tan(a) / math.sqrt(9.0 + 12.0 * math.tan(a) ** 2)
        c = c0 * 3.0 / math.sqrt(9.0 + 12.0 * math.tan(phi) ** 2)
    return f(phi), c, f(psi)


def elastic_tangent(K: float, G: float):
    """C = 2G DEV + K VOL as a 6x6 strain-to-stress matrix (Section 6.3)."""
    return 2.0 * G * DEV + K * VOL


def _tile(M, n):
    return np.repeat(M[:, :, None], n, axis=2)


def vm_kinematic(E, Ep_prev, Hard_prev, K, G, a, Y):
    """Von Mises with linear kinematic hardening (Sections 2.2 and 7.1).

    E, Ep_prev: strain-type [6][n]; Hard_prev: back stress beta (stress-type) [6][n].
    Returns S, DS, plastic, Ep_new, Hard_new, lam.
    """
    n = E.shape[1]
    E_tr = E - Ep_prev
    S_tr = 2.0 * G * (DEV @ E_tr) + K * (VOL @ E_tr)
    SD_tr = DEV @ (2.0 * G * E_tr) - Hard_prev
    norm_SD = np.sqrt(np.sum(SD_tr[:3] ** 2, axis=0) + 2.0 * np.sum(SD_tr[3:] ** 2, axis=0))
    CRIT = norm_SD - Y
    plastic = CRIT > 0
    S = S_tr.copy()
    DS = _tile(elastic_tangent(K, G), n)
    Ep_new, Hard_new = Ep_prev.copy(), Hard_prev.copy()
    lam = np.zeros(n)
    if plastic.any():
        ip = plastic
        Nhat = SD_tr[:, ip] / norm_SD[ip]
        denom = 2.0 * G + a
        lam[ip] = CRIT[ip] / denom
        S[:, ip] -= 2.0 * G * lam[ip] * Nhat
        const = (2.0 * G) ** 2 / denom
        NN = np.einsum("iq,jq->ijq", Nhat, Nhat)
        ID = _tile(DEV, int(ip.sum()))
        DS[:, :, ip] += -const * ID + (const * Y / norm_SD[ip]) * (ID - NN)
        Hard_new[:, ip] += a * lam[ip] * Nhat
        Ep_new[:, ip] += lam[ip] * Nhat * SHEAR2[:, None]
    return S, DS, plastic, Ep_new, Hard_new, lam


def vm_isotropic(E, Ep_prev, alpha_prev, K, G, H, Y):
    """Von Mises with linear isotropic hardening, yield |s| <= Y + H alpha.

    Radial return: lam = (|s_tr| - Y - H alpha_prev)/(2G + H), S = S_tr - 2G lam n,
    DS = C - 4G^2/(2G+H) n(x)n - 4G^2 lam/|s_tr| (DEV - n(x)n), alpha += lam,
    Ep += lam n.  Returns S, DS, plastic, Ep_new, alpha_new, lam.
    """
    n = E.shape[1]
    E_tr = E - Ep_prev
    S_tr = 2.0 * G * (DEV @ E_tr) + K * (VOL @ E_tr)
    SD_tr = DEV @ (2.0 * G * E_tr)
    norm_SD = np.sqrt(np.sum(SD_tr[:3] ** 2, axis=0) + 2.0 * np.sum(SD_tr[3:] ** 2, axis=0))
    CRIT = norm_SD - (Y + H * alpha_prev)
    plastic = CRIT > 0
    S = S_tr.copy()
    DS = _tile(elastic_tangent(K, G), n)
    Ep_new, alpha_new = Ep_prev.copy(), alpha_prev.copy()
    lam = np.zeros(n)
    if plastic.any():
        ip = plastic
        Nhat = SD_tr[:, ip] / norm_SD[ip]
        denom = 2.0 * G + H
        lam[ip] = CRIT[ip] / denom
        S[:, ip] -= 2.0 * G * lam[ip] * Nhat
        NN = np.einsum("iq,jq->ijq", Nhat, Nhat)
        ID = _tile(DEV, int(ip.sum()))
        DS[:, :, ip] += -((2.0 * G) ** 2 / denom) * NN - ((2.0 * G) ** 2 * lam[ip] / norm_SD[ip]) * (ID - NN)
        alpha_new[ip] += lam[ip]
        Ep_new[:, ip] += lam[ip] * Nhat * SHEAR2[:, None]
    return S, DS, plastic, Ep_new, alpha_new, lam


def drucker_prager(E, Ep_prev, alpha_prev, K, G, eta, c, eta_bar=None, Hc=0.0):
    """Drucker-Prager return mapping (Sections 2.3 and 7.2), with the extension above.

    Returns S, DS, plastic (0 elastic, 1 smooth, 2 apex as int8), Ep_new,
    alpha_new, lam, err (1 where the apex is reached but no admissible stress
    exists, i.e. K eta eta_bar + Hc = 0).
    """
    if eta_bar is None:
        eta_bar = eta
    n = E.shape[1]
    E_tr = E - Ep_prev
    S_tr = 2.0 * G * (DEV @ E_tr) + K * (VOL @ E_tr)
    dev_E = DEV @ E_tr
    norm_E = np.sqrt(np.maximum(0.0, np.sum(E_tr * dev_E, axis=0)))
    rho_tr = 2.0 * G * norm_E
    p_tr = K * (IOTA @ E_tr)
    c_k = c + Hc * alpha_prev
    denom_a = K * eta * eta_bar + Hc
    denom_s = G + denom_a
    CRIT1 = rho_tr / math.sqrt(2.0) + eta * p_tr - c_k
    CRIT2 = eta * p_tr - c_k - denom_a * rho_tr / (G * math.sqrt(2.0))
    IND_s = (CRIT1 > 0) & (CRIT2 <= 0)
    IND_a = (CRIT1 > 0) & (CRIT2 > 0)
    S = S_tr.copy()
    DS = _tile(elastic_tangent(K, G), n)
    Ep_new, alpha_new = Ep_prev.copy(), alpha_prev.copy()
    lam = np.zeros(n)
    err = np.zeros(n, dtype=np.int8)
    flag = np.zeros(n, dtype=np.int8)
    flag[IND_s] = 1
    flag[IND_a] = 2
    if IND_s.any():
        s = IND_s
        ls = CRIT1[s] / denom_s
        lam[s] = ls
        N_hat = dev_E[:, s] / norm_E[s]
        M_bar = math.sqrt(2.0) * G * N_hat + K * eta_bar * IOTA[:, None]
        M = math.sqrt(2.0) * G * N_hat + K * eta * IOTA[:, None]
        S[:, s] -= ls * M_bar
        NN = np.einsum("iq,jq->ijq", N_hat, N_hat)
        MM = np.einsum("iq,jq->ijq", M_bar, M)
        ID = _tile(DEV, int(s.sum()))
        DS[:, :, s] += -(2.0 * math.sqrt(2.0) * G * G * ls / rho_tr[s]) * (ID - NN) - MM / denom_s
        Ep_new[:, s] += ls * (N_hat / math.sqrt(2.0) + (eta_bar / 3.0) * IOTA[:, None]) * SHEAR2[:, None]
        alpha_new[s] += ls
    if IND_a.any():
        a = IND_a
        if denom_a == 0.0:
            err[a] = ERR_RETURN_MAP
            S[:, a] = np.nan
            DS[:, :, a] = np.nan
        else:
            la = (eta * p_tr[a] - c_k[a]) / denom_a
            lam[a] = la
            p = p_tr[a] - K * eta_bar * la
            S[:, a] = IOTA[:, None] * p
            DS[:, :, a] = (K * Hc / denom_a) * VOL[:, :, None]
            Ep_new[:, a] = E[:, a] - IOTA[:, None] * (p / (3.0 * K))
            alpha_new[a] += la
    return S, DS, flag, Ep_new, alpha_new, lam, err


# ----------------------------------------------------------------------------
# Model dispatch with 2D (plane strain) embedding
# ----------------------------------------------------------------------------

# plane-strain state layout (11, 22, 12, 33) <-> 3D Voigt indices
PLANE_STATE_IDX = np.array([0, 1, 3, 2])
PLANE_INPLANE_IDX = np.array([0, 1, 3])


def n_comp(dim: int) -> int:
    return 4 if dim == 2 else 6


def embed_strain(E_in: np.ndarray, dim: int) -> np.ndarray:
    """In-plane strain (e11, e22, 2e12) -> 3D Voigt with e33 = e23 = e13 = 0."""
    if dim == 3:
        return E_in
    out = np.zeros((6, E_in.shape[1]))
    out[PLANE_INPLANE_IDX] = E_in
    return out


def embed_state(X: np.ndarray, dim: int) -> np.ndarray:
    """Stored state (11,22,12,33) -> 3D Voigt vector."""
    if dim == 3:
        return X
    out = np.zeros((6, X.shape[1]))
    out[PLANE_STATE_IDX] = X
    return out


def extract_state(X6: np.ndarray, dim: int) -> np.ndarray:
    return X6 if dim == 3 else X6[PLANE_STATE_IDX]


def constitutive(material, dim: int, E_in, ep_prev, hard_prev):
    """Evaluate the model at strains E_in ([3 or 6][n], strain-type, in-plane in 2D).

    ep_prev: stored plastic strain [n_comp][n]; hard_prev: alpha [n] (isotropic
    models) or back stress [n_comp][n] (kinematic).  Returns a dict with
    S (stored-layout stress [n_comp][n]), S_in (stress rows of the B-matrix
    [3 or 6][n]), DS_in (tangent block [3|6][3|6][n]), plastic (int8), and the
    trial state ep, hard, lam, err.
    """
    K, G = moduli(material.E, material.nu)
    E6 = embed_strain(E_in, dim)
    Ep6 = embed_state(ep_prev, dim)
    n = E6.shape[1]
    err = np.zeros(n, dtype=np.int8)
    model = material.model
    if model == 0:   # elastic
        S6 = elastic_tangent(K, G) @ (E6 - Ep6)
        DS6 = _tile(elastic_tangent(K, G), n)
        plastic = np.zeros(n, dtype=np.int8)
        ep_new, hard_new, lam = ep_prev.copy(), np.array(hard_prev, copy=True), np.zeros(n)
        ep6_new = Ep6
    elif model == 1:  # von Mises kinematic
        B6 = embed_state(hard_prev, dim)
        S6, DS6, pl, ep6_new, B6_new, lam = vm_kinematic(E6, Ep6, B6, K, G, material.H, material.Y)
        plastic = pl.astype(np.int8)
        hard_new = extract_state(B6_new, dim)
    elif model == 2:  # von Mises isotropic
        S6, DS6, pl, ep6_new, hard_new, lam = vm_isotropic(E6, Ep6, hard_prev, K, G, material.H, material.Y)
        plastic = pl.astype(np.int8)
    elif model == 3:  # Drucker-Prager
        eta, c, eta_bar = dp_parameters(material.c0, material.phi, material.psi, dim)
        S6, DS6, plastic, ep6_new, hard_new, lam, err = drucker_prager(
            E6, Ep6, hard_prev, K, G, eta, c, eta_bar, material.Hc)
    else:
        raise ValueError(f"unknown model {model}")
    ep_new = extract_state(ep6_new, dim)
    if dim == 2:
        S_in = S6[PLANE_INPLANE_IDX]
        DS_in = DS6[np.ix_(PLANE_INPLANE_IDX, PLANE_INPLANE_IDX)]
    else:
        S_in, DS_in = S6, DS6
    return dict(S=extract_state(S6, dim), S_in=S_in, DS_in=DS_in, DS6=DS6, plastic=plastic,
                ep=ep_new, hard=hard_new, lam=lam, err=err)
