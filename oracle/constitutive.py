"""Constitutive operators T_k, T_k^o and internal-variable updates (plain numpy, FP64).

Test infrastructure: part of the CPU oracle; never used by the product path.

Voigt conventions of Section 5: stresses (s11,s22,s33,s12,s23,s13), strains
(e11,e22,e33,2e12,2e23,2e13).  IOTA, VOL and DEV are the vector I, the matrix
I (x) I and the deviatoric projector that maps a strain-type vector to a
stress-type one (Section 6.3).  All functions work on arrays [6][n] and return
the stress S [6][n], the tangent DS [6][6][n] (row = stress component, column =
strain component), the plastic flag, and the trial internal variables that
become the new state once the step has converged.

Models (written per point in tensor notation from the closed forms of
Section 2; Voigt arrays are converted at entry and exit):
  * von Mises, linear kinematic hardening (Section 2.2, eqs. (T_kinematic),
    (DT_kinematic), (T_other)); a = 0 gives perfect plasticity.
  * von Mises, linear isotropic hardening: yield |s| <= Y + H*alpha with
    alpha incremented by the plastic multiplier (extension; the consistency
    condition and its derivative are worked out in vm_isotropic's docstring;
    on a virgin state with H = a it gives the kinematic result).
  * Drucker-Prager (Section 2.3): elastic / smooth / apex cases, here with a
    plastic potential of slope eta_bar (nonassociated when eta_bar != eta)
    and linear cohesion hardening c + Hc*alpha (extension; eta_bar = eta and
    Hc = 0 give the paper's perfect-plastic formulas).  p_tr is the mean
    trial stress K tr(e_tr): the trace I:sigma in Section 2.3's notation list
    is read as I:sigma/3, which is what the yield function uses.  A point is
    plastic when the trial yield function is > 0 and returns to the apex when
    eta p_tr - c_k - (K eta eta_bar + Hc)|s_tr|/(sqrt(2) G) > 0 (strict, as in
    Section 7.2; the text of Section 2.3 puts the tie on the apex side).
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


# ----------------------------------------------------------------------------
# Tensor form.  The return mappings below work on symmetric 3x3 tensors
# (arrays [n,3,3]) and fourth-order operators (arrays [n,3,3,3,3]) exactly as
# Section 2 writes them; Voigt vectors enter and leave only at the interface.
# ----------------------------------------------------------------------------

_PAIRS = ((0, 0), (1, 1), (2, 2), (0, 1), (1, 2), (0, 2))   # Voigt index -> tensor index
_I2 = np.eye(3)
_II = np.einsum("ij,kl->ijkl", _I2, _I2)                                   # I (x) I
_I4 = 0.5 * (np.einsum("ik,jl->ijkl", _I2, _I2) + np.einsum("il,jk->ijkl", _I2, _I2))
_P_DEV = _I4 - _II / 3.0                                                    # I_D on symmetric tensors


def _to_tensor(v, strain_type: bool):
    """Voigt [6][n] -> symmetric tensors [n,3,3]; strain-type shears are halved."""
    t = np.empty((v.shape[1], 3, 3))
    for a, (i, j) in enumerate(_PAIRS):
        x = v[a] * 0.5 if (strain_type and i != j) else v[a]
        t[:, i, j] = x
        t[:, j, i] = x
    return t


def _to_voigt(t, strain_type: bool):
    """Symmetric tensors [n,3,3] -> Voigt [6][n]; strain-type shears are doubled."""
    return np.stack([t[:, i, j] * (2.0 if (strain_type and i != j) else 1.0) for i, j in _PAIRS])


def _to_voigt_operator(T):
    """Fourth-order operators [n,3,3,3,3] with minor symmetries -> [6][6][n].

    Row I = stress component (i,j), column J = engineering strain component
    (k,l): since 2 eps_kl = eps_kl + eps_lk, the entry is T_ijkl itself.
    """
    return np.stack([np.stack([T[:, i, j, k, l] for (k, l) in _PAIRS]) for (i, j) in _PAIRS])


def _trace(t):
    return np.einsum("nii->n", t)


def _dev(t):
    return t - (_trace(t) / 3.0)[:, None, None] * _I2


def _norm(t):
    """Frobenius norm |t| = sqrt(t:t) (Section 2's |.|)."""
    return np.sqrt(np.einsum("nij,nij->n", t, t))


def _outer(a, b):
    return np.einsum("nij,nkl->nijkl", a, b)


def _hooke(K, G, eps):
    """C eps = K tr(eps) I + 2G I_D eps (Section 2, eq. (elastic_law))."""
    return (K * _trace(eps))[:, None, None] * _I2 + 2.0 * G * _dev(eps)


def _hooke_operator(K, G, n):
    return np.broadcast_to(K * _II + 2.0 * G * _P_DEV, (n, 3, 3, 3, 3)).copy()


def vm_kinematic(E, Ep_prev, Hard_prev, K, G, a, Y):
    """Von Mises with linear kinematic hardening: eqs. (T_kinematic), (DT_kinematic), (T_other).

    E, Ep_prev: strain-type [6][n]; Hard_prev: back stress beta (stress-type) [6][n].
    Returns S, DS, plastic, Ep_new, Hard_new, lam, where lam = (|s_tr| - Y)/(2G + a)
    is the coefficient the updates of Section 2.2 share.
    """
    n = E.shape[1]
    sigma_tr = _hooke(K, G, _to_tensor(E - Ep_prev, True))
    beta = _to_tensor(Hard_prev, False)
    s_tr = _dev(sigma_tr) - beta                       # trial relative deviator
    size = _norm(s_tr)
    plastic = size > Y                                  # second branch of (T_kinematic)
    sigma, D = sigma_tr.copy(), _hooke_operator(K, G, n)
    ep_t, beta_new = _to_tensor(Ep_prev, True), beta.copy()
    lam = np.zeros(n)
    if plastic.any():
        p = plastic
        nrm = s_tr[p] / size[p, None, None]             # n_k^tr
        lam[p] = (size[p] - Y) / (2.0 * G + a)
        sigma[p] -= (2.0 * G * lam[p])[:, None, None] * nrm
        k = 4.0 * G * G / (2.0 * G + a)
        # (DT_kinematic): C - k I_D + k (Y/|s_tr|) (I_D - n (x) n)
        D[p] += -k * _P_DEV + (k * Y / size[p])[:, None, None, None, None] * (_P_DEV - _outer(nrm, nrm))
        beta_new[p] += (a * lam[p])[:, None, None] * nrm
        ep_t[p] += lam[p][:, None, None] * nrm
    return (_to_voigt(sigma, False), _to_voigt_operator(D), plastic,
            _to_voigt(ep_t, True), _to_voigt(beta_new, False), lam)


def vm_isotropic(E, Ep_prev, alpha_prev, K, G, H, Y):
    """Von Mises with linear isotropic hardening, yield |s| <= Y + H alpha (extension).

    The plastic multiplier lam solves the consistency condition
    |s_tr| - 2G lam - (Y + H (alpha_prev + lam)) = 0; the stress returns along
    the trial normal n; differentiating sigma = sigma_tr - 2G lam n with
    dn/deps = 2G/|s_tr| (I_D - n (x) n) gives
    DS = C - 4G^2/(2G+H) n (x) n - 4G^2 lam/|s_tr| (I_D - n (x) n).
    Returns S, DS, plastic, Ep_new, alpha_new, lam.
    """
    n = E.shape[1]
    sigma_tr = _hooke(K, G, _to_tensor(E - Ep_prev, True))
    s_tr = _dev(sigma_tr)
    size = _norm(s_tr)
    radius = Y + H * alpha_prev
    plastic = size > radius
    sigma, D = sigma_tr.copy(), _hooke_operator(K, G, n)
    ep_t, alpha_new = _to_tensor(Ep_prev, True), alpha_prev.copy()
    lam = np.zeros(n)
    if plastic.any():
        p = plastic
        nrm = s_tr[p] / size[p, None, None]
        lam[p] = (size[p] - radius[p]) / (2.0 * G + H)
        sigma[p] -= (2.0 * G * lam[p])[:, None, None] * nrm
        nn = _outer(nrm, nrm)
        D[p] -= (4.0 * G * G / (2.0 * G + H)) * nn
        D[p] -= (4.0 * G * G * lam[p] / size[p])[:, None, None, None, None] * (_P_DEV - nn)
        alpha_new[p] += lam[p]
        ep_t[p] += lam[p][:, None, None] * nrm
    return (_to_voigt(sigma, False), _to_voigt_operator(D), plastic,
            _to_voigt(ep_t, True), alpha_new, lam)


def drucker_prager(E, Ep_prev, alpha_prev, K, G, eta, c, eta_bar=None, Hc=0.0):
    """Drucker-Prager return mapping (Section 2.3), with the extension of the module header.

    Yield function Psi(sigma, alpha) = |s|/sqrt(2) + eta p - (c + Hc alpha),
    p = tr(sigma)/3; plastic potential |s|/sqrt(2) + eta_bar p, so the flow
    direction in stress space is C(n/sqrt(2) + eta_bar/3 I) = sqrt(2) G n + K eta_bar I.
    Smooth return: the multiplier solves Psi = 0 along that direction,
    lam = Psi_tr/(G + K eta eta_bar + Hc).  It overshoots the apex (|s| would
    change sign) exactly when eta p_tr - c_k - (K eta eta_bar + Hc)|s_tr|/(sqrt(2) G) > 0;
    then the stress is hydrostatic, sigma = p I with eta p = c + Hc (alpha_prev + lam).
    Returns S, DS, plastic (0 elastic, 1 smooth, 2 apex as int8), Ep_new,
    alpha_new, lam, err (1 where the apex is reached but no admissible stress
    exists, i.e. K eta eta_bar + Hc = 0).
    """
    if eta_bar is None:
        eta_bar = eta
    n = E.shape[1]
    eps_e = _to_tensor(E - Ep_prev, True)
    sigma_tr = _hooke(K, G, eps_e)
    s_tr = _dev(sigma_tr)
    rho = _norm(s_tr)                                    # varrho_k^tr
    p_tr = _trace(sigma_tr) / 3.0                        # mean stress (reading of I:sigma)
    c_k = c + Hc * alpha_prev
    slope = K * eta * eta_bar + Hc                       # d(eta p - c_k)/d lam at the apex
    psi_tr = rho / math.sqrt(2.0) + eta * p_tr - c_k
    beyond_apex = eta * p_tr - c_k - slope * rho / (math.sqrt(2.0) * G) > 0
    smooth = (psi_tr > 0) & ~beyond_apex
    apex = (psi_tr > 0) & beyond_apex
    sigma, D = sigma_tr.copy(), _hooke_operator(K, G, n)
    ep_t, alpha_new = _to_tensor(Ep_prev, True), alpha_prev.copy()
    lam = np.zeros(n)
    err = np.zeros(n, dtype=np.int8)
    flag = np.zeros(n, dtype=np.int8)
    flag[smooth] = 1
    flag[apex] = 2
    if smooth.any():
        q = smooth
        nrm = s_tr[q] / rho[q, None, None]
        lam[q] = psi_tr[q] / (G + slope)
        flow = math.sqrt(2.0) * G * nrm + K * eta_bar * _I2       # stress-space flow direction
        grad = math.sqrt(2.0) * G * nrm + K * eta * _I2           # d Psi_tr / d eps
        sigma[q] -= lam[q][:, None, None] * flow
        D[q] -= _outer(flow, grad) / (G + slope)
        D[q] -= (2.0 * math.sqrt(2.0) * G * G * lam[q] / rho[q])[:, None, None, None, None] * (
            _P_DEV - _outer(nrm, nrm))
        ep_t[q] += lam[q][:, None, None] * (nrm / math.sqrt(2.0) + (eta_bar / 3.0) * _I2)
        alpha_new[q] += lam[q]
    if apex.any():
        q = apex
        if slope == 0.0:
            err[q] = ERR_RETURN_MAP
            sigma[q] = np.nan
            D[q] = np.nan
        else:
            lam[q] = (eta * p_tr[q] - c_k[q]) / slope
            p = p_tr[q] - K * eta_bar * lam[q]
            sigma[q] = p[:, None, None] * _I2
            D[q] = (K * Hc / slope) * _II
            # all of the total strain beyond the hydrostatic elastic part is plastic
            ep_t[q] = _to_tensor(E[:, q], True) - (p / (3.0 * K))[:, None, None] * _I2
            alpha_new[q] += lam[q]
    return (_to_voigt(sigma, False), _to_voigt_operator(D), flag,
            _to_voigt(ep_t, True), alpha_new, lam, err)


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
