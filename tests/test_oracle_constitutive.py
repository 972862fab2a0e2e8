"""Pins for the oracle's return mappings (Sections 2.2, 2.3 and the extensions).

Independent checks: tangents equal central differences of the stress map,
yield-function invariants after the return, Hooke's law with the returned
plastic strain, reductions between models (isotropic vs kinematic hardening
on a virgin state; nonassociated DP with eta_bar = eta and Hc = 0 vs the
paper's perfect-plastic formulas written from Section 2.3's text form), and
closed-form special cases (elastic points give C, perfect-plastic apex gives 0).
"""
import math

import numpy as np
import pytest

from oracle import constitutive as C

E_MOD, NU = 206900.0, 0.29
K, G = C.moduli(E_MOD, NU)
Y = 450.0 * math.sqrt(2.0 / 3.0)


def _strains(n, scale, seed):
    g = np.random.default_rng(seed)
    return g.standard_normal((6, n)) * scale


def _vm_kin(E, Ep, B, a=1e4):
    return C.vm_kinematic(E, Ep, B, K, G, a, Y)


def _vm_iso(E, Ep, al, H=1e4):
    return C.vm_isotropic(E, Ep, al, K, G, H, Y)


def _dp(E, Ep, al, phi=30.0, psi=10.0, Hc=1e3, c0=450.0):
    eta, c, eta_bar = C.dp_parameters(c0, math.radians(phi), math.radians(psi), 3)
    return C.drucker_prager(E, Ep, al, K, G, eta, c, eta_bar, Hc)


def _fd_tangent(fun, E, h):
    n = E.shape[1]
    D = np.zeros((6, 6, n))
    for j in range(6):
        Ep, Em = E.copy(), E.copy()
        Ep[j] += h
        Em[j] -= h
        D[:, j, :] = (fun(Ep) - fun(Em)) / (2 * h)
    return D


def _check_fd(fun_full, E, mask):
    S, DS = fun_full(E)[:2]
    h = 1e-7 * max(1e-3, np.abs(E).max())
    fd = _fd_tangent(lambda X: fun_full(X)[0], E, h)
    scale = np.abs(DS[:, :, mask]).max()
    err = np.abs(fd[:, :, mask] - DS[:, :, mask]).max()
    assert err <= 1e-6 * scale, err / scale


def test_vm_kinematic_tangent_fd():
    n = 400
    E = _strains(n, 1.5e-3, 1)
    Ep = _strains(n, 3e-4, 2)
    B = C.DEV @ _strains(n, 50.0, 3)
    S, DS, pl, *_ = _vm_kin(E, Ep, B)
    SD = C.DEV @ (2 * G * (E - Ep)) - B
    nrm = np.sqrt((SD[:3] ** 2).sum(0) + 2 * (SD[3:] ** 2).sum(0))
    mask = np.abs(nrm - Y) / Y > 1e-3
    assert pl.sum() > 50 and (~pl).sum() > 50
    _check_fd(lambda X: _vm_kin(X, Ep, B), E, mask)
    # symmetric tangent
    np.testing.assert_allclose(DS, np.transpose(DS, (1, 0, 2)), atol=1e-9 * np.abs(DS).max())
    # elastic points: D = C exactly
    Ce = C.elastic_tangent(K, G)
    assert np.array_equal(DS[:, :, ~pl], np.repeat(Ce[:, :, None], (~pl).sum(), axis=2))


def test_vm_isotropic_tangent_fd_and_invariants():
    n = 400
    E = _strains(n, 1.5e-3, 4)
    Ep = _strains(n, 3e-4, 5)
    al = np.abs(np.random.default_rng(6).standard_normal(n)) * 5e-3
    H = 1e4
    S, DS, pl, Ep_new, al_new, lam = _vm_iso(E, Ep, al, H)
    assert pl.sum() > 50 and (~pl).sum() > 50
    SD = C.DEV @ (2 * G * (E - Ep))
    nrm = np.sqrt((SD[:3] ** 2).sum(0) + 2 * (SD[3:] ** 2).sum(0))
    mask = np.abs(nrm - Y - H * al) / Y > 1e-3
    _check_fd(lambda X: _vm_iso(X, Ep, al, H), E, mask)
    np.testing.assert_allclose(DS, np.transpose(DS, (1, 0, 2)), atol=1e-9 * np.abs(DS).max())
    # yield function after the return: <= 0 everywhere, = 0 at plastic points
    s = S - (S[:3].sum(0) / 3) * C.IOTA[:, None]
    ns = np.sqrt((s[:3] ** 2).sum(0) + 2 * (s[3:] ** 2).sum(0))
    psi = ns - Y - H * al_new
    assert psi.max() <= 1e-12 * Y
    assert np.abs(psi[pl]).max() <= 1e-12 * Y
    assert (lam >= 0).all()
    # Hooke's law with the returned plastic strain
    np.testing.assert_allclose(S, C.elastic_tangent(K, G) @ (E - Ep_new), atol=1e-9 * np.abs(S).max())
    # multiplier equals the increment of the hardening variable
    np.testing.assert_allclose(al_new - al, lam, atol=1e-18)


def test_isotropic_equals_kinematic_on_virgin_state():
    n = 300
    E = _strains(n, 3e-3, 7)
    Z = np.zeros((6, n))
    a = 1e4
    Sk, Dk, pk, Epk, Bk, lk = _vm_kin(E, Z, Z, a)
    Si, Di, pi, Epi, ali, li = _vm_iso(E, Z, np.zeros(n), a)
    assert np.array_equal(pk, pi)
    np.testing.assert_allclose(Si, Sk, rtol=0, atol=1e-10 * np.abs(Sk).max())
    np.testing.assert_allclose(Di, Dk, rtol=0, atol=1e-9 * np.abs(Dk).max())
    np.testing.assert_allclose(Epi, Epk, rtol=0, atol=1e-15)
    np.testing.assert_allclose(li, lk, rtol=0, atol=1e-16)


def _dp_cases(n, seed):
    """Strains spanning elastic, smooth and apex returns."""
    g = np.random.default_rng(seed)
    E = g.standard_normal((6, n)) * 2e-3
    # add a volumetric part ranging from compression to strong tension
    E[:3] += g.uniform(-4e-3, 6e-3, n)
    return E


def test_dp_tangent_fd_all_regimes():
    n = 2000
    E = _dp_cases(n, 8)
    Ep = _strains(n, 2e-4, 9)
    al = np.abs(np.random.default_rng(10).standard_normal(n)) * 1e-3
    phi, psi, Hc, c0 = 30.0, 10.0, 1e3, 450.0
    S, DS, flag, Ep_new, al_new, lam, err = _dp(E, Ep, al, phi, psi, Hc, c0)
    assert (flag == 0).sum() > 100 and (flag == 1).sum() > 100 and (flag == 2).sum() > 100
    assert not err.any()
    eta, c, eta_bar = C.dp_parameters(c0, math.radians(phi), math.radians(psi), 3)
    Et = E - Ep
    devE = C.DEV @ Et
    rho = 2 * G * np.sqrt(np.maximum(0, (Et * devE).sum(0)))
    p = K * Et[:3].sum(0)
    ck = c + Hc * al
    crit1 = rho / math.sqrt(2) + eta * p - ck
    crit2 = eta * p - ck - (K * eta * eta_bar + Hc) * rho / (G * math.sqrt(2))
    mask = (np.abs(crit1) / c > 1e-3) & (np.abs(crit2) / c > 1e-3)
    _check_fd(lambda X: _dp(X, Ep, al, phi, psi, Hc, c0), E, mask)
    # nonassociated: the smooth-return tangent is not symmetric
    sm = flag == 1
    asym = np.abs(DS[:, :, sm] - np.transpose(DS[:, :, sm], (1, 0, 2))).max()
    assert asym > 1e-3 * np.abs(DS).max()
    # yield function <= 0 after return, = 0 at plastic points
    s = S - (S[:3].sum(0) / 3) * C.IOTA[:, None]
    ns = np.sqrt((s[:3] ** 2).sum(0) + 2 * (s[3:] ** 2).sum(0))
    yf = ns / math.sqrt(2) + eta * S[:3].sum(0) / 3 - (c + Hc * al_new)
    assert yf.max() <= 1e-12 * c
    assert np.abs(yf[flag > 0]).max() <= 1e-10 * c
    assert (lam >= 0).all()
    np.testing.assert_allclose(S, C.elastic_tangent(K, G) @ (E - Ep_new), atol=1e-9 * np.abs(S).max())
    # apex: purely hydrostatic stress
    assert np.abs(s[:, flag == 2]).max() <= 1e-9 * c


def test_dp_associated_perfect_matches_section_2_3_text_form():
    """eta_bar = eta, Hc = 0: the text form of Section 2.3 (T, T^o, eps^p for the three cases)."""
    n = 1500
    E = _dp_cases(n, 11)
    Ep = _strains(n, 2e-4, 12)
    al = np.zeros(n)
    phi = math.radians(20.0)
    eta, c, _ = C.dp_parameters(450.0, phi, phi, 3)
    S, DS, flag, Ep_new, *_ = C.drucker_prager(E, Ep, al, K, G, eta, c, eta, 0.0)
    Ce = C.elastic_tangent(K, G)
    for i in range(n):
        e = E[:, i] - Ep[:, i]
        sig_tr = Ce @ e
        p_tr = sig_tr[:3].sum() / 3.0
        s_tr = sig_tr - p_tr * C.IOTA
        rho = math.sqrt((s_tr[:3] ** 2).sum() + 2 * (s_tr[3:] ** 2).sum())
        psi_tr = rho / math.sqrt(2) + eta * p_tr - c
        if psi_tr <= 0:
            assert flag[i] == 0
            np.testing.assert_allclose(S[:, i], sig_tr, rtol=1e-13, atol=1e-9)
            continue
        if eta * p_tr - K * eta * eta / (G * math.sqrt(2)) * rho < c:
            assert flag[i] == 1
            nv = s_tr / rho
            g = G * math.sqrt(2) * nv + K * eta * C.IOTA
            sig = sig_tr - psi_tr / (G + K * eta * eta) * g
            tang = Ce - (1 / (G + K * eta * eta)) * (
                2 * G * G * math.sqrt(2) * psi_tr / rho * (C.DEV - np.outer(nv, nv)) + np.outer(g, g))
            dep = psi_tr / (G + K * eta * eta) * (math.sqrt(2) / 2 * nv + eta / 3 * C.IOTA) * C.SHEAR2
            np.testing.assert_allclose(S[:, i], sig, rtol=1e-12, atol=1e-9)
            np.testing.assert_allclose(DS[:, :, i], tang, rtol=1e-12, atol=1e-6)
            np.testing.assert_allclose(Ep_new[:, i], Ep[:, i] + dep, rtol=1e-12, atol=1e-17)
        else:
            assert flag[i] == 2
            np.testing.assert_allclose(S[:, i], c / eta * C.IOTA, rtol=1e-12, atol=1e-9)
            assert np.abs(DS[:, :, i]).max() == 0.0
            np.testing.assert_allclose(Ep_new[:, i], E[:, i] - c / (3 * K * eta) * C.IOTA, rtol=1e-12, atol=1e-17)


def test_dp_apex_without_dilatancy_or_hardening_is_an_error():
    E = np.zeros((6, 1))
    E[:3] = 1e-2                       # strong hydrostatic tension -> apex
    eta, c, _ = C.dp_parameters(450.0, math.radians(20), 0.0, 3)
    *_, err = C.drucker_prager(E, np.zeros((6, 1)), np.zeros(1), K, G, eta, c, 0.0, 0.0)
    assert err[0] == C.ERR_RETURN_MAP


def test_plane_strain_first_yield_closed_form():
    """Homogeneous plane-strain column: first yield at t = 450/sqrt(1 - nu + nu^2)."""
    from oracle.newton import homogeneous_column
    from synthetic import vm_iso_material
    from synthetic.problems import first_yield_traction_vm
    mat = vm_iso_material()
    t_y = 450.0 / math.sqrt(1 - NU + NU * NU)
    assert abs(first_yield_traction_vm(mat.E, mat.nu, mat.Y) - t_y) < 1e-9
    below = homogeneous_column(mat, [t_y * (1 - 1e-9)])
    above = homogeneous_column(mat, [t_y * (1 + 1e-9)])
    assert below[0]["plastic"] == 0 and above[0]["plastic"] == 1
    # elastic plane strain: sigma_33 = nu * (sigma_11 + sigma_22)
    assert abs(below[0]["stress"][3] - NU * (-t_y * (1 - 1e-9))) < 1e-9


def test_plane_strain_dp_limit_traction():
    """psi = 0: the column's traction tends to 2c/(1-eta) with sigma_33 -> -t/2."""
    from oracle.newton import homogeneous_column
    from synthetic.problems import Material, DP, plane_strain_limit_traction_dp
    mat = Material(DP, E=E_MOD, nu=NU, c0=450.0, phi=math.radians(20.0), psi=0.0)
    t_lim = plane_strain_limit_traction_dp(mat.c0, mat.phi)
    eta, c, _ = C.dp_parameters(450.0, math.radians(20.0), 0.0, 2)
    assert abs(t_lim - 2 * c / (1 - eta)) < 1e-9
    ts = t_lim * np.concatenate([np.linspace(0.05, 0.95, 19), [0.99, 0.999, 0.9999]])
    out = homogeneous_column(mat, ts)
    e22 = np.array([o["strain"][1] for o in out])
    # secant compliance blows up near the limit
    slope_far = (e22[10] - e22[9]) / (ts[10] - ts[9])
    slope_near = (e22[-1] - e22[-2]) / (ts[-1] - ts[-2])
    assert abs(slope_near) > 50 * abs(slope_far)
    assert abs(out[-1]["stress"][3] / ts[-1] + 0.5) < 2e-3
