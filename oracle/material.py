"""Spectral-split phase-field constitutive law, plain NumPy float64 (test infrastructure only).

Strain tensors are d x d per voxel (d = 2: plane strain with eps_zz = 0, which drops
out of the split because its eigenvalue is 0; d = 3: full 3D).
"""
from __future__ import annotations

import numpy as np


def lame(E, nu):
    """Lame constants of an isotropic phase (the same in plane strain and 3D)."""
    E = np.asarray(E, dtype=float)
    nu = np.asarray(nu, dtype=float)
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return lam, mu


def degradation(phi, k_res=0.0):
    """g(phi) = (1 - phi)^2 + k  (Eq. gFunct).

    reading: the paper prints "- k"; Miehe's residual stiffness is "+ k".  k = 0 by default.
    """
    return (1.0 - phi) ** 2 + k_res


def degradation_slope(phi):
    """g'(phi) = -2 (1 - phi)."""
    return -2.0 * (1.0 - phi)


def heaviside_pos(x):
    """H+(x) = 1 for x > 0 else 0 (reading: the Macaulay bracket's slope at 0 is 0)."""
    return (x > 0.0).astype(float)


def split(eps, lam, mu):
    """Positive/negative parts of the strain energy (Eq. PlusNegPsi).

    eps: (..., d, d) symmetric; lam, mu broadcast against eps[..., 0, 0].
    Returns dict with zeta (eigenvalues), Q (eigenvectors as columns), tr,
    psi_p, psi_m, sig_p, sig_m where sig_pm = d psi_pm / d eps.
    """
    d = eps.shape[-1]
    zeta, Q = np.linalg.eigh(eps)
    tr = np.trace(eps, axis1=-2, axis2=-1)
    zp = np.maximum(zeta, 0.0)
    zm = np.minimum(zeta, 0.0)
    trp = np.maximum(tr, 0.0)
    trm = np.minimum(tr, 0.0)
    psi_p = 0.5 * lam * trp ** 2 + mu * np.sum(zp ** 2, axis=-1)
    psi_m = 0.5 * lam * trm ** 2 + mu * np.sum(zm ** 2, axis=-1)
    eps_p = np.einsum("...ia,...a,...ja->...ij", Q, zp, Q)
    eps_m = np.einsum("...ia,...a,...ja->...ij", Q, zm, Q)
    I = np.eye(d)
    sig_p = (lam * trp)[..., None, None] * I + 2.0 * mu[..., None, None] * eps_p
    sig_m = (lam * trm)[..., None, None] * I + 2.0 * mu[..., None, None] * eps_m
    return dict(zeta=zeta, Q=Q, tr=tr, psi_p=psi_p, psi_m=psi_m, sig_p=sig_p, sig_m=sig_m,
                eps_p=eps_p, eps_m=eps_m)


def stress(eps, phi, lam, mu, k_res=0.0, isotropic=False):
    """sigma = g(phi) sigma_0^+ + sigma_0^-  (Eq. OriSystem0a, Eq. C_Calc's stress).

    isotropic=True is the "isotropic" variant (Sec. 5.2): psi = g (psi+ + psi-), no split.
    Returns (sigma, psi_p, parts); for the isotropic variant psi_p is the full energy.
    """
    parts = split(eps, lam, mu)
    g = degradation(phi, k_res)[..., None, None]
    if isotropic:
        sig0 = parts["sig_p"] + parts["sig_m"]
        return g * sig0, parts["psi_p"] + parts["psi_m"], parts
    return g * parts["sig_p"] + parts["sig_m"], parts["psi_p"], parts


def loewner_pos(zeta, rel_tol=1e-12):
    """Divided differences of the Macaulay bracket <x>+ between eigenvalues.

    L_ab = (<z_a>+ - <z_b>+) / (z_a - z_b); for |z_a - z_b| <= rel_tol * max|z| the
    limit H+((z_a + z_b)/2) is used (reading: the tie rule for coincident eigenvalues).
    This is the first divided difference of the Daleckii-Krein formula for the
    derivative of the isotropic tensor function eps -> eps^+.
    """
    za = zeta[..., :, None]
    zb = zeta[..., None, :]
    diff = za - zb
    scale = np.max(np.abs(zeta), axis=-1)[..., None, None]
    tie = np.abs(diff) <= rel_tol * scale
    safe = np.where(tie, 1.0, diff)
    dd = (np.maximum(za, 0.0) - np.maximum(zb, 0.0)) / safe
    return np.where(tie, heaviside_pos(0.5 * (za + zb)), dd)


def d_eps_pos(parts, deps):
    """Directional derivative of eps^+ along deps: Q (L o (Q^T deps Q)) Q^T."""
    Q = parts["Q"]
    L = loewner_pos(parts["zeta"])
    dt = np.einsum("...ai,...ab,...bj->...ij", Q, deps, Q)
    return np.einsum("...ia,...ab,...jb->...ij", Q, L * dt, Q)


def tangent_apply(parts, phi, lam, mu, deps, k_res=0.0, isotropic=False):
    """C : deps with C = g d2psi+/deps2 + d2psi-/deps2  (Eq. C_Calc), as a directional
    derivative of the stress, evaluated from the split of the linearisation point."""
    d = deps.shape[-1]
    I = np.eye(d)
    g = degradation(phi, k_res)
    trd = np.trace(deps, axis1=-2, axis2=-1)
    if isotropic:
        c0 = lam[..., None, None] * trd[..., None, None] * I + 2.0 * mu[..., None, None] * deps
        return g[..., None, None] * c0
    hp = heaviside_pos(parts["tr"])
    hm = 1.0 - hp
    dp = d_eps_pos(parts, deps)
    dm = deps - dp
    vol = (g * lam * hp + lam * hm) * trd
    return vol[..., None, None] * I + 2.0 * (g * mu)[..., None, None] * dp + 2.0 * mu[..., None, None] * dm
