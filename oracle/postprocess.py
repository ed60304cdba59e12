"""Post-processing of crack-controlled runs (test infrastructure only, plain NumPy).

effective_toughness: Eq. JaviGc, G_Ceff(f) = (1/L_g) int Sigma_M : f dE, as the area under
    the (E, Sigma:f) curve.  reading: Sigma_M is a volume average, so the external work of the
    cell is |Omega| int Sigma:f dE; the per-length toughness divides that by L_g.
amplification_factor: the appendix's Fourier-series crack length of the optimal AT2 profile.
    reading: the profile is exp(-|x|/l) (the minimiser of Eq. CrackLenght; the printed
    exp(-|x-a|/(2l)) has a garbled factor) sampled on N voxels of size h = 1, and the
    Fourier sum is |phi_hat_k|^2 / N^2 [1/(2l) + (l/2) (2 pi k / L)^2] L (Parseval; the printed
    "[1 + (i 2 pi k j l / L)^2]" is garbled).  A = Gamma_h / Gamma_continuum.
"""
from __future__ import annotations

import numpy as np

from . import fourier


def effective_toughness(E, sigma_f, area, length):
    """(area / length) * int_0^{E_end} Sigma:f dE by the trapezoid rule over the points of
    the load path, starting from the unloaded state (E, Sigma:f) = (0, 0)."""
    E = np.concatenate([[0.0], np.asarray(E, float)])
    S = np.concatenate([[0.0], np.asarray(sigma_f, float)])
    work = np.sum(0.5 * (S[1:] + S[:-1]) * (E[1:] - E[:-1]))
    return float(area * work / length)


def amplification_factor(ell_h, N=257):
    """Gamma of the sampled optimal profile on an N-voxel periodic line over its continuum
    value (appendix, Fig. A1c / the fit f_ad = 1 + a / (l/h))."""
    ell = float(ell_h)
    x = np.arange(N)
    d = np.minimum(x, N - x).astype(float)
    phi = np.exp(-d / ell).reshape(N, 1)
    gam_h = fourier.crack_length(phi, ell, fourier.xi_squared((N, 1)))
    # continuum value of the periodic profile: phi^2/(2l) + l/2 phi'^2 = exp(-2|x|/l)/l, whose
    # integral over one period [-N/2, N/2] is 1 - exp(-N/l)  (1 on the infinite line)
    gam_c = 1.0 - np.exp(-N / ell)
    return gam_h / gam_c
