"""Post-processing of crack-controlled runs (test infrastructure only, plain NumPy).

effective_toughness: Eq. JaviGc, G_Ceff(f) = (1/L_g) int Sigma_M : f dE, as the area under
    the (E, Sigma:f) curve.  reading: Sigma_M is a volume average, so the external work of the
    cell is |Omega| int Sigma:f dE; the per-length toughness divides that by L_g.
amplification_factor: the appendix's Fourier-series crack length of the optimal AT2 profile.
    reading: the profile is exp(-|x|/l) (the minimiser of Eq. CrackLenght; the printed
    exp(-|x-a|/(2l)) has a garbled factor) sampled on N voxels of size h = 1, and the
    Fourier sum is |phi_hat_k|^2 / N^2 [1/(2l) + (l/2) (2 pi k / L)^2] L (Parseval; the printed
    "[1 + (i 2 pi k j l / L)^2]" is garbled).  A = Gamma_h / Gamma_continuum.
rotation_2d, j_integral: the J-integral around a crack tip of a solved state, the energy
    release rate that the crack-controlled path holds near G_c A (Sec. 4 compares the
    dissipated energy with G_c; the contour form is Rice's, the paper prints none).
    reading: the displacement gradient comes from the compatible strain and the rotation
    that the compatibility relations give (standard frequencies, Nyquist component 0).
"""
from __future__ import annotations

import numpy as np

from . import fourier, material


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


def rotation_2d(eps_t):
    """(J-integral of Sec. 4.2.)  Infinitesimal rotation w = (d1 u2 - d2 u1) / 2 of the
    periodic displacement whose
    symmetric gradient is the compatible field eps_t (2D, shape (ny, nx, 2, 2)), from the
    compatibility relations d1 w = d1 e12 - d2 e11, d2 w = d1 e22 - d2 e12 in Fourier
    space with the standard frequencies (reading: the Nyquist component of xi is 0, as for
    the continuous projector); the mean rotation is 0."""
    shape = eps_t.shape[:2]
    xs = fourier.standard_xi(shape)
    xi = []
    for a in range(2):
        N = shape[1 - a]
        x = np.broadcast_to(xs[a], shape).copy()
        if N % 2 == 0:
            k = np.broadcast_to(fourier.integer_frequencies(shape)[a], shape)
            x = np.where(np.abs(k) == N // 2, 0.0, x)
        xi.append(x)
    e11, e12, e22 = (fourier.fftn(eps_t[..., i, j]) for i, j in ((0, 0), (0, 1), (1, 1)))
    num = xi[0] * (xi[0] * e12 - xi[1] * e11) + xi[1] * (xi[0] * e22 - xi[1] * e12)
    x2 = xi[0] ** 2 + xi[1] ** 2
    w_hat = np.where(x2 > 0.0, num / np.where(x2 > 0.0, x2, 1.0), 0.0)
    return fourier.ifftn(w_hat).real


def j_integral(pb, st, box):
    """The J-integral check of Sec. 4.2 (energy release rate during controlled propagation).
    J = closed-contour sum of (W n_1 - sigma_ij n_j d1 u_i) ds around a crack tip
    (Rice's J in the x direction, plane strain, h = 1), for the rectangle of voxel centres
    box = (x0, y0, x1, y1) traversed once, outward normals, each voxel of a side weighted
    by its length (corners count half on each of their two sides).  W = g psi0+ + psi0- is
    the degraded energy density, sigma the degraded stress; d1 u = E f e_1 + d1 u~ with
    d1 u~_1 = e~11 and d1 u~_2 = e~12 + w (rotation_2d)."""
    x0, y0, x1, y1 = box
    eps = st.eps_t + pb.f * st.E
    sig, _, parts = material.stress(eps, st.phi, pb.lam, pb.mu, pb.k_res, pb.isotropic)
    g = material.degradation(st.phi, pb.k_res)
    W = g * (parts["psi_p"] + parts["psi_m"]) if pb.isotropic else g * parts["psi_p"] + parts["psi_m"]
    w = rotation_2d(st.eps_t)
    du1 = st.E * pb.f[0, 0] + st.eps_t[..., 0, 0]
    du2 = st.E * pb.f[1, 0] + st.eps_t[..., 0, 1] + w
    J = 0.0
    sides = [  # (fixed coordinate, range, normal, along-x?)
        ("x", x1, range(y0, y1 + 1), (1.0, 0.0)),
        ("y", y1, range(x0, x1 + 1), (0.0, 1.0)),
        ("x", x0, range(y0, y1 + 1), (-1.0, 0.0)),
        ("y", y0, range(x0, x1 + 1), (0.0, -1.0)),
    ]
    for kind, c, rng, (n1, n2) in sides:
        pts = list(rng)
        for i, t in enumerate(pts):
            wgt = 0.5 if i in (0, len(pts) - 1) else 1.0
            y, x = (t, c) if kind == "x" else (c, t)
            s = sig[y, x]
            t1 = s[0, 0] * n1 + s[0, 1] * n2
            t2 = s[1, 0] * n1 + s[1, 1] * n2
            J += wgt * (W[y, x] * n1 - (t1 * du1[y, x] + t2 * du2[y, x]))
    return float(J)
