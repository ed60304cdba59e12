"""Fourier-side operators of the FFT solver, plain NumPy float64 (test infrastructure only).

Arrays are indexed [y, x] (2D plane strain) or [z, y, x] (3D); tensor indices run over
(x, y[, z]).  The forward DFT is unnormalised (numpy.fft), the inverse carries 1/n.
"""
from __future__ import annotations

import numpy as np

# FFT library of every transform below: numpy.fft (single-threaded) unless
# set_fft_workers(k) routes the same transforms through scipy.fft with k threads, the
# multi-core CPU baseline.  Either library computes the plain DFT, so the two agree to
# rounding (pinned in tests/test_oracle_fourier.py).
_WORKERS = None


def set_fft_workers(workers=None):
    """None: numpy.fft; an int k >= 1: scipy.fft with k worker threads."""
    global _WORKERS
    _WORKERS = None if workers is None else int(workers)


def fftn(a, axes=None):
    if _WORKERS is None:
        return np.fft.fftn(a, axes=axes)
    import scipy.fft
    return scipy.fft.fftn(a, axes=axes, workers=_WORKERS)


def ifftn(a, axes=None):
    if _WORKERS is None:
        return np.fft.ifftn(a, axes=axes)
    import scipy.fft
    return scipy.fft.ifftn(a, axes=axes, workers=_WORKERS)


def spatial_axes(shape):
    return tuple(range(len(shape)))


def integer_frequencies(shape):
    """Per tensor direction a (x, y[, z]) the integer wave number k_a on the grid.

    k runs over 0..N/2-1, -N/2..-1 (numpy convention; the Nyquist index is -N/2).
    Returned arrays broadcast against a field of ``shape``.
    """
    d = len(shape)
    ks = []
    for a in range(d):  # a = 0 is x = last array axis
        ax = d - 1 - a
        N = shape[ax]
        k = np.fft.fftfreq(N) * N
        sh = [1] * d
        sh[ax] = N
        ks.append(k.reshape(sh))
    return ks


def standard_xi(shape):
    """Standard frequencies xi_a = 2 pi k_a / N_a (h = 1), used by the Helmholtz operator
    (Sec. 3.1: standard frequencies for the phase-field problem)."""
    d = len(shape)
    ks = integer_frequencies(shape)
    return [2.0 * np.pi * ks[a] / shape[d - 1 - a] for a in range(d)]


def xi_squared(shape):
    """|xi|^2 on the full grid.  reading: the paper's xi.xi in Eq. LinearOpe_Helm is the
    square of the derivative symbol i xi, i.e. -|xi|^2; the operator used here is |xi|^2."""
    xs = standard_xi(shape)
    out = np.zeros(shape)
    for x in xs:
        out = out + x * x
    return out


def willot_direction(shape):
    """Unit vectors n(k) of the rotated finite-difference scheme of Willot (Sec. 3.1).

    The rotated scheme differentiates on the 2^d voxel corners; its modified frequency
    along a is proportional to sin(q_a/2) * prod_{b != a} cos(q_b/2), q = 2 pi k / N.
    The common complex phase and scale cancel in the projector, so only the direction
    matters.  n = 0 where the modified frequency vanishes (k = 0 and the checkerboard
    modes).  Returns an array of shape ``shape + (d,)``.
    """
    d = len(shape)
    ks = integer_frequencies(shape)
    q = [2.0 * np.pi * ks[a] / shape[d - 1 - a] for a in range(d)]
    kt = []
    for a in range(d):
        v = np.sin(q[a] / 2.0)
        for b in range(d):
            if b != a:
                v = v * np.cos(q[b] / 2.0)
        kt.append(np.broadcast_to(v, shape))
    kt = np.stack(kt, axis=-1)
    norm = np.sqrt(np.sum(kt * kt, axis=-1))
    n = np.zeros(shape + (d,))
    # cos(pi/2) evaluates to ~6e-17, so the checkerboard modes need a threshold; every
    # other mode has |k~| >= sin(pi/N) cos(pi/2 - pi/N) ~ (pi/N)^2 >> 1e-10 for N <= 4096
    nz = norm > 1e-10
    n[nz] = kt[nz] / norm[nz][:, None]
    return n


def continuous_direction(shape):
    """Unit vectors n = xi / |xi| of the continuous (standard) frequencies, the Galerkin
    projection of Sec. 3.1 without the rotated scheme.

    reading: at the Nyquist index of an even axis the frequency has no sign for a real
    field, so its component of the derivative symbol is taken as 0 there (the projector
    then stays real-symmetric per frequency); n = 0 where that symbol vanishes.  Returns an
    array of shape ``shape + (d,)``.
    """
    d = len(shape)
    ks = integer_frequencies(shape)
    comps = []
    for a in range(d):
        N = shape[d - 1 - a]
        k = np.asarray(ks[a], dtype=float)
        xi = 2.0 * np.pi * k / N
        if N % 2 == 0:
            xi = np.where(np.abs(k) == N // 2, 0.0, xi)
        comps.append(np.broadcast_to(xi, shape))
    xi = np.stack(comps, axis=-1)
    norm = np.sqrt(np.sum(xi * xi, axis=-1))
    n = np.zeros(shape + (d,))
    nz = norm > 0.0
    n[nz] = xi[nz] / norm[nz][:, None]
    return n


def gamma_hat(n):
    """Fourth-order Galerkin projection per frequency (Eq. GFourier, symmetric reading).

    reading: the paper's G_ijkl = delta_ik xi_j xi_l / |xi|^2 is not symmetric, while the
    unknowns are symmetric strains; the orthogonal projector onto compatible symmetric
    strains is used:
        G_ijkl = 1/2 (d_ik n_j n_l + d_il n_j n_k + d_jk n_i n_l + d_jl n_i n_k) - n_i n_j n_k n_l
    and G = 0 where n = 0 (the zero frequency).
    """
    d = n.shape[-1]
    I = np.eye(d)
    t1 = np.einsum("ik,...j,...l->...ijkl", I, n, n)
    t2 = np.einsum("il,...j,...k->...ijkl", I, n, n)
    t3 = np.einsum("jk,...i,...l->...ijkl", I, n, n)
    t4 = np.einsum("jl,...i,...k->...ijkl", I, n, n)
    t5 = np.einsum("...i,...j,...k,...l->...ijkl", n, n, n, n)
    return 0.5 * (t1 + t2 + t3 + t4) - t5


def fft_tensor(tau, shape):
    return fftn(tau, axes=spatial_axes(shape))


def ifft_tensor(tau_hat, shape):
    return ifftn(tau_hat, axes=spatial_axes(shape)).real


def project(tau, G):
    """F^-1 { G : F { tau } } for a real tensor field tau (shape + (d, d))  (Eq. LinearOpe_Mech)."""
    shape = tau.shape[:-2]
    th = fft_tensor(tau, shape)
    ph = np.einsum("...ijkl,...kl->...ij", G, th)
    return ifft_tensor(ph, shape)


def laplace_op(phi, xi2):
    """L phi = F^-1 [ |xi|^2 F[phi] ]  (= - discrete Laplacian, Eq. LinearOpe_Helm)."""
    return ifftn(xi2 * fftn(phi)).real


def crack_length(phi, ell, xi2):
    """Gamma = int phi^2/(2 l) + l/2 |grad phi|^2  (Eq. CrackLenght), h = 1.

    The gradient term is evaluated spectrally (Eq. newGammaFourier) through Parseval:
    sum_v |F^-1(i xi phi_hat)|^2 = (1/n) sum_k |xi_k|^2 |phi_hat_k|^2.
    reading: the same |xi|^2 as the Helmholtz operator (Nyquist xi = pi) so that the
    linearised constraint (Eq. CrackLength_linearization, Delta F3) is its exact derivative.
    """
    n = phi.size
    ph = fftn(phi)
    grad2 = np.sum(xi2 * (ph.real ** 2 + ph.imag ** 2)) / n
    return float(np.sum(phi * phi) / (2.0 * ell) + 0.5 * ell * grad2)


def derivative_symbols(shape):
    """Per direction a (x, y[, z]) the multiplier s_a(k) of the spectral derivative D_a of
    Eq. newGammaFourier: i xi_a with the standard frequencies, except at the Nyquist index of
    an even axis, where it is the real |xi_a| = pi.
    reading: a real field's Nyquist coefficient carries no sign, so i xi there would leave
    the real fields; the real multiplier keeps D_a phi real and keeps Parseval exact,
    sum_v sum_a (D_a phi)^2 = (1/n) sum_k |xi_k|^2 |phi_hat_k|^2, so for homogeneous G_c the
    dissipation below is exactly G_c times crack_length."""
    d = len(shape)
    ks = integer_frequencies(shape)
    xs = standard_xi(shape)
    out = []
    for a in range(d):
        N = shape[d - 1 - a]
        nyq = (N % 2 == 0) & (np.abs(ks[a]) == N // 2)
        s = np.where(nyq, np.abs(xs[a]) + 0j, 1j * xs[a])
        out.append(np.broadcast_to(s, shape))
    return out


def spectral_gradient(phi):
    """[D_a phi for each direction a] = F^-1[s_a F[phi]] (real fields): the gradient
    F^-1(xi phi_hat) of Eq. newGammaFourier."""
    ph = fftn(phi)
    return [ifftn(s * ph).real for s in derivative_symbols(phi.shape)]


def spectral_gradient_adjoint(g):
    """sum_a D_a^T g_a = sum_a F^-1[conj(s_a) F[g_a]], the adjoint of spectral_gradient in
    the plain voxel sum (F / sqrt(n) is unitary)."""
    syms = derivative_symbols(g[0].shape)
    acc = np.zeros(g[0].shape, dtype=complex)
    for s, ga in zip(syms, g):
        acc = acc + np.conj(s) * fftn(ga)
    return ifftn(acc).real


def dissipation(phi, Gc, ell):
    """Dissipated energy int G_c gamma_f (Eq. SystemDisc), h = 1, with gamma_f of
    Eq. newGammaFourier: phi^2/(2 l) + (l/2) sum_a (D_a phi)^2 per voxel, G_c per voxel."""
    grad = spectral_gradient(phi)
    g2 = sum(x * x for x in grad)
    return float(np.sum(Gc * (phi * phi / (2.0 * ell) + 0.5 * ell * g2)))


def dissipation_gradient(phi, Gc, ell):
    """d dissipation / d phi = G_c phi / l + l sum_a D_a^T (G_c D_a phi) per voxel: the
    constraint row Delta F3 of Eq. CrackLength_linearization under energy control (reading:
    the exact derivative; the printed row G_c (phi / l + l L phi) equals it only for
    homogeneous G_c)."""
    grad = spectral_gradient(phi)
    return Gc * phi / ell + ell * spectral_gradient_adjoint([Gc * x for x in grad])
