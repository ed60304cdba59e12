"""Pins of the oracle's Fourier-side operators (FFT conventions, Galerkin projection,
spectral Laplacian, crack length) against brute force and closed forms."""
import math

import numpy as np
import pytest

from oracle import dense, fourier

SHAPES = [(8, 8), (6, 8), (4, 4, 4), (4, 6, 2)]


def _sym(a):
    return 0.5 * (a + np.swapaxes(a, -1, -2))


@pytest.mark.parametrize("shape", [(8, 6), (4, 4, 2), (5, 3)])
def test_dft_convention_matches_dense(shape):
    x = np.random.default_rng(0).standard_normal(shape)
    assert np.allclose(np.fft.fftn(x), dense.dense_dftn(x), atol=1e-12)


@pytest.mark.parametrize("shape", SHAPES)
def test_projector_equals_dense_real_space_projector(shape):
    """Gamma-hat with Willot frequencies (Eq. GFourier, Sec. 3.1) is the orthogonal
    projector onto symmetric gradients of the rotated finite-difference scheme."""
    d = len(shape)
    P = dense.compatible_projector(shape)
    G = fourier.gamma_hat(fourier.willot_direction(shape))
    tau = _sym(np.random.default_rng(1).standard_normal(shape + (d, d)))
    pf = fourier.project(tau, G)
    pd = dense.vec_to_field(P @ dense.field_to_vec(tau), shape)
    assert np.max(np.abs(pf - pd)) < 1e-12


@pytest.mark.parametrize("shape", SHAPES)
def test_projector_idempotent_symmetric_and_kills_constants(shape):
    d = len(shape)
    rng = np.random.default_rng(2)
    G = fourier.gamma_hat(fourier.willot_direction(shape))
    a = _sym(rng.standard_normal(shape + (d, d)))
    b = _sym(rng.standard_normal(shape + (d, d)))
    pa = fourier.project(a, G)
    assert np.max(np.abs(fourier.project(pa, G) - pa)) < 1e-13
    # self-adjoint in the Frobenius metric
    assert abs(np.sum(pa * b) - np.sum(a * fourier.project(b, G))) < 1e-11
    const = np.broadcast_to(_sym(rng.standard_normal((d, d))), shape + (d, d)).copy()
    assert np.max(np.abs(fourier.project(const, G))) < 1e-14
    # symmetric per frequency: G_ijkl = G_klij = G_jikl
    assert np.allclose(G, np.swapaxes(np.swapaxes(G, -4, -2), -3, -1))
    assert np.allclose(G, np.swapaxes(G, -4, -3))


@pytest.mark.parametrize("shape", [(8, 8), (4, 4, 4)])
def test_projector_keeps_compatible_fields(shape):
    d = len(shape)
    B = dense.sym_strain_matrix(shape)
    u = np.random.default_rng(3).standard_normal(B.shape[1])
    eps = dense.vec_to_field(B @ u, shape)
    G = fourier.gamma_hat(fourier.willot_direction(shape))
    assert np.max(np.abs(fourier.project(eps, G) - eps)) < 1e-12


@pytest.mark.parametrize("shape", SHAPES + [(5, 6), (3, 5, 4)])
def test_continuous_projector_equals_dense_spectral_projector(shape):
    """Gamma-hat with continuous frequencies is the orthogonal projector onto symmetric
    gradients of the spectral derivative (dense DFT matrices, Nyquist component 0)."""
    d = len(shape)
    P = dense.compatible_projector(shape, scheme="spectral")
    G = fourier.gamma_hat(fourier.continuous_direction(shape))
    tau = _sym(np.random.default_rng(4).standard_normal(shape + (d, d)))
    pf = fourier.project(tau, G)
    pd = dense.vec_to_field(P @ dense.field_to_vec(tau), shape)
    assert np.max(np.abs(pf - pd)) < 1e-12
    # idempotent, kills constants, keeps spectral symmetric gradients
    assert np.max(np.abs(fourier.project(pf, G) - pf)) < 1e-13
    B = dense.sym_strain_matrix(shape, scheme="spectral")
    u = np.random.default_rng(5).standard_normal(B.shape[1])
    eps = dense.vec_to_field(B @ u, shape)
    assert np.max(np.abs(fourier.project(eps, G) - eps)) < 1e-12


def test_continuous_and_rotated_directions_differ_off_axis():
    """The two schemes agree on the axes and differ off them (a dropped cosine factor in
    the rotated scheme would make them equal)."""
    shape = (8, 8)
    nw, nc = fourier.willot_direction(shape), fourier.continuous_direction(shape)
    assert np.allclose(nw[0, 1], nc[0, 1]) and np.allclose(nw[2, 0], nc[2, 0])
    assert not np.allclose(nw[1, 3], nc[1, 3])
    assert np.all(nc[4, 0] == 0.0) and np.all(nc[4, 4] == 0.0)


def test_checkerboard_mode_is_dropped():
    shape = (8, 8)
    n = fourier.willot_direction(shape)
    assert np.all(n[4, 4] == 0.0) and np.all(n[0, 0] == 0.0)
    assert abs(np.linalg.norm(n[4, 1]) - 1.0) < 1e-14


@pytest.mark.parametrize("N,k", [(16, 1), (16, 3), (16, 8), (12, 5), (9, 4)])
def test_laplacian_on_cosines(N, k):
    """L cos(2 pi k x / N) = (2 pi k / N)^2 cos(...) with the standard frequencies."""
    shape = (3, N)
    x = np.arange(N)[None, :] * np.ones((3, 1))
    phi = np.cos(2 * np.pi * k * x / N)
    xi2 = fourier.xi_squared(shape)
    lap = fourier.laplace_op(phi, xi2)
    assert np.allclose(lap, (2 * np.pi * k / N) ** 2 * phi, atol=1e-12)


def test_crack_length_closed_forms():
    """Gamma (Eq. CrackLenght) for phi = const and for one Fourier mode (Parseval)."""
    ell = 2.0
    shape = (10, 16)
    n = 160
    xi2 = fourier.xi_squared(shape)
    assert abs(fourier.crack_length(np.full(shape, 0.3), ell, xi2) - n * 0.09 / (2 * ell)) < 1e-13
    k = 3
    x = np.arange(16)[None, :] * np.ones((10, 1))
    phi = np.cos(2 * np.pi * k * x / 16)
    q = 2 * np.pi * k / 16
    expect = n * (1.0 / (4 * ell) + ell / 4 * q * q)
    assert abs(fourier.crack_length(phi, ell, xi2) - expect) < 1e-12
    # y-mode in a 3D grid
    shape3 = (4, 6, 8)
    y = np.arange(6)[None, :, None] * np.ones((4, 1, 8))
    phi3 = np.sin(2 * np.pi * 2 * y / 6)
    q = 2 * np.pi * 2 / 6
    assert abs(fourier.crack_length(phi3, ell, fourier.xi_squared(shape3)) - 192 * (1 / (4 * ell) + ell / 4 * q * q)) < 1e-12


@pytest.mark.parametrize("shape", [(12, 18), (4, 6, 8)])
def test_multithreaded_fft_backend_matches_numpy(shape):
    """The multi-core baseline's backend (scipy.fft with several workers) computes the same
    DFT as numpy.fft: projection, Laplacian and crack length agree to rounding."""
    pytest.importorskip("scipy")
    rng = np.random.default_rng(3)
    d = len(shape)
    a = rng.standard_normal(shape + (d, d))
    tau = 0.5 * (a + np.swapaxes(a, -1, -2))
    phi = rng.random(shape)
    G = fourier.gamma_hat(fourier.willot_direction(shape))
    xi2 = fourier.xi_squared(shape)
    ref = (fourier.project(tau, G), fourier.laplace_op(phi, xi2), fourier.crack_length(phi, 2.0, xi2))
    try:
        fourier.set_fft_workers(4)
        got = (fourier.project(tau, G), fourier.laplace_op(phi, xi2), fourier.crack_length(phi, 2.0, xi2))
    finally:
        fourier.set_fft_workers(None)
    assert np.max(np.abs(got[0] - ref[0])) < 1e-13 * np.max(np.abs(ref[0]))
    assert np.max(np.abs(got[1] - ref[1])) < 1e-13 * np.max(np.abs(ref[1]))
    assert abs(got[2] - ref[2]) < 1e-13 * ref[2]
