"""Pins of the energy-controlled constraint (Eq. SystemDisc with gamma_f of Eq.
newGammaFourier): the spectral derivative against closed forms and dense DFT matrices, the
dissipation against G_c times the crack length for homogeneous G_c, its gradient against
exact central differences, and energy control against length control."""
import numpy as np
import pytest

from oracle import dense, fourier, solver
from paper_2412_17445_gb300 import microstructure as ms


@pytest.mark.parametrize("k", [1, 3, 7, 8])
def test_derivative_of_single_modes(k):
    """D_x cos(2 pi k x / N) = -(2 pi k / N) sin(2 pi k x / N) and D_y of it is 0; at the
    Nyquist mode (k = N/2) the real multiplier gives D_x (-1)^x = pi (-1)^x."""
    ny, nx = 6, 16
    x = np.arange(nx)[None, :] * np.ones((ny, 1))
    phi = np.cos(2 * np.pi * k * x / nx)
    dx, dy = fourier.spectral_gradient(phi)
    q = 2 * np.pi * k / nx
    expect = np.pi * phi if 2 * k == nx else -q * np.sin(q * x)
    assert np.max(np.abs(dx - expect)) < 1e-13
    assert np.max(np.abs(dy)) < 1e-13


def test_derivative_along_z_in_3d():
    shape = (8, 4, 6)
    z = np.arange(8)[:, None, None] * np.ones(shape)
    phi = np.sin(2 * np.pi * 3 * z / 8)
    dx, dy, dz = fourier.spectral_gradient(phi)
    assert np.max(np.abs(dz - 2 * np.pi * 3 / 8 * np.cos(2 * np.pi * 3 * z / 8))) < 1e-13
    assert max(np.max(np.abs(dx)), np.max(np.abs(dy))) < 1e-13


@pytest.mark.parametrize("shape", [(4, 6), (5, 4), (3, 5)])
def test_gradient_and_adjoint_equal_dense_matrices(shape):
    """D_a from dense DFT matrices (Kronecker products, real Nyquist multiplier) and its
    transpose as the adjoint."""
    ny, nx = shape
    rng = np.random.default_rng(3)
    phi = rng.standard_normal(shape)
    Dx = np.kron(np.eye(ny), dense.spectral_derivative_1d(nx, nyquist="real"))
    Dy = np.kron(dense.spectral_derivative_1d(ny, nyquist="real"), np.eye(nx))
    dx, dy = fourier.spectral_gradient(phi)
    assert np.max(np.abs(dx.reshape(-1) - Dx @ phi.reshape(-1))) < 1e-12
    assert np.max(np.abs(dy.reshape(-1) - Dy @ phi.reshape(-1))) < 1e-12
    g = [rng.standard_normal(shape) for _ in range(2)]
    adj = fourier.spectral_gradient_adjoint(g)
    assert np.max(np.abs(adj.reshape(-1) - (Dx.T @ g[0].reshape(-1) + Dy.T @ g[1].reshape(-1)))) < 1e-12


@pytest.mark.parametrize("shape", [(8, 8), (6, 10), (5, 7), (4, 6, 2), (3, 5, 4)])
def test_homogeneous_dissipation_is_gc_times_crack_length(shape):
    rng = np.random.default_rng(4)
    phi = rng.random(shape)
    Gc, ell = 2.7e-3, 1.5
    xi2 = fourier.xi_squared(shape)
    D = fourier.dissipation(phi, np.full(shape, Gc), ell)
    assert abs(D - Gc * fourier.crack_length(phi, ell, xi2)) < 1e-13 * abs(D)
    w = fourier.dissipation_gradient(phi, np.full(shape, Gc), ell)
    wl = Gc * (phi / ell + ell * fourier.laplace_op(phi, xi2))
    assert np.max(np.abs(w - wl)) < 1e-13 * np.max(np.abs(wl))


@pytest.mark.parametrize("shape", [(8, 8), (6, 10), (4, 6, 2)])
def test_dissipation_gradient_is_exact_derivative_heterogeneous(shape):
    """The dissipation is quadratic in phi, so a central difference of any step is exact
    up to rounding; with heterogeneous G_c it differs from G_c (phi/l + l L phi)."""
    rng = np.random.default_rng(5)
    phi = rng.random(shape)
    dphi = rng.standard_normal(shape)
    Gc = 1e-3 * (1.0 + 4.0 * (rng.random(shape) < 0.4))
    ell = 2.0
    w = fourier.dissipation_gradient(phi, Gc, ell)
    for h in (0.5, 1e-3):
        fd = (fourier.dissipation(phi + h * dphi, Gc, ell) - fourier.dissipation(phi - h * dphi, Gc, ell)) / (2 * h)
        assert abs(fd - np.sum(w * dphi)) < 1e-10 * np.sum(np.abs(w * dphi))
    naive = Gc * (phi / ell + ell * fourier.laplace_op(phi, fourier.xi_squared(shape)))
    assert np.max(np.abs(w - naive)) > 1e-3 * np.max(np.abs(w))


@pytest.mark.parametrize("shape", [(8, 8), (6, 10), (4, 4, 4)])
def test_energy_jacobian_matches_central_differences(shape):
    """The bordered Jacobian under energy control is the derivative of F (heterogeneous
    G_c): central-difference error O(h^2)."""
    inp = ms.random_rve(shape, 21)
    pb = solver.problem_from_input(inp, constraint="energy")
    eps, E, phi, H = ms.random_state(inp, 22)
    de, dp, dE = ms.random_direction(inp, 23)
    dq = (de, dp * (inp.notch == 0), dE)
    lin = solver.Linearization(pb, eps, E, phi, H)
    J = solver.jacobian_apply(lin, dq, solver.CRACK)
    errs = []
    for h in (1e-5, 1e-6):
        lp = solver.Linearization(pb, eps + h * de, E + h * dE, phi + h * dq[1], H)
        lm = solver.Linearization(pb, eps - h * de, E - h * dE, phi - h * dq[1], H)
        F3p = solver.residual(lp, solver.CRACK, 1.0)[2]
        F3m = solver.residual(lm, solver.CRACK, 1.0)[2]
        errs.append(abs((F3p - F3m) / (2 * h) - J[2]) / abs(J[2]))
    assert errs[1] < 1e-7 and (errs[1] < 0.05 * errs[0] or errs[1] < 1e-9), errs


def test_energy_control_equals_length_control_for_homogeneous_gc():
    """A homogeneous panel under energy control with tau increments G_c * da follows the
    length-controlled path (same scaled Newton systems up to rounding)."""
    inp = ms.homogeneous_panel(16, notch_len=4)
    opt = solver.Options(newton_tol=1e-10)
    runs = []
    for c in ("length", "energy"):
        pb = solver.problem_from_input(inp, constraint=c)
        st, _, _ = solver.startup(pb, opt)
        da = 1.0 if c == "length" else float(inp.Gc[0])
        recs = []
        for _ in range(2):
            r, rec = solver.crack_increment(pb, st, da, opt)
            assert rec is not None
            recs.append((rec["E"], st.phi.copy(), rec["Gamma"]))
        runs.append(recs)
    for (E1, p1, g1), (E2, p2, g2) in zip(*runs):
        assert abs(E1 - E2) < 1e-8 * abs(E1)
        assert np.max(np.abs(p1 - p2)) < 1e-7
        assert abs(g1 - g2) < 1e-8 * g1


def test_energy_controlled_increment_on_a_composite():
    """Heterogeneous G_c (fibres 5x tougher): the converged state dissipates exactly the
    prescribed energy."""
    inp = ms.fibre_composite(n=24, radius=4.0, fraction=0.3, notch_len=8)
    pb = solver.problem_from_input(inp, constraint="energy")
    opt = solver.Options(newton_tol=1e-10)
    st, _, _ = solver.startup(pb, opt)
    tau0 = st.tau
    assert abs(tau0 - fourier.dissipation(st.phi, pb.Gc, pb.ell)) < 1e-14 * tau0
    r, rec = solver.crack_increment(pb, st, 0.5 * float(np.min(pb.Gc)), opt)
    assert rec is not None
    D = fourier.dissipation(st.phi, pb.Gc, pb.ell)
    assert abs(D - st.tau) < 1e-9 * st.tau
    assert abs(st.tau - tau0 - 0.5 * float(np.min(pb.Gc))) < 1e-15 + 1e-12 * tau0


def test_planted_printed_constraint_row_is_caught(monkeypatch):
    """Replacing the exact row with the printed G_c (phi/l + l L phi) (exact only for
    homogeneous G_c) fails the central-difference check of the bordered Jacobian."""
    shape = (8, 8)
    inp = ms.random_rve(shape, 21)
    pb = solver.problem_from_input(inp, constraint="energy")
    eps, E, phi, H = ms.random_state(inp, 22)
    de, dp, dE = ms.random_direction(inp, 23)
    dq = (de, dp * (inp.notch == 0), dE)
    monkeypatch.setattr(fourier, "dissipation_gradient",
                        lambda p, Gc, ell: Gc * (p / ell + ell * fourier.laplace_op(p, fourier.xi_squared(p.shape))))
    lin = solver.Linearization(pb, eps, E, phi, H)
    J3 = solver.jacobian_apply(lin, dq, solver.CRACK)[2]
    h = 1e-6
    lp = solver.Linearization(pb, eps + h * de, E + h * dE, phi + h * dq[1], H)
    lm = solver.Linearization(pb, eps - h * de, E - h * dE, phi - h * dq[1], H)
    fd = (solver.residual(lp, solver.CRACK, 1.0)[2] - solver.residual(lm, solver.CRACK, 1.0)[2]) / (2 * h)
    assert abs(fd - J3) > 1e-4 * abs(fd)
