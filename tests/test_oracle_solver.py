"""Pins of the oracle's residual, linearisation and Newton-Krylov loop (Sec. 3.2,
Algorithm 2) against finite differences, closed forms and dense brute force."""
import math

import numpy as np
import pytest

from oracle import dense, fourier, material, solver
from paper_2412_17445_gb300 import microstructure as ms


def _fd_errors(shape, seed, control, isotropic=False):
    """Max |(F(q+h v) - F(q-h v))/2h - J v| per block, for h = 1e-5 and 1e-6."""
    inp = ms.random_rve(shape, seed)
    pb = solver.problem_from_input(inp, isotropic=isotropic)
    eps, E, phi, H = ms.random_state(inp, seed + 1)
    de, dp, dE = ms.random_direction(inp, seed + 2)
    dq = (de, dp * (inp.notch == 0), dE)
    tgt = 1.0 if control == solver.CRACK else E
    lin = solver.Linearization(pb, eps, E, phi, H)
    J = solver.jacobian_apply(lin, dq, control)
    out = []
    for h in (1e-5, 1e-6):
        lp = solver.Linearization(pb, eps + h * de, E + h * dE, phi + h * dq[1], H)
        lm = solver.Linearization(pb, eps - h * de, E - h * dE, phi - h * dq[1], H)
        Fp = solver.residual(lp, control, tgt)
        Fm = solver.residual(lm, control, tgt)
        out.append([np.max(np.abs((np.asarray(Fp[i]) - np.asarray(Fm[i])) / (2 * h) - np.asarray(J[i])))
                    / max(np.max(np.abs(np.asarray(J[i]))), 1e-300) for i in range(3)])
    return np.array(out)


@pytest.mark.parametrize("shape", [(8, 8), (6, 10), (4, 4, 4)])
@pytest.mark.parametrize("control", [solver.CRACK, solver.STRAIN])
@pytest.mark.parametrize("isotropic", [False, True])
def test_jacobian_matches_central_differences(shape, control, isotropic):
    """Eq. CrackLength_linearization is the derivative of Eq. System_CrackLength:
    the central-difference error is O(h^2) (shrinks ~100x from h = 1e-5 to 1e-6)."""
    err = _fd_errors(shape, 11, control, isotropic)
    assert np.all(err[1] < 1e-7), err
    assert np.all((err[1] < 0.05 * err[0]) | (err[1] < 1e-9)), err


def test_newton_block_symmetric_on_compatible_space():
    """With chi_H = 1 everywhere and a homogeneous toughness the unscaled (eps, phi) block is
    self-adjoint on compatible strains: <x, J y> = <J x, y> (the couplings -2(1-phi) sig0+
    appear in both rows).  With Gc(x) varying, Gc(x) l L is not self-adjoint (Eq. System_
    CrackLength multiplies the Laplacian pointwise), so the toughness is made uniform here."""
    shape = (6, 6)
    inp = ms.random_rve(shape, 3)
    inp.Gc = np.full_like(inp.Gc, 1e-3)
    pb = solver.problem_from_input(inp)
    eps, E, phi, _ = ms.random_state(inp, 4)
    lin = solver.Linearization(pb, eps, E, phi, np.zeros(shape))
    assert np.all(lin.chi == 1.0)
    B = dense.sym_strain_matrix(shape)
    rng = np.random.default_rng(5)

    def vec():
        e = dense.vec_to_field(B @ rng.standard_normal(B.shape[1]), shape)
        return (e, rng.standard_normal(shape) * (inp.notch == 0), 0.0)

    x, y = vec(), vec()
    Jx = solver.jacobian_apply(lin, x, solver.STRAIN)
    Jy = solver.jacobian_apply(lin, y, solver.STRAIN)
    lhs = np.sum(x[0] * Jy[0]) + np.sum(x[1] * Jy[1])
    rhs = np.sum(Jx[0] * y[0]) + np.sum(Jx[1] * y[1])
    assert abs(lhs - rhs) < 1e-12 * max(abs(lhs), 1.0)


@pytest.mark.parametrize("shape", [(8, 8), (4, 4, 4)])
def test_uniform_strain_closed_form(shape):
    """Homogeneous, unnotched RVE under strain control: eps_tilde = 0, phi uniform
    = 2 psi+/(Gc/l + 2 psi+) (Eq. Helm2 with H = psi+), Sigma = g sig0+ + sig0-."""
    d = len(shape)
    E_mod, nu, Gc, ell = 1.0, 0.3, 1e-3, 2.0
    f = np.zeros((d, d))
    f[1, 1] = 1.0
    f[0, 0] = -0.2
    pb = solver.Problem(shape, np.zeros(shape, np.uint8), [E_mod], [nu], [Gc], ell,
                        np.zeros(shape, np.uint8), f)
    st = solver.initial_state(pb)
    Et = 0.02
    r, rec = solver.strain_increment(pb, st, Et, solver.Options(newton_tol=1e-12))
    assert r.converged
    lam, mu = material.lame(E_mod, nu)
    eps = f * Et
    z = np.linalg.eigvalsh(eps)
    tr = np.trace(eps)
    psi = 0.5 * lam * max(tr, 0) ** 2 + mu * np.sum(np.maximum(z, 0) ** 2)
    phi = 2 * psi / (Gc / ell + 2 * psi)
    assert np.max(np.abs(st.phi - phi)) < 1e-10
    assert np.max(np.abs(st.eps_t)) < 1e-12
    sp = lam * max(tr, 0) * np.eye(d) + 2 * mu * np.diag(np.maximum(np.diag(eps), 0))
    sm = lam * min(tr, 0) * np.eye(d) + 2 * mu * np.diag(np.minimum(np.diag(eps), 0))
    Sig = (1 - phi) ** 2 * sp + sm
    assert np.allclose(rec["Sigma"], Sig, rtol=1e-10, atol=1e-14)


@pytest.mark.parametrize("load", ["parallel", "normal"])
def test_laminate_closed_form(load):
    """Layers normal to x: the discrete solution equals the exact piecewise-constant one."""
    shape = (6, 12)
    x = np.arange(12)[None, :] * np.ones((6, 1), int)
    phase = (x < 5).astype(np.uint8)
    E = np.array([1.0, 7.0])
    nu = np.array([0.3, 0.2])
    f = np.zeros((2, 2))
    if load == "parallel":
        f[1, 1] = 1.0
    else:
        f[0, 0] = 1.0
    pb = solver.Problem(shape, phase, E, nu, [1e-3, 1e-3], 2.0, np.zeros(shape, np.uint8), f)
    Et = 1e-3
    eps_t = solver.solve_mechanical(pb, np.zeros(shape), Et)
    eps = eps_t + f * Et
    lam, mu = material.lame(E, nu)
    C = lam + 2 * mu
    v = np.array([np.mean(phase == 0), np.mean(phase == 1)])
    if load == "parallel":
        S = Et * np.sum(v * lam / C) / np.sum(v / C)
        exx = (S - lam * Et) / C
        eyy = np.array([Et, Et])
    else:
        S = Et / np.sum(v / C)
        exx = S / C
        eyy = np.zeros(2)
    for p in (0, 1):
        m = phase == p
        assert np.max(np.abs(eps[m][:, 0, 0] - exx[p])) < 1e-14
        assert np.max(np.abs(eps[m][:, 1, 1] - eyy[p])) < 1e-14
        assert np.max(np.abs(eps[m][:, 0, 1])) < 1e-14


@pytest.mark.parametrize("N,ell", [(32, 2.0), (48, 3.0), (64, 1.5)])
def test_at2_profile_is_discrete_green_function(N, ell):
    """A through-crack (notch row y = 0) at E = 0: the phase field solves
    (1/l + l L) phi = 0 off the crack with phi = 1 on it, i.e. phi = G(y)/G(0) with the
    discrete Green function G(y) = (1/N) sum_k e^{i xi_k y} / (1/l + l xi_k^2)."""
    shape = (N, 4)
    notch = np.zeros(shape, np.uint8)
    notch[0, :] = 1
    pb = solver.Problem(shape, np.zeros(shape, np.uint8), [1.0], [0.3], [1e-3], ell, notch,
                        ms.tensile_f(2))
    st = solver.initial_state(pb)
    r = solver.newton(pb, st, solver.STRAIN, 0.0, solver.Options(newton_tol=1e-13))
    assert r.converged
    k = np.fft.fftfreq(N) * N
    xi = 2 * np.pi * k / N
    y = np.arange(N)
    G = np.real(np.exp(1j * np.outer(y, xi)) @ (1.0 / (1.0 / ell + ell * xi * xi))) / N
    prof = G / G[0]
    assert np.max(np.abs(st.phi[:, 0] - prof)) < 1e-11
    assert np.max(np.abs(st.phi - st.phi[:, :1])) < 1e-13


def test_at2_profile_continuum_limit():
    """For l >> h the discrete profile approaches the periodic minimiser of the AT2
    functional, cosh((L/2 - |y|)/l) / cosh(L/(2 l))  (the exp(-|y|/l) profile)."""
    N, ell = 256, 12.0
    k = np.fft.fftfreq(N) * N
    xi = 2 * np.pi * k / N
    y = np.arange(N)
    G = np.real(np.exp(1j * np.outer(y, xi)) @ (1.0 / (1.0 / ell + ell * xi * xi))) / N
    prof = G / G[0]
    yy = np.minimum(y, N - y)
    exact = np.cosh((N / 2 - yy) / ell) / np.cosh(N / (2 * ell))
    assert np.max(np.abs(prof - exact)) < 0.02
    # and the crack length per unit length tends to tanh(L / 2l) -> 1
    shape = (N, 1)
    gam = fourier.crack_length(prof.reshape(shape), ell, fourier.xi_squared(shape))
    assert abs(gam - math.tanh(N / (2 * ell))) < 0.05


def test_dense_newton_equals_newton_krylov():
    """The converged increment does not depend on the linear solver: Newton with dense
    exact solves (restricted to compatible strains) == Newton-BiCGStab."""
    shape = (8, 8)
    inp = ms.random_rve(shape, 21)
    pb = solver.problem_from_input(inp)
    opt = solver.Options(newton_tol=1e-12, krylov_tol=1e-12)
    st_k, res_k, _ = solver.startup(pb, opt)
    assert all(r.converged for r in res_k)
    st_d, res_d, _ = solver.startup(pb, opt, linear_solver=dense.restricted_solver(shape, 2))
    assert all(r.converged for r in res_d)
    for _ in range(2):
        rk, reck = solver.crack_increment(pb, st_k, 1.0, opt)
        rd, recd = solver.crack_increment(pb, st_d, 1.0, opt, dense.restricted_solver(shape, 2))
        assert rk.converged and rd.converged
        assert abs(reck["E"] - recd["E"]) < 1e-9 * abs(recd["E"])
        assert np.max(np.abs(reck["Sigma"] - recd["Sigma"])) < 1e-9 * np.max(np.abs(recd["Sigma"]))
        assert np.max(np.abs(st_k.phi - st_d.phi)) < 1e-8


def test_crack_control_invariants_and_rollback():
    """Each increment ends with Gamma = tau and tau grows by da; a failed increment leaves
    the committed state untouched; history never decreases (Eq. history)."""
    inp = ms.homogeneous_panel(24, notch_len=6)
    pb = solver.problem_from_input(inp)
    opt = solver.Options()
    st, res, Es = solver.startup(pb, opt)
    assert all(r.converged for r in res[:3]) and Es > 0
    tau0 = st.tau
    H0 = st.Hn.copy()
    r, rec = solver.crack_increment(pb, st, 1.0, opt)
    assert r.converged
    assert abs(st.tau - tau0 - 1.0) < 1e-14
    assert abs(rec["Gamma"] - st.tau) < 1e-8 * st.tau
    assert np.all(st.Hn >= H0)
    snap = st.copy()
    r, rec = solver.crack_increment(pb, st, 1.0, solver.Options(newton_max=1))
    assert not r.converged and rec is None
    assert np.array_equal(st.phi, snap.phi) and st.E == snap.E and st.tau == snap.tau


def test_shadow_hash_is_splitmix64():
    """Reference outputs of SplitMix64 (state 0 -> first outputs of the generator)."""
    z = solver.splitmix64(np.array([0, 0x9E3779B97F4A7C15], dtype=np.uint64))
    assert int(z[0]) == 0xE220A8397B1DCDAF
    assert int(z[1]) == 0x6E789E6AA1B965F4


# ---- planted mistakes: each plausible error in the oracle must fail one of the pins ----

def test_planted_coupling_sign_is_caught(monkeypatch):
    monkeypatch.setattr(material, "degradation_slope", lambda phi: 2.0 * (1.0 - phi))
    err = _fd_errors((8, 8), 11, solver.CRACK)
    assert np.max(err[1]) > 1e-3


def test_planted_nonsymmetric_projector_is_caught(monkeypatch):
    def literal(n):  # the paper's printed G_ijkl = delta_ik n_j n_l
        d = n.shape[-1]
        return np.einsum("ik,...j,...l->...ijkl", np.eye(d), n, n)

    monkeypatch.setattr(fourier, "gamma_hat", literal)
    shape = (6, 8)
    G = fourier.gamma_hat(fourier.willot_direction(shape))
    tau = np.random.default_rng(1).standard_normal(shape + (2, 2))
    tau = 0.5 * (tau + np.swapaxes(tau, -1, -2))
    P = dense.compatible_projector(shape)
    pd = dense.vec_to_field(P @ dense.field_to_vec(tau), shape)
    assert np.max(np.abs(fourier.project(tau, G) - pd)) > 1e-3


def test_planted_laplacian_sign_is_caught(monkeypatch):
    orig = fourier.laplace_op
    monkeypatch.setattr(fourier, "laplace_op", lambda phi, xi2: -orig(phi, xi2))
    N, ell = 32, 2.0
    shape = (N, 4)
    notch = np.zeros(shape, np.uint8)
    notch[0, :] = 1
    pb = solver.Problem(shape, np.zeros(shape, np.uint8), [1.0], [0.3], [1e-3], ell, notch,
                        ms.tensile_f(2))
    st = solver.initial_state(pb)
    solver.newton(pb, st, solver.STRAIN, 0.0, solver.Options(newton_max=5))
    k = np.fft.fftfreq(N) * N
    xi = 2 * np.pi * k / N
    G = np.real(np.exp(1j * np.outer(np.arange(N), xi)) @ (1.0 / (1.0 / ell + ell * xi * xi))) / N
    assert not np.max(np.abs(st.phi[:, 0] - G / G[0])) < 1e-6


def test_planted_dropped_load_term_is_caught(monkeypatch):
    orig = solver.jacobian_apply

    def dropped(lin, dq, control):
        de, dp, dE = dq
        a1, a2, a3 = orig(lin, (de, dp, 0.0), control)
        return a1, a2, (float(dE) if control == solver.STRAIN else a3)

    monkeypatch.setattr(solver, "jacobian_apply", dropped)
    err = _fd_errors((8, 8), 11, solver.CRACK)
    assert np.max(err[1]) > 1e-3


def test_staggered_fixed_point_is_the_monolithic_solution():
    """Algorithm 1 (staggered, strain control) converges to the state the monolithic
    Newton reaches at the same load in the stable regime: both solve F1 = F2 = 0 with
    H = max(psi+, H^n).  (Past the peak the two may reach different branches.)"""
    inp = ms.homogeneous_panel(16, notch_len=4)
    pb = solver.problem_from_input(inp)
    opt = solver.Options(newton_tol=1e-13, krylov_tol=1e-13)
    _, _, Es = solver.startup(pb, opt)
    st = solver.initial_state(pb)
    r, _ = solver.strain_increment(pb, st, 0.6 * Es, opt)
    assert r.converged
    for f in (0.8, 1.0):
        a, b = st.copy(), st.copy()
        sweeps, rec = solver.staggered_increment(pb, a, f * Es, tol=1e-11, mech_tol=1e-10)
        r, mono = solver.strain_increment(pb, b, f * Es, opt)
        assert r.converged and sweeps > 2
        assert np.max(np.abs(a.phi - b.phi)) < 1e-10
        assert np.max(np.abs(rec["Sigma"] - mono["Sigma"])) < 1e-10 * np.max(np.abs(mono["Sigma"]))
        assert np.max(a.phi * (1 - pb.notch)) > 0.5  # the phase field does evolve


def test_phase_solve_is_the_helmholtz_solution():
    """solve_phase satisfies F2 = 0 (free voxels) and phi = 1 on the notch; a dropped
    Laplacian term would fail the residual check."""
    inp = ms.homogeneous_panel(16, notch_len=4)
    pb = solver.problem_from_input(inp)
    H = 1e-4 * np.random.default_rng(3).random(pb.shape)
    phi = solver.solve_phase(pb, H)
    F2 = (pb.Gc / pb.ell + 2 * H) * phi + pb.Gc * pb.ell * fourier.laplace_op(phi, pb.xi2) - 2 * H
    assert np.max(np.abs(np.where(pb.notch, 0.0, F2))) < 1e-12
    assert np.all(phi[pb.notch] == 1.0)


def test_energy_balance_along_controlled_crack_path():
    """Per crack-controlled increment of a 32^2 panel, the external work |Omega| int Sigma:f dE
    (trapezoid) equals the change of the degraded elastic energy plus G_c times the change of
    Gamma, to within 5 % of the dissipated increment (the history-field model is not exactly
    variational; the gap grows slowly with crack length).  A wrong stress, energy or crack-
    length scaling breaks this by order one."""
    n = 32
    inp = ms.homogeneous_panel(n, notch_len=8)
    pb = solver.problem_from_input(inp)
    opt = solver.Options(newton_tol=1e-9, krylov_tol=1e-10)
    st, _, _ = solver.startup(pb, opt)
    Gc = float(np.min(pb.Gc))

    def state_energies():
        eps = st.eps_t + pb.f * st.E
        sig, _, parts = material.stress(eps, st.phi, pb.lam, pb.mu, pb.k_res, pb.isotropic)
        g = material.degradation(st.phi, pb.k_res)
        e_el = float(np.sum(g * parts["psi_p"] + parts["psi_m"]))
        s_f = float(np.sum(sig.reshape(-1, 2, 2).mean(axis=0) * pb.f))
        return st.E, s_f, e_el, fourier.crack_length(st.phi, pb.ell, pb.xi2)

    prev = None
    for _ in range(8):
        _, rec = solver.crack_increment(pb, st, 1.0, opt)
        assert rec is not None
        cur = state_energies()
        if prev is not None:
            dW = n * n * 0.5 * (cur[1] + prev[1]) * (cur[0] - prev[0])
            dD = Gc * (cur[3] - prev[3])
            assert abs(dW - (cur[2] - prev[2]) - dD) < 0.05 * dD
        prev = cur


def test_crack_control_coincides_with_strain_control_in_stable_stage():
    """Before the peak the equilibrium path is unique (Sec. 4.2): a strain-controlled solve
    at the load factor a crack-controlled increment found, from the same committed state,
    lands on the same fields, stress and crack length."""
    inp = ms.homogeneous_panel(32, notch_len=8)
    pb = solver.problem_from_input(inp)
    opt = solver.Options(newton_tol=1e-11, krylov_tol=1e-12)
    st, _, _ = solver.startup(pb, opt)
    for _ in range(2):
        snap = st.copy()
        _, rec = solver.crack_increment(pb, st, 1.0, opt)
        assert rec is not None
        _, rec_s = solver.strain_increment(pb, snap, st.E, opt)
        assert rec_s is not None
        assert np.max(np.abs(snap.phi - st.phi)) < 1e-9
        assert np.max(np.abs(rec_s["Sigma"] - rec["Sigma"])) < 1e-9 * np.max(np.abs(rec["Sigma"]))
        assert abs(rec_s["Gamma"] - rec["tau"]) < 1e-9 * rec["tau"]


def test_accepted_newton_iterates_are_roots():
    """The acceptance rule (a posteriori estimate theta / (1 - theta) err, R23) ends Newton
    without evaluating F at the accepted iterate.  Pinned against the definition of a root of
    Eq. System_CrackLength: at the committed state after each of three crack increments
    (i) the scaled residual, evaluated afresh, is at most 1e-7 of the reference norm, and
    (ii) one more Newton step with an exact (dense) solve, the step the rule skipped, moves
    phi, E and the strain by less than 10 x the Newton tolerance."""
    shape = (8, 8)
    inp = ms.random_rve(shape, 21)
    pb = solver.problem_from_input(inp)
    tol = 1e-8
    opt = solver.Options(newton_tol=tol, krylov_tol=1e-12)
    st, res, _ = solver.startup(pb, opt)
    assert all(r.converged for r in res)
    exact = dense.restricted_solver(shape, 2)
    for _ in range(3):
        r, rec = solver.crack_increment(pb, st, 1.0, opt)
        assert r.converged and rec["cutbacks"] == 0
        lin = solver.Linearization(pb, st.eps_t, st.E, st.phi, st.Hn)
        F1, F2, F3 = solver.residual(lin, solver.CRACK, st.tau)
        s1, s2, s3 = solver.scales(lin, solver.CRACK)
        sf = math.sqrt(float(np.sum((s1 * F1) ** 2) + np.sum((s2 * F2) ** 2)) + (s3 * F3) ** 2)
        assert sf <= 1e-7 * lin.reference_norm(solver.CRACK, st.tau), sf
        trial = st.copy()
        one = solver.newton(pb, trial, solver.CRACK, st.tau, solver.Options(newton_tol=0.0, newton_max=1), exact)
        assert one.iterations == 1
        eps0 = st.eps_t + pb.f * st.E
        d_eps = np.linalg.norm(trial.eps_t - st.eps_t) / np.linalg.norm(eps0)
        d_phi = np.linalg.norm(trial.phi - st.phi) / np.linalg.norm(st.phi)
        d_E = abs(trial.E - st.E) / abs(st.E)
        assert max(d_eps, d_phi, d_E) < 10 * tol, (d_eps, d_phi, d_E)


def test_startup_ramp_stops_where_its_definition_says():
    """Start-up (R13, strain control before crack control) against its definition:
    (b, c) the first committed load is E_s = E_p sqrt(startup_beta / r_p), the elastic
    extrapolation from the probe load E_p = 1e-3 sqrt(min(Gc / l) / C_ref), where r_p is
    max over free voxels of 2 psi+ / (Gc / l) (checked on fresh strain-controlled solves; at
    E_s itself the ratio is startup_beta up to the phase field's response to the load, within
    10 %); (d) the ramp multiplies E by ramp_factor per committed step and stops at the first
    load whose crack length exceeds the one at E_s by ramp_gamma (the step before did not);
    (e) tau_0 = Gamma of the final state, a root of the strain-controlled system."""
    inp = ms.homogeneous_panel(24, notch_len=6)
    pb = solver.problem_from_input(inp)
    opt = solver.Options(newton_tol=1e-10)
    st, res, Es = solver.startup(pb, opt)
    assert all(r.converged for r in res)
    # (b, c) fresh solves at E = 0, the probe load and E_s, history not yet committed
    s0 = solver.initial_state(pb)
    assert solver.newton(pb, s0, solver.STRAIN, 0.0, opt).converged
    Ep = 1e-3 * math.sqrt(float(np.min(pb.Gc / pb.ell)) / pb.C_ref)
    assert solver.newton(pb, s0, solver.STRAIN, Ep, opt).converged
    rp = solver.max_drive_ratio(pb, s0)
    assert abs(Es - Ep * math.sqrt(opt.startup_beta / rp)) <= 1e-12 * Es
    assert solver.newton(pb, s0, solver.STRAIN, Es, opt).converged
    assert abs(solver.max_drive_ratio(pb, s0) / opt.startup_beta - 1.0) < 0.1
    g0 = fourier.crack_length(s0.phi, pb.ell, pb.xi2)
    # (d) the final load is E_s * ramp_factor^k and the ramp stopped at the first k with growth >= ramp_gamma
    k = round(math.log(st.E / Es) / math.log(opt.ramp_factor))
    assert k >= 1 and abs(st.E - Es * opt.ramp_factor ** k) < 1e-12 * st.E
    assert len(res) == 3 + k
    g_final = fourier.crack_length(st.phi, pb.ell, pb.xi2)
    assert g_final - g0 >= opt.ramp_gamma
    prev = s0.copy()
    solver.commit(pb, prev)
    for _ in range(k - 1):
        assert solver.newton(pb, prev, solver.STRAIN, prev.E * opt.ramp_factor, opt).converged
        solver.commit(pb, prev)
    assert fourier.crack_length(prev.phi, pb.ell, pb.xi2) - g0 < opt.ramp_gamma
    # (e)
    assert abs(st.tau - g_final) <= 1e-14 * g_final
    lin = solver.Linearization(pb, st.eps_t, st.E, st.phi, st.Hn)
    F1, F2, _ = solver.residual(lin, solver.STRAIN, st.E)
    s1, s2, _ = solver.scales(lin, solver.STRAIN)
    sf = math.sqrt(float(np.sum((s1 * F1) ** 2) + np.sum((s2 * F2) ** 2)))
    assert sf <= 1e-8 * lin.reference_norm(solver.STRAIN, st.E), sf
