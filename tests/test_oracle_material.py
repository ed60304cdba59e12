"""Pins of the oracle's constitutive law (Eqs. PlusNegPsi, gFunct, C_Calc)."""
import numpy as np
import pytest

from oracle import material


def _sym(a):
    return 0.5 * (a + np.swapaxes(a, -1, -2))


def _rot2(t):
    c, s = np.cos(t), np.sin(t)
    return np.array([[c, -s], [s, c]])


def test_lame_constants():
    lam, mu = material.lame(1.0, 0.3)
    assert abs(lam - 0.3 / (1.3 * 0.4)) < 1e-15 and abs(mu - 1 / 2.6) < 1e-15


def test_degradation():
    assert material.degradation(0.0) == 1.0 and material.degradation(1.0) == 0.0
    assert material.degradation(1.0, 1e-6) == 1e-6
    assert material.degradation_slope(0.25) == -1.5


@pytest.mark.parametrize("a,b,theta", [(2e-3, -1e-3, 0.0), (2e-3, -1e-3, 0.7), (3e-3, 1e-3, 1.1),
                                       (-1e-3, -4e-3, 0.3), (1e-3, -3e-3, 2.0)])
def test_split_closed_form_2d(a, b, theta):
    """Principal strains (a, b) rotated by theta: psi+- from Eq. PlusNegPsi by hand."""
    lam, mu = np.array(0.7), np.array(0.4)
    R = _rot2(theta)
    eps = R @ np.diag([a, b]) @ R.T
    parts = material.split(eps[None], lam[None], mu[None])
    tr = a + b
    pp = 0.5 * lam * max(tr, 0) ** 2 + mu * (max(a, 0) ** 2 + max(b, 0) ** 2)
    pm = 0.5 * lam * min(tr, 0) ** 2 + mu * (min(a, 0) ** 2 + min(b, 0) ** 2)
    assert abs(parts["psi_p"][0] - pp) < 1e-18 and abs(parts["psi_m"][0] - pm) < 1e-18
    sp = lam * max(tr, 0) * np.eye(2) + 2 * mu * R @ np.diag([max(a, 0), max(b, 0)]) @ R.T
    assert np.allclose(parts["sig_p"][0], sp, atol=1e-16)


@pytest.mark.parametrize("d", [2, 3])
def test_split_identities_and_stress_is_gradient(d):
    rng = np.random.default_rng(d)
    eps = _sym(rng.standard_normal((40, d, d))) * 1e-2
    lam = 0.3 + rng.random(40)
    mu = 0.2 + rng.random(40)
    p = material.split(eps, lam, mu)
    tr = np.trace(eps, axis1=1, axis2=2)
    full = 0.5 * lam * tr ** 2 + mu * np.einsum("vij,vij->v", eps, eps)
    assert np.allclose(p["psi_p"] + p["psi_m"], full, rtol=1e-13, atol=1e-20)
    c0 = lam[:, None, None] * tr[:, None, None] * np.eye(d) + 2 * mu[:, None, None] * eps
    assert np.allclose(p["sig_p"] + p["sig_m"], c0, atol=1e-16)
    # sigma+ = d psi+ / d eps (central differences along random symmetric directions)
    de = _sym(rng.standard_normal((40, d, d)))
    h = 1e-7
    fd = (material.split(eps + h * de, lam, mu)["psi_p"] - material.split(eps - h * de, lam, mu)["psi_p"]) / (2 * h)
    assert np.allclose(fd, np.einsum("vij,vij->v", p["sig_p"], de), rtol=1e-6, atol=1e-12)


@pytest.mark.parametrize("d,iso", [(2, False), (3, False), (2, True), (3, True)])
def test_tangent_is_stress_derivative(d, iso):
    """C : de (Eq. C_Calc) equals the central difference of sigma(eps, phi)."""
    rng = np.random.default_rng(10 + d)
    eps = _sym(rng.standard_normal((60, d, d)))
    de = _sym(rng.standard_normal((60, d, d)))
    phi = rng.random(60)
    lam = 0.3 + rng.random(60)
    mu = 0.2 + rng.random(60)
    _, _, parts = material.stress(eps, phi, lam, mu, isotropic=iso)
    an = material.tangent_apply(parts, phi, lam, mu, de, isotropic=iso)
    h = 1e-6
    sp, _, _ = material.stress(eps + h * de, phi, lam, mu, isotropic=iso)
    sm, _, _ = material.stress(eps - h * de, phi, lam, mu, isotropic=iso)
    assert np.max(np.abs((sp - sm) / (2 * h) - an)) < 1e-8 * np.max(np.abs(an))


@pytest.mark.parametrize("d", [2, 3])
def test_tangent_undamaged_is_isotropic_stiffness(d):
    """With g = 1 the split drops out: C = lambda I x I + 2 mu I4 for any strain."""
    rng = np.random.default_rng(20 + d)
    eps = _sym(rng.standard_normal((30, d, d)))
    de = _sym(rng.standard_normal((30, d, d)))
    lam = np.full(30, 0.6)
    mu = np.full(30, 0.4)
    _, _, parts = material.stress(eps, np.zeros(30), lam, mu)
    an = material.tangent_apply(parts, np.zeros(30), lam, mu, de)
    c0 = 0.6 * np.trace(de, axis1=1, axis2=2)[:, None, None] * np.eye(d) + 0.8 * de
    assert np.allclose(an, c0, atol=1e-14)


def test_tangent_continuous_through_coincident_eigenvalues():
    lam, mu = np.full(2, 0.6), np.full(2, 0.4)
    de = np.broadcast_to(_sym(np.random.default_rng(5).standard_normal((3, 3))), (2, 3, 3))
    eps = np.array([np.diag([2e-3, 2e-3, -1e-3]), np.diag([2e-3, 2e-3 + 1e-12, -1e-3])])
    phi = np.full(2, 0.5)
    _, _, parts = material.stress(eps, phi, lam, mu)
    an = material.tangent_apply(parts, phi, lam, mu, de)
    assert np.max(np.abs(an[0] - an[1])) < 1e-8
