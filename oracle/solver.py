"""Monolithic crack-length-controlled Newton-Krylov solver, plain NumPy float64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Unknowns q = {eps_tilde, phi, E} (Sec. 3.2).  A Krylov vector is the triple
(d_eps [shape + (d, d)], d_phi [shape], d_E [float]) with the Frobenius inner product,
which equals the Mandel-vector inner product of the symmetric components.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

from . import fourier, material

CRACK = "crack"     # F3 = C(phi) - tau: C = Gamma (geometric reading, Eq. System_CrackLength)
                    # or C = int G_c gamma_f (energy control, Eq. SystemDisc)
STRAIN = "strain"   # F3 = E - E_target           (classical control, Eq. OriSystemc with E_M = f E)


class Problem:
    """Discrete RVE: grid, phases, toughness, notch, load direction, spectral operators."""

    def __init__(self, shape, phase, E, nu, Gc, ell, notch, f, k_res=0.0, isotropic=False, gamma="willot",
                 constraint="length"):
        self.shape = tuple(int(s) for s in shape)
        self.d = len(self.shape)
        self.n = int(np.prod(self.shape))
        phase = np.asarray(phase).astype(np.int64)
        lam_p, mu_p = material.lame(np.asarray(E, float), np.asarray(nu, float))
        self.lam = lam_p[phase]
        self.mu = mu_p[phase]
        self.Gc = np.asarray(Gc, float)[phase]
        self.ell = float(ell)
        self.notch = np.asarray(notch).astype(bool)
        self.free = (~self.notch).astype(float)
        self.f = np.asarray(f, float)
        self.k_res = float(k_res)
        self.isotropic = bool(isotropic)
        # constrained quantity under crack control: crack length Gamma (Eq. CrackLenght) or
        # dissipated energy int G_c gamma_f (Eq. SystemDisc, gradients of Eq. newGammaFourier)
        if constraint not in ("length", "energy"):
            raise ValueError(constraint)
        self.constraint = constraint
        self.xi2 = fourier.xi_squared(self.shape)
        # Galerkin projector: Willot's rotated scheme (Sec. 3.1) or continuous frequencies
        direction = fourier.continuous_direction if gamma == "continuous" else fourier.willot_direction
        self.G = fourier.gamma_hat(direction(self.shape))
        # row scalings of the Newton system (reading: the paper names no preconditioner;
        # a diagonal row scaling keeps the three blocks at comparable magnitude)
        self.C_ref = float(np.max(lam_p + 2.0 * mu_p))
        self.Lbar = float(np.mean(self.xi2))
        self._zeta_cache = {}

    def zeta(self, k):
        """Shadow direction of BiCGStab restart k (cached)."""
        if k not in self._zeta_cache:
            self._zeta_cache[k] = shadow_direction(self.shape, k)
        return self._zeta_cache[k]


@dataclasses.dataclass
class State:
    eps_t: np.ndarray
    phi: np.ndarray
    E: float
    Hn: np.ndarray
    tau: float = 0.0

    def copy(self):
        return State(self.eps_t.copy(), self.phi.copy(), float(self.E), self.Hn.copy(), float(self.tau))


def initial_state(pb: Problem) -> State:
    """Algorithm 2 initial data: eps_tilde = 0, E = 0, H = 0; phi = 0 except phi = 1 on
    the notch (reading: the initial crack is a Dirichlet phi = 1 set)."""
    return State(np.zeros(pb.shape + (pb.d, pb.d)), pb.notch.astype(float), 0.0,
                 np.zeros(pb.shape), 0.0)


class Linearization:
    """Everything the residual and the Jacobian need at one Newton iterate."""

    def __init__(self, pb: Problem, eps_t, E, phi, Hn):
        self.pb = pb
        self.phi = phi
        self.E = E
        self.eps = eps_t + pb.f * E                                          # Eq. stress_1a
        self.sigma, self.psi_p, self.parts = material.stress(self.eps, phi, pb.lam, pb.mu,
                                                             pb.k_res, pb.isotropic)
        if pb.isotropic:
            self.sig_drive = self.parts["sig_p"] + self.parts["sig_m"]
        else:
            self.sig_drive = self.parts["sig_p"]                              # d psi+ / d eps
        self.H = np.maximum(self.psi_p, Hn)                                   # Eq. history
        # Eq. Delta_history.  reading: at a tie psi+ = H^n the loading branch is taken
        # (chi = 1).  Every increment starts from q^n, where psi+ = H^n on all loading
        # voxels; with the strict "> H" the coupling d F2 / d eps vanishes there, d Gamma /
        # d E = 0 and the bordered system of Eq. LinearSyst_CrackCont is singular.
        self.chi = (self.psi_p >= Hn).astype(float)
        self.Lphi = fourier.laplace_op(phi, pb.xi2)
        self.Gamma = fourier.crack_length(phi, pb.ell, pb.xi2)
        if pb.constraint == "energy":
            self.C = fourier.dissipation(phi, pb.Gc, pb.ell)
            self.w = fourier.dissipation_gradient(phi, pb.Gc, pb.ell) * pb.free  # d C / d phi
        else:
            self.C = self.Gamma
            self.w = (phi / pb.ell + pb.ell * self.Lphi) * pb.free            # d Gamma / d phi
        self.s1 = 1.0 / pb.C_ref
        self.s2 = np.where(pb.notch, 1.0, 1.0 / (pb.Gc / pb.ell + 2.0 * self.H + pb.Gc * pb.ell * pb.Lbar))
        wn = math.sqrt(float(np.sum(self.w * self.w)))
        self.s3_crack = 1.0 / wn if wn > 0 else 1.0
        # magnitude of the terms the residual is assembled from: a residual that has
        # cancelled them down to ~1e-14 of this is at the round-off floor
        free = pb.free
        t2 = [(pb.Gc / pb.ell + 2.0 * self.H) * phi * free, 2.0 * self.H * free,
              pb.Gc * pb.ell * self.Lphi * free]
        self.ref2 = (float(np.sum((self.s1 * self.sigma) ** 2))
                     + sum(float(np.sum((self.s2 * t) ** 2)) for t in t2))

    def reference_norm(self, control, target):
        if control == CRACK:
            g = self.s3_crack * max(abs(self.C), abs(target))
        else:
            g = max(abs(self.E), abs(target))
        return math.sqrt(self.ref2 + g * g)


def residual(lin: Linearization, control: str, target: float):
    """F(q) = (F1, F2, F3)  (Eq. System_CrackLength)."""
    pb = lin.pb
    F1 = fourier.project(lin.sigma, pb.G)
    F2 = (pb.Gc / pb.ell + 2.0 * lin.H) * lin.phi + pb.Gc * pb.ell * lin.Lphi - 2.0 * lin.H
    F2 = np.where(pb.notch, lin.phi - 1.0, F2)
    F3 = (lin.C - target) if control == CRACK else (lin.E - target)
    return F1, F2, float(F3)


def jacobian_apply(lin: Linearization, dq, control: str):
    """Delta F(q; Delta q)  (Eq. CrackLength_linearization with Eq. Delta_history).

    dF1 = F^-1{ G : F[ C:(de + f dE) - 2(1-phi) sig0+ dphi ] }
    dF2 = -2(1-phi) chi sig0+ : (de + f dE) + (Gc/l + 2H) dphi + Gc l L dphi
    dF3 = sum_v (phi/l + l L phi) dphi        (crack control; dE for strain control)
    Notch voxels are Dirichlet rows: dF2 = dphi there and dphi does not enter other rows.
    """
    pb = lin.pb
    de, dp, dE = dq
    dpm = dp * pb.free
    deps = de + pb.f * dE
    t = material.tangent_apply(lin.parts, lin.phi, pb.lam, pb.mu, deps, pb.k_res, pb.isotropic)
    t = t + (material.degradation_slope(lin.phi) * dpm)[..., None, None] * lin.sig_drive
    dF1 = fourier.project(t, pb.G)
    coup = np.einsum("...ij,...ij->...", lin.sig_drive, deps)
    dF2 = (material.degradation_slope(lin.phi) * lin.chi * coup
           + (pb.Gc / pb.ell + 2.0 * lin.H) * dpm + pb.Gc * pb.ell * fourier.laplace_op(dpm, pb.xi2))
    dF2 = np.where(pb.notch, dp, dF2)
    dF3 = float(np.sum(lin.w * dpm)) if control == CRACK else float(dE)
    return dF1, dF2, dF3


def scales(lin: Linearization, control: str):
    return lin.s1, lin.s2, (lin.s3_crack if control == CRACK else 1.0)


# ---- Krylov vectors ------------------------------------------------------------------

def vdot(a, b):
    return float(np.sum(a[0] * b[0]) + np.sum(a[1] * b[1]) + a[2] * b[2])


def vaxpy(alpha, x, y):
    """alpha x + y"""
    return (alpha * x[0] + y[0], alpha * x[1] + y[1], alpha * x[2] + y[2])


def vscale(alpha, x):
    return (alpha * x[0], alpha * x[1], alpha * x[2])


def vzero_like(x):
    return (np.zeros_like(x[0]), np.zeros_like(x[1]), 0.0)


_MASK64 = (1 << 64) - 1


def splitmix64(x):
    """SplitMix64 finaliser (Steele, Lea, Flood, OOPSLA 2014) on uint64 arrays."""
    x = (np.asarray(x, dtype=np.uint64) + np.uint64(0x9E3779B97F4A7C15))
    with np.errstate(over="ignore"):
        z = x
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def unit_hash(idx):
    """Deterministic numbers in [-1, 1): top 53 bits of splitmix64(idx)."""
    z = splitmix64(idx)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -52) - 1.0


def mandel_channels(d):
    """Mandel component order: 2D (xx, yy, xy); 3D (xx, yy, zz, yz, xz, xy)."""
    if d == 2:
        return [(0, 0), (1, 1), (0, 1)]
    return [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]


def shadow_direction(shape, seed=0):
    """Fixed pseudo-random vector zeta for the BiCGStab shadow residual.

    Channel c of voxel v (linear index, x fastest) draws unit_hash(c * n + v + seed * N),
    Mandel strain channels first, then phi (c = m), then E (index (m + 1) * n); N is the
    vector length (m + 1) n + 1.  In tensor form an off-diagonal Mandel value z becomes
    z / sqrt 2 in both (i, j) and (j, i).
    """
    d = len(shape)
    n = int(np.prod(shape))
    ch = mandel_channels(d)
    m = len(ch)
    off = np.uint64(seed * ((m + 1) * n + 1))
    v = np.arange(n, dtype=np.uint64)
    e = np.zeros(tuple(shape) + (d, d))
    for c, (i, j) in enumerate(ch):
        z = unit_hash(np.uint64(c * n) + v + off).reshape(shape)
        if i == j:
            e[..., i, i] = z
        else:
            e[..., i, j] = e[..., j, i] = z / math.sqrt(2.0)
    p = unit_hash(np.uint64(m * n) + v + off).reshape(shape)
    E = float(unit_hash(np.uint64((m + 1) * n) + off))
    return (e, p, E)


def bicgstab(apply, b, tol=1e-10, maxiter=2000, atol=0.0, zeta=None, shape=None,
             check_every=8, max_restarts=6, stall_checks=25):
    """Unpreconditioned BiCGStab (van der Vorst) from x0 = 0 (Sec. 3.2: the bordered
    system is non-symmetric).  Stops when ||r|| <= max(tol ||b||, atol).

    The shadow residual is r^ = r0 + ||r0|| / sqrt(N) zeta_k with a fixed pseudo-random
    direction zeta_k (N = vector length).  reading: the common choice r^ = b breaks down at
    the first Newton step of every increment, where b is nonzero only in its F3 slot.
    Every ``check_every`` iterations the iterate with the smallest residual so far is kept;
    if the residual has grown 1e6-fold over it, is not finite, has not improved on it for
    ``stall_checks`` checks, or the recurrence broke down, the method restarts from that
    iterate (r = b - A x, shadow zeta_{k+1}), at most ``max_restarts`` times (reading: the bordered Jacobian can carry a nearly imaginary
    eigenvalue pair on which BiCGStab's first-degree stabiliser stalls or diverges).
    zeta: None (r^ = b, no restarts) or a callable k -> zeta_k.
    Returns (x, iterations, relative residual, status) with status 0 = converged,
    1 = iteration limit, 2 = breakdown / divergence after the last restart."""
    bn = math.sqrt(vdot(b, b))
    x = vzero_like(b)
    if bn == 0.0:
        return x, 0, 0.0, 0
    thr = max(tol * bn, atol)
    x_best, rn_best = x, bn
    restarts = 0
    it = 0
    stall = 0
    r = b
    while True:
        rn0 = math.sqrt(vdot(r, r))
        if zeta is None:
            rhat = r
        else:
            z = zeta(restarts)
            N = z[1].size * (1 + len(mandel_channels(z[1].ndim))) + 1
            rhat = vaxpy(rn0 / math.sqrt(N), z, r)
        rho = alpha = omega = 1.0
        v = vzero_like(b)
        p = vzero_like(b)
        bad = False
        while it < maxiter:
            it += 1
            rho_new = vdot(rhat, r)
            if rho_new == 0.0:
                bad = True
                break
            beta = (rho_new / rho) * (alpha / omega)
            p = vaxpy(1.0, r, vscale(beta, vaxpy(-omega, v, p)))
            v = apply(p)
            rv = vdot(rhat, v)
            if rv == 0.0:
                bad = True
                break
            alpha = rho_new / rv
            s = vaxpy(-alpha, v, r)
            t = apply(s)
            tt = vdot(t, t)
            omega = vdot(t, s) / tt if tt > 0.0 else 0.0
            x = vaxpy(alpha, p, vaxpy(omega, s, x))
            r = vaxpy(-omega, t, s)
            rn = math.sqrt(vdot(r, r))
            if rn <= thr:
                return x, it, rn / bn, 0
            if omega == 0.0:
                bad = True
                break
            rho = rho_new
            if zeta is not None and it % check_every == 0:
                if not math.isfinite(rn) or rn > 1e6 * rn_best:
                    bad = True
                    break
                if rn < rn_best:
                    x_best, rn_best = x, rn
                    stall = 0
                else:
                    stall += 1
                    if stall >= stall_checks:
                        stall = 0
                        bad = True
                        break
        if not bad:
            rn = math.sqrt(vdot(r, r))
            if zeta is not None and not rn < rn_best:
                return x_best, it, rn_best / bn, 1
            return x, it, rn / bn, 1
        if zeta is None or restarts >= max_restarts:
            return x_best, it, rn_best / bn, 2
        restarts += 1
        x = x_best
        r = vaxpy(-1.0, apply(x), b)


@dataclasses.dataclass
class Options:
    alpha: float = 1.0            # relaxation of the Newton update (Algorithm 2)
    rho_E: float = 1.0            # crack control: |a dE| <= rho_E |E_i| when E grows (reading)
    rho_E_down: float = 0.5       # ... and <= rho_E_down |E_i| when E shrinks (E never vanishes)
    rho_phi: float = 1.0          # max |a d_phi| <= rho_phi (the phase field lives in [0, 1])
    newton_tol: float = 1e-10
    newton_max: int = 50
    krylov_tol: float = 1e-10
    krylov_max: int = 4000
    floor: float = 1e-13          # round-off floor, relative to Linearization.reference_norm
    e_scale: float = 0.1          # crack control: unknown E scaled so |S J e_E| = e_scale (reading)
    restarts: int = 6             # BiCGStab restarts on divergence / breakdown / stagnation
    startup_beta: float = 0.25    # start-up load level: max 2 psi+ / (Gc/l) over free voxels
    ramp_gamma: float = 0.5       # start-up strain ramp until Gamma grew by this much
    ramp_factor: float = 1.25     # load factor per start-up ramp step
    ramp_max: int = 40
    ls_growth: float = 1.5        # backtrack when |b| grows beyond this factor
    ls_max: int = 6               # at most this many step halvings


@dataclasses.dataclass
class NewtonResult:
    converged: bool
    iterations: int
    krylov_iterations: int
    err: float
    history: list


def _rel(a, b):
    if a == 0.0:
        return 0.0
    return a / b if b > 0.0 else math.inf


def newton(pb: Problem, st: State, control: str, target: float, opt: Options,
           linear_solver=None) -> NewtonResult:
    """Algorithm 2 inner loop: Newton-Raphson on F(q) = 0 with the linear system of
    Eq. LinearSyst_CrackCont solved by BiCGStab.  Updates ``st`` in place (eps_t, phi, E);
    the history Hn is not touched (committed by the caller).

    Convergence (reading of the garbled Eq. errors_crack):
      err = max(||a d_eps||/||eps||, |a dE|/|E|, ||a d_phi||/||phi||, |Gamma - tau|/tau)
    with a the applied step length, counted only after a step whose Krylov solve reached its
    tolerance.  A Krylov solve that stops above its tolerance but at least halved the
    residual still gives a step (inexact Newton): near unstable propagation the bordered
    system can be nearly singular at an iterate, and the next iterate usually is not.
    An iterate is also accepted when the a posteriori error estimate theta / (1 - theta) * err
    (theta = err_k / err_{k-1} < 0.5, the observed contraction of two consecutive exact steps)
    is within the tolerance (reading: the certification step that would only confirm a
    contracting sequence is skipped).
    Step length (reading: the paper gives only the relaxation alpha): alpha, reduced under
    crack control so that E at most doubles or halves per iteration, and so that no
    phase-field value moves by more than 1; without such bounds the first increment from a
    low start-up load can overshoot into a diverging branch.
    """
    hist = []
    kry_total = 0
    bn_prev = None
    last = None          # (step length, d_eps, d_phi, dE) of the step just taken
    halvings = 0
    err_prev = None      # err of the previous full step, when it was an exact step
    it = 0
    while it < opt.newton_max:
        lin = Linearization(pb, st.eps_t, st.E, st.phi, st.Hn)
        F1, F2, F3 = residual(lin, control, target)
        s1, s2, s3 = scales(lin, control)
        b = (-s1 * F1, -s2 * F2, -s3 * F3)
        ref = lin.reference_norm(control, target)
        bn = math.sqrt(vdot(b, b))
        # backtracking (reading: the paper takes full or alpha-relaxed steps): a step that
        # grew the scaled residual norm more than ls_growth-fold is halved, up to ls_max times
        if last is not None and bn > opt.ls_growth * bn_prev and halvings < opt.ls_max:
            a_l, de_l, dp_l, dE_l = last
            h = 0.5 * a_l
            st.eps_t = fourier.project(st.eps_t - h * de_l, pb.G)
            st.phi = st.phi - h * dp_l
            st.E = st.E - h * dE_l
            last = (h, de_l, dp_l, dE_l)
            halvings += 1
            err_prev = None
            continue
        it += 1
        halvings = 0
        relres = bn / ref if ref > 0.0 else 0.0
        if it > 1 and bn <= opt.floor * ref:
            # the residual is at its round-off floor: the previous step converged
            hist.append(dict(it=it, step=0.0, err=0.0, krylov=0, krylov_rel=0.0, krylov_status=0,
                             e_eps=0.0, e_E=0.0, e_phi=0.0, res=relres))
            return NewtonResult(True, it - 1, kry_total, 0.0, hist)

        def A0(v):
            a1, a2, a3 = jacobian_apply(lin, v, control)
            return (s1 * a1, s2 * a2, s3 * a3)

        # column scaling of the E unknown under crack control: the constraint row and the
        # E column form a border with a zero diagonal whose eigenvalue pair lies near the
        # imaginary axis; shrinking the column to norm e_scale keeps the pair small
        kE = 1.0
        if control == CRACK and opt.e_scale > 0.0:
            cE = A0((np.zeros_like(st.eps_t), np.zeros_like(st.phi), 1.0))
            cn = math.sqrt(vdot(cE, cE))
            if cn > 0.0:
                kE = opt.e_scale / cn

        def A(v):
            return A0((v[0], v[1], kE * v[2]))

        if linear_solver is None:
            dq, kits, krel, kstat = bicgstab(A, b, opt.krylov_tol, opt.krylov_max, 0.1 * opt.floor * ref,
                                             pb.zeta, max_restarts=opt.restarts)
        else:
            dq, kits, krel, kstat = linear_solver(lin, A, b, control)
        dq = (dq[0], dq[1], kE * dq[2])
        kry_total += kits
        if kstat != 0 and not krel < 0.5:
            hist.append(dict(it=it, step=0.0, err=math.inf, krylov=kits, krylov_rel=krel,
                             krylov_status=kstat, e_eps=0.0, e_E=0.0, e_phi=0.0, res=relres))
            return NewtonResult(False, it, kry_total, math.inf, hist)
        de, dp, dE = dq
        a = opt.alpha
        if control == CRACK and dE != 0.0:
            rho = opt.rho_E if dE > 0.0 else opt.rho_E_down
            if abs(a * dE) > rho * abs(st.E):
                a = rho * abs(st.E) / abs(dE)
        dpmax = float(np.max(np.abs(dp)))
        if dpmax > 0.0 and a * dpmax > opt.rho_phi:
            a = opt.rho_phi / dpmax
        # the update keeps eps_tilde compatible (G projection): Newton corrections act only on
        # compatible directions, so incompatible round-off in a step would never be removed
        st.eps_t = fourier.project(st.eps_t + a * de, pb.G)
        st.phi = st.phi + a * dp
        st.E = st.E + a * dE
        last = (a, de, dp, dE)
        bn_prev = bn
        if not (np.all(np.isfinite(st.eps_t)) and np.all(np.isfinite(st.phi)) and math.isfinite(st.E)):
            return NewtonResult(False, it, kry_total, math.inf, hist)
        eps = st.eps_t + pb.f * st.E
        e_eps = _rel(a * math.sqrt(float(np.sum(de * de))), math.sqrt(float(np.sum(eps * eps))))
        e_E = _rel(abs(a * dE), abs(st.E))
        e_phi = _rel(a * math.sqrt(float(np.sum(dp * dp))), math.sqrt(float(np.sum(st.phi * st.phi))))
        err = max(e_eps, e_E, e_phi)
        if control == CRACK:
            err = max(err, _rel(abs(constraint_value(pb, st.phi) - target), abs(target)))
        hist.append(dict(it=it, step=a, err=err, krylov=kits, krylov_rel=krel, krylov_status=kstat,
                         e_eps=e_eps, e_E=e_E, e_phi=e_phi, res=relres))
        # an inexact step (Krylov stopped above its tolerance) never ends the loop
        est = err
        if kstat == 0 and err_prev is not None and err_prev > 0.0:
            theta = err / err_prev
            if theta < 0.5:
                est = min(err, theta / (1.0 - theta) * err)
        if est <= opt.newton_tol and kstat == 0:
            return NewtonResult(True, it, kry_total, err, hist)
        err_prev = err if kstat == 0 else None
    return NewtonResult(False, opt.newton_max, kry_total, hist[-1]["err"] if hist else math.inf, hist)


def constraint_value(pb: Problem, phi):
    """The quantity crack control prescribes: Gamma, or int G_c gamma_f under energy control."""
    if pb.constraint == "energy":
        return fourier.dissipation(phi, pb.Gc, pb.ell)
    return fourier.crack_length(phi, pb.ell, pb.xi2)


def commit(pb: Problem, st: State):
    """History update at the end of a converged increment (Eq. history)."""
    eps = st.eps_t + pb.f * st.E
    _, psi_p, _ = material.stress(eps, st.phi, pb.lam, pb.mu, pb.k_res, pb.isotropic)
    st.Hn = np.maximum(psi_p, st.Hn)


def macro_stress(pb: Problem, st: State):
    """Sigma_M = <sigma> (volume average) at the current state."""
    eps = st.eps_t + pb.f * st.E
    sig, _, _ = material.stress(eps, st.phi, pb.lam, pb.mu, pb.k_res, pb.isotropic)
    return sig.reshape(-1, pb.d, pb.d).mean(axis=0)


def max_drive_ratio(pb: Problem, st: State):
    """max over free voxels of 2 psi+ / (Gc / l) at the current state."""
    eps = st.eps_t + pb.f * st.E
    _, psi_p, _ = material.stress(eps, st.phi, pb.lam, pb.mu, pb.k_res, pb.isotropic)
    r = 2.0 * psi_p / (pb.Gc / pb.ell)
    return float(np.max(np.where(pb.notch, 0.0, r)))


def startup(pb: Problem, opt: Options, st: Optional[State] = None, linear_solver=None):
    """Start-up before the first crack-controlled increment.

    reading: at E = 0 the bordered system is singular (every E-derivative vanishes), and
    from a small load the linearised crack length responds to E so weakly that a crack-
    controlled Newton step overshoots; crack control therefore starts from a loaded state:
      (a) strain control at E = 0 gives the phase-field profile around the notch;
      (b) strain control at a probe load E_p (damage response ~1e-6) gives the elastic
          scaling of psi+ with E^2;
      (c) strain control at E_s, where max over free voxels 2 psi+/(Gc/l) = startup_beta,
          and the history is committed;
      (d) strain-controlled loading E <- ramp_factor E (history committed each step) until
          Gamma has grown by ramp_gamma over its value at (c) or a step fails to converge
          (the pre-peak part of the load path);
      (e) tau_0 = the constrained quantity (Gamma, or the dissipated energy) of the last
          committed state.
    Returns (state, [NewtonResult a, b, c, ramp...], E_s).
    """
    st = initial_state(pb) if st is None else st
    res = []
    r = newton(pb, st, STRAIN, 0.0, opt, linear_solver)
    res.append(r)
    if not r.converged:
        return st, res, None
    gmin = float(np.min(pb.Gc / pb.ell))
    Ep = 1e-3 * math.sqrt(gmin / pb.C_ref)
    r = newton(pb, st, STRAIN, Ep, opt, linear_solver)
    res.append(r)
    if not r.converged:
        return st, res, None
    ratio = max_drive_ratio(pb, st)
    if not ratio > 0.0:
        raise ValueError("load direction produces no tensile energy")
    Es = Ep * math.sqrt(opt.startup_beta / ratio)
    r = newton(pb, st, STRAIN, Es, opt, linear_solver)
    res.append(r)
    if not r.converged:
        return st, res, Es
    commit(pb, st)
    g0 = fourier.crack_length(st.phi, pb.ell, pb.xi2)
    gam = g0
    for _ in range(opt.ramp_max):
        if gam - g0 >= opt.ramp_gamma:
            break
        trial = st.copy()
        r = newton(pb, trial, STRAIN, st.E * opt.ramp_factor, opt, linear_solver)
        res.append(r)
        if not r.converged:
            break
        commit(pb, trial)
        st.eps_t, st.phi, st.E, st.Hn = trial.eps_t, trial.phi, trial.E, trial.Hn
        gam = fourier.crack_length(st.phi, pb.ell, pb.xi2)
    st.tau = constraint_value(pb, st.phi)
    return st, res, Es


def crack_increment(pb: Problem, st: State, da: float, opt: Options, linear_solver=None,
                    max_depth: int = 3, _depth: int = 0):
    """One crack-length increment (Algorithm 2 outer loop): tau <- tau + da * h^(d-1),
    Newton under crack control from the last committed state, commit on convergence.

    reading (cut-back, not in the paper): if Newton fails, the increment is retried as two
    half increments (each committed), recursively down to da / 2^max_depth.  On failure the
    state is left unchanged.  Returns (NewtonResult, record); record["cutbacks"] counts the
    halvings used."""
    snap = st.copy()
    trial = st.copy()
    tau = st.tau + da
    r = newton(pb, trial, CRACK, tau, opt, linear_solver)
    if not r.converged:
        if _depth >= max_depth:
            return r, None
        r1, rec1 = crack_increment(pb, st, 0.5 * da, opt, linear_solver, max_depth, _depth + 1)
        if rec1 is None:
            return r1, None
        r2, rec2 = crack_increment(pb, st, 0.5 * da, opt, linear_solver, max_depth, _depth + 1)
        if rec2 is None:
            st.eps_t, st.phi, st.E, st.Hn, st.tau = snap.eps_t, snap.phi, snap.E, snap.Hn, snap.tau
            return r2, None
        rec2["cutbacks"] = 1 + rec1["cutbacks"] + rec2["cutbacks"]
        rec2["newton"] += rec1["newton"] + r.iterations
        rec2["krylov"] += rec1["krylov"] + r.krylov_iterations
        return r2, rec2
    commit(pb, trial)
    trial.tau = tau
    st.eps_t, st.phi, st.E, st.Hn, st.tau = trial.eps_t, trial.phi, trial.E, trial.Hn, trial.tau
    lin = Linearization(pb, st.eps_t, st.E, st.phi, st.Hn)
    rec = dict(E=st.E, Sigma=macro_stress(pb, st), Gamma=lin.Gamma, tau=st.tau,
               newton=r.iterations, krylov=r.krylov_iterations, cutbacks=0)
    return r, rec


def strain_increment(pb: Problem, st: State, E_target: float, opt: Options):
    """Strain-controlled monolithic increment (E fixed), for start-up and comparison."""
    trial = st.copy()
    r = newton(pb, trial, STRAIN, E_target, opt)
    if not r.converged:
        return r, None
    commit(pb, trial)
    st.eps_t, st.phi, st.E, st.Hn = trial.eps_t, trial.phi, trial.E, trial.Hn
    st.tau = constraint_value(pb, st.phi)
    return r, dict(E=st.E, Sigma=macro_stress(pb, st), Gamma=fourier.crack_length(st.phi, pb.ell, pb.xi2))


def problem_from_input(inp, **kw) -> Problem:
    """Build a Problem from any object with the RVE input attributes
    (shape, phase, E, nu, Gc, ell, notch, f)."""
    return Problem(inp.shape, inp.phase, inp.E, inp.nu, inp.Gc, inp.ell, inp.notch, inp.f, **kw)


def cg(apply, b, tol=1e-12, maxiter=5000):
    """Conjugate gradients on the (symmetric) mechanical sub-problem (Sec. 3.1)."""
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = float(np.sum(r * r))
    bn = math.sqrt(rr)
    if bn == 0.0:
        return x, 0
    for it in range(1, maxiter + 1):
        Ap = apply(p)
        pAp = float(np.sum(p * Ap))
        if pAp <= 0.0:  # the residual reached round-off (or a non-positive direction): stop
            return x, it
        a = rr / pAp
        x = x + a * p
        r = r - a * Ap
        rr_new = float(np.sum(r * r))
        if math.sqrt(rr_new) <= tol * bn:
            return x, it
        p = r + (rr_new / rr) * p
        rr = rr_new
    return x, maxiter


def solve_mechanical(pb: Problem, phi, E, eps_t=None, tol=1e-12, newton_max=30):
    """Mechanical sub-problem of Algorithm 1 at fixed phi and fixed E: Newton on
    F1 = F^-1{G : F[sigma]} = 0 (Eq. FouGal_equil) with the linear system of
    Eq. LinearOpe_Mech solved by CG.  Returns eps_tilde."""
    eps_t = np.zeros(pb.shape + (pb.d, pb.d)) if eps_t is None else eps_t.copy()
    for _ in range(newton_max):
        eps = eps_t + pb.f * E
        sig, _, parts = material.stress(eps, phi, pb.lam, pb.mu, pb.k_res, pb.isotropic)
        F1 = fourier.project(sig, pb.G)
        ref = math.sqrt(float(np.sum(sig * sig)))
        if math.sqrt(float(np.sum(F1 * F1))) <= tol * max(ref, 1e-300):
            return eps_t

        def A(de):
            return fourier.project(material.tangent_apply(parts, phi, pb.lam, pb.mu, de, pb.k_res,
                                                          pb.isotropic), pb.G)

        de, _ = cg(A, -F1, tol * 1e-2)
        eps_t = eps_t + de
    raise RuntimeError("mechanical Newton did not converge")


def solve_phase(pb: Problem, H):
    """Phase-field sub-problem of Algorithm 1 at fixed history H (Eq. Helm2 with R2):
    (Gc/l + 2H) phi + Gc l L phi = 2H on the free voxels, phi = 1 on the notch.  The free
    block is symmetric positive definite; solved by CG on it, with the notch values moved
    to the right-hand side."""
    free = ~pb.notch
    fixed = pb.notch.astype(float)
    a = pb.Gc / pb.ell + 2.0 * H

    def A(v):
        return a * v + pb.Gc * pb.ell * fourier.laplace_op(v, pb.xi2)

    def Af(v):
        return np.where(free, A(np.where(free, v, 0.0)), 0.0)

    b = np.where(free, 2.0 * H - A(fixed), 0.0)
    x, _ = cg(Af, b, tol=1e-14, maxiter=20000)
    return np.where(free, x, 0.0) + fixed


def staggered_increment(pb: Problem, st: State, E_target: float, tol=1e-10, max_iter=500, mech_tol=1e-11):
    """Strain-controlled staggered increment (Algorithm 1): alternate the mechanical
    solve at fixed phi and the phase-field solve at fixed H = max(psi+, H^n) until the
    relative phase-field change is within tol; commit H.

    reading: the paper's stopping test is on the iterates; the relative change of phi
    (and of eps_tilde) between two sweeps is used.  The fixed point solves F1 = F2 = 0 at
    E_target, i.e. it is the monolithic strain-controlled solution.  Returns (sweeps,
    record)."""
    st.E = float(E_target)
    for it in range(1, max_iter + 1):
        eps_t = solve_mechanical(pb, st.phi, st.E, st.eps_t, tol=mech_tol)
        eps = eps_t + pb.f * st.E
        _, psi_p, _ = material.stress(eps, st.phi, pb.lam, pb.mu, pb.k_res, pb.isotropic)
        H = np.maximum(psi_p, st.Hn)
        phi = solve_phase(pb, H)
        dphi = _rel(math.sqrt(float(np.sum((phi - st.phi) ** 2))), math.sqrt(float(np.sum(phi * phi))))
        deps = _rel(math.sqrt(float(np.sum((eps_t - st.eps_t) ** 2))), math.sqrt(float(np.sum(eps * eps))))
        st.eps_t, st.phi = eps_t, phi
        if max(dphi, deps) <= tol:
            break
    else:
        raise RuntimeError("staggered iteration did not converge")
    commit(pb, st)
    st.tau = constraint_value(pb, st.phi)
    return it, dict(E=st.E, Sigma=macro_stress(pb, st), Gamma=fourier.crack_length(st.phi, pb.ell, pb.xi2),
                    sweeps=it)
