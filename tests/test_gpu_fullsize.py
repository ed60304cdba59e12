"""Parity at the full 512^2 size of the headline workload (seeded fibre composites, r = 12,
40 % fibres, notch 32), in the launch configuration the bench times.

* The grouped apply of 4 RVEs (rve_apply_device_batch, one launch per pass, as in the batched
  BiCGStab chunks) equals each RVE's own apply bit for bit.
* One 512^2 apply against the float64 oracle's Jacobian (0.2 s in NumPy): FP64 at 1e-11 and
  MIXED at 1e-5, element by element.
* A batched crack increment of 4 composites (MIXED, Newton 1e-8, Krylov 1e-2, as in the bench),
  checked through properties the oracle evaluates on the library's converged fields: the
  crack-length constraint Gamma(phi) = tau, the macroscopic stress, and the scaled residual
  of Eq. System_CrackLength at the Newton tolerance's level.
* The apply at the other workloads' full sizes (the 128^3 porous RVE and ragged-batch grids
  on runtime-length axes) against the oracle, MIXED at 1e-5."""
import math

import numpy as np
import pytest

from oracle import solver
from paper_2412_17445_gb300 import binding as B
from paper_2412_17445_gb300 import microstructure as ms

pytestmark = pytest.mark.gpu

N = 512


def _composite(k):
    return ms.fibre_composite(n=N, radius=12.0, fraction=0.4, notch_len=32, seed=ms.SEED_BASE + 1 + 1000 * k)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2412_17445_gb300 import build
    build.build()
    B.lib()


def test_grouped_apply_512_equals_single_applies():
    import torch
    gs = []
    for k in range(4):
        inp = _composite(k)
        g = B.RVE(inp, precision=B.RVE_MIXED)
        eps, E, phi, H = ms.random_state(inp, 60 + k)
        g.set_state(B.mandel_from_tensor(eps), phi, H, E, 0.0)
        g.linearize(B.RVE_CTRL_CRACK, 1.0)
        gs.append(g)
    for g in gs:
        g.autotune()
    c, nv = gs[0].m + 1, gs[0].n
    gen = torch.Generator().manual_seed(7)
    xs = [torch.randn(c * nv, generator=gen, dtype=torch.float32).cuda() for _ in gs]
    xEs = [torch.tensor([0.2 * (k + 1)], dtype=torch.float64).cuda() for k in range(4)]
    ys1 = [torch.empty_like(x) for x in xs]
    yE1 = [torch.zeros(1, dtype=torch.float64).cuda() for _ in gs]
    for g, x, xE, y, yE in zip(gs, xs, xEs, ys1, yE1):
        g.apply_device(x.data_ptr(), xE.data_ptr(), y.data_ptr(), yE.data_ptr())
    torch.cuda.synchronize()
    ys2 = [torch.empty_like(x) for x in xs]
    yE2 = [torch.zeros(1, dtype=torch.float64).cuda() for _ in gs]
    B.apply_device_batch(gs, [x.data_ptr() for x in xs], [e.data_ptr() for e in xEs],
                         [y.data_ptr() for y in ys2], [e.data_ptr() for e in yE2])
    torch.cuda.synchronize()
    for a, b, ea, eb in zip(ys1, ys2, yE1, yE2):
        assert torch.equal(a, b)
        assert torch.equal(ea, eb)
    for g in gs:
        g.close()


@pytest.mark.parametrize("precision", [B.RVE_FP64, B.RVE_MIXED])
def test_apply_512_against_oracle(precision):
    inp = _composite(0)
    eps, E, phi, H = ms.random_state(inp, 70)
    pb = solver.problem_from_input(inp)
    lin = solver.Linearization(pb, eps, E, phi, H)
    de, dp, dE = ms.random_direction(inp, 71)
    Jo = solver.jacobian_apply(lin, (de, dp, dE), solver.CRACK)
    g = B.RVE(inp, precision=precision)
    g.set_state(B.mandel_from_tensor(eps), phi, H, E)
    g.linearize(B.RVE_CTRL_CRACK, lin.Gamma + 0.5)
    Je, Jp, JE = g.apply(B.mandel_from_tensor(de), dp, dE)
    tol = 1e-11 if precision == B.RVE_FP64 else 1e-5
    assert np.max(np.abs(Je - B.mandel_from_tensor(Jo[0]))) < tol * np.max(np.abs(Jo[0]))
    assert np.max(np.abs(Jp - Jo[1].reshape(-1))) < tol * np.max(np.abs(Jo[1]))
    assert abs(JE - Jo[2]) < tol * max(abs(Jo[2]), 1.0)
    g.close()


def test_batched_increment_512_converged_fields():
    inps = [_composite(k) for k in range(4)]
    gs = [B.RVE(inp, precision=B.RVE_MIXED, newton_tol=1e-8, krylov_tol=1e-2) for inp in inps]
    for g in gs:
        g.startup()
    out, st = B.batch_crack_increment(gs, [1.0] * len(gs))
    assert st == [0] * len(gs)
    for k in (0, 3):
        g, inp, rec = gs[k], inps[k], out[k]
        pb = solver.problem_from_input(inp)
        eps_t = B.tensor_from_mandel(g.field(B.RVE_FIELD_EPS_T), (N, N))
        phi = g.field(B.RVE_FIELD_PHI).reshape(N, N)
        # the history the increment started from is not kept; H = max(psi+, H^n) at the
        # converged state is what the constitutive law sees, and the committed H is exactly that
        H = g.field(B.RVE_FIELD_H).reshape(N, N)
        lin = solver.Linearization(pb, eps_t, rec["E"], phi, H)
        # constraint Gamma(phi) = tau
        assert abs(lin.Gamma - rec["tau"]) <= 1e-6 * rec["tau"]
        # macroscopic stress of the converged fields
        sig_o = B.mandel_from_tensor(solver.macro_stress(pb, solver.State(eps_t, phi, rec["E"], H))[None])[:, 0]
        assert np.max(np.abs(np.array(rec["sigma"][:3]) - sig_o)) <= 1e-12 * np.max(np.abs(sig_o))
        # scaled residual of the bordered system at the converged state
        F1, F2, F3 = solver.residual(lin, solver.CRACK, rec["tau"])
        s1, s2, s3 = solver.scales(lin, solver.CRACK)
        b = (s1 * F1, s2 * F2, s3 * F3)
        assert math.sqrt(solver.vdot(b, b)) <= 1e-5 * lin.reference_norm(solver.CRACK, rec["tau"])
    for g in gs:
        g.close()


@pytest.mark.parametrize("case", ["porous128", "ragged384x192", "ragged512x384", "ragged96x64x48"])
def test_apply_other_full_sizes_against_oracle(case):
    """The apply at the other workloads' full sizes against the oracle, MIXED at 1e-5: the
    128^3 porous RVE, and 2D/3D sizes of the ragged batch whose axes run the runtime-length
    FFT kernels (192, 384, 96, 48)."""
    if case == "porous128":
        inp = ms.porous_solid(n=128, radius=8.0, porosity=0.15, notch_radius=10.0)
    elif case == "ragged384x192":
        inp = ms.fibre_composite(n=192, ny=384, radius=12.0, fraction=0.4, notch_len=32, seed=ms.SEED_BASE + 81)
    elif case == "ragged512x384":
        inp = ms.fibre_composite(n=384, ny=512, radius=12.0, fraction=0.2, notch_len=32, seed=ms.SEED_BASE + 82)
    else:
        inp = ms.porous_solid(shape=(96, 64, 48), radius=4.0, porosity=0.1, notch_radius=8.0,
                              seed=ms.SEED_BASE + 83, E_pore=1e-3)
    eps, E, phi, H = ms.random_state(inp, 80)
    pb = solver.problem_from_input(inp)
    lin = solver.Linearization(pb, eps, E, phi, H)
    de, dp, dE = ms.random_direction(inp, 81)
    Jo = solver.jacobian_apply(lin, (de, dp, dE), solver.CRACK)
    g = B.RVE(inp, precision=B.RVE_MIXED)
    g.set_state(B.mandel_from_tensor(eps), phi, H, E)
    g.linearize(B.RVE_CTRL_CRACK, lin.Gamma + 0.5)
    Je, Jp, JE = g.apply(B.mandel_from_tensor(de), dp, dE)
    assert np.max(np.abs(Je - B.mandel_from_tensor(Jo[0]))) < 1e-5 * np.max(np.abs(Jo[0]))
    assert np.max(np.abs(Jp - Jo[1].reshape(-1))) < 1e-5 * np.max(np.abs(Jo[1]))
    assert abs(JE - Jo[2]) < 1e-5 * max(abs(Jo[2]), 1.0)
    g.close()


@pytest.mark.parametrize("precision", [B.RVE_FP64, B.RVE_MIXED])
def test_apply_1024_against_oracle(precision):
    """The largest 2D grid of the served mix (1024^2 composite; compile-time line length 1024
    in both passes) against the oracle: FP64 at 1e-11, MIXED at 1e-5."""
    inp = ms.fibre_composite(n=1024, radius=12.0, fraction=0.4, notch_len=32, seed=ms.SEED_BASE + 84)
    eps, E, phi, H = ms.random_state(inp, 90)
    pb = solver.problem_from_input(inp)
    lin = solver.Linearization(pb, eps, E, phi, H)
    de, dp, dE = ms.random_direction(inp, 91)
    Jo = solver.jacobian_apply(lin, (de, dp, dE), solver.CRACK)
    g = B.RVE(inp, precision=precision)
    g.set_state(B.mandel_from_tensor(eps), phi, H, E)
    g.linearize(B.RVE_CTRL_CRACK, lin.Gamma + 0.5)
    Je, Jp, JE = g.apply(B.mandel_from_tensor(de), dp, dE)
    tol = 1e-11 if precision == B.RVE_FP64 else 1e-5
    assert np.max(np.abs(Je - B.mandel_from_tensor(Jo[0]))) < tol * np.max(np.abs(Jo[0]))
    assert np.max(np.abs(Jp - Jo[1].reshape(-1))) < tol * np.max(np.abs(Jo[1]))
    assert abs(JE - Jo[2]) < tol * max(abs(Jo[2]), 1.0)
    g.close()


@pytest.mark.parametrize("precision", [B.RVE_FP64, B.RVE_MIXED])
def test_crack_length_sum_near_cancelling_constraint_1024(precision):
    """The crack-length sum behind F3 = Gamma - tau (Eq. CrackLenght via Parseval, float64 and
    compensated in both precisions) on a 1024^2 composite with the target set to the
    oracle's Gamma, so F3 cancels to the difference of the two sums: within 1e-12 of Gamma."""
    inp = ms.fibre_composite(n=1024, radius=12.0, fraction=0.4, notch_len=32, seed=ms.SEED_BASE + 84)
    eps, E, phi, H = ms.random_state(inp, 92)
    pb = solver.problem_from_input(inp)
    lin = solver.Linearization(pb, eps, E, phi, H)
    _, _, F3o = solver.residual(lin, solver.CRACK, lin.Gamma)
    assert F3o == 0.0
    g = B.RVE(inp, precision=precision)
    g.set_state(B.mandel_from_tensor(eps), phi, H, E)
    g.linearize(B.RVE_CTRL_CRACK, lin.Gamma)
    _, _, F3 = g.residual()
    assert abs(F3) <= 1e-12 * lin.Gamma, (F3, lin.Gamma)
    g.close()


def test_apply_192cube_mixed_against_fp64():
    """The largest 3D grid of the serving spec (192^3 porous solid, runtime-length axes): the
    oracle needs 85 s and 29 GB for one apply there, so the MIXED apply is checked against the
    library's FP64 apply (oracle-pinned at the smaller sizes) at 1e-5."""
    inp = ms.porous_solid(n=192, radius=8.0, porosity=0.15, notch_radius=10.0, seed=ms.SEED_BASE + 85)
    eps, E, phi, H = ms.random_state(inp, 92)
    de, dp, dE = ms.random_direction(inp, 93)
    outs = []
    for prec in (B.RVE_FP64, B.RVE_MIXED):
        g = B.RVE(inp, precision=prec)
        g.set_state(B.mandel_from_tensor(eps), phi, H, E)
        g.linearize(B.RVE_CTRL_CRACK, 1e3)
        outs.append(g.apply(B.mandel_from_tensor(de), dp, dE))
        g.close()
    (e64, p64, E64), (e32, p32, E32) = outs
    assert np.max(np.abs(e32 - e64)) < 1e-5 * np.max(np.abs(e64))
    assert np.max(np.abs(p32 - p64)) < 1e-5 * np.max(np.abs(p64))
    assert abs(E32 - E64) < 1e-5 * max(abs(E64), 1.0)
