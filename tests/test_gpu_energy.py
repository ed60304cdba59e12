"""Energy control on the GPU (RVE_CONSTRAINT_ENERGY, Eq. SystemDisc): the constraint value,
its derivative row in the scaled operator, and energy-controlled increments against the
oracle's Problem(constraint="energy").  Float64 path 1e-11 on single evaluations and 1e-10 on
converged increments; mixed path 1e-5."""
import numpy as np
import pytest

from oracle import fourier, solver
from paper_2412_17445_gb300 import binding as B
from paper_2412_17445_gb300 import microstructure as ms

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2412_17445_gb300 import build
    build.build()
    B.lib()


@pytest.mark.parametrize("shape", [(16, 16), (18, 12), (24, 36), (64, 128), (128, 48), (8, 8, 6), (12, 6, 4),
                                   (8, 64, 128)])
@pytest.mark.parametrize("precision", [B.RVE_FP64, B.RVE_MIXED])
def test_residual_and_apply_energy_constraint(shape, precision):
    inp = ms.random_rve(shape, 41)
    eps, E, phi, H = ms.random_state(inp, 42)
    pb = solver.problem_from_input(inp, constraint="energy")
    lin = solver.Linearization(pb, eps, E, phi, H)
    target = lin.C * 1.01
    F1o, F2o, F3o = solver.residual(lin, solver.CRACK, target)
    g = B.RVE(inp, precision=precision, constraint=B.RVE_CONSTRAINT_ENERGY)
    g.set_state(B.mandel_from_tensor(eps), phi, H, E)
    g.linearize(B.RVE_CTRL_CRACK, target)
    F1, F2, F3 = g.residual()
    assert abs(F3 - F3o) < 1e-11 * abs(target)
    assert np.max(np.abs(F1 - B.mandel_from_tensor(F1o))) < 1e-11 * np.max(np.abs(lin.sigma))
    de, dp, dE = ms.random_direction(inp, 43)
    Jo = solver.jacobian_apply(lin, (de, dp, dE), solver.CRACK)
    Je, Jp, JE = g.apply(B.mandel_from_tensor(de), dp, dE)
    tol = 1e-11 if precision == B.RVE_FP64 else 1e-5
    assert abs(JE - Jo[2]) < tol * np.sum(np.abs(lin.w * dp))
    assert np.max(np.abs(Jp - Jo[1].reshape(-1))) < tol * np.max(np.abs(Jo[1]))
    assert np.max(np.abs(Je - B.mandel_from_tensor(Jo[0]))) < tol * np.max(np.abs(Jo[0]))
    g.close()


def _oracle_energy_run(inp, n_inc, dtau):
    pb = solver.problem_from_input(inp, constraint="energy")
    opt = solver.Options(newton_tol=1e-12, krylov_tol=1e-12)
    st, res, _ = solver.startup(pb, opt)
    assert all(r.converged for r in res[:3])
    recs = []
    for _ in range(n_inc):
        r, rec = solver.crack_increment(pb, st, dtau, opt)
        assert r.converged
        rec["phi"] = st.phi.copy()
        rec["D"] = fourier.dissipation(st.phi, pb.Gc, pb.ell)
        recs.append(rec)
    return recs


@pytest.mark.parametrize("case", ["composite32", "porous8"])
def test_energy_controlled_increments_fp64(case):
    """Heterogeneous G_c under energy control: start-up and increments of prescribed
    dissipated energy match the oracle (E, Sigma, Gamma, tau at 1e-10; phi at 1e-8)."""
    if case == "composite32":
        inp = ms.fibre_composite(n=32, radius=4.0, fraction=0.3, notch_len=8, seed=21)
    else:
        inp = ms.porous_solid(n=8, radius=1.5, porosity=0.1, notch_radius=2.0, seed=6, E_pore=0.05)
    dtau = float(np.min(inp.Gc))
    orc = _oracle_energy_run(inp, 3, dtau)
    g = B.RVE(inp, precision=B.RVE_FP64, newton_tol=1e-12, krylov_tol=1e-12, constraint=B.RVE_CONSTRAINT_ENERGY)
    su = g.startup()
    for k in range(3):
        s = g.crack_increment(dtau)
        o = orc[k]
        sig_o = B.mandel_from_tensor(o["Sigma"][None])[:, 0]
        assert abs(s["E"] - o["E"]) <= 1e-10 * abs(o["E"]), (k, s["E"], o["E"])
        assert np.max(np.abs(np.array(s["sigma"][: g.m]) - sig_o)) <= 1e-10 * np.max(np.abs(sig_o))
        assert abs(s["gamma"] - o["Gamma"]) <= 1e-10 * o["Gamma"]
        assert abs(s["tau"] - o["tau"]) <= 1e-10 * o["tau"]
    assert abs(su["tau"] + 3 * dtau - s["tau"]) < 1e-12 * s["tau"]
    phi = g.field(B.RVE_FIELD_PHI)
    assert np.max(np.abs(phi - orc[-1]["phi"].reshape(-1))) < 1e-8
    g.close()


def test_energy_controlled_increments_mixed():
    inp = ms.fibre_composite(n=32, radius=3.0, fraction=0.3, notch_len=6, seed=11)
    dtau = float(np.min(inp.Gc))
    orc = _oracle_energy_run(inp, 3, dtau)
    g = B.RVE(inp, precision=B.RVE_MIXED, constraint=B.RVE_CONSTRAINT_ENERGY)
    g.startup()
    for k in range(3):
        s = g.crack_increment(dtau)
        o = orc[k]
        sig_o = B.mandel_from_tensor(o["Sigma"][None])[:, 0]
        assert abs(s["E"] - o["E"]) <= 1e-5 * abs(o["E"])
        assert np.max(np.abs(np.array(s["sigma"][:3]) - sig_o)) <= 1e-5 * np.max(np.abs(sig_o))
    g.close()


@pytest.mark.parametrize("precision", [B.RVE_FP64, B.RVE_MIXED])
def test_energy_control_equals_length_control_for_homogeneous_gc(precision):
    """A homogeneous panel: energy increments G_c * da give the length-controlled path."""
    inp = ms.homogeneous_panel(32, notch_len=8)
    Gc = float(inp.Gc[0])
    out = []
    for c, da in ((B.RVE_CONSTRAINT_LENGTH, 1.0), (B.RVE_CONSTRAINT_ENERGY, Gc)):
        g = B.RVE(inp, precision=precision, constraint=c)
        g.startup()
        out.append([g.crack_increment(da) for _ in range(3)] + [g.field(B.RVE_FIELD_PHI)])
        g.close()
    tol = 1e-9 if precision == B.RVE_FP64 else 1e-5
    for a, b in zip(out[0][:3], out[1][:3]):
        assert abs(a["E"] - b["E"]) <= tol * abs(a["E"])
        assert abs(a["gamma"] - b["gamma"]) <= tol * a["gamma"]
        assert abs(Gc * a["tau"] - b["tau"]) <= tol * b["tau"]
    assert np.max(np.abs(out[0][3] - out[1][3])) < (1e-7 if precision == B.RVE_FP64 else 1e-3)


@pytest.mark.parametrize("precision", [B.RVE_FP64, B.RVE_MIXED])
def test_energy_control_batch_equals_alone(precision):
    """Energy- and length-controlled RVEs mixed in one batch (grouped launches for the three
    composites of one shape): every result equals the RVE run alone, bit for bit."""
    inps = [ms.fibre_composite(n=32, radius=3.0, fraction=0.3, notch_len=6, seed=11 + k) for k in range(3)]
    inps.append(ms.porous_solid(n=8, radius=1.5, porosity=0.1, notch_radius=2.0, seed=6, E_pore=0.05))
    cons = [B.RVE_CONSTRAINT_ENERGY, B.RVE_CONSTRAINT_LENGTH, B.RVE_CONSTRAINT_ENERGY, B.RVE_CONSTRAINT_ENERGY]
    das = [float(np.min(inp.Gc)) if c == B.RVE_CONSTRAINT_ENERGY else 1.0 for inp, c in zip(inps, cons)]
    alone = []
    for inp, c, da in zip(inps, cons, das):
        g = B.RVE(inp, precision=precision, constraint=c)
        g.startup()
        for _ in range(2):
            r = g.crack_increment(da)
        alone.append(r)
        g.close()
    gs = [B.RVE(inp, precision=precision, constraint=c) for inp, c in zip(inps, cons)]
    for g in gs:
        g.startup()
    for _ in range(2):
        out, st = B.batch_crack_increment(gs, das)
        assert st == [0] * len(gs)
    for a, b in zip(alone, out):
        assert a["E"] == b["E"] and a["sigma"] == b["sigma"] and a["tau"] == b["tau"]
    for g in gs:
        g.close()
