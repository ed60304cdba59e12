"""GPU parity: the CUDA library (through the C ABI) against the float64 CPU oracle on the
same seeded inputs.  Float64 path: relative 1e-10 on converged macroscopic quantities and
round-off level (1e-11 of the operand scale) on single operator evaluations; mixed path
(float32 FFTs / Krylov, float64 residual): relative 1e-5 and identical {phi > 0.5} sets."""
import json
import os

import numpy as np
import pytest

from oracle import fourier, solver
from paper_2412_17445_gb300 import binding as B
from paper_2412_17445_gb300 import microstructure as ms

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2412_17445_gb300 import build
    build.build()
    B.lib()


def _gpu_state_from(inp, eps, E, phi, H, prec, split, tau=0.0):
    g = B.RVE(inp, precision=prec, split=split)
    g.set_state(B.mandel_from_tensor(eps), phi, H, E, tau)
    return g


# (ny, nx) / (nz, ny, nx).  The library compiles the FFT passes for line lengths 48, 64, 96,
# 128, 192, 256, 384, 512 and 1024 (2D) and 48, 64, 96, 128 (3D), with a radix-3 stage at 48,
# 96, 192 and 384; other lengths run the runtime-length kernels.  The shapes mix both kinds
# on different axes, with several tiles and a ragged last tile, and include odd extents (no
# Nyquist index; an odd row count leaves the last row pair half empty).
SHAPES = [(16, 16), (18, 12), (24, 36), (8, 8, 6), (12, 6, 4),
          (64, 128), (96, 256), (128, 48), (8, 64, 128), (64, 12, 64),
          (9, 27), (27, 9), (3, 9, 27),
          (192, 36), (36, 384), (48, 96, 24), (24, 48, 96)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("split", [B.RVE_SPLIT_SPECTRAL, B.RVE_SPLIT_NONE])
@pytest.mark.parametrize("control", [B.RVE_CTRL_CRACK, B.RVE_CTRL_STRAIN])
def test_residual_and_apply_fp64(shape, split, control):
    """Rows a1-a9: constitutive update, residual F1..F3 and the operator apply."""
    inp = ms.random_rve(shape, 7)
    eps, E, phi, H = ms.random_state(inp, 8)
    pb = solver.problem_from_input(inp, isotropic=split == B.RVE_SPLIT_NONE)
    lin = solver.Linearization(pb, eps, E, phi, H)
    octrl = solver.CRACK if control == B.RVE_CTRL_CRACK else solver.STRAIN
    target = lin.Gamma + 0.5 if control == B.RVE_CTRL_CRACK else E * 1.1
    F1o, F2o, F3o = solver.residual(lin, octrl, target)
    g = _gpu_state_from(inp, eps, E, phi, H, B.RVE_FP64, split)
    g.linearize(control, target)
    F1, F2, F3 = g.residual()
    sig_scale = np.max(np.abs(lin.sigma))
    assert np.max(np.abs(F1 - B.mandel_from_tensor(F1o))) < 1e-11 * sig_scale
    assert np.max(np.abs(F2 - F2o.reshape(-1))) < 1e-11 * np.max(np.abs(F2o))
    assert abs(F3 - F3o) < 1e-11 * max(abs(target), 1.0)
    de, dp, dE = ms.random_direction(inp, 9)
    Jo = solver.jacobian_apply(lin, (de, dp, dE), octrl)
    Je, Jp, JE = g.apply(B.mandel_from_tensor(de), dp, dE)
    s1 = np.max(np.abs(Jo[0]))
    assert np.max(np.abs(Je - B.mandel_from_tensor(Jo[0]))) < 1e-11 * s1
    assert np.max(np.abs(Jp - Jo[1].reshape(-1))) < 1e-11 * np.max(np.abs(Jo[1]))
    assert abs(JE - Jo[2]) < 1e-11 * max(abs(Jo[2]), 1.0)
    g.close()


@pytest.mark.parametrize("shape", [(16, 16), (24, 36), (8, 8, 6), (64, 128), (128, 48), (8, 64, 128),
                                   (384, 192), (96, 384), (48, 96, 24), (24, 48, 96)])
def test_apply_mixed_precision(shape):
    """float32 apply (mixed path) within 1e-5 of the float64 oracle."""
    inp = ms.random_rve(shape, 17)
    eps, E, phi, H = ms.random_state(inp, 18)
    pb = solver.problem_from_input(inp)
    lin = solver.Linearization(pb, eps, E, phi, H)
    target = lin.Gamma + 0.5
    g = _gpu_state_from(inp, eps, E, phi, H, B.RVE_MIXED, B.RVE_SPLIT_SPECTRAL)
    g.linearize(B.RVE_CTRL_CRACK, target)
    de, dp, dE = ms.random_direction(inp, 19)
    Jo = solver.jacobian_apply(lin, (de, dp, dE), solver.CRACK)
    Je, Jp, JE = g.apply(B.mandel_from_tensor(de), dp, dE)
    assert np.max(np.abs(Je - B.mandel_from_tensor(Jo[0]))) < 1e-5 * np.max(np.abs(Jo[0]))
    assert np.max(np.abs(Jp - Jo[1].reshape(-1))) < 1e-5 * np.max(np.abs(Jo[1]))
    assert abs(JE - Jo[2]) < 1e-5 * max(abs(Jo[2]), 1.0)
    g.close()


class _OracleAlong:
    """The oracle advanced along the cut-back path the library took (Algorithm 2 with the
    cut-back reading R17): an increment the library took in one step is one oracle step, an
    increment it split into two committed halves (cutbacks == 1) is two oracle half steps.
    The oracle may not cut back on its own (max_depth = 0), so both sides run the same
    sequence of Newton solves and their converged states must agree."""

    def __init__(self, inp, isotropic=False, tol=1e-12):
        self.pb = solver.problem_from_input(inp, isotropic=isotropic)
        self.opt = solver.Options(newton_tol=tol, krylov_tol=tol)
        self.st, res, _ = solver.startup(self.pb, self.opt)
        assert all(r.converged for r in res[:3])

    def step(self, da, cutbacks):
        assert cutbacks in (0, 1), f"path with {cutbacks} cut-backs is not replayed"
        parts = [da] if cutbacks == 0 else [0.5 * da, 0.5 * da]
        for d in parts:
            r, rec = solver.crack_increment(self.pb, self.st, d, self.opt, max_depth=0)
            assert r.converged, ("the oracle does not converge on the library's path", cutbacks)
        rec["phi"] = self.st.phi.copy()
        return rec


def _case_input(case):
    if case == "panel32":
        return ms.homogeneous_panel(32, notch_len=8)
    if case == "composite24":
        return ms.fibre_composite(n=24, radius=3.0, fraction=0.3, notch_len=6, seed=5)
    if case == "composite32":
        return ms.fibre_composite(n=32, radius=4.0, fraction=0.3, notch_len=8, seed=21)
    if case == "composite48":
        return ms.fibre_composite(n=48, radius=5.0, fraction=0.35, notch_len=8, seed=7)
    return ms.porous_solid(n=8, radius=1.5, porosity=0.1, notch_radius=2.0, seed=6, E_pore=0.05)


@pytest.mark.parametrize("case", ["panel32", "composite24", "composite32", "composite48", "porous8"])
def test_crack_increments_fp64(case):
    """Rows a10-a11 end to end: start-up and crack-length-controlled increments, float64,
    against the oracle on the same cut-back path (1e-10 on E, Sigma, Gamma; 1e-8 on phi)."""
    inp = _case_input(case)
    n_inc = 3
    orc = _OracleAlong(inp)
    g = B.RVE(inp, precision=B.RVE_FP64, newton_tol=1e-12, krylov_tol=1e-12)
    g.startup()
    cuts = []
    for k in range(n_inc):
        s = g.crack_increment(1.0)
        cuts.append(s["cutbacks"])
        o = orc.step(1.0, s["cutbacks"])
        sig_o = B.mandel_from_tensor(o["Sigma"][None])[:, 0]
        sig = np.array(s["sigma"][: g.m])
        assert abs(s["E"] - o["E"]) <= 1e-10 * abs(o["E"]), (k, s["E"], o["E"], cuts)
        assert np.max(np.abs(sig - sig_o)) <= 1e-10 * np.max(np.abs(sig_o)), (k, sig, sig_o, cuts)
        assert abs(s["gamma"] - o["Gamma"]) <= 1e-10 * o["Gamma"]
        assert abs(s["tau"] - o["tau"]) <= 1e-10 * o["tau"]
    phi = g.field(B.RVE_FIELD_PHI)
    assert np.max(np.abs(phi - o["phi"].reshape(-1))) < 1e-8
    print(case, "cut-back path", cuts)
    g.close()


@pytest.mark.parametrize("case", ["panel32", "composite32"])
def test_crack_increments_mixed_precision(case):
    """Mixed path: 1e-5 on E and Sigma per increment, identical crack path {phi > 0.5}, against
    the float64 oracle on the same cut-back path."""
    if case == "panel32":
        inp = ms.homogeneous_panel(32, notch_len=8)
    else:
        inp = ms.fibre_composite(n=32, radius=3.0, fraction=0.3, notch_len=6, seed=11)
    n_inc = 3
    orc = _OracleAlong(inp)
    g = B.RVE(inp, precision=B.RVE_MIXED)
    g.startup()
    for k in range(n_inc):
        s = g.crack_increment(1.0)
        o = orc.step(1.0, s["cutbacks"])
        sig_o = B.mandel_from_tensor(o["Sigma"][None])[:, 0]
        assert abs(s["E"] - o["E"]) <= 1e-5 * abs(o["E"])
        assert np.max(np.abs(np.array(s["sigma"][:3]) - sig_o)) <= 1e-5 * np.max(np.abs(sig_o))
    phi = g.field(B.RVE_FIELD_PHI)
    po = o["phi"].reshape(-1)
    tie = np.abs(po - 0.5) < 1e-6
    assert np.array_equal((phi > 0.5)[~tie], (po > 0.5)[~tie])
    g.close()


@pytest.mark.parametrize("shape", [(16, 16), (24, 36), (64, 128), (8, 8, 6), (8, 64, 128)])
@pytest.mark.parametrize("precision", [B.RVE_FP64, B.RVE_MIXED])
def test_residual_and_apply_continuous_projector(shape, precision):
    """Galerkin projection with continuous frequencies (RVE_GAMMA_CONTINUOUS): residual and
    scaled apply against the oracle's Problem(gamma="continuous")."""
    inp = ms.random_rve(shape, 9)
    pb = solver.problem_from_input(inp, gamma="continuous")
    eps, E, phi, H = ms.random_state(inp, 5)
    lin = solver.Linearization(pb, eps, E, phi, H)
    F1o, F2o, _ = solver.residual(lin, solver.CRACK, lin.Gamma + 1.0)
    g = B.RVE(inp, precision=precision, gamma_op=B.RVE_GAMMA_CONTINUOUS)
    g.set_state(B.mandel_from_tensor(eps), phi, H, E, 0.0)
    g.linearize(B.RVE_CTRL_CRACK, lin.Gamma + 1.0)
    F1, F2, _ = g.residual()
    sig_scale = np.max(np.abs(lin.sigma))
    assert np.max(np.abs(F1 - B.mandel_from_tensor(F1o))) < 1e-11 * sig_scale
    assert np.max(np.abs(F2 - F2o.reshape(-1))) < 1e-11 * np.max(np.abs(F2o))
    de, dp, dE = ms.random_direction(inp, 6)
    Jo = solver.jacobian_apply(lin, (de, dp, dE), solver.CRACK)
    Je, Jp, JE = g.apply(B.mandel_from_tensor(de), dp, dE)
    tol = 1e-11 if precision == B.RVE_FP64 else 1e-5
    assert np.max(np.abs(Je - B.mandel_from_tensor(Jo[0]))) < tol * np.max(np.abs(Jo[0]))
    assert np.max(np.abs(Jp - Jo[1].reshape(-1))) < tol * np.max(np.abs(Jo[1]))
    assert abs(JE - Jo[2]) < tol * max(abs(Jo[2]), 1.0)
    g.close()


def test_crack_increments_shear_loading():
    """Shear control tensor f = e_x e_y + e_y e_x: start-up and increments, float64, against
    the oracle (variant of Table 1 loading)."""
    inp = ms.homogeneous_panel(32, notch_len=8)
    inp.f = ms.shear_f(2)
    n_inc = 2
    orc = _OracleAlong(inp)
    g = B.RVE(inp, precision=B.RVE_FP64, newton_tol=1e-12, krylov_tol=1e-12)
    g.startup()
    for k in range(n_inc):
        s = g.crack_increment(1.0)
        o = orc.step(1.0, s["cutbacks"])
        sig_o = B.mandel_from_tensor(o["Sigma"][None])[:, 0]
        assert abs(s["E"] - o["E"]) <= 1e-10 * abs(o["E"]), (k, s["E"], o["E"])
        assert np.max(np.abs(np.array(s["sigma"][:3]) - sig_o)) <= 1e-10 * np.max(np.abs(sig_o))
    g.close()


@pytest.mark.parametrize("precision", [B.RVE_FP64, B.RVE_MIXED])
def test_staggered_increments_against_oracle(precision):
    """Algorithm 1 on the GPU (rve_staggered_increment) against the oracle's staggered
    increments, and equal to the monolithic strain-controlled increment (stable regime)."""
    inp = ms.homogeneous_panel(16, notch_len=4)
    pb = solver.problem_from_input(inp)
    opt = solver.Options(newton_tol=1e-13, krylov_tol=1e-13)
    _, _, Es = solver.startup(pb, opt)
    st = solver.initial_state(pb)
    r, _ = solver.strain_increment(pb, st, 0.6 * Es, opt)
    recs = []
    for f in (0.8, 1.0):
        _, rec = solver.staggered_increment(pb, st, f * Es, tol=1e-11, mech_tol=1e-10)
        rec["phi"] = st.phi.copy()
        recs.append(rec)
    kw = dict(newton_tol=1e-12, krylov_tol=1e-12) if precision == B.RVE_FP64 else dict(newton_tol=1e-10)
    tol = 1e-9 if precision == B.RVE_FP64 else 1e-5
    g = B.RVE(inp, precision=precision, **kw)
    mono = B.RVE(inp, precision=precision, **kw)
    g.strain_increment(0.6 * Es)
    mono.strain_increment(0.6 * Es)
    for f, o in zip((0.8, 1.0), recs):
        s = g.staggered_increment(f * Es, tol=1e-11)
        m = mono.strain_increment(f * Es)
        sig_o = B.mandel_from_tensor(o["Sigma"][None])[:, 0]
        sig = np.array(s["sigma"][:3])
        assert s["sweeps"] > 2
        assert np.max(np.abs(sig - sig_o)) <= tol * np.max(np.abs(sig_o)), (f, sig, sig_o)
        assert np.max(np.abs(sig - np.array(m["sigma"][:3]))) <= tol * np.max(np.abs(sig_o))
        assert abs(s["gamma"] - o["Gamma"]) <= tol * o["Gamma"]
    phi = g.field(B.RVE_FIELD_PHI)
    assert np.max(np.abs(phi - recs[-1]["phi"].reshape(-1))) < (1e-8 if precision == B.RVE_FP64 else 1e-4)
    g.close()
    mono.close()


def test_panel64_against_stored_oracle():
    """64 x 64 panel, 20 increments (stored oracle values, tests/golden/make_golden.py)."""
    path = os.path.join(HERE, "golden", "panel64_crack.json")
    gold = json.load(open(path))
    inp = ms.homogeneous_panel(64, notch_len=16)
    g = B.RVE(inp, precision=B.RVE_FP64, newton_tol=1e-12, krylov_tol=1e-12)
    g.startup()
    for row in gold["rows"][1:]:
        s = g.crack_increment(1.0)
        sig_o = B.mandel_from_tensor(np.array(row["Sigma"])[None])[:, 0]
        assert abs(s["E"] - row["E"]) <= 1e-10 * abs(row["E"]), row["inc"]
        assert np.max(np.abs(np.array(s["sigma"][:3]) - sig_o)) <= 1e-10 * np.max(np.abs(sig_o)), row["inc"]
    g.close()


def test_panel64_mixed_against_stored_oracle():
    """Mixed path on the 64 x 64 panel (compile-time FFT lengths): 1e-5 on E and Sigma."""
    gold = json.load(open(os.path.join(HERE, "golden", "panel64_crack.json")))
    inp = ms.homogeneous_panel(64, notch_len=16)
    g = B.RVE(inp, precision=B.RVE_MIXED)
    g.startup()
    for row in gold["rows"][1:9]:
        s = g.crack_increment(1.0)
        sig_o = B.mandel_from_tensor(np.array(row["Sigma"])[None])[:, 0]
        assert abs(s["E"] - row["E"]) <= 1e-5 * abs(row["E"]), row["inc"]
        assert np.max(np.abs(np.array(s["sigma"][:3]) - sig_o)) <= 1e-5 * np.max(np.abs(sig_o)), row["inc"]
    g.close()


def test_rollback_and_checkpoint(tmp_path):
    """A failed increment leaves the committed state; a checkpoint resumes bit-exactly."""
    inp = ms.homogeneous_panel(16, notch_len=4)
    g = B.RVE(inp)
    g.startup()
    g.crack_increment(1.0)
    phi0 = g.field(B.RVE_FIELD_PHI)
    sig0, E0 = g.macro_stress()
    path = str(tmp_path / "rve.ckpt")
    g.save(path)
    a = g.crack_increment(1.0)
    g2 = B.RVE.load(path)
    b = g2.crack_increment(1.0)
    assert a["E"] == b["E"] and a["sigma"] == b["sigma"]
    # a Newton limit of 1 fails (RVE_E_NOCONV) and leaves the committed state untouched
    g3 = B.RVE(inp, newton_max=1)
    g3.set_state(g2.field(B.RVE_FIELD_EPS_T), g2.field(B.RVE_FIELD_PHI), g2.field(B.RVE_FIELD_H),
                 b["E"], b["tau"])
    before = g3.field(B.RVE_FIELD_PHI)
    with pytest.raises(B.RVEError) as ei:
        g3.crack_increment(1.0)
    assert ei.value.code == B.RVE_E_NOCONV
    assert np.array_equal(g3.field(B.RVE_FIELD_PHI), before)
    assert g3.macro_stress()[1] == b["E"]
    g.close()
    g2.close()
    g3.close()


def test_merged_vector_update_option_matches_oracle():
    """The opt-in merged BiCGStab vector update (RVE_MERGED_UPDATE=1, read once per process, so
    run in a child process): mixed crack increments of a 32^2 composite within 1e-5 of the
    oracle, like the default path."""
    import subprocess
    import sys
    code = (
        "import json, sys\n"
        "sys.path.insert(0, %r)\n"
        "from paper_2412_17445_gb300 import binding as B, microstructure as ms\n"
        "inp = ms.fibre_composite(n=32, radius=3.0, fraction=0.3, notch_len=6, seed=11)\n"
        "g = B.RVE(inp, precision=B.RVE_MIXED)\n"
        "g.startup()\n"
        "print(json.dumps([g.crack_increment(1.0) for _ in range(3)]))\n"
    ) % os.path.dirname(HERE)
    env = dict(os.environ, RVE_MERGED_UPDATE="1")
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    recs = json.loads(out.stdout.strip().splitlines()[-1])
    inp = ms.fibre_composite(n=32, radius=3.0, fraction=0.3, notch_len=6, seed=11)
    orc = _OracleAlong(inp)
    for s in recs:
        o = orc.step(1.0, s["cutbacks"])
        sig_o = B.mandel_from_tensor(o["Sigma"][None])[:, 0]
        assert abs(s["E"] - o["E"]) <= 1e-5 * abs(o["E"])
        assert np.max(np.abs(np.array(s["sigma"][:3]) - sig_o)) <= 1e-5 * np.max(np.abs(sig_o))


@pytest.mark.parametrize("variant", [1, 2, 3])
@pytest.mark.parametrize("shape", [(72, 36), (64, 128), (12, 24, 32)])
def test_residual_and_apply_with_forced_radix_plan(shape, variant, monkeypatch):
    """The radix plans the autotuner chooses among (variant 1: the default radices reversed;
    2: radix 4 instead of 8; 3: those reversed), forced on every axis through RVE_RADIX_PLAN
    (compile-time lengths then run the runtime-length kernels): residual FP64 at 1e-11, apply
    FP64 at 1e-11 and MIXED at 1e-5 against the oracle."""
    monkeypatch.setenv("RVE_RADIX_PLAN", str(variant))
    inp = ms.random_rve(shape, 27)
    eps, E, phi, H = ms.random_state(inp, 28)
    pb = solver.problem_from_input(inp)
    lin = solver.Linearization(pb, eps, E, phi, H)
    target = lin.Gamma + 0.5
    F1o, F2o, F3o = solver.residual(lin, solver.CRACK, target)
    de, dp, dE = ms.random_direction(inp, 29)
    Jo = solver.jacobian_apply(lin, (de, dp, dE), solver.CRACK)
    for prec, tol in ((B.RVE_FP64, 1e-11), (B.RVE_MIXED, 1e-5)):
        g = _gpu_state_from(inp, eps, E, phi, H, prec, B.RVE_SPLIT_SPECTRAL)
        g.linearize(B.RVE_CTRL_CRACK, target)
        if prec == B.RVE_FP64:
            F1, F2, F3 = g.residual()
            assert np.max(np.abs(F1 - B.mandel_from_tensor(F1o))) < 1e-11 * np.max(np.abs(lin.sigma))
            assert np.max(np.abs(F2 - F2o.reshape(-1))) < 1e-11 * np.max(np.abs(F2o))
            assert abs(F3 - F3o) < 1e-11 * max(abs(target), 1.0)
        Je, Jp, JE = g.apply(B.mandel_from_tensor(de), dp, dE)
        assert np.max(np.abs(Je - B.mandel_from_tensor(Jo[0]))) < tol * np.max(np.abs(Jo[0])), prec
        assert np.max(np.abs(Jp - Jo[1].reshape(-1))) < tol * np.max(np.abs(Jo[1])), prec
        assert abs(JE - Jo[2]) < tol * max(abs(Jo[2]), 1.0), prec
        g.close()


@pytest.mark.parametrize("shape", [(72, 36), (12, 24, 32)])
def test_tuned_radix_plans_match_the_oracle(shape):
    """Lengths without compile-time kernels (72, 36, 32, 24, 12) get their radix plans from the
    autotuner's timings: the tuned handle's apply still equals the oracle's Jacobian."""
    inp = ms.random_rve(shape, 31)
    eps, E, phi, H = ms.random_state(inp, 32)
    pb = solver.problem_from_input(inp)
    lin = solver.Linearization(pb, eps, E, phi, H)
    target = lin.Gamma + 0.5
    de, dp, dE = ms.random_direction(inp, 33)
    Jo = solver.jacobian_apply(lin, (de, dp, dE), solver.CRACK)
    for prec, tol in ((B.RVE_FP64, 1e-11), (B.RVE_MIXED, 1e-5)):
        g = _gpu_state_from(inp, eps, E, phi, H, prec, B.RVE_SPLIT_SPECTRAL)
        g.autotune()
        g.linearize(B.RVE_CTRL_CRACK, target)
        Je, Jp, JE = g.apply(B.mandel_from_tensor(de), dp, dE)
        assert np.max(np.abs(Je - B.mandel_from_tensor(Jo[0]))) < tol * np.max(np.abs(Jo[0])), prec
        assert np.max(np.abs(Jp - Jo[1].reshape(-1))) < tol * np.max(np.abs(Jo[1])), prec
        g.close()
