"""Full-size parity on the workload the headline benchmark times: the 512 x 512 fibre
composite (RSA discs r = 12 at 40 %, E_f/E_m = 10, Gc_f/Gc_m = 5, l = 2, central notch of
32 voxels, seed base + 1), start-up plus crack-length increments of da = 1, against the
float64 oracle's values stored by tests/golden/make_golden.py (Algorithm 2, Sec. 3.2).

  float64 path (Newton / Krylov 1e-12): E, Sigma, Gamma and tau within 1e-10 relative, the
      same cut-back path, the crack path {phi > 0.5} voxel-identical and phi near the notch
      within 1e-8;
  mixed path, run as the benchmark runs it (a batch of independent 512^2 composites through
      rve_batch_crack_increment, grouped launches, Newton 1e-8, Krylov 1e-2): E and Sigma
      within 1e-5 relative and the crack path {phi > 0.5} voxel-identical, voxels within
      1e-6 of 0.5 in the oracle excepted (ties).
"""
import json
import os

import numpy as np
import pytest

from paper_2412_17445_gb300 import binding as B
from paper_2412_17445_gb300 import microstructure as ms

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = os.path.join(HERE, "golden", "composite512_crack.json")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2412_17445_gb300 import build
    build.build()
    B.lib()


@pytest.fixture(scope="module")
def gold():
    with open(GOLD) as f:
        g = json.load(f)
    assert len(g["rows"]) >= 4, "the stored run holds the start-up and at least 3 increments"
    return g


def _inp(k=0):
    return ms.fibre_composite(n=512, radius=12.0, fraction=0.4, notch_len=32, seed=ms.SEED_BASE + 1 + k)


def _crack_ok(phi, row):
    """{phi > 0.5} equals the oracle's crack voxels, except at the oracle's ties."""
    got = set(np.flatnonzero(phi > 0.5).tolist())
    want = set(row["crack"])
    ties = set(row["ties"])
    return (got ^ want) <= ties, sorted((got ^ want) - ties)[:10]


def _window(phi, row):
    w = row["phi_window"]
    a = phi.reshape(512, 512)[w["y0"]:w["y0"] + w["rows"], w["x0"]:w["x0"] + w["cols"]]
    return a.reshape(-1), np.array(w["values"])


def test_composite512_fp64_against_stored_oracle(gold):
    g = B.RVE(_inp(), precision=B.RVE_FP64, newton_tol=1e-12, krylov_tol=1e-12)
    s0 = g.startup()
    r0 = gold["rows"][0]
    assert abs(s0["E"] - r0["E"]) <= 1e-10 * abs(r0["E"])
    assert abs(s0["tau"] - r0["tau"]) <= 1e-10 * abs(r0["tau"])
    for row in gold["rows"][1:]:
        s = g.crack_increment(1.0)
        k = row["inc"]
        sig_o = B.mandel_from_tensor(np.array(row["Sigma"])[None])[:, 0]
        assert s["cutbacks"] == row["cutbacks"], (k, s["cutbacks"], row["cutbacks"])
        assert abs(s["E"] - row["E"]) <= 1e-10 * abs(row["E"]), (k, s["E"], row["E"])
        assert np.max(np.abs(np.array(s["sigma"][:3]) - sig_o)) <= 1e-10 * np.max(np.abs(sig_o)), k
        assert abs(s["gamma"] - row["Gamma"]) <= 1e-10 * row["Gamma"], k
        assert abs(s["tau"] - row["tau"]) <= 1e-10 * row["tau"], k
        phi = g.field(B.RVE_FIELD_PHI)
        ok, diff = _crack_ok(phi, row)
        assert ok, (k, diff)
        got, want = _window(phi, row)
        assert np.max(np.abs(got - want)) < 1e-8, k
    g.close()


def test_composite512_mixed_batched_against_stored_oracle(gold):
    """The benchmark's configuration: four independent composites (the stored one first) in
    one rve_batch_crack_increment per increment, MIXED, Newton 1e-8, Krylov 1e-2."""
    gs = [B.RVE(_inp(k), precision=B.RVE_MIXED, newton_tol=1e-8, krylov_tol=1e-2) for k in range(4)]
    for x in gs:
        x.startup()
    r0 = gold["rows"][0]
    s0, E0 = gs[0].macro_stress()
    assert abs(E0 - r0["E"]) <= 1e-5 * abs(r0["E"])
    errs = []
    for row in gold["rows"][1:]:
        out, st = B.batch_crack_increment(gs, [1.0] * len(gs))
        assert st == [0] * len(gs)
        s = out[0]
        k = row["inc"]
        sig_o = B.mandel_from_tensor(np.array(row["Sigma"])[None])[:, 0]
        eE = abs(s["E"] - row["E"]) / abs(row["E"])
        eS = np.max(np.abs(np.array(s["sigma"][:3]) - sig_o)) / np.max(np.abs(sig_o))
        errs.append((k, eE, eS))
        assert eE <= 1e-5 and eS <= 1e-5, (k, eE, eS)
        assert abs(s["gamma"] - row["Gamma"]) <= 1e-5 * row["Gamma"], k
        ok, diff = _crack_ok(gs[0].field(B.RVE_FIELD_PHI), row)
        assert ok, (k, diff)
    print("mixed vs oracle (inc, rel E, rel Sigma):", errs)
    for x in gs:
        x.close()
