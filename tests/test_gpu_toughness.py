"""Effective toughness from a solved crack-controlled curve (Sec. 2.4, Eq. JaviGc; Sec. 4.2;
Appendix A): a homogeneous panel is cracked across the whole periodic cell on the GPU, the
area under its (E, Sigma:f) curve gives G_Ceff through rve_effective_toughness, and

  * on a 32 x 32 panel the float64 GPU curve and its G_Ceff equal the oracle's stored curve
    (tests/golden/panel32_crossing.json) increment by increment;
  * on a 256 x 256 panel the mixed-precision G_Ceff lies within 5 % of G_c A(l/h) with the
    appendix amplification factor A(2) of the discrete crack functional.

Reading (Eq. JaviGc with an initial crack): the external work only pays for the crack that
grows, so L_g is the cell width minus the initial notch length.
"""
import json
import os

import numpy as np
import pytest

from oracle import postprocess
from paper_2412_17445_gb300 import binding as B
from paper_2412_17445_gb300 import microstructure as ms

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2412_17445_gb300 import build
    build.build()
    B.lib()


def _crack_across(g, n, max_inc, peak0):
    """Crack-length increments of 1 until {phi > 0.5} covers the notch row and Sigma_yy is
    below 1 % of its peak.  Returns the (E, Sigma_yy) points after the start-up point."""
    E, S = [], []
    peak = peak0
    for _ in range(max_inc):
        r = g.crack_increment(1.0)
        E.append(r["E"])
        S.append(r["sigma"][1])
        peak = max(peak, r["sigma"][1])
        row = g.field(B.RVE_FIELD_PHI).reshape(n, n)[n // 2]
        if np.all(row > 0.5) and r["sigma"][1] < 0.01 * peak:
            return E, S, True
    return E, S, False


def test_panel32_curve_and_toughness_match_the_oracle():
    gold = json.load(open(os.path.join(HERE, "golden", "panel32_crossing.json")))
    n, a0 = gold["n"], gold["notch"]
    g = B.RVE(ms.homogeneous_panel(n, notch_len=a0), precision=B.RVE_FP64, newton_tol=1e-10, krylov_tol=1e-12)
    s0 = g.startup()
    rows = gold["rows"]
    E, S = [s0["E"]], [s0["sigma"][1]]
    for row in rows[1:]:
        r = g.crack_increment(1.0)
        assert r["cutbacks"] == row["cutbacks"], row["inc"]
        assert abs(r["E"] - row["E"]) <= 1e-8 * abs(row["E"]), (row["inc"], r["E"], row["E"])
        assert abs(r["sigma"][1] - row["Sigma"][1][1]) <= 1e-8 * max(abs(x["Sigma"][1][1]) for x in rows), row["inc"]
        E.append(r["E"])
        S.append(r["sigma"][1])
    g.close()
    Eo = [r["E"] for r in rows]
    So = [r["Sigma"][1][1] for r in rows]
    G_o = postprocess.effective_toughness(Eo, So, n * n, n - a0)
    G = B.effective_toughness(E, S, area=n * n, length=n - a0)
    assert abs(G - G_o) <= 1e-8 * G_o, (G, G_o)


def test_panel256_effective_toughness_near_gc_times_amplification():
    n, a0, Gc = 256, 32, 1e-3
    g = B.RVE(ms.homogeneous_panel(n, notch_len=a0, Gc=Gc), precision=B.RVE_MIXED, newton_tol=1e-8)
    s0 = g.startup()
    E, S, crossed = _crack_across(g, n, 600, s0["sigma"][1])
    g.close()
    assert crossed, (len(E), S[-3:])
    G = B.effective_toughness([s0["E"]] + E, [s0["sigma"][1]] + S, area=n * n, length=n - a0)
    A = postprocess.amplification_factor(2.0)
    print(f"G_Ceff {G:.6e}  G_c A(2) {Gc * A:.6e}  ratio {G / (Gc * A):.4f}  increments {len(E)}")
    assert abs(G / (Gc * A) - 1.0) < 0.05
