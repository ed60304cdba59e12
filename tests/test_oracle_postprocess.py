"""Pins of the post-processing (Eq. JaviGc, appendix amplification factor) against the
numbers the paper prints (tests/golden/paper_values.json) and closed forms."""
import json
import os

import numpy as np
import pytest

from oracle import postprocess

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_amplification_fit_matches_paper():
    """Least-squares fit A = 1 + a/(l/h) over l/h in [1, 8] gives the printed a = 0.298."""
    r = np.array([1.0, 1.5, 2.0, 3.0, 4.0, 6.0, 8.0])
    A = np.array([postprocess.amplification_factor(x) for x in r])
    a = np.sum((A - 1.0) / r) / np.sum(1.0 / r ** 2)
    assert abs(a - GOLD["fft_amplification_fit_a"]["value"]) < 0.01 * 0.298
    # and it lies below Bourdin's FEM value (Eq. BourdinGc) at every l/h
    assert np.all(A < 1.0 + GOLD["fem_bourdin_a"]["value"] / r)


def test_amplification_continuum_limit():
    assert abs(postprocess.amplification_factor(40.0, N=2049) - 1.0) < 0.01


def test_paper_griffith_average_consistent_with_fit():
    """The printed panel average 3232.6 is within the printed 5% of G_c (1 + a/(l/h))."""
    g = GOLD["griffith_panels_Gceff_avg"]
    Gc_o = g["Gc"] * postprocess.amplification_factor(g["l_over_h"])
    assert abs(g["value"] / Gc_o - 1.0) < g["tolerance_vs_Gceff_o"]


def test_effective_toughness_closed_form():
    """Linear loading to E_f then linear softening to zero: area = S_max E_end / 2."""
    E = np.linspace(0.1, 1.0, 10)
    S = 2.0 * E
    assert abs(postprocess.effective_toughness(E, S, area=4.0, length=2.0) - 4.0 / 2.0 * 1.0) < 1e-14
    E2 = np.array([1.0, 1.5, 2.0])
    S2 = np.array([2.0, 1.0, 0.0])
    assert abs(postprocess.effective_toughness(E2, S2, 1.0, 1.0) - (1.0 + 0.75 + 0.25)) < 1e-14


def test_c_abi_effective_toughness_matches_oracle():
    """rve_effective_toughness (host arithmetic of librve, no GPU) equals the oracle's."""
    import ctypes
    from paper_2412_17445_gb300 import binding as B, build
    build.build()
    rng = np.random.default_rng(3)
    E = np.cumsum(rng.random(30)) * 1e-3
    S = rng.random(30) * 1e-2
    want = postprocess.effective_toughness(E, S, area=4096.0, length=64.0)
    got = B.effective_toughness(E, S, area=4096.0, length=64.0)
    assert abs(got - want) <= 1e-14 * abs(want)
