"""Failure handling, with every fault made on the host (nothing here faults, traps or hangs
the GPU): a non-finite host input, a BiCGStab breakdown forced through the library's
RVE_FAULT hook, and a device allocation failure forced through the same hook.  Each call
fails with its status code and leaves the RVE (or the device memory) as it was."""
import numpy as np
import pytest

from paper_2412_17445_gb300 import binding as B
from paper_2412_17445_gb300 import microstructure as ms

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2412_17445_gb300 import build
    build.build()
    B.lib()


def _started_panel():
    g = B.RVE(ms.homogeneous_panel(16, notch_len=4))
    g.startup()
    g.crack_increment(1.0)
    return g


def test_non_finite_host_state_is_rejected_and_state_kept():
    g = _started_panel()
    eps = g.field(B.RVE_FIELD_EPS_T)
    phi = g.field(B.RVE_FIELD_PHI)
    H = g.field(B.RVE_FIELD_H)
    sig0, E0 = g.macro_stress()
    for bad in ("eps", "phi", "H", "E"):
        e2, p2, h2, E2 = eps.copy(), phi.copy(), H.copy(), E0
        if bad == "eps":
            e2[1, 7] = np.nan
        elif bad == "phi":
            p2[3] = np.inf
        elif bad == "H":
            h2[5] = -np.inf
        else:
            E2 = np.nan
        with pytest.raises(B.RVEError) as ei:
            g.set_state(e2, p2, h2, E2, 5.0)
        assert ei.value.code == B.RVE_E_ARG
        assert "finite" in str(ei.value)
    assert np.array_equal(g.field(B.RVE_FIELD_PHI), phi)
    sig1, E1 = g.macro_stress()
    assert E1 == E0 and np.array_equal(sig1, sig0)
    g.crack_increment(1.0)  # the handle still works
    g.close()


def test_forced_krylov_breakdown_fails_the_increment_and_keeps_the_state(tmp_path, monkeypatch):
    g = _started_panel()
    path = str(tmp_path / "panel.ckpt")
    g.save(path)
    phi0 = g.field(B.RVE_FIELD_PHI)
    sig0, E0 = g.macro_stress()
    g.close()
    monkeypatch.setenv("RVE_FAULT", "krylov_breakdown")
    h = B.RVE.load(path)  # rve_load creates the handle: the hook is armed for it
    monkeypatch.delenv("RVE_FAULT")
    with pytest.raises(B.RVEError) as ei:
        h.crack_increment(1.0)
    assert ei.value.code == B.RVE_E_NOCONV
    assert np.array_equal(h.field(B.RVE_FIELD_PHI), phi0)
    sig1, E1 = h.macro_stress()
    assert E1 == E0 and np.array_equal(sig1, sig0)
    h.close()
    ok = B.RVE.load(path)  # the same checkpoint without the hook advances normally
    r = ok.crack_increment(1.0)
    assert r["tau"] > 0 and r["newton_iters"] >= 1
    ok.close()


@pytest.mark.parametrize("k", [1, 3, 7])
def test_forced_allocation_failure_is_oom_without_leak(monkeypatch, k):
    import torch
    torch.cuda.synchronize()
    inp = ms.fibre_composite(n=64, radius=6.0, fraction=0.3, notch_len=8, seed=3)
    probe = B.RVE(inp, precision=B.RVE_MIXED)  # warm the context and the library's static state
    probe.close()
    free0, _ = torch.cuda.mem_get_info()
    monkeypatch.setenv("RVE_FAULT", f"alloc:{k}")
    with pytest.raises(B.RVEError) as ei:
        B.RVE(inp, precision=B.RVE_MIXED)
    monkeypatch.delenv("RVE_FAULT")
    assert ei.value.code == B.RVE_E_OOM
    assert "injected" in str(ei.value)
    free1, _ = torch.cuda.mem_get_info()
    assert free1 >= free0 - (2 << 20)
    g = B.RVE(inp, precision=B.RVE_MIXED)  # creation works again
    g.close()
