"""Batched and served RVEs of uneven sizes (2D and 3D): every result is the same
alone and in the mix, and admission keeps the resident RVEs within the HBM budget."""
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


def _inputs():
    return [ms.homogeneous_panel(32, notch_len=8),
            ms.fibre_composite(n=32, radius=3.0, fraction=0.3, notch_len=6, seed=11),
            ms.porous_solid(n=8, radius=1.5, porosity=0.1, notch_radius=2.0, seed=6, E_pore=0.05),
            ms.homogeneous_panel(48, notch_len=12)]


@pytest.mark.parametrize("precision", [B.RVE_FP64, B.RVE_MIXED])
def test_batch_equals_separate_increments(precision):
    n_inc = 2
    alone = []
    for inp in _inputs():
        g = B.RVE(inp, precision=precision)
        g.startup()
        for _ in range(n_inc):
            r = g.crack_increment(1.0)
        alone.append(r)
        g.close()
    gs = [B.RVE(inp, precision=precision) for inp in _inputs()]
    for g in gs:
        g.startup()
    for _ in range(n_inc):
        out, st = B.batch_crack_increment(gs, [1.0] * len(gs))
        assert st == [0] * len(gs)
    for a, b in zip(alone, out):
        assert a["E"] == b["E"] and a["sigma"] == b["sigma"] and a["gamma"] == b["gamma"]
    for g in gs:
        g.close()


@pytest.mark.parametrize("precision", [B.RVE_FP64, B.RVE_MIXED])
def test_grouped_launches_equal_separate_increments(precision):
    """Five RVEs of one shape in a batch run their Krylov chunks as grouped launches (groups
    of up to four members, one launch per pass); every result equals the RVE run alone."""
    inps = [ms.fibre_composite(n=32, radius=3.0, fraction=0.3, notch_len=6, seed=11 + k) for k in range(5)]
    n_inc = 2
    alone = []
    for inp in inps:
        g = B.RVE(inp, precision=precision)
        g.startup()
        for _ in range(n_inc):
            r = g.crack_increment(1.0)
        alone.append(r)
        g.close()
    gs = [B.RVE(inp, precision=precision) for inp in inps]
    for g in gs:
        g.startup()
    for _ in range(n_inc):
        out, st = B.batch_crack_increment(gs, [1.0] * len(gs))
        assert st == [0] * len(gs)
    for a, b in zip(alone, out):
        assert a["E"] == b["E"] and a["sigma"] == b["sigma"] and a["gamma"] == b["gamma"]
        assert a["krylov_iters"] == b["krylov_iters"]
    for g in gs:
        g.close()


def test_server_results_same_alone_and_in_mix():
    reqs = _inputs()
    alone = []
    for inp in reqs:
        s = B.Server(hbm_budget_bytes=8 << 30, max_active=4)
        s.submit(inp, n_increments=2, precision=B.RVE_MIXED)
        s.drain()
        (r,) = s.poll()
        assert r["status"] == 0, r["error"]
        alone.append(r)
        s.close()
    s = B.Server(hbm_budget_bytes=8 << 30, max_active=8)
    ids = [s.submit(inp, n_increments=2, precision=B.RVE_MIXED) for inp in reqs]
    s.drain()
    mix = {r["id"]: r for r in s.poll()}
    s.close()
    assert sorted(mix) == sorted(ids)
    for rid, a in zip(ids, alone):
        b = mix[rid]
        assert b["status"] == 0 and b["n_increments"] == 2
        assert a["E"] == b["E"] and a["sigma"] == b["sigma"] and a["gamma"] == b["gamma"]


def test_server_admission_respects_budget():
    inp = ms.homogeneous_panel(48, notch_len=12)
    fp = B.footprint(inp, B.RVE_MIXED)
    budget = int(2.5 * fp)  # room for two resident RVEs
    s = B.Server(hbm_budget_bytes=budget, max_active=16)
    for _ in range(6):
        s.submit(inp, n_increments=1, precision=B.RVE_MIXED)
    s.drain()
    res = s.poll()
    s.close()
    assert len(res) == 6 and all(r["status"] == 0 for r in res)
    for r in res:
        t = r["t_start"]
        resident = sum(q["footprint"] for q in res if q["t_start"] <= t < q["t_end"])
        assert resident <= budget
    # with two slots the six requests needed at least three admission waves
    starts = sorted(r["t_start"] for r in res)
    ends = sorted(r["t_end"] for r in res)
    assert starts[2] >= ends[0] - 1e-9


def _threads():
    import os
    return len(os.listdir("/proc/self/task"))


def test_server_threads_bounded():
    """The server runs requests on a fixed pool of max_active worker threads: serving many
    more requests than slots keeps the process's thread count where server creation left it,
    and destroying the server returns it to the count before."""
    inp = ms.homogeneous_panel(16, notch_len=4)
    before = _threads()
    s = B.Server(hbm_budget_bytes=1 << 30, max_active=2)
    created = _threads()
    assert created <= before + 3  # two workers and the scheduler
    for _ in range(12):
        s.submit(inp, n_increments=1, precision=B.RVE_MIXED)
    peak = created
    import time
    while True:
        st = s.stats()
        peak = max(peak, _threads())
        if st["active"] == 0 and st["queued"] == 0:
            break
        time.sleep(0.002)
    s.drain()
    res = s.poll()
    assert len(res) == 12 and all(r["status"] == 0 for r in res)
    assert peak == created and _threads() == created
    s.close()
    assert _threads() == before


def test_server_admits_past_a_blocked_head():
    """A request that does not fit beside the resident RVEs does not block a later one that
    does: with A resident, B (too large to join A) waits while C (small) is admitted."""
    a = ms.homogeneous_panel(128, notch_len=32)
    b = ms.homogeneous_panel(256, notch_len=64)
    c = ms.homogeneous_panel(32, notch_len=8)
    fa, fb, fc = (B.footprint(x, B.RVE_MIXED) for x in (a, b, c))
    budget = max(fb, fa + fc)
    assert fa + fb > budget and fc < fb
    s = B.Server(hbm_budget_bytes=budget, max_active=4)
    ia = s.submit(a, n_increments=3, precision=B.RVE_MIXED)
    ib = s.submit(b, n_increments=1, precision=B.RVE_MIXED)
    ic = s.submit(c, n_increments=1, precision=B.RVE_MIXED)
    s.drain()
    res = {r["id"]: r for r in s.poll()}
    s.close()
    assert all(r["status"] == 0 for r in res.values())
    ra, rb, rc = res[ia], res[ib], res[ic]
    assert rc["t_start"] < ra["t_end"] <= rb["t_start"]
    for r in res.values():
        t = r["t_start"]
        assert sum(q["footprint"] for q in res.values() if q["t_start"] <= t < q["t_end"]) <= budget


@pytest.mark.parametrize("precision,shape", [(B.RVE_MIXED, (64, 128)), (B.RVE_FP64, (16, 16)), (B.RVE_MIXED, (8, 8, 6))])
def test_apply_device_batch_equals_single_applies(precision, shape):
    """rve_apply_device_batch (one launch per pass over three RVEs) gives, bit for bit, the
    outputs of rve_apply_device on each RVE."""
    import torch
    n = 3
    inps = [ms.random_rve(shape, 30 + k) for k in range(n)]
    gs = []
    for k, inp in enumerate(inps):
        g = B.RVE(inp, precision=precision)
        eps, E, phi, H = ms.random_state(inp, 40 + k)
        g.set_state(B.mandel_from_tensor(eps), phi, H, E, 0.0)
        g.linearize(B.RVE_CTRL_CRACK if k != 1 else B.RVE_CTRL_STRAIN, 1.0)
        gs.append(g)
    for g in gs:
        g.autotune()  # the first tunes this shape, the others take its tiles from the process cache
    dt = torch.float32 if precision == B.RVE_MIXED else torch.float64
    c, nv = gs[0].m + 1, gs[0].n
    gen = torch.Generator().manual_seed(5)
    xs = [torch.randn(c * nv, generator=gen, dtype=dt).cuda() for _ in gs]
    xEs = [torch.tensor([0.3 * (k + 1)], dtype=torch.float64).cuda() for k in range(n)]
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
