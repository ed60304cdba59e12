"""Host-only logic of librve (no GPU call): footprint accounting, descriptor validation,
and the multi-rank helpers of bench.py on CPU gloo ranks."""
import os
import socket

import numpy as np
import pytest

from paper_2412_17445_gb300 import microstructure as ms


@pytest.fixture(scope="module")
def B():
    from paper_2412_17445_gb300 import binding, build
    build.build()
    binding.lib()
    return binding


def test_footprint_scales_with_grid_and_precision(B):
    a = B.footprint(ms.homogeneous_panel(64), B.RVE_FP64)
    b = B.footprint(ms.homogeneous_panel(128), B.RVE_FP64)
    c = B.footprint(ms.homogeneous_panel(128), B.RVE_MIXED)
    assert 3.5 * a < b < 4.5 * a          # ~ linear in the voxel count
    assert c < b                          # float32 Krylov vectors and tangent
    n = 128 * 128
    assert 300 * n < c < 500 * n          # bytes per voxel of the mixed 2D solver


def test_server_rejects_requests_beyond_budget(B):
    import ctypes
    inp = ms.homogeneous_panel(64)
    need = B.footprint(inp)
    d, keep = B.make_desc(inp)
    h = ctypes.c_void_p()
    L = B.lib()
    assert L.rve_server_create(need // 2, 4, ctypes.byref(h)) == B.RVE_OK
    rid = ctypes.c_longlong()
    assert L.rve_server_submit(h, ctypes.byref(d), None, 1, 1.0, ctypes.byref(rid)) == B.RVE_E_OOM
    assert L.rve_server_submit(h, None, None, 1, 1.0, ctypes.byref(rid)) == B.RVE_E_ARG
    used, act, q = ctypes.c_longlong(), ctypes.c_int(), ctypes.c_int()
    L.rve_server_stats(h, ctypes.byref(used), ctypes.byref(act), ctypes.byref(q))
    assert (used.value, act.value, q.value) == (0, 0, 0)
    L.rve_server_destroy(h)


def test_footprint_counts_energy_control_work_space(B):
    """Energy control adds exactly m x n float64 of work space (2D m = 3, 3D m = 6)."""
    for inp, m in ((ms.homogeneous_panel(64), 3), (ms.porous_solid(n=16, radius=2.0, notch_radius=3.0), 6)):
        n = int(np.prod(inp.shape))
        for prec in (B.RVE_FP64, B.RVE_MIXED):
            extra = B.footprint(inp, prec, B.RVE_CONSTRAINT_ENERGY) - B.footprint(inp, prec)
            assert extra == 8 * m * n


def _supported(N):
    while N % 2 == 0:
        N //= 2
    while N % 3 == 0:
        N //= 3
    return N == 1


def test_workload_generators_only_make_supported_grids():
    """Every grid of the ragged batch and of the served stream has extents 2^a 3^b <= 4096 (the
    library's FFT plans), a phase map of its shape and a non-empty notch."""
    from paper_2412_17445_gb300 import workloads_bench as wb
    inps = wb._ragged_inputs() + [inp for inp, _ in wb._serve_requests(32)]
    assert len(inps) == 96
    for inp in inps:
        assert all(_supported(s) and s <= 4096 for s in inp.shape), inp.shape
        assert inp.phase.shape == tuple(inp.shape) and inp.notch.shape == tuple(inp.shape)
        assert inp.notch.any()
