"""GPU test of rve_apply_device_noalloc, the allocation-free variant of rve_apply_device.

Callers that cannot allocate device memory when they call (CUDA graph capture, a host
allocator that owns the device memory, services that reserve everything at start-up) use
it; it must give the same result as rve_apply_device, bit for bit and call after call, while
drawing its scratch from the library's built-in device array.  Collected last (file name) so that a
run stopping at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from oracle import solver
from paper_2412_17445_gb300 import binding as B
from paper_2412_17445_gb300 import microstructure as ms

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2412_17445_gb300 import build
    build.build()
    B.lib()


def _linearized(shape, precision, seed=31):
    inp = ms.random_rve(shape, seed)
    eps, E, phi, H = ms.random_state(inp, seed + 1)
    pb = solver.problem_from_input(inp)
    gamma = solver.Linearization(pb, eps, E, phi, H).Gamma
    g = B.RVE(inp, precision=precision)
    g.set_state(B.mandel_from_tensor(eps), phi, H, E, 0.0)
    g.linearize(B.RVE_CTRL_CRACK, gamma + 0.5)
    return g


@pytest.mark.parametrize("precision,shape", [(B.RVE_FP64, (48, 36)), (B.RVE_MIXED, (64, 64)),
                                             (B.RVE_FP64, (12, 8, 6)), (B.RVE_MIXED, (16, 16, 16))])
def test_noalloc_apply_matches_apply_device(precision, shape):
    import torch
    g = _linearized(shape, precision)
    g.set_stream(torch.cuda.current_stream().cuda_stream)
    dt = torch.float32 if precision == B.RVE_MIXED else torch.float64
    c, n = g.m + 1, g.n
    rng = np.random.default_rng(7)
    x = torch.tensor(rng.standard_normal(c * n), dtype=dt, device="cuda")
    xE = torch.tensor([0.3], dtype=torch.float64, device="cuda")
    y_ref = torch.zeros_like(x)
    yE_ref = torch.zeros(1, dtype=torch.float64, device="cuda")
    g.apply_device(x.data_ptr(), xE.data_ptr(), y_ref.data_ptr(), yE_ref.data_ptr())
    torch.cuda.synchronize()
    L = B.lib()
    for _ in range(2):  # two calls in a row share (and reuse) the built-in scratch
        y = torch.full_like(x, float("nan"))
        yE = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        rc = L.rve_apply_device_noalloc(g.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(xE.data_ptr()),
                                        ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(yE.data_ptr()))
        assert rc == B.RVE_OK, L.rve_last_error(g.h)
        torch.cuda.synchronize()
        assert torch.isfinite(y).all()
        # the same kernels, launch shapes and reduction order on the same inputs, with only the
        # scratch in another place: the outputs are the same bits
        assert torch.equal(y, y_ref)
        assert torch.equal(yE, yE_ref)
    g.close()


def test_noalloc_apply_rejects_grids_beyond_its_scratch():
    """A 768 x 768 float64 grid needs ~18.9 MB of spectral scratch (> 16 MiB): RVE_E_ARG."""
    import torch
    inp = ms.homogeneous_panel(768, notch_len=64)
    g = B.RVE(inp, precision=B.RVE_FP64)
    g.set_state(np.zeros((3, g.n)), inp.notch.astype(float).reshape(-1), np.zeros(g.n), 1e-3, 0.0)
    g.linearize(B.RVE_CTRL_STRAIN, 1e-3)
    x = torch.zeros(4 * g.n, dtype=torch.float64, device="cuda")
    e = torch.zeros(1, dtype=torch.float64, device="cuda")
    L = B.lib()
    rc = L.rve_apply_device_noalloc(g.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(e.data_ptr()),
                                    ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(e.data_ptr()))
    assert rc == B.RVE_E_ARG
    assert b"built-in array" in L.rve_last_error(g.h)
    g.close()
