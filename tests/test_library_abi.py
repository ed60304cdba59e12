"""The C ABI library builds, loads and exports every entry point include/rve.h declares
(no GPU needed: nothing here calls into CUDA)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "rve.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(rve_[a-z_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2412_17445_gb300 import build
    return build.build()


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    names = _declared()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_header(libpath):
    from paper_2412_17445_gb300 import binding
    bound = {name for name, _, _ in binding.SIGNATURES}
    assert set(_declared()) <= bound


def test_desc_defaults_and_error_paths(libpath):
    """Host-only calls: defaults and argument validation return codes, no device work."""
    from paper_2412_17445_gb300 import binding
    L = binding.lib()
    d = binding.rve_desc()
    L.rve_desc_defaults(ctypes.byref(d))
    assert d.nz == 1 and d.ell == 2.0 and d.newton_tol == 1e-10 and d.precision == binding.RVE_FP64
    h = ctypes.c_void_p()
    # no phase map / properties -> RVE_E_ARG before any CUDA call
    assert L.rve_create(ctypes.byref(d), ctypes.byref(h)) == binding.RVE_E_ARG
    assert h.value is None
    assert b"invalid" in L.rve_last_error(None)
    assert L.rve_crack_increment(None, 1.0, None) == binding.RVE_E_ARG
