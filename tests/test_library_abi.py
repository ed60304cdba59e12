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


def test_ctypes_structs_match_the_header(tmp_path):
    """sizeof and every field offset of rve_desc, rve_step and rve_result, compiled from
    include/rve.h with the host C compiler, equal the binding's ctypes structures."""
    import shutil
    import subprocess
    from paper_2412_17445_gb300 import binding
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    structs = [("rve_desc", binding.rve_desc), ("rve_step", binding.rve_step), ("rve_result", binding.rve_result)]
    lines = ["#include <stddef.h>", "#include <stdio.h>", "#include <stdint.h>", '#include "rve.h"', "int main(void) {"]
    for cname, cls in structs:
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        s, f, v = line.split()
        got[(s, f)] = int(v)
    for cname, cls in structs:
        assert got[(cname, "sizeof")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)


def test_invalid_constraint_is_rejected_before_device_work(libpath):
    from paper_2412_17445_gb300 import binding
    from paper_2412_17445_gb300 import microstructure as ms
    d, keep = binding.make_desc(ms.homogeneous_panel(16, notch_len=4))
    assert d.constraint == binding.RVE_CONSTRAINT_LENGTH
    d.constraint = 7
    h = ctypes.c_void_p()
    assert binding.lib().rve_create(ctypes.byref(d), ctypes.byref(h)) == binding.RVE_E_ARG
    assert h.value is None
