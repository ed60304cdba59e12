"""Compile-time resource checks of the float32 apply passes (no GPU: nvcc cross-compiles).

The 3D x-forward prologue reads 38 operands per voxel.  Holding both voxels of a row pair at
once spilled 260 bytes per thread at the 64-register cap of four resident blocks per SM, and the
spill traffic took a third of the pass's time at 128^3.  This test compiles the 128-point
and 512-point translation units with ptxas's resource report and requires every float32 3D apply
pass, the 2D passes the Krylov chunks run (two row pairs per block, prologue / epilogue modes
0-2) and the fused 512-point column pass to use no local memory.
"""
import os
import re
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2412_17445_gb300", "csrc")


def _ptxas_report(tu, tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    from paper_2412_17445_gb300 import build
    tmp_path.mkdir(parents=True, exist_ok=True)
    cmd = [nvcc] + build.ARCH + build.FLAGS + ["-Xptxas", "-v", "-c", os.path.join(CSRC, tu),
                                               "-o", str(tmp_path / "k.o")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    # one entry per kernel: "Compiling entry function '<mangled>'" followed by its frame and spill line
    out = {}
    name = None
    for line in r.stderr.splitlines():
        m = re.search(r"Compiling entry function '([^']+)'", line)
        if m:
            name = m.group(1)
            continue
        m = re.search(r"(\d+) bytes stack frame, (\d+) bytes spill stores, (\d+) bytes spill loads", line)
        if m and name is not None:
            out[name] = tuple(int(v) for v in m.groups())
            name = None
    return out


def test_float32_apply_passes_do_not_spill(tmp_path):
    import concurrent.futures as cf
    with cf.ThreadPoolExecutor(2) as ex:
        f128 = ex.submit(_ptxas_report, "kernels_fft_128.cu", tmp_path / "a")
        f512 = ex.submit(_ptxas_report, "kernels_fft_512.cu", tmp_path / "b")
        rep, rep512 = f128.result(), f512.result()
    # Itanium mangling of the template arguments: I f (float), Li6E (M = 6), Li128E (N = 128)
    three_d = [k for k in rep if re.match(r"_Z\d+(k_xfwd_apply|k_xinv_apply|k_col)IfLi6E", k)]
    assert len(three_d) == 5, sorted(rep)   # x-forward, x-inverse, three column passes
    hot_2d = [k for k in rep
              if re.match(r"_Z\d+(k_xfwd_apply|k_xinv_apply)IfLi3ELi128ELi2ELi[012]E", k)]
    assert len(hot_2d) == 6, sorted(rep)
    spilling = {k: rep[k] for k in three_d + hot_2d if rep[k] != (0, 0, 0)}
    assert not spilling, spilling
    # the benchmarked 512^2 grouped apply: its x passes and the fused column pass of one column
    hot_512 = [k for k in rep512
               if re.match(r"_Z\d+(k_xfwd_apply|k_xinv_apply)IfLi3ELi512ELi2ELi[012]E", k)
               or re.match(r"_Z\d+k_col_fused2dILi512ELi1EE", k)]
    assert len(hot_512) == 7, sorted(rep512)
    spilling = {k: rep512[k] for k in hot_512 if rep512[k] != (0, 0, 0)}
    assert not spilling, spilling
