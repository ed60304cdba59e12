"""Write the stored oracle values used by the GPU parity tests.

Calls only the float64 CPU oracle (oracle/) on seeded synthetic inputs from
paper_2412_17445_gb300.microstructure; nothing here touches the CUDA library.

  python tests/golden/make_golden.py panel64
  python tests/golden/make_golden.py composite512 [n_increments]
  python tests/golden/make_golden.py composite512_cost [n_increments]
  python tests/golden/make_golden.py panel32_crossing

  panel64_crack.json       64 x 64 homogeneous panel (E = 1, nu = 0.3, Gc = 1e-3, l = 2),
                           notch x in [0, 16) at y = 32, tensile f = e_y e_y, spectral split,
                           start-up + 20 crack-length increments of da = 1 (float64).
  composite512_crack.json  the 512 x 512 fibre composite the headline benchmark times (RSA
                           discs r = 12 at 40 %, E_f/E_m = 10, nu 0.25/0.35, Gc_f/Gc_m = 5,
                           l = 2, central notch of 32 voxels, seed base + 1): start-up +
                           n crack-length increments of da = 1 (float64, Newton and Krylov
                           tolerance 1e-12).  Per increment: E, Sigma, Gamma, tau, the
                           oracle's own Newton / Krylov counts and wall time, the voxels
                           with phi > 0.5 (the crack path), the voxels within 1e-6 of 0.5
                           (ties), and phi on a window of rows around the notch.  The file
                           is rewritten after every increment, so a partial run is usable.
  panel32_crossing.json    32 x 32 homogeneous panel, notch of 4: start-up + increments of
                           da = 1 until the crack has crossed the cell and the stress has
                           dropped (float64, Newton 1e-10, Krylov 1e-12): the (E, Sigma)
                           curve whose area gives the effective toughness of Eq. JaviGc.
  composite512_oracle_cost.json
                           the oracle's own cost of the benchmark's increments on the same
                           composite at the float64 solver's benchmark tolerances (Newton
                           1e-8, Krylov 1e-10): wall time, Newton and Krylov iterations of
                           the start-up and of each increment, one thread.
"""
import json
import os
import platform
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from oracle import solver  # noqa: E402
from paper_2412_17445_gb300 import microstructure as ms  # noqa: E402

# phi window stored per increment of the composite: rows y0 .. y0+WIN_ROWS, columns
# x0 .. x0+WIN_COLS around the central notch
WIN_ROWS = 8
WIN_COLS = 96


def panel64(n_inc=20):
    inp = ms.homogeneous_panel(64, notch_len=16)
    pb = solver.problem_from_input(inp)
    opt = solver.Options(newton_tol=1e-12, krylov_tol=1e-12)
    t0 = time.time()
    st, res, Es = solver.startup(pb, opt)
    assert all(r.converged for r in res[:3])
    rows = [dict(inc=0, E=st.E, tau=st.tau, Sigma=solver.macro_stress(pb, st).tolist())]
    for k in range(1, n_inc + 1):
        r, rec = solver.crack_increment(pb, st, 1.0, opt)
        assert r.converged, k
        rows.append(dict(inc=k, E=rec["E"], tau=rec["tau"], Gamma=rec["Gamma"], Sigma=rec["Sigma"].tolist(),
                         newton=rec["newton"], krylov=rec["krylov"]))
        print(k, rec["E"], rec["Sigma"][1, 1], time.time() - t0, flush=True)
    return dict(workload="panel64_crack", Es=Es, newton_tol=1e-12, krylov_tol=1e-12, rows=rows)


def _cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def _crack_record(st):
    phi = st.phi
    ny, nx = phi.shape
    y0 = ny // 2 - WIN_ROWS // 2
    x0 = nx // 2 - WIN_COLS // 2
    flat = phi.reshape(-1)
    return dict(crack=np.flatnonzero(flat > 0.5).tolist(),
                ties=np.flatnonzero(np.abs(flat - 0.5) < 1e-6).tolist(),
                phi_window=dict(y0=int(y0), x0=int(x0), rows=WIN_ROWS, cols=WIN_COLS,
                                values=phi[y0:y0 + WIN_ROWS, x0:x0 + WIN_COLS].reshape(-1).tolist()))


def composite512(n_inc=5, path=None):
    inp = ms.fibre_composite(n=512, radius=12.0, fraction=0.4, notch_len=32, seed=ms.SEED_BASE + 1)
    pb = solver.problem_from_input(inp)
    tol = 1e-12
    opt = solver.Options(newton_tol=tol, krylov_tol=tol)
    path = path or os.path.join(HERE, "composite512_crack.json")
    out = dict(workload="composite512_crack",
               input="fibre_composite(n=512, radius=12, fraction=0.4, notch_len=32, seed=SEED_BASE+1)",
               newton_tol=tol, krylov_tol=tol, da=1.0,
               host=dict(cpu=_cpu_model(), threads=1, numpy=np.__version__), rows=[])
    t0 = time.time()
    st, res, Es = solver.startup(pb, opt)
    assert all(r.converged for r in res[:3])
    t_start = time.time() - t0
    lin = solver.Linearization(pb, st.eps_t, st.E, st.phi, st.Hn)
    out["startup"] = dict(Es=Es, steps=len(res), newton=[r.iterations for r in res],
                          krylov=[r.krylov_iterations for r in res], seconds=t_start)
    row0 = dict(inc=0, E=st.E, tau=st.tau, Gamma=lin.Gamma, Sigma=solver.macro_stress(pb, st).tolist(),
                seconds=t_start)
    row0.update(_crack_record(st))
    out["rows"].append(row0)
    _write(out, path)
    print("startup", st.E, st.tau, t_start, flush=True)
    for k in range(1, n_inc + 1):
        t1 = time.time()
        r, rec = solver.crack_increment(pb, st, 1.0, opt)
        assert r.converged, k
        row = dict(inc=k, E=rec["E"], tau=rec["tau"], Gamma=rec["Gamma"], Sigma=rec["Sigma"].tolist(),
                   newton=rec["newton"], krylov=rec["krylov"], cutbacks=rec["cutbacks"],
                   seconds=time.time() - t1)
        row.update(_crack_record(st))
        out["rows"].append(row)
        _write(out, path)
        print(k, rec["E"], rec["Sigma"][1, 1], rec["newton"], rec["krylov"], rec["cutbacks"],
              time.time() - t1, flush=True)
    return out


def panel32_crossing(path=None):
    """32 x 32 homogeneous panel (E = 1, nu = 0.3, Gc = 1e-3, l = 2), notch x in [0, 4) at
    y = 16: start-up and crack-length increments of da = 1 until the crack crosses the cell
    ({phi > 0.5} covers the notch row) and Sigma_yy has dropped below 1 % of its peak; float64,
    Newton 1e-10, Krylov 1e-12.  Stores the (E, Sigma) curve of Eq. JaviGc."""
    n, a0 = 32, 4
    inp = ms.homogeneous_panel(n, notch_len=a0)
    pb = solver.problem_from_input(inp)
    opt = solver.Options(newton_tol=1e-10, krylov_tol=1e-12)
    st, res, Es = solver.startup(pb, opt)
    assert all(r.converged for r in res[:3])
    rows = [dict(inc=0, E=st.E, tau=st.tau, Sigma=solver.macro_stress(pb, st).tolist())]
    peak = rows[0]["Sigma"][1][1]
    for k in range(1, 200):
        r, rec = solver.crack_increment(pb, st, 1.0, opt)
        assert r.converged, k
        rows.append(dict(inc=k, E=rec["E"], tau=rec["tau"], Gamma=rec["Gamma"], Sigma=rec["Sigma"].tolist(),
                         cutbacks=rec["cutbacks"]))
        peak = max(peak, rec["Sigma"][1, 1])
        if np.all(st.phi[n // 2] > 0.5) and rec["Sigma"][1, 1] < 0.01 * peak:
            break
    out = dict(workload="panel32_crossing", n=n, notch=a0, newton_tol=1e-10, krylov_tol=1e-12, rows=rows)
    with open(path or os.path.join(HERE, "panel32_crossing.json"), "w") as f:
        json.dump(out, f, indent=1)
    return out


def composite512_cost(n_inc=3, path=None):
    """The oracle's own cost of the benchmark's crack increments: the same composite at the
    float64 solver's benchmark tolerances (Newton 1e-8, Krylov 1e-10), start-up + n
    increments, with the wall time, Newton and Krylov iterations of each (single thread)."""
    inp = ms.fibre_composite(n=512, radius=12.0, fraction=0.4, notch_len=32, seed=ms.SEED_BASE + 1)
    pb = solver.problem_from_input(inp)
    opt = solver.Options(newton_tol=1e-8, krylov_tol=1e-10)
    path = path or os.path.join(HERE, "composite512_oracle_cost.json")
    out = dict(workload="composite512_oracle_cost",
               input="fibre_composite(n=512, radius=12, fraction=0.4, notch_len=32, seed=SEED_BASE+1)",
               newton_tol=1e-8, krylov_tol=1e-10, da=1.0,
               host=dict(cpu=_cpu_model(), threads=1, numpy=np.__version__), rows=[])
    t0 = time.time()
    st, res, Es = solver.startup(pb, opt)
    assert all(r.converged for r in res[:3])
    out["startup"] = dict(seconds=time.time() - t0, steps=len(res), newton=[r.iterations for r in res],
                          krylov=[r.krylov_iterations for r in res])
    _write(out, path)
    for k in range(1, n_inc + 1):
        t1 = time.time()
        r, rec = solver.crack_increment(pb, st, 1.0, opt)
        assert r.converged, k
        out["rows"].append(dict(inc=k, E=rec["E"], newton=rec["newton"], krylov=rec["krylov"],
                                cutbacks=rec["cutbacks"], seconds=time.time() - t1))
        _write(out, path)
        print(k, rec["newton"], rec["krylov"], time.time() - t1, flush=True)
    return out


def _write(out, path):
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(out, f, indent=None, separators=(",", ":"))
    os.replace(tmp, path)


if __name__ == "__main__":
    which = sys.argv[1] if len(sys.argv) > 1 else "panel64"
    if which == "panel64":
        out = panel64()
        with open(os.path.join(HERE, "panel64_crack.json"), "w") as f:
            json.dump(out, f, indent=1)
    elif which == "composite512":
        composite512(int(sys.argv[2]) if len(sys.argv) > 2 else 5)
    elif which == "panel32_crossing":
        panel32_crossing()
    elif which == "composite512_cost":
        composite512_cost(int(sys.argv[2]) if len(sys.argv) > 2 else 3)
    else:
        raise SystemExit(f"unknown golden set {which}")
