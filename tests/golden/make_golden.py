"""Write the stored oracle values used by the GPU parity tests.

Calls only the float64 CPU oracle (oracle/) on seeded synthetic inputs from
paper_2412_17445_gb300.microstructure; nothing here touches the CUDA library.

  panel64_crack.json   64 x 64 homogeneous panel (E = 1, nu = 0.3, Gc = 1e-3, l = 2),
                       notch x in [0, 16) at y = 32, tensile f = e_y e_y, spectral split,
                       start-up + 20 crack-length increments of da = 1 (float64).
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import solver  # noqa: E402
from paper_2412_17445_gb300 import microstructure as ms  # noqa: E402


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


if __name__ == "__main__":
    out = panel64()
    with open(os.path.join(HERE, "panel64_crack.json"), "w") as f:
        json.dump(out, f, indent=1)
