"""J-integral on the GPU (rve_j_integral): the rotation from the compatibility relations and
Rice's contour sum (oracle.postprocess.j_integral restates both on the host).

Parity: the library's J equals the oracle's on the same state, float64 round-off level, on
random states of compile-time and runtime line lengths, both energy splits, contours that
touch the grid border and contours inside it.  Physics on a crack-controlled run of the
64^2 panel (Sec. 4.2): contours around the tip outside the process zone agree, and J sits
near G_c times the amplification factor of the appendix."""
import numpy as np
import pytest

from oracle import postprocess, solver
from paper_2412_17445_gb300 import binding as B
from paper_2412_17445_gb300 import microstructure as ms

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2412_17445_gb300 import build
    build.build()
    B.lib()


def _boxes(ny, nx):
    return [(0, 0, nx - 1, ny - 1), (1, 2, nx // 2, ny - 2), (nx // 3, ny // 4, nx - 2, (3 * ny) // 4),
            (nx - 3, 0, nx - 1, 2)]


@pytest.mark.parametrize("shape", [(16, 16), (18, 12), (24, 36), (64, 128), (128, 48), (96, 256)])
@pytest.mark.parametrize("split", [B.RVE_SPLIT_SPECTRAL, B.RVE_SPLIT_NONE])
def test_j_integral_matches_oracle_on_random_states(shape, split):
    inp = ms.random_rve(shape, 31)
    eps, E, phi, H = ms.random_state(inp, 32)
    pb = solver.problem_from_input(inp, isotropic=split == B.RVE_SPLIT_NONE)
    st = solver.initial_state(pb)
    st.eps_t, st.phi, st.E = eps, phi, E
    g = B.RVE(inp, precision=B.RVE_FP64, split=split)
    g.set_state(B.mandel_from_tensor(eps), phi, H, E)
    ny, nx = shape
    for box in _boxes(ny, nx):
        Jo = postprocess.j_integral(pb, st, box)
        Jg = g.j_integral(box)
        npts = 2 * (box[2] - box[0] + 1) + 2 * (box[3] - box[1] + 1)
        scale = npts * float(np.max(pb.C_ref)) * (np.max(np.abs(eps)) + abs(E)) ** 2
        assert abs(Jg - Jo) < 1e-12 * scale, (box, Jg, Jo)
    g.close()


def test_j_integral_rejects_bad_contours_and_3d():
    g = B.RVE(ms.random_rve((16, 16), 33), precision=B.RVE_FP64)
    for box in [(0, 0, 16, 8), (-1, 0, 4, 4), (4, 4, 4, 8), (5, 6, 3, 8)]:
        with pytest.raises(B.RVEError):
            g.j_integral(box)
    g.close()
    g3 = B.RVE(ms.random_rve((8, 8, 6), 34), precision=B.RVE_FP64)
    with pytest.raises(B.RVEError):
        g3.j_integral((0, 0, 4, 4))
    g3.close()


@pytest.mark.parametrize("prec", [B.RVE_FP64, B.RVE_MIXED])
def test_j_integral_during_crack_growth_panel64(prec):
    """Ten crack-length increments (Delta a = 1) on the 64^2 panel: J on square contours of
    half-size 8, 11 and 14 around the tip agree within 5 %, 0.7 < J / (G_c A) < 1.05, and
    the library's J equals the oracle's contour sum on the library's own fields."""
    n = 64
    inp = ms.homogeneous_panel(n, notch_len=16)
    g = B.RVE(inp, precision=prec, newton_tol=1e-9 if prec == B.RVE_FP64 else 1e-8)
    g.startup()
    for _ in range(10):
        g.crack_increment(1.0)
    phi = g.field(B.RVE_FIELD_PHI).reshape(n, n)
    tip = int(np.max(np.nonzero(phi[n // 2, : 3 * n // 4] > 0.5)[0]))
    boxes = [(tip - d, n // 2 - d, tip + d, n // 2 + d) for d in (8, 11, 14)]
    Js = [g.j_integral(b) for b in boxes]
    assert max(Js) - min(Js) < 0.05 * max(Js), Js
    pb = solver.problem_from_input(inp)
    ref = float(np.min(pb.Gc)) * postprocess.amplification_factor(pb.ell)
    assert 0.7 < np.mean(Js) / ref < 1.05, (np.mean(Js) / ref, Js)
    st = solver.initial_state(pb)
    st.eps_t = B.tensor_from_mandel(g.field(B.RVE_FIELD_EPS_T), (n, n))
    st.phi = phi
    st.E = g.macro_stress()[1]
    for b, Jg in zip(boxes, Js):
        assert abs(Jg - postprocess.j_integral(pb, st, b)) < 1e-10 * abs(Jg)
    g.close()
