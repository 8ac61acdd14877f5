"""GPU parity of the two-dimensional Galerkin operators (bem_planar_operators) with the
oracle (oracle.planar), element by element: the same quadrature in FP64, so the
bound is the device Hankel functions' accuracy (about 2e-10 relative near the
series / asymptotic switch) times the sums' condition: 1e-9 of the largest entry."""
import numpy as np
import pytest

import workloads as W
from oracle import planar as PL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2310_15644_gb300.build import build

    build()
    import paper_2310_15644_gb300.bem as mod

    return mod


CASES = [("circle64", lambda: W.circle_polygon(64), 3.0 + 0j),
         ("ellipse96_lossy", lambda: W.ellipse_polygon(96, 1.5, 2 * np.pi), 4.0 - 0.7j),
         ("airfoil80", lambda: W.airfoil_polygon(80), 6.0 + 0j),
         ("ellipse90_ktilde", lambda: W.ellipse_polygon(90, 1.5, 2 * np.pi), PL.k_tilde(5.0, 1.0))]


@pytest.mark.parametrize("name,mesh,k", CASES, ids=[c[0] for c in CASES])
def test_planar_operators_equal_oracle(B, name, mesh, k):
    verts = mesh()
    n = len(verts)
    mats = [torch.empty(n, n, dtype=torch.complex128, device=DEV) for _ in range(3)]
    B.bem_planar_operators(None, verts, k, mats[0].data_ptr(), mats[1].data_ptr(), mats[2].data_ptr(),
                      torch.cuda.current_stream().cuda_stream)
    S, D, Dt, N, G = PL.operators(PL.Polygon(verts), k)
    for got, ref in zip(mats, (S, D, N)):
        g = got.cpu().numpy()
        assert np.abs(g - ref).max() <= 1e-9 * np.abs(ref).max(), name
