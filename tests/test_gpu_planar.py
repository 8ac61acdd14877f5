"""GPU parity of the two-dimensional Galerkin operators (bem_planar_operators) with the
oracle (oracle.planar), element by element.  FP64 form: the oracle's quadrature on
the near pairs and a 5 x 5 rule with error below 1e-13 on the well-separated ones,
so the bound is the device Hankel functions' accuracy (about 2e-10 relative near
the series / asymptotic switch) times the sums' condition: 1e-9 of the largest
entry.  FP32 form (well-separated pairs with |k R| >= 8 in FP32): 3e-6 of the
largest entry, on ellipses at N = 18 k0 where most pairs take that path."""
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


@pytest.mark.parametrize("n,k", [(288, 16.0 + 0j), (576, 32.0 - 0.4j), (576, PL.k_tilde(32.0, 1.0))],
                         ids=["ellipse288", "ellipse576_lossy", "ellipse576_ktilde"])
def test_planar_fp32_form_equals_oracle(B, n, k):
    verts = W.ellipse_polygon(n, 1.5, 2 * np.pi)
    mats = [torch.empty(n, n, dtype=torch.complex128, device=DEV) for _ in range(3)]
    B.bem_planar_operators(None, verts, k, mats[0].data_ptr(), mats[1].data_ptr(), mats[2].data_ptr(),
                           torch.cuda.current_stream().cuda_stream, fp32=True)
    S, D, Dt, N, G = PL.operators(PL.Polygon(verts), k)
    for got, ref in zip(mats, (S, D, N)):
        g = got.cpu().numpy()
        assert np.abs(g - ref).max() <= 3e-6 * np.abs(ref).max()
