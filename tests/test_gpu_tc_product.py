"""Tensor-core product (BEM_C64_TC): the complex64 operator applied to passes of 64
vectors on the tcgen05 tensor cores, against the float64 oracle's dense product and
against the CUDA-core complex64 product of the same stored operator.

Bound: element-wise error against Z @ X (largest entry-wise error over the largest
reference entry) at most twice that of the CUDA-core complex64 product on the same
vectors -- both read the same FP32 entries, and the three-term TF32 split keeps the
contraction's own rounding near FP32's; the two products agree with each other to
5e-6 of max |y| (each product's FP32 rounding over up to a few thousand terms)."""
import numpy as np
import pytest

import workloads as W
from oracle import operators as O
from oracle import rwg as R

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
EPS = 3.2 - 1.9j


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2310_15644_gb300.build import build

    build()
    import paper_2310_15644_gb300.bem as mod

    return mod


def _stream():
    return torch.cuda.current_stream().cuda_stream


def make(B, v, t, k0, leaf, eta, aca_tol):
    opt = B.bem_default_options()
    opt.precision = B.BEM_PREC_C64
    opt.leaf_size = leaf
    opt.eta = eta
    opt.aca_tol = aca_tol
    h = B.bem_create(opt)
    B.bem_set_mesh(h, v, t)
    B.bem_set_media(h, k0, EPS)
    B.bem_assemble(h, _stream())
    return h


def matvec(B, h, X, dtype):
    xd = torch.from_numpy(np.ascontiguousarray(X.T)).to(DEV, torch.complex64)
    yd = torch.full_like(xd, complex("nan"))
    B.bem_matvec(h, xd.data_ptr(), yd.data_ptr(), X.shape[1], dtype, _stream())
    torch.cuda.synchronize()
    return yd.cpu().numpy().astype(np.complex128).T


def elem(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


CASES = [
    # name, mesh, k0, leaf, eta, aca tol, vectors
    ("ico3_leaf32_aca1e-6_n64", lambda: W.icosphere(3), 10.0, 32, 2.0, 1e-6, 64),
    ("ico3_leaf32_aca1e-4_n13", lambda: W.icosphere(3), 10.0, 32, 2.0, 1e-4, 13),
    ("ico2_dense_leaf16_n70", lambda: W.icosphere(2), 2.0, 16, 0.0, 1e-6, 70),
    ("box_leaf37_n130", lambda: W.box_mesh(1.0, 0.8, 0.3, 8, 6, 3), 6.0, 37, 2.0, 1e-5, 130),
]


@pytest.mark.parametrize("name,mesh,k0,leaf,eta,aca_tol,nrhs", CASES, ids=[c[0] for c in CASES])
def test_tc_product_matches_oracle_and_cuda_cores(B, name, mesh, k0, leaf, eta, aca_tol, nrhs):
    v, t = mesh()
    g = R.build(v, t)
    A, Bm, C = O.pmchwt_blocks(g, k0, EPS)
    Z = np.block([[A, Bm], [-Bm, C]])
    h = make(B, v, t, k0, leaf, eta, aca_tol)
    try:
        X = W.complex_normal(2 * g.ne, seed=31, nrhs=nrhs).astype(np.complex64).astype(np.complex128)
        ref = Z @ X
        y_cc = matvec(B, h, X, B.BEM_C64)
        y_tc = matvec(B, h, X, B.BEM_C64_TC)
        assert np.all(np.isfinite(y_tc))
        e_cc, e_tc = elem(y_cc, ref), elem(y_tc, ref)
        print(f"{name}: tensor {e_tc:.3e}, CUDA cores {e_cc:.3e}, between {elem(y_tc, y_cc):.3e}")
        assert e_tc <= 2.0 * e_cc, (e_tc, e_cc)
        assert elem(y_tc, y_cc) <= 5e-6, elem(y_tc, y_cc)
        # repeated calls are bit-identical (no atomics on the result)
        assert np.array_equal(y_tc, matvec(B, h, X, B.BEM_C64_TC))
    finally:
        B.bem_destroy(h)


def test_tc_product_full_size(B):
    """61440 unknowns in the benchmark's configuration, 64 vectors in one pass:
    sampled rows of two vectors against the oracle (bound as the single-vector
    full-size test, 5e-5 of rms) and every vector against the CUDA-core product."""
    v, t = W.icosphere(5)
    g = R.build(v, t)
    h = make(B, v, t, 10.0, 64, 2.0, 1e-4)
    try:
        X = W.complex_normal(2 * g.ne, seed=0, nrhs=64).astype(np.complex64).astype(np.complex128)
        y_tc = matvec(B, h, X, B.BEM_C64_TC)
        rows = np.random.default_rng(11).choice(2 * g.ne, 12, replace=False)
        for r in (0, 37):
            ref = O.pmchwt_rows_apply(g, 10.0, EPS, X[:, r].copy(), rows)
            err = np.abs(y_tc[rows, r] - ref).max() / np.sqrt(np.mean(np.abs(y_tc[:, r]) ** 2))
            assert err <= 5e-5, (r, err)
        y_cc = matvec(B, h, X[:, :8], B.BEM_C64)
        print(f"full size: tensor vs CUDA cores {elem(y_tc[:, :8], y_cc):.3e}")
        assert elem(y_tc[:, :8], y_cc) <= 5e-6
    finally:
        B.bem_destroy(h)
