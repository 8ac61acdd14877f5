"""GPU tests of the BF16-factor product (precision bit BEM_PREC_BF16F, product
dtype BEM_C64_BF16F) and of the solve that uses it inside FP64 iterative
refinement against the complex64 operator.

Tolerances.  BF16 keeps 8 significand bits: rounding to nearest changes each
real component of a factor entry by at most 2^-9 ~ 2e-3 of itself.  The far part
U (V^H x) therefore moves by at most ~2 x 2^-9 of sum |U||V^H||x|, and only the
far part is affected (near entries stay complex64), so the whole product moves by
a few 1e-3 at most: 4e-3 against the complex64 product and 5e-3 against the
dense oracle (which adds the ACA tolerance 1e-4).  With refinement the solution
is that of the complex64 operator: 1e-3 against the dense LU solution (ACA
tolerance 1e-4 on the same discretisation, as in the complex64 solve tests) and
2e-5 against the complex64-only solve (both refined to residuals of 1e-8 or
below with the same FP64-sum residual).
"""
import numpy as np
import pytest

import workloads as W
from oracle import excitation as E
from oracle import operators as O
from oracle import rwg as R

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

K0, EPS = 10.0, 3.2 - 1.9j
DEV = "cuda:0"


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


@pytest.fixture(scope="module")
def sphere3():
    v, t = W.icosphere(3)
    g = R.build(v, t)
    A, Bm, C = O.pmchwt_blocks(g, K0, EPS)
    return v, t, g, np.block([[A, Bm], [-Bm, C]])


def make(B, v, t, prec, **kw):
    opt = B.bem_default_options()
    opt.precision = prec
    opt.leaf_size = 32
    opt.eta = 2.0
    opt.aca_tol = 1e-4
    for k, val in kw.items():
        setattr(opt, k, val)
    h = B.bem_create(opt)
    B.bem_set_mesh(h, v, t)
    B.bem_set_media(h, K0, EPS)
    B.bem_assemble(h, _stream())
    return h


def matvec(B, h, X, dtype):
    xd = torch.from_numpy(np.ascontiguousarray(X.T)).to(DEV, torch.complex64)
    yd = torch.empty_like(xd)
    B.bem_matvec(h, xd.data_ptr(), yd.data_ptr(), X.shape[1], dtype, _stream())
    torch.cuda.synchronize()
    return yd.cpu().numpy().astype(np.complex128).T


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_bf16_product(B, sphere3):
    v, t, g, Z = sphere3
    h = make(B, v, t, B.BEM_PREC_C64 | B.BEM_PREC_BF16F)
    try:
        st = B.bem_stats_get(h)
        assert sum(st["factor_entries"]) > 0
        assert 0 < st["matvec_bytes_bf16f"] < st["matvec_bytes_c64"]
        X = W.complex_normal(2 * g.ne, seed=21, nrhs=13).astype(np.complex64).astype(np.complex128)
        y64 = matvec(B, h, X, B.BEM_C64)
        ybf = matvec(B, h, X, B.BEM_C64_BF16F)
        d = rel(ybf, y64)
        assert 0 < d <= 4e-3, d
        assert rel(ybf, Z @ X) <= 5e-3
        # entry-wise as well: no row block may carry the whole error
        assert np.abs(ybf - Z @ X).max() <= 5e-3 * np.abs(Z @ X).max()
        # batched (8 + 4 + 1) equals one at a time; repeated calls are identical
        single = np.stack([matvec(B, h, X[:, r:r + 1], B.BEM_C64_BF16F)[:, 0] for r in range(13)], axis=1)
        assert np.abs(ybf - single).max() <= 1e-6 * np.abs(single).max()
        assert np.array_equal(ybf, matvec(B, h, X, B.BEM_C64_BF16F))
    finally:
        B.bem_destroy(h)


def test_bf16_dtype_needs_its_operator(B, sphere3):
    v, t, g, Z = sphere3
    h = make(B, v, t, B.BEM_PREC_C64)
    try:
        x = torch.zeros(2 * g.ne, dtype=torch.complex64, device=DEV)
        y = torch.empty_like(x)
        with pytest.raises(B.BemError):
            B.bem_matvec(h, x.data_ptr(), y.data_ptr(), 1, B.BEM_C64_BF16F, _stream())
    finally:
        B.bem_destroy(h)


def test_bf16_inner_solve_refined(B, sphere3):
    v, t, g, Z = sphere3
    b = E.rhs_planewave(g, K0, [0.0, 0.0, 1.0], [1.0, 0.0, 0.0])
    xr = np.linalg.solve(Z, b)
    ne = g.ne
    bd = torch.from_numpy(b).to(DEV)
    h = make(B, v, t, B.BEM_PREC_C64 | B.BEM_PREC_BF16F, tol=1e-3, refine_tol=1e-8, maxit=3000)
    try:
        xd = torch.zeros_like(bd)
        it, relres, status = B.bem_solve(h, bd.data_ptr(), xd.data_ptr(), 1, _stream())
        assert relres[0] <= 1e-8
        x = xd.cpu().numpy()
    finally:
        B.bem_destroy(h)
    h = make(B, v, t, B.BEM_PREC_C64, tol=1e-4, refine_tol=1e-10, maxit=3000)
    try:
        xd = torch.zeros_like(bd)
        B.bem_solve(h, bd.data_ptr(), xd.data_ptr(), 1, _stream())
        x64 = xd.cpu().numpy()
    finally:
        B.bem_destroy(h)
    for sl in (slice(0, ne), slice(ne, 2 * ne)):
        assert rel(x[sl], xr[sl]) <= 1e-3
        assert rel(x[sl], x64[sl]) <= 2e-5


def test_c64_refinement_with_fp64_residual(B, sphere3):
    """Refinement on the complex64 operator alone: the residual is recomputed with
    FP64 vectors and sums through the complex64 entries, so it converges far below
    the FP32 rounding level of the inner solve, to the complex64 operator's own
    solution."""
    v, t, g, Z = sphere3
    b = E.rhs_planewave(g, K0, [0.0, 0.0, 1.0], [1.0, 0.0, 0.0])
    xr = np.linalg.solve(Z, b)
    ne = g.ne
    bd = torch.from_numpy(b).to(DEV)
    h = make(B, v, t, B.BEM_PREC_C64, tol=1e-4, refine_tol=1e-10, maxit=3000)
    try:
        xd = torch.zeros_like(bd)
        it, relres, status = B.bem_solve(h, bd.data_ptr(), xd.data_ptr(), 1, _stream())
        assert relres[0] <= 1e-10
        x = xd.cpu().numpy()
    finally:
        B.bem_destroy(h)
    for sl in (slice(0, ne), slice(ne, 2 * ne)):
        assert rel(x[sl], xr[sl]) <= 1e-3
