"""GPU tests of the batched GMRES of bem_solve: the right-hand sides of one call
advance together (one product per iteration over every active basis vector, on
the tensor cores for 16 or more complex64 right-hand sides), with Gram-Schmidt,
Givens rotations, residual estimates and restarts on the device.

Right-hand sides: seeded plane waves with Fibonacci-sphere directions and random
polarisations.  References: the oracle's LU solution of the dense FP64 PMCHWT
system (Eq. 7 with the Galerkin entries of Eq. 8).

Tolerances: refined solves (FP64 refinement to a relative residual of 1e-9 through
the complex64 operator with ACA tolerance 1e-6) match LU to 1e-4 per column, the
bound of the single-solve tests; a batch and the same columns solved one at a time
(refined through the same operator) agree to 1e-6, about cond(Z) times the
refinement target; complex128 dense solves refined to 1e-10 match LU to 1e-8.
"""
import numpy as np
import pytest

import workloads as W
from oracle import excitation as E
from oracle import operators as O
from oracle import rwg as R

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
K0 = 6.0
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


def make(B, v, t, k0, prec, eta, aca_tol, **kw):
    opt = B.bem_default_options()
    opt.precision = prec
    opt.leaf_size = 16
    opt.eta = eta
    opt.aca_tol = aca_tol
    for k, val in kw.items():
        setattr(opt, k, val)
    h = B.bem_create(opt)
    B.bem_set_mesh(h, v, t)
    B.bem_set_media(h, k0, EPS)
    B.bem_assemble(h, _stream())
    return h


def colrel(X, REF):
    """Relative error of each column."""
    return np.linalg.norm(X - REF, axis=0) / np.linalg.norm(REF, axis=0)


@pytest.fixture(scope="module")
def sphere3():
    v, t = W.icosphere(3)
    g = R.build(v, t)
    Z = O.pmchwt_matrix(g, K0, EPS)
    khat, e0 = W.plane_wave_batch(20, seed=4)
    b = E.rhs_planewave(g, K0, khat, e0)  # (2ne, 20)
    ref = np.linalg.solve(Z, b)
    return v, t, g, Z, b, ref


def solve(B, h, b, adjoint=False, raise_on_noconv=True):
    """b: (n, nrhs) complex128 -> (x (n, nrhs), iterations, relres, status)."""
    bd = torch.from_numpy(np.ascontiguousarray(b.T)).to(DEV)
    xd = torch.zeros_like(bd)
    f = B.bem_solve_adjoint if adjoint else B.bem_solve
    it, rr, st = f(h, bd.data_ptr(), xd.data_ptr(), b.shape[1], _stream(), raise_on_noconv=raise_on_noconv)
    return xd.cpu().numpy().T, it, rr, st


def test_batch_of_20_refined_matches_lu(B, sphere3):
    v, t, g, Z, b, ref = sphere3
    h = make(B, v, t, K0, 1, 2.0, 1e-6, tol=1e-4, refine_tol=1e-9, maxit=4000, gmres_restart=60)
    try:
        x, it, rr, _ = solve(B, h, b)
        assert np.all(rr <= 1e-9), rr
        ne = g.ne
        assert np.max(colrel(x[:ne], ref[:ne])) <= 1e-4
        assert np.max(colrel(x[ne:], ref[ne:])) <= 1e-4
        # the tensor-core product ran (20 right-hand sides of a complex64 solve)
        st = B.bem_stats_get(h)
        assert st["tc_passes"] > 0
    finally:
        B.bem_destroy(h)


def test_batch_equals_one_at_a_time(B, sphere3):
    v, t, g, Z, b, ref = sphere3
    h = make(B, v, t, K0, 1, 2.0, 1e-6, tol=1e-4, refine_tol=1e-9, maxit=4000, gmres_restart=60)
    try:
        xb, _, rrb, _ = solve(B, h, b)
        for r in (0, 7, 19):
            x1, _, rr1, _ = solve(B, h, b[:, r:r + 1])
            assert rr1[0] <= 1e-9
            assert colrel(xb[:, r:r + 1], x1)[0] <= 1e-6
    finally:
        B.bem_destroy(h)


def test_short_restarts_zero_column_and_unrefined(B, sphere3):
    """Restart length 8 (many device-side restarts), a zero right-hand side in the
    batch, no refinement: every relative residual reaches the inner tolerance, the
    zero column stays zero."""
    v, t, g, Z, b, ref = sphere3
    bz = b.copy()
    bz[:, 5] = 0
    h = make(B, v, t, K0, 1, 2.0, 1e-6, tol=1e-5, maxit=4000, gmres_restart=8)
    try:
        x, it, rr, _ = solve(B, h, bz)
        assert rr[5] == 0 and np.all(x[:, 5] == 0)
        # inner residual 1e-5 on the complex64 operator; measured through the same operator in FP64
        keep = [r for r in range(20) if r != 5]
        assert np.all(rr[keep] <= 1.5e-5), rr
        # the solution is that of the complex64 operator: against LU about cond * 1e-5 + ACA error
        assert np.max(colrel(x[:, keep], ref[:, keep])) <= 1e-2
    finally:
        B.bem_destroy(h)


def test_iteration_cap_reports_each_column(B, sphere3):
    v, t, g, Z, b, ref = sphere3
    h = make(B, v, t, K0, 1, 2.0, 1e-6, tol=1e-8, maxit=5, gmres_restart=50)
    try:
        x, it, rr, st = solve(B, h, b, raise_on_noconv=False)
        assert st == B.BEM_ENOCONV
        assert it == 5 * 20  # every column stopped at the cap
        assert np.all(rr > 1e-8) and np.all(rr < 1.0)
    finally:
        B.bem_destroy(h)


def test_adjoint_batch_refined(B, sphere3):
    v, t, g, Z, b, ref = sphere3
    g3 = b[:, :3]
    refH = np.linalg.solve(Z.conj().T, g3)
    h = make(B, v, t, K0, 1, 2.0, 1e-6, tol=1e-4, refine_tol=1e-9, maxit=4000, gmres_restart=60)
    try:
        lam, it, rr, _ = solve(B, h, g3, adjoint=True)
        assert np.all(rr <= 1e-9)
        assert np.max(colrel(lam, refH)) <= 1e-4
    finally:
        B.bem_destroy(h)


def test_dense_complex128_batch(B):
    """FP64 vectors and FP64 Gram-Schmidt (the complex128 instantiation)."""
    v, t = W.icosphere(2)
    g = R.build(v, t)
    Z = O.pmchwt_matrix(g, 2.0, EPS)
    khat, e0 = W.plane_wave_batch(3, seed=9)
    b = E.rhs_planewave(g, 2.0, khat, e0)
    ref = np.linalg.solve(Z, b)
    h = make(B, v, t, 2.0, 2, 0.0, 1e-6, tol=1e-6, refine_tol=1e-10, maxit=4000, gmres_restart=100)
    try:
        x, it, rr, _ = solve(B, h, b)
        assert np.all(rr <= 1e-10)
        assert np.max(colrel(x, ref)) <= 1e-8
    finally:
        B.bem_destroy(h)
