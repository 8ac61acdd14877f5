"""GPU tests of the inner Krylov solvers (bem_options.solver): GMRES, CGS,
BiCGStab and CGNR (CG on the normal equations, through the adjoint product), on
the dense complex128 operator of a small sphere against the oracle's LU solution,
and inside FP64 refinement on the compressed complex64 operator, for Z x = b and
Z^H lambda = g.

Tolerances: complex128 dense solves (inner 1e-6, refined to a relative residual
of 1e-10 -- CGS alone stagnates well above 1e-10 in rounding, as squared-residual
methods do) must match LU to 1e-8 (J and M separately); refined complex64 solves
to 1e-9 must match LU to 1e-4 (ACA tolerance 1e-6 and FP32 entries, as the
forward product tests).
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
SOLVERS = [0, 1, 2, 3]
IDS = ["gmres", "cgs", "bicgstab", "cgnr"]


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
    B.bem_set_media(h, k0, 3.2 - 1.9j)
    B.bem_assemble(h, _stream())
    return h


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def sphere2():
    v, t = W.icosphere(2)
    g = R.build(v, t)
    Z = O.pmchwt_matrix(g, 2.0, 3.2 - 1.9j)
    b = E.rhs_planewave(g, 2.0, [0.0, 0.0, 1.0], [1.0, 0.0, 0.0])
    return v, t, g, Z, b


def _solve(B, h, rhs, adjoint):
    bd = torch.from_numpy(rhs).to(DEV)
    xd = torch.zeros_like(bd)
    f = B.bem_solve_adjoint if adjoint else B.bem_solve
    it, relres, status = f(h, bd.data_ptr(), xd.data_ptr(), 1, _stream())
    return xd.cpu().numpy(), it, relres[0]


@pytest.mark.parametrize("solver", SOLVERS, ids=IDS)
@pytest.mark.parametrize("adjoint", [False, True], ids=["Z", "ZH"])
def test_dense_complex128(B, sphere2, solver, adjoint):
    v, t, g, Z, b = sphere2
    M = Z.conj().T if adjoint else Z
    ref = np.linalg.solve(M, b)
    h = make(B, v, t, 2.0, 2, 0.0, 1e-6, solver=solver, tol=1e-6, refine_tol=1e-10, maxit=4000,
             gmres_restart=100)
    try:
        x, it, rr = _solve(B, h, b, adjoint)
        assert rr <= 1e-10
        ne = g.ne
        assert rel(x[:ne], ref[:ne]) <= 1e-8
        assert rel(x[ne:], ref[ne:]) <= 1e-8
    finally:
        B.bem_destroy(h)


@pytest.mark.parametrize("solver", SOLVERS, ids=IDS)
def test_compressed_complex64_refined(B, solver):
    v, t = W.icosphere(3)
    g = R.build(v, t)
    Z = O.pmchwt_matrix(g, 6.0, 3.2 - 1.9j)
    b = E.rhs_planewave(g, 6.0, [0.0, 0.0, 1.0], [1.0, 0.0, 0.0])
    ref = np.linalg.solve(Z, b)
    h = make(B, v, t, 6.0, 1, 2.0, 1e-6, solver=solver, tol=1e-4, refine_tol=1e-9, maxit=8000, gmres_restart=80)
    try:
        x, it, rr = _solve(B, h, b, False)
        assert rr <= 1e-9
        ne = g.ne
        assert rel(x[:ne], ref[:ne]) <= 1e-4
        assert rel(x[ne:], ref[ne:]) <= 1e-4
    finally:
        B.bem_destroy(h)
