"""GPU parity tests: every kernel of the path, called through the C interface,
against the float64 CPU oracle on the same seeded inputs.

Tolerances (relative, 2-norm unless stated):
  * partition (cluster order, near and far block lists): exact equality;
  * complex64 operator entries: |err| <= 2e-5 x max|entry| of that operator --
    FP32 rounding (2^-24 ~ 6e-8) accumulated over the 4 x 49 point pairs of an
    entry and through exp/sincos of arguments up to |k1| R ~ 40;
  * complex128 entries: 1e-11 x max|entry| (same formulas, summation order only);
  * dense products: 2e-5 (c64), 1e-11 (c128);
  * compressed products: ACA tolerance plus the above;
  * solves: <= 1e-4 with the complex64 operator and GMRES tolerance 1e-6;
    <= 1e-8 with FP64 iterative refinement on the complex128 operator (dense).
"""
import numpy as np
import pytest

import workloads as W
from oracle import excitation as E
from oracle import operators as O
from oracle import power as P
from oracle import rwg as R
from oracle import tree as TR

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

K0, EPS = 2.0, 3.2 - 1.9j


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2310_15644_gb300.build import build

    build()
    import paper_2310_15644_gb300.bem as mod

    return mod


DEV = "cuda:0"


def _stream():
    return torch.cuda.current_stream().cuda_stream


def make(B, v, t, k0=K0, eps=EPS, prec=3, leaf=32, eta=2.0, aca_tol=1e-6, **kw):
    opt = B.bem_default_options()
    opt.precision = prec
    opt.leaf_size = leaf
    opt.eta = eta
    opt.aca_tol = aca_tol
    for k, val in kw.items():
        setattr(opt, k, val)
    h = B.bem_create(opt)
    B.bem_set_mesh(h, v, t)
    B.bem_set_media(h, k0, eps)
    B.bem_assemble(h, _stream())
    return h


def matvec(B, h, x, dtype):
    ct = torch.complex128 if dtype == B.BEM_C128 else torch.complex64   # every other form takes complex64
    xd = torch.from_numpy(np.ascontiguousarray(x)).to(DEV, ct)
    nrhs = 1 if x.ndim == 1 else x.shape[1]
    if x.ndim == 2:
        xd = xd.t().contiguous()       # column-major: one right-hand side after another
    yd = torch.empty_like(xd)
    B.bem_matvec(h, xd.data_ptr(), yd.data_ptr(), nrhs, dtype, _stream())
    torch.cuda.synchronize()
    y = yd.cpu().numpy().astype(np.complex128)
    return y if x.ndim == 1 else y.T


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def elem(a, b):
    """Largest entry-wise error against the largest reference entry: one wrong row
    block cannot hide under a global norm."""
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.fixture(scope="module")
def sphere2():
    v, t = W.icosphere(2)
    g = R.build(v, t)
    A, Bm, C = O.pmchwt_blocks(g, K0, EPS)
    return v, t, g, (A, Bm, C)


CASES = [
    ("ico2_leaf16", lambda: W.icosphere(2), 16, 2.0),
    ("ico3_leaf64", lambda: W.icosphere(3), 64, 2.0),
    ("ico3_leaf37", lambda: W.icosphere(3), 37, 2.0),
    ("box_leaf8_eta1.5", lambda: W.box_mesh(1.0, 0.8, 0.3, 6, 5, 2), 8, 1.5),
    ("geodesic7_leaf20", lambda: W.geodesic_sphere(7, 1.3), 20, 3.0),
]


@pytest.mark.parametrize("name,mesh,leaf,eta", CASES, ids=[c[0] for c in CASES])
def test_partition_equals_oracle(B, name, mesh, leaf, eta):
    v, t = mesh()
    h = make(B, v, t, prec=1, leaf=leaf, eta=eta, aca_tol=1e-3)
    try:
        perm, near, far = B.bem_partition(h)
        g = R.build(v, t)
        root, perm_o = TR.cluster_tree(g.midpoints(), leaf)
        near_o, far_o = TR.block_partition(root, eta)
        assert np.array_equal(perm, perm_o)
        assert np.array_equal(near.astype(np.int64), near_o)
        assert np.array_equal(far.astype(np.int64), far_o)
    finally:
        B.bem_destroy(h)


def _entry_sample(g, rng, count):
    rows = rng.integers(0, g.ne, count)
    cols = rng.integers(0, g.ne, count)
    # every self entry and every entry between edges sharing a triangle (singular pairs)
    diag = np.arange(g.ne)
    nb_r = np.repeat(g.tri_edge, 3, axis=1).ravel()
    nb_c = np.tile(g.tri_edge, (1, 3)).ravel()
    return np.concatenate([rows, diag, nb_r]).astype(np.int32), np.concatenate([cols, diag, nb_c]).astype(np.int32)


@pytest.mark.parametrize("dtype,tol", [(0, 2e-5), (1, 1e-11)], ids=["c64", "c128"])
def test_entries_equal_oracle(B, sphere2, dtype, tol):
    v, t, g, ops = sphere2
    h = make(B, v, t, prec=3, eta=0.0)
    try:
        rows, cols = _entry_sample(g, np.random.default_rng(7), 3000)
        rd = torch.from_numpy(rows).to(DEV)
        cd = torch.from_numpy(cols).to(DEV)
        ct = torch.complex64 if dtype == 0 else torch.complex128
        out = torch.empty(3 * len(rows), dtype=ct, device=DEV)
        B.bem_eval_entries(h, rd.data_ptr(), cd.data_ptr(), len(rows), out.data_ptr(), dtype, _stream())
        torch.cuda.synchronize()
        got = out.cpu().numpy().reshape(-1, 3).astype(np.complex128)
        for q in range(3):
            ref = ops[q][rows, cols]
            err = np.abs(got[:, q] - ref).max() / np.abs(ops[q]).max()
            assert err <= tol, (q, err)
    finally:
        B.bem_destroy(h)


@pytest.mark.parametrize("dtype,tol", [(0, 2e-5), (1, 1e-11)], ids=["c64", "c128"])
def test_dense_product_equals_oracle(B, sphere2, dtype, tol):
    v, t, g, (A, Bm, C) = sphere2
    Z = np.block([[A, Bm], [-Bm, C]])
    h = make(B, v, t, prec=3, eta=0.0, leaf=32)
    try:
        st = B.bem_stats_get(h)
        assert st["n_far"] == 0 and st["near_entries"] == g.ne * g.ne
        x = W.complex_normal(2 * g.ne, seed=1)
        if dtype == 0:
            x = x.astype(np.complex64).astype(np.complex128)
        y = matvec(B, h, x, dtype)
        assert rel(y, Z @ x) <= tol
        assert elem(y, Z @ x) <= tol
        # several right-hand sides in one call
        X = W.complex_normal(2 * g.ne, seed=2, nrhs=3)
        if dtype == 0:
            X = X.astype(np.complex64).astype(np.complex128)
        Y = matvec(B, h, X, dtype)
        assert rel(Y, Z @ X) <= tol
        assert elem(Y, Z @ X) <= tol
    finally:
        B.bem_destroy(h)


@pytest.fixture(scope="module")
def sphere3():
    v, t = W.icosphere(3)
    g = R.build(v, t)
    A, Bm, C = O.pmchwt_blocks(g, 10.0, EPS)
    return v, t, g, np.block([[A, Bm], [-Bm, C]])


@pytest.mark.parametrize("dtype,aca_tol,tol", [(0, 1e-6, 2e-5), (1, 1e-10, 1e-8), (0, 1e-4, 1e-3)],
                         ids=["c64_tol1e-6", "c128_tol1e-10", "c64_tol1e-4"])
def test_compressed_product_equals_oracle(B, sphere3, dtype, aca_tol, tol):
    v, t, g, Z = sphere3
    h = make(B, v, t, k0=10.0, prec=1 if dtype == 0 else 2, leaf=32, eta=2.0, aca_tol=aca_tol)
    try:
        st = B.bem_stats_get(h)
        assert st["n_far"] > 0
        if aca_tol >= 1e-4:
            # blocks below the break-even rank are kept as factors
            assert sum(st["factor_entries"]) > 0 and st["near_entries"] < g.ne * g.ne
        else:
            # tight tolerances push blocks past the break-even rank: they are stored densely
            assert st["n_far_dense"] > 0
        x = W.complex_normal(2 * g.ne, seed=4)
        if dtype == 0:
            x = x.astype(np.complex64).astype(np.complex128)
        y = matvec(B, h, x, dtype)
        assert rel(y, Z @ x) <= tol
        assert elem(y, Z @ x) <= tol
        y2 = matvec(B, h, x, dtype)
        assert np.array_equal(y, y2), "product is not deterministic"
    finally:
        B.bem_destroy(h)


@pytest.mark.parametrize("mesh,leaf", [(lambda: W.icosphere(0), 64), (lambda: W.icosphere(1), 2),
                                       (lambda: W.box_mesh(1.0, 0.6, 0.4, 4, 3, 2), 5)],
                         ids=["single_leaf", "leaf2", "box_coplanar"])
def test_edge_cases_dense_oracle(B, mesh, leaf):
    v, t = mesh()
    g = R.build(v, t)
    A, Bm, C = O.pmchwt_blocks(g, K0, EPS)
    Z = np.block([[A, Bm], [-Bm, C]])
    h = make(B, v, t, prec=2, leaf=leaf, eta=2.0, aca_tol=1e-12)
    try:
        x = W.complex_normal(2 * g.ne, seed=5)
        y = matvec(B, h, x, B.BEM_C128)
        assert rel(y, Z @ x) <= 1e-9
        assert elem(y, Z @ x) <= 1e-9
    finally:
        B.bem_destroy(h)


def test_rhs_equals_oracle(B, sphere2):
    v, t, g, _ = sphere2
    h = make(B, v, t, prec=1, eta=0.0)
    try:
        kh, e0 = W.plane_wave_batch(4, seed=0)
        ref = E.rhs_planewave(g, K0, kh, e0)
        for dtype, tol in ((B.BEM_C128, 1e-13), (B.BEM_C64, 1e-6)):
            ct = torch.complex64 if dtype == B.BEM_C64 else torch.complex128
            bd = torch.empty(4 * 2 * g.ne, dtype=ct, device=DEV)
            B.bem_rhs_planewave(h, kh, e0, bd.data_ptr(), dtype, _stream())
            torch.cuda.synchronize()
            got = bd.cpu().numpy().reshape(4, 2 * g.ne).T.astype(np.complex128)
            assert rel(got, ref) <= tol
    finally:
        B.bem_destroy(h)


def test_solve_refined_matches_dense_lu(B, sphere2):
    v, t, g, (A, Bm, C) = sphere2
    Z = np.block([[A, Bm], [-Bm, C]])
    b = E.rhs_planewave(g, K0, [0.0, 0.0, 1.0], [1.0, 0.0, 0.0])
    xr = np.linalg.solve(Z, b)
    h = make(B, v, t, prec=3, eta=0.0, refine_tol=1e-11)
    try:
        bd = torch.from_numpy(b).to(DEV)
        xd = torch.zeros_like(bd)
        it, relres, st = B.bem_solve(h, bd.data_ptr(), xd.data_ptr(), 1, _stream())
        x = xd.cpu().numpy()
        ne = g.ne
        assert relres[0] <= 1e-11
        assert rel(x[:ne], xr[:ne]) <= 1e-8
        assert rel(x[ne:], xr[ne:]) <= 1e-8
    finally:
        B.bem_destroy(h)


def test_solve_mixed_precision_meets_1e4(B, sphere3):
    v, t, g, Z = sphere3
    b = E.rhs_planewave(g, 10.0, [0.0, 0.0, 1.0], [1.0, 0.0, 0.0])
    xr = np.linalg.solve(Z, b)
    h = make(B, v, t, k0=10.0, prec=1, leaf=32, eta=2.0, aca_tol=1e-5, tol=1e-6)
    try:
        bd = torch.from_numpy(b).to(DEV)
        xd = torch.zeros_like(bd)
        it, relres, st = B.bem_solve(h, bd.data_ptr(), xd.data_ptr(), 1, _stream())
        x = xd.cpu().numpy()
        ne = g.ne
        assert rel(x[:ne], xr[:ne]) <= 1e-4
        assert rel(x[ne:], xr[ne:]) <= 1e-4
        pa, pe, ps = B.bem_power(h, xd.data_ptr(), bd.data_ptr(), 1, _stream())
        assert abs(pa[0] - P.absorbed(g, xr)) <= 1e-4 * abs(P.absorbed(g, xr))
    finally:
        B.bem_destroy(h)


def test_powers_equal_oracle(B, sphere2):
    v, t, g, (A, Bm, C) = sphere2
    Z = np.block([[A, Bm], [-Bm, C]])
    kh, e0 = W.plane_wave_batch(2, seed=3)
    b = E.rhs_planewave(g, K0, kh, e0)
    x = np.linalg.solve(Z, b)
    h = make(B, v, t, prec=1, eta=0.0)
    try:
        xd = torch.from_numpy(np.ascontiguousarray(x.T)).to(DEV)
        bd = torch.from_numpy(np.ascontiguousarray(b.T)).to(DEV)
        pa, pe, ps = B.bem_power(h, xd.data_ptr(), bd.data_ptr(), 2, _stream())
        for r in range(2):
            assert abs(pa[r] - P.absorbed(g, x[:, r])) <= 1e-12 * abs(pa[r])
            assert abs(pe[r] - P.extinguished(g, x[:, r], b[:, r])) <= 1e-12 * abs(pe[r])
            assert abs(ps[r] - P.scattered(g, K0, x[:, r])) <= 1e-10 * abs(ps[r])
        dens = torch.empty(g.nt, dtype=torch.float64, device=DEV)
        B.bem_power_density(h, xd.data_ptr(), dens.data_ptr(), _stream())
        torch.cuda.synchronize()
        ref = P.absorbed_density(g, x[:, 0])
        assert rel(dens.cpu().numpy(), ref) <= 1e-12
    finally:
        B.bem_destroy(h)


@pytest.fixture(scope="module")
def full_size(B):
    """61440 unknowns, k0 a = 10, leaf 64, eta 2, ACA 1e-4 (the benchmark's operator),
    with the BF16 copy of the factors; 12 sampled rows of the dense product of two
    vectors, computed one by one by the oracle (no dense matrix)."""
    v, t = W.icosphere(5)
    g = R.build(v, t)
    h = make(B, v, t, k0=10.0, prec=B.BEM_PREC_C64 | B.BEM_PREC_BF16F, leaf=64, eta=2.0, aca_tol=1e-4)
    X = W.complex_normal(2 * g.ne, seed=0, nrhs=8).astype(np.complex64).astype(np.complex128)
    rows = np.random.default_rng(11).choice(2 * g.ne, 12, replace=False)
    refs = [O.pmchwt_rows_apply(g, 10.0, EPS, X[:, r].copy(), rows) for r in (0, 5)]
    yield h, g, X, rows, refs
    B.bem_destroy(h)


def _sampled_err(y, rows, ref):
    return float(np.abs(y[rows] - ref).max() / np.sqrt(np.mean(np.abs(y) ** 2)))


def test_full_size_sampled_rows(B, full_size):
    """Complex64 product in the launch configuration the benchmark times.  Measured
    error on these rows 4.8e-6 of rms (ACA 1e-4 compression of the far part, FP32
    rounding far below); bound 5e-5."""
    h, g, X, rows, refs = full_size
    y = matvec(B, h, X[:, 0].copy(), B.BEM_C64)
    err = _sampled_err(y, rows, refs[0])
    assert err <= 5e-5, err


def test_full_size_sampled_rows_bf16_factors(B, full_size):
    """Complex64 near entries with the BF16 copy of the far factors (8 significant bits
    per component, relative rounding 2^-9 ~ 2e-3 of the far part, which is a few
    percent of |y|): bound 5e-4 of rms."""
    h, g, X, rows, refs = full_size
    y = matvec(B, h, X[:, 0].copy(), B.BEM_C64_BF16F)
    err = _sampled_err(y, rows, refs[0])
    assert err <= 5e-4, err


def test_full_size_eight_vectors(B, full_size):
    """Eight right-hand sides in one operator pass at full size: every column equals
    its single-vector product to FP32 rounding, and two columns match the oracle's
    rows like the single product."""
    h, g, X, rows, refs = full_size
    Y = matvec(B, h, X, B.BEM_C64)
    for r, ref in zip((0, 5), refs):
        assert _sampled_err(Y[:, r], rows, ref) <= 5e-5
    for r in (0, 3, 7):
        y1 = matvec(B, h, X[:, r].copy(), B.BEM_C64)
        assert np.abs(Y[:, r] - y1).max() <= 1e-5 * np.abs(y1).max()


@pytest.mark.parametrize("dtype", [0, 1], ids=["c64", "c128"])
def test_batched_product_equals_one_at_a_time(B, sphere3, dtype):
    """13 right-hand sides (chunks of 8 + 4 + 1 streaming the operator once per chunk)
    give the same columns as 13 single products, and match the oracle."""
    v, t, g, Z = sphere3
    h = make(B, v, t, k0=10.0, prec=1 if dtype == 0 else 2, leaf=32, eta=2.0, aca_tol=1e-4)
    try:
        X = W.complex_normal(2 * g.ne, seed=8, nrhs=13)
        if dtype == 0:
            X = X.astype(np.complex64).astype(np.complex128)
        Y = matvec(B, h, X, dtype)
        single = np.stack([matvec(B, h, X[:, r].copy(), dtype) for r in range(13)], axis=1)
        tol = 1e-6 if dtype == 0 else 1e-14
        assert np.abs(Y - single).max() <= tol * np.abs(single).max()
        assert rel(Y, Z @ X) <= 1e-3
        assert elem(Y, Z @ X) <= 1e-3
    finally:
        B.bem_destroy(h)


def test_solver_reports_nonconvergence_and_bad_input(B, sphere2):
    """maxit = 1: BEM_ENOCONV with the residual of the last iterate reported (below 1,
    one GMRES step); a non-finite right-hand side is refused (BEM_EINVAL)."""
    v, t, g, _ = sphere2
    b = E.rhs_planewave(g, K0, [0.0, 0.0, 1.0], [1.0, 0.0, 0.0])
    h = make(B, v, t, prec=1, maxit=1, tol=1e-12)
    try:
        bd = torch.from_numpy(b).to(DEV)
        xd = torch.zeros_like(bd)
        it, relres, st = B.bem_solve(h, bd.data_ptr(), xd.data_ptr(), 1, _stream(), raise_on_noconv=False)
        assert st == B.BEM_ENOCONV and it == 1
        assert 0.0 < relres[0] < 1.0
        with pytest.raises(B.BemError) as ei:
            B.bem_solve(h, bd.data_ptr(), xd.data_ptr(), 1, _stream())
        assert ei.value.status == B.BEM_ENOCONV
        bad = b.copy()
        bad[3] = np.nan
        bdd = torch.from_numpy(bad).to(DEV)
        with pytest.raises(B.BemError) as ei:
            B.bem_solve(h, bdd.data_ptr(), xd.data_ptr(), 1, _stream())
        assert ei.value.status == B.BEM_EINVAL
    finally:
        B.bem_destroy(h)
