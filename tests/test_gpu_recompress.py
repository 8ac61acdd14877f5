"""GPU tests of the SVD recompression of ACA factors (bem_options.aca_recompress):
the same operator assembled with and without it.

Pins: the recompressed factors hold fewer entries; their total is at most the sum
over the far blocks of (SVD eps-rank + 2) (m + n), the eps-ranks taken from the
exact blocks of the oracle's dense PMCHWT matrix (Eq. 8) with numpy's SVD; and the
product against the oracle's dense product stays within twice the error of the
ACA factors alone (truncation adds at most tol |B|_F per block)."""
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


_cache = {}


def sphere3(k0):
    if k0 not in _cache:
        v, t = W.icosphere(3)
        g = R.build(v, t)
        ops = O.pmchwt_blocks(g, k0, EPS)
        Z = np.block([[ops[0], ops[1]], [-ops[1], ops[2]]])
        _cache[k0] = (v, t, g, ops, Z)
    return _cache[k0]


def _stream():
    return torch.cuda.current_stream().cuda_stream


def make(B, v, t, k0, prec, aca_tol, recompress, leaf=64):
    opt = B.bem_default_options()
    opt.precision = prec
    opt.leaf_size = leaf
    opt.eta = 2.0
    opt.aca_tol = aca_tol
    opt.aca_recompress = recompress
    h = B.bem_create(opt)
    B.bem_set_mesh(h, v, t)
    B.bem_set_media(h, k0, EPS)
    B.bem_assemble(h, _stream())
    return h


def product_error(B, h, Z, prec):
    n = Z.shape[0]
    x = W.complex_normal(n, seed=8)
    dt = B.BEM_C64 if prec == 1 else B.BEM_C128
    npdt = np.complex64 if prec == 1 else np.complex128
    xd = torch.from_numpy(x.astype(npdt)).to(DEV)
    yd = torch.empty_like(xd)
    B.bem_matvec(h, xd.data_ptr(), yd.data_ptr(), 1, dt, _stream())
    torch.cuda.synchronize()
    ref = Z @ x.astype(npdt).astype(np.complex128)
    y = yd.cpu().numpy().astype(np.complex128)
    return float(np.max(np.abs(y - ref)) / np.max(np.abs(ref)))


def svd_bound(B, h, ops, tol):
    """sum over the far blocks of (eps-rank + 2) (m + n), eps-ranks of the exact blocks."""
    perm, near, far = B.bem_partition(h)
    total = np.zeros(3, dtype=np.int64)
    for r0, m, c0, n in far:
        rows, cols = perm[r0:r0 + m], perm[c0:c0 + n]
        for q in range(3):
            s = np.linalg.svd(ops[q][np.ix_(rows, cols)], compute_uv=False)
            tail = np.sqrt(np.cumsum((s ** 2)[::-1])[::-1]) / np.linalg.norm(s)
            total[q] += (int(np.sum(tail > tol)) + 2) * (m + n)
    return total


# k0 a = 10 at 1e-4, where no far block of the 1280-triangle sphere needs more than
# its break-even rank (none is split), so the SVD bound applies block by block; at
# 1e-5 (k0 a = 2) about a third of the blocks split into dense children and only the
# savings and the accuracy are checked
@pytest.mark.parametrize("k0,prec,tol", [(10.0, 1, 1e-4), (2.0, 1, 1e-5), (2.0, 2, 1e-5)],
                         ids=["c64_1e-4", "c64_1e-5", "c128_1e-5"])
def test_recompression_saves_entries_within_svd_bound(B, k0, prec, tol):
    v, t, g, ops, Z = sphere3(k0)
    h0 = make(B, v, t, k0, prec, tol, 0)
    h1 = make(B, v, t, k0, prec, tol, 1)
    try:
        s0, s1 = B.bem_stats_get(h0), B.bem_stats_get(h1)
        f0, f1 = np.array(s0["factor_entries"]), np.array(s1["factor_entries"])
        print(f"{prec} {tol}: factor entries {f0.sum()} -> {f1.sum()} ({f1.sum() / f0.sum():.3f}), "
              f"max rank {s0['max_rank']} -> {s1['max_rank']}")
        assert s1["n_far_split"] == s0["n_far_split"]  # the same blocks are factored
        assert f1.sum() < 0.95 * f0.sum()
        assert np.all(f1 <= f0)
        assert s1["max_rank"] <= s0["max_rank"]
        if s1["n_far_split"] == 0:
            bound = svd_bound(B, h1, ops, tol)
            assert np.all(f1 <= bound), (f1, bound)
        else:
            assert tol < 1e-4  # the bound case must not split
        e0, e1 = product_error(B, h0, Z, prec), product_error(B, h1, Z, prec)
        print(f"   product error vs oracle: {e0:.3e} -> {e1:.3e}")
        assert e1 <= 2.0 * e0, (e0, e1)
    finally:
        B.bem_destroy(h0)
        B.bem_destroy(h1)
