"""Pins of the oracle's cluster/block partition and of its cross approximation."""
import numpy as np
import pytest

import workloads as W
from oracle import aca as A
from oracle import operators as O
from oracle import rwg as R
from oracle import tree as TR


@pytest.mark.parametrize("level,leaf,eta", [(2, 16, 2.0), (3, 64, 2.0), (3, 32, 1.0), (2, 16, 0.0)])
def test_partition_covers_matrix_once(level, leaf, eta):
    v, t = W.icosphere(level)
    g = R.build(v, t)
    pts = g.midpoints()
    root, perm = TR.cluster_tree(pts, leaf)
    assert np.array_equal(np.sort(perm), np.arange(g.ne))
    for c in TR.leaves(root):
        assert 0 < c.size <= leaf
    near, far = TR.block_partition(root, eta)
    cover = np.zeros((g.ne, g.ne), dtype=np.int32)
    for r0, m, c0, n in np.concatenate([near, far]):
        cover[r0:r0 + m, c0:c0 + n] += 1
    assert np.all(cover == 1)
    leaf_ranges = {(c.lo, c.size) for c in TR.leaves(root)}
    for r0, m, c0, n in near:
        assert (r0, m) in leaf_ranges and (c0, n) in leaf_ranges
    if eta == 0.0:
        assert len(far) == 0
    # far blocks satisfy the admissibility condition, recomputed from the points
    for r0, m, c0, n in far:
        P, Q = pts[perm[r0:r0 + m]], pts[perm[c0:c0 + n]]
        dt = np.linalg.norm(P.max(0) - P.min(0))
        ds = np.linalg.norm(Q.max(0) - Q.min(0))
        gap = np.maximum(0, np.maximum(Q.min(0) - P.max(0), P.min(0) - Q.max(0)))
        assert min(dt, ds) <= eta * np.linalg.norm(gap) * (1 + 1e-12)


def test_children_split_at_median_along_longest_axis():
    v, t = W.icosphere(2)
    g = R.build(v, t)
    pts = g.midpoints()
    root, perm = TR.cluster_tree(pts, 16)
    stack = [root]
    while stack:
        c = stack.pop()
        if c.is_leaf:
            continue
        left, right = c.children
        assert left.size == c.size // 2 and left.lo == c.lo and right.hi == c.hi
        axis = int(np.argmax(c.bbmax - c.bbmin))
        lk = pts[perm[left.lo:left.hi], axis]
        rk = pts[perm[right.lo:right.hi], axis]
        assert lk.max() <= rk.min()
        stack += c.children


def test_aca_recovers_exact_low_rank():
    rng = np.random.default_rng(0)
    U = rng.standard_normal((70, 5)) + 1j * rng.standard_normal((70, 5))
    V = rng.standard_normal((50, 5)) + 1j * rng.standard_normal((50, 5))
    B = U @ V.conj().T
    Ua, Va = A.aca_dense(B, 1e-12)
    assert Ua.shape[1] <= 6
    assert np.linalg.norm(B - Ua @ Va.conj().T) <= 1e-12 * np.linalg.norm(B)


@pytest.fixture(scope="module")
def far_blocks():
    v, t = W.icosphere(3)
    g = R.build(v, t)
    root, perm = TR.cluster_tree(g.midpoints(), 64)
    near, far = TR.block_partition(root, 2.0)
    A_, B_, C_ = O.pmchwt_blocks(g, 10.0, 3.2 - 1.9j)
    return perm, far, (A_, B_, C_)


@pytest.mark.parametrize("tol", [1e-4, 1e-6])
def test_aca_error_and_rank_vs_svd(far_blocks, tol):
    perm, far, ops = far_blocks
    order = np.argsort(-(far[:, 1] * far[:, 3]))
    for bi in order[:6]:
        r0, m, c0, n = far[bi]
        for Op in ops:
            Bk = Op[np.ix_(perm[r0:r0 + m], perm[c0:c0 + n])]
            U, V = A.aca_dense(Bk, tol)
            err = np.linalg.norm(Bk - U @ V.conj().T) / np.linalg.norm(Bk)
            s = np.linalg.svd(Bk, compute_uv=False)
            tail = np.sqrt(np.cumsum((s ** 2)[::-1])[::-1]) / np.linalg.norm(s)
            eps_rank = int(np.sum(tail > tol))
            assert err <= 10 * tol, (bi, err)
            assert U.shape[1] <= 2 * eps_rank + 2, (U.shape[1], eps_rank)


def _eps_rank(s, tol):
    tail = np.sqrt(np.cumsum((s ** 2)[::-1])[::-1]) / np.linalg.norm(s)
    return int(np.sum(tail > tol))


def test_recompress_keeps_an_exact_low_rank_product():
    rng = np.random.default_rng(4)
    B = (rng.standard_normal((60, 3)) + 1j * rng.standard_normal((60, 3))) @ \
        (rng.standard_normal((3, 45)) + 1j * rng.standard_normal((3, 45)))
    # an over-long factorisation of the rank-3 block: 7 columns
    U = B[:, :7]
    V = np.linalg.lstsq(U, B, rcond=None)[0].conj().T
    assert np.linalg.norm(U @ V.conj().T - B) <= 1e-10 * np.linalg.norm(B)
    U2, V2 = A.recompress(U, V, 1e-12)
    assert U2.shape[1] == 3
    assert np.linalg.norm(U2 @ V2.conj().T - B) <= 1e-10 * np.linalg.norm(B)


@pytest.mark.parametrize("tol", [1e-4, 1e-6])
def test_recompress_is_the_truncated_svd(far_blocks, tol):
    """The singular values of U' V'^H are the leading ones of U V^H, and what it drops
    is within tol of |U V^H|_F (the definition of the truncated SVD)."""
    perm, far, ops = far_blocks
    order = np.argsort(-(far[:, 1] * far[:, 3]))
    for bi in order[:4]:
        r0, m, c0, n = far[bi]
        Bk = ops[1][np.ix_(perm[r0:r0 + m], perm[c0:c0 + n])]
        U, V = A.aca_dense(Bk, tol)
        P = U @ V.conj().T
        U2, V2 = A.recompress(U, V, tol)
        r = U2.shape[1]
        s = np.linalg.svd(P, compute_uv=False)
        s2 = np.linalg.svd(U2 @ V2.conj().T, compute_uv=False)[:r]
        assert np.allclose(s2, s[:r], rtol=1e-9, atol=1e-12 * s[0])
        assert np.linalg.norm(P - U2 @ V2.conj().T) <= tol * np.linalg.norm(P) * (1 + 1e-9)
        assert r == _eps_rank(s[:U.shape[1]], tol)


@pytest.mark.parametrize("tol", [1e-4, 1e-6])
def test_recompressed_rank_within_two_of_the_svd_rank(far_blocks, tol):
    """Against the exact block: after recompression every far block's rank is at
    most its SVD eps-rank + 2, and the block error stays within the ACA bound (10 tol)
    plus the truncation (2 tol)."""
    perm, far, ops = far_blocks
    order = np.argsort(-(far[:, 1] * far[:, 3]))
    for bi in order[:8]:
        r0, m, c0, n = far[bi]
        for Op in ops:
            Bk = Op[np.ix_(perm[r0:r0 + m], perm[c0:c0 + n])]
            U, V = A.aca_dense(Bk, tol)
            U2, V2 = A.recompress(U, V, tol)
            s = np.linalg.svd(Bk, compute_uv=False)
            assert U2.shape[1] <= _eps_rank(s, tol) + 2, (bi, U2.shape[1], _eps_rank(s, tol))
            assert U2.shape[1] <= U.shape[1]
            err = np.linalg.norm(Bk - U2 @ V2.conj().T) / np.linalg.norm(Bk)
            assert err <= 10 * tol + 2 * tol, err
