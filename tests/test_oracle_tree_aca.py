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
