"""Cluster tree and block partition (oracle, test infrastructure).

The paper's compressed block (Eq. 17) is global; the library splits the
operator into a hierarchy of blocks instead, each either stored densely (near)
or compressed (far).  The partition is defined here exactly, so that the GPU
builder can be checked for equality:

  cluster tree over the RWG edge midpoints ((v0 + v1) * 0.5, float64):
    a cluster is a contiguous range of a permutation of the edges; the root
    holds all edges in index order; a cluster with more than ``leaf_size``
    edges is split: its bounding box picks the axis of largest extent (first
    axis on ties), its points are ordered by (coordinate on that axis,
    original edge index), the first floor(size/2) form the left child.
  block tree from (root, root):
    admissible (far) if eta > 0, dist > 0 and min(diam_t, diam_s) <= eta dist,
      tested as min(diam_t^2, diam_s^2) <= (eta*eta) * dist^2 with
      diam^2 = (dx*dx + dy*dy) + dz*dz of the bounding-box extents and dist^2
      the same sum of the per-axis box gaps max(0, lo_s - hi_t, lo_t - hi_s);
    else near if both clusters are leaves;
    else recurse into the children of every non-leaf side.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Cluster:
    lo: int
    hi: int
    bbmin: np.ndarray
    bbmax: np.ndarray
    children: list = field(default_factory=list)

    @property
    def size(self) -> int:
        return self.hi - self.lo

    @property
    def is_leaf(self) -> bool:
        return not self.children


def cluster_tree(points: np.ndarray, leaf_size: int = 64):
    """Return (root, perm): perm[k] is the edge at position k of the tree order."""
    points = np.asarray(points, dtype=np.float64)
    perm = np.arange(len(points), dtype=np.int64)

    def build(lo, hi):
        P = points[perm[lo:hi]]
        c = Cluster(lo, hi, P.min(axis=0), P.max(axis=0))
        if hi - lo > leaf_size:
            ext = c.bbmax - c.bbmin
            axis = int(np.argmax(ext))
            order = np.lexsort((perm[lo:hi], P[:, axis]))
            perm[lo:hi] = perm[lo:hi][order]
            mid = lo + (hi - lo) // 2
            c.children = [build(lo, mid), build(mid, hi)]
        return c

    root = build(0, len(points))
    return root, perm


def _sq3(v):
    return (v[0] * v[0] + v[1] * v[1]) + v[2] * v[2]


def admissible(t: Cluster, s: Cluster, eta: float) -> bool:
    if eta <= 0.0:
        return False
    gap = np.maximum(0.0, np.maximum(s.bbmin - t.bbmax, t.bbmin - s.bbmax))
    dist2 = _sq3(gap)
    if not dist2 > 0.0:
        return False
    d2 = min(_sq3(t.bbmax - t.bbmin), _sq3(s.bbmax - s.bbmin))
    return bool(d2 <= (eta * eta) * dist2)


def block_partition(root: Cluster, eta: float):
    """Near and far block lists as int64 arrays of (row_lo, m, col_lo, n), sorted by (row_lo, col_lo)."""
    near, far = [], []
    stack = [(root, root)]
    while stack:
        t, s = stack.pop()
        if admissible(t, s, eta):
            far.append((t.lo, t.size, s.lo, s.size))
        elif t.is_leaf and s.is_leaf:
            near.append((t.lo, t.size, s.lo, s.size))
        elif t.is_leaf:
            stack += [(t, sc) for sc in s.children]
        elif s.is_leaf:
            stack += [(tc, s) for tc in t.children]
        else:
            stack += [(tc, sc) for tc in t.children for sc in s.children]

    def canon(lst):
        a = np.array(lst, dtype=np.int64).reshape(-1, 4)
        return a[np.lexsort((a[:, 2], a[:, 0]))] if len(a) else a

    return canon(near), canon(far)


def leaves(root: Cluster):
    out = []
    stack = [root]
    while stack:
        c = stack.pop()
        if c.is_leaf:
            out.append(c)
        else:
            stack += c.children[::-1]
    return sorted(out, key=lambda c: c.lo)
