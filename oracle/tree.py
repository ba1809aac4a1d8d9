"""Cluster tree (paper section 2.1, "HSS Representation"; section 3).

The tree is binary, numbered level by level from 0 at the root; every node
owns a contiguous index range and its two children partition it.  The same
tree is used for rows and columns.

Readings:
* P13 -- a node of size m > leaf splits into floor(m/2) and ceil(m/2); for a
  point set, recursive coordinate bisection (RCB) first orders the points:
  at each node the coordinate of largest extent (lowest coordinate on ties)
  is sorted by (value, original index) and the first floor(m/2) points go to
  the first child.  The RCB tree is then the halving tree of the permuted
  order.
"""
from __future__ import annotations

import numpy as np


class Node:
    """One node of the cluster tree plus the per-node temporaries of
    Algorithms 1-3 (tau.S^r, tau.R^r, tau.J^r, tau.I^r, ...)."""

    def __init__(self, idx, lo, size, level, parent):
        self.idx, self.lo, self.size, self.level, self.parent = idx, lo, size, level, parent
        self.children: list[int] = []
        self.reset()

    def reset(self):
        self.state = "U"           # UNTOUCHED / "PC" / "C"
        self.D = None
        self.B12 = self.B21 = None
        self.Sr = self.Sc = None   # local samples, m x d
        self.Rr = self.Rc = None   # reduced random blocks
        self.U = self.V = None
        self.Jr = self.Jc = None   # skeleton rows (local indices, pivot order)
        self.Xr = self.Xc = None   # R1^{-1} R2  (E^T)
        self.piv_r = self.piv_c = None
        self.d_id = None           # sample columns the ID was taken from
        self.Ir = self.Ic = None   # skeleton rows as global indices
        self.inc = {}              # Incrementing per-side state

    @property
    def is_leaf(self):
        return not self.children

    @property
    def I(self):
        return np.arange(self.lo, self.lo + self.size)


def halving_tree(n: int, leaf: int) -> list[Node]:
    """Level-order list of nodes; node 0 is the root (level 0)."""
    nodes = [Node(0, 0, n, 0, -1)]
    i = 0
    while i < len(nodes):
        t = nodes[i]
        if t.size > leaf:
            h = t.size // 2
            for lo, m in ((t.lo, h), (t.lo + h, t.size - h)):
                c = Node(len(nodes), lo, m, t.level + 1, i)
                t.children.append(c.idx)
                nodes.append(c)
        i += 1
    return nodes


def rcb_order(points: np.ndarray, leaf: int) -> np.ndarray:
    """Recursive coordinate bisection.  Returns perm with perm[new] = old."""
    points = np.asarray(points, dtype=np.float64)
    n = points.shape[0]
    perm = np.arange(n, dtype=np.int64)
    stack = [(0, n)]
    while stack:
        lo, m = stack.pop()
        if m <= leaf:
            continue
        idx = perm[lo:lo + m]
        P = points[idx]
        ext = P.max(axis=0) - P.min(axis=0)
        c = int(np.argmax(ext))
        order = np.lexsort((idx, P[:, c]))
        perm[lo:lo + m] = idx[order]
        h = m // 2
        stack.append((lo + h, m - h))
        stack.append((lo, h))
    return perm
