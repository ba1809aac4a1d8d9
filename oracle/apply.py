"""Dense expansion, product and error of an HSS result.

* ``to_dense`` -- the nested-basis expansion of eq. nestedUV and of the
  two-level example eq. HSSexamplematrix: leaves hold D_tau; the sibling
  blocks are U^big_nu1 B12 (V^big_nu2)^T and U^big_nu2 B21 (V^big_nu1)^T;
  U^big_tau = blockdiag(U^big_nu1, U^big_nu2) U_tau.
* ``matvec`` -- H X from the dense expansion (the plain definition).
* ``rel_error`` -- ||A - H||_F / ||A||_F, the error of Table 3.
* ``column_block`` / ``rel_error_blocks`` -- the same expansion one block of
  columns at a time, for matrices too large to hold densely (A's columns
  taken from the source's entries).
"""
from __future__ import annotations

import numpy as np


def to_dense(res) -> np.ndarray:
    nodes = res.nodes
    H = np.zeros((res.n, res.n))
    Ubig, Vbig = {}, {}
    for t in reversed(nodes):
        if t.is_leaf:
            H[t.lo:t.lo + t.size, t.lo:t.lo + t.size] = t.D
            if t.parent >= 0:
                Ubig[t.idx], Vbig[t.idx] = t.U, t.V
            continue
        a, b = nodes[t.children[0]], nodes[t.children[1]]
        H[a.lo:a.lo + a.size, b.lo:b.lo + b.size] = Ubig[a.idx] @ t.B12 @ Vbig[b.idx].T
        H[b.lo:b.lo + b.size, a.lo:a.lo + a.size] = Ubig[b.idx] @ t.B21 @ Vbig[a.idx].T
        if t.parent >= 0:
            ka_r, ka_c = Ubig[a.idx].shape[1], Vbig[a.idx].shape[1]
            Ubig[t.idx] = np.vstack([Ubig[a.idx] @ t.U[:ka_r], Ubig[b.idx] @ t.U[ka_r:]])
            Vbig[t.idx] = np.vstack([Vbig[a.idx] @ t.V[:ka_c], Vbig[b.idx] @ t.V[ka_c:]])
    return H


def matvec(res, X: np.ndarray) -> np.ndarray:
    return to_dense(res) @ X


def rel_error(res, A: np.ndarray) -> float:
    return float(np.linalg.norm(A - to_dense(res)) / np.linalg.norm(A))


def abs_error(res, A: np.ndarray) -> float:
    return float(np.linalg.norm(A - to_dense(res)))


def _big_bases(res):
    """U^big_tau and V^big_tau of every non-root node (eq. nestedUV)."""
    nodes = res.nodes
    Ubig, Vbig = {}, {}
    for t in reversed(nodes):
        if t.parent < 0:
            continue
        if t.is_leaf:
            Ubig[t.idx], Vbig[t.idx] = t.U, t.V
            continue
        a, b = nodes[t.children[0]], nodes[t.children[1]]
        ka_r, ka_c = Ubig[a.idx].shape[1], Vbig[a.idx].shape[1]
        Ubig[t.idx] = np.vstack([Ubig[a.idx] @ t.U[:ka_r], Ubig[b.idx] @ t.U[ka_r:]])
        Vbig[t.idx] = np.vstack([Vbig[a.idx] @ t.V[:ka_c], Vbig[b.idx] @ t.V[ka_c:]])
    return Ubig, Vbig


def column_block(res, j0: int, j1: int, bases=None) -> np.ndarray:
    """H(:, j0:j1) from the same expansion as ``to_dense``: the leaf blocks D
    that meet the columns, and for every node the sibling blocks
    U^big_nu1 B12 (V^big_nu2)^T and U^big_nu2 B21 (V^big_nu1)^T restricted to
    them."""
    Ubig, Vbig = bases if bases is not None else _big_bases(res)
    out = np.zeros((res.n, j1 - j0))
    for t in res.nodes:
        if t.is_leaf:
            lo, hi = max(t.lo, j0), min(t.lo + t.size, j1)
            if lo < hi:
                out[t.lo:t.lo + t.size, lo - j0:hi - j0] = t.D[:, lo - t.lo:hi - t.lo]
            continue
        a, b = res.nodes[t.children[0]], res.nodes[t.children[1]]
        for x, y, B in ((a, b, t.B12), (b, a, t.B21)):
            lo, hi = max(y.lo, j0), min(y.lo + y.size, j1)
            if lo < hi:
                Vy = Vbig[y.idx][lo - y.lo:hi - y.lo]
                out[x.lo:x.lo + x.size, lo - j0:hi - j0] = Ubig[x.idx] @ (B @ Vy.T)
    return out


def rel_error_blocks(res, src, block: int = 2048) -> float:
    """||A - H||_F / ||A||_F with A's columns from ``src.entries`` and H's
    from ``column_block``, one block of columns at a time."""
    bases = _big_bases(res)
    rows = np.arange(res.n)
    num = den = 0.0
    for j0 in range(0, res.n, block):
        j1 = min(res.n, j0 + block)
        Ab = src.entries(rows, np.arange(j0, j1))
        num += float(np.sum((Ab - column_block(res, j0, j1, bases)) ** 2))
        den += float(np.sum(Ab ** 2))
    return float(np.sqrt(num / den))
