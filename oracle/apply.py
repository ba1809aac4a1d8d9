"""Dense expansion, product and error of an HSS result.

* ``to_dense`` -- the nested-basis expansion of eq. nestedUV and of the
  two-level example eq. HSSexamplematrix: leaves hold D_tau; the sibling
  blocks are U^big_nu1 B12 (V^big_nu2)^T and U^big_nu2 B21 (V^big_nu1)^T;
  U^big_tau = blockdiag(U^big_nu1, U^big_nu2) U_tau.
* ``matvec`` -- H X from the dense expansion (the plain definition).
* ``rel_error`` -- ||A - H||_F / ||A||_F, the error of Table 3.
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
