"""QR with column pivoting and the interpolative decomposition.

Paper references: eq. ID / eq. QRCPSr (section 2.2): the ID of a local
sample S (m x d) is computed from a QRCP of S^* (d x m):
    S^* Pi = Q [R1 R2],  E = (R1^{-1} R2)^*,  U = Pi [I; E],
and the skeleton rows J are the first k pivots.

Rank rules:
* ``plain_rule`` (P4/P5): k = number of leading pivots j with
  |R_jj| > eps_a and |R_jj| > eps_r |R_11|, i.e. the factorisation stops at
  the first pivot that fails.
* ``hmt_rule`` (eq. RRQRHMTstop, section 2.4.1): at the k-th pivot (1-based)
  the tolerances are divided by f(k) = 1 + 4 sqrt(d)/(d-k-1) sqrt(min(m,n)),
  where d is the number of sample columns and m, n are the sizes of the
  Hankel block; f = infinity (no stop) when d-k-1 <= 0 (P6).

The factorisation is the textbook Businger-Golub Householder QRCP: at every
step the 2-norms of all trailing columns are recomputed exactly (no
down-dating), the largest is taken as pivot (lowest index on ties, P14),
and a Householder reflector annihilates the pivot column below the
diagonal.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.linalg import solve_triangular


def plain_rule(eps_r: float, eps_a: float):
    def stop(j, rjj, r11):
        return rjj <= eps_a or rjj <= eps_r * r11
    return stop


def hmt_factor(k1: int, d: int, mh: int, nh: int) -> float:
    """f(k) of eq. RRQRHMTstop for the 1-based pivot index k1."""
    den = d - k1 - 1
    if den <= 0:
        return math.inf
    return 1.0 + 4.0 * math.sqrt(d) / den * math.sqrt(min(mh, nh))


def hmt_rule(eps_r: float, eps_a: float, d: int, mh: int, nh: int):
    def stop(j, rjj, r11):
        f = hmt_factor(j + 1, d, mh, nh)
        return rjj <= eps_a / f or rjj <= eps_r * r11 / f
    return stop


def qrcp(W: np.ndarray, stop):
    """Truncated Householder QRCP of W (d x m).

    Returns (piv, R, k, stopped): piv is the full column permutation, R the
    first k rows of the triangular factor in pivoted column order (k x m),
    and ``stopped`` tells whether the rule fired before min(d, m) pivots.
    """
    W = np.array(W, dtype=np.float64, copy=True)
    d, m = W.shape
    piv = np.arange(m)
    r11 = None
    for j in range(min(d, m)):
        norms = np.sqrt(np.sum(W[j:, j:] ** 2, axis=0))
        p = j + int(np.argmax(norms))
        rjj = float(norms[p - j])
        if r11 is None:
            r11 = rjj
        if stop(j, rjj, r11):
            return piv, W[:j, :].copy(), j, True
        if p != j:
            W[:, [j, p]] = W[:, [p, j]]
            piv[[j, p]] = piv[[p, j]]
        x = W[j:, j]
        s = 1.0 if x[0] >= 0 else -1.0
        v = x.copy()
        v[0] += s * rjj
        vn = np.linalg.norm(v)
        if vn > 0:
            v /= vn
            W[j:, j:] -= 2.0 * np.outer(v, v @ W[j:, j:])
        W[j + 1:, j] = 0.0
    k = min(d, m)
    return piv, np.triu(W[:k, :]), k, False


def interpolative(piv, R, k):
    """From a truncated QRCP, the ID of S (m x d): returns
    (J, X, U) with J = piv[:k], X = R1^{-1} R2 (k x (m-k)) and the m x k
    basis U = Pi [I; X^T] so that S ~= U S(J, :)."""
    m = piv.size
    J = piv[:k].copy()
    if k > 0 and m > k:
        X = solve_triangular(R[:k, :k], R[:k, k:m], lower=False)
    else:
        X = np.zeros((k, m - k))
    U = np.zeros((m, k))
    U[piv[:k], np.arange(k)] = 1.0
    U[piv[k:], :] = X.T
    return J, X, U


def near_threshold_count(S: np.ndarray, er: float, ea: float, rule: str, mh: int = 0, nh: int = 0,
                         band: float = 0.1, noise: float = 0.0) -> int:
    """Number of singular values of a local sample S (m x d) within +-band
    of the rank threshold that the ID's rule applies at their position:
    max(eps_a, eps_r |R_11|) (P4; |R_11| = the largest row norm of S, the
    first pivot's norm whatever the pivot order), divided by the HMT factor
    f(j + 1) of eq. RRQRHMTstop under ``rule == "hmt"``.  Where pivot order
    diverges at near ties, a rank can cross such a value but not more of
    them than there are (the tie rule of the rank comparison).  ``noise``:
    a bound on the 2-norm of a perturbation of S (a sample computed in
    another arithmetic); by Weyl's inequality it moves every singular value
    by at most that much, so the band widens by it."""
    sv = np.linalg.svd(np.asarray(S, dtype=np.float64), compute_uv=False)
    if sv.size == 0:
        return 0
    r11 = float(np.max(np.linalg.norm(S, axis=1)))
    d = S.shape[1]
    cnt = 0
    for j, s in enumerate(sv):
        f = hmt_factor(j + 1, d, mh, nh) if rule == "hmt" else 1.0
        thr = max(ea, er * r11) / f
        if abs(s - thr) <= band * thr + noise:
            cnt += 1
    return cnt


def near_threshold_count_qr(S: np.ndarray, er: float, ea: float, rule: str, mh: int = 0, nh: int = 0,
                            band: float = 0.1, noise: float = 0.0) -> int:
    """Number of pivots j of the full QRCP of S^* (d x m) whose |R_jj| lies
    within +-band of the rank threshold at its position -- the quantity the
    ID's rule itself compares (P4; eq. RRQRHMTstop divides the threshold by
    f(j + 1) under ``rule == "hmt"``), where near_threshold_count looks at
    the singular values.  Two QRCPs of the same sample in different
    arithmetic can stop one pivot apart at each such |R_jj|.  ``noise``
    widens the band as there."""
    W = np.asarray(S, dtype=np.float64).T
    d, m = W.shape
    if min(d, m) == 0:
        return 0
    _, R, _, _ = qrcp(W, lambda j, rjj, r11: False)
    rd = np.abs(np.diag(R))
    r11 = float(rd[0])
    cnt = 0
    for j, r in enumerate(rd):
        f = hmt_factor(j + 1, d, mh, nh) if rule == "hmt" else 1.0
        thr = max(ea, er * r11) / f
        if abs(r - thr) <= band * thr + noise:
            cnt += 1
    return cnt
