"""Adaptive randomized HSS compression (Algorithm 3) with Algorithm 2.

The compression is written as the paper's recursive post-order traversal
(CompressNodeAdaptive) inside the outer loop of HSSCompressAdaptive:

  d <- d0; R, S^r = A R, S^c = A^T R;  all nodes UNTOUCHED
  while root is not COMPRESSED:
      CompressNodeAdaptive(root)
      grow R by dd columns (Incrementing) or by d columns (Doubling) and
      append A R_new to S^r and A^T R_new to S^c            (P1)

CompressNodeAdaptive(tau):
  leaf: D = A(I, I) when UNTOUCHED.  non-leaf: recurse into both children,
  return unless both are COMPRESSED, extract B12 = A(nu1.I^r, nu2.I^c),
  B21 = A(nu2.I^r, nu1.I^c) when UNTOUCHED.  root: mark COMPRESSED.
  Local samples (Algorithm 2): all columns when UNTOUCHED, the new ones
  otherwise.  A node that is not COMPRESSED runs the strategy's test and,
  on success, the ID of both samples at eps/level(tau) (P3), is marked
  COMPRESSED and reduces all columns; on failure it is marked
  PARTIALLY_COMPRESSED.  A COMPRESSED node reduces the new columns.

Readings (see the design notes for the full list):
 P1  S^c grows with A^T R_new (the algorithm's S^r there is a typo).
 P2  the merge uses nu2.S^r(nu2.J^r) and B12 nu2.R^r, as in Algorithm 2.
 P3  tolerances eps_r/level(tau), eps_a/level(tau), root at level 0.
 P4  ID rank = leading pivots passing both tolerances.
 P5  Incrementing's final RRQR uses the P4 rule on all columns.
 P6  Doubling: d0 columns first, then Delta d = d; a node is accepted iff
     RRQR_HMT stops at rank k <= d - p, or selects all m rows (P9).
 P7  the absolute Incrementing test divides by sqrt(#columns in the block).
 P8  rho = |(R_1)_11| of the side's first block.
 P9  a sample whose rows are all selected is exact: accept (Doubling), and
     an Incrementing basis Q with m columns is sufficient.
 P17 the column ranges of Algorithm 3 are "all columns so far" for an
     UNTOUCHED node and "the columns added by the last growth" otherwise.
 P18 Incrementing tests a side's columns in the blocks in which they were
     drawn (d0 columns, then Delta d per growth), in order, stopping at the
     first sufficient block: a node touched for the first time after growth
     runs Algorithm 5 over its earlier blocks within the pass, exactly as if
     it had been tested at every pass.  A side that passed stays passed; the
     node is COMPRESSED when both sides have passed.
 P19 the loop ends after a failed pass at d = d_max (NOT_CONVERGED); the
     last growth is clipped so that d <= d_max.
 P21 symmetric option (A = A^T): Algorithm 3 with A^T = A makes the
     column side a copy of the row side — S^c = S^r, the same ID (J^c = J^r,
     V = U), R^c = R^r and B21 = B12^T — so only the row side is sampled,
     tested and factored, and the column side takes its results.
 P22 HMT criterion option (Lemma 4.1, eq. HMT_IQQH): Incrementing with the
     test of each block S_k replaced by  alpha sqrt(2/pi) max_i
     |((I - Q Q^T)^2 S_k)(:, i)|_2 <= eps_a  on the node's local sample
     (the only sample the construction has); on failure the block's
     orthonormal basis joins Q, as in Algorithm 5.  The criterion has no
     relative form, so rtol is ignored and the final RRQR keeps the pivots
     with |R_jj| > eps_a.
 P23 hard restart (section 4.3.2, Table 4): attempts with d = d0, 2 d0,
     4 d0, ... (the last clipped to d_max), each Algorithm 3 with no growth
     (d_max = d) on the first d columns of R and nothing carried over; the
     strategy's own test is the failure check; the first converged attempt
     is the result.  The known-rank mode is one attempt with d0 = d_max.
 P24 user sampling operator (section 3.1, partially matrix-free): with
     ``product`` the samples A R and A^T R come from the caller's product;
     the leaf diagonal blocks D R(I) are still removed from the source's
     entries (Algorithm 2), which also give every generator.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

from .qrcp import qrcp, interpolative, plain_rule, hmt_rule
from .tree import halving_tree


@dataclass
class Options:
    leaf: int = 64
    rtol: float = 1e-6
    atol: float = 1e-12
    d0: int = 64
    dd: int = 32
    d_max: int = 1024
    strategy: str = "incrementing"     # or "doubling"
    p: int = 10
    level_tol_scaling: bool = True
    criterion: str = "new"             # or "hmt" (P22; Incrementing only)
    hmt_alpha: float = 10.0
    symmetric: bool = False            # A = A^T: one sample, V = U (see P21)


@dataclass
class Result:
    n: int
    nodes: list
    d_final: int
    n_adapt: int
    converged: bool
    passes: list = field(default_factory=list)

    def ranks(self):
        return {t.idx: (len(t.Jr), len(t.Jc)) for t in self.nodes
                if t.idx != 0 and t.Jr is not None}

    def max_rank(self):
        r = self.ranks()
        return max((max(a, b) for a, b in r.values()), default=0)


class _Sampler:
    """S^r = A R and S^c = A^T R for the new columns of R, through the
    source's entries in row panels (a plain product, no structure used), or
    through a user product(X, trans) -> A X / A^T X (section 3.1)."""

    def __init__(self, src, product=None):
        self.src = src
        self.n = src.n
        self.product = product
        self.dense = (src.to_dense() if product is None and (src.dense is not None or src.n <= 8192)
                      else None)

    def sample(self, Rnew, symmetric=False):
        if self.product is not None:
            Sr = self.product(Rnew, False)
            return Sr, (Sr if symmetric else self.product(Rnew, True))
        if self.dense is not None:
            Sr = self.dense @ Rnew
            return Sr, (Sr if symmetric else self.dense.T @ Rnew)
        n = self.n
        Sr = np.zeros((n, Rnew.shape[1]))
        Sc = np.zeros((n, Rnew.shape[1]))
        idx = np.arange(n)
        step = max(1, (1 << 24) // n)
        for i0 in range(0, n, step):
            blk = self.src.entries(idx[i0:i0 + step], idx)
            Sr[i0:i0 + step] = blk @ Rnew
            if not symmetric:
                Sc += blk.T @ Rnew[i0:i0 + step]
        return Sr, (Sr if symmetric else Sc)

    def entries(self, I, J):
        if self.dense is not None:
            return self.dense[np.ix_(np.asarray(I, dtype=np.int64), np.asarray(J, dtype=np.int64))]
        return self.src.entries(I, J)


def compress(src, R: np.ndarray, opts: Options, product=None) -> Result:
    """HSSCompressAdaptive (Algorithm 3).  ``R`` is the caller's n x d_max
    Gaussian matrix; the pass with d columns uses R[:, :d].  ``product``:
    optional user sampling operator, product(X, trans) = A X or A^T X (the
    partially matrix-free interface of section 3.1); the entries for the
    generators and the leaf diagonal blocks still come from ``src``."""
    if opts.criterion not in ("new", "hmt"):
        raise ValueError(f"unknown criterion {opts.criterion!r}")
    if opts.criterion == "hmt" and (opts.strategy != "incrementing" or not opts.hmt_alpha > 1.0):
        raise ValueError("the HMT criterion is an Incrementing test with alpha > 1")
    n = src.n
    nodes = halving_tree(n, opts.leaf)
    A = _Sampler(src, product)
    d_max = min(opts.d_max, R.shape[1])
    d = min(opts.d0, d_max)
    Sr, Sc = A.sample(R[:, :d], opts.symmetric)
    ctx = dict(A=A, R=R, opts=opts, nodes=nodes, d_prev=0, d=d, bounds=[d])
    n_adapt = 0
    passes = []
    while True:
        ctx["Sr"], ctx["Sc"] = Sr, Sc
        _compress_node(ctx, nodes[0])
        passes.append(dict(d=d, states=[t.state for t in nodes]))
        if nodes[0].state == "C":
            return Result(n, nodes, d, n_adapt, True, passes)
        if d >= d_max:
            return Result(n, nodes, d, n_adapt, False, passes)
        dd = d if opts.strategy == "doubling" else opts.dd
        dd = min(dd, d_max - d)
        Srn, Scn = A.sample(R[:, d:d + dd], opts.symmetric)
        Sr = np.hstack([Sr, Srn])
        Sc = Sr if opts.symmetric else np.hstack([Sc, Scn])
        ctx["d_prev"], ctx["d"] = d, d + dd
        d += dd
        ctx["bounds"].append(d)
        n_adapt += 1


def compress_hard_restart(src, R: np.ndarray, opts: Options):
    """The "hard-restart" mode the paper compares against (section 4.3.2,
    Table 4, P23): without adaptivity a user restarts the compression from
    scratch with more random vectors when it fails.  Returns the first
    converged attempt (or the last one, at d_max) and the number of
    restarts."""
    d_cap = min(opts.d_max, R.shape[1])
    d = min(opts.d0, d_cap)
    restarts = 0
    while True:
        res = compress(src, R, replace(opts, d0=d, d_max=d))
        if res.converged or d >= d_cap:
            return res, restarts
        d = min(2 * d, d_cap)
        restarts += 1


def _tols(opts: Options, level: int):
    if opts.level_tol_scaling:
        return opts.rtol / level, opts.atol / level
    return opts.rtol, opts.atol


def _compress_node(ctx, t):
    nodes, A, opts = ctx["nodes"], ctx["A"], ctx["opts"]
    d_prev, d = ctx["d_prev"], ctx["d"]
    if t.is_leaf:
        if t.state == "U":
            t.D = A.entries(t.I, t.I)
    else:
        c1, c2 = nodes[t.children[0]], nodes[t.children[1]]
        _compress_node(ctx, c1)
        _compress_node(ctx, c2)
        if c1.state != "C" or c2.state != "C":
            return
        if t.state == "U":
            t.B12 = A.entries(c1.Ir, c2.Ic)
            t.B21 = A.entries(c2.Ir, c1.Ic)
    if t.parent < 0:
        t.state = "C"
        return
    cols = slice(0, d) if t.state == "U" else slice(d_prev, d)
    _local_samples(ctx, t, cols)
    if t.state != "C":
        if _node_sufficient(ctx, t):
            t.state = "C"
            _reduce_local_samples(ctx, t, slice(0, d))
        else:
            t.state = "PC"
    else:
        _reduce_local_samples(ctx, t, slice(d_prev, d))


def _local_samples(ctx, t, cols):
    """ComputeLocalSamples (Algorithm 2) for the columns ``cols``."""
    nodes, R = ctx["nodes"], ctx["R"]
    d = ctx["d"]
    sym = ctx["opts"].symmetric
    if t.is_leaf:
        I = t.I
        sr = ctx["Sr"][I, cols] - t.D @ R[I, cols]
        sc = sr if sym else ctx["Sc"][I, cols] - t.D.T @ R[I, cols]
        m_r = m_c = t.size
    else:
        c1, c2 = nodes[t.children[0]], nodes[t.children[1]]
        sr = np.vstack([c1.Sr[c1.Jr, cols] - t.B12 @ c2.Rr[:, cols],
                        c2.Sr[c2.Jr, cols] - t.B21 @ c1.Rr[:, cols]])
        sc = sr if sym else np.vstack([c1.Sc[c1.Jc, cols] - t.B21.T @ c2.Rc[:, cols],
                                       c2.Sc[c2.Jc, cols] - t.B12.T @ c1.Rc[:, cols]])
        m_r, m_c = len(c1.Jr) + len(c2.Jr), len(c1.Jc) + len(c2.Jc)
    if t.Sr is None:
        t.Sr, t.Sc = np.zeros((m_r, d)), np.zeros((m_c, d))
    elif t.Sr.shape[1] < d:
        t.Sr = np.hstack([t.Sr, np.zeros((m_r, d - t.Sr.shape[1]))])
        t.Sc = np.hstack([t.Sc, np.zeros((m_c, d - t.Sc.shape[1]))])
    t.Sr[:, cols] = sr
    t.Sc[:, cols] = sc
    if ctx["opts"].symmetric:
        t.Sc = t.Sr


def _reduce_local_samples(ctx, t, cols):
    """ReduceLocalSamples (Algorithm 2): tau.R^r = V^* [..], tau.R^c = U^* [..]
    and the global skeleton index sets tau.I^r, tau.I^c."""
    nodes, R = ctx["nodes"], ctx["R"]
    d = ctx["d"]
    if t.is_leaf:
        xr = xc = R[t.I, cols]
        Ibase_r = Ibase_c = t.I
    else:
        c1, c2 = nodes[t.children[0]], nodes[t.children[1]]
        xr = np.vstack([c1.Rr[:, cols], c2.Rr[:, cols]])
        xc = np.vstack([c1.Rc[:, cols], c2.Rc[:, cols]])
        Ibase_r = np.concatenate([c1.Ir, c2.Ir])
        Ibase_c = np.concatenate([c1.Ic, c2.Ic])
    if t.Rr is None:
        t.Rr, t.Rc = np.zeros((len(t.Jc), d)), np.zeros((len(t.Jr), d))
    elif t.Rr.shape[1] < d:
        t.Rr = np.hstack([t.Rr, np.zeros((t.Rr.shape[0], d - t.Rr.shape[1]))])
        t.Rc = np.hstack([t.Rc, np.zeros((t.Rc.shape[0], d - t.Rc.shape[1]))])
    t.Rr[:, cols] = t.V.T @ xr
    if ctx["opts"].symmetric:
        t.Rc = t.Rr
    else:
        t.Rc[:, cols] = t.U.T @ xc
    t.Ir = Ibase_r[t.Jr]
    t.Ic = Ibase_c[t.Jc]


def _hankel_sizes(ctx, t):
    return t.size, ctx["A"].n - t.size


def _node_sufficient(ctx, t) -> bool:
    """Strategy test plus the ID of both local samples (the try-block of
    Algorithm 3).  Returns True when the node may be marked COMPRESSED."""
    opts = ctx["opts"]
    er, ea = _tols(opts, t.level)
    d = ctx["d"]
    sides = (t.Sr,) if opts.symmetric else (t.Sr, t.Sc)
    if opts.strategy == "doubling":
        mh, nh = _hankel_sizes(ctx, t)
        out = []
        for S in sides:
            m = S.shape[0]
            piv, Rf, k, stopped = qrcp(S[:, :d].T, hmt_rule(er, ea, d, mh, nh))
            if stopped:
                ok = k <= d - opts.p
            else:
                ok = k == m          # every row selected: exact (P9)
            if not ok:
                return False
            out.append((piv, Rf, k))
        _set_id(t, out * 2 if opts.symmetric else out, d)
        return True
    # Incrementing (Algorithm 5 applied to the node's samples, block by
    # block as they were drawn, P18)
    for side, S in ((("r", t.Sr),) if opts.symmetric else (("r", t.Sr), ("c", t.Sc))):
        st = t.inc.setdefault(side, dict(Q=np.zeros((S.shape[0], 0)), rho=None,
                                         tested=0, done=False))
        while not st["done"] and st["tested"] < d:
            end = min(b for b in ctx["bounds"] if b > st["tested"])
            blk = S[:, st["tested"]:end]
            st["tested"] = end
            if opts.criterion == "hmt":
                st["done"] = hmt_block_test(blk, st, ea, opts.hmt_alpha)
            else:
                st["done"] = incrementing_block_test(blk, st, er, ea)
        if st["done"]:
            st["tested"] = d
    if opts.symmetric:
        t.inc["c"] = t.inc["r"]
    if not (t.inc["r"]["done"] and t.inc["c"]["done"]):
        return False
    out = []
    for S in sides:
        piv, Rf, k, _ = qrcp(S[:, :d].T, plain_rule(0.0 if opts.criterion == "hmt" else er, ea))
        out.append((piv, Rf, k))
    _set_id(t, out * 2 if opts.symmetric else out, d)
    return True


def incrementing_block_test(Sk: np.ndarray, st: dict, er: float, ea: float) -> bool:
    """One step of Algorithm 5 on the new block S_k (m x b) with the side's
    accumulated orthonormal basis Q: iterated block Gram-Schmidt, the four
    tests of eq. stopping_criteria, and on failure Q <- [Q Q_k]."""
    Q = st["Q"]
    m, b = Sk.shape
    Sh = Sk.copy()
    if Q.shape[1]:
        Sh = Sh - Q @ (Q.T @ Sh)
        Sh = Sh - Q @ (Q.T @ Sh)
    nS = np.linalg.norm(Sk)
    nSh = np.linalg.norm(Sh)
    if b == 0:
        return False
    if nS == 0.0 or nSh < er * nS or nSh / math.sqrt(b) < ea:
        return True
    Qk, Rk = np.linalg.qr(Sh)
    dg = np.abs(np.diag(Rk))
    if st["rho"] is None:
        st["rho"] = float(dg[0])
    mn = float(dg.min())
    if mn < ea or mn < er * st["rho"]:
        return True
    room = m - Q.shape[1]
    st["Q"] = np.hstack([Q, Qk[:, :min(b, room)]])
    return st["Q"].shape[1] >= m


def hmt_estimate(Y: np.ndarray, alpha: float) -> float:
    """The right-hand side of Lemma 4.1 (eq. HMT_err_bound): for Y = B W with
    W of p independent standard Gaussian columns, alpha sqrt(2/pi) times the
    largest column 2-norm of Y bounds |B|_2 except with probability alpha^-p."""
    if Y.shape[1] == 0:
        return 0.0
    return alpha * math.sqrt(2.0 / math.pi) * float(np.max(np.linalg.norm(Y, axis=0)))


def hmt_block_test(Sk: np.ndarray, st: dict, ea: float, alpha: float) -> bool:
    """Incrementing step with the HMT criterion (eq. HMT_IQQH, P22) on the
    new block S_k (m x b): the part of S_k outside span(Q), by the same
    iterated block Gram-Schmidt as Algorithm 5, gives the estimate of
    Lemma 4.1; the block is sufficient when the estimate is <= eps_a,
    otherwise its orthonormal basis joins Q."""
    Q = st["Q"]
    m, b = Sk.shape
    if b == 0:
        return False
    Sh = Sk.copy()
    if Q.shape[1]:
        Sh = Sh - Q @ (Q.T @ Sh)
        Sh = Sh - Q @ (Q.T @ Sh)
    if hmt_estimate(Sh, alpha) <= ea:
        return True
    Qk, _ = np.linalg.qr(Sh)
    room = m - Q.shape[1]
    st["Q"] = np.hstack([Q, Qk[:, :min(b, room)]])
    return st["Q"].shape[1] >= m


def _set_id(t, out, d):
    t.d_id = d
    (pr, Rr_, kr), (pc, Rc_, kc) = out
    t.Jr, t.Xr, t.U = interpolative(pr, Rr_, kr)
    t.Jc, t.Xc, t.V = interpolative(pc, Rc_, kc)
    t.piv_r, t.piv_c = pr, pc
