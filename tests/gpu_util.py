"""Helpers shared by the GPU tests: marshalling of the seeded inputs to the
C ABI and comparison of a GPU result with the oracle."""
from __future__ import annotations

import numpy as np

import workloads as w
from oracle import apply, qrcp
from oracle.tree import halving_tree


def dev():
    import torch
    return torch.device("cuda:0")


def col_major(A: np.ndarray):
    """Device tensor with A's entries stored column-major (stride(0) == 1)."""
    import torch
    return torch.from_numpy(np.ascontiguousarray(np.asarray(A, dtype=np.float64).T)).to(dev()).t()


def device_source(src: w.Source):
    from paper_1810_04125_gb300 import hss
    if src.kind == w.SRC_DENSE:
        return hss.dense_source(col_major(src.dense))
    if src.kind == w.SRC_TOEPLITZ:
        import torch
        return hss.toeplitz_source(torch.from_numpy(src.col).to(dev()),
                                   torch.from_numpy(src.row).to(dev()))
    return hss.points_source(src.kind, col_major(src.points), src.p0, src.p1)


STRAT = {"incrementing": 1, "doubling": 0}
PREC = {"fp64": 0, "tf32x2": 1, "bf16x3": 2}


def toeplitz_fft_operator(col, row):
    """A user sampling operator for a Toeplitz matrix (device tensors col,
    row): S = T R through the FFT of its circulant embedding of size 2n
    (torch.fft on the library's stream), the GPU counterpart of
    oracle.operator.toeplitz_product."""
    import torch
    n = col.numel()

    def spectrum(c_, r_):
        c = torch.zeros(2 * n, dtype=torch.float64, device=col.device)
        c[:n] = c_
        c[n + 1:] = r_[1:].flip(0)
        return torch.fft.rfft(c)

    F, FT = spectrum(col, row), spectrum(row, col)
    torch.cuda.synchronize()
    calls = []

    def fn(trans, R, S, stream):
        calls.append(trans)
        Y = torch.zeros((2 * n, R.shape[1]), dtype=torch.float64, device=R.device)
        Y[:n] = R
        Z = torch.fft.irfft((FT if trans else F)[:, None] * torch.fft.rfft(Y, dim=0), n=2 * n, dim=0)
        S.copy_(Z[:n])

    fn.calls = calls
    return fn


def gpu_compress(src, R, o, precision="fp64", pass_R=True, seed=0, allow_not_converged=False, op=None):
    from paper_1810_04125_gb300 import hss
    s = device_source(src)
    Rd = col_major(R) if pass_R else None
    opts = hss.make_opts(o.leaf, o.rtol, o.atol, o.d0, o.dd, o.d_max, STRAT[o.strategy],
                         PREC[precision], o.p, seed, Rd, int(o.level_tol_scaling),
                         int(getattr(o, "symmetric", False)),
                         1 if getattr(o, "criterion", "new") == "hmt" else 0, getattr(o, "hmt_alpha", 10.0),
                         op=op)
    return hss.hss_compress(s, opts, allow_not_converged=allow_not_converged)


def gpu_compress_restart(src, R, o, precision="fp64", pass_R=True, seed=0):
    """The hard-restart mode through the C ABI: (handle, restarts)."""
    from paper_1810_04125_gb300 import hss
    s = device_source(src)
    Rd = col_major(R) if pass_R else None
    opts = hss.make_opts(o.leaf, o.rtol, o.atol, o.d0, o.dd, o.d_max, STRAT[o.strategy],
                         PREC[precision], o.p, seed, Rd, int(o.level_tol_scaling),
                         int(getattr(o, "symmetric", False)),
                         1 if getattr(o, "criterion", "new") == "hmt" else 0, getattr(o, "hmt_alpha", 10.0))
    return hss.hss_compress_restart(s, opts, allow_not_converged=True)


def gpu_dense(H, n):
    import torch
    from paper_1810_04125_gb300 import hss
    X = torch.eye(n, dtype=torch.float64, device=dev()).t()
    Y = torch.empty((n, n), dtype=torch.float64, device=dev()).t()
    hss.hss_matvec(H, X, Y)
    torch.cuda.synchronize()
    return Y.cpu().numpy()


class _Res:
    def __init__(self, n, nodes):
        self.n, self.nodes = n, nodes


def expand_exported(H, n, leaf):
    """The GPU generators put into the oracle's node objects, so that the
    oracle's plain expansion (eq. nestedUV) can be applied to them."""
    nodes = halving_tree(n, leaf)
    for t in nodes:
        e = H.export_node(t.idx)
        if t.is_leaf:
            t.D = e["D"]
        if t.idx == 0:
            if not t.is_leaf:
                t.B12, t.B21 = e["B12"], e["B21"]
            continue
        for side in ("r", "c"):
            piv, X = e["P" + side], e["X" + side]
            k = X.shape[0]
            m = piv.size
            U = np.zeros((m, k))
            U[piv[:k], np.arange(k)] = 1.0
            U[piv[k:], :] = X.T
            setattr(t, "U" if side == "r" else "V", U)
            setattr(t, "J" + side, piv[:k])
            setattr(t, "I" + side, e["I" + side])
        if not t.is_leaf:
            t.B12, t.B21 = e["B12"], e["B21"]
    return _Res(n, nodes)


def node_tolerances(level, o):
    """(eps_r, eps_a) of a node's ID: level-scaled (P3); the HMT criterion's
    final RRQR knows eps_a only."""
    scale = 1.0 / level if o.level_tol_scaling else 1.0
    er, ea = o.rtol * scale, o.atol * scale
    if getattr(o, "criterion", "new") == "hmt":
        er = 0.0
    return er, ea


def rank_mismatch_allowed(t, side, o, d, k_a, k_b, n, band=0.1, noise=0.0):
    """Ranks may differ only where singular values of the node's sample lie
    within +-10% of the rank threshold, and by at most the number of such
    values (pivot order may legitimately diverge at near ties, which can move
    the rank across such a value but not further).  ``noise``: a bound on
    the error of the GPU's sample against the oracle's (mixed forms), which
    widens the band by Weyl's inequality."""
    S = (t.Sr if side == "r" else t.Sc)[:, :d]
    er, ea = node_tolerances(t.level, o)
    rule = "hmt" if o.strategy == "doubling" else "plain"
    return abs(k_a - k_b) <= qrcp.near_threshold_count(S, er, ea, rule, t.size, n - t.size, band, noise)


# tested bound of the mixed sampling error relative to the sample (Frobenius
# norm; test_gpu_mixed measures 0.4-1.8e-7 for TF32x2 and BF16x3)
MIXED_NOISE = 5e-7


def mixed_noise(src, R, ref, delta=MIXED_NOISE):
    """noise(t, side): a bound on the error of a node's local sample when the
    sampling product S = (A - D^(L)) R runs in a mixed form.  The sampling
    error enters the local samples only through the rows of the global
    sample at the node's sample rows (the merges subtract exactly formed
    terms), so it is bounded by delta times the norm of those rows."""
    A = src.to_dense()
    n = src.n
    for t in ref.nodes:
        if t.is_leaf:
            A[np.ix_(t.I, t.I)] = 0.0
    Sr = A @ R
    Sc = A.T @ R

    def noise(t, side):
        if t.is_leaf:
            rows = t.I
        else:
            c1, c2 = (ref.nodes[c] for c in t.children)
            rows = np.concatenate([c1.Ir, c2.Ir] if side == "r" else [c1.Ic, c2.Ic])
        G = Sr if side == "r" else Sc
        return delta * float(np.linalg.norm(G[rows, :t.d_id]))

    return noise


def _near_report(t, side, o, d, k_lo, k_hi, n):
    """sigma_j / thr and |R_jj| / thr of the oracle's sample around the two
    ranks (for the failure message)."""
    S = (t.Sr if side == "r" else t.Sc)[:, :d]
    er, ea = node_tolerances(t.level, o)
    _, Rf, _, _ = qrcp.qrcp(S.T, lambda j, r, r1: False)
    diag = np.abs(np.diag(Rf))
    sv = np.linalg.svd(S, compute_uv=False)
    r11 = float(np.max(np.linalg.norm(S, axis=1)))
    out = []
    for j in range(max(0, k_lo - 2), min(sv.size, k_hi + 2)):
        f = qrcp.hmt_factor(j + 1, d, t.size, n - t.size) if o.strategy == "doubling" else 1.0
        thr = max(ea, er * r11) / f
        out.append(f"{j + 1}:sv {sv[j] / thr:.3f} R {diag[j] / thr:.3f}")
    return " ".join(out)


def compare_with_oracle(H, ref, o, n, noise=None):
    """Ranks node by node; returns the list of unexplained mismatches.
    ``noise``: for a GPU result sampled in a mixed form, mixed_noise(...)."""
    bad = []
    gr = H.ranks()
    for t in ref.nodes[1:]:
        if t.Jr is None:
            continue
        kg = gr[t.idx]
        ko = (len(t.Jr), len(t.Jc))
        for s, a, b in (("r", kg[0], ko[0]), ("c", kg[1], ko[1])):
            if a != b and not rank_mismatch_allowed(t, s, o, t.d_id, a, b, n,
                                                    noise=noise(t, s) if noise else 0.0):
                bad.append((t.idx, s, a, b, _near_report(t, s, o, t.d_id, min(a, b), max(a, b), n)))
    return bad


def rel_err(A, H_dense):
    return float(np.linalg.norm(A - H_dense) / np.linalg.norm(A))
