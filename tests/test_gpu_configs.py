"""The five workload configurations at their full sizes, in the launch
shapes the benchmark uses.  The oracle cannot compress these sizes, so the
checks are on outputs it computes one at a time, or on properties that hold
at any size:

* sampled rows of the off-diagonal samples (A - D^(L)) R  (eq. sample_off_diag)
  against the oracle's entries, element by element;
* convergence, and the product H x against the oracle's A x on sampled rows
  (the error of the compressed matrix, eq. nestedUV);
* the interpolative decomposition of sampled leaves: A(I, C) = U A(I(J), C)
  on sampled columns C outside the leaf (eq. ID), and U(J, :) = I;
* the mixed forms against the FP64 form of the same compression: ranks within
  the noise band, errors of the same size.
"""
from __future__ import annotations

import numpy as np
import pytest

import gpu_util as gu
import workloads as w
from oracle import hss as ohss
from oracle.tree import halving_tree

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    if not _t.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1810_04125_gb300 import build
    build.build()
    return _t


@pytest.fixture(scope="module")
def hss(torch):
    from paper_1810_04125_gb300 import hss as h
    return h

STRAT = {"doubling": 0, "incrementing": 1}


def _prepared(wl):
    src = wl.source
    if wl.needs_rcb:
        from paper_1810_04125_gb300 import hss
        src = src.permuted(hss.hss_rcb_order(src.points, wl.leaf))
    return src


def _dense_on_device(src):
    """A point-kernel source as a dense FP64 matrix built on the device (the
    form the benchmark compresses), column-major, from the same points."""
    import torch
    X = torch.from_numpy(src.points).to(gu.dev())
    n = src.n
    A = torch.empty((n, n), dtype=torch.float64, device=gu.dev())   # row j of this = column j of A
    for j0 in range(0, n, 1024):
        Xj = X[j0:j0 + 1024]
        r2 = torch.zeros((Xj.shape[0], n), dtype=torch.float64, device=gu.dev())
        for c in range(X.shape[1]):
            r2 += (Xj[:, c:c + 1] - X[:, c][None, :]) ** 2
        A[j0:j0 + 1024] = torch.exp(-r2 / (2.0 * src.p0 * src.p0))
    A.diagonal().add_(src.p1)
    return A.t()


def _device(src, dense):
    from paper_1810_04125_gb300 import hss
    if dense:
        A = _dense_on_device(src)
        s = hss.dense_source(A)
        s._keep = A
        return s
    return gu.device_source(src)


def _compress(wl, dsrc, prec):
    from paper_1810_04125_gb300 import hss
    o = hss.make_opts(wl.leaf, wl.rtol, wl.atol, wl.d0, wl.dd, wl.d_max, STRAT[wl.strategy],
                      gu.PREC[prec], wl.p, wl.seed)
    return hss.hss_compress(dsrc, o)


def _sampled_rows_check(src, dsrc, leaf, prec, rng, ncols=32, nrows=48):
    """(A - D^(L)) R on sampled rows, element by element."""
    import torch
    from paper_1810_04125_gb300 import hss
    n = src.n
    R = w.gaussian_matrix(17, n, 0, ncols)
    if prec == "tf32x2":
        R = w.round_to_tf32(R)
    elif prec == "bf16x3":
        R = w.round_to_bf16(R)
    Sr = torch.full((n, ncols), float("nan"), dtype=torch.float64, device=gu.dev())
    Sc = torch.full((n, ncols), float("nan"), dtype=torch.float64, device=gu.dev())
    hss.hss_sample_offdiag(dsrc, leaf, gu.PREC[prec], gu.col_major(R), Sr, Sc)
    torch.cuda.synchronize()
    rows = np.sort(rng.choice(n, nrows, replace=False))
    smp = ohss._Sampler(src)
    leaves = [t for t in halving_tree(n, leaf) if t.is_leaf]
    lo = np.array([t.I[0] for t in leaves])
    ref_r, ref_c = np.zeros((nrows, ncols)), np.zeros((nrows, ncols))
    bnd_r, bnd_c = np.zeros((nrows, ncols)), np.zeros((nrows, ncols))
    for a in range(0, n, 8192):
        J = np.arange(a, min(n, a + 8192))
        Er = smp.entries(rows, J)
        Ec = smp.entries(J, rows).T
        for q, i in enumerate(rows):      # the leaf block of row i is not sampled
            t = leaves[np.searchsorted(lo, i, side="right") - 1]
            inside = (J >= t.I[0]) & (J <= t.I[-1])
            Er[q, inside] = 0.0
            Ec[q, inside] = 0.0
        ref_r += Er @ R[J]
        ref_c += Ec @ R[J]
        bnd_r += np.abs(Er) @ np.abs(R[J])
        bnd_c += np.abs(Ec) @ np.abs(R[J])
    rel = 1e-13 if prec == "fp64" else 2.0 ** -21 + n * 2.0 ** -24
    for got, ref, bnd in ((Sr, ref_r, bnd_r), (Sc, ref_c, bnd_c)):
        g = got.cpu().numpy()[rows]
        assert np.all(np.isfinite(g))
        assert np.all(np.abs(g - ref) <= rel * bnd + 1e-300)
        if prec != "fp64":
            assert np.linalg.norm(g - ref) <= 5e-7 * np.linalg.norm(ref)


def _product_error(H, src, rng, nrows=96):
    """||(H x - A x)(rows)|| / ||(A x)(rows)|| for a Gaussian x."""
    import torch
    from paper_1810_04125_gb300 import hss
    n = src.n
    x = rng.standard_normal(n)
    X = torch.from_numpy(x).to(gu.dev()).reshape(1, n).t()
    Y = torch.empty((1, n), dtype=torch.float64, device=gu.dev()).t()
    hss.hss_matvec(H, X, Y)
    torch.cuda.synchronize()
    y = Y.cpu().numpy()[:, 0]
    rows = np.sort(rng.choice(n, nrows, replace=False))
    smp = ohss._Sampler(src)
    ex = np.zeros(nrows)
    for a in range(0, n, 8192):
        J = np.arange(a, min(n, a + 8192))
        ex += smp.entries(rows, J) @ x[J]
    return float(np.linalg.norm(y[rows] - ex) / np.linalg.norm(ex))


def _leaf_id_check(H, src, leaf, rtol, rng, nleaves=3, ncols=256):
    """A(I, C) = U A(I(J), C) on sampled columns outside the leaf."""
    n = src.n
    nodes = halving_tree(n, leaf)
    leaves = [t for t in nodes if t.is_leaf]
    level = max(t.level for t in leaves)
    smp = ohss._Sampler(src)
    for t in [leaves[i] for i in rng.choice(len(leaves), nleaves, replace=False)]:
        e = H.export_node(t.idx)
        piv, X = e["Pr"], e["Xr"]
        k, m = X.shape[0], piv.size
        U = np.zeros((m, k))
        U[piv[:k], np.arange(k)] = 1.0
        U[piv[k:], :] = X.T
        assert np.array_equal(U[piv[:k]], np.eye(k))
        outside = np.setdiff1d(np.arange(n), t.I)
        C = np.sort(rng.choice(outside, min(ncols, outside.size), replace=False))
        Ablk = smp.entries(t.I, C)
        err = np.linalg.norm(Ablk - U @ Ablk[piv[:k]]) / np.linalg.norm(Ablk)
        # the ID of the sample at eps / level, with room for the randomized
        # estimate and the (1 + |X|) growth of an interpolative decomposition
        assert err <= 100.0 * rtol / level, (t.idx, err)


# (name, workload, precisions, dense A on the device)
CONFIGS = [
    ("toeplitz_inv_n1024", w.workload_toeplitz_1024, ["fp64", "tf32x2"], False),
    ("gauss8_n16384_dense", w.workload_gauss8_16384, ["tf32x2", "fp64"], True),
    ("laplace_sphere_n32768", w.workload_laplace_sphere, ["bf16x3", "fp64"], False),
    ("toeplitz_cos_n131072", w.workload_toeplitz_cos, ["tf32x2"], False),
]


@pytest.mark.parametrize("name,mk,precs,dense", CONFIGS, ids=[c[0] for c in CONFIGS])
def test_full_size_config(hss, torch, name, mk, precs, dense):
    wl = mk()
    src = _prepared(wl)
    dsrc = _device(src, dense)
    rng = np.random.default_rng(11)
    _sampled_rows_check(src, dsrc, wl.leaf, precs[0], rng)
    results = {}
    for prec in precs:
        H = _compress(wl, dsrc, prec)
        st = H.stats()
        assert st.converged == 1
        err = _product_error(H, src, np.random.default_rng(3))
        # the compressed matrix meets the tolerance up to the accumulation
        # over the levels of the tree
        assert err <= 10.0 * wl.rtol, (prec, err)
        _leaf_id_check(H, src, wl.leaf, wl.rtol, np.random.default_rng(5))
        results[prec] = (st.d_final, max(st.max_rank_r, st.max_rank_c), err)
        del H
    if len(precs) == 2:
        # the mixed form (precs[0]) is not less accurate than the FP64 form;
        # under Incrementing its sampling noise can make it draw more
        # columns than the FP64 form and so end with a smaller error, which
        # is no fault of it
        (d0, r0, e0), (d1, r1, e1) = results[precs[0]], results[precs[1]]
        assert abs(r0 - r1) <= max(2, 0.02 * r1), results
        assert e0 <= 1.5 * e1 + 1e-12, results


def test_batch_members_full_size(hss, torch):
    """Members of the 64-matrix batch (sizes log-uniform in [2048, 16384]):
    the smallest and the largest of each kind, Doubling from d0 = 64."""
    sizes = w.batch_sizes()
    picks = []
    for kind in ("toeplitz", "gauss3"):
        idx = range(0, 32) if kind == "toeplitz" else range(32, 64)
        ns = sorted(int(sizes[i]) for i in idx)
        picks += [(kind, ns[0]), (kind, ns[-1])]
    for kind, n in picks:
        if kind == "toeplitz":
            src = w.toeplitz_power(n, 1.5)
        else:
            from paper_1810_04125_gb300 import hss as H_
            pts = w.uniform_points(n, 3, seed=n)
            src = w.gaussian_kernel(pts[H_.hss_rcb_order(pts, 128)], 1.0, 0.0)
        wl = w.Workload(f"{kind}_{n}", src, leaf=128, rtol=1e-5, atol=1e-8, strategy="doubling",
                        d0=64, dd=64, d_max=min(n, 4096), precision="tf32x2")
        H = _compress(wl, gu.device_source(src), "tf32x2")
        assert H.stats().converged == 1
        err = _product_error(H, src, np.random.default_rng(7))
        assert err <= 10.0 * wl.rtol, (kind, n, err)
        del H
