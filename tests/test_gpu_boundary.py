"""The partially matrix-free boundary of section 3.1 through the C ABI:
products with H and H^T, entries H(I, J) of a compressed handle, a matrix
known only through a user product and a user element extraction (no entries
on the device), a compressed HSS product, and the partial result of a
compression that reaches d_max."""
import numpy as np
import pytest

import workloads as w
from oracle import apply
from oracle.hss import Options, compress
from oracle.operator import toeplitz_product
from oracle.tree import halving_tree

import gpu_util as gu

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


def _dense_T(H, n, torch, hss):
    """H^T through the transposed product applied to the identity."""
    X = torch.eye(n, dtype=torch.float64, device=gu.dev()).t()
    Y = torch.empty((n, n), dtype=torch.float64, device=gu.dev()).t()
    hss.hss_matvec(H, X, Y, transpose=True)
    torch.cuda.synchronize()
    return Y.cpu().numpy()


def _entries(H, I, J, torch, hss):
    Id = torch.from_numpy(np.asarray(I, dtype=np.int32)).to(gu.dev())
    Jd = torch.from_numpy(np.asarray(J, dtype=np.int32)).to(gu.dev())
    out = torch.full((len(J), len(I)), float("nan"), dtype=torch.float64, device=gu.dev()).t()
    hss.hss_get_entries(H, Id, Jd, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


CASES = [
    ("nonsym_toeplitz", lambda: w.toeplitz_nonsymmetric(1000),
     Options(leaf=64, rtol=1e-8, atol=1e-14, d0=32, dd=16, d_max=512)),
    ("udv_dbl", lambda: w.dense_source(w.udv_matrix(777, 40, seed=5)),
     Options(leaf=50, rtol=1e-8, atol=1e-14, d0=16, dd=16, d_max=512, strategy="doubling")),
    ("laplace_ragged", lambda: w.laplace_kernel(w.fibonacci_sphere(901)[
        __import__("oracle").tree.rcb_order(w.fibonacci_sphere(901), 40)]),
     Options(leaf=40, rtol=1e-6, atol=1e-12, d0=32, dd=16, d_max=600)),
]


@pytest.mark.parametrize("name,mk,o", CASES, ids=[c[0] for c in CASES])
def test_transposed_product_and_entries(hss, torch, name, mk, o):
    """H^T X equals the transpose of the expansion; H(I, J) from the nested
    bases equals the expansion's entries (same leaf, siblings, distant
    leaves, repeated and unsorted indices)."""
    src = mk()
    n = src.n
    H = gu.gpu_compress(src, w.gaussian_matrix(3, n, 0, o.d_max), o)
    Hd = gu.gpu_dense(H, n)
    scale = np.abs(Hd).max()
    np.testing.assert_allclose(_dense_T(H, n, torch, hss), Hd.T, rtol=0, atol=1e-13 * scale)
    rng = np.random.default_rng(1)
    I = np.concatenate([rng.integers(0, n, 300), [0, n - 1, 5, 5, n // 2]])
    J = np.concatenate([rng.integers(0, n, 200), [n - 1, 0, 6, 7, n // 2 + 1]])
    np.testing.assert_allclose(_entries(H, I, J, torch, hss), Hd[np.ix_(I, J)], rtol=0, atol=1e-13 * scale)
    # a whole block row and the full matrix
    np.testing.assert_allclose(_entries(H, np.arange(n), np.arange(n), torch, hss), Hd, rtol=0,
                               atol=1e-13 * scale)
    with pytest.raises(hss.HSSError) as ei:
        _entries(H, [0, n], [1], torch, hss)
    assert ei.value.status == hss.HSS_ERR_ARG


def _toeplitz_extractor(col, row, torch):
    calls = []

    def fn(blocks, stream):
        calls.append(len(blocks))
        for I, J, out in blocks:
            d = I.long()[:, None] - J.long()[None, :]
            out.copy_(torch.where(d >= 0, col[d.clamp(min=0)], row[(-d).clamp(min=0)]))

    fn.calls = calls
    return fn


@pytest.mark.parametrize("n,leaf,strategy,sym", [(2000, 100, "incrementing", False),
                                                 (1537, 64, "doubling", False),
                                                 (4096, 128, "incrementing", True)])
def test_product_and_extraction_only(hss, torch, n, leaf, strategy, sym):
    """A Toeplitz matrix known only through an FFT product (sampling) and an
    element extraction routine (generators): no entries of A on the device.
    Same passes, ranks (within the tie rule) and error as the oracle
    sampling through its own FFT product and reading the entries."""
    src = w.toeplitz_cos(n) if sym else w.toeplitz_nonsymmetric(n)
    o = Options(leaf=leaf, rtol=1e-6, atol=1e-12, d0=32, dd=32, d_max=1024, strategy=strategy, symmetric=sym)
    R = w.gaussian_matrix(9, n, 0, o.d_max)
    ref = compress(src, R, o, product=lambda X, tr: toeplitz_product(src.col, src.row, X, tr))
    col = torch.from_numpy(src.col).to(gu.dev())
    row = torch.from_numpy(src.row).to(gu.dev())
    ext = _toeplitz_extractor(col, row, torch)
    op = hss.make_operator(gu.toeplitz_fft_operator(col, row))
    s = hss.extract_source(n, ext)
    opts = hss.make_opts(leaf, o.rtol, o.atol, o.d0, o.dd, o.d_max, gu.STRAT[strategy], R=gu.col_major(R),
                         symmetric=int(sym), op=op)
    H = hss.hss_compress(s, opts)
    st = H.stats()
    assert st.converged and ref.converged
    assert (st.d_final, st.n_adapt) == (ref.d_final, ref.n_adapt)
    assert not gu.compare_with_oracle(H, ref, o, n)
    A = src.to_dense()
    assert gu.rel_err(A, gu.gpu_dense(H, n)) <= 1.1 * apply.rel_error(ref, A) + 1e-15
    # the leaf blocks in one call, then one call per level with B blocks
    assert ext.calls[0] == len([t for t in halving_tree(n, leaf) if not t.children])
    assert len(ext.calls) <= H.stats().levels + 1
    # an extraction routine that raises stops the compression with a status
    def bad(blocks, stream):
        raise RuntimeError("no entries today")
    with pytest.raises(hss.HSSError) as ei:
        hss.hss_compress(hss.extract_source(n, bad), opts)
    assert ei.value.status == hss.HSS_ERR_OPERATOR


def test_hss_product_compressed(hss, torch):
    """HSS times HSS (section 3.1: a fast multiply from hierarchical
    matrices): C = H1 H2 sampled as H1 (H2 R) and H2^T (H1^T R) through
    hss_matvec, its entries C(I, J) = H1(I, :) H2(:, J) from hss_get_entries;
    against the oracle's compression of the dense product on the same R."""
    n, leaf = 2048, 128
    P = w.uniform_points(n, 3, seed=4)
    P = P[__import__("oracle").tree.rcb_order(P, leaf)]
    o1 = Options(leaf=leaf, rtol=1e-10, atol=1e-14, d0=64, dd=32, d_max=1024)
    H1 = gu.gpu_compress(w.gaussian_kernel(P, 0.5, 1.0), w.gaussian_matrix(1, n, 0, 1024), o1)
    H2 = gu.gpu_compress(w.toeplitz_nonsymmetric(n), w.gaussian_matrix(2, n, 0, 1024), o1)
    C = gu.gpu_dense(H1, n) @ gu.gpu_dense(H2, n)
    allidx = torch.arange(n, dtype=torch.int32, device=gu.dev())

    def prod(trans, R, S, stream):
        T = torch.empty((R.shape[1], n), dtype=torch.float64, device=gu.dev()).t()
        first, second = (H1, H2) if trans else (H2, H1)     # C^T R = H2^T (H1^T R)
        hss.hss_matvec(first, R, T, stream=stream, transpose=bool(trans))
        hss.hss_matvec(second, T, S, stream=stream, transpose=bool(trans))

    def ext(blocks, stream):
        for I, J, out in blocks:
            rows = torch.empty((n, I.numel()), dtype=torch.float64, device=gu.dev()).t()
            cols = torch.empty((J.numel(), n), dtype=torch.float64, device=gu.dev()).t()
            hss.hss_get_entries(H1, I, allidx, rows, stream=stream)
            hss.hss_get_entries(H2, allidx, J, cols, stream=stream)
            out.copy_(rows @ cols)

    o = Options(leaf=leaf, rtol=1e-6, atol=1e-12, d0=64, dd=32, d_max=1024)
    R = w.gaussian_matrix(6, n, 0, o.d_max)
    ref = compress(w.dense_source(C), R, o)
    opts = hss.make_opts(leaf, o.rtol, o.atol, o.d0, o.dd, o.d_max, hss.HSS_INCREMENTING, R=gu.col_major(R),
                         op=hss.make_operator(prod))
    H = hss.hss_compress(hss.extract_source(n, ext), opts)
    st = H.stats()
    assert st.converged and ref.converged and (st.d_final, st.n_adapt) == (ref.d_final, ref.n_adapt)
    assert not gu.compare_with_oracle(H, ref, o, n)
    assert gu.rel_err(C, gu.gpu_dense(H, n)) <= 1.1 * apply.rel_error(ref, C) + 1e-15


PARTIAL = [
    # the level-1 sides (32 rows, rank 20) fail at d = 20, everything below compresses
    ("synthetic_inc", lambda: w.synthetic_hss(1024, 64, {4: 8, 3: 12, 2: 16, 1: 20}, seed=3),
     Options(leaf=64, rtol=1e-10, atol=1e-14, d0=8, dd=4, d_max=20)),
    ("synthetic_dbl", lambda: w.synthetic_hss(1024, 64, {4: 8, 3: 12, 2: 16, 1: 20}, seed=3),
     Options(leaf=64, rtol=1e-10, atol=1e-14, d0=5, dd=4, d_max=20, strategy="doubling", p=2)),
    # no leaf passes: every block outside the leaves kept dense
    ("udv_inc", lambda: w.udv_matrix(1000, 90, seed=2),
     Options(leaf=64, rtol=1e-10, atol=1e-15, d0=16, dd=8, d_max=48)),
]


@pytest.mark.parametrize("name,mk,o", PARTIAL, ids=[c[0] for c in PARTIAL])
def test_not_converged_partial_result(hss, torch, name, mk, o):
    """A compression that reaches d_max returns a usable partial result: the
    node states of the oracle's last pass, the blocks between the children
    of every uncompressed node (and its leaves' D) equal to A exactly, the
    compressed subtrees as accurate as their tolerance, and the products,
    H^T and the entries consistent with the expansion."""
    A = mk()
    n, leaf = A.shape[0], o.leaf
    R = w.gaussian_matrix(0, n, 0, o.d_max)
    ref = compress(w.dense_source(A), R, o)
    assert not ref.converged
    H = gu.gpu_compress(w.dense_source(A), R, o, allow_not_converged=True)
    st = H.stats()
    assert st.converged == 0 and st.d_final == ref.d_final
    states = [H.node(i).state for i in range(st.n_nodes)]
    assert states == [{"U": 0, "PC": 1, "C": 2}[s] for s in ref.passes[-1]["states"]]
    Hd = gu.gpu_dense(H, n)
    nodes = halving_tree(n, leaf)
    for t in nodes:
        if t.children and states[t.idx] != 2:
            a, b = (nodes[c] for c in t.children)
            assert np.array_equal(Hd[np.ix_(a.I, b.I)], A[np.ix_(a.I, b.I)])
            assert np.array_equal(Hd[np.ix_(b.I, a.I)], A[np.ix_(b.I, a.I)])
        if not t.children and states[t.idx] != 2:
            assert np.array_equal(Hd[np.ix_(t.I, t.I)], A[np.ix_(t.I, t.I)])
    # the compressed subtrees: their diagonal blocks within the tolerance
    for t in nodes:
        if states[t.idx] == 2 and t.parent >= 0 and states[t.parent] != 2:
            blk = np.ix_(t.I, t.I)
            assert np.linalg.norm(Hd[blk] - A[blk]) <= 1e-8 * np.linalg.norm(A[blk]), t.idx
    np.testing.assert_allclose(_dense_T(H, n, torch, hss), Hd.T, rtol=0, atol=1e-13 * np.abs(Hd).max())
    I = np.random.default_rng(3).integers(0, n, 150)
    J = np.random.default_rng(4).integers(0, n, 170)
    np.testing.assert_allclose(_entries(H, I, J, torch, hss), Hd[np.ix_(I, J)], rtol=0,
                               atol=1e-13 * np.abs(Hd).max())
