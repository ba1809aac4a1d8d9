"""The two non-adaptive modes of the paper's adaptivity-cost comparison
(section 4.3.2, Table 4) on the GPU against the oracle: the hard restart
(attempts at d0, 2 d0, 4 d0, ... from scratch) with the same number of
restarts, final d, ranks under the tie rule and error <= 1.1x the oracle's;
the known-rank mode (d0 = d_max) converging or failing as the oracle does."""
from __future__ import annotations

import numpy as np
import pytest

import gpu_util as gu
import workloads as w
from oracle import apply
from oracle.hss import Options, compress, compress_hard_restart

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


RANKS = {4: 8, 3: 12, 2: 16, 1: 20}


@pytest.mark.parametrize("d0", [3, 8, 21])
def test_hard_restart_exact_ranks(hss, torch, d0):
    """Closed form on the synthetic matrix with ranks 8/12/16/20: restarts
    until d >= 21, exact ranks."""
    n, leaf = 1024, 64
    A = w.synthetic_hss(n, leaf, RANKS, seed=3)
    R = w.gaussian_matrix(5, n, 0, 512)
    o = Options(leaf=leaf, rtol=1e-10, atol=1e-14, d0=d0, dd=8, d_max=512)
    H, k = gu.gpu_compress_restart(w.dense_source(A), R, o)
    want = 0
    while d0 * 2 ** want < 21:
        want += 1
    st = H.stats()
    assert st.converged == 1 and k == want and st.d_final == d0 * 2 ** want and st.n_adapt == 0
    for i, (kr, kc) in H.ranks().items():
        assert kr == kc == RANKS[H.node(i).level], (i, kr, kc)
    assert gu.rel_err(A, gu.gpu_dense(H, n)) < 1e-12


CASES = [
    ("udv1000_inc", lambda: w.dense_source(w.udv_matrix(1000, 60, seed=3)),
     Options(leaf=64, rtol=1e-8, atol=1e-14, d0=16, dd=16, d_max=1000)),
    ("toeplitz1024_dbl", lambda: w.toeplitz_inverse_distance(1024),
     Options(leaf=64, rtol=1e-6, atol=1e-12, d0=16, dd=16, d_max=1024, strategy="doubling")),
    ("udv1024_hmt", lambda: w.dense_source(w.udv_matrix(1024, 200, seed=1)),
     Options(leaf=128, rtol=0.0, atol=1e-10, d0=64, dd=64, d_max=1024, criterion="hmt")),
]


@pytest.mark.parametrize("name,mk,o", CASES, ids=[c[0] for c in CASES])
def test_hard_restart_parity(hss, torch, name, mk, o):
    src = mk()
    n = src.n
    R = w.gaussian_matrix(7, n, 0, o.d_max)
    ref, k_ref = compress_hard_restart(src, R, o)
    H, k = gu.gpu_compress_restart(src, R, o)
    st = H.stats()
    assert st.converged == 1 and ref.converged
    assert k == k_ref and st.d_final == ref.d_final, (k, k_ref, st.d_final, ref.d_final)
    bad = gu.compare_with_oracle(H, ref, o, n)
    assert not bad, bad
    A = src.to_dense()
    err_g = gu.rel_err(A, gu.gpu_dense(H, n))
    assert err_g <= 1.1 * apply.rel_error(ref, A) + 1e-15


def test_hard_restart_generated_R(hss, torch):
    """With R generated on the device every attempt uses the leading columns
    of the same generated matrix: the result equals one pass at the final d."""
    src = w.toeplitz_inverse_distance(1024)
    o = Options(leaf=64, rtol=1e-8, atol=1e-14, d0=8, dd=8, d_max=1024)
    H, k = gu.gpu_compress_restart(src, None, o, pass_R=False, seed=11)
    d = H.stats().d_final
    assert H.stats().converged == 1 and d == 8 * 2 ** k and k >= 1
    o1 = Options(leaf=64, rtol=1e-8, atol=1e-14, d0=d, dd=8, d_max=d)
    H1 = gu.gpu_compress(src, None, o1, pass_R=False, seed=11)
    assert H1.ranks() == H.ranks()
    n = src.n
    np.testing.assert_array_equal(gu.gpu_dense(H, n), gu.gpu_dense(H1, n))


def test_known_rank_mode(hss, torch):
    """d0 = d_max: one pass; NOT_CONVERGED with the oracle's node states when
    the fixed number of vectors is too small, converged with no growth when
    it is large enough."""
    n, leaf = 1024, 64
    A = w.synthetic_hss(n, leaf, RANKS, seed=3)
    R = w.gaussian_matrix(5, n, 0, 512)
    for d, ok in ((20, False), (21, True)):
        o = Options(leaf=leaf, rtol=1e-10, atol=1e-14, d0=d, dd=8, d_max=d)
        ref = compress(w.dense_source(A), R, o)
        H = gu.gpu_compress(w.dense_source(A), R, o, allow_not_converged=True)
        st = H.stats()
        assert bool(st.converged) == ok == ref.converged and st.n_adapt == 0 and st.d_final == d
        states = [H.node(t.idx).state for t in ref.nodes]
        want = [{"U": 0, "PC": 1, "C": 2}[t.state] for t in ref.nodes]
        assert states == want
