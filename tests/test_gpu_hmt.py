"""The HMT stopping criterion (Lemma 4.1 in the form of eq. HMT_IQQH, an
alternative Incrementing test) on the GPU against the oracle's HMT option on
the same R: d_final and the number of adaptations equal, ranks under the tie
rule, error <= 1.1x the oracle's.  The cases cover both forms of the test
kernel (one CTA per node side where the sides outnumber the SMs, a group of
CTAs per side otherwise), the symmetric option, and a mixed-precision
compression against the FP64 one."""
from __future__ import annotations

import numpy as np
import pytest

import gpu_util as gu
import workloads as w
from oracle import apply
from oracle.hss import Options, compress
from oracle.tree import rcb_order

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


def _gauss(n, seed, h, leaf):
    pts = w.uniform_points(n, 3, seed=seed)
    return w.gaussian_kernel(pts[rcb_order(pts, leaf)], h, 0.0)


CASES = [
    ("udv1000_ragged", lambda: w.dense_source(w.udv_matrix(1000, 60, seed=3)),
     Options(leaf=64, rtol=0.0, atol=1e-8, d0=32, dd=16, d_max=1000, criterion="hmt")),
    ("toeplitz1024_adapt", lambda: w.toeplitz_inverse_distance(1024),
     Options(leaf=64, rtol=0.0, atol=1e-6, d0=16, dd=8, d_max=1024, criterion="hmt")),
    # 128 leaves: 256 node sides at the leaf level (one CTA per side)
    ("udv2048_leaf16", lambda: w.dense_source(w.udv_matrix(2048, 100, seed=5)),
     Options(leaf=16, rtol=0.0, atol=1e-8, d0=16, dd=16, d_max=1024, criterion="hmt")),
    ("gauss1200_symmetric", lambda: _gauss(1200, 3, 0.4, 64),
     Options(leaf=64, rtol=0.0, atol=1e-8, d0=32, dd=32, d_max=1024, criterion="hmt", symmetric=True)),
    ("udv1024_alpha2", lambda: w.dense_source(w.udv_matrix(1024, 200, seed=1)),
     Options(leaf=128, rtol=0.0, atol=1e-10, d0=128, dd=64, d_max=1024, criterion="hmt", hmt_alpha=2.0)),
]


@pytest.mark.parametrize("name,mk,o", CASES, ids=[c[0] for c in CASES])
def test_hmt_parity(hss, torch, name, mk, o):
    src = mk()
    n = src.n
    R = w.gaussian_matrix(7, n, 0, o.d_max)
    ref = compress(src, R, o)
    H = gu.gpu_compress(src, R, o)
    st = H.stats()
    assert st.converged == 1 and ref.converged
    assert st.d_final == ref.d_final and st.n_adapt == ref.n_adapt, (st.d_final, ref.d_final)
    bad = gu.compare_with_oracle(H, ref, o, n)
    assert not bad, bad
    A = src.to_dense()
    err_g = gu.rel_err(A, gu.gpu_dense(H, n))
    err_o = apply.rel_error(ref, A)
    assert err_g <= 1.1 * err_o + 1e-15, (err_g, err_o)


def test_hmt_against_new_criterion(hss, torch):
    """Table 3's comparison on the GPU: at the same absolute tolerance the
    HMT criterion takes at least as many samples as the new criterion with
    rtol = atol, with ranks at least as large and errors no larger."""
    n = 2048
    A = w.udv_matrix(n, 200, seed=1)
    src = w.dense_source(A)
    R = w.gaussian_matrix(1, n, 0, 1024)
    for tol in (1e-6, 1e-10):
        Hn = gu.gpu_compress(src, R, Options(leaf=128, rtol=tol, atol=tol, d0=128, dd=64, d_max=1024))
        Hh = gu.gpu_compress(src, R, Options(leaf=128, rtol=tol, atol=tol, d0=128, dd=64, d_max=1024,
                                             criterion="hmt"))
        sn, sh = Hn.stats(), Hh.stats()
        en, eh = gu.rel_err(A, gu.gpu_dense(Hn, n)), gu.rel_err(A, gu.gpu_dense(Hh, n))
        assert sh.d_final >= sn.d_final
        assert max(sh.max_rank_r, sh.max_rank_c) >= max(sn.max_rank_r, sn.max_rank_c)
        assert eh <= 1.01 * en and eh <= tol, (tol, en, eh)


def test_hmt_mixed_precision(hss, torch):
    """TF32x2 sampling with the HMT criterion against the FP64 form of the
    same compression: ranks within the noise band, errors of the same size."""
    src = w.toeplitz_cos(4096)
    n = src.n
    o = Options(leaf=256, rtol=0.0, atol=1e-4, d0=128, dd=64, d_max=1024, criterion="hmt")
    A = src.to_dense()
    out = {}
    for prec in ("fp64", "tf32x2"):
        H = gu.gpu_compress(src, None, o, precision=prec, pass_R=False, seed=3)
        st = H.stats()
        assert st.converged == 1
        out[prec] = (max(st.max_rank_r, st.max_rank_c), gu.rel_err(A, gu.gpu_dense(H, n)))
    (r64, e64), (r32, e32) = out["fp64"], out["tf32x2"]
    assert abs(r64 - r32) <= max(2, 0.02 * r64), out
    assert e32 <= 1.5 * e64 + 1e-12 and e64 <= 1.5 * e32 + 1e-12, out
