"""Sampling through a user operator (the partially matrix-free interface of
section 3.1): a Toeplitz matrix sampled by the FFT of its circulant
embedding (torch.fft on the library's stream) with the entries for the
generators from the Toeplitz source.  Against the oracle sampling through
its own FFT product on the same R: d_final, adaptations, ranks under the tie
rule, error <= 1.1x the oracle's; the symmetric option calls the operator
for A R only; a failing operator stops the compression with
HSS_ERR_OPERATOR; at n = 131072 the operator form matches the entry form's
ranks and error."""
from __future__ import annotations

import numpy as np
import pytest

import gpu_util as gu
import workloads as w
from oracle import apply
from oracle import hss as ohss
from oracle.hss import Options, compress
from oracle.operator import toeplitz_product

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


def _op(hss, torch, src):
    fn = gu.toeplitz_fft_operator(torch.from_numpy(src.col).to(gu.dev()), torch.from_numpy(src.row).to(gu.dev()))
    return hss.make_operator(fn), fn


CASES = [
    ("toeplitz_cos1500_inc", lambda: w.toeplitz_cos(1500),
     Options(leaf=100, rtol=1e-6, atol=1e-12, d0=32, dd=32, d_max=1024)),
    ("toeplitz_inv1024_dbl", lambda: w.toeplitz_inverse_distance(1024),
     Options(leaf=64, rtol=1e-8, atol=1e-14, d0=32, dd=32, d_max=1024, strategy="doubling")),
    ("toeplitz_pow2048_adapt", lambda: w.toeplitz_power(2048, 1.5),
     Options(leaf=128, rtol=1e-6, atol=1e-12, d0=16, dd=8, d_max=1024)),
    # A^T != A: the transposed product and the transposed leaf blocks matter
    ("toeplitz_nonsym1200_inc", lambda: w.toeplitz_nonsymmetric(1200),
     Options(leaf=100, rtol=1e-6, atol=1e-12, d0=32, dd=16, d_max=1024)),
]


@pytest.mark.parametrize("name,mk,o", CASES, ids=[c[0] for c in CASES])
def test_operator_parity(hss, torch, name, mk, o):
    src = mk()
    n = src.n
    R = w.gaussian_matrix(7, n, 0, o.d_max)
    ref = compress(src, R, o, product=lambda X, tr: toeplitz_product(src.col, src.row, X, tr))
    op, fn = _op(hss, torch, src)
    H = gu.gpu_compress(src, R, o, op=op)
    st = H.stats()
    assert st.converged == 1 and ref.converged
    assert st.d_final == ref.d_final and st.n_adapt == ref.n_adapt
    assert fn.calls.count(0) == fn.calls.count(1) == st.n_adapt + 1   # one product per orientation and pass
    bad = gu.compare_with_oracle(H, ref, o, n)
    assert not bad, bad
    A = src.to_dense()
    err_g = gu.rel_err(A, gu.gpu_dense(H, n))
    assert err_g <= 1.1 * apply.rel_error(ref, A) + 1e-15


def test_operator_symmetric(hss, torch):
    """A symmetric Toeplitz matrix with the symmetric option: only A R is
    requested, and the result equals the general form's."""
    src = w.toeplitz_inverse_distance(1024)
    R = w.gaussian_matrix(3, src.n, 0, 512)
    o = Options(leaf=64, rtol=1e-6, atol=1e-12, d0=32, dd=32, d_max=512, symmetric=True)
    op, fn = _op(hss, torch, src)
    H = gu.gpu_compress(src, R, o, op=op)
    assert H.stats().converged == 1 and set(fn.calls) == {0}
    ref = compress(src, R, o, product=lambda X, tr: toeplitz_product(src.col, src.row, X, tr))
    assert H.stats().d_final == ref.d_final
    assert not gu.compare_with_oracle(H, ref, o, src.n)


def test_operator_failure_status(hss, torch):
    """An operator that fails (an exception in the callable) stops the
    compression with HSS_ERR_OPERATOR; the library stays usable."""
    src = w.toeplitz_inverse_distance(512)

    def broken(trans, R, S, stream):
        raise RuntimeError("no product")

    op = hss.make_operator(broken)
    o = Options(leaf=64, rtol=1e-6, atol=1e-12, d0=32, dd=32, d_max=256)
    with pytest.raises(hss.HSSError) as ei:
        gu.gpu_compress(src, w.gaussian_matrix(1, 512, 0, 256), o, op=op)
    assert ei.value.status == hss.HSS_ERR_OPERATOR
    assert isinstance(hss.last_operator_error, RuntimeError)
    H = gu.gpu_compress(src, w.gaussian_matrix(1, 512, 0, 256), o)
    assert H.stats().converged == 1


def test_operator_full_size_toeplitz_cos(hss, torch):
    """n = 131072 (the Toeplitz cos configuration): the FFT operator form in
    FP64 against the entry form of the same compression (TF32x2 sampling, the
    configuration's form): converged, ranks within the noise band, H x on
    sampled rows within 10 rtol of A x."""
    src = w.toeplitz_cos(131072)
    n = src.n
    o = Options(leaf=256, rtol=1e-4, atol=1e-10, d0=128, dd=64, d_max=1024)
    op, fn = _op(hss, torch, src)
    H = gu.gpu_compress(src, None, o, pass_R=False, seed=0, op=op)
    H2 = gu.gpu_compress(src, None, o, precision="tf32x2", pass_R=False, seed=0)
    s1, s2 = H.stats(), H2.stats()
    assert s1.converged == 1 and s2.converged == 1
    r1, r2 = max(s1.max_rank_r, s1.max_rank_c), max(s2.max_rank_r, s2.max_rank_c)
    assert abs(r1 - r2) <= max(2, 0.02 * r2), (r1, r2)
    rng = np.random.default_rng(5)
    x = rng.standard_normal(n)
    X = torch.from_numpy(x).to(gu.dev()).reshape(1, n).t()
    Y = torch.empty((1, n), dtype=torch.float64, device=gu.dev()).t()
    hss.hss_matvec(H, X, Y)
    torch.cuda.synchronize()
    rows = np.sort(rng.choice(n, 64, replace=False))
    ex = ohss._Sampler(src).entries(rows, np.arange(n)) @ x
    err = np.linalg.norm(Y.cpu().numpy()[rows, 0] - ex) / np.linalg.norm(ex)
    assert err <= 10 * o.rtol, err
