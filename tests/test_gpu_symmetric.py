"""The symmetric option (A = A^T; the column side copies the row side) on the
GPU against the oracle's symmetric option on the same R: d_final, ranks
under the tie rule, error <= 1.1x the oracle's, V = U and B21 = B12^T in the
exported generators; and against the GPU's own general form."""
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
    ("toeplitz1000_inc_fp64", lambda: w.toeplitz_inverse_distance(1000), "fp64",
     Options(leaf=64, rtol=1e-6, atol=1e-12, d0=32, dd=32, d_max=512, symmetric=True)),
    ("gauss1200_dbl_fp64", lambda: _gauss(1200, 3, 0.4, 64), "fp64",
     Options(leaf=64, rtol=1e-6, atol=1e-12, d0=32, dd=32, d_max=1024, strategy="doubling",
             symmetric=True)),
    ("gauss2048_dbl_tf32", lambda: _gauss(2048, 4, 0.5, 128), "tf32x2",
     Options(leaf=128, rtol=1e-4, atol=1e-8, d0=64, dd=64, d_max=2048, strategy="doubling",
             symmetric=True)),
    ("synthetic_sym1024_inc_fp64", lambda: w.dense_source(
        w.synthetic_hss(1024, 64, {4: 8, 3: 12, 2: 16, 1: 20}, seed=4, symmetric=True)), "fp64",
     Options(leaf=64, rtol=1e-6, atol=1e-12, d0=16, dd=16, d_max=512, symmetric=True)),
    ("laplace1536_inc_bf16", lambda: w.laplace_kernel(
        (lambda P: P[rcb_order(P, 96)])(w.fibonacci_sphere(1536))), "bf16x3",
     Options(leaf=96, rtol=1e-5, atol=1e-8, d0=64, dd=32, d_max=1024, symmetric=True)),
]


@pytest.mark.parametrize("name,mk,prec,o", CASES, ids=[c[0] for c in CASES])
def test_symmetric_parity(hss, torch, name, mk, prec, o):
    src = mk()
    n = src.n
    R = w.gaussian_matrix(9, n, 0, o.d_max)
    if prec == "tf32x2":
        R = w.round_to_tf32(R)
    elif prec == "bf16x3":
        R = w.round_to_bf16(R)
    ref = compress(src, R, o)
    H = gu.gpu_compress(src, R, o, precision=prec)
    st = H.stats()
    assert st.converged == 1 and ref.converged
    assert st.d_final == ref.d_final
    bad = gu.compare_with_oracle(H, ref, o, n, noise=None if prec == "fp64" else gu.mixed_noise(src, R, ref))
    assert not bad, bad
    A = src.to_dense()
    err_g = gu.rel_err(A, gu.gpu_dense(H, n))
    assert err_g <= 1.1 * apply.rel_error(ref, A) + 1e-15, err_g
    for i in range(1, st.n_nodes):
        e = H.export_node(i)
        assert np.array_equal(e["Pr"], e["Pc"]) and np.array_equal(e["Xr"], e["Xc"])
        if e.get("B12") is not None and e["B12"].size:
            assert np.array_equal(e["B21"], e["B12"].T)


def test_symmetric_matches_general_form(hss, torch):
    """Same matrix and R: the symmetric option and the general algorithm give
    the same d_final, ranks within the tie rule and the same error."""
    src = _gauss(1500, 5, 0.4, 64)
    o = Options(leaf=64, rtol=1e-6, atol=1e-12, d0=64, dd=64, d_max=1024, strategy="doubling")
    R = w.gaussian_matrix(10, src.n, 0, 1024)
    Hg = gu.gpu_compress(src, R, o)
    o.symmetric = True
    Hs = gu.gpu_compress(src, R, o)
    sg, ss = Hg.stats(), Hs.stats()
    assert sg.d_final == ss.d_final
    A = src.to_dense()
    eg, es = gu.rel_err(A, gu.gpu_dense(Hg, src.n)), gu.rel_err(A, gu.gpu_dense(Hs, src.n))
    assert abs(eg - es) <= 0.05 * eg, (eg, es)
    rg, rs = Hg.ranks(), Hs.ranks()
    assert sum(1 for i in rg if rg[i] != rs[i]) <= 2, (rg, rs)
