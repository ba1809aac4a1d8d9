"""The CUDA path at the settings of the oracle's closed-form pins: Doubling's
acceptance rule (k <= d - p, all rows selected; Algorithm 4, eq.
RRQRHMTstop) on matrices of exact HSS ranks, and Incrementing driven by its
absolute tests alone (rtol = 0; eq. stopping_criteria)."""
import numpy as np
import pytest

import workloads as w
from oracle import apply
from oracle.hss import Options, compress

import gpu_util as gu
from test_oracle_pins import doubling_closed_form

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hss():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1810_04125_gb300 import build, hss as h
    build.build()
    return h


CASES = [({4: 8, 3: 12, 2: 16, 1: 20}, d0, p) for d0, p in ((12, 0), (12, 10), (15, 10), (7, 0), (11, 10))]
CASES += [({4: 8, 3: 16, 2: 20, 1: 24}, 8, 10), ({4: 8, 3: 15, 2: 20, 1: 24}, 16, 3)]


@pytest.mark.parametrize("ranks,d0,p", CASES)
def test_doubling_acceptance_closed_form_gpu(hss, ranks, d0, p):
    n, leaf = 1024, 64
    A = w.synthetic_hss(n, leaf, ranks, seed=3)
    R = w.gaussian_matrix(5, n, 0, 128)
    o = Options(leaf=leaf, rtol=1e-10, atol=1e-14, d0=d0, dd=d0, d_max=128, strategy="doubling", p=p)
    H = gu.gpu_compress(w.dense_source(A), R, o)
    st = H.stats()
    kept = {}
    assert (bool(st.converged), st.d_final, st.n_adapt) == doubling_closed_form(n, leaf, ranks, d0, p, 128, kept)
    # rows and kept ranks: the exact rank where the rule stopped, every row
    # where it selected all of them (P9), at the pass that accepted the node
    for i in range(1, st.n_nodes):
        nd = H.node(i)
        m, k = kept[i]
        assert (nd.mr, nd.mc, nd.kr, nd.kc) == (m, m, k, k), (i, nd.mr, nd.kr, m, k)
    assert gu.rel_err(A, gu.gpu_dense(H, n)) < 1e-12


ATOL_CASES = [
    ("toeplitz1000_atol", lambda: w.toeplitz_inverse_distance(1000),
     Options(leaf=50, rtol=0.0, atol=1e-6, d0=16, dd=8, d_max=512)),
    ("udv900_atol", lambda: w.dense_source(w.udv_matrix(900, 50, seed=4)),
     Options(leaf=64, rtol=0.0, atol=1e-9, d0=8, dd=8, d_max=512)),
    ("toeplitzcos2048_atol_dbl", lambda: w.toeplitz_cos(2048),
     Options(leaf=128, rtol=0.0, atol=1e-7, d0=16, dd=16, d_max=1024, strategy="doubling", p=4)),
]


@pytest.mark.parametrize("name,mk,o", ATOL_CASES, ids=[c[0] for c in ATOL_CASES])
def test_absolute_tolerance_only_parity(hss, name, mk, o):
    src = mk()
    n = src.n
    R = w.gaussian_matrix(11, n, 0, o.d_max)
    ref = compress(src, R, o)
    H = gu.gpu_compress(src, R, o)
    st = H.stats()
    assert st.converged == 1 and ref.converged
    assert (st.d_final, st.n_adapt) == (ref.d_final, ref.n_adapt)
    assert not gu.compare_with_oracle(H, ref, o, n)
    A = src.to_dense()
    assert gu.rel_err(A, gu.gpu_dense(H, n)) <= 1.1 * apply.rel_error(ref, A) + 1e-15
