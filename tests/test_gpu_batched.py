"""hss_compress_batched: members of a mixed batch (two Toeplitz families and
3-D Gaussian kernels of different orders, both strategies, FP64 and TF32x2)
compressed side by side, each against the oracle on the same R (ranks under
the tie rule of the single-matrix tests, error <= 1.1x the oracle's)."""
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


def _members():
    out = []
    for n in (512, 777, 1024):
        out.append((w.toeplitz_power(n, 1.5),
                    Options(leaf=64, rtol=1e-6, atol=1e-12, d0=32, dd=32, d_max=512), "fp64"))
    for n, seed in ((640, 1), (1000, 2)):
        pts = w.uniform_points(n, 3, seed=seed)
        out.append((w.gaussian_kernel(pts[rcb_order(pts, 64)], 0.3, 0.0),
                    Options(leaf=64, rtol=1e-5, atol=1e-10, d0=64, dd=64, d_max=512,
                            strategy="doubling"), "tf32x2"))
    out.append((w.toeplitz_cos(900),
                Options(leaf=100, rtol=1e-4, atol=1e-10, d0=64, dd=32, d_max=512), "tf32x2"))
    return out


def test_batched_matches_oracle(hss, torch):
    mem = _members()
    srcs, opts, Rs, keep = [], [], [], []
    for i, (src, o, prec) in enumerate(mem):
        R = w.gaussian_matrix(20 + i, src.n, 0, o.d_max)
        if prec == "tf32x2":
            R = w.round_to_tf32(R)
        Rs.append(R)
        s = gu.device_source(src)
        Rd = gu.col_major(R)
        keep += [s, Rd]
        srcs.append(s)
        opts.append(hss.make_opts(o.leaf, o.rtol, o.atol, o.d0, o.dd, o.d_max, gu.STRAT[o.strategy],
                                  gu.PREC[prec], o.p, 0, Rd, int(o.level_tol_scaling)))
    Hs = hss.hss_compress_batched(srcs, opts)
    assert len(Hs) == len(mem)
    for (src, o, prec), R, H in zip(mem, Rs, Hs):
        ref = compress(src, R, o)
        st = H.stats()
        assert st.converged == 1 and ref.converged
        assert st.d_final == ref.d_final
        bad = gu.compare_with_oracle(H, ref, o, src.n,
                                     noise=None if prec == "fp64" else gu.mixed_noise(src, R, ref))
        assert not bad, (src.name, bad)
        A = src.to_dense()
        err_g = gu.rel_err(A, gu.gpu_dense(H, src.n))
        assert err_g <= 1.1 * apply.rel_error(ref, A) + 1e-15, (src.name, err_g)


def test_batched_error_frees_everything(hss, torch):
    """A member with an invalid source fails the whole call: every handle is
    freed and the failing member is named."""
    good = gu.device_source(w.toeplitz_inverse_distance(256))
    bad = hss.hss_source(hss.HSS_SRC_DENSE, 256, 0, 0, None, None, 256, 0.0, 0.0)   # no data
    o = hss.make_opts(32, 1e-6, 1e-12, 32, 32, 256, hss.HSS_INCREMENTING)
    with pytest.raises(hss.HSSError) as e:
        hss.hss_compress_batched([good, bad, good], [o, o, o])
    assert "matrix 1" in str(e.value)


def test_batched_levels_share_launches(hss, torch):
    """Lockstep batching: every phase of a tree level is one launch over the
    nodes of all matrices, so eight equal matrices take far fewer launches
    than eight single calls (only the sampling launches are per matrix), with
    the same ranks and an error within 1.1x the oracle's."""
    src = w.toeplitz_power(1024, 1.5)
    o = Options(leaf=64, rtol=1e-6, atol=1e-12, d0=16, dd=16, d_max=512)
    R = w.gaussian_matrix(3, src.n, 0, o.d_max)
    ref = compress(src, R, o)
    s = gu.device_source(src)
    Rd = gu.col_major(R)
    opt = hss.make_opts(o.leaf, o.rtol, o.atol, o.d0, o.dd, o.d_max, gu.STRAT[o.strategy], R=Rd)
    single = hss.hss_compress(s, opt)
    Hs = hss.hss_compress_batched([s] * 8, [opt] * 8)
    launches_batch = sum(H.stats().launches for H in Hs)
    launches_single = single.stats().launches
    assert launches_batch <= 0.5 * 8 * launches_single, (launches_batch, launches_single)
    A = src.to_dense()
    for H in Hs:
        st = H.stats()
        assert (st.d_final, st.n_adapt) == (ref.d_final, ref.n_adapt)
        assert H.ranks() == single.ranks()
        assert not gu.compare_with_oracle(H, ref, o, src.n)
        assert gu.rel_err(A, gu.gpu_dense(H, src.n)) <= 1.1 * apply.rel_error(ref, A) + 1e-15
