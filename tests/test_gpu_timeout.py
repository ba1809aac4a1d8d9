"""Failure detection without a GPU fault: the device-side waits of the
kernels whose CTAs share a node side are bounded, and a wait that runs out
makes the kernels return and the call report HSS_ERR_TIMEOUT.  A limit of
one nanosecond makes the first wait that has to spin give up; the library
stays usable and the next compression in the process matches the oracle."""
import pytest

import workloads as w
from oracle import apply
from oracle.hss import Options, compress

import gpu_util as gu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hss():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1810_04125_gb300 import build, hss as h
    build.build()
    return h


def _compress(hss, src, R, o, wait_ns):
    opts = hss.make_opts(o.leaf, o.rtol, o.atol, o.d0, o.dd, o.d_max, gu.STRAT[o.strategy], R=gu.col_major(R),
                         wait_limit_ns=wait_ns)
    return hss.hss_compress(gu.device_source(src), opts)


@pytest.mark.parametrize("strategy", ["doubling", "incrementing"])
def test_group_wait_runs_out_then_recovers(hss, strategy):
    # four leaves of 256 rows: eight node sides, each worked on by a group of
    # CTAs (QRCP; with Incrementing also the test kernel's groups)
    src = w.toeplitz_cos(1024)
    o = Options(leaf=256, rtol=1e-6, atol=1e-12, d0=64, dd=64, d_max=512, strategy=strategy)
    R = w.gaussian_matrix(5, src.n, 0, o.d_max)
    with pytest.raises(hss.HSSError) as ei:
        _compress(hss, src, R, o, 1)
    assert ei.value.status == hss.HSS_ERR_TIMEOUT
    assert b"gave up" in hss.lib().hss_last_error()
    # the same compression with the default limit, in the same process
    ref = compress(src, R, o)
    H = _compress(hss, src, R, o, 0)
    st = H.stats()
    assert st.converged and (st.d_final, st.n_adapt) == (ref.d_final, ref.n_adapt)
    assert not gu.compare_with_oracle(H, ref, o, src.n)
    A = src.to_dense()
    assert gu.rel_err(A, gu.gpu_dense(H, src.n)) <= 1.1 * apply.rel_error(ref, A) + 1e-15
