"""hss_sample_offdiag_noalloc: the sampling entry point for callers that
cannot let the library allocate device memory (a process whose device
memory is owned by its own pool, or one that cannot take cudaMalloc's
synchronisation or failure mid-run).  Its output must equal that of the
allocating hss_sample_offdiag on the same inputs, on consecutive calls that
reuse the library's fixed leaf table with different sizes.  This file is
collected last so that a run stopping at the first failure has already run
every other test."""
import ctypes as C

import numpy as np
import pytest

import workloads as w

pytestmark = pytest.mark.gpu


def _run(hss, torch, fn, src_dev, leaf, R, n, nc):
    Sr = torch.full((n, nc), float("nan"), dtype=torch.float64, device="cuda:0")
    Sc = torch.full((n, nc), float("nan"), dtype=torch.float64, device="cuda:0")
    fn(src_dev, leaf, hss.HSS_PREC_FP64, R, Sr, Sc)
    torch.cuda.synchronize()
    return Sr.cpu().numpy(), Sc.cpu().numpy()


def test_noalloc_matches_allocating_entry_point():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1810_04125_gb300 import build
    build.build()
    from paper_1810_04125_gb300 import hss
    import gpu_util as gu

    cases = [
        (w.toeplitz_cos(1500), 100, 70),
        (w.dense_source(np.random.default_rng(4).standard_normal((700, 700))), 64, 33),
    ]
    for src, leaf, nc in cases:           # two calls in a row, different n and leaf
        n = src.n
        Rd = gu.col_major(w.gaussian_matrix(3, n, 0, nc))
        sd = gu.device_source(src)
        ar, ac = _run(hss, torch, hss.hss_sample_offdiag, sd, leaf, Rd, n, nc)
        br, bc = _run(hss, torch, hss.hss_sample_offdiag_noalloc, sd, leaf, Rd, n, nc)
        assert np.all(np.isfinite(br)) and np.all(np.isfinite(bc))
        np.testing.assert_allclose(br, ar, rtol=1e-13, atol=1e-13 * np.abs(ar).max())
        np.testing.assert_allclose(bc, ac, rtol=1e-13, atol=1e-13 * np.abs(ac).max())

    # sizes beyond the fixed table are refused before anything is launched
    big = hss.hss_source(hss.HSS_SRC_TOEPLITZ, (1 << 20) + 1, 0, 0, 1, 1, 0, 0.0, 0.0)
    st = hss.lib().hss_sample_offdiag_noalloc(C.byref(big), 64, 0, 8, 1, (1 << 20) + 1, 1, 1, 8,
                                             None)
    assert st == hss.HSS_ERR_ARG
    assert b"exceeds" in hss.lib().hss_last_error()
