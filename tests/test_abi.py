"""The C-ABI library loads and exports every entry point of include/hss.h;
host-side entry points and argument validation work without a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import workloads as w
from oracle import tree as otree

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def hss():
    from paper_1810_04125_gb300 import build, hss as binding
    build.build()
    return binding


def header_functions():
    txt = open(os.path.join(ROOT, "include", "hss.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(hss_\w+)\s*\(", txt)))


def test_exports_every_declared_symbol(hss):
    names = header_functions()
    assert len(names) >= 11
    lib = hss.lib()
    for nm in names:
        assert hasattr(lib, nm), nm
    assert set(names) == set(hss.EXPORTS)


def test_status_strings(hss):
    L = hss.lib()
    assert L.hss_status_str(0) == b"HSS_OK"
    assert L.hss_status_str(4) == b"HSS_ERR_NOT_CONVERGED"


def test_rcb_matches_oracle_bitwise(hss):
    rng = np.random.default_rng(0)
    for n, dim, leaf in [(1000, 3, 64), (4096, 8, 128), (777, 2, 50)]:
        P = rng.random((n, dim))
        assert np.array_equal(hss.hss_rcb_order(P, leaf), otree.rcb_order(P, leaf))
    # ties: many equal coordinates
    P = np.floor(rng.random((600, 3)) * 4)
    assert np.array_equal(hss.hss_rcb_order(P, 16), otree.rcb_order(P, 16))
    # sphere points
    P = w.fibonacci_sphere(2048)
    assert np.array_equal(hss.hss_rcb_order(P, 64), otree.rcb_order(P, 64))


def test_argument_validation_without_gpu(hss):
    L = hss.lib()
    h = C.c_void_p()
    o = hss.make_opts(64, 1e-6, 1e-12, 64, 32, 256, hss.HSS_INCREMENTING)
    assert L.hss_compress(None, C.byref(o), None, C.byref(h)) == hss.HSS_ERR_ARG
    s = hss.hss_source(hss.HSS_SRC_DENSE, 100, 0, 0, 1234, None, 50, 0.0, 0.0)  # ld < n
    assert L.hss_compress(C.byref(s), C.byref(o), None, C.byref(h)) == hss.HSS_ERR_ARG
    assert b"ld" in L.hss_last_error()
    s = hss.hss_source(hss.HSS_SRC_TOEPLITZ, 100, 0, 0, 1234, 1234, 0, 0.0, 0.0)
    bad = hss.make_opts(0, 1e-6, 1e-12, 64, 32, 256, hss.HSS_INCREMENTING)
    assert L.hss_compress(C.byref(s), C.byref(bad), None, C.byref(h)) == hss.HSS_ERR_ARG
    bad = hss.make_opts(64, -1.0, 1e-12, 64, 32, 256, hss.HSS_INCREMENTING)
    assert L.hss_compress(C.byref(s), C.byref(bad), None, C.byref(h)) == hss.HSS_ERR_ARG
    bad = hss.make_opts(64, 1e-6, 1e-12, 64, 0, 256, hss.HSS_INCREMENTING)
    assert L.hss_compress(C.byref(s), C.byref(bad), None, C.byref(h)) == hss.HSS_ERR_ARG
    bad = hss.make_opts(64, 1e-6, 1e-12, 64, 32, 256, 7)
    assert L.hss_compress(C.byref(s), C.byref(bad), None, C.byref(h)) == hss.HSS_ERR_ARG
    # a user operator needs an apply function and the FP64 form
    op = hss.make_operator(lambda *a: None)
    bad = hss.make_opts(64, 1e-6, 1e-12, 64, 32, 256, hss.HSS_INCREMENTING, hss.HSS_PREC_TF32X2, op=op)
    assert L.hss_compress(C.byref(s), C.byref(bad), None, C.byref(h)) == hss.HSS_ERR_ARG
    null_op = hss.hss_operator()
    bad = hss.make_opts(64, 1e-6, 1e-12, 64, 32, 256, hss.HSS_INCREMENTING, op=null_op)
    assert L.hss_compress(C.byref(s), C.byref(bad), None, C.byref(h)) == hss.HSS_ERR_ARG
    assert L.hss_status_str(hss.HSS_ERR_OPERATOR) == b"HSS_ERR_OPERATOR"
    # checkpoints: arguments and files checked on the host
    assert L.hss_save(None, b"/nonexistent/x") == hss.HSS_ERR_ARG
    hh = C.c_void_p(123)
    assert L.hss_load(b"/nonexistent/dir/file", C.byref(hh)) == hss.HSS_ERR_ARG and not hh.value
    import tempfile
    with tempfile.NamedTemporaryFile(suffix=".hss", delete=False) as tf:
        tf.write(b"not a checkpoint at all")
    try:
        hh = C.c_void_p(123)
        assert L.hss_load(tf.name.encode(), C.byref(hh)) == hss.HSS_ERR_ARG and not hh.value
    finally:
        os.unlink(tf.name)
    # launch-shape parameters: validated, settable, restorable
    saved = hss.get_tuning()
    bad_t = hss.hss_tuning(0, 4, 2)
    assert L.hss_set_tuning(C.byref(bad_t)) == hss.HSS_ERR_ARG
    hss.set_tuning()
    assert hss.get_tuning() == {"qrcp_wide_max_sides": 8, "sample_waves_packed": 4, "sample_waves_generated": 2}
    hss.set_tuning(qrcp_wide_max_sides=16)
    assert hss.get_tuning()["qrcp_wide_max_sides"] == 16
    hss.set_tuning(**saved)
    assert hss.get_tuning() == saved
    # the HMT criterion: Incrementing only, alpha > 1 and finite, known criterion codes
    for kw in (dict(strategy=hss.HSS_DOUBLING, criterion=hss.HSS_CRIT_HMT),
               dict(strategy=hss.HSS_INCREMENTING, criterion=hss.HSS_CRIT_HMT, hmt_alpha=1.0),
               dict(strategy=hss.HSS_INCREMENTING, criterion=hss.HSS_CRIT_HMT, hmt_alpha=float("inf")),
               dict(strategy=hss.HSS_INCREMENTING, criterion=2)):
        bad = hss.make_opts(64, 1e-6, 1e-12, 64, 32, 256, **kw)
        assert L.hss_compress(C.byref(s), C.byref(bad), None, C.byref(h)) == hss.HSS_ERR_ARG, kw
    assert h.value is None
    assert L.hss_matvec(None, 1, None, 1, None, 1, None) == hss.HSS_ERR_ARG
    hs = (C.c_void_p * 1)()
    assert L.hss_compress_batched(None, None, -1, None, hs) == hss.HSS_ERR_ARG
    assert L.hss_compress_batched(None, C.byref(o), 1, None, hs) == hss.HSS_ERR_ARG
    assert L.hss_compress_batched(None, None, 0, None, None) == hss.HSS_OK
    k = C.c_int(5)
    assert L.hss_compress_restart(None, C.byref(o), None, C.byref(h), C.byref(k)) == hss.HSS_ERR_ARG
    assert k.value == 0
    bad = hss.make_opts(0, 1e-6, 1e-12, 64, 32, 256, hss.HSS_INCREMENTING)
    assert L.hss_compress_restart(C.byref(s), C.byref(bad), None, C.byref(h), None) == hss.HSS_ERR_ARG
    assert L.hss_rcb_order(None, 10, 2, 10, 4, None) == hss.HSS_ERR_ARG
    assert L.hss_random_normal(0, 10, 0, 1, None, 10, 0, None) == hss.HSS_ERR_ARG
