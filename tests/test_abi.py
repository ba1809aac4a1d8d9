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
    assert L.hss_load(b"/nonexistent/dir/file", C.byref(hh)) == hss.HSS_ERR_IO and not hh.value
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
    bad_t = hss.hss_tuning(0, 4, 2, 4, 0)
    assert L.hss_set_tuning(C.byref(bad_t)) == hss.HSS_ERR_ARG
    bad_t = hss.hss_tuning(8, 4, 2, 4, 3)    # CTAs per SM: 0, 1, 2 or 4
    assert L.hss_set_tuning(C.byref(bad_t)) == hss.HSS_ERR_ARG
    hss.set_tuning()
    assert hss.get_tuning() == {"qrcp_wide_max_sides": 8, "sample_waves_packed": 4, "sample_waves_generated": 2,
                                "qrcp_min_cols": 4, "qrcp_sm_ctas": 0}
    hss.set_tuning(qrcp_sm_ctas=1)
    assert hss.get_tuning()["qrcp_sm_ctas"] == 1
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
    assert L.hss_matvec(None, 1, None, 1, None, 1, 0, None) == hss.HSS_ERR_ARG
    assert L.hss_get_entries(None, 1, None, 1, None, None, 1, None) == hss.HSS_ERR_ARG
    # an extraction source needs its routine, and a sampling operator
    s_x = hss.hss_source(hss.HSS_SRC_EXTRACT, 100, 0, 0, None, None, 0, 0.0, 0.0)
    assert L.hss_compress(C.byref(s_x), C.byref(o), None, C.byref(h)) == hss.HSS_ERR_ARG
    s_x = hss.extract_source(100, lambda blocks, stream: None)
    assert L.hss_compress(C.byref(s_x), C.byref(o), None, C.byref(h)) == hss.HSS_ERR_ARG
    assert b"operator" in L.hss_last_error()
    assert L.hss_sample_offdiag(C.byref(s_x), 16, 0, 1, 1234, 100, None, None, 1, None) == hss.HSS_ERR_ARG
    assert L.hss_status_str(hss.HSS_ERR_IO) == b"HSS_ERR_IO"
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


# ------------------------------------------------------------ checkpoint files
def _checkpoint_bytes(hss, n=8, leaf=2, mutate=None):
    """A well-formed checkpoint of a handle on the halving tree of (n, leaf)
    with rank 1 at every node, written field by field in the file format of
    hss_save (magic, header, statistics, then per node its record and
    arrays as count + elements).  ``mutate(name, value)`` may replace a field
    before it is written."""
    import struct
    nodes = otree.halving_tree(n, leaf)
    mx = max(t.level for t in nodes)
    mut = mutate or (lambda name, v: v)
    out = [b"HSSGEN01"]
    hdr = mut("hdr", [n, len(nodes), mx, 1, 1, 4, 0, leaf])
    out.append(struct.pack("8i", *hdr))
    sst = C.sizeof(hss.hss_stats)
    out.append(struct.pack("q", sst) + bytes(sst))

    def arr(name, vals, fmt):
        vals = mut(name, vals)
        if vals is None:
            return struct.pack("q", -1)
        return struct.pack("q", len(vals)) + struct.pack(f"{len(vals)}{fmt}", *vals)

    for t in nodes:
        root, leafn = t.idx == 0, not t.children
        m = 0 if root else (t.size if leafn else 2)
        k = 0 if root else 1
        rec = mut(f"rec{t.idx}", [t.lo, t.size, t.level, t.parent,
                                  t.children[0] if t.children else -1, t.children[1] if t.children else -1,
                                  1 if leafn else 0, 2, m, k, m, k])
        out.append(struct.pack("12i", *rec))
        for side in "rc":
            piv = None if root else list(range(m))[::-1]
            X = None if root else [0.5] * (k * (m - k))
            # skeleton index: the global index of the first pivot's row
            I = None if root else [t.lo + (piv[0] if leafn else 0)]
            out.append(arr(f"piv{t.idx}{side}", piv, "i"))
            out.append(arr(f"X{t.idx}{side}", X, "d"))
            out.append(arr(f"I{t.idx}{side}", I, "i"))
        out.append(arr(f"D{t.idx}", [1.0] * (t.size * t.size) if leafn else None, "d"))
        out.append(arr(f"B12{t.idx}", None if leafn else [0.7], "d"))
        out.append(arr(f"B21{t.idx}", None if leafn else [0.3], "d"))
    return b"".join(out)


def _load_status(hss, blob, tmp_path):
    p = tmp_path / "c.hss"
    p.write_bytes(blob)
    h = C.c_void_p(123)
    st = hss.lib().hss_load(str(p).encode(), C.byref(h))
    if st == hss.HSS_OK:
        hss.lib().hss_free(h)
    else:
        assert not h.value
    return st


def test_checkpoint_checks_on_host(hss, tmp_path):
    """hss_load checks the whole file on the host before it uploads
    anything: a well-formed file gets past every check (without a GPU it then
    fails at the device copy, HSS_ERR_CUDA), and each damaged variant is
    rejected as HSS_ERR_ARG."""
    import torch
    good = _checkpoint_bytes(hss)
    if not torch.cuda.is_available():
        assert _load_status(hss, good, tmp_path) == hss.HSS_ERR_CUDA
    else:
        assert _load_status(hss, good, tmp_path) == hss.HSS_OK

    def bad(name, fn):
        return _checkpoint_bytes(hss, mutate=lambda nm, v: fn(v) if nm == name else v)

    damaged = {
        "truncated": good[:-8],
        "trailing bytes": good + b"\0",
        "pivot repeated": bad("piv3r", lambda v: [v[0], v[0]]),
        "pivot out of range": bad("piv1c", lambda v: [2, 0]),
        "pivot array short": bad("piv4r", lambda v: v[:1]),
        "X count": bad("X2c", lambda v: v + [0.0]),
        "X missing": bad("X5r", lambda v: None),
        "skeleton index outside the node": bad("I6r", lambda v: [0]),
        "B12 count": bad("B121", lambda v: v + [1.0, 2.0]),
        "B21 missing": bad("B210", lambda v: None),
        "D short": bad("D3", lambda v: v[:3]),
        "D at a non-leaf": bad("D1", lambda v: [1.0]),
        "tree record": bad("rec2", lambda v: [v[0], v[1] + 1] + v[2:]),
        "sample rows of a non-leaf": bad("rec1", lambda v: v[:8] + [3, 1, 3, 1]),
        "rank above rows": bad("rec3", lambda v: v[:8] + [2, 3, 2, 1]),
        "not converged": bad("hdr", lambda v: v[:4] + [0] + v[5:]),
        "leaf size": bad("hdr", lambda v: v[:7] + [4]),   # a 3-node tree
        "node count": bad("hdr", lambda v: [v[0], v[1] + 2] + v[2:]),
    }
    for what, blob in damaged.items():
        assert _load_status(hss, blob, tmp_path) == hss.HSS_ERR_ARG, what
