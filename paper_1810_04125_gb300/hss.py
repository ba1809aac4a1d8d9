"""Thin ctypes binding of libhss.so (include/hss.h).

The functions carry the C names and only marshal arguments: device buffers
are passed as torch CUDA tensors (their data pointers), host buffers as
numpy arrays.  Every step of the method runs in the CUDA library; if the
library has not been built, loading fails loudly.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhss.so")
# launch-shape table written by tune.py for this GPU family (applied on load)
TUNING_PATH = os.path.join(_HERE, "tuning_sm103.json")

HSS_OK, HSS_ERR_ARG, HSS_ERR_NOMEM, HSS_ERR_CUDA = 0, 1, 2, 3
HSS_ERR_NOT_CONVERGED, HSS_ERR_NONFINITE, HSS_ERR_TIMEOUT, HSS_ERR_UNSUPPORTED = 4, 5, 6, 7
HSS_ERR_OPERATOR, HSS_ERR_IO = 8, 9
HSS_DOUBLING, HSS_INCREMENTING = 0, 1
HSS_CRIT_NEW, HSS_CRIT_HMT = 0, 1
HSS_PREC_FP64, HSS_PREC_TF32X2, HSS_PREC_BF16X3 = 0, 1, 2
HSS_SRC_DENSE, HSS_SRC_TOEPLITZ, HSS_SRC_GAUSS, HSS_SRC_LAPLACE, HSS_SRC_EXTRACT = 0, 1, 2, 3, 4
HSS_UNTOUCHED, HSS_PARTIALLY_COMPRESSED, HSS_COMPRESSED = 0, 1, 2

EXPORTS = ["hss_compress", "hss_compress_restart", "hss_compress_batched", "hss_save", "hss_load", "hss_matvec", "hss_get_entries", "hss_to_dense", "hss_get_stats", "hss_get_node", "hss_export_node",
           "hss_free", "hss_release_cached", "hss_set_tuning", "hss_get_tuning", "hss_status_str",
           "hss_last_error", "hss_rcb_order",
           "hss_random_normal", "hss_sample_offdiag", "hss_sample_offdiag_noalloc"]


class hss_block(C.Structure):
    _fields_ = [("nr", C.c_int), ("nc", C.c_int), ("I", C.c_void_p), ("J", C.c_void_p),
                ("out", C.c_void_p), ("ldo", C.c_longlong)]


EXTRACT_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_int, C.POINTER(hss_block), C.c_void_p)


class hss_source(C.Structure):
    _fields_ = [("kind", C.c_int), ("n", C.c_int), ("dim", C.c_int), ("reserved", C.c_int),
                ("a", C.c_void_p), ("b", C.c_void_p), ("ld", C.c_longlong),
                ("p0", C.c_double), ("p1", C.c_double), ("extract", EXTRACT_FN), ("ctx", C.c_void_p)]


APPLY_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_longlong, C.c_void_p,
                       C.c_longlong, C.c_void_p)


class hss_operator(C.Structure):
    _fields_ = [("apply", APPLY_FN), ("ctx", C.c_void_p)]


class hss_opts(C.Structure):
    _fields_ = [("leaf", C.c_int), ("strategy", C.c_int), ("precision", C.c_int),
                ("level_tol_scaling", C.c_int), ("rtol", C.c_double), ("atol", C.c_double),
                ("d0", C.c_int), ("dd", C.c_int), ("d_max", C.c_int), ("oversample_p", C.c_int),
                ("seed", C.c_ulonglong), ("R", C.c_void_p), ("symmetric", C.c_int),
                ("criterion", C.c_int), ("hmt_alpha", C.c_double), ("op", C.POINTER(hss_operator)),
                ("wait_limit_ns", C.c_longlong)]


class hss_stats(C.Structure):
    _fields_ = [("n", C.c_int), ("n_nodes", C.c_int), ("levels", C.c_int), ("d_final", C.c_int),
                ("n_adapt", C.c_int), ("converged", C.c_int), ("max_rank_r", C.c_int),
                ("max_rank_c", C.c_int), ("ms_total", C.c_double), ("ms_sample", C.c_double),
                ("ms_rng", C.c_double), ("ms_id", C.c_double), ("ms_test", C.c_double),
                ("ms_merge", C.c_double), ("flop_sample", C.c_double),
                ("bytes_sample", C.c_double), ("launches", C.c_longlong),
                ("sample_launches", C.c_longlong), ("bytes_h2d", C.c_longlong),
                ("bytes_d2h", C.c_longlong), ("flop_id", C.c_double)]


class hss_tuning(C.Structure):
    _fields_ = [("qrcp_wide_max_sides", C.c_int), ("sample_waves_packed", C.c_int),
                ("sample_waves_generated", C.c_int), ("qrcp_min_cols", C.c_int), ("qrcp_sm_ctas", C.c_int)]


class hss_node_info(C.Structure):
    _fields_ = [(f, C.c_int) for f in ("lo", "size", "level", "parent", "child0", "child1",
                                       "state", "mr", "mc", "kr", "kc")]


_lib = None


def lib():
    """Load libhss.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_1810_04125_gb300.build` (needs nvcc)")
        L = C.CDLL(LIB_PATH)
        vp, i, ll, d = C.c_void_p, C.c_int, C.c_longlong, C.c_double
        L.hss_compress.argtypes = [C.POINTER(hss_source), C.POINTER(hss_opts), vp, C.POINTER(vp)]
        L.hss_compress_batched.argtypes = [C.POINTER(hss_source), C.POINTER(hss_opts), i, vp, C.POINTER(vp)]
        L.hss_compress_restart.argtypes = [C.POINTER(hss_source), C.POINTER(hss_opts), vp, C.POINTER(vp),
                                           C.POINTER(i)]
        L.hss_matvec.argtypes = [vp, i, vp, ll, vp, ll, i, vp]
        L.hss_get_entries.argtypes = [vp, i, vp, i, vp, vp, ll, vp]
        L.hss_to_dense.argtypes = [vp, vp, ll, vp]
        L.hss_get_stats.argtypes = [vp, C.POINTER(hss_stats)]
        L.hss_get_node.argtypes = [vp, i, C.POINTER(hss_node_info)]
        L.hss_export_node.argtypes = [vp, i] + [vp] * 11
        L.hss_free.argtypes = [vp]
        L.hss_release_cached.argtypes = []
        L.hss_save.argtypes = [vp, C.c_char_p]
        L.hss_load.argtypes = [C.c_char_p, C.POINTER(vp)]
        L.hss_set_tuning.argtypes = [C.POINTER(hss_tuning)]
        L.hss_get_tuning.argtypes = [C.POINTER(hss_tuning)]
        L.hss_free.restype = None
        L.hss_status_str.argtypes = [i]
        L.hss_status_str.restype = C.c_char_p
        L.hss_last_error.argtypes = []
        L.hss_last_error.restype = C.c_char_p
        L.hss_rcb_order.argtypes = [vp, i, i, ll, i, vp]
        L.hss_random_normal.argtypes = [C.c_ulonglong, i, i, i, vp, ll, i, vp]
        L.hss_sample_offdiag.argtypes = [C.POINTER(hss_source), i, i, i, vp, ll, vp, vp, ll, vp]
        L.hss_sample_offdiag_noalloc.argtypes = [C.POINTER(hss_source), i, i, i, vp, ll, vp, vp,
                                                 ll, vp]
        for f in EXPORTS:
            if f not in ("hss_free", "hss_status_str", "hss_last_error"):
                getattr(L, f).restype = C.c_int
        _lib = L
        _apply_tuning_table()
    return _lib


def _apply_tuning_table():
    """Apply the launch-shape table of tune.py when one is present."""
    if not os.path.exists(TUNING_PATH):
        return
    import json
    t = json.load(open(TUNING_PATH))
    set_tuning(**{k: int(t[k]) for k in ("qrcp_wide_max_sides", "sample_waves_packed",
                                         "sample_waves_generated", "qrcp_min_cols", "qrcp_sm_ctas") if k in t})


def get_tuning() -> dict:
    t = hss_tuning()
    _check(lib().hss_get_tuning(C.byref(t)))
    return {f: getattr(t, f) for f, _ in hss_tuning._fields_}


def set_tuning(**kw):
    """hss_set_tuning with the given fields changed (no arguments: defaults)."""
    if not kw:
        _check(lib().hss_set_tuning(None))
        return
    t = hss_tuning()
    _check(lib().hss_get_tuning(C.byref(t)))
    for k, v in kw.items():
        setattr(t, k, int(v))
    _check(lib().hss_set_tuning(C.byref(t)))


class HSSError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{lib().hss_status_str(status).decode()}: {msg}")
        self.status = status


def _check(status):
    if status != HSS_OK:
        msg = lib().hss_last_error().decode()
        if status == HSS_ERR_OPERATOR:   # the caller's callback raised: say what
            cause = last_extract_error if "extraction" in msg else last_operator_error
            if cause is not None:
                msg += f" ({type(cause).__name__}: {cause})"
        raise HSSError(status, msg)
    return status


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        return None
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else stream


# ------------------------------------------------------------------ wrappers
def make_source(kind, n, a, b=None, ld=0, dim=0, p0=0.0, p1=0.0):
    """hss_source over device tensors (kept alive by the returned object)."""
    s = hss_source(kind, n, dim, 0, _ptr(a), _ptr(b), ld, p0, p1)
    s._keep = (a, b)
    return s


last_extract_error = None


def _device_ints(ptr, count):
    """A view of `count` int32 entries of device memory owned by the library."""
    import torch

    class _View:
        __cuda_array_interface__ = {"shape": (count,), "strides": None, "typestr": "<i4",
                                    "data": (ptr, False), "version": 3}
    return torch.as_tensor(_View(), device="cuda")


def extract_source(n, fn):
    """hss_source of kind HSS_SRC_EXTRACT around fn(blocks, stream): blocks is
    a list of (I, J, out) per requested block — I, J int32 device views of
    the global indices, out a column-major view of the library's buffer — and
    stream the library's stream (made current); fn enqueues
    out[i, j] = A[I[i], J[j]] for every block.  An exception becomes a
    nonzero status (HSS_ERR_OPERATOR); it is kept in last_extract_error."""
    import torch

    def cb(ctx, nblocks, blocks, stream):
        global last_extract_error
        try:
            st = torch.cuda.ExternalStream(stream) if stream else torch.cuda.default_stream()
            with torch.cuda.stream(st):
                req = []
                for q in range(nblocks):
                    b = blocks[q]
                    req.append((_device_ints(b.I, b.nr), _device_ints(b.J, b.nc),
                                _device_matrix(b.out, b.nr, b.nc, b.ldo)))
                fn(req, st)
            return 0
        except Exception as e:   # the status carries the failure back through the C ABI
            last_extract_error = e
            return 1

    c = EXTRACT_FN(cb)
    s = hss_source(HSS_SRC_EXTRACT, n, 0, 0, None, None, 0, 0.0, 0.0, c, None)
    s._keep = (c, fn)
    return s


def make_opts(leaf, rtol, atol, d0, dd, d_max, strategy, precision=HSS_PREC_FP64, p=10, seed=0,
              R=None, level_tol_scaling=1, symmetric=0, criterion=0, hmt_alpha=10.0, op=None,
              wait_limit_ns=0):
    o = hss_opts(leaf, strategy, precision, level_tol_scaling, rtol, atol, d0, dd, d_max, p,
                 seed, _ptr(R), int(symmetric), int(criterion), float(hmt_alpha),
                 C.pointer(op) if op is not None else None, int(wait_limit_ns))
    o._keep = (R, op)
    return o


def _device_matrix(ptr, rows, cols, ld):
    """A column-major rows x cols view (leading dimension ld) of FP64 device
    memory owned by the library."""
    import torch

    class _View:
        __cuda_array_interface__ = {"shape": (rows, cols), "strides": (8, 8 * ld), "typestr": "<f8",
                                    "data": (ptr, False), "version": 3}
    return torch.as_tensor(_View(), device="cuda")


last_operator_error = None


def make_operator(fn):
    """hss_operator around fn(trans, R, S, stream): R and S are n x ncols
    column-major views of the library's buffers and stream the library's
    stream (made current); fn enqueues S = A R (trans 0) or S = A^T R
    (trans 1).  An exception becomes a nonzero status (HSS_ERR_OPERATOR);
    it is kept in last_operator_error."""
    import torch

    def cb(ctx, trans, n, ncols, R, ldr, S, lds, stream):
        global last_operator_error
        try:
            st = torch.cuda.ExternalStream(stream) if stream else torch.cuda.default_stream()
            with torch.cuda.stream(st):
                fn(trans, _device_matrix(R, n, ncols, ldr), _device_matrix(S, n, ncols, lds), st)
            return 0
        except Exception as e:   # the status carries the failure back through the C ABI
            last_operator_error = e
            return 1

    c = APPLY_FN(cb)
    op = hss_operator(c, None)
    op._keep = (c, fn)
    return op


def hss_compress(source, opts, stream=None, allow_not_converged=False):
    """Returns an HSSMatrix; raises HSSError on failure."""
    h = C.c_void_p()
    st = lib().hss_compress(C.byref(source), C.byref(opts), _stream(stream), C.byref(h))
    if st == HSS_ERR_NOT_CONVERGED and h.value and allow_not_converged:
        return HSSMatrix(h.value, converged=False)
    _check(st)
    return HSSMatrix(h.value)


def hss_compress_restart(source, opts, stream=None, allow_not_converged=False):
    """The hard-restart mode; returns (HSSMatrix, number of restarts)."""
    h = C.c_void_p()
    k = C.c_int(0)
    st = lib().hss_compress_restart(C.byref(source), C.byref(opts), _stream(stream), C.byref(h), C.byref(k))
    if st == HSS_ERR_NOT_CONVERGED and h.value and allow_not_converged:
        return HSSMatrix(h.value, converged=False), k.value
    _check(st)
    return HSSMatrix(h.value), k.value


def hss_save(H, path):
    """Write H's generators to the file `path` (a checkpoint)."""
    _check(lib().hss_save(H.handle, os.fsencode(path)))


def hss_load(path):
    """A new handle on the current device from a checkpoint file."""
    h = C.c_void_p()
    _check(lib().hss_load(os.fsencode(path), C.byref(h)))
    return HSSMatrix(h.value)


def hss_release_cached():
    """Return the device memory cached from freed handles (current device)."""
    _check(lib().hss_release_cached())


def hss_to_dense(H, out, stream=None):
    """out (n x n device tensor, column-major) = H."""
    if out.stride(0) != 1:
        raise ValueError("hss_to_dense needs a column-major out (stride(0) == 1)")
    _check(lib().hss_to_dense(H.handle, _ptr(out), out.stride(1), _stream(stream)))


def hss_matvec(H, X, Y, stream=None, transpose=False):
    """Y = H X (or H^T X); X, Y column-major device tensors."""
    if X.dim() == 2 and (X.stride(0) != 1 or Y.stride(0) != 1):
        raise ValueError("hss_matvec needs column-major X and Y (stride(0) == 1)")
    n, nrhs = X.shape[0], (X.shape[1] if X.dim() == 2 else 1)
    ldx = X.stride(1) if X.dim() == 2 else n
    ldy = Y.stride(1) if Y.dim() == 2 else n
    _check(lib().hss_matvec(H.handle, nrhs, _ptr(X), ldx, _ptr(Y), ldy, int(bool(transpose)), _stream(stream)))


def hss_get_entries(H, I, J, out, stream=None):
    """out (len(I) x len(J), column-major device tensor) = H[I, J]; I, J
    int32 device tensors."""
    if out.dim() != 2 or (out.stride(0) != 1 and out.shape[0] > 1):
        raise ValueError("hss_get_entries needs a column-major 2-D out")
    _check(lib().hss_get_entries(H.handle, I.numel(), _ptr(I), J.numel(), _ptr(J), _ptr(out),
                                 max(out.stride(1), out.shape[0], 1), _stream(stream)))


def hss_rcb_order(points: np.ndarray, leaf: int) -> np.ndarray:
    P = np.asfortranarray(points, dtype=np.float64)
    n, dim = P.shape
    perm = np.empty(n, dtype=np.int32)
    _check(lib().hss_rcb_order(P.ctypes.data, n, dim, n, leaf, perm.ctypes.data))
    return perm.astype(np.int64)


def hss_random_normal(seed, n, col0, ncols, R, round_mode=0, stream=None):
    _check(lib().hss_random_normal(seed, n, col0, ncols, _ptr(R), R.stride(1) if R.dim() == 2 else n,
                                   round_mode, _stream(stream)))


def hss_sample_offdiag(source, leaf, precision, R, Sr, Sc, stream=None):
    ncols = R.shape[1]
    lds = (Sr if Sr is not None else Sc).stride(0)
    _check(lib().hss_sample_offdiag(C.byref(source), leaf, precision, ncols, _ptr(R), R.stride(1),
                                    _ptr(Sr), _ptr(Sc), lds, _stream(stream)))


def hss_sample_offdiag_noalloc(source, leaf, precision, R, Sr, Sc, stream=None):
    """hss_sample_offdiag for callers that cannot have the library allocate
    device memory (the leaf table lives in a fixed array inside the library,
    n <= 2^20; overlapping calls race on it)."""
    ncols = R.shape[1]
    lds = (Sr if Sr is not None else Sc).stride(0)
    _check(lib().hss_sample_offdiag_noalloc(C.byref(source), leaf, precision, ncols, _ptr(R),
                                            R.stride(1), _ptr(Sr), _ptr(Sc), lds, _stream(stream)))


def hss_compress_batched(sources, opts, stream=None, allow_not_converged=False):
    """One HSSMatrix per (source, opts) pair, compressed side by side."""
    n = len(sources)
    if len(opts) != n:
        raise ValueError("one opts per source")
    src_arr = (hss_source * n)(*sources)
    opt_arr = (hss_opts * n)(*opts)
    hs = (C.c_void_p * n)()
    st = lib().hss_compress_batched(src_arr, opt_arr, n, _stream(stream), hs)
    if not (st == HSS_ERR_NOT_CONVERGED and allow_not_converged):
        _check(st)
    out = [HSSMatrix(h) for h in hs]
    for m in out:
        m.converged = bool(m.stats().converged)
    return out


class HSSMatrix:
    def __init__(self, handle, converged=True):
        self.handle = handle
        self.converged = converged

    def __del__(self):
        if getattr(self, "handle", None):
            try:
                lib().hss_free(self.handle)
            except Exception:
                pass
            self.handle = None

    def stats(self) -> hss_stats:
        s = hss_stats()
        _check(lib().hss_get_stats(self.handle, C.byref(s)))
        return s

    def node(self, i) -> hss_node_info:
        inf = hss_node_info()
        _check(lib().hss_get_node(self.handle, i, C.byref(inf)))
        return inf

    def export_node(self, i) -> dict:
        inf = self.node(i)
        out = dict(info=inf)
        kr, kc, mr, mc = inf.kr, inf.kc, inf.mr, inf.mc
        comp = inf.state == HSS_COMPRESSED and i != 0
        Jr = np.zeros(max(kr, 1), np.int32); Jc = np.zeros(max(kc, 1), np.int32)
        Pr = np.zeros(max(mr, 1), np.int32); Pc = np.zeros(max(mc, 1), np.int32)
        Xr = np.zeros((max(kr, 1), max(mr - kr, 1)), order="F")
        Xc = np.zeros((max(kc, 1), max(mc - kc, 1)), order="F")
        Ir = np.zeros(max(kr, 1), np.int32); Ic = np.zeros(max(kc, 1), np.int32)
        leaf = inf.child0 < 0
        D = np.zeros((inf.size, inf.size), order="F") if leaf else None
        B12 = B21 = None
        if not leaf and inf.state == HSS_COMPRESSED:
            a, b = self.node(inf.child0), self.node(inf.child1)
            B12 = np.zeros((max(a.kr, 1), max(b.kc, 1)), order="F")
            B21 = np.zeros((max(b.kr, 1), max(a.kc, 1)), order="F")
        args = [Jr, Jc, Pr, Pc, Xr, Xc, Ir, Ic] if comp else [None] * 8
        _check(lib().hss_export_node(self.handle, i, *[_ptr(x) for x in args], _ptr(D), _ptr(B12),
                                     _ptr(B21)))
        if comp:
            out.update(Jr=Jr[:kr].astype(np.int64), Jc=Jc[:kc].astype(np.int64),
                       Pr=Pr[:mr].astype(np.int64), Pc=Pc[:mc].astype(np.int64),
                       Xr=Xr.ravel(order="F")[:kr * (mr - kr)].reshape((kr, mr - kr), order="F"),
                       Xc=Xc.ravel(order="F")[:kc * (mc - kc)].reshape((kc, mc - kc), order="F"),
                       Ir=Ir[:kr].astype(np.int64), Ic=Ic[:kc].astype(np.int64))
        if D is not None:
            out["D"] = D
        if B12 is not None:
            a, b = self.node(inf.child0), self.node(inf.child1)
            out["B12"] = B12.ravel(order="F")[:a.kr * b.kc].reshape((a.kr, b.kc), order="F")
            out["B21"] = B21.ravel(order="F")[:b.kr * a.kc].reshape((b.kr, a.kc), order="F")
        return out

    def ranks(self) -> dict:
        st = self.stats()
        return {i: (self.node(i).kr, self.node(i).kc) for i in range(1, st.n_nodes)}


# ------------------------------------------------------- source constructors
def dense_source(A):
    """A: device float64 tensor holding A column-major (e.g. a transposed
    contiguous tensor, ``A_t.t()`` with ``A_t`` row-major A^T)."""
    n = A.shape[0]
    ld = A.stride(1) if A.dim() == 2 else n
    return make_source(HSS_SRC_DENSE, n, A, None, ld)


def toeplitz_source(col, row=None):
    return make_source(HSS_SRC_TOEPLITZ, col.shape[0], col, row if row is not None else col)


def points_source(kind, P, p0, p1=0.0):
    """P: device float64 tensor n x dim stored column-major (stride(0) == 1)."""
    n, dim = P.shape
    assert P.stride(0) == 1
    return make_source(kind, n, P, None, P.stride(1), dim, p0, p1)
