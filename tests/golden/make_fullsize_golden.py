"""Oracle results at the benchmark sizes, for the full-size parity test.

Writes ``tests/golden/fullsize_<case>.txt`` from the plain CPU oracle alone
(``oracle/`` and ``workloads/``; nothing of the CUDA library is imported or
run): the passes (d_final, adaptations), every node's ranks, the number of
singular values of each node's sample within 10 % of its rank threshold
(the tie rule of the rank comparison), the same count for the diagonal of
the node's full QRCP (|R_jj| near the threshold: the ID rule's own
decision quantity) and, for the cases whose GPU form samples in TF32 x 2,
both counts with the band widened by the tested bound of the mixed sampling
error (5e-7 of the rows of the sample the node's local sample is formed
from; Weyl's inequality for the singular values), the error
||A - H||_F / ||A||_F (paper section 4.4.1) and the oracle's wall time on
this host.

Cases (the workloads of the benchmark, with R drawn by the Philox generator
of ``workloads`` and rounded once to TF32 where the GPU form samples in
TF32 x 2, reading P10):
  c2_tf32  Gaussian kernel exp(-|x-y|^2/2) + I, n = 16384 points uniform in
           [0,1]^8 ordered by RCB, leaf 128, rtol 1e-4, atol 1e-8, Doubling
           from d0 = 128, d_max 4096, p = 10; R rounded to TF32
  c2_fp64  the same with the FP64 R
  c5_tf32  Toeplitz cos(0.3 k)/(1 + k), n = 131072 (entries generated),
           leaf 256, rtol 1e-4, atol 1e-10, Incrementing d0 = 256, dd = 128,
           d_max 1024; R rounded to TF32

Usage:  python tests/golden/make_fullsize_golden.py c2_tf32 [c2_fp64 c5_tf32 ...]
"""
from __future__ import annotations

import os
import platform
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as w  # noqa: E402
from oracle import apply, qrcp  # noqa: E402
from oracle.hss import Options, compress  # noqa: E402
from oracle.tree import rcb_order  # noqa: E402

MIXED_NOISE = 5e-7   # tested bound of the TF32 x 2 / BF16 x 3 sampling error, relative


def case(name):
    if name.startswith("c2"):
        n, leaf = 16384, 128
        P = w.uniform_points(n, 8, seed=0)
        src = w.gaussian_kernel(P[rcb_order(P, leaf)], 1.0, 1.0)
        o = Options(leaf=leaf, rtol=1e-4, atol=1e-8, d0=128, dd=128, d_max=4096, strategy="doubling", p=10)
        desc = ("Gaussian kernel exp(-|x-y|^2/2) + I, n = 16384 uniform points in [0,1]^8 (seed 0), RCB order, "
                "leaf 128, rtol 1e-4, atol 1e-8, Doubling d0 = 128, d_max = 4096, p = 10")
    elif name.startswith("c5"):
        n, leaf = 131072, 256
        src = w.toeplitz_cos(n)
        o = Options(leaf=leaf, rtol=1e-4, atol=1e-10, d0=256, dd=128, d_max=1024, strategy="incrementing")
        desc = ("Toeplitz cos(0.3k)/(1+k), n = 131072 generated, leaf 256, rtol 1e-4, atol 1e-10, "
                "Incrementing d0 = 256, dd = 128, d_max = 1024")
    else:
        raise SystemExit(f"unknown case {name}")
    R = w.gaussian_matrix(0, src.n, 0, o.d_max)
    if name.endswith("tf32"):
        R = w.round_to_tf32(R)
        desc += "; R = Philox seed 0 rounded to TF32"
    else:
        desc += "; R = Philox seed 0 (FP64)"
    return src, o, R, desc


def sample_row_norms(src, R, res):
    """norms(t, side): the Frobenius norm of the rows of the global sample
    (A - D^(L)) R (or its transpose's) at a node's sample rows and its ID's
    columns: the sampling error reaches a local sample only through those
    rows (the merges subtract exactly formed terms)."""
    n, d = src.n, R.shape[1]
    leaf_of = np.empty(n, dtype=np.int64)
    for t in res.nodes:
        if t.is_leaf:
            leaf_of[t.lo:t.lo + t.size] = t.idx
    Sr = np.zeros((n, d))
    Sc = np.zeros((n, d))
    idx = np.arange(n)
    step = max(1, (1 << 24) // n)
    for i0 in range(0, n, step):
        rows = idx[i0:i0 + step]
        blk = src.entries(rows, idx)
        blk[leaf_of[rows][:, None] == leaf_of[None, :]] = 0.0      # the leaf blocks D
        Sr[rows] = blk @ R
        Sc += blk.T @ R[rows]

    def norms(t, side):
        if t.is_leaf:
            rows = t.I
        else:
            c1, c2 = (res.nodes[c] for c in t.children)
            rows = np.concatenate([c1.Ir, c2.Ir] if side == "r" else [c1.Ic, c2.Ic])
        return float(np.linalg.norm((Sr if side == "r" else Sc)[rows, :t.d_id]))

    return norms


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def main(names):
    for name in names:
        src, o, R, desc = case(name)
        t0 = time.time()
        res = compress(src, R, o)
        t_compress = time.time() - t0
        err = apply.rel_error_blocks(res, src)
        n = src.n
        lines = [f"# oracle compression at full size: {desc}",
                 f"# written by: python tests/golden/make_fullsize_golden.py {name}",
                 f"# host: {os.cpu_count()} cores, {cpu_model()}; oracle compression {t_compress:.1f} s",
                 f"case {name}", f"n {n}", f"leaf {o.leaf}", f"converged {int(res.converged)}",
                 f"d_final {res.d_final}", f"n_adapt {res.n_adapt}", f"rel_error {err:.6e}",
                 f"oracle_seconds {t_compress:.1f}", f"cores {os.cpu_count()}",
                 "# node level kr kc near_r near_c near_mixed_r near_mixed_c d_id "
                 "qr_near_r qr_near_c qr_near_mixed_r qr_near_mixed_c"]
        rule = "hmt" if o.strategy == "doubling" else "plain"
        norms = sample_row_norms(src, R, res) if name.endswith("tf32") else None
        for t in res.nodes[1:]:
            if t.Jr is None:
                continue
            scale = 1.0 / t.level if o.level_tol_scaling else 1.0
            er, ea = o.rtol * scale, o.atol * scale
            near, near_m, qnear, qnear_m = [], [], [], []
            for side, S in (("r", t.Sr), ("c", t.Sc)):
                S = S[:, :t.d_id]
                near.append(qrcp.near_threshold_count(S, er, ea, rule, t.size, n - t.size))
                qnear.append(qrcp.near_threshold_count_qr(S, er, ea, rule, t.size, n - t.size))
                if norms is None:
                    near_m.append(near[-1])
                    qnear_m.append(qnear[-1])
                else:
                    noise = MIXED_NOISE * norms(t, side)
                    near_m.append(qrcp.near_threshold_count(S, er, ea, rule, t.size, n - t.size, noise=noise))
                    qnear_m.append(qrcp.near_threshold_count_qr(S, er, ea, rule, t.size, n - t.size, noise=noise))
            lines.append(f"{t.idx} {t.level} {len(t.Jr)} {len(t.Jc)} {near[0]} {near[1]} {near_m[0]} {near_m[1]} "
                         f"{t.d_id} {qnear[0]} {qnear[1]} {qnear_m[0]} {qnear_m[1]}")
        path = os.path.join(HERE, f"fullsize_{name}.txt")
        open(path, "w").write("\n".join(lines) + "\n")
        print(f"{name}: d_final {res.d_final}, adaptations {res.n_adapt}, max rank {res.max_rank()}, "
              f"error {err:.3e}, {t_compress:.1f} s -> {path}", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["c2_tf32"])
