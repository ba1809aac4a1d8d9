"""The benchmark workloads at full size against the oracle's compression of
the same matrices on the same R, stored by tests/golden/make_fullsize_golden.py
(which runs the oracle alone): Gaussian kernel 8-D, n = 16384 dense,
Doubling, TF32 x 2 sampling (the benchmark configuration), and the FP64
form of it when its file is there.  Required: the same passes, every node's
ranks equal except across singular values within the tie band (widened by
the tested bound of the mixed sampling error for the TF32 x 2 form), and an
error ||A - H||_F / ||A||_F within 1.1x the oracle's."""
import os

import numpy as np
import pytest

import workloads as w
from oracle.tree import rcb_order

import gpu_util as gu

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_golden(name):
    path = os.path.join(GOLDEN, f"fullsize_{name}.txt")
    if not os.path.exists(path):
        return None
    kv, nodes = {}, {}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        if len(f) == 2:
            kv[f[0]] = f[1]
        else:
            idx, lev, kr, kc, nr, nc, nmr, nmc, d_id = (int(x) for x in f)
            nodes[idx] = dict(level=lev, kr=kr, kc=kc, near=(nr, nc), near_mixed=(nmr, nmc), d_id=d_id)
    return kv, nodes


@pytest.mark.parametrize("name,prec", [("c2_tf32", "tf32x2"), ("c2_fp64", "fp64")])
def test_benchmark_configuration_against_oracle(name, prec):
    g = read_golden(name)
    if g is None:
        pytest.skip(f"no golden file for {name}")
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1810_04125_gb300 import build, hss
    build.build()
    kv, nodes = g
    n, leaf = int(kv["n"]), int(kv["leaf"])
    P = w.uniform_points(n, 8, seed=0)
    A = w.gaussian_kernel(P[rcb_order(P, leaf)], 1.0, 1.0).to_dense()
    R = w.gaussian_matrix(0, n, 0, 4096)
    if prec == "tf32x2":
        R = w.round_to_tf32(R)
    Ad = gu.col_major(A)
    opts = hss.make_opts(leaf, 1e-4, 1e-8, 128, 128, 4096, hss.HSS_DOUBLING, gu.PREC[prec], 10, 0, gu.col_major(R))
    H = hss.hss_compress(hss.dense_source(Ad), opts)
    st = H.stats()
    assert st.converged == int(kv["converged"]) == 1
    assert (st.d_final, st.n_adapt) == (int(kv["d_final"]), int(kv["n_adapt"]))
    key = "near_mixed" if prec != "fp64" else "near"
    bad, diffs = [], []
    for i, (kr, kc) in H.ranks().items():
        ref = nodes[i]
        for k_g, k_o, band in ((kr, ref["kr"], ref[key][0]), (kc, ref["kc"], ref[key][1])):
            diffs.append(abs(k_g - k_o))
            if abs(k_g - k_o) > band:
                bad.append((i, k_g, k_o, band))
    print(f"{name}: {len(diffs)} node sides, rank differences: max {max(diffs)}, "
          f"sum {sum(diffs)}, nonzero {sum(1 for x in diffs if x)}")
    assert not bad, bad
    # the error on the whole matrix, from the expansion on the GPU
    D = torch.empty((n, n), dtype=torch.float64, device=gu.dev()).t()
    hss.hss_to_dense(H, D)
    err = float(torch.linalg.norm(D - Ad) / torch.linalg.norm(Ad))
    print(f"{name}: error {err:.4e}, oracle {float(kv['rel_error']):.4e}")
    assert err <= 1.1 * float(kv["rel_error"]), (err, kv["rel_error"])
