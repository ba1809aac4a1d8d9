"""Launch-shape autotuner.

Times the candidate values of the hss_tuning parameters on representative
compressions on the GPU at hand and writes the fastest to
tuning_sm103.json beside this file; the binding applies that table when it
loads the library.  Only launch shapes change: every candidate computes the
same method (rounding aside).

  python -m paper_1810_04125_gb300.tune [--out PATH] [--reps K]

Workloads (synthetic, seeded):
  * dense Gaussian kernel exp(-|x - y|^2 / 2) + I on 16384 points uniform in
    [0, 1]^8 (seed 0), recursive-coordinate-bisection order, leaf 128,
    TF32x2 sampling, Doubling from 128 at rtol 1e-4: the QRCP shapes (CTAs
    per SM, ID phase time) and the K split of the packed sampling kernel (sampling
    phase time);
  * Toeplitz cos(0.3 k) / (1 + k), n = 131072, generated entries, leaf 256,
    TF32x2 sampling, Incrementing from 256 by 128 at rtol 1e-4: the K split
    of the generated-entry sampling kernel (sampling phase time).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics

import numpy as np


def _gauss_dense(hss, torch, n, dim, seed, leaf):
    pts = np.random.default_rng(seed).random((n, dim))
    pts = pts[hss.hss_rcb_order(pts, leaf)]
    X = torch.from_numpy(np.ascontiguousarray(pts)).cuda()
    A = torch.empty((n, n), dtype=torch.float64, device="cuda")
    for j0 in range(0, n, 2048):
        A[j0:j0 + 2048] = torch.exp(-torch.cdist(X[j0:j0 + 2048], X,
                                                 compute_mode="donot_use_mm_for_euclid_dist") ** 2 / 2.0)
    A.diagonal().add_(1.0)
    return A


def _phase_ms(hss, torch, src, opts, reps):
    """Median over `reps` compressions (after one warm-up) of the ID and
    sampling phase times (CUDA events inside the library)."""
    H = hss.hss_compress(src, opts)
    del H
    ids, samples = [], []
    for _ in range(reps):
        H = hss.hss_compress(src, opts)
        st = H.stats()
        ids.append(st.ms_id)
        samples.append(st.ms_sample)
        del H
    torch.cuda.synchronize()
    return statistics.median(ids), statistics.median(samples)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning_sm103.json"))
    ap.add_argument("--reps", type=int, default=3)
    args = ap.parse_args()
    import torch

    from . import build
    build.build()
    from . import hss
    hss.set_tuning()   # start from the defaults
    meas = {}
    A = _gauss_dense(hss, torch, 16384, 8, 0, 128)
    src = hss.dense_source(A.t())
    opts = hss.make_opts(128, 1e-4, 1e-8, 128, 128, 4096, hss.HSS_DOUBLING, hss.HSS_PREC_TF32X2, 10, 0)
    cand = {}
    for c in (4, 8, 16):
        hss.set_tuning(qrcp_wide_max_sides=c)
        cand[c] = _phase_ms(hss, torch, src, opts, args.reps)[0]
    best_q = min(cand, key=cand.get)
    meas["qrcp_wide_max_sides_ms_id"] = cand
    hss.set_tuning(qrcp_wide_max_sides=best_q)
    cand = {}
    for c in (0, 1, 2, 4):
        hss.set_tuning(qrcp_sm_ctas=c)
        cand[c] = _phase_ms(hss, torch, src, opts, args.reps)[0]
    best_s = min(cand, key=cand.get)
    meas["qrcp_sm_ctas_ms_id"] = cand
    hss.set_tuning(qrcp_sm_ctas=best_s)
    cand = {}
    for c in (4, 16, 32, 64, 128):
        hss.set_tuning(qrcp_min_cols=c)
        cand[c] = _phase_ms(hss, torch, src, opts, args.reps)[0]
    best_mc = min(cand, key=cand.get)
    meas["qrcp_min_cols_ms_id"] = cand
    hss.set_tuning(qrcp_min_cols=best_mc)
    cand = {}
    for c in (1, 2, 4, 8):
        hss.set_tuning(sample_waves_packed=c)
        cand[c] = _phase_ms(hss, torch, src, opts, args.reps)[1]
    best_p = min(cand, key=cand.get)
    meas["sample_waves_packed_ms_sample"] = cand
    hss.set_tuning(sample_waves_packed=best_p)
    del src, A
    torch.cuda.empty_cache()
    n = 131072
    k = torch.arange(n, dtype=torch.float64, device="cuda")
    coef = torch.cos(0.3 * k) / (1.0 + k)
    tsrc = hss.toeplitz_source(coef, coef)
    topts = hss.make_opts(256, 1e-4, 1e-10, 256, 128, 1024, hss.HSS_INCREMENTING, hss.HSS_PREC_TF32X2, 10, 0)
    cand = {}
    for c in (1, 2, 4):
        hss.set_tuning(sample_waves_generated=c)
        cand[c] = _phase_ms(hss, torch, tsrc, topts, max(1, args.reps - 1))[1]
    best_g = min(cand, key=cand.get)
    meas["sample_waves_generated_ms_sample"] = cand
    out = {"qrcp_wide_max_sides": best_q, "sample_waves_packed": best_p, "sample_waves_generated": best_g,
           "qrcp_min_cols": best_mc, "qrcp_sm_ctas": best_s,
           "device": torch.cuda.get_device_name(), "measured_ms": meas}
    with open(args.out, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
