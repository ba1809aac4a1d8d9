"""CUDA path against the CPU oracle, element by element where the result is
unique (random matrix, samples, extracted blocks) and by rank / error where
pivot ties may legitimately differ (paper section 2.2: the ID is defined by
a greedy pivot choice)."""
import math

import numpy as np
import pytest

import workloads as w
from oracle import apply, hss as ohss, tree as otree
from oracle.hss import Options, compress

import gpu_util as gu

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


# --------------------------------------------------------------- random R
@pytest.mark.parametrize("round_mode", [0, 1, 2])
def test_random_normal_matches_generator(hss, torch, round_mode):
    n, c0, nc = 1001, 5, 37
    R = torch.zeros((nc, n), dtype=torch.float64, device=gu.dev()).t()
    hss.hss_random_normal(12345, n, c0, nc, R, round_mode)
    torch.cuda.synchronize()
    got = R.cpu().numpy()
    ref = w.gaussian_matrix(12345, n, c0, nc)
    if round_mode == 0:
        np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-15)
    else:
        rnd = w.round_to_tf32 if round_mode == 1 else w.round_to_bf16
        frac = np.mean(got == rnd(ref))
        assert frac > 0.999, frac
        np.testing.assert_allclose(got, rnd(ref), rtol=2.0 ** (-10 if round_mode == 1 else -7))


# --------------------------------------------------------------- sampling
def _rcb(P, leaf):
    return P[otree.rcb_order(P, leaf)]


SOURCES = [
    ("dense", lambda: w.dense_source(np.random.default_rng(4).standard_normal((700, 700))), 64),
    ("toeplitz", lambda: w.toeplitz_inverse_distance(1000), 64),
    ("toeplitz_cos", lambda: w.toeplitz_cos(1500), 100),
    ("gauss", lambda: w.gaussian_kernel(_rcb(w.uniform_points(1200, 8, seed=2), 128), 1.0, 1.0), 128),
    ("laplace", lambda: w.laplace_kernel(_rcb(w.fibonacci_sphere(1300), 100)), 100),
]


@pytest.mark.parametrize("name,mk,leaf", SOURCES, ids=[s[0] for s in SOURCES])
def test_sample_offdiag_parity(hss, torch, name, mk, leaf):
    src = mk()
    n, nc = src.n, 70
    R = w.gaussian_matrix(3, n, 0, nc)
    Rd = gu.col_major(R)
    Sr = torch.full((n, nc), float("nan"), dtype=torch.float64, device=gu.dev())
    Sc = torch.full((n, nc), float("nan"), dtype=torch.float64, device=gu.dev())
    hss.hss_sample_offdiag(gu.device_source(src), leaf, 0, Rd, Sr, Sc)
    torch.cuda.synchronize()
    # oracle: S = A R, then the leaf diagonal blocks' D R removed (Algorithm 2)
    smp = ohss._Sampler(src)
    er, ec = smp.sample(R)
    A = src.to_dense()
    absA = np.abs(A).copy()
    for t in otree.halving_tree(n, leaf):
        if t.is_leaf:
            I = t.I
            D = smp.entries(I, I)
            er[I] -= D @ R[I]
            ec[I] -= D.T @ R[I]
            absA[np.ix_(I, I)] = 0.0
    bound_r = 1e-13 * (absA @ np.abs(R)) + 1e-300
    bound_c = 1e-13 * (absA.T @ np.abs(R)) + 1e-300
    assert np.all(np.abs(Sr.cpu().numpy() - er) <= bound_r + 1e-12 * np.abs(er))
    assert np.all(np.abs(Sc.cpu().numpy() - ec) <= bound_c + 1e-12 * np.abs(ec))


# ----------------------------------------------------------- compression
def _cases():
    c = []
    c.append(("toeplitz1024_inc", lambda: w.toeplitz_inverse_distance(1024),
              Options(leaf=64, rtol=1e-6, atol=1e-12, d0=64, dd=32, d_max=1024)))
    c.append(("toeplitz1024_dbl", lambda: w.toeplitz_inverse_distance(1024),
              Options(leaf=64, rtol=1e-6, atol=1e-12, d0=64, dd=32, d_max=1024, strategy="doubling")))
    c.append(("toeplitz1024_inc_adapt", lambda: w.toeplitz_inverse_distance(1024),
              Options(leaf=64, rtol=1e-6, atol=1e-12, d0=16, dd=8, d_max=1024)))
    c.append(("gauss8_2048_dbl", lambda: w.gaussian_kernel(
        (lambda P: P[otree.rcb_order(P, 128)])(w.uniform_points(2048, 8, 0)), 1.0, 1.0),
        Options(leaf=128, rtol=1e-4, atol=1e-8, d0=64, dd=64, d_max=2048, strategy="doubling")))
    c.append(("laplace2048_inc", lambda: w.laplace_kernel(
        (lambda P: P[otree.rcb_order(P, 128)])(w.fibonacci_sphere(2048))),
        Options(leaf=128, rtol=1e-6, atol=1e-8, d0=64, dd=32, d_max=2048)))
    c.append(("toeplitzcos4096_inc", lambda: w.toeplitz_cos(4096),
              Options(leaf=256, rtol=1e-4, atol=1e-10, d0=128, dd=64, d_max=1024)))
    c.append(("udv1000_ragged_inc", lambda: w.dense_source(w.udv_matrix(1000, 60, seed=3)),
              Options(leaf=64, rtol=1e-8, atol=1e-14, d0=32, dd=16, d_max=1000)))
    # 256 leaves: the leaf level has more node sides than SMs (one CTA per
    # node side), the upper levels use CTA groups
    c.append(("toeplitz4096_leaf16_dbl", lambda: w.toeplitz_power(4096, 1.5),
              Options(leaf=16, rtol=1e-8, atol=1e-14, d0=32, dd=32, d_max=1024, strategy="doubling")))
    return c


@pytest.mark.parametrize("name,mk,o", _cases(), ids=[x[0] for x in _cases()])
def test_compress_parity(hss, torch, name, mk, o):
    src = mk()
    n = src.n
    R = w.gaussian_matrix(7, n, 0, o.d_max)
    ref = compress(src, R, o)
    H = gu.gpu_compress(src, R, o)
    st = H.stats()
    assert st.converged == 1 and ref.converged
    assert st.d_final == ref.d_final and st.n_adapt == ref.n_adapt
    bad = gu.compare_with_oracle(H, ref, o, n)
    assert not bad, bad
    A = src.to_dense()
    err_g = gu.rel_err(A, gu.gpu_dense(H, n))
    err_o = apply.rel_error(ref, A)
    assert err_g <= 1.1 * err_o + 1e-15, (err_g, err_o)


@pytest.mark.parametrize("strategy", ["incrementing", "doubling"])
def test_synthetic_hss_exact_ranks_gpu(hss, torch, strategy):
    n, leaf = 1024, 64
    ranks = {4: 8, 3: 12, 2: 16, 1: 20}
    A = w.synthetic_hss(n, leaf, ranks, seed=3)
    o = Options(leaf=leaf, rtol=1e-10, atol=1e-14, d0=8, dd=8, d_max=512, strategy=strategy)
    R = w.gaussian_matrix(5, n, 0, 512)
    H = gu.gpu_compress(w.dense_source(A), R, o)
    for i, (kr, kc) in H.ranks().items():
        lev = H.node(i).level
        assert kr == kc == ranks[lev], (i, kr, kc)
    assert gu.rel_err(A, gu.gpu_dense(H, n)) < 1e-12


def test_generators_and_matvec(hss, torch):
    """B blocks are exact sub-blocks of A at the skeleton indices, the
    skeleton rows compose as [I^r_nu1 I^r_nu2](J^r), and the GPU product
    equals the oracle's plain expansion of the same generators."""
    n, leaf = 1000, 64
    A = w.udv_matrix(n, 40, seed=9)
    o = Options(leaf=leaf, rtol=1e-8, atol=1e-14, d0=48, dd=16, d_max=512)
    H = gu.gpu_compress(w.dense_source(A), w.gaussian_matrix(2, n, 0, 512), o)
    res = gu.expand_exported(H, n, leaf)
    for t in res.nodes:
        if t.is_leaf:
            assert np.array_equal(t.D, A[t.lo:t.lo + t.size, t.lo:t.lo + t.size])
            if t.idx:
                assert np.array_equal(t.Ir, t.lo + t.Jr) and np.array_equal(t.Ic, t.lo + t.Jc)
            continue
        a, b = (res.nodes[c] for c in t.children)
        assert np.array_equal(t.B12, A[np.ix_(a.Ir, b.Ic)])
        assert np.array_equal(t.B21, A[np.ix_(b.Ir, a.Ic)])
        if t.idx:
            assert np.array_equal(t.Ir, np.concatenate([a.Ir, b.Ir])[t.Jr])
            assert np.array_equal(t.Ic, np.concatenate([a.Ic, b.Ic])[t.Jc])
    Hd = apply.to_dense(res)
    G = gu.gpu_dense(H, n)
    np.testing.assert_allclose(G, Hd, rtol=0, atol=1e-12 * np.abs(Hd).max())
    # a few right-hand sides with a leading dimension larger than n
    X = np.random.default_rng(1).standard_normal((n, 5))
    Xd = torch.zeros((5, n + 3), dtype=torch.float64, device=gu.dev()).t()[:n]
    Xd.copy_(torch.from_numpy(X))
    Yd = torch.zeros((5, n + 7), dtype=torch.float64, device=gu.dev()).t()[:n]
    hss.hss_matvec(H, Xd, Yd)
    torch.cuda.synchronize()
    np.testing.assert_allclose(Yd.cpu().numpy(), Hd @ X, rtol=0, atol=1e-11 * np.abs(Hd @ X).max())
    # hss_to_dense, into a buffer with ld > n: the same expansion
    D = torch.full(((n + 5) * n,), float("nan"), dtype=torch.float64, device=gu.dev())
    Dv = torch.as_strided(D, (n, n), (1, n + 5))      # column-major, ld n + 5
    hss.hss_to_dense(H, Dv)
    torch.cuda.synchronize()
    np.testing.assert_allclose(Dv.cpu().numpy(), Hd, rtol=0, atol=1e-12 * np.abs(Hd).max())


# -------------------------------------------------------------- edge cases
def test_root_is_leaf(hss, torch):
    n = 50
    A = np.random.default_rng(0).standard_normal((n, n))
    o = Options(leaf=64, rtol=1e-6, atol=1e-12, d0=8, dd=8, d_max=50)
    H = gu.gpu_compress(w.dense_source(A), w.gaussian_matrix(0, n, 0, 50), o)
    assert H.stats().n_nodes == 1
    assert np.array_equal(gu.gpu_dense(H, n), A)


@pytest.mark.parametrize("strategy", ["incrementing", "doubling"])
def test_block_diagonal_rank_zero(hss, torch, strategy):
    n, leaf = 256, 32
    A = np.zeros((n, n))
    for lo in range(0, n, leaf):
        A[lo:lo + leaf, lo:lo + leaf] = np.random.default_rng(lo).standard_normal((leaf, leaf))
    o = Options(leaf=leaf, d0=16, dd=16, d_max=64, strategy=strategy)
    H = gu.gpu_compress(w.dense_source(A), w.gaussian_matrix(0, n, 0, 64), o)
    assert all(k == (0, 0) for k in H.ranks().values())
    assert np.array_equal(gu.gpu_dense(H, n), A)


def test_not_converged_status(hss, torch):
    n = 512
    A = w.udv_matrix(n, 80, seed=2)
    o = Options(leaf=64, rtol=1e-12, atol=1e-16, d0=16, dd=8, d_max=24)
    ref = compress(w.dense_source(A), w.gaussian_matrix(0, n, 0, 24), o)
    with pytest.raises(hss.HSSError) as ei:
        gu.gpu_compress(w.dense_source(A), w.gaussian_matrix(0, n, 0, 24), o)
    assert ei.value.status == hss.HSS_ERR_NOT_CONVERGED
    H = gu.gpu_compress(w.dense_source(A), w.gaussian_matrix(0, n, 0, 24), o,
                        allow_not_converged=True)
    st = H.stats()
    assert st.converged == 0 and st.d_final == 24 and st.n_adapt == ref.n_adapt
    states = [H.node(i).state for i in range(st.n_nodes)]
    assert states == [{"U": 0, "PC": 1, "C": 2}[s] for s in ref.passes[-1]["states"]]


def test_nonfinite_input(hss, torch):
    n = 300
    A = np.random.default_rng(0).standard_normal((n, n))
    A[5, 200] = np.nan
    o = Options(leaf=64, d0=16, dd=16, d_max=64)
    with pytest.raises(hss.HSSError) as ei:
        gu.gpu_compress(w.dense_source(A), w.gaussian_matrix(0, n, 0, 64), o)
    assert ei.value.status == hss.HSS_ERR_NONFINITE


def test_device_generated_R(hss, torch):
    """Without a caller R the library draws the same Philox stream."""
    src = w.toeplitz_inverse_distance(1024)
    o = Options(leaf=64, rtol=1e-6, atol=1e-12, d0=64, dd=32, d_max=1024)
    R = w.gaussian_matrix(42, 1024, 0, 1024)
    ref = compress(src, R, o)
    H = gu.gpu_compress(src, R, o, pass_R=False, seed=42)
    assert not gu.compare_with_oracle(H, ref, o, 1024)
    A = src.to_dense()
    assert gu.rel_err(A, gu.gpu_dense(H, 1024)) <= 1.1 * apply.rel_error(ref, A) + 1e-15


def test_freed_memory_is_reused(hss, torch):
    """A freed handle's device chunks serve the next compression (the chunk
    cache), and hss_release_cached returns them: the results of the second
    and third compressions equal the first's."""
    src = w.toeplitz_inverse_distance(1024)
    o = Options(leaf=64, rtol=1e-6, atol=1e-12, d0=32, dd=32, d_max=512)
    R = w.gaussian_matrix(7, src.n, 0, 512)
    H = gu.gpu_compress(src, R, o)
    ranks, dense = H.ranks(), gu.gpu_dense(H, src.n)
    del H
    H = gu.gpu_compress(src, R, o)
    assert H.ranks() == ranks
    np.testing.assert_allclose(gu.gpu_dense(H, src.n), dense, rtol=0, atol=1e-13)
    del H
    hss.hss_release_cached()
    H = gu.gpu_compress(src, R, o)
    assert H.ranks() == ranks


def test_release_cached_returns_work_buffers(hss, torch):
    """The work buffers of a call (packed operands, job lists) come from the
    library's own memory pool, which keeps freed memory for the next call,
    and the arena chunks of a freed handle stay cached: device memory stays
    held after a mixed-form compression, and hss_release_cached gives all of
    it back (the free memory returns to what it was before the call)."""
    src = w.toeplitz_inverse_distance(2048)
    o = Options(leaf=64, rtol=1e-6, atol=1e-12, d0=32, dd=32, d_max=512)
    R = w.gaussian_matrix(7, src.n, 0, 512)

    def free_after(release):
        if release:
            hss.hss_release_cached()
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        return torch.cuda.mem_get_info()[0]

    H = gu.gpu_compress(src, R, o, precision="tf32x2")
    del H
    free0 = free_after(True)
    H = gu.gpu_compress(src, R, o, precision="tf32x2")
    assert H.stats().converged
    del H
    assert free_after(False) < free0 - (64 << 20)        # a 256 MB chunk at least, and the pool
    assert free_after(True) >= free0 - (32 << 20)


def test_checkpoint_round_trip(hss, torch, tmp_path):
    """hss_save / hss_load: the loaded handle has the same tree, ranks,
    statistics and generators, and its products equal the original's."""
    for o, src in ((Options(leaf=64, rtol=1e-6, atol=1e-12, d0=32, dd=32, d_max=512),
                    w.toeplitz_inverse_distance(1024)),
                   (Options(leaf=64, rtol=1e-6, atol=1e-12, d0=32, dd=32, d_max=512, symmetric=True),
                    w.toeplitz_power(1000, 1.5))):
        n = src.n
        H = gu.gpu_compress(src, w.gaussian_matrix(7, n, 0, 512), o)
        path = str(tmp_path / "h.hss")
        hss.hss_save(H, path)
        H2 = hss.hss_load(path)
        assert H2.ranks() == H.ranks()
        s1, s2 = H.stats(), H2.stats()
        assert (s1.d_final, s1.n_adapt, s1.converged) == (s2.d_final, s2.n_adapt, s2.converged)
        for i in range(H.stats().n_nodes):
            e1, e2 = H.export_node(i), H2.export_node(i)
            for k in e1:
                if k == "info":
                    continue
                if e1[k] is None:
                    assert e2[k] is None
                else:
                    np.testing.assert_array_equal(e1[k], e2[k])
        np.testing.assert_allclose(gu.gpu_dense(H2, n), gu.gpu_dense(H, n), rtol=0, atol=1e-15)
        import os
        assert not os.path.exists(path + ".tmp")
    # a failed save (no such directory) is an I/O error and leaves no file
    bad = str(tmp_path / "missing" / "h.hss")
    with pytest.raises(hss.HSSError) as ei:
        hss.hss_save(H, bad)
    assert ei.value.status == hss.HSS_ERR_IO
    assert not (tmp_path / "missing").exists()
