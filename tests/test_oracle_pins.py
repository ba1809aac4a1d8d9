"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test is chosen so that a plausible mistake in the oracle (a dropped
term, a wrong sign or index, a transposed operand, a wrong rank rule)
fails at least one of them.  None of them compares the oracle with itself.
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla

import workloads as w
from oracle import apply, hss, qrcp, tree
from oracle.hss import Options, compress

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- generator
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    for r in rows:
        v = [int(x, 16) for x in r]
        out = w.philox4x32_10(np.array(v[:4], dtype=np.uint32), np.array(v[4:6], dtype=np.uint32))
        assert [int(x) for x in out] == v[6:]


def test_gaussian_moments():
    R = w.gaussian_matrix(7, 4096, 0, 64)
    z = R.ravel()
    assert abs(z.mean()) < 4 / math.sqrt(z.size)
    assert abs(z.var() - 1) < 4 * math.sqrt(2 / z.size)
    # columns drawn separately equal the corresponding block of a wide draw
    assert np.array_equal(w.gaussian_matrix(7, 4096, 10, 5), R[:, 10:15])


# --------------------------------------------------------------------- tree
def test_halving_tree_partition():
    for n, leaf in [(1024, 64), (1000, 64), (2048 + 77, 128), (64, 64), (65, 64)]:
        nodes = tree.halving_tree(n, leaf)
        assert nodes[0].lo == 0 and nodes[0].size == n
        for t in nodes:
            if t.children:
                a, b = (nodes[c] for c in t.children)
                assert a.lo == t.lo and a.size == t.size // 2
                assert b.lo == a.lo + a.size and a.size + b.size == t.size
                assert a.level == b.level == t.level + 1
            else:
                assert t.size <= leaf
        # level order numbering
        assert [t.level for t in nodes] == sorted(t.level for t in nodes)
    assert len(tree.halving_tree(1024, 64)) == 31


def test_rcb_properties():
    rng = np.random.default_rng(3)
    P = rng.random((1000, 3)) * np.array([1.0, 4.0, 2.0])
    perm = tree.rcb_order(P, 64)
    assert sorted(perm) == list(range(1000))
    Q = P[perm]
    for t in tree.halving_tree(1000, 64):
        if not t.children:
            continue
        blk = Q[t.lo:t.lo + t.size]
        c = int(np.argmax(blk.max(0) - blk.min(0)))
        h = t.size // 2
        assert blk[:h, c].max() <= blk[h:, c].min()
    # 1-D points: RCB is a sort
    x = rng.random((300, 1))
    assert np.array_equal(tree.rcb_order(x, 8), np.argsort(x[:, 0], kind="stable"))


# --------------------------------------------------------------------- QRCP
def _graded(d, m, seed):
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((d, m))
    return G * (10.0 ** -np.linspace(0, 6, m))[rng.permutation(m)]


def test_qrcp_matches_lapack_pivoting():
    W = _graded(80, 50, 0)
    piv, R, k, stopped = qrcp.qrcp(W, lambda j, r, r1: False)
    Q2, R2, P2 = sla.qr(W, pivoting=True, mode="economic")
    assert not stopped and k == 50
    assert np.array_equal(piv, P2)
    np.testing.assert_allclose(np.abs(np.diag(R)), np.abs(np.diag(R2)), rtol=1e-12)
    # W Pi = Q R with Q orthonormal: R^T R = (W Pi)^T (W Pi)
    WP = W[:, piv]
    np.testing.assert_allclose(R.T @ R, WP.T @ WP, rtol=1e-10, atol=1e-12)


def test_plain_rule_rank_and_id_exact():
    rng = np.random.default_rng(1)
    m, d, k = 60, 40, 13
    S = rng.standard_normal((m, k)) @ rng.standard_normal((k, d))   # m x d, rank k
    piv, R, kk, stopped = qrcp.qrcp(S.T, qrcp.plain_rule(1e-10, 1e-14))
    assert stopped and kk == k
    J, X, U = qrcp.interpolative(piv, R, kk)
    np.testing.assert_array_equal(U[J], np.eye(k))
    np.testing.assert_allclose(U @ S[J], S, rtol=0, atol=1e-11 * np.abs(S).max())


def test_id_matches_scipy_interpolative():
    import scipy.linalg.interpolative as sli
    S = _graded(30, 45, 4).T            # 45 x 30 sample; ID of its rows
    k = 12
    idx, proj = sli.interp_decomp(np.asfortranarray(S.T), k, rand=False)
    piv, R, kk, _ = qrcp.qrcp(S.T, lambda j, r, r1: j >= k)
    J, X, U = qrcp.interpolative(piv, R, kk)
    assert np.array_equal(J, idx[:k])
    np.testing.assert_allclose(X, proj, rtol=1e-9, atol=1e-12)


def test_hmt_rule_is_more_conservative():
    rng = np.random.default_rng(2)
    m, d = 80, 64
    sv = 10.0 ** -np.linspace(0, 12, m)
    U, _ = np.linalg.qr(rng.standard_normal((m, m)))
    S = (U * sv) @ rng.standard_normal((m, d))
    _, _, k_plain, _ = qrcp.qrcp(S.T, qrcp.plain_rule(1e-6, 1e-30))
    _, _, k_hmt, st = qrcp.qrcp(S.T, qrcp.hmt_rule(1e-6, 1e-30, d, m, 1000))
    assert st and k_hmt > k_plain
    # the factor grows without bound as the oversampling d-k-1 vanishes
    assert qrcp.hmt_factor(d - 2, d, m, 1000) > qrcp.hmt_factor(10, d, m, 1000) > 1
    assert qrcp.hmt_factor(d - 1, d, m, 1000) == math.inf


# ------------------------------------------------------ Incrementing block test
def test_incrementing_block_cases():
    rng = np.random.default_rng(5)
    m = 50
    Q, _ = np.linalg.qr(rng.standard_normal((m, 10)))
    # a block inside span(Q): the projected block vanishes -> sufficient
    st = dict(Q=Q.copy(), rho=1.0)
    assert hss.incrementing_block_test(Q @ rng.standard_normal((10, 8)), st, 1e-8, 1e-30)
    # a full-rank block: not sufficient, Q grows by the block width, stays orthonormal
    st = dict(Q=Q.copy(), rho=None)
    assert not hss.incrementing_block_test(rng.standard_normal((m, 8)), st, 1e-8, 1e-30)
    assert st["Q"].shape == (m, 18)
    np.testing.assert_allclose(st["Q"].T @ st["Q"], np.eye(18), atol=1e-13)
    # a rank-deficient block outside span(Q): min |diag R| is tiny -> sufficient
    st = dict(Q=Q.copy(), rho=None)
    blk = rng.standard_normal((m, 3)) @ rng.standard_normal((3, 8))
    assert hss.incrementing_block_test(blk, st, 1e-8, 1e-30)


def test_incrementing_residual_estimator():
    """E ||(I-QQ^T) F R||_F^2 / b = ||(I-QQ^T) F||_F^2 (section 2.5): the
    projected block norm estimates the residual of the Hankel block."""
    rng = np.random.default_rng(6)
    m, ncol, b = 40, 200, 16
    F = rng.standard_normal((m, 5)) @ rng.standard_normal((5, ncol)) + 1e-3 * rng.standard_normal((m, ncol))
    Q, _ = np.linalg.qr(F @ rng.standard_normal((ncol, 5)))
    truth = np.linalg.norm(F - Q @ (Q.T @ F)) ** 2
    est = []
    for s in range(300):
        Rk = w.gaussian_matrix(100 + s, ncol, 0, b)
        Sk = F @ Rk
        Sh = Sk - Q @ (Q.T @ Sk)
        Sh = Sh - Q @ (Q.T @ Sh)
        est.append(np.linalg.norm(Sh) ** 2 / b)
    est = np.array(est)
    assert abs(est.mean() - truth) < 4 * est.std() / math.sqrt(est.size)


def test_norm_estimator_theorem1():
    """E ||A R||_F^2 / d = ||A||_F^2 (Theorem 1 and the estimate after it)."""
    rng = np.random.default_rng(8)
    A = rng.standard_normal((30, 60)) * (0.7 ** np.arange(60))
    vals = np.array([np.linalg.norm(A @ w.gaussian_matrix(s, 60, 0, 8)) ** 2 / 8 for s in range(500)])
    assert abs(vals.mean() - np.linalg.norm(A) ** 2) < 4 * vals.std() / math.sqrt(vals.size)


# ------------------------------------------------------------ compression
@pytest.mark.parametrize("strategy", ["incrementing", "doubling"])
@pytest.mark.parametrize("d0,dd", [(32, 16), (8, 8)])
def test_synthetic_hss_exact_ranks(strategy, d0, dd):
    n, leaf = 1024, 64
    ranks = {4: 8, 3: 12, 2: 16, 1: 20}
    A = w.synthetic_hss(n, leaf, ranks, seed=3)
    R = w.gaussian_matrix(5, n, 0, 512)
    res = compress(w.dense_source(A), R, Options(leaf=leaf, rtol=1e-10, atol=1e-14, d0=d0,
                                                 dd=dd, d_max=512, strategy=strategy))
    assert res.converged
    for t in res.nodes[1:]:
        assert len(t.Jr) == len(t.Jc) == ranks[t.level], (t.idx, t.level)
    assert apply.rel_error(res, A) < 1e-12
    if d0 == 8:
        assert res.n_adapt >= 1


@pytest.mark.parametrize("strategy", ["incrementing", "doubling"])
def test_symmetric_option_exact_ranks(strategy):
    """Symmetric option (P21) on an exactly symmetric HSS matrix: the known
    ranks, V = U, B21 = B12^T, and the reconstruction exact to rounding."""
    n, leaf = 1024, 64
    ranks = {4: 8, 3: 12, 2: 16, 1: 20}
    A = w.synthetic_hss(n, leaf, ranks, seed=4, symmetric=True)
    assert np.array_equal(A, A.T)
    R = w.gaussian_matrix(6, n, 0, 512)
    res = compress(w.dense_source(A), R, Options(leaf=leaf, rtol=1e-10, atol=1e-14, d0=16, dd=16,
                                                 d_max=512, strategy=strategy, symmetric=True))
    assert res.converged
    for t in res.nodes[1:]:
        assert len(t.Jr) == ranks[t.level], (t.idx, t.level)
        assert np.array_equal(t.Jr, t.Jc) and np.array_equal(t.U, t.V)
    for t in res.nodes:
        if not t.is_leaf:
            assert np.array_equal(t.B21, t.B12.T)
    assert apply.rel_error(res, A) < 1e-12


def test_symmetric_option_matches_general_on_symmetric_matrix():
    """On a symmetric kernel matrix the symmetric option reproduces the
    general algorithm: same d_final, ranks and the same error to rounding."""
    n, leaf = 768, 64
    pts = w.uniform_points(n, 3, seed=2)
    src = w.gaussian_kernel(pts[tree.rcb_order(pts, leaf)], 0.4, 0.0)
    R = w.gaussian_matrix(8, n, 0, 512)
    o = dict(leaf=leaf, rtol=1e-6, atol=1e-12, d0=32, dd=32, d_max=512)
    gen = compress(src, R, Options(**o))
    sym = compress(src, R, Options(**o, symmetric=True))
    assert gen.converged and sym.converged and gen.d_final == sym.d_final
    assert gen.ranks() == sym.ranks()
    A = src.to_dense()
    e_g, e_s = apply.rel_error(gen, A), apply.rel_error(sym, A)
    assert abs(e_g - e_s) <= 1e-3 * e_g, (e_g, e_s)


def _hankel(A, t):
    I = t.I
    mask = np.ones(A.shape[0], bool)
    mask[I] = False
    return A[np.ix_(I, np.flatnonzero(mask))], A[np.ix_(np.flatnonzero(mask), I)]


@pytest.mark.parametrize("strategy", ["incrementing", "doubling"])
def test_bruteforce_svd_small(strategy):
    """n = 512: every node's ID rank against the singular values of its
    Hankel blocks, the interpolation error of the leaf Hankel blocks, and
    the final error bound rtol."""
    n, leaf = 512, 32
    A = w.toeplitz_inverse_distance(n).to_dense()
    R = w.gaussian_matrix(11, n, 0, 512)
    rtol = 1e-6
    opts = Options(leaf=leaf, rtol=rtol, atol=1e-14, d0=32, dd=16, d_max=512, strategy=strategy)
    res = compress(w.toeplitz_inverse_distance(n), R, opts)
    assert res.converged
    L = max(t.level for t in res.nodes)
    for t in res.nodes[1:]:
        eps = rtol / t.level
        Fr, Fc = _hankel(A, t)
        for F, k in ((Fr, len(t.Jr)), (Fc.T, len(t.Jc))):
            s = np.linalg.svd(F, compute_uv=False)
            lo = int(np.sum(s > eps * s[0] * 30.0))
            hi = int(np.sum(s > eps * s[0] / 30.0))
            assert lo <= k <= hi + 16, (t.idx, k, lo, hi)
        if t.is_leaf:
            # rows J interpolate the true Hankel row block
            err = np.linalg.norm(Fr - t.U @ Fr[t.Jr]) / np.linalg.norm(Fr)
            assert err < 100 * eps, (t.idx, err)
            err = np.linalg.norm(Fc.T - t.V @ Fc.T[t.Jc]) / np.linalg.norm(Fc)
            assert err < 100 * eps, (t.idx, err)
    assert apply.rel_error(res, A) <= rtol


def test_structural_invariants():
    n = 1024
    src = w.toeplitz_inverse_distance(n)
    A = src.to_dense()
    res = compress(src, w.gaussian_matrix(0, n, 0, 1024), Options())
    Ubig, Vbig = {}, {}
    for t in reversed(res.nodes[1:]):
        np.testing.assert_array_equal(t.U[t.Jr], np.eye(len(t.Jr)))
        np.testing.assert_array_equal(t.V[t.Jc], np.eye(len(t.Jc)))
        if t.is_leaf:
            Ubig[t.idx], Vbig[t.idx] = t.U, t.V
        else:
            a, b = (res.nodes[c] for c in t.children)
            # B blocks are exact sub-blocks of A at the skeleton indices
            assert np.array_equal(t.B12, A[np.ix_(a.Ir, b.Ic)])
            assert np.array_equal(t.B21, A[np.ix_(b.Ir, a.Ic)])
            ka = Ubig[a.idx].shape[1]
            Ubig[t.idx] = np.vstack([Ubig[a.idx] @ t.U[:ka], Ubig[b.idx] @ t.U[ka:]])
            kc = Vbig[a.idx].shape[1]
            Vbig[t.idx] = np.vstack([Vbig[a.idx] @ t.V[:kc], Vbig[b.idx] @ t.V[kc:]])
        # nested skeleton: the big basis is the identity on the global rows I^r
        np.testing.assert_allclose(Ubig[t.idx][t.Ir - t.lo], np.eye(len(t.Ir)), atol=1e-12)
        np.testing.assert_allclose(Vbig[t.idx][t.Ic - t.lo], np.eye(len(t.Ic)), atol=1e-12)
    x = np.random.default_rng(0).standard_normal((n, 3))
    np.testing.assert_allclose(apply.matvec(res, x), A @ x, rtol=0, atol=5e-6 * np.abs(A @ x).max())


def test_toeplitz_1024_error_bound():
    wl = w.workload_toeplitz_1024()
    A = wl.source.to_dense()
    res = compress(wl.source, w.gaussian_matrix(0, 1024, 0, 1024),
                   Options(leaf=64, rtol=1e-6, atol=1e-12, d0=64, dd=32, d_max=1024))
    assert res.converged
    assert apply.rel_error(res, A) <= 1e-6


def test_not_converged_when_dmax_too_small():
    n = 512
    A = w.udv_matrix(n, 80, seed=2)
    res = compress(w.dense_source(A), w.gaussian_matrix(0, n, 0, 24),
                   Options(leaf=64, rtol=1e-12, atol=1e-16, d0=16, dd=8, d_max=24))
    assert not res.converged and res.d_final == 24 and res.n_adapt == 1


def test_block_diagonal_rank_zero():
    """Zero off-diagonal blocks: every node has rank 0 and H = A exactly."""
    n, leaf = 256, 32
    A = np.zeros((n, n))
    for lo in range(0, n, leaf):
        A[lo:lo + leaf, lo:lo + leaf] = np.random.default_rng(lo).standard_normal((leaf, leaf))
    for strat in ("incrementing", "doubling"):
        res = compress(w.dense_source(A), w.gaussian_matrix(0, n, 0, 64),
                       Options(leaf=leaf, d0=16, dd=16, d_max=64, strategy=strat))
        assert res.converged and res.max_rank() == 0
        np.testing.assert_array_equal(apply.to_dense(res), A)


def test_table3_rank_band():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "table3_udv_ranks.txt"))
            if l.strip() and not l.startswith("#")]
    n, r = 2048, 200
    A = w.udv_matrix(n, r, seed=1)
    R = w.gaussian_matrix(1, n, 0, 1024)
    for rtol, atol, _err, rank in rows:
        rtol, atol, rank = float(rtol), float(atol), int(rank)
        res = compress(w.dense_source(A), R, Options(leaf=128, rtol=rtol, atol=atol, d0=128,
                                                     dd=64, d_max=1024))
        assert res.converged
        assert 0.7 * rank <= res.max_rank() <= 1.3 * rank, (rtol, res.max_rank(), rank)
        assert apply.rel_error(res, A) <= rtol


# ------------------------------------------------------ HMT criterion (P22)
def test_hmt_estimate_rank_one_failure_probability():
    """Lemma 4.1 on a rank-one B = u v^T with unit u, v (|B|_2 = 1): B w =
    u (v^T w) with v^T w standard normal, so the estimate alpha sqrt(2/pi)
    max_i |B w_i|_2 falls below |B|_2 exactly when every |g_i| < 1 / (alpha
    sqrt(2/pi)), which has probability erf(sqrt(pi) / (2 alpha))^p <= alpha^-p.
    The frequency over many draws pins the constant and the max."""
    rng = np.random.default_rng(21)
    u = rng.standard_normal(7)
    v = rng.standard_normal(5)
    B = np.outer(u / np.linalg.norm(u), v / np.linalg.norm(v))
    alpha, T = 2.0, 40000
    for p in (1, 3):
        W = rng.standard_normal((T, 5, p))
        fails = sum(hss.hmt_estimate(B @ W[t], alpha) < 1.0 for t in range(T))
        prob = math.erf(math.sqrt(math.pi) / (2.0 * alpha)) ** p
        assert prob <= alpha ** -p
        assert abs(fails / T - prob) < 5.0 * math.sqrt(prob * (1.0 - prob) / T), (p, fails / T, prob)
    # a full-rank B: the bound of the lemma fails with frequency <= alpha^-p
    B = rng.standard_normal((6, 9))
    nB = np.linalg.norm(B, 2)
    p, T = 3, 20000
    W = rng.standard_normal((T, 9, p))
    fails = sum(hss.hmt_estimate(B @ W[t], alpha) < nB for t in range(T)) / T
    assert fails <= alpha ** -p + 5.0 * math.sqrt(alpha ** -p / T)


def test_hmt_criterion_leaves_meet_lemma():
    """At a leaf the local sample is exactly F R(outside) with F the Hankel
    block A(I, complement) (eq. sample_off_diag), so Lemma 4.1 holds with
    B = (I - Q Q^T) F: when the HMT test accepts a block,
    |(I - Q Q^T) F|_2 <= eps_a / level except with probability alpha^-b."""
    n, leaf, atol = 1024, 128, 1e-6
    A = w.udv_matrix(n, 120, seed=4)
    o = Options(leaf=leaf, rtol=0.0, atol=atol, d0=16, dd=16, d_max=512, criterion="hmt")
    res = compress(w.dense_source(A), w.gaussian_matrix(2, n, 0, 512), o)
    assert res.converged
    grew = 0
    for t in res.nodes:
        if not t.is_leaf:
            continue
        out = np.setdiff1d(np.arange(n), t.I)
        ea = atol / t.level
        for side, F in (("r", A[np.ix_(t.I, out)]), ("c", A[np.ix_(out, t.I)].T)):
            Q = t.inc[side]["Q"]
            resid = np.linalg.norm(F - Q @ (Q.T @ F), 2)
            assert resid <= ea, (t.idx, side, resid, ea)
            if 0 < Q.shape[1] < t.size and np.linalg.norm(F, 2) > ea:
                grew += 1
    assert grew > 0      # the test had to grow bases: it was not vacuous


def test_hmt_criterion_table3_shape():
    """Table 3: at the same absolute tolerance the HMT criterion (rtol
    ignored) takes at least as many samples as the new criterion with
    rtol = atol, and gives ranks at least as large and errors no larger."""
    n = 1024
    A = w.udv_matrix(n, 200, seed=1)
    R = w.gaussian_matrix(1, n, 0, n)
    for tol in (1e-6, 1e-10):
        new = compress(w.dense_source(A), R, Options(leaf=128, rtol=tol, atol=tol, d0=128, dd=64,
                                                     d_max=1024))
        hmt = compress(w.dense_source(A), R, Options(leaf=128, rtol=tol, atol=tol, d0=128, dd=64,
                                                     d_max=1024, criterion="hmt"))
        assert new.converged and hmt.converged
        e_new, e_hmt = apply.rel_error(new, A), apply.rel_error(hmt, A)
        assert hmt.d_final >= new.d_final and hmt.max_rank() >= new.max_rank(), tol
        assert e_hmt <= e_new * 1.01 and e_hmt <= tol, (tol, e_new, e_hmt)


def test_hmt_criterion_options_checked():
    A = w.udv_matrix(64, 8, seed=0)
    for o in (Options(leaf=16, strategy="doubling", criterion="hmt"),
              Options(leaf=16, criterion="hmt", hmt_alpha=1.0), Options(leaf=16, criterion="x")):
        with pytest.raises(ValueError):
            compress(w.dense_source(A), w.gaussian_matrix(0, 64, 0, 64), o)


def test_hmt_block_test_cases():
    """The HMT block test on blocks whose projected columns are known: a block
    inside span(Q) is sufficient; orthogonal columns of norms 1, 2, 1/2
    outside span(Q) have the estimate alpha sqrt(2/pi) 2, and a failed block
    extends Q by its width with orthonormal columns."""
    rng = np.random.default_rng(9)
    m = 40
    full, _ = np.linalg.qr(rng.standard_normal((m, m)))
    Q, P = full[:, :6], full[:, 6:]
    st = dict(Q=Q.copy())
    assert hss.hmt_block_test(Q @ rng.standard_normal((6, 8)), st, 1e-12, 10.0)
    Sk = P[:, :3] * np.array([1.0, 2.0, 0.5]) + Q @ rng.standard_normal((6, 3))
    for alpha in (2.0, 10.0):
        thr = alpha * math.sqrt(2.0 / math.pi) * 2.0
        st = dict(Q=Q.copy())
        assert hss.hmt_block_test(Sk, st, 1.001 * thr, alpha) and st["Q"].shape[1] == 6
        st = dict(Q=Q.copy())
        assert not hss.hmt_block_test(Sk, st, 0.999 * thr, alpha)
        assert st["Q"].shape[1] == 9
        np.testing.assert_allclose(st["Q"].T @ st["Q"], np.eye(9), atol=1e-13)


# ----------------------------------------- known-rank and hard restart (P23)
@pytest.mark.parametrize("d0", [3, 5, 8, 20, 21])
def test_hard_restart_on_exact_ranks(d0):
    """A synthetic HSS matrix with per-level ranks 8/12/16/20 (level 4 ... 1):
    one pass with d vectors converges exactly when d >= 21 — every local
    sample then has more columns than its rank, while at d <= 20 the level-1
    sides (32 rows, rank 20) fail the Incrementing test.  So the hard restart
    doubles d0 until it reaches 21: the number of restarts and the final d
    follow in closed form, and the ranks are the exact ones."""
    n, leaf = 1024, 64
    ranks = {4: 8, 3: 12, 2: 16, 1: 20}
    A = w.synthetic_hss(n, leaf, ranks, seed=3)
    R = w.gaussian_matrix(5, n, 0, 512)
    o = Options(leaf=leaf, rtol=1e-10, atol=1e-14, d0=d0, dd=8, d_max=512)
    res, k = hss.compress_hard_restart(w.dense_source(A), R, o)
    want = 0
    while d0 * 2 ** want < 21:
        want += 1
    assert res.converged and k == want and res.d_final == d0 * 2 ** want and res.n_adapt == 0
    for t in res.nodes[1:]:
        assert len(t.Jr) == len(t.Jc) == ranks[t.level], t.idx
    assert apply.rel_error(res, A) < 1e-12


def test_known_rank_single_pass():
    """Known-rank mode (d0 = d_max): one pass, no growth; it converges at
    d = 21 and reports NOT_CONVERGED at d = 20 on the matrix above."""
    n, leaf = 1024, 64
    A = w.synthetic_hss(n, leaf, {4: 8, 3: 12, 2: 16, 1: 20}, seed=3)
    R = w.gaussian_matrix(5, n, 0, 512)
    for d, ok in ((20, False), (21, True)):
        res = compress(w.dense_source(A), R, Options(leaf=leaf, rtol=1e-10, atol=1e-14, d0=d, dd=8, d_max=d))
        assert res.converged == ok and res.n_adapt == 0 and res.d_final == d


# --------------------------------------- user sampling operator (section 3.1)
def test_toeplitz_fft_product_is_the_toeplitz_product():
    """The circulant embedding gives T X exactly up to rounding: against the
    dense Toeplitz matrix built from its definition, both orientations,
    n odd and even."""
    from oracle.operator import toeplitz_product
    rng = np.random.default_rng(31)
    for n in (1, 2, 7, 64, 301):
        col, row = rng.standard_normal(n), rng.standard_normal(n)
        row[0] = col[0]
        T = np.array([[col[i - j] if i >= j else row[j - i] for j in range(n)] for i in range(n)])
        X = rng.standard_normal((n, 5))
        for trans in (False, True):
            ref = (T.T if trans else T) @ X
            got = toeplitz_product(col, row, X, trans)
            assert np.max(np.abs(got - ref)) <= 1e-13 * (np.abs(T).max() * np.abs(X).sum(axis=0).max() + 1.0)


def test_compress_with_user_product_matches_entries():
    """Sampling through the user product instead of the entries changes only
    the rounding of S = A R: the same adaptations, ranks and error."""
    from oracle.operator import toeplitz_product
    src = w.toeplitz_cos(1500)
    col, row = src.col, src.row
    R = w.gaussian_matrix(4, src.n, 0, 1024)
    o = Options(leaf=100, rtol=1e-6, atol=1e-12, d0=32, dd=32, d_max=1024)
    a = compress(src, R, o)
    b = compress(src, R, o, product=lambda X, tr: toeplitz_product(col, row, X, tr))
    assert a.converged and b.converged and a.d_final == b.d_final and a.n_adapt == b.n_adapt
    assert a.ranks() == b.ranks()
    A = src.to_dense()
    assert abs(apply.rel_error(a, A) - apply.rel_error(b, A)) <= 1e-3 * apply.rel_error(a, A)


# ------------------------------- Doubling acceptance in closed form (Alg. 4)
def doubling_side_accepts(m: int, r: int, d: int, p: int):
    """Whether RRQR_HMT (eq. RRQRHMTstop) accepts a local sample of m rows
    and exact rank r <= m drawn with d Gaussian vectors, and the rank it
    keeps, worked out from the rule rather than run: the sample has rank
    min(r, d), so in exact arithmetic the first vanishing pivot is the
    1-based index r + 1, which exists when r < min(d, m); the scaled stop can
    fire there only when the oversampling d - (r + 1) - 1 is positive (the
    factor is infinite otherwise, and also at every later index).  A stop at
    rank r is accepted when r <= d - p (Algorithm 4); without a stop the
    factorisation selects min(d, m) rows and is accepted only when that is
    every row (P9)."""
    if r < min(d, m) and d - (r + 1) - 1 > 0:
        return r <= d - p, r
    k = min(d, m)
    return k == m, k


def doubling_closed_form(n, leaf, ranks, d0, p, d_max, kept_out=None):
    """(converged, d_final, n_adapt) of Algorithm 3 with Doubling on the
    synthetic HSS matrix of the given per-level ranks: passes at d0, 2 d0,
    ... (the last clipped to d_max); in a pass the levels are swept from the
    leaves up, a node is tried once both children are COMPRESSED, and its
    sample has m rows = its leaf size, or the sum of its children's kept
    ranks.  ``kept_out`` (a dict) receives node -> (rows, kept rank)."""
    nodes = tree.halving_tree(n, leaf)
    state, kept = {}, {}
    d, n_adapt = min(d0, d_max), 0
    while True:
        for t in sorted(nodes[1:], key=lambda t: -t.level):
            if state.get(t.idx) or (t.children and not all(state.get(c) for c in t.children)):
                continue
            m = t.size if not t.children else sum(kept[c] for c in t.children)
            ok, k = doubling_side_accepts(m, ranks[t.level], d, p)
            if ok:
                state[t.idx], kept[t.idx] = True, k
                if kept_out is not None:
                    kept_out[t.idx] = (m, k)
        if all(state.get(c) for c in nodes[0].children):
            return True, d, n_adapt
        if d >= d_max:
            return False, d, n_adapt
        d += min(d, d_max - d)
        n_adapt += 1


def test_doubling_side_rule_by_hand():
    """A few values of the side rule checked by hand: a leaf of 64 rows and
    rank 8 stops at rank 8 from d = 11 on (8 + 3) and needs d >= 18 with
    p = 10; a full-rank side (r = m) is accepted as soon as d >= m; with
    r < m <= r + 2 the window d in {r + 1, r + 2} selects every row."""
    assert doubling_side_accepts(64, 8, 10, 0) == (False, 10)
    assert doubling_side_accepts(64, 8, 11, 0) == (True, 8)
    assert doubling_side_accepts(64, 8, 17, 10) == (False, 8)
    assert doubling_side_accepts(64, 8, 18, 10) == (True, 8)
    assert doubling_side_accepts(16, 16, 15, 10) == (False, 15)
    assert doubling_side_accepts(16, 16, 16, 10) == (True, 16)
    assert doubling_side_accepts(16, 15, 16, 10) == (True, 16)
    assert doubling_side_accepts(16, 15, 18, 10) == (False, 15)
    assert doubling_side_accepts(16, 15, 25, 10) == (True, 15)


# (ranks per level, d0, p): sequences that land between r + 3 and r + p at
# the level-1 sides (rank 20: d = 24, 26, 28 accept with p = 0, not with
# p = 10), exactly at k = d - p (d = 30), below the HMT window (d = 22 = r + 2
# with 32 rows: no stop, not every row), a full-rank level (level 3: 16 rows,
# rank 16, accepted only by selecting every row) and the all-rows window
# (level 3: 16 rows, rank 15, d = 16)
DOUBLING_PINS = [({4: 8, 3: 12, 2: 16, 1: 20}, d0, p)
                 for d0 in (5, 7, 8, 11, 12, 13, 15, 16) for p in (0, 10)]
DOUBLING_PINS += [({4: 8, 3: 16, 2: 20, 1: 24}, d0, p) for d0 in (8, 12, 15, 16) for p in (0, 10)]
DOUBLING_PINS += [({4: 8, 3: 15, 2: 20, 1: 24}, d0, p) for d0 in (8, 16) for p in (0, 3)]


@pytest.mark.parametrize("ranks,d0,p", DOUBLING_PINS)
def test_doubling_acceptance_closed_form(ranks, d0, p):
    """Doubling on a matrix of exact HSS ranks: the passes, the final d and
    the ranks kept follow from the acceptance rule k <= d - p / all rows
    selected (Algorithm 4, eq. RRQRHMTstop, P6, P9) in closed form."""
    n, leaf = 1024, 64
    A = w.synthetic_hss(n, leaf, ranks, seed=3)
    R = w.gaussian_matrix(5, n, 0, 128)
    kept = {}
    want = doubling_closed_form(n, leaf, ranks, d0, p, 128, kept)
    res = compress(w.dense_source(A), R, Options(leaf=leaf, rtol=1e-10, atol=1e-14, d0=d0, dd=d0,
                                                 d_max=128, strategy="doubling", p=p))
    assert (res.converged, res.d_final, res.n_adapt) == want
    for t in res.nodes[1:]:
        m, k = kept[t.idx]
        assert t.Sr.shape[0] == t.Sc.shape[0] == m and len(t.Jr) == len(t.Jc) == k, t.idx
    assert apply.rel_error(res, A) < 1e-12


def test_doubling_closed_form_distinguishes_p():
    """The pins above are not vacuous: p = 0 and p = 10, and k <= d - p
    against k < d - p, give different passes on them."""
    r = {4: 8, 3: 12, 2: 16, 1: 20}
    assert doubling_closed_form(1024, 64, r, 12, 0, 128)[1:] == (24, 1)
    assert doubling_closed_form(1024, 64, r, 12, 10, 128)[1:] == (48, 2)
    assert doubling_closed_form(1024, 64, r, 15, 10, 128)[1:] == (30, 1)   # 20 <= 30 - 10
    assert doubling_closed_form(1024, 64, {4: 8, 3: 16, 2: 20, 1: 24}, 8, 10, 128)[1:] == (64, 3)


# ---------------------------------------- the RRQR_HMT factor by hand (P6)
def _orthogonal_columns(d, norms, seed):
    """d x m matrix with mutually orthogonal columns of the given norms (in
    a shuffled order): its QRCP takes the columns by decreasing norm and has
    |R_jj| equal to the sorted norms."""
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((d, len(norms))))
    perm = rng.permutation(len(norms))
    return (Q * np.asarray(norms)[perm])


# d = 64 sample columns, Hankel block 100 x 900: f(k) = 1 + 4 sqrt(64) /
# (64 - k - 1) sqrt(min(100, 900)) = 1 + 320 / (63 - k), so with
# eps |R_11| = 1e-2 the thresholds of the 1-based pivots k = 2 .. 5 are
# 1e-2 / (1 + 320/61) = 1.60105e-3, 1e-2 / (1 + 320/60) = 1.57895e-3,
# 1e-2 / (1 + 320/59) = 1.55673e-3, 1e-2 / (1 + 320/58) = 1.53439e-3.
# Pivots 2-4 sit 0.2 % above their thresholds and pivot 5 0.2 % below, so
# the rule stops at k = 5 (rank 4).  Each plausible slip moves the stop: a 2
# for the 4, d - k for d - k - 1 (or a 0-based k), a missing "1 +", or an
# unscaled relative threshold stop at k = 2; d for sqrt(d), max for min, or
# min(m, n) unsquare-rooted run past k = 5 to the tiny sixth pivot.
HMT_NORMS = [1.0, 1.60425e-3, 1.58211e-3, 1.55984e-3, 1.53132e-3, 1e-6, 5e-7, 2e-7]


@pytest.mark.parametrize("tol", ["relative", "absolute"])
def test_hmt_stop_index_by_hand(tol):
    W = _orthogonal_columns(64, HMT_NORMS, seed=17)
    er, ea = (1e-2, 0.0) if tol == "relative" else (0.0, 1e-2)
    piv, R, k, stopped = qrcp.qrcp(W, qrcp.hmt_rule(er, ea, 64, 100, 900))
    assert stopped and k == 4
    np.testing.assert_allclose(np.abs(np.diag(R)), HMT_NORMS[:4], rtol=1e-12)
    # unscaled (the plain rule of the ID) the same tolerance stops at the
    # second pivot, 1.6e-3 <= 1e-2
    _, _, k_plain, st_plain = qrcp.qrcp(W, qrcp.plain_rule(er, ea))
    assert st_plain and k_plain == 1
    # with m and n swapped the factor is the same (min of the two)
    assert qrcp.qrcp(W, qrcp.hmt_rule(er, ea, 64, 900, 100))[2] == 4


# ----------------------- Incrementing's absolute and relative tests (eq. stopping_criteria)
def _block_outside(Q, norms, seed, inside=None):
    """m x b block S = Q G + Z with Z's columns orthogonal to span(Q) and to
    each other, of the given norms; Q G (optional, scale ``inside``) lies in
    span(Q), so (I - Q Q^T)^2 S = Z exactly up to rounding."""
    rng = np.random.default_rng(seed)
    m, q = Q.shape
    b = len(norms)
    Y = rng.standard_normal((m, b))
    if q:
        Y -= Q @ (Q.T @ Y)
    Z, _ = np.linalg.qr(Y)
    Z = Z * np.asarray(norms)
    G = rng.standard_normal((q, b)) * (inside or 0.0)
    return Q @ G + Z


def _basis(m, q, seed):
    return np.linalg.qr(np.random.default_rng(seed).standard_normal((m, q)))[0] if q else np.zeros((m, 0))


@pytest.mark.parametrize("q", [0, 6])
def test_incrementing_absolute_norm_test(q):
    """|S^|_F / sqrt(b) < eps_a (P7).  The projected block has b = 8
    orthogonal columns of norm 2, so |S^|_F / sqrt(b) = 2 and min |diag R| = 2:
    atol just above 2 is sufficient, just below is not (a /b instead of
    /sqrt(b) would make 0.707 < 1.98 sufficient).  The norm test comes
    before the QR of S^ (Algorithm 5), so when it decides no |R_11| is
    recorded for the side; if only the diagonal test fired, it would be."""
    Q = _basis(40, q, 3)
    S = _block_outside(Q, [2.0] * 8, seed=4, inside=5.0)
    st = dict(Q=Q.copy(), rho=None)
    assert hss.incrementing_block_test(S, st, 0.0, 2.02)
    assert st["rho"] is None and st["Q"].shape[1] == q
    st = dict(Q=Q.copy(), rho=None)
    assert not hss.incrementing_block_test(S, st, 0.0, 1.98)
    assert st["Q"].shape[1] == q + 8 and abs(st["rho"] - 2.0) < 1e-12


@pytest.mark.parametrize("q", [0, 6])
def test_incrementing_absolute_diagonal_test(q):
    """min |diag R^| < eps_a alone decides: columns of norms 1, ..., 1, 1e-3
    give |S^|_F / sqrt(8) = 0.935 but min |diag R| = 1e-3, and |R_11| = 1 is
    recorded before the decision."""
    Q = _basis(40, q, 5)
    norms = [1.0] * 7 + [1e-3]
    S = _block_outside(Q, norms, seed=6, inside=3.0)
    for ea, want in ((0.5, True), (1.001e-3, True), (0.999e-3, False)):
        st = dict(Q=Q.copy(), rho=None)
        assert hss.incrementing_block_test(S, st, 0.0, ea) == want, ea
        assert abs(st["rho"] - 1.0) < 1e-12


def test_incrementing_relative_tests():
    """|S^|_F < eps_r |S_k|_F and min |diag R^| < eps_r rho (rho = |R_11| of
    the side's first block, P8), each deciding alone."""
    m, q = 40, 6
    Q = _basis(m, q, 7)
    # |S^|_F = 0.1 * sqrt(8); |S_k|_F^2 = |Q G|_F^2 + 0.08 (Q G large)
    S = _block_outside(Q, [0.1] * 8, seed=8, inside=10.0)
    ratio = math.sqrt(0.08) / np.linalg.norm(S)
    st = dict(Q=Q.copy(), rho=None)
    assert hss.incrementing_block_test(S, st, 1.01 * ratio, 0.0) and st["rho"] is None
    # just below: the norm test fails; the diagonal test (min 0.1 against
    # eps_r rho with rho = 0.1 set by this block) fails too
    st = dict(Q=Q.copy(), rho=None)
    assert not hss.incrementing_block_test(S, st, 0.99 * ratio, 0.0)
    # diagonal relative test against an earlier block's rho
    S2 = _block_outside(_basis(m, 0, 9), [1.0] * 7 + [0.05], seed=10)
    for rho, want in ((10.0, True), (4.0, False)):
        st = dict(Q=np.zeros((m, 0)), rho=rho)
        assert hss.incrementing_block_test(S2, st, 0.0051, 0.0) == want, rho


def test_near_threshold_count_qr_by_hand():
    """The tie count on the QRCP diagonal (the rank rule's own quantity).
    Orthogonal rows of prescribed norms: the pivots take them in decreasing
    order and |R_jj| are the norms themselves, so the count follows by hand.
    Two nearly parallel rows e1 and e1 + 1e-3 e2: |R_22| is the distance of
    e1 from the first pivot's line, 1e-3 / sqrt(1 + 1e-6), right at a
    threshold of 1e-3, while the smaller singular value is near
    1e-3 / sqrt(2): only the diagonal count sees the tie."""
    rng = np.random.default_rng(3)
    Qm, _ = np.linalg.qr(rng.standard_normal((8, 8)))
    norms = np.array([1.0, 0.5, 1.05e-3, 0.95e-3, 1e-5])
    S = norms[:, None] * Qm[:5, :]          # 5 orthogonal rows, d = 8
    assert qrcp.near_threshold_count_qr(S, 1e-3, 0.0, "plain") == 2
    assert qrcp.near_threshold_count_qr(S, 1e-3, 0.0, "plain", band=0.01) == 0
    assert qrcp.near_threshold_count_qr(S, 1e-3, 0.0, "plain", band=0.01, noise=1e-4) == 2
    assert qrcp.near_threshold_count_qr(S, 0.0, 1e-5, "plain") == 1          # absolute threshold
    T = np.array([[1.0, 0.0, 0.0, 0.0], [1.0, 1e-3, 0.0, 0.0]])
    er = 1e-3 / np.sqrt(1.0 + 1e-6)    # threshold er |R_11| = 1e-3
    assert qrcp.near_threshold_count_qr(T, er, 0.0, "plain") == 1
    assert qrcp.near_threshold_count(T, er, 0.0, "plain") == 0
