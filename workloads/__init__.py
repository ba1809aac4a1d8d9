"""Seeded synthetic inputs for adaptive randomized HSS compression.

This module is shared by the CPU oracle and the CUDA path.  It holds NO
arithmetic of the compression method: only the definitions of the test
matrices (point sets, Toeplitz coefficient tables, entry formulas for the
small host-side cases) and the counter-based Gaussian generator whose draws
are passed as the random matrix R to both sides.

Matrix families (all synthetic; the paper's own BEM / quantum-chemistry /
Schur matrices are not reproduced):

* Toeplitz ``A_ij = a_|i-j|`` -- ``1/(1+k)`` (n=1024), ``(1+k)^-1.5``,
  ``cos(0.3 k)/(1+k)`` (n=131072).
* Gaussian kernel ``exp(-|x_i-x_j|^2/(2 h^2)) + s delta_ij`` on points
  uniform in the unit hypercube.
* Laplace single layer ``1/(4 pi |x_i-x_j|)`` on a Fibonacci lattice of the
  unit sphere, with a constant diagonal.
* ``alpha I + beta U D V^T`` with ``D_kk = 2^(-53 (k-1)/r)`` (paper section
  "Test Problems", the parametrised example of Table 1 and Table 3).
* A synthetic HSS matrix with prescribed per-level ranks (exactly
  representable, used to pin exact rank recovery).

Random matrix R: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
numbers: as easy as 1, 2, 3", SC 2011) keyed by the 64-bit seed; entry
(i, c) takes counter (i >> 1, c, 0, 0); the four 32-bit words give two
53-bit uniforms u1 = ((w0 >> 5) * 2^26 + (w1 >> 6)) * 2^-53 and u2 likewise
from (w2, w3); Box-Muller gives z0 = sqrt(-2 ln(1-u1)) cos(2 pi u2) and
z1 = sqrt(-2 ln(1-u1)) sin(2 pi u2); row i takes z_(i & 1).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# ---------------------------------------------------------------------------
# Philox4x32-10 counter-based generator (published definition, SC 2011).
# ---------------------------------------------------------------------------
_PHILOX_M0 = np.uint64(0xD2511F53)
_PHILOX_M1 = np.uint64(0xCD9E8D57)
_PHILOX_W0 = np.uint32(0x9E3779B9)
_PHILOX_W1 = np.uint32(0xBB67AE85)
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr: np.ndarray, key: np.ndarray) -> np.ndarray:
    """Ten rounds of Philox4x32 on arrays of counters.

    ``ctr``: uint32 array (..., 4); ``key``: uint32 array (..., 2)
    (broadcastable).  Returns uint32 (..., 4).
    """
    c = [ctr[..., i].astype(np.uint32) for i in range(4)]
    k0 = np.broadcast_to(key[..., 0], c[0].shape).astype(np.uint32)
    k1 = np.broadcast_to(key[..., 1], c[0].shape).astype(np.uint32)
    with np.errstate(over="ignore"):
        for _ in range(10):
            p0 = _PHILOX_M0 * c[0].astype(np.uint64)
            p1 = _PHILOX_M1 * c[2].astype(np.uint64)
            hi0 = (p0 >> np.uint64(32)).astype(np.uint32)
            lo0 = (p0 & _MASK32).astype(np.uint32)
            hi1 = (p1 >> np.uint64(32)).astype(np.uint32)
            lo1 = (p1 & _MASK32).astype(np.uint32)
            c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
            k0 = (k0 + _PHILOX_W0).astype(np.uint32)
            k1 = (k1 + _PHILOX_W1).astype(np.uint32)
    return np.stack(c, axis=-1)


def gaussian_matrix(seed: int, n: int, col0: int, ncols: int) -> np.ndarray:
    """R(:, col0:col0+ncols) as an n x ncols float64 Fortran-ordered array."""
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint32)
    rows = np.arange(n, dtype=np.int64)
    cols = np.arange(col0, col0 + ncols, dtype=np.int64)
    ctr = np.zeros((ncols, n, 4), dtype=np.uint32)
    ctr[:, :, 0] = (rows >> 1).astype(np.uint32)[None, :]
    ctr[:, :, 1] = cols.astype(np.uint32)[:, None]
    w = philox4x32_10(ctr, key).astype(np.float64)
    u1 = (np.floor(w[..., 0] / 32.0) * 67108864.0 + np.floor(w[..., 1] / 64.0)) * 2.0 ** -53
    u2 = (np.floor(w[..., 2] / 32.0) * 67108864.0 + np.floor(w[..., 3] / 64.0)) * 2.0 ** -53
    rad = np.sqrt(-2.0 * np.log1p(-u1))
    ang = 2.0 * math.pi * u2
    z = np.where((rows & 1)[None, :] == 0, rad * np.cos(ang), rad * np.sin(ang))
    return np.asfortranarray(z.T)


def round_to_tf32(x: np.ndarray) -> np.ndarray:
    """Round float64 values to the nearest value with an 11-bit significand
    (the TF32 significand), ties to even, keeping the float32 exponent range
    for the magnitudes used here."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)                       # x = m 2^e, 0.5 <= |m| < 1
    return np.ldexp(np.round(m * 2048.0) / 2048.0, e)


def round_to_bf16(x: np.ndarray) -> np.ndarray:
    """Round float64 values to the nearest value with an 8-bit significand
    (the bfloat16 significand), ties to even."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)
    return np.ldexp(np.round(m * 256.0) / 256.0, e)


# ---------------------------------------------------------------------------
# Matrix sources.  Each exposes entries(I, J) (float64, len(I) x len(J)),
# the raw arrays the device path consumes, and ``kind`` matching the C ABI.
# ---------------------------------------------------------------------------
SRC_DENSE, SRC_TOEPLITZ, SRC_GAUSS, SRC_LAPLACE = 0, 1, 2, 3


@dataclass
class Source:
    kind: int
    n: int
    dense: np.ndarray | None = None          # SRC_DENSE: n x n, Fortran order
    col: np.ndarray | None = None            # SRC_TOEPLITZ: A_ij = col[i-j], i >= j
    row: np.ndarray | None = None            # SRC_TOEPLITZ: A_ij = row[j-i], j > i
    points: np.ndarray | None = None         # SRC_GAUSS/LAPLACE: n x dim (rows are points)
    p0: float = 0.0                          # GAUSS: h; LAPLACE: diagonal value
    p1: float = 0.0                          # GAUSS: diagonal shift
    name: str = ""
    meta: dict = field(default_factory=dict)

    def entries(self, I, J) -> np.ndarray:
        I = np.asarray(I, dtype=np.int64)
        J = np.asarray(J, dtype=np.int64)
        if self.kind == SRC_DENSE:
            return np.array(self.dense[np.ix_(I, J)], dtype=np.float64)
        if self.kind == SRC_TOEPLITZ:
            k = I[:, None] - J[None, :]
            return np.where(k >= 0, self.col[np.maximum(k, 0)], self.row[np.maximum(-k, 0)])
        X = self.points
        diff = X[I][:, None, :] - X[J][None, :, :]
        r2 = np.einsum("ijk,ijk->ij", diff, diff)
        same = I[:, None] == J[None, :]
        if self.kind == SRC_GAUSS:
            h = self.p0
            return np.exp(-r2 / (2.0 * h * h)) + np.where(same, self.p1, 0.0)
        if self.kind == SRC_LAPLACE:
            with np.errstate(divide="ignore"):
                v = 1.0 / (4.0 * math.pi * np.sqrt(r2))
            return np.where(same, self.p0, v)
        raise ValueError(self.kind)

    def to_dense(self) -> np.ndarray:
        if self.kind == SRC_DENSE:
            return np.asfortranarray(self.dense)
        idx = np.arange(self.n)
        out = np.empty((self.n, self.n), dtype=np.float64, order="F")
        step = max(1, (1 << 22) // max(self.n, 1))
        for j0 in range(0, self.n, step):
            out[:, j0:j0 + step] = self.entries(idx, idx[j0:j0 + step])
        return out

    def permuted(self, perm: np.ndarray) -> "Source":
        """The same operator with rows/columns reordered by ``perm``
        (new index -> old index); only meaningful for point sources."""
        assert self.points is not None
        return Source(self.kind, self.n, points=np.ascontiguousarray(self.points[perm]),
                      p0=self.p0, p1=self.p1, name=self.name, meta=dict(self.meta))


def toeplitz_source(coef: np.ndarray, name: str = "toeplitz") -> Source:
    coef = np.ascontiguousarray(coef, dtype=np.float64)
    return Source(SRC_TOEPLITZ, coef.size, col=coef, row=coef, name=name)


def toeplitz_inverse_distance(n: int) -> Source:
    """A_ij = 1/(1+|i-j|)."""
    return toeplitz_source(1.0 / (1.0 + np.arange(n)), name=f"toeplitz_1/(1+k)_n{n}")


def toeplitz_power(n: int, p: float = 1.5) -> Source:
    """A_ij = (1+|i-j|)^-p."""
    return toeplitz_source((1.0 + np.arange(n)) ** (-p), name=f"toeplitz_(1+k)^-{p}_n{n}")


def toeplitz_cos(n: int, w: float = 0.3) -> Source:
    """A_ij = cos(w |i-j|)/(1+|i-j|)."""
    k = np.arange(n, dtype=np.float64)
    return toeplitz_source(np.cos(w * k) / (1.0 + k), name=f"toeplitz_cos{w}k/(1+k)_n{n}")


def toeplitz_nonsymmetric(n: int, p: float = 1.5, w: float = 0.3) -> Source:
    """A_ij = (1+(i-j))^-p below the diagonal, cos(w (j-i))/(1+(j-i)) above
    (both 1 on it): a Toeplitz matrix with A^T != A."""
    k = np.arange(n, dtype=np.float64)
    col = np.ascontiguousarray((1.0 + k) ** (-p))
    row = np.ascontiguousarray(np.cos(w * k) / (1.0 + k))
    return Source(SRC_TOEPLITZ, n, col=col, row=row, name=f"toeplitz_nonsym_n{n}")


def uniform_points(n: int, dim: int, seed: int = 0) -> np.ndarray:
    return np.random.default_rng(seed).random((n, dim))


def gaussian_kernel(points: np.ndarray, h: float = 1.0, shift: float = 0.0) -> Source:
    n = points.shape[0]
    return Source(SRC_GAUSS, n, points=np.ascontiguousarray(points, dtype=np.float64),
                  p0=h, p1=shift, name=f"gauss_d{points.shape[1]}_n{n}")


def fibonacci_sphere(n: int) -> np.ndarray:
    """Quasi-uniform points on the unit sphere (Fibonacci lattice):
    z_i = 1 - (2i+1)/n, azimuth i * pi (3 - sqrt 5)."""
    i = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / n
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = i * (math.pi * (3.0 - math.sqrt(5.0)))
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


def laplace_diag_value(points: np.ndarray) -> float:
    """2 * mean_i 1/(4 pi min_{j != i} |x_i - x_j|)."""
    from scipy.spatial import cKDTree
    dist, _ = cKDTree(points).query(points, k=2)
    return float(2.0 * np.mean(1.0 / (4.0 * math.pi * dist[:, 1])))


def laplace_kernel(points: np.ndarray, diag: float | None = None) -> Source:
    points = np.ascontiguousarray(points, dtype=np.float64)
    if diag is None:
        diag = laplace_diag_value(points)
    return Source(SRC_LAPLACE, points.shape[0], points=points, p0=diag,
                  name=f"laplace_sphere_n{points.shape[0]}")


def dense_source(A: np.ndarray, name: str = "dense") -> Source:
    A = np.asfortranarray(A, dtype=np.float64)
    return Source(SRC_DENSE, A.shape[0], dense=A, name=name)


def udv_matrix(n: int, r: int, alpha: float = 1.0, beta: float = 1.0, seed: int = 0) -> np.ndarray:
    """alpha I + beta U D V^T, U and V with r orthonormal columns (QR of
    Gaussian matrices), D_kk = 2^(-53 (k-1)/r)."""
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((n, r)))
    V, _ = np.linalg.qr(rng.standard_normal((n, r)))
    D = 2.0 ** (-53.0 * np.arange(r) / r)
    return np.asfortranarray(alpha * np.eye(n) + beta * (U * D) @ V.T)


def halving_tree_ranges(n: int, leaf: int):
    """Level-order list of (lo, size, level, parent) for the binary halving
    tree: a node of size m > leaf splits into floor(m/2) and ceil(m/2)."""
    nodes = [(0, n, 0, -1)]
    i = 0
    while i < len(nodes):
        lo, m, lev, _ = nodes[i]
        if m > leaf:
            h = m // 2
            nodes.append((lo, h, lev + 1, i))
            nodes.append((lo + h, m - h, lev + 1, i))
        i += 1
    return nodes


def synthetic_hss(n: int, leaf: int, ranks_per_level: dict, seed: int = 0,
                  symmetric: bool = False) -> np.ndarray:
    """Dense matrix that is exactly HSS on the halving tree with the given
    off-diagonal rank at each level (level -> rank).  Nested bases: leaf U, V
    are orthonormal ``m x r``; a parent's basis is blockdiag(children) times
    an orthonormal ``(r1+r2) x r`` transfer matrix; sibling blocks are
    ``U_big B V_big^T`` with a Gaussian B (full rank).  ``symmetric``: V = U,
    symmetric leaf blocks and B21 = B12^T, so that A = A^T."""
    rng = np.random.default_rng(seed)
    nodes = halving_tree_ranges(n, leaf)
    children = {i: [] for i in range(len(nodes))}
    for i, (_, _, _, p) in enumerate(nodes):
        if p >= 0:
            children[p].append(i)
    A = np.zeros((n, n))
    Ubig, Vbig = {}, {}

    def orth(m, r):
        q, _ = np.linalg.qr(rng.standard_normal((m, r)))
        return q

    for i in reversed(range(len(nodes))):
        lo, m, lev, _ = nodes[i]
        ch = children[i]
        if not ch:
            Dl = rng.standard_normal((m, m))
            A[lo:lo + m, lo:lo + m] = (Dl + Dl.T) / 2 if symmetric else Dl
        if i == 0:
            pass
        else:
            r = ranks_per_level[lev]
            if not ch:
                Ubig[i] = orth(m, r)
                Vbig[i] = Ubig[i] if symmetric else orth(m, r)
            else:
                a, b = ch
                ra, rb = Ubig[a].shape[1], Ubig[b].shape[1]
                Tu = orth(ra + rb, r)
                Tv = Tu if symmetric else orth(ra + rb, r)
                Ubig[i] = np.vstack([Ubig[a] @ Tu[:ra], Ubig[b] @ Tu[ra:]])
                Vbig[i] = np.vstack([Vbig[a] @ Tv[:ra], Vbig[b] @ Tv[ra:]])
        if ch:
            a, b = ch
            la, ma = nodes[a][0], nodes[a][1]
            lb, mb = nodes[b][0], nodes[b][1]
            B12 = rng.standard_normal((Ubig[a].shape[1], Vbig[b].shape[1]))
            B21 = B12.T if symmetric else rng.standard_normal((Ubig[b].shape[1], Vbig[a].shape[1]))
            A[la:la + ma, lb:lb + mb] = Ubig[a] @ B12 @ Vbig[b].T
            if symmetric:
                A[lb:lb + mb, la:la + ma] = A[la:la + ma, lb:lb + mb].T
            else:
                A[lb:lb + mb, la:la + ma] = Ubig[b] @ B21 @ Vbig[a].T
    return np.asfortranarray(A)


# ---------------------------------------------------------------------------
# Workload configurations (sizes and parameters of the benchmark cases).
# ---------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    source: Source
    leaf: int
    rtol: float
    atol: float
    strategy: str            # "incrementing" | "doubling"
    d0: int
    dd: int
    d_max: int
    precision: str           # "fp64" | "tf32x2" | "bf16x3"
    p: int = 10
    seed: int = 0
    needs_rcb: bool = False


def workload_toeplitz_1024() -> Workload:
    return Workload("toeplitz_inv_n1024", toeplitz_inverse_distance(1024), leaf=64,
                    rtol=1e-6, atol=1e-12, strategy="incrementing", d0=64, dd=32,
                    d_max=1024, precision="fp64")


def workload_gauss8_16384(n: int = 16384, precision: str = "tf32x2") -> Workload:
    src = gaussian_kernel(uniform_points(n, 8, seed=0), h=1.0, shift=1.0)
    return Workload(f"gauss8_n{n}", src, leaf=128, rtol=1e-4, atol=1e-8,
                    strategy="doubling", d0=128, dd=128, d_max=min(n, 4096),
                    precision=precision, needs_rcb=True)


def workload_laplace_sphere(n: int = 32768, precision: str = "bf16x3") -> Workload:
    pts = fibonacci_sphere(n)
    return Workload(f"laplace_sphere_n{n}", laplace_kernel(pts), leaf=256, rtol=1e-6,
                    atol=1e-8, strategy="incrementing", d0=128, dd=64,
                    d_max=min(n, 4096), precision=precision, needs_rcb=True)


def workload_toeplitz_cos(n: int = 131072, precision: str = "tf32x2") -> Workload:
    return Workload(f"toeplitz_cos_n{n}", toeplitz_cos(n), leaf=256, rtol=1e-4,
                    atol=1e-10, strategy="incrementing", d0=256, dd=128,
                    d_max=1024, precision=precision)


def batch_sizes(count: int = 64, lo: int = 2048, hi: int = 16384, seed: int = 0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), size=count))).astype(np.int64)
