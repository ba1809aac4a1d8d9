"""Plain FP64 CPU oracle for adaptive randomized HSS compression.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports, calls or
executes this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference arm of ``bench.py`` use it.  It shares no code with
the CUDA library; both sides consume the same seeded inputs from
``workloads``.

Modules
-------
tree     cluster tree by recursive halving and recursive coordinate
         bisection (paper section 2.1 and section 3).
qrcp     Householder QR with column pivoting and the two rank rules (eq. ID
         truncation; eq. RRQRHMTstop), interpolative decomposition.
hss      Algorithm 3 (adaptive compression) with Algorithm 2 (local samples,
         reduction), the Incrementing test (Algorithm 5, eq.
         stopping_criteria) and the Doubling test (Algorithm 4).
apply    expansion of the generators to a dense matrix (eq. nestedUV),
         matrix-vector product and the relative error of Table 3.
operator a user sampling product for Toeplitz matrices through the FFT of
         a circulant embedding (section 3.1, partially matrix-free).

Every function is written in FP64 and follows the paper's order of steps;
the readings taken where the paper is ambiguous are listed in the module
docstrings (P-numbers refer to the same list in the design notes).
"""
from . import tree, qrcp, hss, apply, operator  # noqa: F401
