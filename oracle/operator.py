"""A user sampling operator for the partially matrix-free interface
(section 3.1: the construction needs products with A and A^T plus selected
entries of A), for Toeplitz matrices: the product through the circulant
embedding of size N = 2n and NumPy's FFT, O(n log n) per column instead of
the O(n^2) of a dense product.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle``.

With T(i, j) = col[i - j] for i >= j and row[j - i] for j > i, the circulant
C of size N whose first column is
    c = [col[0], ..., col[n-1], 0, row[n-1], ..., row[1]]
has C(i, j) = c[(i - j) mod N], which equals T(i, j) for i, j < n; hence
T x = (C [x; 0])[:n] and C y = ifft(fft(c) * fft(y)).  T^T is the Toeplitz
matrix with col and row exchanged.
"""
from __future__ import annotations

import numpy as np


def circulant_column(col: np.ndarray, row: np.ndarray) -> np.ndarray:
    n = col.size
    c = np.zeros(2 * n)
    c[:n] = col
    c[n + 1:] = row[1:][::-1]
    return c


def toeplitz_product(col: np.ndarray, row: np.ndarray, X: np.ndarray, trans: bool = False) -> np.ndarray:
    """T X (or T^T X) for the n x w block X through the circulant embedding."""
    n = col.size
    c = circulant_column(row, col) if trans else circulant_column(col, row)
    Y = np.zeros((2 * n, X.shape[1]))
    Y[:n] = X
    Z = np.fft.irfft(np.fft.rfft(c)[:, None] * np.fft.rfft(Y, axis=0), n=2 * n, axis=0)
    return Z[:n]
