"""Block-CSR matrix-vector products, written as plain loops (oracle).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

The linear solver of the FIM step iterates on the assembled block-CSR
Jacobian (LinearSystem module, Sec. 3.3.3); its kernel is y = alpha*A*x +
beta*y, and the adjoint needs the transposed product.  Vectors are
block-interleaved: x[nb*c + v].
"""
from __future__ import annotations

import numpy as np


def bsr_spmv(row_ptr, col_idx, val, x, alpha=1.0, beta=0.0, y=None, transpose=False, rows=None):
    """y <- alpha * A x + beta * y  (or A^T x).  Also returns the magnitude
    |alpha| |A| |x| + |beta| |y| used as the per-entry tolerance scale.
    With ``rows`` given (non-transposed only), only those block rows are
    computed; the other entries of the result are left at zero."""
    nb = val.shape[1]
    N = len(row_ptr) - 1
    X = np.asarray(x, dtype=np.float64).reshape(N, nb)
    Y0 = np.zeros((N, nb)) if y is None else np.asarray(y, dtype=np.float64).reshape(N, nb)
    acc = np.zeros((N, nb))
    mag = np.zeros((N, nb))
    if rows is not None and transpose:
        raise ValueError("row sampling is for the plain product only")
    for r in (range(N) if rows is None else rows):
        for s in range(row_ptr[r], row_ptr[r + 1]):
            c = col_idx[s]
            blk = val[s]
            if not transpose:
                acc[r] += blk @ X[c]
                mag[r] += np.abs(blk) @ np.abs(X[c])
            else:
                acc[c] += blk.T @ X[r]
                mag[c] += np.abs(blk.T) @ np.abs(X[r])
    out = alpha * acc + beta * Y0
    m = abs(alpha) * mag + abs(beta) * np.abs(Y0)
    return out.ravel(), m.ravel()


def bsr_to_dense(row_ptr, col_idx, val):
    nb = val.shape[1]
    N = len(row_ptr) - 1
    A = np.zeros((N * nb, N * nb))
    for r in range(N):
        for s in range(row_ptr[r], row_ptr[r + 1]):
            c = col_idx[s]
            A[r * nb:(r + 1) * nb, c * nb:(c + 1) * nb] = val[s]
    return A


def bsr_to_scipy(row_ptr, col_idx, val):
    import scipy.sparse as sp
    nb = val.shape[1]
    N = len(row_ptr) - 1
    return sp.bsr_matrix((val, col_idx, row_ptr), shape=(N * nb, N * nb))
