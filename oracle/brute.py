"""Alg. 1 of the paper written literally with dense 0/1 matrices (tiny graphs).

Test infrastructure only.  Alg. 1 states S <- A^T A o A for the adjacency A;
Sec. II-A says S[i,j] is the number of triangles on edge (i,j).  With A stored
upper-triangular (Sec. II-B) that count is ((A + A^T)(A + A^T)) o A, which is
the form used here: each round computes every live edge's support from the
symmetric live adjacency, builds M = S >= K-2 on the live edges, sets A <- A o M
and stops when M removes nothing (isUnchanged).  Rounds count executions of
the support step; the loop also stops when A has no edge left.
"""
from __future__ import annotations

import numpy as np


def ktruss_dense(n: int, row_ptr, col, K: int, tri_out: list | None = None):
    """Returns (mask[m] uint8, support[m] int64, rounds) in CSR slot order.
    When tri_out is a list, the triangle count of each round's live graph is
    appended to it, as trace(B^3) / 6 for the symmetric live adjacency B."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    m = col.shape[0]
    rows = np.repeat(np.arange(n), np.diff(row_ptr))
    A = np.zeros((n, n), dtype=np.int64)
    A[rows, col] = 1
    rounds = 0
    S = np.zeros((n, n), dtype=np.int64)
    while A.any():
        rounds += 1
        Asym = A + A.T
        if tri_out is not None:
            tri_out.append(int(np.trace(Asym @ Asym @ Asym)) // 6)
        S = (Asym @ Asym) * A
        M = (S >= K - 2).astype(np.int64) * A
        unchanged = np.array_equal(M, A)
        A = M
        if unchanged:
            break
    mask = A[rows, col].astype(np.uint8)
    support = np.where(mask == 1, S[rows, col], 0).astype(np.int64)
    return mask, support, rounds
