"""Sparse pencil helpers: DIA storage to SciPy CSR, and matrix 1-norms.

The pencil (A, B) of Sec. 1 Eq. (problem) arrives in DIA form:
M[i, i + offsets[d]] = dia[d, i].
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def dia_to_csr(offsets, dia, n: int) -> sp.csr_matrix:
    """Assemble M with M[i, i+off_d] = dia[d, i] (entries outside 0..n-1 dropped)."""
    rows, cols, vals = [], [], []
    for d, off in enumerate(offsets):
        i = np.arange(n)
        j = i + int(off)
        ok = (j >= 0) & (j < n)
        rows.append(i[ok])
        cols.append(j[ok])
        vals.append(np.asarray(dia[d])[ok])
    M = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n), dtype=np.complex128)
    M = M.tocsr()
    M.eliminate_zeros()
    return M


def norm1(M) -> float:
    """Matrix 1-norm: maximum absolute column sum."""
    return float(np.max(np.asarray(abs(M).sum(axis=0)).ravel()))


def pencil_matrices(pen):
    """(A, B) as CSR matrices from an ie_inputs.Pencil."""
    A = dia_to_csr(pen.offsets, pen.A_dia, pen.n)
    B = dia_to_csr(pen.offsets, pen.B_dia, pen.n)
    return A, B
