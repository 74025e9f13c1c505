"""Reference eigenvalues near a point, by shift-invert Arnoldi.

Sec. 6.2 computes its reference eigenvalues with MATLAB's eigs; this is the same
kind of computation: the eigenvalues theta of (A - sigma B)^{-1} B of largest
modulus give the eigenvalues lambda = sigma + 1/theta of (A, B) nearest sigma.
(SciPy ARPACK on a LinearOperator; SuperLU for A - sigma B.)
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse.linalg as spla


def nearest_eigenvalues(A, B, sigma: complex, count: int, tol: float = 1e-14, seed: int = 0):
    n = A.shape[0]
    lu = spla.splu((A - sigma * B).tocsc())
    op = spla.LinearOperator((n, n), matvec=lambda x: lu.solve(B @ x), dtype=np.complex128)
    v0 = np.random.default_rng(seed).standard_normal(n).astype(np.complex128)
    theta = spla.eigs(op, k=count, which="LM", tol=tol, v0=v0, ncv=max(2 * count + 1, 40),
                      return_eigenvectors=False)
    lam = sigma + 1.0 / theta
    return lam[np.argsort(np.abs(lam - sigma))]


def all_eigenvalues(A, B):
    """Dense QZ eigenvalues (small pencils only)."""
    return sla.eigvals(A.toarray(), B.toarray())


def median_eigenvalue(lam):
    """Median eigenvalue: index floor(n/2) (0-based) after sorting by real part,
    ties by imaginary part."""
    o = np.lexsort((lam.imag, lam.real))
    return lam[o][len(lam) // 2]


def disk_radius(distances, count: int) -> float:
    """Radius enclosing exactly `count` eigenvalues: midpoint of the count-th and
    (count+1)-th smallest distances from the centre."""
    d = np.sort(np.asarray(distances))
    return 0.5 * (float(d[count - 1]) + float(d[count]))
