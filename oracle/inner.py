"""Inner operator G (Sec. 3.2, Eq. linearsolve2; the set-up steps of Alg. 1).

K_i = p_i B - A for the q inner trapezoidal poles, each factorised once
(sparse LU, SciPy SuperLU, as the paper uses MATLAB's default sparse LU,
Sec. 3.2 footnote), and
    G(V) = sum_{i=1}^{q} w_i K_i^{-1} B V.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from .coeffs import trapezoid_poles_weights


class InnerOperator:
    """Pre-factorised G for the disk (c, r) with q inner poles."""

    def __init__(self, A, B, c: complex, r: float, q: int):
        self.A, self.B = A, B
        self.n = A.shape[0]
        self.poles, self.weights = trapezoid_poles_weights(c, r, q)
        self.factors = []
        for p in self.poles:
            K = (p * B - A).tocsc()           # K_i = p_i B - A (Alg. 1)
            self.factors.append(spla.splu(K))
        self.n_applies = 0                    # columns G has been applied to

    def apply(self, V: np.ndarray) -> np.ndarray:
        """G(V) = sum_i w_i K_i^{-1} (B V), V of shape (n,) or (n, k)."""
        V = np.asarray(V, dtype=np.complex128)
        BV = self.B @ V
        out = np.zeros_like(BV)
        for w, lu in zip(self.weights, self.factors):
            out += w * lu.solve(BV)
        self.n_applies += 1 if V.ndim == 1 else V.shape[1]
        return out
