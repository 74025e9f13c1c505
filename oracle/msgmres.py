"""Outer rational function by multi-shift GMRES (Sec. 3.2, Eq. linearsolve1abs;
the filter steps of Alg. 1 and Alg. 2).

For one column ytilde = G(y) the Krylov space K_J(G, ytilde) is built once by
Arnoldi and shared by every outer shift, because K_J(G - sI, y) = K_J(G, y) and
(G - sI) V_J = V_{J+1} (Hbar_J - s Ibar_J). For each shift s_j the GMRES iterate
from x0 = 0 minimises || beta e_1 - (Hbar - s_j Ibar) y || (Saad, GMRES), here
solved as a plain least-squares problem.

The filtered column (Thm 2 with the corrected sign, see coeffs) is
    u = sum_j c_j (s_j I - G)^{-1} ytilde + odd_coef * ytilde,
where (s_j I - G)^{-1} ytilde = -(G - s_j I)^{-1} ytilde = -V_J y_j.

reading (Arnoldi): one independent Krylov space per column, not block GMRES;
orthogonalisation by classical Gram-Schmidt applied twice (CGS2).
reading (stopping): shift j of a column has converged when the GMRES residual
||ytilde - (G - s_j I) x_j|| <= tol * ||ytilde||; a column stops extending its
basis when all its shifts have converged, after a lucky breakdown, or at m_max.
"""
from __future__ import annotations

import numpy as np

from .coeffs import outer_shifts_weights


class ColumnKrylov:
    """Arnoldi basis of K_J(G, ytilde) for one column, extendable (Alg. 2 reuses it)."""

    def __init__(self, G_apply, ytilde: np.ndarray, m_max: int):
        self.G_apply = G_apply
        self.m_max = m_max
        self.beta = float(np.linalg.norm(ytilde))
        n = ytilde.shape[0]
        self.V = np.zeros((n, m_max + 1), dtype=np.complex128)
        self.H = np.zeros((m_max + 1, m_max), dtype=np.complex128)
        self.J = 0                     # number of Arnoldi steps taken
        self.breakdown = self.beta == 0.0
        if not self.breakdown:
            self.V[:, 0] = ytilde / self.beta

    def step(self) -> None:
        """One Arnoldi step with CGS2: w = G v_J; h = V^H w, w -= V h, twice."""
        j = self.J
        w = self.G_apply(self.V[:, j])
        wn0 = float(np.linalg.norm(w))
        Vj = self.V[:, : j + 1]
        h = Vj.conj().T @ w
        w = w - Vj @ h
        h2 = Vj.conj().T @ w
        w = w - Vj @ h2
        h = h + h2
        hn = float(np.linalg.norm(w))
        self.H[: j + 1, j] = h
        self.H[j + 1, j] = hn
        self.J = j + 1
        # lucky breakdown: K_J is invariant under G, the GMRES solutions are exact
        if hn <= 1e-14 * wn0:
            self.breakdown = True
            self.H[j + 1, j] = 0.0
        else:
            self.V[:, j + 1] = w / hn

    def solve_shift(self, s: complex):
        """GMRES iterate for (G - sI) x = ytilde in the current basis.
        Returns (y, relative residual)."""
        J = self.J
        if self.beta == 0.0:
            return np.zeros(0, dtype=np.complex128), 0.0
        Hs = self.H[: J + 1, :J].copy()
        Hs[np.arange(J), np.arange(J)] -= s          # Hbar_J - s Ibar_J
        rhs = np.zeros(J + 1, dtype=np.complex128)
        rhs[0] = self.beta
        y, *_ = np.linalg.lstsq(Hs, rhs, rcond=None)
        res = float(np.linalg.norm(rhs - Hs @ y)) / self.beta
        return y, res

    def converged(self, shifts, tol: float) -> bool:
        if self.beta == 0.0:
            return True
        if self.J == 0:
            return False
        if self.breakdown:
            return True
        return all(self.solve_shift(s)[1] <= tol for s in shifts)

    def run(self, shifts, tol: float) -> bool:
        """Extend the basis until every shift meets tol. Returns False at m_max."""
        while not self.converged(shifts, tol):
            if self.J >= self.m_max:
                return False
            self.step()
        return True

    def combine(self, shifts, weights, odd: float) -> np.ndarray:
        """u = sum_j c_j (s_j I - G)^{-1} ytilde + odd * ytilde (Thm 2, corrected sign)."""
        n = self.V.shape[0]
        if self.beta == 0.0:
            return np.zeros(n, dtype=np.complex128)
        z = np.zeros(self.J, dtype=np.complex128)
        for s, c in zip(shifts, weights):
            y, _ = self.solve_shift(s)
            z -= c * y                       # (s I - G)^{-1} ytilde = -V y
        u = self.V[:, : self.J] @ z
        u = u + odd * self.beta * self.V[:, 0]
        return u


def filter_apply(G, Y: np.ndarray, p: int, tol: float = 1e-12, m_max: int = 100,
                 return_stats: bool = False):
    """U = R_{c,r,pq}(B^{-1}A) Y by the composite rule (filter step of Alg. 1):
    Ytilde = G(Y); per column multi-shift GMRES for the p outer shifts; combine."""
    s, c, odd = outer_shifts_weights(p)
    Y = np.asarray(Y, dtype=np.complex128)
    n, k = Y.shape
    U = np.zeros((n, k), dtype=np.complex128)
    iters, ok = [], True
    for col in range(k):
        yt = G.apply(Y[:, col])
        kr = ColumnKrylov(G.apply, yt, m_max)
        ok &= kr.run(s, tol)
        U[:, col] = kr.combine(s, c, odd)
        iters.append(kr.J)
    if return_stats:
        return U, {"gmres_iters": iters, "converged": ok}
    return U
