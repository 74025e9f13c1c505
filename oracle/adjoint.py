"""Left eigenvectors and first-order eigenvalue sensitivities.

TEST INFRASTRUCTURE ONLY (see the package header).

The paper computes right eigenpairs only. This module carries its method over to the
adjoint pencil, which gives the left eigenvectors, and from them the derivatives of
the eigenvalues.

Left eigenvectors. y is a left eigenvector of (A, B) for lambda when
y^H A = lambda y^H B, that is A^H y = conj(lambda) B^H y: y is a right eigenvector of
the adjoint pencil (A^H, B^H) for conj(lambda). The eigenvalues of (A^H, B^H) inside
D(conj c, r) are the conjugates of those of (A, B) inside D(c, r), so the eigensolver
of Sec. 3 (drivers.solve, Alg. 1 / Alg. 2) run on (A^H, B^H, conj c, r) finds them.
Its inner operator (Eq. linearsolve2 for the adjoint pencil) uses the trapezoidal
nodes of D(conj c, r) (Eq. pwtp). The angles (2i-1) pi / q form a set that is closed
under negation modulo 2 pi, so those nodes and weights are the conjugates of the nodes
p_i and weights w_i of D(c, r), and each shifted matrix is conj(p_i) B^H - A^H = K_i^H:
    G_adj(V) = sum_i conj(w_i) K_i^{-H} B^H V.

Sensitivity. For a simple eigenvalue with right vector x and left vector y, and a
perturbation (dA, dB) of the pencil, first-order perturbation theory gives
    d lambda = y^H (dA - lambda dB) x / (y^H B x).
Changing the diagonal entry A_jj by delta gives d lambda = delta conj(y_j) x_j / (y^H B x).
The convection-diffusion pencil carries + i gamma_j on the diagonal of A (and B does not
depend on gamma), so d lambda / d gamma_j = i conj(y_j) x_j / (y^H B x).
"""
from __future__ import annotations

import numpy as np

from .drivers import solve
from .inner import InnerOperator


def adjoint_pencil(A, B):
    """(A^H, B^H) in CSR form."""
    return A.conj().T.tocsr(), B.conj().T.tocsr()


def adjoint_inner(A, B, c: complex, r: float, q: int) -> InnerOperator:
    """G_adj for the disk D(c, r) of (A, B): the inner operator of (A^H, B^H) on
    D(conj c, r), each K_i^H factorised on its own (SuperLU)."""
    AH, BH = adjoint_pencil(A, B)
    return InnerOperator(AH, BH, np.conj(c), r, q)


def left_eigenpairs(A, B, c: complex, r: float, p: int, q: int, Y0: np.ndarray,
                    sigma: complex | None = None, **kw) -> dict:
    """Alg. 1 / Alg. 2 on the adjoint pencil. Returns the solver's dict with 'lam'
    conjugated back to eigenvalues of (A, B) and the left vectors under 'Y' (unit 2-norm,
    same order as 'lam')."""
    AH, BH = adjoint_pencil(A, B)
    res = solve(AH, BH, np.conj(c), r, p, q, Y0,
                sigma=None if sigma is None else np.conj(sigma), **kw)
    out = dict(res)
    out["lam"] = np.conj(res["lam"])
    out["Y"] = res["X"]
    return out


def pair_left(lam_right: np.ndarray, lam_left: np.ndarray) -> np.ndarray:
    """Index into lam_left of the eigenvalue nearest each lam_right entry (one-to-one
    required: raises ValueError if two right eigenvalues pick the same left one)."""
    lam_right = np.asarray(lam_right)
    lam_left = np.asarray(lam_left)
    d = np.abs(lam_right[:, None] - lam_left[None, :])
    d[~np.isfinite(d)] = np.inf
    idx = np.argmin(d, axis=1)
    if len(set(idx.tolist())) != len(idx):
        raise ValueError("left/right eigenvalues do not pair one-to-one")
    return idx


def diag_sensitivity(B, X: np.ndarray, Y: np.ndarray, alpha: complex = 1.0) -> np.ndarray:
    """S[j, i] = alpha conj(Y[j, i]) X[j, i] / (Y[:, i]^H B X[:, i]): the derivative of
    eigenvalue i with respect to the parameter t of A_jj(t) = A_jj + alpha t
    (alpha = 1j for gamma_j of the convection-diffusion pencil). Invariant under
    rescaling of either vector."""
    X = np.asarray(X, dtype=np.complex128)
    Y = np.asarray(Y, dtype=np.complex128)
    den = np.sum(np.conj(Y) * (B @ X), axis=0)
    return alpha * np.conj(Y) * X / den[None, :]


def vjp(S: np.ndarray, gbar: np.ndarray) -> np.ndarray:
    """Gradient of a real loss J(lambda) with respect to the parameters:
    grad_j = Re sum_i conj(gbar_i) S[j, i], where gbar_i = dJ/d Re(lambda_i)
    + i dJ/d Im(lambda_i) (so that dJ = Re sum_i conj(gbar_i) d lambda_i)."""
    return np.real(np.asarray(S) @ np.conj(np.asarray(gbar, dtype=np.complex128)))
