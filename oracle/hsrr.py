"""Harmonic subspace Rayleigh-Ritz extraction "HSRR" (Sec. 2.1, the extraction
steps of Alg. SIsketch) and the error measures of Sec. 3.2.

    V = orth(U);  W = orth(A V - sigma B V);
    (W^* A V, W^* B V) -> QZ: P_L^* (W^*AV) P_R = H_A, P_L^* (W^*BV) P_R = H_B;
    lambda_i = (H_A)_ii / (H_B)_ii;  x_i = V P_R V_R(:, i),
with V_R the right eigenvectors of the triangular pair (H_A, H_B).

reading (orth): column-by-column classical Gram-Schmidt with each projection
applied twice (CGS2). Rank guard: a column whose norm after projection is
<= 1e-12 times its norm before projection (or that is zero) is replaced by a
seeded random vector, itself projected twice and normalised, so V and W keep
k columns (sigma = c can be an eigenvalue, making A V - sigma B V rank deficient).
reading (Ritz vectors): each x_i is scaled to unit 2-norm; the next block of
Alg. 1 is Y = (x_1 .. x_k) without re-orthogonalisation.
reading (infinite Ritz values): (H_B)_ii = 0 gives lambda_i = inf, never in D.
Errors: e_i of Eq. (rel-error), ||A x - B x lambda||_2 / ((|c| + r) ||B x||_2), and
rho_i = ||A x - lambda B x||_2 / ((||A||_1 + |lambda| ||B||_1) ||x||_2).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

RANK_TOL = 1e-12


def orth_cgs2(U: np.ndarray, rng: np.random.Generator | None = None):
    """Orthonormal basis of the columns of U (CGS2 with the rank guard).
    Returns (Q, replaced_column_indices)."""
    U = np.asarray(U, dtype=np.complex128)
    n, k = U.shape
    Q = np.zeros((n, k), dtype=np.complex128)
    replaced = []
    for j in range(k):
        u = U[:, j].copy()
        nrm0 = float(np.linalg.norm(u))
        for _ in range(2):
            u = u - Q[:, :j] @ (Q[:, :j].conj().T @ u)
        nrm = float(np.linalg.norm(u))
        if nrm0 == 0.0 or nrm <= RANK_TOL * nrm0:
            g = rng if rng is not None else np.random.Generator(np.random.PCG64(12345 + j))
            u = g.standard_normal(n) + 1j * g.standard_normal(n)
            for _ in range(2):
                u = u - Q[:, :j] @ (Q[:, :j].conj().T @ u)
            nrm = float(np.linalg.norm(u))
            replaced.append(j)
        Q[:, j] = u / nrm
    return Q, replaced


def triangular_right_eigvecs(S: np.ndarray, T: np.ndarray) -> np.ndarray:
    """Right eigenvectors of an upper-triangular pair (S, T): for each i solve
    (beta_i S - alpha_i T) v = 0 with v_i = 1, v_l = 0 for l > i, by back substitution
    (alpha_i = S_ii, beta_i = T_ii). Near-zero pivots (repeated eigenvalues) are
    replaced by eps times the scale of the pair."""
    k = S.shape[0]
    Vr = np.zeros((k, k), dtype=np.complex128)
    eps = np.finfo(float).eps
    snorm = np.abs(S).max() if k else 0.0
    tnorm = np.abs(T).max() if k else 0.0
    for i in range(k):
        a, b = S[i, i], T[i, i]
        M = b * S - a * T
        small = eps * (abs(b) * snorm + abs(a) * tnorm)
        v = np.zeros(k, dtype=np.complex128)
        v[i] = 1.0
        for j in range(i - 1, -1, -1):
            rhs = -np.dot(M[j, j + 1 : i + 1], v[j + 1 : i + 1])
            d = M[j, j]
            if abs(d) <= small:
                d = small if small > 0 else eps
            v[j] = rhs / d
        Vr[:, i] = v
    return Vr


def residuals(A, B, lam: np.ndarray, X: np.ndarray, c: complex, r: float,
              normA: float, normB: float):
    """Returns (e, rho) for the pairs (lam_i, X[:, i])."""
    AX = A @ X
    BX = B @ X
    R = AX - BX * lam[None, :]
    rn = np.linalg.norm(R, axis=0)
    bxn = np.linalg.norm(BX, axis=0)
    xn = np.linalg.norm(X, axis=0)
    with np.errstate(divide="ignore", invalid="ignore"):
        e = rn / ((abs(c) + r) * bxn)
        rho = rn / ((normA + np.abs(lam) * normB) * xn)
    bad = ~np.isfinite(lam)
    e[bad] = np.inf
    rho[bad] = np.inf
    return e, rho


def hsrr(A, B, U: np.ndarray, sigma: complex, c: complex, r: float,
         normA: float, normB: float, rng: np.random.Generator | None = None) -> dict:
    """[Y, Lambda, X] = HSRR(A, B, U, sigma) (extraction steps of Alg. SIsketch) plus errors."""
    V, rep_v = orth_cgs2(U, rng)
    AV = A @ V
    BV = B @ V
    W, rep_w = orth_cgs2(AV - sigma * BV, rng)
    Ah = W.conj().T @ AV
    Bh = W.conj().T @ BV
    HA, HB, PL, PR = sla.qz(Ah, Bh, output="complex")   # PL^* Ah PR = HA
    alpha = np.diag(HA).copy()
    beta = np.diag(HB).copy()
    with np.errstate(divide="ignore", invalid="ignore"):
        lam = np.where(beta != 0, alpha / np.where(beta != 0, beta, 1), np.inf + 0j)
    VR = triangular_right_eigvecs(HA, HB)
    X = V @ (PR @ VR)
    X = X / np.linalg.norm(X, axis=0)[None, :]
    e, rho = residuals(A, B, lam, X, c, r, normA, normB)
    return {"lam": lam, "X": X, "e": e, "rho": rho, "V": V, "W": W,
            "Ah": Ah, "Bh": Bh, "replaced": (rep_v, rep_w)}


def in_disk(lam: np.ndarray, c: complex, r: float) -> np.ndarray:
    """Strict membership |lambda - c| < r (eigenvalues on the contour are excluded,
    Sec. 2.2 footnote)."""
    lam = np.asarray(lam)
    with np.errstate(invalid="ignore"):
        return np.isfinite(lam) & (np.abs(lam - c) < r)


def ghost_filter(lam, e, c: complex, r: float, tau_g: float) -> np.ndarray:
    """Filtered pairs (Sec. 3.2): Ritz value in D and relative error e_i < tau_g."""
    return in_disk(lam, c, r) & (np.asarray(e) < tau_g)


def order_pairs(lam, filt, c: complex) -> np.ndarray:
    """Output order: filtered pairs first, each group by |lambda - c| ascending."""
    d = np.where(np.isfinite(lam), np.abs(lam - c), np.inf)
    return np.lexsort((d, ~np.asarray(filt)))
