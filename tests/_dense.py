"""Dense spectral definitions used to pin the oracle (Sec. 2.2, Eq. CIoperator):
for a diagonalizable pencil A X = B X Lambda, f(B^{-1}A) = X f(Lambda) X^{-1}.
Computed with SciPy's dense generalized eigensolver; shares nothing with the oracle."""
import numpy as np
import scipy.linalg as sla


def spectral_apply(A, B, f, Y):
    Ad = A.toarray() if hasattr(A, "toarray") else np.asarray(A)
    Bd = B.toarray() if hasattr(B, "toarray") else np.asarray(B)
    lam, X = sla.eig(Ad, Bd)
    coef = np.linalg.solve(X, Y)
    return X @ (f(lam)[:, None] * coef), lam, np.linalg.cond(X)


def planted_pencil(n, lam, seed=0, b_identity=False):
    """Sparse-format pencil with prescribed eigenvalues: B SPD (or I), A = B T diag(lam) T^{-1}."""
    import scipy.sparse as sp
    g = np.random.default_rng(seed)
    T = np.eye(n) + 0.3 * (g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))) / np.sqrt(n)
    if b_identity:
        Bd = np.eye(n)
    else:
        Mr = g.standard_normal((n, n)) / np.sqrt(n)
        Bd = np.eye(n) + 0.2 * (Mr @ Mr.T)
    Ad = Bd @ T @ np.diag(lam) @ np.linalg.inv(T)
    return sp.csr_matrix(Ad.astype(np.complex128)), sp.csr_matrix(Bd.astype(np.complex128))
