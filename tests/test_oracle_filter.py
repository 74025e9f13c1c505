"""Pins of the oracle's inner operator G and its multi-shift GMRES filter against
dense spectral definitions (Sec. 2.2 Eq. CIoperator; Sec. 3.2 Eqs. linearsolve1,
linearsolve2, linearsolve1abs; Thm 2)."""
import numpy as np
import pytest

import ie_inputs
from oracle import coeffs, inner, msgmres, pencil
from _dense import spectral_apply, planted_pencil


@pytest.fixture(scope="module")
def small_pencil():
    pen = ie_inputs.make_pencil(8, seed=5)          # n = 64 convection-diffusion pencil
    A, B = pencil.pencil_matrices(pen)
    import scipy.linalg as sla
    lam = sla.eigvals(A.toarray(), B.toarray())
    o = np.lexsort((lam.imag, lam.real))
    c = lam[o][len(lam) // 2]
    d = np.sort(np.abs(lam - c))
    r = 0.5 * (d[5] + d[6])
    return A, B, c, r


def test_dia_to_csr_matches_stencil():
    """DIA assembly against the stencil written entry by entry (m = 3)."""
    pen = ie_inputs.make_pencil(3, seed=1)
    A, B = pencil.pencil_matrices(pen)
    m, h = 3, 0.25
    Ad = A.toarray()
    for iy in range(m):
        for ix in range(m):
            i = ix + m * iy
            assert Ad[i, i] == pytest.approx(4 / h**2 + 1j * pen.gamma[i])
            if ix + 1 < m:
                assert Ad[i, i + 1] == pytest.approx(-1 / h**2 + 3 / (2 * h))
            if ix > 0:
                assert Ad[i, i - 1] == pytest.approx(-1 / h**2 - 3 / (2 * h))
            if iy + 1 < m:
                assert Ad[i, i + m] == pytest.approx(-1 / h**2 + 1 / h)
            if iy > 0:
                assert Ad[i, i - m] == pytest.approx(-1 / h**2 - 1 / h)
    Bd = B.toarray()
    assert np.allclose(Bd, Bd.T) and np.all(np.diag(Bd).real >= 1.0)
    assert np.count_nonzero(Ad) == 5 * 9 - 4 * 3
    assert pencil.norm1(A) == pytest.approx(np.abs(Ad).sum(axis=0).max())


@pytest.mark.parametrize("q", [2, 3, 4, 8])
def test_inner_operator_is_Rq_of_pencil(small_pencil, q):
    A, B, c, r = small_pencil
    G = inner.InnerOperator(A, B, c, r, q)
    Y = ie_inputs.random_block(A.shape[0], 5, seed=2)
    got = G.apply(Y)
    ref, lam, condX = spectral_apply(A, B, lambda z: 1.0 / (1.0 + ((z - c) / r) ** q), Y)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-10 * max(1.0, condX / 1e3)


@pytest.mark.parametrize("p", [2, 3, 4, 8])
def test_multishift_gmres_each_shift_matches_dense_solve(small_pencil, p):
    """Every shift of one shared Krylov space reaches the dense (G - s_j I)^{-1} ytilde."""
    A, B, c, r = small_pencil
    q = 4
    G = inner.InnerOperator(A, B, c, r, q)
    n = A.shape[0]
    y = ie_inputs.random_block(n, 1, seed=9)[:, 0]
    yt = G.apply(y)
    Gd = G.apply(np.eye(n))
    s, _, _ = coeffs.outer_shifts_weights(p)
    kr = msgmres.ColumnKrylov(G.apply, yt, m_max=n)
    assert kr.run(s, 1e-13)
    for sj in s:
        yv, res = kr.solve_shift(sj)
        x = kr.V[:, : kr.J] @ yv
        xd = np.linalg.solve(Gd - sj * np.eye(n), yt)
        assert res <= 1e-13
        assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-9
    # Arnoldi relation (G - sI) V_J = V_{J+1} (Hbar - s Ibar) at s = 0, orthonormal basis
    J = kr.J
    V = kr.V[:, : J + 1]
    assert np.linalg.norm(V.conj().T @ V - np.eye(J + 1)) < 1e-12
    assert np.linalg.norm(Gd @ kr.V[:, :J] - V @ kr.H[: J + 1, :J]) < 1e-11 * np.linalg.norm(Gd)


@pytest.mark.parametrize("p,q", [(4, 4), (3, 4), (2, 3), (8, 2), (1, 4)])
def test_composite_filter_equals_full_rule_on_pencil(small_pencil, p, q):
    """Thm 2 at matrix level: composite U equals the pq-pole simple rule (Eq.
    discretizedCIoperator with pq sparse solves) and X R_pq(Lambda) X^{-1} Y."""
    A, B, c, r = small_pencil
    G = inner.InnerOperator(A, B, c, r, q)
    n = A.shape[0]
    Y = ie_inputs.random_block(n, 4, seed=11)
    U = msgmres.filter_apply(G, Y, p, tol=1e-13, m_max=n)
    full = inner.InnerOperator(A, B, c, r, p * q).apply(Y)
    ref, lam, condX = spectral_apply(A, B, lambda z: 1.0 / (1.0 + ((z - c) / r) ** (p * q)), Y)
    assert np.linalg.norm(U - full) / np.linalg.norm(full) < 1e-9
    assert np.linalg.norm(U - ref) / np.linalg.norm(ref) < 1e-9 * max(1.0, condX / 1e3)


def test_filter_on_planted_spectrum():
    """Planted eigenvalues: the filter keeps eigenvector components inside D and damps
    the rest exactly as 1/(1 + ((lambda-c)/r)^{pq})."""
    lam = np.array([0.1, 0.3j, -0.2 + 0.1j, 0.5, 0.45j, 1.5, 2.0 + 1j, -3.0, 1.2j, 5.0] + list(np.linspace(3, 9, 20)))
    A, B = planted_pencil(len(lam), lam, seed=4)
    c, r, p, q = 0.0, 1.0, 4, 4
    G = inner.InnerOperator(A, B, c, r, q)
    Y = ie_inputs.random_block(len(lam), 3, seed=1)
    U = msgmres.filter_apply(G, Y, p, tol=1e-13, m_max=len(lam))
    ref, _, _ = spectral_apply(A, B, lambda z: 1.0 / (1.0 + ((z - c) / r) ** (p * q)), Y)
    assert np.linalg.norm(U - ref) / np.linalg.norm(ref) < 1e-9
