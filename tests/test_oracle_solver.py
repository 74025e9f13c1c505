"""Pins of the oracle's HSRR step (Sec. 2.1) and its two drivers (Alg. 1, Alg. 2)
against planted spectra, the definition of an eigenpair, and dense QZ."""
import numpy as np
import pytest
import scipy.linalg as sla

import ie_inputs
from oracle import drivers, hsrr, pencil
from _dense import planted_pencil


def test_cgs2_orthonormal_and_span():
    g = np.random.default_rng(0)
    U = g.standard_normal((50, 8)) + 1j * g.standard_normal((50, 8))
    Q, rep = hsrr.orth_cgs2(U)
    assert rep == []
    assert np.linalg.norm(Q.conj().T @ Q - np.eye(8)) < 1e-14
    # same span, triangular relation: Q^H U upper triangular
    R = Q.conj().T @ U
    assert np.linalg.norm(np.tril(R, -1)) < 1e-12 * np.linalg.norm(U)
    assert np.linalg.norm(Q @ R - U) < 1e-12 * np.linalg.norm(U)


def test_cgs2_rank_guard():
    g = np.random.default_rng(1)
    U = g.standard_normal((40, 6)) + 1j * g.standard_normal((40, 6))
    U[:, 3] = U[:, 0] * (2 - 1j) + 1e-15 * U[:, 1]     # dependent column
    U[:, 5] = 0.0                                     # zero column
    Q, rep = hsrr.orth_cgs2(U)
    assert rep == [3, 5]
    assert np.linalg.norm(Q.conj().T @ Q - np.eye(6)) < 1e-13
    for j in (0, 1, 2, 4):                            # independent columns stay in the span
        u = U[:, j]
        assert np.linalg.norm(u - Q @ (Q.conj().T @ u)) < 1e-12 * np.linalg.norm(u)


def test_triangular_eigvecs_definition():
    g = np.random.default_rng(2)
    k = 12
    S = np.triu(g.standard_normal((k, k)) + 1j * g.standard_normal((k, k)))
    T = np.triu(g.standard_normal((k, k)) + 1j * g.standard_normal((k, k))) + 3 * np.eye(k)
    V = hsrr.triangular_right_eigvecs(S, T)
    for i in range(k):
        a, b = S[i, i], T[i, i]
        assert np.linalg.norm((b * S - a * T) @ V[:, i]) < 1e-12 * np.linalg.norm(V[:, i]) * (np.abs(S).max() + np.abs(T).max()) * 10


def test_residual_definitions_closed_form():
    import scipy.sparse as sp
    lamv = np.array([1.0, 2.0 + 1j, -1.0, 3.0])
    A = sp.csr_matrix(np.diag(lamv).astype(complex))
    B = sp.csr_matrix(np.eye(4, dtype=complex))
    X = np.eye(4, dtype=complex)[:, :2].copy()
    X[1, 0] = 1e-3                          # perturb the first pair
    lam = lamv[:2].copy()
    e, rho = hsrr.residuals(A, B, lam, X, c=0.5, r=1.0, normA=3.0, normB=1.0)
    # A x - lambda B x = (2+1j - 1) * 1e-3 e_2 for the perturbed pair
    rn = abs(1.0 + 1j) * 1e-3
    assert e[0] == pytest.approx(rn / (1.5 * np.sqrt(1 + 1e-6)), rel=1e-12)
    assert rho[0] == pytest.approx(rn / ((3.0 + 1.0) * np.sqrt(1 + 1e-6)), rel=1e-12)
    assert e[1] == 0.0 and rho[1] == 0.0


def test_in_disk_is_strict_and_ghost_filter():
    lam = np.array([0.0, 1.0, 0.999, np.inf, 0.5j])
    assert list(hsrr.in_disk(lam, 0.0, 1.0)) == [True, False, True, False, True]
    f = hsrr.ghost_filter(lam, np.array([1e-9, 1e-9, 0.5, 1e-9, 1e-3]), 0.0, 1.0, 1e-2)
    assert list(f) == [True, False, False, False, True]


PLANT = np.array([0.1, 0.3j, -0.2 + 0.1j, 0.5 - 0.4j, 0.45j,            # 5 inside D
                  1.15, 1.4 + 0.9j, -1.3, 1.25j, 2.0, -2.2j, 3.0 + 1j]
                 + list(np.linspace(3.5, 12.0, 28)) + list(-np.linspace(2.5, 9.0, 20) * 1j))


@pytest.mark.parametrize("driver", [1, 2])
@pytest.mark.parametrize("p,q", [(4, 4), (3, 4)])
def test_drivers_on_planted_spectrum(driver, p, q):
    n = len(PLANT)
    A, B = planted_pencil(n, PLANT, seed=7)
    c, r = 0.0, 1.0
    Y0 = ie_inputs.orthonormal_random_block(n, 8, seed=3)
    res = drivers.solve(A, B, c, r, p, q, Y0, driver=driver, m_max=n)
    assert res["status"] == "ok"
    assert res["n_found"] == 5
    got = res["lam"][:5]
    ref = PLANT[:5]
    dist = np.abs(got[:, None] - ref[None, :])
    assert sorted(np.argmin(dist, axis=1)) == list(range(5))    # one-to-one
    assert np.max(np.min(dist, axis=1)) < 1e-10
    assert np.all(res["rho"][:5] <= 1e-10)


def test_alg1_on_small_convection_diffusion_vs_dense_qz():
    """m = 12 pencil (n = 144): Alg. 1 and Alg. 2 find exactly the QZ eigenvalues in D."""
    pen = ie_inputs.make_pencil(12, seed=0)
    A, B = pencil.pencil_matrices(pen)
    lam = sla.eigvals(A.toarray(), B.toarray())
    o = np.lexsort((lam.imag, lam.real))
    c = lam[o][len(lam) // 2]
    d = np.sort(np.abs(lam - c))
    r = 0.5 * (d[6] + d[7])
    inD = lam[np.abs(lam - c) < r]
    Y0 = ie_inputs.orthonormal_random_block(pen.n, 12, seed=0)
    for drv in (1, 2):
        res = drivers.solve(A, B, c, r, 4, 4, Y0, driver=drv)
        assert res["status"] == "ok"
        assert res["n_found"] == len(inD) == 7
        for l in res["lam"][: res["n_found"]]:
            assert np.min(np.abs(inD - l)) / abs(l) < 1e-10
        assert np.all(res["rho"][: res["n_found"]] <= 1e-10)
