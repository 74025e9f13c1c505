"""Pins of the oracle's adjoint pencil, left eigenvectors and eigenvalue sensitivities
(oracle/adjoint.py) against dense LAPACK left eigenvectors, the spectral definition of
the adjoint filter, an identity linking G_adj to G, and central finite differences of
dense eigenvalues."""
import numpy as np
import pytest
import scipy.linalg as sla

import ie_inputs
from oracle import adjoint, coeffs, inner, pencil
from _dense import spectral_apply


@pytest.fixture(scope="module")
def c1():
    w = ie_inputs.load_workload("c1_m24")
    pen = ie_inputs.make_pencil(w["m"], seed=w["seed"])
    A, B = pencil.pencil_matrices(pen)
    return w, pen, A, B


def _dense(M):
    return M.toarray() if hasattr(M, "toarray") else np.asarray(M)


@pytest.fixture(scope="module")
def c1_eig(c1):
    """LAPACK (ggev) eigenvalues with left and right eigenvectors of the dense C1 pencil."""
    _, _, A, B = c1
    return sla.eig(_dense(A), _dense(B), left=True, right=True)


def test_adjoint_inner_is_spectral_filter_of_adjoint_pencil(c1):
    """G_adj = X' R_q(Lambda') X'^{-1} for the eigendecomposition of (A^H, B^H) and the
    q-point filter of the conjugate disk (Eq. CIoperator)."""
    w, _, A, B = c1
    c, r, q = w["center"], w["radius"], w["q"]
    G = adjoint.adjoint_inner(A, B, c, r, q)
    V = ie_inputs.random_block(A.shape[0], 3, seed=5)
    AH, BH = adjoint.adjoint_pencil(A, B)
    ref, _, cond = spectral_apply(AH, BH, lambda z: coeffs.compact_filter(z, np.conj(c), r, q), V)
    got = G.apply(V)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-9 * max(1.0, cond / 1e3)


def test_adjoint_inner_identity_with_primal(c1):
    """B^H G_adj = G^H B^H, because G = (sum_i w_i K_i^{-1}) B and
    G_adj = (sum_i conj(w_i) K_i^{-H}) B^H. G^H comes from the primal operator applied to
    the identity, so conjugated weights or transposed factors would show here."""
    w, _, A, B = c1
    c, r, q = w["center"], w["radius"], w["q"]
    n = A.shape[0]
    Gp = inner.InnerOperator(A, B, c, r, q)
    Gd = Gp.apply(np.eye(n, dtype=np.complex128))          # dense G
    Ga = adjoint.adjoint_inner(A, B, c, r, q)
    V = ie_inputs.random_block(n, 4, seed=6)
    Bh = _dense(B).conj().T
    lhs = Bh @ Ga.apply(V)
    rhs = Gd.conj().T @ (Bh @ V)
    assert np.linalg.norm(lhs - rhs) / np.linalg.norm(rhs) < 1e-11


def test_left_eigenpairs_match_dense_left_vectors(c1, c1_eig):
    """The oracle's left eigenpairs (Alg. 1 on the adjoint pencil) against LAPACK's left
    eigenvectors of (A, B): same eigenvalues, parallel vectors, and y^H A = lambda y^H B."""
    w, _, A, B = c1
    n, k = A.shape[0], w["k"]
    Y0 = ie_inputs.orthonormal_random_block(n, k, seed=w["seed"])
    res = adjoint.left_eigenpairs(A, B, w["center"], w["radius"], w["p"], w["q"], Y0)
    nf = res["n_found"]
    assert res["status"] == "ok" and nf == len(w["eig_in_disk_re"])
    Ad, Bd = _dense(A), _dense(B)
    lam, VL, VR = c1_eig
    for i in range(nf):
        li, yi = res["lam"][i], res["Y"][:, i]
        j = int(np.argmin(np.abs(lam - li)))
        assert abs(lam[j] - li) <= 1e-10 * abs(li)
        vl = VL[:, j]
        cosang = abs(np.vdot(vl, yi)) / (np.linalg.norm(vl) * np.linalg.norm(yi))
        assert cosang > 1 - 1e-9, (i, cosang)
        r = yi.conj() @ Ad - li * (yi.conj() @ Bd)
        assert np.linalg.norm(r) <= 1e-10 * (pencil.norm1(A) + abs(li) * pencil.norm1(B))


def test_pair_left_one_to_one():
    lr = np.array([1.0 + 1j, 2.0, 3.0 - 1j])
    ll = np.array([3.0 - 1j + 1e-12, 1.0 + 1j, 2.0 + 1e-13, 9.0])
    assert adjoint.pair_left(lr, ll).tolist() == [1, 2, 0]
    with pytest.raises(ValueError):
        adjoint.pair_left(np.array([1.0, 1.0 + 1e-9]), np.array([1.0, 5.0]))


def _fd_derivatives(Ad, Bd, j, lam0, h, alpha=1j):
    """Central differences of the eigenvalues nearest each lam0 entry under
    A_jj -> A_jj + alpha t (eigenvalues of B^{-1} A(t); B is well conditioned)."""
    out = []
    for t in (h, -h):
        Ap = Ad.copy()
        Ap[j, j] += alpha * t
        lam = np.linalg.eigvals(np.linalg.solve(Bd, Ap))
        out.append(np.array([lam[np.argmin(np.abs(lam - l0))] for l0 in np.atleast_1d(lam0)]))
    return (out[0] - out[1]) / (2 * h)


def test_sensitivity_matches_central_differences(c1, c1_eig):
    """d lambda_i / d gamma_j = i conj(y_j) x_j / (y^H B x) against central differences of
    dense eigenvalues, at 6 seeded nodes and the eigenvalues of the disk that are at least
    0.5 apart from every other eigenvalue. Step h = 1e-2: the dense eigenvalues (~2440)
    carry rounding errors near 5e-12, so the difference quotient is good to ~3e-10
    against derivatives of 1e-5..1e-3; the O(h^2) term is far below that."""
    w, _, A, B = c1
    Ad, Bd = _dense(A), _dense(B)
    lam, VL, VR = c1_eig
    c, r = w["center"], w["radius"]
    inside = np.flatnonzero(np.abs(lam - c) < r)
    gaps = np.array([np.min(np.abs(np.delete(lam, i) - lam[i])) for i in inside])
    sel = inside[gaps > 0.5]
    assert len(sel) >= 4
    S = adjoint.diag_sensitivity(B, VR[:, sel], VL[:, sel], alpha=1j)
    nodes = np.random.default_rng(11).choice(Ad.shape[0], size=6, replace=False)
    for j in nodes:
        fd = _fd_derivatives(Ad, Bd, j, lam[sel], 1e-2)
        for col, i in enumerate(sel):
            assert abs(S[j, col] - fd[col]) <= 1e-5 * abs(fd[col]) + 1e-9, (j, i, S[j, col], fd[col])


def test_sensitivity_uses_the_b_weighted_denominator(c1, c1_eig):
    """sum_j S[j, i] / alpha = y^H x / (y^H B x) is the derivative of lambda_i along
    A -> A + t I. With B = I it would be exactly 1; this pencil's B != I makes it differ,
    so a denominator without B fails against the dense difference."""
    w, _, A, B = c1
    Ad, Bd = _dense(A), _dense(B)
    lam, VL, VR = c1_eig
    i = int(np.argmin(np.abs(lam - w["center"])))
    S = adjoint.diag_sensitivity(B, VR[:, [i]], VL[:, [i]], alpha=1.0)
    # A -> A + t I moves lambda by t * y^H x / (y^H B x): compare with a dense difference
    h = 1e-2
    lp = np.linalg.eigvals(np.linalg.solve(Bd, Ad + h * np.eye(len(Ad))))
    lm = np.linalg.eigvals(np.linalg.solve(Bd, Ad - h * np.eye(len(Ad))))
    fd = (lp[np.argmin(np.abs(lp - lam[i]))] - lm[np.argmin(np.abs(lm - lam[i]))]) / (2 * h)
    assert abs(S[:, 0].sum() - fd) <= 1e-6 * abs(fd)
    assert abs(fd - 1.0) > 1e-3          # B != I makes this differ from 1


def test_vjp_matches_finite_difference_of_a_loss(c1, c1_eig):
    """J = sum_i Re(conj(g_i) lambda_i) with complex g: dJ/d gamma_j from vjp(S, g)
    against a central difference of J."""
    w, _, A, B = c1
    Ad, Bd = _dense(A), _dense(B)
    lam, VL, VR = c1_eig
    c, r = w["center"], w["radius"]
    inside = np.flatnonzero(np.abs(lam - c) < r)
    gaps = np.array([np.min(np.abs(np.delete(lam, i) - lam[i])) for i in inside])
    sel = inside[gaps > 0.5][:4]
    g = np.random.default_rng(12)
    gbar = g.uniform(0, 1, len(sel)) + 1j * g.uniform(-1, 1, len(sel))
    S = adjoint.diag_sensitivity(B, VR[:, sel], VL[:, sel], alpha=1j)
    grad = adjoint.vjp(S, gbar)
    for j in (3, 100, 400):
        dl = _fd_derivatives(Ad, Bd, j, lam[sel], 1e-2)
        fd = np.real(np.sum(np.conj(gbar) * dl))
        assert abs(grad[j] - fd) <= 1e-5 * np.sum(np.abs(gbar) * np.abs(dl)), (j, grad[j], fd)
