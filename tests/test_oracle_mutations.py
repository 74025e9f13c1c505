"""Planted mistakes: each plausible slip in the oracle (an index, a sign, a dropped
term, a transposed operand) is caught by one of the pins. The mistakes are planted
in the oracle on the CPU with monkeypatch; the pins are the functions of the pin tests."""
import numpy as np
import pytest

import ie_inputs
from oracle import coeffs, inner, msgmres, pencil
from test_oracle_coeffs import compact_form_error, composite_error
from _dense import spectral_apply


def test_wrong_pole_angle_is_caught(monkeypatch):
    def bad(c, r, k):                      # theta_i = 2 i pi / k  (index slip)
        i = np.arange(1, k + 1)
        e = np.exp(1j * 2 * i * np.pi / k)
        return c + r * e, r * e / k
    monkeypatch.setattr(coeffs, "trapezoid_poles_weights", bad)
    assert compact_form_error(8, 0.0, 1.0) > 1e-3


def test_missing_weight_factor_is_caught(monkeypatch):
    good = coeffs.trapezoid_poles_weights
    monkeypatch.setattr(coeffs, "trapezoid_poles_weights", lambda c, r, k: (good(c, r, k)[0], good(c, r, k)[1] * k))
    assert compact_form_error(4, 0.0, 1.0) > 1e-3


def test_dropped_odd_term_is_caught(monkeypatch):
    good = coeffs.outer_shifts_weights
    monkeypatch.setattr(coeffs, "outer_shifts_weights", lambda p: good(p)[:2] + (0.0,))
    assert composite_error(3, 4) > 1e-3
    assert composite_error(4, 4) < 1e-9      # even p unaffected: the odd pin is what catches it


def test_statement_sign_is_caught(monkeypatch):
    good = coeffs.outer_shifts_weights
    monkeypatch.setattr(coeffs, "outer_shifts_weights", lambda p: (good(p)[0], -good(p)[1], good(p)[2]))
    assert composite_error(4, 4) > 1e-3


def _gmres_error():
    pen = ie_inputs.make_pencil(6, seed=2)
    A, B = pencil.pencil_matrices(pen)
    c, r = A.diagonal().mean(), 20.0
    G = inner.InnerOperator(A, B, c, r, 4)
    Y = ie_inputs.random_block(pen.n, 2, seed=1)
    U = msgmres.filter_apply(G, Y, 4, tol=1e-13, m_max=pen.n)
    ref, _, _ = spectral_apply(A, B, lambda z: 1 / (1 + ((z - c) / r) ** 16), Y)
    return np.linalg.norm(U - ref) / np.linalg.norm(ref)


def test_gmres_pin_passes_unmutated():
    assert _gmres_error() < 1e-8


def test_transposed_projection_is_caught(monkeypatch):
    def bad_step(self):                      # V^T w instead of V^H w
        j = self.J
        w = self.G_apply(self.V[:, j])
        Vj = self.V[:, : j + 1]
        for _ in range(2):
            h = Vj.T @ w
            w = w - Vj @ h
        self.H[: j + 1, j] = Vj.conj().T @ self.G_apply(self.V[:, j])
        hn = np.linalg.norm(w)
        self.H[j + 1, j] = hn
        self.J = j + 1
        self.V[:, j + 1] = w / hn
    monkeypatch.setattr(msgmres.ColumnKrylov, "step", bad_step)
    assert _gmres_error() > 1e-4


def test_wrong_shift_sign_is_caught(monkeypatch):
    good = msgmres.ColumnKrylov.solve_shift
    monkeypatch.setattr(msgmres.ColumnKrylov, "solve_shift", lambda self, s: good(self, -s))
    assert _gmres_error() > 1e-4


# ---------------------------------------------------------------- adjoint / sensitivities
def _small_pencil():
    pen = ie_inputs.make_pencil(6, seed=4)
    return pencil.pencil_matrices(pen)


def _adjoint_identity_error():
    """B^H G_adj V against G^H B^H V (the identity pin of the adjoint operator)."""
    from oracle import adjoint
    A, B = _small_pencil()
    n = A.shape[0]
    c, r = A.diagonal().mean(), 20.0
    Gd = inner.InnerOperator(A, B, c, r, 4).apply(np.eye(n, dtype=np.complex128))
    V = ie_inputs.random_block(n, 2, seed=3)
    Bh = B.toarray().conj().T
    lhs = Bh @ adjoint.adjoint_inner(A, B, c, r, 4).apply(V)
    rhs = Gd.conj().T @ (Bh @ V)
    return np.linalg.norm(lhs - rhs) / np.linalg.norm(rhs)


def _sensitivity_error():
    """Largest relative gap between diag_sensitivity and central differences of dense
    eigenvalues on a 36 x 36 pencil (the finite-difference pin)."""
    import scipy.linalg as sla
    from oracle import adjoint
    A, B = _small_pencil()
    Ad, Bd = A.toarray(), B.toarray()
    lam, VL, VR = sla.eig(Ad, Bd, left=True, right=True)
    gaps = np.array([np.min(np.abs(np.delete(lam, i) - lam[i])) for i in range(len(lam))])
    sel = np.argsort(-gaps)[:3]
    S = adjoint.diag_sensitivity(B, VR[:, sel], VL[:, sel], alpha=1j)
    worst = 0.0
    for j in (0, 7, 20):
        d = []
        for t in (1e-3, -1e-3):
            Ap = Ad.copy()
            Ap[j, j] += 1j * t
            lt = np.linalg.eigvals(np.linalg.solve(Bd, Ap))
            d.append(np.array([lt[np.argmin(np.abs(lt - lam[i]))] for i in sel]))
        fd = (d[0] - d[1]) / 2e-3
        worst = max(worst, float(np.max(np.abs(S[j] - fd) / np.abs(fd))))
    return worst


def test_adjoint_pins_pass_unmutated():
    assert _adjoint_identity_error() < 1e-11
    assert _sensitivity_error() < 1e-5


def test_unconjugated_adjoint_nodes_are_caught(monkeypatch):
    from oracle import adjoint

    def bad(A, B, c, r, q):                  # the primal disk's nodes for the adjoint pencil
        AH, BH = adjoint.adjoint_pencil(A, B)
        return inner.InnerOperator(AH, BH, c, r, q)
    monkeypatch.setattr(adjoint, "adjoint_inner", bad)
    assert _adjoint_identity_error() > 1e-3


def test_unconjugated_left_vector_is_caught(monkeypatch):
    from oracle import adjoint
    good = adjoint.diag_sensitivity
    monkeypatch.setattr(adjoint, "diag_sensitivity",
                        lambda B, X, Y, alpha=1.0: good(B, X, np.conj(Y), alpha))
    assert _sensitivity_error() > 1e-3


def test_denominator_without_b_is_caught(monkeypatch):
    from oracle import adjoint

    def bad(B, X, Y, alpha=1.0):             # y^H x instead of y^H B x
        den = np.sum(np.conj(Y) * X, axis=0)
        return alpha * np.conj(Y) * X / den[None, :]
    monkeypatch.setattr(adjoint, "diag_sensitivity", bad)
    assert _sensitivity_error() > 1e-3


# ---------------------------------------------------------------- reference eigenvalues
from oracle import reference_eigs
from test_oracle_reference_eigs import nearest_error


def test_reference_eigs_pin_passes_unmutated():
    assert nearest_error(12, 0, 10, 0.37 + 0.11j) < 1e-12


def _bad_nearest(sign, which):
    import scipy.sparse.linalg as spla

    def bad(A, B, sigma, count, tol=1e-14, seed=0):
        n = A.shape[0]
        lu = spla.splu((A - sigma * B).tocsc())
        op = spla.LinearOperator((n, n), matvec=lambda x: lu.solve(B @ x), dtype=np.complex128)
        v0 = np.random.default_rng(seed).standard_normal(n).astype(np.complex128)
        theta = spla.eigs(op, k=count, which=which, tol=tol, v0=v0, ncv=max(2 * count + 1, 40),
                          return_eigenvectors=False)
        lam = sigma + sign / theta
        return lam[np.argsort(np.abs(lam - sigma))]
    return bad


def test_wrong_shift_invert_sign_is_caught(monkeypatch):
    monkeypatch.setattr(reference_eigs, "nearest_eigenvalues", _bad_nearest(-1.0, "LM"))
    assert nearest_error(12, 0, 10, 0.37 + 0.11j) > 1e-3


def test_wrong_end_of_spectrum_is_caught(monkeypatch):
    from scipy.sparse.linalg import ArpackNoConvergence
    monkeypatch.setattr(reference_eigs, "nearest_eigenvalues", _bad_nearest(1.0, "SM"))
    try:
        err = nearest_error(12, 0, 10, 0.37 + 0.11j)
    except ArpackNoConvergence:      # the far end of (A - sigma B)^{-1} B does not even converge
        err = np.inf
    assert err > 1e-3


def test_radius_off_by_one_is_caught(monkeypatch):
    def bad(distances, count):
        d = np.sort(np.asarray(distances))
        return 0.5 * (float(d[count]) + float(d[count + 1]))
    monkeypatch.setattr(reference_eigs, "disk_radius", bad)
    import test_oracle_reference_eigs as pins
    with pytest.raises(AssertionError):
        pins.test_disk_radius_hand_built_and_exact_count()


def test_median_without_tie_break_is_caught(monkeypatch):
    monkeypatch.setattr(reference_eigs, "median_eigenvalue",
                        lambda lam: np.asarray(lam)[np.argsort(np.asarray(lam).real, kind="stable")][len(lam) // 2])
    import test_oracle_reference_eigs as pins
    with pytest.raises(AssertionError):
        pins.test_median_eigenvalue_hand_built()
