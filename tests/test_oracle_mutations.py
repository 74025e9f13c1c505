"""Planted mistakes: each plausible slip in the oracle (an index, a sign, a dropped
term, a transposed operand) is caught by one of the pins. The mistakes are planted
in the oracle on the CPU with monkeypatch; the pins are the functions of the pin tests."""
import numpy as np

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
