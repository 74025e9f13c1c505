"""Pins of the oracle's quadrature coefficients against closed forms fixed by the
paper (Sec. 4.3 Lemma 1 and toy cases, Sec. 4.4 Corollary, Sec. 5 Thm 2,
Eq. mobiustrans, Prop. 1, Fig. mobius caption)."""
import os

import numpy as np
import pytest

from oracle import coeffs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _sample_points(c, r, n=400, seed=3):
    g = np.random.default_rng(seed)
    rad = r * np.concatenate([g.uniform(0.0, 0.95, n // 2), g.uniform(1.05, 3.0, n // 2)])
    ang = g.uniform(0, 2 * np.pi, n)
    return c + rad * np.exp(1j * ang)


def compact_form_error(k, c, r):
    z = _sample_points(c, r)
    p, w = coeffs.trapezoid_poles_weights(c, r, k)
    got = coeffs.rational_filter(z, p, w)
    ref = 1.0 / (1.0 + ((z - c) / r) ** k)          # Lemma 1 generalised, retyped from Sec. 4.3
    return float(np.max(np.abs(got - ref) / np.maximum(np.abs(ref), 1e-3)))


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 7, 8, 16, 33, 64])
@pytest.mark.parametrize("c,r", [(0.0, 1.0), (3.0 - 2.0j, 0.5), (2438.1 + 2.46j, 10.07)])
def test_lemma1_compact_form(k, c, r):
    # rounding of z - c and p_i - c grows with |c|/r; a wrong pole, weight or angle is O(1)
    assert compact_form_error(k, c, r) < 1e-13 * k * max(1.0, abs(c) / r)


def test_toy_cases_k2_k4():
    rows = [l.split() for l in open(os.path.join(GOLD, "trapezoid_k2_k4.txt")) if l.strip() and l[0] != "#"]
    for k in (2, 4):
        sel = [r for r in rows if int(r[0]) == k]
        p, w = coeffs.trapezoid_poles_weights(0.0, 1.0, k)
        for r in sel:
            i = int(r[1]) - 1
            pole = np.exp(1j * np.pi * float(r[2]))
            assert abs(p[i] - pole) < 1e-15
            assert abs(w[i] - pole * float(r[3])) < 1e-15
    z = _sample_points(0.0, 1.0)
    p2, w2 = coeffs.trapezoid_poles_weights(0.0, 1.0, 2)
    p4, w4 = coeffs.trapezoid_poles_weights(0.0, 1.0, 4)
    R2 = coeffs.rational_filter(z, p2, w2)
    R4 = coeffs.rational_filter(z, p4, w4)
    assert np.allclose(R2, 1.0 / (1.0 + z * z), rtol=1e-12, atol=1e-14)
    assert np.allclose(R4, coeffs.rational_filter(z * z, p2, w2), rtol=1e-12, atol=1e-14)


def composite_error(p, q, c=0.3 + 0.1j, r=2.0):
    z = _sample_points(c, r, seed=p * 100 + q)
    got = coeffs.composite_filter(z, c, r, p, q)
    ref = 1.0 / (1.0 + ((z - c) / r) ** (p * q))
    return float(np.max(np.abs(got - ref) / np.maximum(np.abs(ref), 1e-3)))


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 7, 8, 16])
@pytest.mark.parametrize("q", [1, 2, 3, 4, 8])
def test_thm2_composite_equals_full_rule(p, q):
    """Thm 2: R_{c,r,pq} = R_{0,1,p}(M(R_{c,r,q})) in summation form (even and odd p)."""
    assert composite_error(p, q) < 1e-9


def test_thm2_statement_sign_negates_even():
    """The sign as printed in the statement of Thm 2, sum c_j (R - s_j)^{-1} R,
    gives -R_{c,r,pq} for even p: the oracle's (s_j - R)^{-1} R reading is the one
    that reproduces the full rule."""
    c, r, p, q = 0.0, 1.0, 4, 4
    z = _sample_points(c, r)
    pp, ww = coeffs.trapezoid_poles_weights(c, r, q)
    t = coeffs.rational_filter(z, pp, ww)
    s, cc, _ = coeffs.outer_shifts_weights(p)
    stmt = sum(cj * t / (t - sj) for sj, cj in zip(s, cc))
    ref = 1.0 / (1.0 + ((z - c) / r) ** (p * q))
    assert np.allclose(stmt, -ref, rtol=1e-9, atol=1e-12)


def test_mobius_identity_on_figure_grid():
    """Eq. mobiustrans: M(R_{k1}(z)) = z^{k1}; grid of the Fig. mobius caption
    (201 x 201 points on [-2,2]^2, k1 = 8)."""
    x = np.linspace(-2, 2, 201)
    z = (x[None, :] + 1j * x[:, None]).ravel()
    p, w = coeffs.trapezoid_poles_weights(0.0, 1.0, 8)
    dmin = np.min(np.abs(z[:, None] - p[None, :]), axis=1)
    z = z[(dmin > 1e-3) & (np.abs(z) > 1e-3)]
    lhs = coeffs.mobius(coeffs.rational_filter(z, p, w))
    rhs = z ** 8
    assert np.max(np.abs(lhs - rhs) / np.maximum(np.abs(rhs), 1.0)) < 1e-9


@pytest.mark.parametrize("p,q", [(2, 4), (4, 4), (8, 8), (3, 4), (5, 2)])
def test_prop1_pole_transfer(p, q):
    """Prop. 1: R_{c,r,q}(p_i^{(pq)}) equals some s_j^{(p)} (or is infinite, odd p)."""
    c, r = 1.0 + 1.0j, 3.0
    poles, _ = coeffs.trapezoid_poles_weights(c, r, p * q)
    s, _, _ = coeffs.outer_shifts_weights(p)
    for pole in poles:
        y = (pole - c) / r
        denom = 1.0 + y ** q                      # R_q = 1/denom (Lemma 1)
        if p % 2 == 1 and abs(denom) < 1e-12:
            continue                              # the infinite shift of odd p
        t = 1.0 / denom
        assert np.min(np.abs(s - t)) < 1e-10 * max(1.0, abs(t))
    # every s_j is hit (the map is onto the shifts)
    y = (poles - c) / r
    hit = [1.0 / (1.0 + v ** q) for v in y if abs(1.0 + v ** q) > 1e-12]
    for sj in s:
        assert np.min(np.abs(np.array(hit) - sj)) < 1e-10


@pytest.mark.parametrize("p", [1, 2, 3, 4, 8, 16, 64])
def test_shifts_on_half_line(p):
    """Fig. mobius caption: the poles map onto the line Re(z) = 1/2."""
    s, c, odd = coeffs.outer_shifts_weights(p)
    assert np.allclose(s.real, 0.5, atol=1e-13)
    assert len(s) == p - (p % 2)
    assert odd == (1.0 / p if p % 2 else 0.0)


def separation_brute(k, a=1.0, b=1.1, nang=4096):
    """Spectrum separation Eq. (ratio) of the k-point trapezoidal rule on the circle |z| = a,
    by brute force over circles |z| = a (inf over the inner disk, max modulus principle)
    and |z| = b (sup over the outer region)."""
    p, w = coeffs.trapezoid_poles_weights(0.0, a, k)
    ang = np.linspace(0, 2 * np.pi, nang, endpoint=False)
    ang = np.concatenate([ang, np.pi * (2 * np.arange(k) + 1) / k, np.array([0.0])])
    inner = np.abs(coeffs.rational_filter(a * 0.999999 * np.exp(1j * ang), p, w)).min()
    outer = np.abs(coeffs.rational_filter(b * np.exp(1j * ang), p, w)).max()
    return outer / inner


@pytest.mark.parametrize("k", [2, 4, 8, 16, 32, 64, 128])
def test_corollary_trapezoid_separation(k):
    """Corollary (Sec. 4.4): separation 2/((b/a)^k - 1), a = 1, b = 1.1 (Sec. 6.1), and it
    is never below the inverse-power optimum (a/b)^k of Thm 4.2."""
    got = separation_brute(k)
    ref = 2.0 / (1.1 ** k - 1.0)
    assert abs(got - ref) / ref < 1e-4
    assert got >= (1.0 / 1.1) ** k
