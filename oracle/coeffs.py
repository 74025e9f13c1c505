"""Quadrature coefficients of the trapezoidal rule and of its composite form.

Sec. 2.2 Eq. (pwtp): poles p_i = r e^{i theta_i} + c, weights w_i = r e^{i theta_i}/k,
theta_i = (2i-1) pi / k, i = 1..k.
Sec. 2.2 Eq. (discretizedCI): R_k(z) = sum_i w_i / (p_i - z).
Sec. 4.3 Lemma 1 (and its generalisation below it): R_{c,r,k}(z) = 1 / (1 + ((z-c)/r)^k).
Sec. 5 Eq. (mobiustrans): M(z) = (1 - z) / z.
Sec. 5 Thm 2 Eqs. (Rcrm), (Rcrmodd): the composite summation form with outer roots
sigma_j of z^{k2} = -1, c_j = -(1/k2) sigma_j / (1 + sigma_j), s_j = 1 / (1 + sigma_j).

reading (sign): the statement of Thm 2 writes (R - s_j)^{-1} R, the last line of
its proof writes (s_j - R)^{-1} R. Only the latter equals R_{c,r,k1 k2}; the
statement's sign negates the even-k2 result. The oracle uses (s_j - R)^{-1} R.
reading (odd k2): the extra term for sigma = -1 is (1/k2) R_{c,r,k1} (the
statement's 1/k2; the proof's 1/k1 is a typo).
Notation: q = k1 (inner order, number of factorisations), p = k2 (outer order).
"""
from __future__ import annotations

import numpy as np


def trapezoid_poles_weights(c: complex, r: float, k: int):
    """Eq. (pwtp). Returns (poles, weights), complex arrays of length k."""
    if k < 1:
        raise ValueError("k >= 1")
    i = np.arange(1, k + 1)
    theta = (2 * i - 1) * np.pi / k
    e = np.exp(1j * theta)
    return c + r * e, r * e / k


def rational_filter(z, poles, weights):
    """Eq. (discretizedCI): R_k(z) = sum_i w_i / (p_i - z), elementwise in z."""
    z = np.asarray(z, dtype=np.complex128)
    out = np.zeros(z.shape, dtype=np.complex128)
    for p, w in zip(poles, weights):
        out += w / (p - z)
    return out


def compact_filter(z, c: complex, r: float, k: int):
    """Lemma 1 generalised (Sec. 4.3): R_{c,r,k}(z) = 1 / (1 + ((z - c)/r)^k)."""
    z = np.asarray(z, dtype=np.complex128)
    return 1.0 / (1.0 + ((z - c) / r) ** k)


def mobius(z):
    """Eq. (mobiustrans): M(z) = (1 - z)/z."""
    z = np.asarray(z, dtype=np.complex128)
    return (1.0 - z) / z


def outer_roots(p: int) -> np.ndarray:
    """The p roots of z^p = -1, sigma_j = e^{i (2j-1) pi / p}, j = 1..p (Thm 2)."""
    j = np.arange(1, p + 1)
    return np.exp(1j * (2 * j - 1) * np.pi / p)


def outer_shifts_weights(p: int):
    """Thm 2 summation form. Returns (s, c, odd_coef):
    s_j = 1/(1+sigma_j), c_j = -(1/p) sigma_j/(1+sigma_j) over the roots with
    sigma_j != -1, and odd_coef = 1/p when p is odd (the sigma = -1 term,
    Eq. (Rcrmodd)), else 0. The sigma = -1 root is j = (p+1)/2, dropped by index."""
    if p < 1:
        raise ValueError("p >= 1")
    sig = outer_roots(p)
    keep = np.ones(p, dtype=bool)
    odd = 0.0
    if p % 2 == 1:
        keep[(p + 1) // 2 - 1] = False
        odd = 1.0 / p
    sig = sig[keep]
    s = 1.0 / (1.0 + sig)
    c = -(1.0 / p) * sig / (1.0 + sig)
    return s, c, odd


def composite_filter(z, c: complex, r: float, p: int, q: int):
    """Thm 2: R_{c,r,pq}(z) = sum_j c_j (s_j - t)^{-1} t + odd_coef * t, t = R_{c,r,q}(z),
    with the inner R_{c,r,q} evaluated as the q-pole sum of Eq. (discretizedCI)."""
    poles, weights = trapezoid_poles_weights(c, r, q)
    t = rational_filter(z, poles, weights)
    s, cc, odd = outer_shifts_weights(p)
    out = odd * t
    for sj, cj in zip(s, cc):
        out = out + cj * t / (sj - t)
    return out
