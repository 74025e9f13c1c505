"""The two eigensolvers of Sec. 3: Alg. 1 (fixed outer order, subspace
iteration) and Alg. 2 (outer order doubled each iteration, Krylov reuse).

reading (stop test, Sec. 3.2 and Sec. 6.3): with n_found the number of filtered
pairs (Ritz value in D and e_i < tau_g), stop when
  t >= 2, n_found_t == n_found_{t-1} and every filtered pair has rho_i < tau, or
  t == 1, n_found >= 1 and every filtered pair has rho_i < tau,
or when max_outer iterations are spent. tau applies to rho_i (the residual
||Ax - lambda Bx|| / ((||A||_1 + |lambda| ||B||_1) ||x||)), tau_g to e_i (Eq. rel-error).
reading (Alg. 2 nesting): the roots of z^p = -1 are not roots of z^{2p} = -1, so
the shifts s^{(p)} are not a subset of s^{(2p)} and U/2 + sum_new c_j U_j is not
R_{c,r,2pq}. Each doubling therefore solves all 2p shifts in the existing
per-column Krylov bases (extending them only where a shift misses tol) and
forms U = sum over all 2p shifts, which equals R_{c,r,2pq}(B^{-1}A) Y.
"""
from __future__ import annotations

import time

import numpy as np

from .coeffs import outer_shifts_weights
from .hsrr import hsrr, ghost_filter, order_pairs
from .inner import InnerOperator
from .msgmres import ColumnKrylov, filter_apply
from .pencil import norm1


DEFAULTS = dict(tau_g=1e-2, tau=1e-10, gmres_tol=1e-12, m_max=100, max_outer=10)


def _stop(t, n_found, prev, rho, filt, tau):
    conv = bool(np.all(rho[filt] < tau))
    if t == 1:
        return n_found >= 1 and conv
    return n_found == prev and conv


def _finish(res, c, tau_g, r):
    filt = ghost_filter(res["lam"], res["e"], c, r, tau_g)
    order = order_pairs(res["lam"], filt, c)
    return filt, order


def solve(A, B, c: complex, r: float, p: int, q: int, Y0: np.ndarray, driver: int = 1,
          sigma: complex | None = None, tau_g: float = DEFAULTS["tau_g"],
          tau: float = DEFAULTS["tau"], gmres_tol: float = DEFAULTS["gmres_tol"],
          m_max: int = DEFAULTS["m_max"], max_outer: int = DEFAULTS["max_outer"],
          seed: int = 0, G: InnerOperator | None = None) -> dict:
    """All eigenpairs of (A, B) in D = {|z - c| < r}. Returns a dict with the
    pairs ordered filtered-first, n_found, history and counters."""
    sigma = c if sigma is None else sigma           # sigma = c (Sec. 6 preamble)
    t0 = time.perf_counter()
    if G is None:
        G = InnerOperator(A, B, c, r, q)            # set-up of Alg. 1/2
    t_factor = time.perf_counter() - t0
    nA, nB = norm1(A), norm1(B)
    rng = np.random.Generator(np.random.PCG64(seed + 7))
    Y = np.asarray(Y0, dtype=np.complex128)
    n, k = Y.shape
    hist = []
    prev = None
    status = "noconv"
    if driver == 1:
        res = None
        for t in range(1, max_outer + 1):
            U, st = filter_apply(G, Y, p, gmres_tol, m_max, return_stats=True)   # filter step
            res = hsrr(A, B, U, sigma, c, r, nA, nB, rng)                        # extraction step
            filt, order = _finish(res, c, tau_g, r)                              # ghost filter
            n_found = int(filt.sum())
            hist.append({"t": t, "n_found": n_found, "gmres_iters": st["gmres_iters"],
                         "max_rho_filtered": float(np.max(res["rho"][filt])) if n_found else 0.0,
                         "p": p})
            if _stop(t, n_found, prev, res["rho"], filt, tau):
                status = "ok"
                break
            prev = n_found
            Y = res["X"]                               # Y <- Ritz vectors
    elif driver == 2:
        Yt = G.apply(Y)                                # Alg. 2: G(Y) once
        cols = [ColumnKrylov(G.apply, Yt[:, j], m_max) for j in range(k)]
        pc = p
        res = None
        for t in range(1, max_outer + 1):
            s, cw, odd = outer_shifts_weights(pc)
            iters = []
            for kr in cols:                             # all shifts, reuse + expand
                kr.run(s, gmres_tol)
                iters.append(kr.J)
            U = np.stack([kr.combine(s, cw, odd) for kr in cols], axis=1)   # combination step
            res = hsrr(A, B, U, sigma, c, r, nA, nB, rng)                  # extraction step
            filt, order = _finish(res, c, tau_g, r)
            n_found = int(filt.sum())
            hist.append({"t": t, "n_found": n_found, "gmres_iters": iters,
                         "max_rho_filtered": float(np.max(res["rho"][filt])) if n_found else 0.0,
                         "p": pc})
            if _stop(t, n_found, prev, res["rho"], filt, tau):
                status = "ok"
                break
            prev = n_found
            pc *= 2                                     # doubling step
    else:
        raise ValueError("driver must be 1 or 2")
    filt, order = _finish(res, c, tau_g, r)
    return {"lam": res["lam"][order], "X": res["X"][:, order], "e": res["e"][order],
            "rho": res["rho"][order], "n_found": int(filt.sum()), "status": status,
            "history": hist, "t_factor": t_factor,
            "n_G_columns": G.n_applies, "time": time.perf_counter() - t0}
