"""Seeded synthetic pencil and block generator.

Workload: A is the 5-point finite-difference discretisation of
    -Laplace(u) + (3, 2) . grad(u) + i * gamma(x, y) * u     on (0,1)^2, u = 0 on the boundary,
with gamma = 5 sin(pi x) sin(pi y) + N(0, 0.1^2) per node, and
    B = I + 0.05 * S,   S symmetric on the 5-point pattern (diagonal included), S_ij ~ U(0, 1).
Grid: m x m interior nodes, h = 1/(m+1), node (ix, iy) -> row ix + m*iy (x fastest).
Central differences for the convection term (cell Peclet number 3h/2 < 1 for m >= 2).

Random draws, in this order, from numpy PCG64(seed): gamma noise (n), S diagonal (n),
S horizontal edges (m*(m-1), row-major), S vertical edges (m*(m-1)), then any block
(complex Gaussian: real parts then imaginary parts, column-major n x k).

DIA layout (shared by every consumer): offsets = [-m, -1, 0, 1, m];
dia[d, i] = M[i, i + offsets[d]], zero where i + offsets[d] leaves the grid row/column range.
The problem statement (Ax = lambda Bx, lambda in a disk) is Sec. 1, Eq. (problem).
"""
from __future__ import annotations

import json
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
WORKLOADS_JSON = os.path.join(_HERE, "..", "tests", "golden", "workloads.json")


@dataclass
class Pencil:
    m: int
    n: int
    offsets: np.ndarray  # int64 (ndiag,)
    A_dia: np.ndarray    # complex128 (ndiag, n)
    B_dia: np.ndarray    # complex128 (ndiag, n), real-valued
    gamma: np.ndarray    # float64 (n,) coefficient field

    @property
    def half_bw(self) -> int:
        return int(np.max(np.abs(self.offsets)))


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def make_pencil(m: int, seed: int = 0, rng: np.random.Generator | None = None) -> Pencil:
    """Build the DIA pencil for an m x m grid (n = m^2). Returns host arrays."""
    if m < 2:
        raise ValueError("m must be >= 2")
    g = _rng(seed) if rng is None else rng
    n = m * m
    h = 1.0 / (m + 1)
    ix = np.tile(np.arange(m), m)          # x index of row i
    iy = np.repeat(np.arange(m), m)        # y index of row i
    x = (ix + 1) * h
    y = (iy + 1) * h
    gamma = 5.0 * np.sin(np.pi * x) * np.sin(np.pi * y) + 0.1 * g.standard_normal(n)
    s_diag = g.random(n)
    s_h = g.random(m * (m - 1))            # edge (ix, iy)-(ix+1, iy), iy-major
    s_v = g.random(m * (m - 1))            # edge (ix, iy)-(ix, iy+1), iy-major

    offsets = np.array([-m, -1, 0, 1, m], dtype=np.int64)
    A = np.zeros((5, n), dtype=np.complex128)
    Bd = np.zeros((5, n), dtype=np.complex128)
    inv_h2 = 1.0 / (h * h)
    # diagonal
    A[2] = 4.0 * inv_h2 + 1j * gamma
    Bd[2] = 1.0 + 0.05 * s_diag
    # east (+1) / west (-1): same grid row only
    has_e = ix < m - 1
    has_w = ix > 0
    A[3, has_e] = -inv_h2 + 3.0 / (2.0 * h)
    A[1, has_w] = -inv_h2 - 3.0 / (2.0 * h)
    # north (+m) / south (-m)
    has_n = iy < m - 1
    has_s = iy > 0
    A[4, has_n] = -inv_h2 + 2.0 / (2.0 * h)
    A[0, has_s] = -inv_h2 - 2.0 / (2.0 * h)
    # symmetric S on the same pattern
    eh = np.zeros(n)                       # value of edge (i, i+1) stored at i
    eh_idx = np.flatnonzero(has_e)         # rows with an east neighbour, iy-major order
    eh[eh_idx] = s_h
    ev = np.zeros(n)                       # value of edge (i, i+m) stored at i
    ev_idx = np.flatnonzero(has_n)
    ev[ev_idx] = s_v
    Bd[3] = 0.05 * eh                      # B[i, i+1]
    Bd[1, 1:] = 0.05 * eh[:-1]             # B[i, i-1] = B[i-1, i]
    Bd[1, ~has_w] = 0.0
    Bd[4] = 0.05 * ev                      # B[i, i+m]
    Bd[0, m:] = 0.05 * ev[:-m]             # B[i, i-m] = B[i-m, i]
    return Pencil(m=m, n=n, offsets=offsets, A_dia=A, B_dia=Bd, gamma=gamma)


def random_block(n: int, k: int, seed: int, stream: int = 0) -> np.ndarray:
    """Complex Gaussian n x k block (column-major semantics; returned as a numpy array).

    `stream` selects an independent PCG64 stream (jumped) so several blocks can be
    drawn from one seed without touching the pencil's draws.
    """
    bitgen = np.random.PCG64(seed)
    if stream:
        bitgen = bitgen.jumped(stream)
    g = np.random.Generator(bitgen)
    re = g.standard_normal((k, n))
    im = g.standard_normal((k, n))
    return np.ascontiguousarray((re + 1j * im).T)


def orthonormal_random_block(n: int, k: int, seed: int, stream: int = 1) -> np.ndarray:
    """Random orthonormal n x k block: the starting block the drivers draw
    (Alg. 1 and Alg. 2, "generate an orthonormal random matrix Y").
    The draw is the Q factor of a complex Gaussian block (numpy QR)."""
    z = random_block(n, k, seed, stream)
    q, r = np.linalg.qr(z)
    # fix the phase so the draw is unique: diag(R) real positive
    d = np.diag(r)
    ph = d / np.abs(d)
    return np.asfortranarray(q * ph[None, :].conj())


def workload_names() -> list[str]:
    with open(WORKLOADS_JSON) as f:
        return sorted(json.load(f).keys())


def load_workload(name: str) -> dict:
    """Workload definition (grid, seed, disk, orders, block width), as written by
    tests/golden/make_golden.py from the oracle's eigenvalue computations."""
    with open(WORKLOADS_JSON) as f:
        w = json.load(f)[name]
    w = dict(w)
    w["center"] = complex(w["center_re"], w["center_im"])
    return w


def closed_form_spectrum(m: int) -> np.ndarray:
    """Eigenvalues of the constant-coefficient part of A (-Laplace + (3, 2) . grad, central
    differences, h = 1/(m+1)): (2/h^2)[2 - sqrt(1-(3h/2)^2) cos(j pi h) - sqrt(1-h^2) cos(k pi h)],
    j, k = 1..m (each 1D factor is a tridiagonal Toeplitz matrix). Real, ascending. Used only
    to place disks of the batch workload."""
    h = 1.0 / (m + 1)
    j = np.arange(1, m + 1)
    ax = np.sqrt(1.0 - (1.5 * h) ** 2) * np.cos(j * np.pi * h)
    ay = np.sqrt(1.0 - h ** 2) * np.cos(j * np.pi * h)
    lam = (2.0 / h ** 2) * (2.0 - ax[:, None] - ay[None, :])
    return np.sort(lam.ravel())


BATCH_GRIDS = (64, 96, 128, 160, 192)


def batch_problems(count: int = 12, seed: int = 0, grids=BATCH_GRIDS) -> list[dict]:
    """Recipe of a seeded mix of independent problems (pencils and disks) for the batched
    solver. Pencil j has grid grids[j mod len(grids)] and pencil seed 100 + j; it gets 1 or 2
    disks. Disk d of a pencil: N = n_in in {6, 10, 16} eigenvalues with block width
    k = 16, 24, 32, q in {4, 6, 8}, p in {4, 8}, driver 1. Its centre is placed near the
    closed-form eigenvalue at the fraction proxy_frac = 1/4 + d/16 of the sorted spectrum (away
    from the cluster at the middle of the 2D spectrum); tests/golden/make_golden.py fixes the
    exact centre and radius from the oracle's eigenvalues and stores them in workloads.json
    under `name`. Draws from PCG64(seed), independent of the pencils' own draws."""
    g = _rng(seed)
    out = []
    j = 0
    while len(out) < count:
        m = int(grids[j % len(grids)])
        ndisk = 1 + int(g.integers(0, 2))
        for d in range(ndisk):
            if len(out) == count:
                break
            N = int(g.choice([6, 10, 16]))
            out.append({"name": f"b{len(out)}_m{m}_d{d}", "m": m, "seed": 100 + j,
                        "k": {6: 16, 10: 24, 16: 32}[N], "q": int(g.choice([4, 6, 8])),
                        "p": int(g.choice([4, 8])), "n_in": N, "driver": 1,
                        "proxy_frac": 0.25 + d / 16.0})
        j += 1
    return out


def batch_workload_names(count: int = 12, seed: int = 0) -> list[str]:
    return [b["name"] for b in batch_problems(count, seed)]
