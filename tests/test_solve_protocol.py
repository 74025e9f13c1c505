"""CPU emulations of the band-solve kernels' orders: the look-ahead protocol
(`band_solve_la_kernel`) and the synchronised one (`band_solve_kernel`,
`band_solve_pipe_kernel`).

The kernel splits each sweep of the blocked band solve (Sec. 3.2, the inner operator's
K_i^{-1}: P, L forward, U backward, in LAPACK gbtrs order) into head warps and update warps
that run one panel apart. This test replays that split in Python, with the most aggressive
order the kernel's waits allow -- head(P+1) runs before update(P) -- and checks:

* every head input IN(P) is delivered exactly once per row (an arrival count per panel that
  must reach 2*NB, as the mbarrier's count does), and no head reads a value not yet delivered
  (inputs start as NaN);
* the slot of each row the update warps deliver (row, or the slot's next row) is the one the
  kernel computes;
* the result equals a dense solve of the matrix that LAPACK factored (zgbtrf), for bands from
  0 to 40, ragged n and n smaller than two panels.

The per-panel transforms T (16x16 over the set H of head rows and pivot members) and
inv(U_block) are formed here from their definitions, independently of the CUDA code.
"""
import numpy as np
import pytest
from scipy.linalg import lapack

NB = 8


def _band_factor(n, kl, seed):
    g = np.random.default_rng(seed)
    K = np.zeros((n, n), complex)
    for i in range(n):
        for j in range(max(0, i - kl), min(n, i + kl + 1)):
            K[i, j] = g.standard_normal() + 1j * g.standard_normal()
    band = np.zeros((3 * kl + 1, n), complex, order="F")
    for j in range(n):
        for r in range(max(0, j - kl), min(n, j + kl + 1)):
            band[2 * kl + r - j, j] = K[r, j]
    lu, piv, info = lapack.zgbtrf(band, kl, kl)
    assert info == 0
    return K, lu, piv


def _panels(n, kl, lu, piv):
    """Per panel: H (16 rows, -1 absent), T (H <- T H), inv(U_block) (zero for rows >= n)."""
    kv = 2 * kl
    npan = (n + NB - 1) // NB

    def L(r, j):
        return lu[kv + r - j, j] if (j < n and r < n and 1 <= r - j <= kl) else 0

    def U(r, j):
        return lu[kv + r - j, j] if (j < n and 0 <= r and 0 <= j - r <= kv) else 0

    out = []
    for P in range(npan):
        j0, nvalid = P * NB, min(n - P * NB, NB)
        pst = [piv[j0 + jj] if jj < nvalid else -1 for jj in range(NB)]

        def hidx(r):
            if j0 <= r < j0 + NB:
                return r - j0
            for jj in range(nvalid):
                if pst[jj] == r:
                    return NB + jj
            return -1

        H = [j0 + l if l < NB else -1 for l in range(16)]
        for jj in range(nvalid):
            if pst[jj] >= j0 + NB and hidx(pst[jj]) == NB + jj:
                H[NB + jj] = pst[jj]
        T = np.zeros((16, 16), complex)
        for m in range(16):
            if H[m] < 0:
                continue
            val = np.zeros(16, complex)
            val[m] = 1
            for jj in range(nvalid):
                j, b = j0 + jj, hidx(pst[jj])
                val[jj], val[b] = val[b], val[jj]
                x = val[jj]
                for l in range(16):
                    if H[l] > j and H[l] <= j + kl:
                        val[l] -= L(H[l], j) * x
            T[:, m] = [val[l] if H[l] >= 0 else 0 for l in range(16)]
        Ub = np.array([[U(j0 + i, j0 + c) if (j0 + c < n and j0 + i < n) else float(i == c)
                        for c in range(NB)] for i in range(NB)])
        Ui = np.linalg.inv(Ub)
        for i in range(NB):
            if j0 + i >= n:
                Ui[i, :] = 0
                Ui[:, i] = 0
        out.append((H, T, Ui))
    return out, L, U


def _look_ahead_solve(n, kl, lu, piv, b):
    kv = 2 * kl
    npan = (n + NB - 1) // NB
    n_pad = npan * NB
    pans, L, U = _panels(n, kl, lu, piv)
    R = lambda r: b[r] if 0 <= r < n else 0

    # ---------------- forward: window of Sf slots, slot of row r is (r - NB) mod Sf
    Sf = max(kl, 2 * NB)
    frow = [NB + s for s in range(Sf)]
    v = [R(r) for r in frow]
    nxt = [R(r + Sf) for r in frow]
    IN = {P: np.full(16, np.nan, complex) for P in range(npan)}
    arrivals = {P: 0 for P in range(npan)}
    OUT = {}
    y = np.zeros(n, complex)

    def head(P):
        H, T, _ = pans[P]
        j0, nvalid = P * NB, min(n - P * NB, NB)
        if P < 2:                                   # untouched rows: read directly
            IN[P][:] = [R(r) if r >= 0 else 0 for r in H]
            arrivals[P] += 2 * NB
        else:                                       # head warp 0 completes the absent members
            arrivals[P] += NB - sum(1 for r in H[NB:] if r >= 0)
        assert arrivals[P] == 2 * NB, (P, arrivals[P])
        val = np.zeros(16, complex)
        for i, r in enumerate(H):
            if r < 0:
                continue
            x = IN[P][i]
            assert not np.isnan(x), ("read before delivery", P, i)
            if P >= 1:                              # catch-up: apply panel P-1
                Hq, oq = pans[P - 1][0], OUT[P - 1]
                if r in Hq[NB:]:
                    x = oq[Hq.index(r)]
                else:
                    jq = j0 - NB
                    for jj in range(min(n - jq, NB)):
                        if r - (jq + jj) <= kl:
                            x -= L(r, jq + jj) * oq[jj]
            val[i] = x
        out = np.array([T[i] @ val if H[i] >= 0 else 0 for i in range(16)])
        y[j0:j0 + nvalid] = out[:nvalid]
        OUT[P] = out

    def update(P):
        H = pans[P][0]
        j0, nvalid = P * NB, min(n - P * NB, NB)
        H2 = pans[P + 2][0] if P + 2 < npan else None
        for s in range(Sf):
            r = frow[s]
            assert r - j0 >= NB and (r - NB) % Sf == s
            for jj in range(nvalid):
                if r - (j0 + jj) <= kl:
                    v[s] -= L(r, j0 + jj) * OUT[P][jj]
            if r in H[NB:]:
                v[s] = OUT[P][H.index(r)]
            if H2 is not None:                      # rows of panel P+2, after panel P
                for m in range(16):
                    if H2[m] == r:
                        IN[P + 2][m] = v[s]
                        arrivals[P + 2] += 1
                    elif m >= NB and H2[m] == r + Sf:
                        assert H2[m] > j0 + NB - 1 + Sf     # only beyond the window
                        IN[P + 2][m] = nxt[s]
                        arrivals[P + 2] += 1
            if r - j0 < 2 * NB:                     # a head row of P+1: take row r + Sf
                frow[s] = r + Sf
                v[s], nxt[s] = nxt[s], R(r + 2 * Sf)

    head(0)
    for P in range(npan):
        if P + 1 < npan:
            head(P + 1)
        update(P)

    # ---------------- backward: window of Sb slots below the head
    Sb = max(kv, 2 * NB)
    Y = lambda r: y[r] if 0 <= r < n else 0
    top = n_pad - 1
    row = [top - NB - s for s in range(Sb)]
    v = [Y(r) for r in row]
    nxt = [Y(r - Sb) for r in row]
    IN = {B: np.full(NB, np.nan, complex) for B in range(npan)}
    arrivals = {B: 0 for B in range(npan)}
    OUT = {}
    x = np.zeros(n, complex)

    def bhead(Bp):
        j0 = top - Bp * NB
        Ui = pans[(j0 - NB + 1) // NB][2]
        if Bp < 2:
            IN[Bp][:] = [Y(j0 - t) for t in range(NB)]
            arrivals[Bp] += 2 * NB
        else:
            arrivals[Bp] += NB
        assert arrivals[Bp] == 2 * NB, (Bp, arrivals[Bp])
        val = np.zeros(NB, complex)
        for t in range(NB):
            w = IN[Bp][t]
            assert not np.isnan(w), ("read before delivery", Bp, t)
            if Bp >= 1:
                jq, r = j0 + NB, j0 - t
                for s2 in range(NB):
                    if (jq - r) - s2 <= kv:
                        w -= U(r, jq - s2) * OUT[Bp - 1][s2]
            val[t] = w
        xs = np.array([Ui[NB - 1 - t, ::-1] @ val for t in range(NB)])
        for t in range(NB):
            if j0 - t < n:
                x[j0 - t] = xs[t]
        OUT[Bp] = xs

    def bupdate(Bp):
        j0 = top - Bp * NB
        for s in range(Sb):
            r = row[s]
            base = j0 - r
            assert base >= NB
            for s2 in range(NB):
                if base - s2 <= kv:
                    v[s] -= U(r, j0 - s2) * OUT[Bp][s2]
            if Bp + 2 < npan and 0 <= base - 2 * NB < NB:
                IN[Bp + 2][base - 2 * NB] = v[s]
                arrivals[Bp + 2] += 1
            if base < 2 * NB:
                row[s] = r - Sb
                v[s], nxt[s] = nxt[s], Y(r - 2 * Sb)

    bhead(0)
    for Bp in range(npan):
        if Bp + 1 < npan:
            bhead(Bp + 1)
        bupdate(Bp)
    return x


@pytest.mark.parametrize("n,kl,seed", [(37, 3, 0), (64, 1, 1), (83, 11, 3), (20, 12, 4),
                                        (9, 4, 7), (5, 1, 9), (16, 0, 12), (150, 33, 11),
                                        (120, 20, 6)])
def test_look_ahead_protocol_solves_the_factored_matrix(n, kl, seed):
    K, lu, piv = _band_factor(n, kl, seed)
    b = np.random.default_rng(9).standard_normal(n) + 1j
    x = _look_ahead_solve(n, kl, lu, piv, b)
    ref = np.linalg.solve(K, b)
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) < 1e-12


def test_emulation_detects_a_missing_delivery():
    """Planted mistake: the update side forgets the next-row deliveries (members of panel
    P+2 beyond the window). The arrival count must then fall short."""
    import inspect
    n, kl = 120, 20
    K, lu, piv = _band_factor(n, kl, 6)
    b = np.random.default_rng(9).standard_normal(n) + 1j
    code = inspect.getsource(_look_ahead_solve)
    assert "elif m >= NB and H2[m] == r + Sf:" in code
    g = dict(globals())
    exec(code.replace("elif m >= NB and H2[m] == r + Sf:", "elif False:"), g)
    with pytest.raises(AssertionError):
        g["_look_ahead_solve"](n, kl, lu, piv, b)


def _synchronised_solve(n, kl, lu, piv, b):
    """The barrier-synchronised kernels' order (`band_solve_kernel`, `band_solve_pipe_kernel`):
    per panel the head (T H forward, inv(U_block) h backward), then the window update, whose
    first NB rows become the next head; the window holds max(kl, NB) / max(kv, NB) rows."""
    kv = 2 * kl
    npan = (n + NB - 1) // NB
    n_pad = npan * NB
    pans, L, U = _panels(n, kl, lu, piv)
    R = lambda r: b[r] if 0 <= r < n else 0
    Sf = max(kl, NB)
    hd = [R(t) for t in range(NB)]
    frow = [NB + s for s in range(Sf)]
    v = [R(r) for r in frow]
    y = np.zeros(n, complex)
    for P in range(npan):
        H, T, _ = pans[P]
        j0, nvalid = P * NB, min(n - P * NB, NB)
        hv = np.zeros(16, complex)
        hv[:NB] = hd
        mem = [-1] * Sf
        for s in range(Sf):
            if frow[s] in H[NB:]:
                mem[s] = H.index(frow[s])
                hv[mem[s]] = v[s]
        out = np.array([T[i] @ hv if H[i] >= 0 else 0 for i in range(16)])
        y[j0:j0 + nvalid] = out[:nvalid]
        for s in range(Sf):
            r = frow[s]
            if mem[s] >= NB:
                v[s] = out[mem[s]]
            else:
                for jj in range(nvalid):
                    if r - (j0 + jj) <= kl:
                        v[s] -= L(r, j0 + jj) * out[jj]
            if r - j0 - NB < NB:
                hd[r - j0 - NB] = v[s]
                frow[s] = r + Sf
                v[s] = R(r + Sf)
    Sb = max(kv, NB)
    Y = lambda r: y[r] if 0 <= r < n else 0
    top = n_pad - 1
    hd = [Y(top - t) for t in range(NB)]
    row = [top - NB - s for s in range(Sb)]
    v = [Y(r) for r in row]
    x = np.zeros(n, complex)
    for Bp in range(npan):
        j0 = top - Bp * NB
        Ui = pans[(j0 - NB + 1) // NB][2]
        xs = np.array([Ui[NB - 1 - t, ::-1] @ np.array(hd) for t in range(NB)])
        for t in range(NB):
            if j0 - t < n:
                x[j0 - t] = xs[t]
        for s in range(Sb):
            r = row[s]
            base = j0 - r
            for s2 in range(NB):
                if base - s2 <= kv:
                    v[s] -= U(r, j0 - s2) * xs[s2]
            if base - NB < NB:
                hd[base - NB] = v[s]
                row[s] = r - Sb
                v[s] = Y(r - Sb)
    return x


@pytest.mark.parametrize("n,kl,seed", [(37, 3, 0), (64, 1, 1), (50, 5, 2), (83, 11, 3),
                                        (20, 12, 4), (17, 2, 5), (16, 0, 12)])
def test_synchronised_order_solves_the_factored_matrix(n, kl, seed):
    K, lu, piv = _band_factor(n, kl, seed)
    b = np.random.default_rng(9).standard_normal(n) + 1j
    x = _synchronised_solve(n, kl, lu, piv, b)
    ref = np.linalg.solve(K, b)
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) < 1e-12
