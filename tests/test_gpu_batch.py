"""GPU parity of the batched solver (ie_solve_batch): several independent problems run
concurrently give the same eigenpairs as ie_solve on each problem alone, and match the
reference eigenvalues of every problem (tests/golden)."""
import numpy as np
import pytest

import ie_inputs

from test_gpu_parity import Case, dblock, dzeros, golden_eigs, match_eigs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NAMES = ["c1_m24", "r1_m37", "m1_m64", "b0_m64_d0", "b2_m96_d0", "b10_m96_d0"]


@pytest.fixture(scope="module")
def ie():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_18043_gb300 import build as b
    b.build()
    import paper_2310_18043_gb300.ie as ie_
    return ie_


def _start(c):
    return ie_inputs.orthonormal_random_block(c.n, c.w["k"], seed=c.w["seed"])


def test_batch_equals_individual_solves_and_golden(ie):
    cases = [Case(ie, nm) for nm in NAMES]
    try:
        probs, outs = [], []
        for i, c in enumerate(cases):
            k = c.w["k"]
            # one item writes to a host buffer, the rest to device memory
            X = (np.zeros((c.n, k), dtype=np.complex128, order="F") if i == 1 else dzeros(c.n, k))
            outs.append(X)
            probs.append((c.h, dblock(_start(c)), X, k))
        st, res = ie.ie_solve_batch(probs, max_workers=4)
        assert st == ie.IE_OK, [ie.ie_status_str(r["status"]) for r in res]
        for c, r, X in zip(cases, res, outs):
            nf = r["n_found"]
            ref = golden_eigs(c.w)
            assert nf == len(ref), c.w
            match_eigs(r["lam"][:nf], ref)
            assert np.all(r["rho"][:nf] <= 1e-10)
            # the same problem alone through ie_solve
            k = c.w["k"]
            Xs = dzeros(c.n, k)
            st1, lam1, rho1, _, nf1, _ = ie.ie_solve(c.h, dblock(_start(c)), Xs, k)
            assert st1 == ie.IE_OK and nf1 == nf
            assert np.max(np.abs(lam1[:nf] - r["lam"][:nf]) / np.abs(lam1[:nf])) < 1e-12
            Xb = X.cpu().numpy() if isinstance(X, torch.Tensor) else X
            Xa = Xs.cpu().numpy()
            for j in range(nf):   # same vectors up to a unit scalar
                cosang = abs(np.vdot(Xa[:, j], Xb[:, j])) / (np.linalg.norm(Xa[:, j]) * np.linalg.norm(Xb[:, j]))
                assert cosang > 1 - 1e-10
    finally:
        for c in cases:
            c.close()


def test_batch_rejects_shared_handles_and_empty(ie):
    c = Case(ie, "c1_m24")
    try:
        k = c.w["k"]
        X1, X2 = dzeros(c.n, k), dzeros(c.n, k)
        st, _ = ie.ie_solve_batch([(c.h, None, X1, k), (c.h, None, X2, k)])
        assert st == ie.IE_ERR_ARG
        st, _ = ie.ie_solve_batch([])
        assert st == ie.IE_ERR_ARG
    finally:
        c.close()


def test_mixed_precision_batch_equals_individual_solves(ie):
    """The batch with mixed-precision handles (complex64 factors, FP64 refinement): each item
    equals its one-at-a-time ie_solve and matches the reference eigenvalues at rho <= 1e-10."""
    names = ["m1_m64", "b0_m64_d0", "b2_m96_d0"]
    cases = [Case(ie, nm, precision=1) for nm in names]
    try:
        probs = [(c.h, dblock(_start(c)), dzeros(c.n, c.w["k"]), c.w["k"]) for c in cases]
        st, res = ie.ie_solve_batch(probs, max_workers=3)
        assert st == ie.IE_OK, [ie.ie_status_str(r["status"]) for r in res]
        for c, r in zip(cases, res):
            nf = r["n_found"]
            ref = golden_eigs(c.w)
            assert nf == len(ref)
            match_eigs(r["lam"][:nf], ref)
            assert np.all(r["rho"][:nf] <= 1e-10)
            k = c.w["k"]
            st1, lam1, _, _, nf1, _ = ie.ie_solve(c.h, dblock(_start(c)), dzeros(c.n, k), k)
            assert st1 == ie.IE_OK and nf1 == nf
            assert np.max(np.abs(lam1[:nf] - r["lam"][:nf]) / np.abs(lam1[:nf])) < 1e-12
    finally:
        for c in cases:
            c.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_fused_batch_equals_individual_solves_and_golden(ie, precision):
    """ie_solve_batch_fused: one band-solve launch per Arnoldi step serves every problem of the
    batch (uneven n, band, poles, block widths, odd p, both drivers). Each item matches its
    reference eigenvalues at rho <= 1e-10 and its one-at-a-time ie_solve (complex128: the same
    kernels in the same order per problem, so the same eigenvalues to rounding)."""
    names = NAMES if precision == 0 else ["m1_m64", "b0_m64_d0", "b2_m96_d0", "r1_m37"]
    cases = [Case(ie, nm, precision=precision, driver=(2 if i % 2 else 1))
             for i, nm in enumerate(names)]
    try:
        probs, outs = [], []
        for i, c in enumerate(cases):
            k = c.w["k"]
            X = (np.zeros((c.n, k), dtype=np.complex128, order="F") if i == 1 else dzeros(c.n, k))
            outs.append(X)
            probs.append((c.h, dblock(_start(c)), X, k))
        st, res = ie.ie_solve_batch_fused(probs)
        assert st == ie.IE_OK, [ie.ie_status_str(r["status"]) for r in res]
        for c, r in zip(cases, res):
            nf = r["n_found"]
            ref = golden_eigs(c.w)
            assert nf == len(ref), (c.w, nf)
            match_eigs(r["lam"][:nf], ref)
            assert np.all(r["rho"][:nf] <= 1e-10)
            k = c.w["k"]
            st1, lam1, _, _, nf1, _ = ie.ie_solve(c.h, dblock(_start(c)), dzeros(c.n, k), k)
            assert st1 == ie.IE_OK and nf1 == nf
            assert np.max(np.abs(lam1[:nf] - r["lam"][:nf]) / np.abs(lam1[:nf])) < 1e-11
    finally:
        for c in cases:
            c.close()


def test_fused_batch_rejects_shared_handles_and_empty(ie):
    c = Case(ie, "c1_m24")
    try:
        k = c.w["k"]
        st, _ = ie.ie_solve_batch_fused([(c.h, None, dzeros(c.n, k), k), (c.h, None, dzeros(c.n, k), k)])
        assert st == ie.IE_ERR_ARG
        st, _ = ie.ie_solve_batch_fused([])
        assert st == ie.IE_ERR_ARG
    finally:
        c.close()
