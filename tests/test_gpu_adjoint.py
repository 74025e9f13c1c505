"""GPU parity of the adjoint path: the conjugate-transpose band solves (ie_apply_GH), left
eigenvectors (ie_solve_left) and eigenvalue sensitivities (ie_eig_sensitivity), through the
C ABI, against the FP64 oracle (oracle/adjoint.py) and dense LAPACK left eigenvectors.

Tolerances: G_adj(V) 1e-11 relative, as G(V) (direct solves with the same factors);
left eigenvalues equal to the right ones within the first-order bound of their residuals;
left vectors parallel to LAPACK's to 1e-9; sensitivities (scale-invariant) 1e-8 relative
per eigenvalue against the oracle's formula on LAPACK vectors."""
import numpy as np
import pytest
import scipy.linalg as sla

import ie_inputs
from oracle import adjoint as oadj, pencil as opencil

from test_gpu_parity import colerr, Case, dblock, dzeros

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ie():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_18043_gb300 import build as b
    b.build()
    import paper_2310_18043_gb300.ie as ie_
    return ie_


@pytest.mark.parametrize("name,k", [("c1_m24", 16), ("r1_m37", 11), ("m1_m64", 24)])
def test_apply_GH_matches_oracle(ie, name, k):
    """All q poles and k columns in one conjugate-transpose launch (several column groups,
    ragged n at r1) against sum_i conj(w_i) K_i^{-H} B^H V from SuperLU factors of K_i^H."""
    c = Case(ie, name, adjoint=1)
    try:
        V = ie_inputs.random_block(c.n, k, seed=7)
        GVd = dzeros(c.n, k)
        assert ie.ie_apply_GH(c.h, dblock(V), GVd) == ie.IE_OK
        ref = oadj.adjoint_inner(c.A, c.B, c.w["center"], c.w["radius"], c.w["q"]).apply(V)
        err = np.linalg.norm(GVd.cpu().numpy() - ref, axis=0) / np.linalg.norm(ref, axis=0)
        assert err.max() < 1e-11, err.max()
        assert colerr(GVd.cpu().numpy(), ref).max() < 1e-11
        _, st = ie.ie_get_stats(c.h)
        assert st["adj_launches"] == 1
    finally:
        c.close()


def test_apply_GH_ragged_ld_and_host_buffers(ie):
    c = Case(ie, "r1_m37", adjoint=1)
    try:
        k = 5
        V = ie_inputs.random_block(c.n, k, seed=8)
        Vpad = np.zeros((c.n + 3, k), dtype=np.complex128, order="F")
        Vpad[: c.n] = V
        Vd = torch.zeros((k, c.n + 3), dtype=torch.complex128, device="cuda:0")
        Vd[:, : c.n] = torch.from_numpy(np.ascontiguousarray(V.T)).to("cuda:0")
        Gd = torch.zeros((k, c.n + 5), dtype=torch.complex128, device="cuda:0")
        assert ie.ie_apply_GH(c.h, Vd.T[: c.n], Gd.T[: c.n]) == ie.IE_OK   # ld = n + 3, n + 5
        Gh = np.zeros((c.n, k), dtype=np.complex128, order="F")
        assert ie.ie_apply_GH(c.h, Vpad[: c.n], Gh) == ie.IE_OK              # host, ld = n + 3
        ref = oadj.adjoint_inner(c.A, c.B, c.w["center"], c.w["radius"], c.w["q"]).apply(V)
        for got in (Gd.T.cpu().numpy()[: c.n], Gh):
            assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-11
    finally:
        c.close()


def test_apply_GH_mixed_precision(ie):
    """complex64 factors, FP32 conjugate-transpose solves, FP64 refinement against K_i^H."""
    c = Case(ie, "m1_m64", adjoint=1, precision=1)
    try:
        k = 24
        V = ie_inputs.random_block(c.n, k, seed=9)
        GVd = dzeros(c.n, k)
        assert ie.ie_apply_GH(c.h, dblock(V), GVd) == ie.IE_OK
        ref = oadj.adjoint_inner(c.A, c.B, c.w["center"], c.w["radius"], c.w["q"]).apply(V)
        err = np.linalg.norm(GVd.cpu().numpy() - ref, axis=0) / np.linalg.norm(ref, axis=0)
        assert err.max() < 1e-11, err.max()
        assert colerr(GVd.cpu().numpy(), ref).max() < 1e-11
        _, st = ie.ie_get_stats(c.h)
        assert st["refine_solves"] >= 1
        assert st["adj_launches"] == 1 + st["refine_solves"] and st["solve_launches"] == 0
    finally:
        c.close()


def test_apply_GH_needs_adjoint_handle(ie):
    c = Case(ie, "c1_m24")
    try:
        V = dblock(ie_inputs.random_block(c.n, 2, seed=1))
        assert ie.ie_apply_GH(c.h, V, dzeros(c.n, 2)) == ie.IE_ERR_ARG
        Y = dzeros(c.n, 2)
        st, _, _, _ = ie.ie_solve_left(c.h, np.array([1.0 + 0j, 2.0]), Y)
        assert st == ie.IE_ERR_ARG
    finally:
        c.close()


def _right_then_left(ie, c):
    k = c.w["k"]
    Y0 = ie_inputs.orthonormal_random_block(c.n, k, seed=c.w["seed"])
    Xd = dzeros(c.n, k)
    st, lam, rho, e, nf, _ = ie.ie_solve(c.h, dblock(Y0), Xd, k)
    assert st == ie.IE_OK, ie.ie_status_str(st)
    Yd = dzeros(c.n, k)
    st, ll, rl, stats = ie.ie_solve_left(c.h, lam[:nf], Yd)
    assert st == ie.IE_OK, ie.ie_status_str(st)
    return lam[:nf], rho[:nf], Xd[:, :nf], ll, rl, Yd[:, :nf], stats


@pytest.mark.parametrize("name,driver", [("c1_m24", 1), ("r1_m37", 2)])
def test_left_eigenvectors_match_lapack(ie, name, driver):
    c = Case(ie, name, adjoint=1, driver=driver)
    try:
        lam, rho, Xd, ll, rl, Yd, stats = _right_then_left(ie, c)
        assert stats["adj_launches"] > 0
        nA, nB = opencil.norm1(c.A), opencil.norm1(c.B)
        # the paired left eigenvalue is the same eigenvalue, within both residual bounds
        scale = (nA + np.abs(lam) * nB) / np.abs(lam)
        assert np.all(rl <= 1e-10), rl.max()
        assert np.all(np.abs(ll - lam) / np.abs(lam) <= 4 * (rho + rl) * scale + 1e-13)
        Ad, Bd = c.A.toarray(), c.B.toarray()
        lam_d, VL, VR = sla.eig(Ad, Bd, left=True, right=True)
        Y = Yd.cpu().numpy()
        X = Xd.cpu().numpy()
        for i in range(len(lam)):
            j = int(np.argmin(np.abs(lam_d - lam[i])))
            vl = VL[:, j]
            cosang = abs(np.vdot(vl, Y[:, i])) / (np.linalg.norm(vl) * np.linalg.norm(Y[:, i]))
            assert cosang > 1 - 1e-9, (i, cosang)
            r = Y[:, i].conj() @ Ad - lam[i] * (Y[:, i].conj() @ Bd)
            assert np.linalg.norm(r) <= 1e-9 * (nA + abs(lam[i]) * nB)
        # sensitivities against the oracle's formula on LAPACK's left/right vectors
        sel = [int(np.argmin(np.abs(lam_d - l))) for l in lam]
        Sref = oadj.diag_sensitivity(c.B, VR[:, sel], VL[:, sel], alpha=1j)
        Sd = dzeros(c.n, len(lam))
        g = np.random.default_rng(3)
        gbar = g.uniform(0, 1, len(lam)) + 1j * g.uniform(-1, 1, len(lam))
        grad = torch.zeros(c.n, dtype=torch.float64, device="cuda:0")
        assert ie.ie_eig_sensitivity(c.h, Xd, Yd, 1j, Sd, gbar, grad) == ie.IE_OK
        S = Sd.cpu().numpy()
        err = np.linalg.norm(S - Sref, axis=0) / np.linalg.norm(Sref, axis=0)
        assert err.max() < 1e-8, err.max()
        gref = oadj.vjp(Sref, gbar)
        assert np.linalg.norm(grad.cpu().numpy() - gref) <= 1e-8 * np.linalg.norm(gref)
    finally:
        c.close()


def test_sensitivity_kernel_matches_oracle_formula_host_buffers(ie):
    """The sensitivity kernel alone, on arbitrary (non-eigen) host blocks: S and the VJP
    against the oracle's formula on the same X, Y; grad into a host array, S omitted."""
    c = Case(ie, "m1_m64")
    try:
        nf = 6
        X = np.asfortranarray(ie_inputs.random_block(c.n, nf, seed=11))
        Y = np.asfortranarray(ie_inputs.random_block(c.n, nf, seed=12))
        Sh = np.zeros((c.n, nf), dtype=np.complex128, order="F")
        assert ie.ie_eig_sensitivity(c.h, X, Y, 0.5 - 2j, Sh) == ie.IE_OK
        Sref = oadj.diag_sensitivity(c.B, X, Y, alpha=0.5 - 2j)
        assert np.linalg.norm(Sh - Sref) <= 1e-13 * np.linalg.norm(Sref)
        gbar = np.linspace(0.2, 1.0, nf) - 0.3j
        gh = np.zeros(c.n)
        assert ie.ie_eig_sensitivity(c.h, X, Y, 0.5 - 2j, None, gbar, gh) == ie.IE_OK
        gref = oadj.vjp(Sref, gbar)
        assert np.linalg.norm(gh - gref) <= 1e-13 * np.linalg.norm(gref)
        # grad without gbar is refused
        assert ie.ie_eig_sensitivity(c.h, X, Y, 1j, None, None, gh) == ie.IE_ERR_ARG
    finally:
        c.close()


def test_autograd_function_gradient_matches_oracle(ie):
    """DiskEigenvalues (torch.autograd.Function over the C ABI): the eigenvalues in D of the
    C1 pencil as a function of gamma, and d/dgamma of L = sum_i w_i Re(lambda_i) + Im(lambda_0)
    by loss.backward(), against the oracle's VJP on LAPACK's left and right eigenvectors."""
    from paper_2310_18043_gb300.autograd import DiskEigenvalues
    w = ie_inputs.load_workload("c1_m24")
    pen = ie_inputs.make_pencil(w["m"], w["seed"])
    main = int(np.flatnonzero(pen.offsets == 0)[0])
    A0 = pen.A_dia.copy()
    A0[main] -= 1j * pen.gamma
    dev = "cuda:0"
    gamma = torch.tensor(pen.gamma, dtype=torch.float64, device=dev, requires_grad=True)
    opts = ie.ie_opts_default(k=w["k"], driver=1)
    lam = DiskEigenvalues.apply(gamma, torch.from_numpy(A0).to(dev),
                                torch.from_numpy(pen.B_dia).to(dev), pen.offsets, w["center"],
                                w["radius"], w["p"], w["q"], opts)
    nf = lam.shape[0]
    assert nf == len(w["eig_in_disk_re"])
    wts = torch.from_numpy(np.random.default_rng(4).uniform(0, 1, nf)).to(dev)
    loss = (wts * lam.real).sum() + lam[0].imag
    loss.backward()
    A, B = opencil.pencil_matrices(pen)
    lam_d, VL, VR = sla.eig(A.toarray(), B.toarray(), left=True, right=True)
    lam_h = lam.detach().cpu().numpy()
    sel = [int(np.argmin(np.abs(lam_d - l))) for l in lam_h]
    Sref = oadj.diag_sensitivity(B, VR[:, sel], VL[:, sel], alpha=1j)
    gbar = wts.cpu().numpy().astype(np.complex128)
    gbar[0] += 1j
    gref = oadj.vjp(Sref, gbar)
    got = gamma.grad.cpu().numpy()
    assert np.linalg.norm(got - gref) <= 1e-8 * np.linalg.norm(gref)
