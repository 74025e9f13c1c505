"""Mixed precision (opts.precision = 1): complex64 factors and FP32 band solves, each
K_i^{-1} b refined in FP64. Same tolerances as the complex128 path: G(V) to 1e-11, the
filtered block to 1e-9, eigenvalues in D to 1e-10 with rho <= 1e-10."""
import numpy as np
import pytest

import ie_inputs
from oracle import coeffs, inner, msgmres

from test_gpu_parity import Case, colerr, dblock, dzeros, golden_eigs, match_eigs

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


def mixed(ie, name, **over):
    over.setdefault("precision", 1)
    return Case(ie, name, **over)


@pytest.mark.parametrize("name,k", [("c1_m24", 16), ("r1_m37", 11), ("m1_m64", 24)])
def test_mixed_apply_G_matches_oracle(ie, name, k):
    c = mixed(ie, name)
    try:
        V = ie_inputs.random_block(c.n, k, seed=5)
        GVd = dzeros(c.n, k)
        assert ie.ie_apply_G(c.h, dblock(V), GVd) == ie.IE_OK
        G = inner.InnerOperator(c.A, c.B, c.w["center"], c.w["radius"], c.w["q"])
        ref = G.apply(V)
        err = np.linalg.norm(GVd.cpu().numpy() - ref, axis=0) / np.linalg.norm(ref, axis=0)
        assert err.max() < 1e-11, err.max()
        assert colerr(GVd.cpu().numpy(), ref).max() < 1e-11
        _, st = ie.ie_get_stats(c.h)
        # one plain solve, then measured refinement steps down to the FP64 floor
        assert st["refine_solves"] >= 1
        assert st["solve32_launches"] == 1 + st["refine_solves"] and st["solve_launches"] == 0
    finally:
        c.close()


def test_mixed_filter_matches_oracle(ie):
    c = mixed(ie, "r1_m37")
    try:
        k = c.w["k"]
        Y = ie_inputs.orthonormal_random_block(c.n, k, seed=2)
        Ud = dzeros(c.n, k)
        assert ie.ie_filter_apply(c.h, dblock(Y), Ud) == ie.IE_OK
        G = inner.InnerOperator(c.A, c.B, c.w["center"], c.w["radius"], c.w["q"])
        ref = msgmres.filter_apply(G, Y, c.w["p"], tol=1e-12, m_max=100)
        err = np.linalg.norm(Ud.cpu().numpy() - ref) / np.linalg.norm(ref)
        assert err < 1e-9, err
        assert colerr(Ud.cpu().numpy(), ref).max() < 1e-9
    finally:
        c.close()


@pytest.mark.parametrize("name,driver", [("c1_m24", 1), ("r1_m37", 2), ("m1_m64", 1),
                                         ("c2_m256", 2)])
def test_mixed_solve_matches_golden(ie, name, driver):
    c = mixed(ie, name, driver=driver, m_max=150)
    try:
        k = c.w["k"]
        Y0 = ie_inputs.orthonormal_random_block(c.n, k, seed=c.w["seed"])
        Xd = dzeros(c.n, k)
        st, lam, rho, e, nf, stats = ie.ie_solve(c.h, dblock(Y0), Xd, k)
        assert st == ie.IE_OK, ie.ie_status_str(st)
        ref = golden_eigs(c.w)
        assert nf == len(ref)
        match_eigs(lam[:nf], ref)
        assert np.all(rho[:nf] <= 1e-10)
    finally:
        c.close()


def test_mixed_handle_has_no_complex128_factors(ie):
    """A precision = 1 handle has complex64 factors only: the complex128 static G path
    refuses it instead of touching factors it does not have."""
    c = mixed(ie, "c1_m24")
    try:
        V = dblock(ie_inputs.random_block(c.n, 2, seed=1))
        assert ie.ie_apply_G_static(c.h, V, dzeros(c.n, 2)) == ie.IE_ERR_ARG
    finally:
        c.close()


@pytest.mark.parametrize("name", ["c1_m24", "r1_m37"])
def test_mixed_lu_is_cgbtrf(ie, name):
    """The mixed handle factors K_i = p_i B - A, assembled in complex64, by the band LU in FP32
    arithmetic (LAPACK cgbtf2 semantics: pivot = first max of |re| + |im|). Against LAPACK's
    cgbtrf on the same complex64 band: the same pivot rows (the two round the rank-1 updates
    in different orders, so a near-tie could flip one; none does on these pencils), factors
    equal to FP32 rounding, and the factors solve K x = b to an FP32-level backward error."""
    from scipy.linalg import lapack
    c = mixed(ie, name)
    try:
        n, m = c.n, c.pen.half_bw
        ldab = 3 * m + 1
        poles, _ = coeffs.trapezoid_poles_weights(c.w["center"], c.w["radius"], c.w["q"])
        for i, pole in enumerate(poles):
            st, ab, ipiv, kl = ie.ie_get_factor(c.h, i, n, ldab)
            assert st == ie.IE_OK and kl == m
            K = (pole * c.B - c.A).toarray()
            K32 = K.astype(np.complex64)
            band = np.zeros((ldab, n), dtype=np.complex64, order="F")
            for j in range(n):
                for r in range(max(0, j - m), min(n, j + m + 1)):
                    band[2 * m + r - j, j] = K32[r, j]
            lu, piv_ref, info = lapack.cgbtrf(band, m, m)
            assert info == 0
            assert np.array_equal(ipiv, piv_ref + 1), "pivot rows differ from cgbtrf"
            scale = np.abs(lu).max()
            assert np.max(np.abs(ab - lu)) <= 1e-4 * scale
            b = ie_inputs.random_block(n, 2, seed=i)
            x, info = lapack.zgbtrs(ab, m, m, b, ipiv - 1)
            assert info == 0
            res = np.linalg.norm(K @ x - b) / (np.linalg.norm(K, 1) * np.linalg.norm(x))
            assert res < 1e-5, res
    finally:
        c.close()


def test_mixed_every_solve_shape_matches_oracle(ie):
    """Repeated mixed-precision G applications walk through every candidate launch shape of
    the complex64 band solve (synchronised, warp-specialised and look-ahead kernels); each
    result matches the oracle element by element, and since every shape performs the same
    operations in the same order, every call returns the same bits."""
    c = mixed(ie, "r1_m37")
    try:
        k = c.w["k"]
        V = ie_inputs.random_block(c.n, k, seed=13)
        Vd = dblock(V)
        ref = inner.InnerOperator(c.A, c.B, c.w["center"], c.w["radius"], c.w["q"]).apply(V)
        first = None
        for call in range(20):                    # each call launches several solves
            GVd = dzeros(c.n, k)
            assert ie.ie_apply_G(c.h, Vd, GVd) == ie.IE_OK
            got = GVd.cpu().numpy()
            err = colerr(got, ref).max()
            assert err < 1e-11, (call, err)
            if first is None:
                first = got
            assert np.array_equal(got, first), f"call {call} differs"
    finally:
        c.close()


def test_mixed_singular_pencil_reports_zero_pivot(ie):
    """The complex64 blocked LU on a pencil with an exactly zero column (band 1, n not a
    multiple of the 16-column panel): IE_ERR_SINGULAR on the host, no GPU fault, and the
    context stays usable."""
    n = 70
    offsets = np.array([-1, 0, 1], dtype=np.int64)
    A = np.zeros((3, n), dtype=np.complex128)
    B = np.zeros((3, n), dtype=np.complex128)
    A[1] = np.arange(1, n + 1)
    B[1] = 1.0
    A[1, 37] = 0.0
    B[1, 37] = 0.0
    st, h = ie.ie_create(n, offsets, torch.from_numpy(A).to("cuda:0"), torch.from_numpy(B).to("cuda:0"),
                         10.0, 2.5, 4, 4, ie.ie_opts_default(k=4, precision=1))
    assert st == ie.IE_ERR_SINGULAR
    ie.ie_destroy(h)
    c = mixed(ie, "c1_m24")
    c.close()
