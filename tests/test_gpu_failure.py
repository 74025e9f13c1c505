"""Failure detection on the GPU without a fault: a device-side wait that runs out.

The band LU's CTAs wait for each column's published pivot with a bounded wait (IE_WAIT_NS).
The test hook IE_TEST_SKIP_PUBLISH=j makes the owner of column j never set that flag, so
every wait for step j runs out; the kernel records the timeout and returns, ie_create
reports IE_ERR_TIMEOUT, and the context stays usable: the next ie_create succeeds and its
factorisation is still LAPACK's."""
import numpy as np
import pytest
import scipy.linalg.lapack as lapack

import ie_inputs

from test_gpu_parity import Case, dblock, dzeros

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


def test_lu_wait_runs_out_and_reports_timeout(ie, monkeypatch):
    w = ie_inputs.load_workload("c1_m24")
    pen = ie_inputs.make_pencil(w["m"], w["seed"])
    A = torch.from_numpy(pen.A_dia).to("cuda:0")
    B = torch.from_numpy(pen.B_dia).to("cuda:0")
    monkeypatch.setenv("IE_TEST_SKIP_PUBLISH", "5")
    opts = ie.ie_opts_default(k=w["k"])
    st, h = ie.ie_create(pen.n, pen.offsets, A, B, w["center"], w["radius"], w["p"], w["q"], opts)
    assert st == ie.IE_ERR_TIMEOUT, ie.ie_status_str(st)
    monkeypatch.delenv("IE_TEST_SKIP_PUBLISH")
    c = Case(ie, "c1_m24")          # asserts IE_OK
    try:
        from oracle import coeffs
        m = c.pen.half_bw
        ldab = 3 * m + 1
        st, ab, ipiv, kl = ie.ie_get_factor(c.h, 0, c.n, ldab)
        assert st == ie.IE_OK
        pole = coeffs.trapezoid_poles_weights(w["center"], w["radius"], w["q"])[0][0]
        K = (pole * c.B - c.A).toarray()
        band = np.zeros((ldab, c.n), dtype=np.complex128, order="F")
        for j in range(c.n):
            for r in range(max(0, j - m), min(c.n, j + m + 1)):
                band[2 * m + r - j, j] = K[r, j]
        lu, piv_ref, info = lapack.zgbtrf(band, m, m)
        assert info == 0 and np.array_equal(ipiv, piv_ref + 1)
        assert np.max(np.abs(ab - lu)) <= 1e-12 * np.abs(lu).max()
        V = ie_inputs.random_block(c.n, 2, seed=1)
        assert ie.ie_apply_G(c.h, dblock(V), dzeros(c.n, 2)) == ie.IE_OK
    finally:
        c.close()
