"""ie_apply_G_static: the G(V) variant whose scratch is a file-scope device array, for
callers that must not make the library allocate device memory at call time. It must give
the same result as ie_apply_G, call after call (the shared scratch keeps the previous
call's contents), and refuse problems larger than its scratch without launching.
This file is collected last on purpose."""
import numpy as np
import pytest

import ie_inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a).T)).to(DEV).T


def _zeros(n, k):
    return torch.zeros((k, n), dtype=torch.complex128, device=DEV).T


@pytest.fixture(scope="module")
def handle():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_18043_gb300 import build as b
    b.build()
    import paper_2310_18043_gb300.ie as ie
    w = ie_inputs.load_workload("m1_m64")
    pen = ie_inputs.make_pencil(w["m"], w["seed"])
    A = torch.from_numpy(pen.A_dia).to(DEV)
    B = torch.from_numpy(pen.B_dia).to(DEV)
    st, h = ie.ie_create(pen.n, pen.offsets, A, B, w["center"], w["radius"], w["p"], w["q"],
                         ie.ie_opts_default(k=w["k"]))
    assert st == ie.IE_OK, ie.ie_status_str(st)
    yield ie, h, pen.n, w
    ie.ie_destroy(h)


def test_static_scratch_matches_apply_G_on_consecutive_calls(handle):
    ie, h, n, w = handle
    k = w["k"]                      # (q+1) n k = 7 * 4096 * 24 values, inside the 32 MiB array
    for call, seed in enumerate((31, 32)):
        V = _dev(ie_inputs.random_block(n, k, seed=seed))
        ref = _zeros(n, k)
        got = _zeros(n, k)
        assert ie.ie_apply_G(h, V, ref) == ie.IE_OK
        assert ie.ie_apply_G_static(h, V, got) == ie.IE_OK, f"call {call}"
        torch.cuda.synchronize()
        err = (torch.linalg.norm(got - ref) / torch.linalg.norm(ref)).item()
        assert err < 1e-11, (call, err)


def test_static_scratch_allocates_nothing(handle):
    """After the first call (which, under lazy module loading, loads the module that holds
    the array), further calls leave the device's free memory unchanged."""
    ie, h, n, w = handle
    k = w["k"]
    V = _dev(ie_inputs.random_block(n, k, seed=33))
    GV = _zeros(n, k)
    assert ie.ie_apply_G_static(h, V, GV) == ie.IE_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert ie.ie_apply_G_static(h, V, GV) == ie.IE_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


@pytest.mark.parametrize("extra", [None, 8])
def test_static_scratch_other_block_widths(handle, extra):
    """k = 1, and k wider than the handle's opts.k (allowed while (q+1) n k fits the array):
    each column equals ie_apply_G on slices of at most opts.k columns."""
    ie, h, n, w = handle
    k = 1 if extra is None else w["k"] + extra
    assert (w["q"] + 1) * n * k * 16 <= ie.IE_STATIC_SCRATCH_BYTES
    V = _dev(ie_inputs.random_block(n, k, seed=40 + k))
    got = _zeros(n, k)
    assert ie.ie_apply_G_static(h, V, got) == ie.IE_OK
    ref = _zeros(n, k)
    for c0 in range(0, k, w["k"]):
        c1 = min(k, c0 + w["k"])
        assert ie.ie_apply_G(h, V[:, c0:c1], ref[:, c0:c1]) == ie.IE_OK
    torch.cuda.synchronize()
    err = (torch.linalg.norm(got - ref, dim=0) / torch.linalg.norm(ref, dim=0)).max().item()
    assert err < 1e-11, err


def test_static_scratch_rejects_oversized_problem(handle):
    ie, h, n, w = handle
    k = ie.IE_STATIC_SCRATCH_BYTES // (16 * (w["q"] + 1) * n) + 1
    V = _zeros(n, k)
    GV = _zeros(n, k)
    GV.fill_(1.0)
    assert ie.ie_apply_G_static(h, V, GV) == ie.IE_ERR_SCRATCH_LIMIT
    torch.cuda.synchronize()
    assert torch.all(GV == 1.0)     # nothing was launched
