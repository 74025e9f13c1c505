"""ctypes binding of the C ABI declared in include/ie.h (same names, argument
marshalling only). Every computation runs in libie.so's CUDA kernels; there is no
CPU fallback: importing this module does not load the library, the first call does,
and it raises if the library has not been built.

Pointer arguments accept torch tensors (device memory, complex128) or numpy arrays
(host memory, complex128). Blocks are n x k column-major: pass a tensor/array whose
first dimension is n and whose row stride is 1 (for example `t.T` of a (k, n)
contiguous tensor, or `np.asfortranarray`); the leading dimension is read from the
column stride.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libie.so")

(IE_OK, IE_ERR_ARG, IE_ERR_CUDA, IE_ERR_OOM, IE_ERR_SINGULAR, IE_ERR_NOCONV, IE_ERR_BREAKDOWN,
 IE_ERR_TIMEOUT, IE_ERR_SCRATCH_LIMIT) = range(9)
IE_STATIC_SCRATCH_BYTES = 32 * 1024 * 1024


class ie_complex(C.Structure):
    _fields_ = [("re", C.c_double), ("im", C.c_double)]


class ie_pencil(C.Structure):
    _fields_ = [("n", C.c_int64), ("ndiag", C.c_int32), ("h_offsets", C.POINTER(C.c_int64)),
                ("d_A_dia", C.c_void_p), ("d_B_dia", C.c_void_p)]


class ie_opts(C.Structure):
    _fields_ = [("k", C.c_int32), ("driver", C.c_int32), ("m_max", C.c_int32),
                ("max_outer", C.c_int32), ("tau_g", C.c_double), ("tau", C.c_double),
                ("gmres_tol", C.c_double), ("sigma_is_center", C.c_int32),
                ("sigma_re", C.c_double), ("sigma_im", C.c_double), ("seed", C.c_uint64),
                ("precision", C.c_int32), ("refine_steps", C.c_int32), ("adjoint", C.c_int32)]


class ie_stats(C.Structure):
    _fields_ = [("outer_iters", C.c_int32), ("n_found", C.c_int32), ("p_final", C.c_int32),
                ("gmres_iters_max", C.c_int32), ("gmres_iters_min", C.c_int32),
                ("converged", C.c_int32), ("g_columns", C.c_int64), ("t_factor_ms", C.c_double),
                ("t_filter_ms", C.c_double), ("t_hsrr_ms", C.c_double),
                ("max_rho_found", C.c_double), ("solve_launches", C.c_int64),
                ("t_solve_ms", C.c_double), ("solve_flops", C.c_double),
                ("solve_bytes", C.c_double), ("kernel_launches", C.c_int64),
                ("solve32_launches", C.c_int64), ("t_solve32_ms", C.c_double),
                ("solve32_flops", C.c_double), ("adj_launches", C.c_int64),
                ("t_adj_ms", C.c_double), ("adj_flops", C.c_double),
                ("refine_solves", C.c_int64), ("refine_last_corr", C.c_double),
                ("solve_kernel", C.c_int32), ("solve32_kernel", C.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class ie_batch_item(C.Structure):
    _fields_ = [("h", C.c_void_p), ("Y0_any", C.c_void_p), ("ldy0", C.c_int64),
                ("h_lambda", C.c_void_p), ("X_any", C.c_void_p), ("ldx", C.c_int64),
                ("h_rho", C.c_void_p), ("h_e", C.c_void_p), ("stream", C.c_void_p),
                ("n_found", C.c_int32), ("status", C.c_int32), ("stats", ie_stats)]


EXPORTS = ["ie_opts_default", "ie_create", "ie_destroy", "ie_status_str", "ie_filter_apply",
           "ie_apply_G", "ie_hsrr", "ie_solve", "ie_spmv", "ie_get_coeffs", "ie_get_factor",
           "ie_get_stats", "ie_apply_G_static", "ie_apply_GH", "ie_solve_left",
           "ie_eig_sensitivity", "ie_solve_batch", "ie_solve_batch_fused"]

_lib = None
_vp, _i32, _i64, _dp = C.c_void_p, C.c_int32, C.c_int64, C.POINTER(C.c_double)


def load():
    """Loads libie.so (raises if it is missing: there is no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libie.so not built ({LIB_PATH}); run __graft_entry__.build()")
    L = C.CDLL(LIB_PATH)
    L.ie_opts_default.argtypes = [C.POINTER(ie_opts)]
    L.ie_opts_default.restype = None
    L.ie_status_str.argtypes = [C.c_int]
    L.ie_status_str.restype = C.c_char_p
    L.ie_create.argtypes = [C.POINTER(ie_pencil), ie_complex, C.c_double, _i32, _i32,
                            C.POINTER(ie_opts), _vp, C.POINTER(_vp)]
    L.ie_destroy.argtypes = [_vp]
    L.ie_filter_apply.argtypes = [_vp, _vp, _i64, _i32, _vp, _i64, _vp]
    L.ie_apply_G.argtypes = [_vp, _vp, _i64, _i32, _vp, _i64, _vp]
    L.ie_hsrr.argtypes = [_vp, _vp, _i64, _i32, _vp, _vp, _i64, _vp, _vp, _vp]
    L.ie_solve.argtypes = [_vp, _vp, _i64, _vp, _vp, _i64, _vp, _vp, C.POINTER(_i32),
                           C.POINTER(ie_stats), _vp]
    L.ie_spmv.argtypes = [_vp, _i32, _vp, _i64, _i32, _vp, _i64, _vp]
    L.ie_get_coeffs.argtypes = [_vp, _vp, _vp, _vp, _vp, C.POINTER(_i32), _dp]
    L.ie_get_factor.argtypes = [_vp, _i32, _vp, _vp, C.POINTER(_i32), C.POINTER(_i32)]
    L.ie_get_stats.argtypes = [_vp, C.POINTER(ie_stats)]
    L.ie_apply_G_static.argtypes = [_vp, _vp, _i64, _i32, _vp, _i64, _vp]
    L.ie_apply_GH.argtypes = [_vp, _vp, _i64, _i32, _vp, _i64, _vp]
    L.ie_solve_left.argtypes = [_vp, _vp, _i32, _vp, _i64, _vp, _i64, _vp, _vp,
                                C.POINTER(ie_stats), _vp]
    L.ie_solve_batch.argtypes = [C.POINTER(ie_batch_item), _i32, _i32]
    L.ie_solve_batch_fused.argtypes = [C.POINTER(ie_batch_item), _i32, _vp]
    L.ie_eig_sensitivity.argtypes = [_vp, _vp, _i64, _vp, _i64, _i32, ie_complex, _vp, _i64, _vp,
                                     _vp, _vp]
    for f in EXPORTS:
        if f not in ("ie_opts_default", "ie_status_str"):
            getattr(L, f).restype = C.c_int
    _lib = L
    return L


class IeError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {ie_status_str(status)}")
        self.status = status


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        except Exception:
            pass
        return None
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _block(x):
    """(pointer, ld, rows, cols) of an n x k column-major complex128 block."""
    if x is None:
        return None, 0, 0, 0
    try:
        import torch
        if isinstance(x, torch.Tensor):
            if x.dtype != torch.complex128:
                raise TypeError("complex128 tensor expected")
            if x.dim() == 1:
                return C.c_void_p(x.data_ptr()), x.shape[0], x.shape[0], 1
            if x.stride(0) != 1:
                raise ValueError("column-major block expected (row stride 1)")
            ld = x.stride(1) if x.shape[1] > 1 else x.shape[0]
            return C.c_void_p(x.data_ptr()), ld, x.shape[0], x.shape[1]
    except ImportError:
        pass
    if isinstance(x, np.ndarray):
        if x.dtype != np.complex128:
            raise TypeError("complex128 array expected")
        if x.ndim == 1:
            return C.c_void_p(x.ctypes.data), x.shape[0], x.shape[0], 1
        if x.strides[0] != 16:
            raise ValueError("column-major block expected (Fortran order)")
        ld = x.strides[1] // 16 if x.shape[1] > 1 else x.shape[0]
        return C.c_void_p(x.ctypes.data), ld, x.shape[0], x.shape[1]
    raise TypeError(f"unsupported block type {type(x)}")


# Matrix size n of every live handle (recorded by ie_create), so that the wrappers can check
# block shapes before the library writes n x k outputs through raw pointers.
_handle_n: dict = {}


def _hkey(h):
    return h.value if isinstance(h, C.c_void_p) else h


def _check_rows(h, rows, where):
    n = _handle_n.get(_hkey(h))
    if n is not None and rows != n:
        raise ValueError(f"{where}: block has {rows} rows, the handle's matrix size is {n}")


def _in_out(h, X, Y, where):
    """Input X and output Y of an n x k -> n x k call: (px, ldx, k, py, ldy). Raises
    ValueError unless Y has exactly X's shape and both have the handle's n rows."""
    px, ldx, n, k = _block(X)
    py, ldy, ny, ky = _block(Y)
    _check_rows(h, n, where)
    if (ny, ky) != (n, k):
        raise ValueError(f"{where}: output block is {ny} x {ky}, input block is {n} x {k}")
    return px, ldx, k, py, ldy


def _out_cols(h, X, cols, where):
    """An output block that receives `cols` columns: (pointer, ld)."""
    px, ldx, n, k = _block(X)
    _check_rows(h, n, where)
    if k < cols:
        raise ValueError(f"{where}: output block has {k} columns, {cols} are written")
    return px, ldx


def _vec(x):
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return C.c_void_p(x.ctypes.data)
    return C.c_void_p(x.data_ptr())


def ie_status_str(status: int) -> str:
    return load().ie_status_str(int(status)).decode()


def ie_opts_default(**overrides) -> ie_opts:
    o = ie_opts()
    load().ie_opts_default(C.byref(o))
    for k_, v in overrides.items():
        setattr(o, k_, v)
    return o


def ie_create(n, offsets, A_dia, B_dia, center, radius, p, q, opts=None, stream=None):
    """Returns (status, handle). A_dia, B_dia: (ndiag, n) complex128 (device tensor or host array)."""
    L = load()
    offs = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    pen = ie_pencil(int(n), len(offs), offs.ctypes.data_as(C.POINTER(C.c_int64)), _vec(A_dia),
                    _vec(B_dia))
    h = C.c_void_p()
    o = opts if opts is not None else ie_opts_default()
    st = L.ie_create(C.byref(pen), ie_complex(complex(center).real, complex(center).imag),
                     float(radius), int(p), int(q), C.byref(o), _stream(stream), C.byref(h))
    if h.value:
        _handle_n[h.value] = int(n)
    return st, h


def ie_destroy(h):
    if h is not None:
        _handle_n.pop(_hkey(h), None)
    return load().ie_destroy(h)


def ie_filter_apply(h, Y, U, stream=None):
    py, ldy, k, pu, ldu = _in_out(h, Y, U, "ie_filter_apply")
    return load().ie_filter_apply(h, py, ldy, k, pu, ldu, _stream(stream))


def ie_apply_G(h, V, GV, stream=None):
    pv, ldv, k, pg, ldg = _in_out(h, V, GV, "ie_apply_G")
    return load().ie_apply_G(h, pv, ldv, k, pg, ldg, _stream(stream))


def ie_apply_G_static(h, V, GV, stream=None):
    """G(V) with the library's static scratch: no device allocation by the call.
    V, GV must be device tensors."""
    pv, ldv, k, pg, ldg = _in_out(h, V, GV, "ie_apply_G_static")
    return load().ie_apply_G_static(h, pv, ldv, k, pg, ldg, _stream(stream))


def ie_spmv(h, which, X, Y, stream=None):
    px, ldx, k, py, ldy = _in_out(h, X, Y, "ie_spmv")
    return load().ie_spmv(h, int(which), px, ldx, k, py, ldy, _stream(stream))


def ie_hsrr(h, U, X=None, stream=None):
    """Returns (status, lambda (k,), e (k,), rho (k,)); Ritz vectors into X when given."""
    pu, ldu, n, k = _block(U)
    _check_rows(h, n, "ie_hsrr")
    px, ldx = _out_cols(h, X, k, "ie_hsrr") if X is not None else (None, 0)
    lam = np.zeros(k, dtype=np.complex128)
    e = np.zeros(k)
    rho = np.zeros(k)
    st = load().ie_hsrr(h, pu, ldu, k, _vec(lam), px, ldx if X is not None else 0, _vec(e),
                        _vec(rho), _stream(stream))
    return st, lam, e, rho


def ie_solve(h, Y0, X, k, stream=None):
    """Returns (status, lambda (k,), rho (k,), e (k,), n_found, stats dict)."""
    p0, ld0, n0, k0 = _block(Y0)
    if Y0 is not None:
        _check_rows(h, n0, "ie_solve")
        if k0 < k:
            raise ValueError(f"ie_solve: starting block has {k0} columns, {k} are read")
    px, ldx = _out_cols(h, X, k, "ie_solve")
    lam = np.zeros(k, dtype=np.complex128)
    rho = np.zeros(k)
    e = np.zeros(k)
    nf = C.c_int32()
    stt = ie_stats()
    st = load().ie_solve(h, p0, ld0 if Y0 is not None else 0, _vec(lam), px, ldx, _vec(rho),
                         _vec(e), C.byref(nf), C.byref(stt), _stream(stream))
    return st, lam, rho, e, nf.value, stt.as_dict()


def ie_apply_GH(h, V, GV, stream=None):
    """GV = sum_i conj(w_i) K_i^{-H} B^H V (handles created with opts.adjoint = 1)."""
    pv, ldv, k, pg, ldg = _in_out(h, V, GV, "ie_apply_GH")
    return load().ie_apply_GH(h, pv, ldv, k, pg, ldg, _stream(stream))


def ie_solve_left(h, lam, Y, Y0=None, stream=None):
    """Left eigenvectors for the eigenvalues `lam` (nl,) into the first nl columns of Y.
    Returns (status, lambda_left (nl,), rho_left (nl,), stats dict)."""
    lam = np.ascontiguousarray(np.asarray(lam, dtype=np.complex128))
    nl = len(lam)
    p0, ld0, n0, _ = _block(Y0)
    if Y0 is not None:
        _check_rows(h, n0, "ie_solve_left")
    py, ldy = _out_cols(h, Y, nl, "ie_solve_left")
    ll = np.zeros(nl, dtype=np.complex128)
    rl = np.zeros(nl)
    stt = ie_stats()
    st = load().ie_solve_left(h, _vec(lam), nl, p0, ld0 if Y0 is not None else 0, py, ldy,
                              _vec(ll), _vec(rl), C.byref(stt), _stream(stream))
    return st, ll, rl, stt.as_dict()


def ie_eig_sensitivity(h, X, Y, alpha=1j, S=None, gbar=None, grad=None, stream=None):
    """S[j, i] = alpha conj(Y[j, i]) X[j, i] / (Y_i^H B X_i) into S (n x nf) and
    grad[j] = Re sum_i conj(gbar_i) S[j, i] into grad (n doubles); either may be None."""
    px, ldx, nf, py, ldy = _in_out(h, X, Y, "ie_eig_sensitivity")
    ps, lds = _out_cols(h, S, nf, "ie_eig_sensitivity") if S is not None else (None, 0)
    gb = None
    if gbar is not None:
        gb = np.ascontiguousarray(np.asarray(gbar, dtype=np.complex128))
        if gb.shape != (nf,):
            raise ValueError(f"ie_eig_sensitivity: gbar has shape {gb.shape}, expected ({nf},)")
    if grad is not None:
        n = _handle_n.get(_hkey(h), grad.shape[0])
        if tuple(grad.shape) != (n,) or "float64" not in str(grad.dtype):
            raise ValueError(f"ie_eig_sensitivity: grad must be a vector of {n} float64 values")
    a = complex(alpha)
    return load().ie_eig_sensitivity(h, px, ldx, py, ldy, nf, ie_complex(a.real, a.imag), ps,
                                     lds if S is not None else 0, _vec(gb), _vec(grad),
                                     _stream(stream))


def _batch_items(problems, streams, where):
    nb = len(problems)
    items = (ie_batch_item * nb)()
    keep = []
    for i, (h, Y0, X, k) in enumerate(problems):
        p0, ld0, n0, k0 = _block(Y0)
        if Y0 is not None:
            _check_rows(h, n0, where)
            if k0 < k:
                raise ValueError(f"{where}: item {i} starting block has {k0} columns")
        px, ldx = _out_cols(h, X, k, f"{where} item {i}")
        lam = np.zeros(k, dtype=np.complex128)
        rho = np.zeros(k)
        e = np.zeros(k)
        keep.append((lam, rho, e))
        it = items[i]
        it.h = h.value if isinstance(h, C.c_void_p) else h
        it.Y0_any = p0.value if p0 is not None else None
        it.ldy0 = ld0 if Y0 is not None else 0
        it.h_lambda = lam.ctypes.data
        it.X_any = px.value
        it.ldx = ldx
        it.h_rho = rho.ctypes.data
        it.h_e = e.ctypes.data
        s_ = streams[i] if streams is not None else None
        it.stream = (s_ if isinstance(s_, int) else s_.cuda_stream) if s_ is not None else None
    return items, keep


def _batch_results(items, keep):
    out = []
    for i in range(len(keep)):
        lam, rho, e = keep[i]
        out.append({"status": items[i].status, "lam": lam, "rho": rho, "e": e,
                    "n_found": items[i].n_found, "stats": items[i].stats.as_dict()})
    return out


def ie_solve_batch(problems, max_workers=0, streams=None):
    """problems: list of (handle, Y0 or None, X, k). Runs their drivers concurrently
    (ie_solve_batch). Returns (status, [dict(status, lam, rho, e, n_found, stats)])."""
    items, keep = _batch_items(problems, streams, "ie_solve_batch")
    st = load().ie_solve_batch(items, len(problems), int(max_workers))
    return st, _batch_results(items, keep)


def ie_solve_batch_fused(problems, stream=None):
    """problems: list of (handle, Y0 or None, X, k). All drivers advance in lockstep with one
    batched band-solve launch per Arnoldi step (ie_solve_batch_fused).
    Returns (status, [dict(status, lam, rho, e, n_found, stats)])."""
    items, keep = _batch_items(problems, None, "ie_solve_batch_fused")
    st = load().ie_solve_batch_fused(items, len(problems), _stream(stream))
    return st, _batch_results(items, keep)


def ie_get_coeffs(h, p, q):
    poles = np.zeros(q, dtype=np.complex128)
    w = np.zeros(q, dtype=np.complex128)
    s = np.zeros(max(p, 1), dtype=np.complex128)
    c = np.zeros(max(p, 1), dtype=np.complex128)
    ns = C.c_int32()
    odd = C.c_double()
    st = load().ie_get_coeffs(h, _vec(poles), _vec(w), _vec(s), _vec(c), C.byref(ns), C.byref(odd))
    return st, poles, w, s[: ns.value], c[: ns.value], odd.value


def ie_get_factor(h, pole, n, ldab):
    ab = np.zeros((n, ldab), dtype=np.complex128)        # row j = band column j
    ipiv = np.zeros(n, dtype=np.int32)
    kl = C.c_int32()
    ld = C.c_int32()
    st = load().ie_get_factor(h, int(pole), _vec(ab), _vec(ipiv), C.byref(kl), C.byref(ld))
    return st, np.asfortranarray(ab.T), ipiv, kl.value


def ie_get_stats(h):
    s = ie_stats()
    st = load().ie_get_stats(h, C.byref(s))
    return st, s.as_dict()
