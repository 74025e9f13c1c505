"""torch.autograd.Function over the C ABI: the eigenvalues of (A, B) in the disk D as a
function of the coefficient field gamma on the diagonal of A (A = A0 + i diag(gamma)).

Forward: ie_create (adjoint = 1), ie_solve, then ie_solve_left for the eigenvalues found.
Backward: ie_eig_sensitivity with alpha = i, which returns the vector-Jacobian product
grad_j = Re sum_i conj(gbar_i) d lambda_i / d gamma_j. PyTorch hands a complex output's
gradient to backward as gbar_i = dL/dRe(lambda_i) + i dL/dIm(lambda_i) for a real loss L,
which is the convention of that entry point. This module only marshals arguments: the solves,
the left eigenvectors and the product run in libie.so's kernels. Forming A0 + i diag(gamma)
is the input of ie_create, done with one torch add on the device.
"""
from __future__ import annotations

import numpy as np
import torch

from . import ie


class _Handle:
    """Owns an ie_handle until garbage collection (backward may never run)."""

    def __init__(self, h):
        self.h = h

    def __del__(self):
        if self.h is not None:
            ie.ie_destroy(self.h)
            self.h = None


def _check(st, where):
    if st != ie.IE_OK:
        raise ie.IeError(st, where)


class DiskEigenvalues(torch.autograd.Function):
    """lam = DiskEigenvalues.apply(gamma, A0_dia, B_dia, offsets, center, radius, p, q, opts)

    gamma: real (n,) tensor on the device (requires_grad for gradients); A0_dia, B_dia:
    complex128 (ndiag, n) device tensors in the DIA layout of include/ie.h, A0 without the
    i*gamma diagonal; offsets: the ndiag diagonal offsets (one of them 0). opts: an ie_opts
    (its k, driver, precision and tolerances are used; adjoint is set). Returns the n_found
    eigenvalues in D (complex128, ordered as by ie_solve). Raises ie.IeError when a call of
    the library fails or does not converge."""

    @staticmethod
    def forward(ctx, gamma, A0_dia, B_dia, offsets, center, radius, p, q, opts):
        offs = np.asarray(offsets, dtype=np.int64)
        main = int(np.flatnonzero(offs == 0)[0])
        A = A0_dia.clone()
        A[main] += 1j * gamma.to(torch.complex128)
        n = A.shape[1]
        o = ie.ie_opts()
        for f, _ in ie.ie_opts._fields_:
            setattr(o, f, getattr(opts, f))
        o.adjoint = 1
        k = o.k
        st, h = ie.ie_create(n, offs, A, B_dia, center, radius, p, q, o)
        _check(st, "ie_create")
        hh = _Handle(h)
        dev = A.device
        X = torch.zeros((k, n), dtype=torch.complex128, device=dev).T
        st, lam, rho, e, nf, _ = ie.ie_solve(h, None, X, k)
        _check(st, "ie_solve")
        Y = torch.zeros((k, n), dtype=torch.complex128, device=dev).T
        if nf > 0:
            st, _, _, _ = ie.ie_solve_left(h, lam[:nf], Y)
            _check(st, "ie_solve_left")
        ctx.handle = hh
        ctx.nf = nf
        ctx.save_for_backward(X[:, :nf], Y[:, :nf])
        return torch.from_numpy(np.array(lam[:nf])).to(dev)

    @staticmethod
    def backward(ctx, gbar):
        X, Y = ctx.saved_tensors
        n = X.shape[0]
        grad = torch.zeros(n, dtype=torch.float64, device=X.device)
        if ctx.nf > 0:
            g = gbar.detach().to(torch.complex128).cpu().numpy()
            st = ie.ie_eig_sensitivity(ctx.handle.h, X, Y, 1j, None, g, grad)
            _check(st, "ie_eig_sensitivity")
        return grad, None, None, None, None, None, None, None, None
