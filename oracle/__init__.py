"""FP64 CPU oracle for the composite-rule rational filter eigensolver.

TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the CPU-baseline
leg of the benchmark may import this package. The CUDA library never calls it,
and it shares no code with the CUDA path (only the seeded inputs in `ie_inputs`).

Every function restates a passage of Chen & Li, "Interior Eigensolver Based on
Rational Filter with Composite Rule" (arXiv 2310.18043), cited by section and
equation. Readings of passages that are ambiguous or in error are marked
"reading:" in the docstrings.

Pins (tests/test_oracle_*.py), each against something other than the oracle:
  coeffs   - Lemma 1 closed form, the k=2,4 worked examples (Sec. 4.3), the
             Moebius identity (Eq. mobiustrans) on the Fig. mobius grid,
             Prop. 1, Re(s_j)=1/2, the Corollary's separation 2/((b/a)^k-1).
  inner    - dense spectral definition X R_q(Lambda) X^{-1} (Eq. CIoperator).
  msgmres  - dense (G - s_j I)^{-1} per shift; composite filter equals the
             pq-pole simple rule and X R_pq(Lambda) X^{-1} Y (Thm 2).
  hsrr / drivers - tiny pencils with planted spectra; dense QZ on the small
             convection-diffusion pencil; eigen-residuals.
  adjoint  - dense spectral definition for the adjoint pencil; the identity
             B^H G_adj = G^H B^H; LAPACK left eigenvectors; central finite
             differences of dense eigenvalues for the sensitivities and the VJP.
  reference_eigs - shift-invert Arnoldi against dense QZ on the m = 12 and m = 24
             pencils; median and radius against hand-built arrays with ties and the
             exact-count property (tests/test_oracle_reference_eigs.py).
No function is "parity unpinned".
"""
from . import coeffs, pencil, inner, msgmres, hsrr, drivers, adjoint  # noqa: F401
