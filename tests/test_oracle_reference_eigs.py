"""Pins of oracle/reference_eigs.py, the routines that fix the disk (centre, radius) and the
reference eigenvalues of every workload too large for dense QZ (Sec. 6.2 takes its reference
eigenvalues from a shift-invert eigs run; the workload's disk is centred at the median
eigenvalue and encloses a given count).

Each routine is checked against something other than itself: shift-invert Arnoldi against
dense QZ (scipy.linalg.eigvals) on the m = 12 and m = 24 pencils, the median and the radius
against hand-built arrays with ties, and the exact-count property of the radius."""
import numpy as np
import pytest
import scipy.linalg as sla

import ie_inputs
from oracle import pencil, reference_eigs


def _dense_nearest(A, B, sigma, count):
    lam = sla.eigvals(A.toarray(), B.toarray())
    lam = lam[np.isfinite(lam)]
    return lam[np.argsort(np.abs(lam - sigma))][:count], lam


def nearest_error(m, seed, count, offset):
    """Max relative distance between the oracle's `count` eigenvalues nearest sigma and dense
    QZ's, matched one to one. sigma = the dense median eigenvalue + offset (not an
    eigenvalue), with count chosen so the count-th and (count+1)-th distances are distinct."""
    pen = ie_inputs.make_pencil(m, seed)
    A, B = pencil.pencil_matrices(pen)
    lam_all = sla.eigvals(A.toarray(), B.toarray())
    sigma = reference_eigs.median_eigenvalue(lam_all) + offset
    d = np.sort(np.abs(lam_all - sigma))
    assert d[count] - d[count - 1] > 1e-6 * d[count], "ambiguous count for this pin"
    ref, _ = _dense_nearest(A, B, sigma, count)
    got = reference_eigs.nearest_eigenvalues(A, B, sigma, count)
    assert len(got) == count
    D = np.abs(got[:, None] - ref[None, :])
    j = np.argmin(D, axis=1)
    if sorted(j) != list(range(count)):
        return np.inf
    return float(np.max(np.min(D, axis=1) / np.abs(ref[j])))


@pytest.mark.parametrize("m,seed,count,offset", [(12, 0, 10, 0.37 + 0.11j), (24, 0, 20, -0.5 + 0.2j)])
def test_nearest_eigenvalues_match_dense_qz(m, seed, count, offset):
    assert nearest_error(m, seed, count, offset) < 1e-12


def test_nearest_eigenvalues_sorted_by_distance():
    pen = ie_inputs.make_pencil(12, 1)
    A, B = pencil.pencil_matrices(pen)
    sigma = A.diagonal().mean() + 0.3j
    got = reference_eigs.nearest_eigenvalues(A, B, sigma, 8)
    d = np.abs(got - sigma)
    assert np.all(np.diff(d) >= 0)


def test_median_eigenvalue_hand_built():
    lam = np.array([3 + 1j, 1 + 0j, 2 + 5j, 2 - 1j, 0 + 0j])
    # sorted by real part, ties by imaginary part: 0, 1, 2-1j, 2+5j, 3+1j -> index 2
    assert reference_eigs.median_eigenvalue(lam) == 2 - 1j
    for perm in ([4, 3, 2, 1, 0], [2, 0, 4, 1, 3]):
        assert reference_eigs.median_eigenvalue(lam[perm]) == 2 - 1j
    # even length: index n // 2 (0-based) of the sorted list, i.e. the upper of the two
    lam4 = np.array([4 + 0j, 1 + 2j, 1 - 2j, 3 + 0j])
    assert reference_eigs.median_eigenvalue(lam4) == 3 + 0j
    # all real parts tied: ordered by imaginary part alone
    lam3 = np.array([1 + 3j, 1 - 1j, 1 + 0j])
    assert reference_eigs.median_eigenvalue(lam3) == 1 + 0j


def test_disk_radius_hand_built_and_exact_count():
    assert reference_eigs.disk_radius([5.0, 1.0, 3.0, 2.0, 4.0], 2) == 2.5
    assert reference_eigs.disk_radius([1.0, 1.0, 2.0, 3.0], 2) == 1.5   # tie below the cut
    g = np.random.default_rng(0)
    d = g.uniform(0, 10, 200)
    for count in (1, 10, 40, 199):
        r = reference_eigs.disk_radius(d, count)
        assert np.sum(d < r) == count
        s = np.sort(d)
        assert s[count - 1] < r < s[count]
