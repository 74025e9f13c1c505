"""Writes tests/golden/workloads.json: the workload definitions (grid, seed,
disk centre and radius, orders p and q, block k) and the reference eigenvalues
inside each disk. Calls only the oracle (dense QZ for n <= 1600; shift-invert
Arnoldi otherwise, as the paper's reference eigenvalues come from eigs, Sec. 6.2).

Disk recipe: centre = the median eigenvalue (sort by real part, ties by imaginary
part, index floor(n/2)); radius = midpoint of the N-th and (N+1)-th distances from
the centre, so the disk holds exactly N eigenvalues. For n > 1600 the median is not
computed exactly: the centre is the eigenvalue nearest the point
(4/h^2)/1.025 + i*mean(gamma) -- the median of the unperturbed operator scaled by
the mean of B's diagonal (checked against the exact median at small m by this script).

Batch workloads (ie_inputs.batch_problems): the proxy point is the closed-form eigenvalue
of the constant-coefficient operator at the fraction proxy_frac of its sorted spectrum,
scaled by 1/1.025, plus i*mean(gamma); then the same nearest-eigenvalue centre and
N-eigenvalue radius.

Usage: python tests/golden/make_golden.py [names...]
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import ie_inputs  # noqa: E402
from oracle import pencil as opencil, reference_eigs as ref  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "workloads.json")

SPECS = {
    # tiny parity case: m=24, seed 0, q=p=4, k=16, ~10 eigenvalues, driver 1
    "c1_m24": dict(m=24, seed=0, p=4, q=4, k=16, n_in=10, driver=1),
    # ragged: n=1369, odd p, k not a multiple of any tile width
    "r1_m37": dict(m=37, seed=1, p=5, q=3, k=11, n_in=7, driver=1),
    # medium: n=4096, several column groups per pole
    "m1_m64": dict(m=64, seed=2, p=4, q=6, k=24, n_in=16, driver=2),
    # profiling size: band 160, factors 1.6 GB (> L2, a few GB on the device)
    "p1_m160": dict(m=160, seed=3, p=8, q=8, k=64, n_in=30, driver=1),
    # at scale: m=256 (n=65,536, band 256), q=p=8, k=64, ~40 eigenvalues, both drivers
    "c2_m256": dict(m=256, seed=0, p=8, q=8, k=64, n_in=40, driver=1),
    # precision: m=512 (n=262,144, band 512), q=p=8, k=96, mixed-precision solves
    "c4_m512": dict(m=512, seed=0, p=8, q=8, k=96, n_in=60, driver=2, precision=1),
}
# the batched-solver mix (12 problems: grids 64..192, 1-2 disks each)
for _b in ie_inputs.batch_problems(12, 0):
    SPECS[_b["name"]] = {k_: v for k_, v in _b.items() if k_ != "name"}


def proxy_center(pen, frac=None):
    if frac is None:
        h = 1.0 / (pen.m + 1)
        return (4.0 / h**2) / 1.025 + 1j * float(np.mean(pen.gamma))
    lam = ie_inputs.closed_form_spectrum(pen.m)
    return lam[int(frac * pen.n)] / 1.025 + 1j * float(np.mean(pen.gamma))


def build(name, spec):
    t0 = time.time()
    pen = ie_inputs.make_pencil(spec["m"], spec["seed"])
    A, B = opencil.pencil_matrices(pen)
    n_in = spec["n_in"]
    info = {}
    if pen.n <= 1600:
        lam = ref.all_eigenvalues(A, B)
        c = ref.median_eigenvalue(lam)
        d = np.abs(lam - c)
        r = ref.disk_radius(d, n_in)
        inside = lam[d < r]
        info["median_exact"] = True
        info["proxy_center_offset"] = abs(proxy_center(pen) - c)
    else:
        c0 = proxy_center(pen, spec.get("proxy_frac"))
        near0 = ref.nearest_eigenvalues(A, B, c0, 8)
        c = near0[0]
        # Shift-invert from two shifts that are not eigenvalues (c itself is one): the
        # proxy point c0 and c offset by a quarter of the distance to c's nearest neighbour.
        # Both runs must agree on every eigenvalue near c.
        gap = float(np.sort(np.abs(near0 - c))[1])
        runA = ref.nearest_eigenvalues(A, B, c0, n_in + 24)
        runB = ref.nearest_eigenvalues(A, B, c + 0.25 * gap * np.exp(1j * np.pi / 3), n_in + 24)
        near = runB[np.argsort(np.abs(runB - c))][: n_in + 8]
        xerr = max(float(np.min(np.abs(runA - v)) / abs(v)) for v in near)
        assert xerr < 1e-12, f"shift-invert runs disagree: {xerr}"
        d = np.abs(near - c)
        r = ref.disk_radius(d, n_in)
        inside = near[d < r]
        info["median_exact"] = False
        info["proxy_center"] = [c0.real, c0.imag]
        info["crosscheck_rel"] = xerr
    inside = inside[np.argsort(np.abs(inside - c))]
    d_sorted = np.sort(np.abs(inside - c))
    out = dict(spec)
    out.update(n=pen.n, center_re=float(c.real), center_im=float(c.imag), radius=float(r),
               eig_in_disk_re=[float(v.real) for v in inside],
               eig_in_disk_im=[float(v.imag) for v in inside],
               boundary_gap_rel=float((r - d_sorted[-1]) / r), **info,
               seconds=time.time() - t0)
    return out


def main(names):
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            data = json.load(f)
    for name in names or list(SPECS):
        data[name] = build(name, SPECS[name])
        print(name, {k: v for k, v in data[name].items() if not k.startswith("eig_")}, flush=True)
        with open(OUT, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main(sys.argv[1:])
