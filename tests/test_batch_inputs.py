"""CPU checks of the batch workload: the recipe is seeded and stable, the stored disks
(tests/golden/workloads.json, written by make_golden.py from the oracle) match it, and the
closed-form spectrum used to place the disks is the spectrum of the constant-coefficient
operator."""
import numpy as np

import ie_inputs
from oracle import pencil as opencil


def test_recipe_is_deterministic_and_in_range():
    a = ie_inputs.batch_problems(12, 0)
    b = ie_inputs.batch_problems(12, 0)
    assert a == b and len(a) == 12
    assert len({x["name"] for x in a}) == 12
    for x in a:
        assert x["m"] in ie_inputs.BATCH_GRIDS
        assert x["k"] in (16, 24, 32) and x["q"] in (4, 6, 8) and x["p"] in (4, 8)
        assert x["n_in"] < x["k"]


def test_stored_disks_match_recipe():
    for x in ie_inputs.batch_problems(12, 0):
        w = ie_inputs.load_workload(x["name"])
        for key in ("m", "seed", "k", "q", "p", "n_in", "driver"):
            assert w[key] == x[key], (x["name"], key)
        lam = np.array(w["eig_in_disk_re"]) + 1j * np.array(w["eig_in_disk_im"])
        assert len(lam) == x["n_in"]
        assert np.all(np.abs(lam - w["center"]) < w["radius"])
        assert w["boundary_gap_rel"] > 0


def test_closed_form_spectrum_is_the_constant_coefficient_operator():
    m = 7
    pen = ie_inputs.make_pencil(m, seed=3)
    A, _ = opencil.pencil_matrices(pen)
    Acc = A.toarray() - 1j * np.diag(pen.gamma)        # drop the + i gamma diagonal
    ev = np.sort(np.linalg.eigvals(Acc).real)
    assert np.allclose(ev, ie_inputs.closed_form_spectrum(m), rtol=1e-12, atol=1e-9)
