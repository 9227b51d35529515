"""Pins of the degree-2 and degree-3 rational maps of Table 1 (Section 4.1):
their degree (the baryon number of the seed) and the symmetry they impose on
the seed (Section 4.1: the Skyrmion inherits the map's symmetry), seen in the
inertia tensors of Section 5."""
import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("B,scale", [(2, 1.2), (3, 1.3)])
def test_seed_charge_is_the_degree(B, scale):
    # the lattice deficit is set by the spacing (the degree-3 map turns sharply
    # between its faces), and shrinks as h falls
    coarse = oracle.energy(oracle.seed_rational_map((40, 40, 40), 0.24, B, scale), 0.24, 0.0)["B"]
    mid = oracle.energy(oracle.seed_rational_map((80, 80, 80), 0.12, B, scale), 0.12, 0.0)["B"]
    fine = oracle.energy(oracle.seed_rational_map((120, 120, 120), 0.08, B, scale), 0.08, 0.0)["B"]
    assert abs(fine - B) < 1e-2 and abs(fine - B) < abs(mid - B) < abs(coarse - B)


def test_degree_two_seed_is_axially_symmetric_and_degree_three_is_tetrahedral():
    n, h = (60, 60, 60), 0.15
    o2 = oracle.observables(oracle.seed_rational_map(n, h, 2, 1.2), h, 1.0)
    o3 = oracle.observables(oracle.seed_rational_map(n, h, 3, 1.3), h, 1.0)
    for o in (o2, o3):
        for key in ("U", "V", "W"):
            T = np.asarray(o[key])
            assert np.max(np.abs(T - np.diag(np.diag(T)))) < 1e-6 * np.max(np.abs(T)) + 1e-9, key
    # z^2 winds twice about the z axis: symmetric about it, not isotropic.
    # A quarter turn of space (a lattice symmetry) swaps V's first two axes
    # exactly; U's are swapped only by the eighth turn paired with a quarter
    # isorotation, which the lattice lacks, so they agree to the lattice error.
    U2, V2, W2 = np.diag(o2["U"]), np.diag(o2["V"]), np.diag(o2["W"])
    assert V2[0] == pytest.approx(V2[1], rel=1e-9) and abs(V2[2] - V2[0]) > 0.05 * V2[0]
    assert U2[0] == pytest.approx(U2[1], rel=5e-3) and abs(U2[2] - U2[0]) > 0.05 * U2[0]
    assert abs(W2[0]) < 1e-6 * abs(W2[2]) and abs(W2[1]) < 1e-6 * abs(W2[2])
    # tetrahedral symmetry makes every inertia tensor isotropic, the mixed one
    # included (and non-zero), and the quadrupole vanish
    for key in ("U", "V", "W"):
        d = np.diag(o3[key])
        assert np.max(np.abs(d - d.mean())) < 2e-3 * abs(d.mean()), (key, d)
    assert abs(np.diag(o3["W"]).mean()) > 0.1 * np.diag(o3["U"]).mean()
    assert np.max(np.abs(o3["Q"])) < 1e-3 * o3["R"] ** 2 * o3["B"]
