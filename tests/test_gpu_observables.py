"""GPU Section 5 observables (skyrme_observables, 4-vector reduction) against
the oracle (su(2) matrix formulas), on the same field values."""
import numpy as np
import pytest

import oracle
import paper_2604_25876_gb300 as sk
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
KEYS = ("B", "R", "D", "E")
MATS = ("X", "Q", "U", "V", "W")


def on_gpu(phi, h, m, prec):
    lat = sk.Lattice(phi.shape[:3], h, m, prec)
    st = sk.State(lat, DEV)
    sk.load_field(lat, st, phi)
    return lat, st


def compare(g, o, rel):
    for k in KEYS:
        assert g[k] == pytest.approx(o[k], rel=rel), k
    for k in MATS:
        a, b = np.array(g[k]), np.array(o[k])
        scale = max(np.max(np.abs(b)), 1.0)
        assert np.max(np.abs(a - b)) <= rel * scale, (k, a, b)


def generic_field(n, h, seed=5):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(-0.8, 0.8, size=(2, 3))
    q = rng.normal(size=(2, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return oracle.seed_product(n, h, pos, q, 0.9, False)


@pytest.mark.parametrize("prec", [64, 32])
def test_observables_match_oracle_on_a_generic_field(prec):
    n, h, m = (28, 30, 26), 0.25, 1.0
    phi = generic_field(n, h)
    if prec == 32:
        phi = phi.astype(np.float32).astype(np.float64)  # the values the GPU holds
    lat, st = on_gpu(phi, h, m, prec)
    g = sk.observables(lat, st)
    o = oracle.observables(phi, h, m)
    # an FP32 field is a unit vector to ~1e-7 only; for |phi| != 1 the su(2)
    # currents of the oracle and the 4-vector tangent projection of the kernel
    # differ at that level
    compare(g, o, 1e-11 if prec == 64 else 1e-6)
    assert sk.observables(lat, st) == g  # fixed summation order: bitwise repeatable


def test_observables_match_oracle_on_the_128_cubed_b4_seed():
    wl = workloads.b4_cubic_128()
    lat = sk.Lattice(wl.n, wl.h, wl.m, 32)
    st = sk.State(lat, DEV)
    sk.init_field(lat, sk.Seed.from_spec(wl.seed), st)
    g = sk.observables(lat, st)
    phi = st.field().cpu().numpy().astype(np.float64)
    o = oracle.observables(phi, wl.h, wl.m)
    compare(g, o, 1e-6)  # FP32 field: see above
    # the cubic B=4 map: centre at the origin, no quadrupole, isotropic U
    assert np.max(np.abs(g["X"])) < 1e-6 and np.max(np.abs(np.array(g["Q"]))) < 1e-4 * g["R"] ** 2
    U = np.array(g["U"])
    assert np.max(np.abs(U - np.diag(np.diag(U)))) < 1e-5 * U[0, 0]


def test_observables_of_the_vacuum_are_rejected():
    lat = sk.Lattice((16, 16, 16), 0.25, 1.0, 64)
    st = sk.State(lat, DEV)
    sk.init_field(lat, sk.Seed.vacuum(), st)
    with pytest.raises(sk.SkyrmeError):
        sk.observables(lat, st)
