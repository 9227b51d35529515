"""The FP32 streaming path's reductions, isolated from its per-site rounding.

The streaming kernel adds each thread's per-site densities in FP32 over at
most 40 planes, then in double-float (hi, lo) pairs over the block and the
grid, and compares the rounded FP64 total in the arrest test.
skyrme_step_densities runs one ordinary iteration that also writes the very
FP32 values the kernel added.  Their exact sum (math.fsum, in FP64) against
the iteration's reported E_n, B and virial is the error of the reduction
alone: it must be far below the FP32 flow's arrest-noise floor (consecutive
FP32 fields differ in energy by a few 1e-6 relative to E late in a
relaxation)."""
import math

import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
sk = pytest.importorskip("paper_2604_25876_gb300")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
KB = -1.0 / (2.0 * math.pi ** 2)  # baryon density = KB * det


def exact_sums(dens, n):
    d = dens[2:n[0] - 2, 2:n[1] - 2, 2:n[2] - 2].double().cpu().numpy().reshape(-1, 4)
    sums = [math.fsum(d[:, q]) for q in range(4)]
    abs_det = math.fsum(np.abs(d[:, 3]))
    return sums, abs_det


@pytest.mark.parametrize("name", ["b4_cubic_128", "b8_cluster_256"])
def test_reported_sums_equal_the_exact_sum_of_the_kernel_densities(name):
    wl = workloads.ALL[name]()
    lat = sk.Lattice(wl.n, wl.h, wl.m, 32)
    st = sk.State(lat, DEV)
    sk.init_field(lat, sk.Seed.from_spec(wl.seed), st)
    # a few ordinary iterations first: a field that is not a seed
    sk.flow_step(lat, wl.dt, 5, sk.ARRESTED, st)
    dens, rep = sk.step_densities(lat, wl.dt, sk.ARRESTED, st)
    (s2, s4, su, sdet), abs_det = exact_sums(dens, wl.n)
    h3 = wl.h ** 3
    E2, E4, E0 = h3 * s2, h3 * s4, h3 * 2.0 * wl.m ** 2 * su
    E, B = E2 + E4 + E0, h3 * KB * sdet
    V = -E2 + E4 - 3.0 * E0
    err = {"E": abs(rep["E"] - E) / E, "E2": abs(rep["E2"] - E2) / E2,
           "E4": abs(rep["E4"] - E4) / E4, "E0": abs(rep["E0"] - E0) / E0,
           "B": abs(rep["B"] - B) / (h3 * abs(KB) * abs_det),
           "virial": abs(rep["virial"] - V) / E}
    print(name, {k: f"{v:.2e}" for k, v in err.items()})
    for k, v in err.items():
        assert v <= 1e-10, (k, v)
    assert rep["steps"] == 6 and rep["status"] == 0


def test_dumped_densities_match_the_oracle_site_by_site():
    n, h, m = (24, 22, 26), 0.25, 1.0
    phi = oracle.apply_vacuum_boundary(
        np.ascontiguousarray(oracle.rational_map_field(n, h, 2, 1.0, X=(0.3, 0.1, -0.2))))
    lat = sk.Lattice(n, h, m, 32)
    st = sk.State(lat, DEV)
    sk.load_field(lat, st, phi)
    f32 = st.field().double().cpu().numpy()  # the FP32 field the kernel sees
    dens, _ = sk.step_densities(lat, 0.01, sk.ARRESTED, st)
    _, _, d = oracle.forces(f32, h, m)
    got = dens.double().cpu().numpy()
    inner = (slice(2, -2),) * 3
    scale = np.abs(d[inner]).max(axis=(0, 1, 2))
    # {e2, e4, u, det}: u = e0 / 2 m^2, det = b / KB
    expect = np.stack([d[..., 0], d[..., 1], d[..., 2] / (2 * m * m), d[..., 3] / KB], -1)
    scale[2] /= 2 * m * m
    scale[3] /= abs(KB)
    err = np.abs(got[inner] - expect[inner]).max(axis=(0, 1, 2)) / scale
    assert np.all(err < 2e-5), err
    # sites outside the interior are not written
    assert np.all(got[:2] == 0) and np.all(got[:, -2:] == 0)
