"""GPU parity of the Section 7.8 extension models (modified-pion, loosely and
lightly bound potentials, BPS sextic term) with the oracle, through the C ABI.

Tolerances are those of the standard-model parity tests: FP64 forces and
densities within 1e-12 of the oracle relative to their max-norm and energies
within 1e-12 relative; FP32 forces within 1e-5 normwise (the sextic gradient
is a product of first and second lattice derivatives like the quartic one,
so the same per-stencil rounding bound applies) and energies within ~2e-6."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

sk = pytest.importorskip("paper_2604_25876_gb300")

DEV = "cuda:0"
EXT = dict(m_y=0.9, m_z=0.6, m_w=1.1, c6=0.35)
MX = 0.7


def model(**kw):
    e = dict(EXT, **kw)
    return oracle.Model(MX, e["m_y"], e["m_z"], e["m_w"], e["c6"])


def generic_field(n, h, seed=3):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(-0.9, 0.9, size=(3, 3))
    q = rng.normal(size=(3, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return oracle.seed_product(n, h, pos, q, 0.9, True)


def on_gpu(phi, h, prec, **kw):
    lat = sk.Lattice(phi.shape[:3], h, MX, prec, **dict(EXT, **kw))
    st = sk.State(lat, DEV)
    sk.load_field(lat, st, phi)
    return lat, st


TERMS = [dict(), dict(c6=0.0), dict(m_y=0.0, m_z=0.0, m_w=0.0), dict(m_y=0.0, m_z=0.0, c6=0.0)]


@pytest.mark.parametrize("terms", range(len(TERMS)))
@pytest.mark.parametrize("prec,tol", [(64, 1e-12), (32, 1e-5)])
def test_forces_and_densities_match_oracle(terms, prec, tol):
    kw = TERMS[terms]
    n, h = (27, 30, 33), 0.22  # ragged against the 2 x 4 x 32 tile
    phi = generic_field(n, h)
    if prec == 32:
        phi = phi.astype(np.float32).astype(np.float64)
    _, Fo, Do = oracle.forces(phi, h, model(**kw))
    lat, st = on_gpu(phi, h, prec, **kw)
    F, D = sk.forces(lat, st)
    Fg, Dg = F.double().cpu().numpy(), D.double().cpu().numpy()
    scale = np.max(np.abs(Fo))
    assert scale > 1.0
    assert np.max(np.abs(Fg - Fo)) <= tol * scale
    for q in range(4):
        s = np.max(np.abs(Do[..., q]))
        assert np.max(np.abs(Dg[..., q] - Do[..., q])) <= tol * s * 4, q


@pytest.mark.parametrize("prec,tol", [(64, 1e-12), (32, 2e-6)])
def test_energy_sextic_part_and_virial_match_oracle(prec, tol):
    n, h = (36, 40, 44), 0.2
    phi = oracle.seed_rational_map(n, h, 4, 1.5)
    if prec == 32:
        phi = phi.astype(np.float32).astype(np.float64)
    eo = oracle.energy(phi, h, model())
    assert eo["E6"] > 0.05 * eo["E"]
    lat, st = on_gpu(phi, h, prec)
    eg = sk.energy(lat, st)
    for k in ("E", "E2", "E4", "E0"):
        assert eg[k] == pytest.approx(eo[k], rel=tol), k
    assert eg["B"] == pytest.approx(eo["B"], rel=tol)
    assert eg["virial"] == pytest.approx(eo["virial"], rel=tol * 10, abs=tol * eo["E"])
    assert sk.sextic_energy(lat, st) == pytest.approx(eo["E6"], rel=tol)
    # the allocation-free entry point computes the same sums
    es = sk.energy_static(lat, st.field())
    for k in ("E", "E2", "E4", "E0", "B", "virial"):
        assert es[k] == pytest.approx(eo[k], rel=tol * 4, abs=tol * 1e-3), k


@pytest.mark.parametrize("mode", [sk.ARRESTED, sk.NEWTON, sk.GRADIENT])
def test_fp64_trajectory_matches_oracle(mode):
    n, h = (26, 29, 31), 0.25
    dt = 0.05 * h if mode != sk.GRADIENT else 1e-4
    phi = oracle.seed_rational_map(n, h, 1, 0.9)
    ost = oracle.new_state(phi)
    oreps = oracle.flow(ost, h, model(), dt, 60, mode=mode, reports=True)
    lat, st = on_gpu(phi, h, 64)
    for _ in range(3):
        rep = sk.flow_step(lat, dt, 20, mode, st)
    g = st.field().cpu().numpy()
    assert np.max(np.abs(g - ost.phi)) < 1e-11
    if mode != sk.GRADIENT:
        assert np.max(np.abs(st.velocity().cpu().numpy() - ost.v)) < 1e-11
    last = oreps[-1]
    for k in ("E", "E6", "B", "virial"):
        assert rep[k] == pytest.approx(last[k], rel=1e-11), k
    assert rep["delta"] == pytest.approx(last["delta"], rel=1e-10)
    assert rep["steps"] == 60
    assert rep["arrests"] == sum(r["arrested"] for r in oreps)


def test_fp32_trajectory_tracks_fp64_oracle():
    n, h = (40, 40, 40), 0.2
    phi = oracle.seed_rational_map(n, h, 4, 2.0)
    ost = oracle.new_state(phi)
    oreps = oracle.flow(ost, h, model(), 0.05 * h, 50, reports=True)
    lat, st = on_gpu(phi, h, 32)
    rep = sk.flow_step(lat, 0.05 * h, 50, sk.ARRESTED, st)
    assert np.max(np.abs(st.field().double().cpu().numpy() - ost.phi)) < 1e-4
    assert rep["E"] == pytest.approx(oreps[-1]["E"], rel=1e-5)
    assert rep["E6"] == pytest.approx(oreps[-1]["E6"], rel=1e-5)


POTENTIALS = [dict(m_y=0.9, m_z=0.0, m_w=0.0), dict(m_y=0.0, m_z=0.6, m_w=0.0),
              dict(m_y=0.0, m_z=0.0, m_w=1.1), dict(m_y=0.9, m_z=0.6, m_w=1.1)]


@pytest.mark.parametrize("pot", range(len(POTENTIALS)))
def test_fp32_potentials_flow_on_the_streaming_kernel_tracks_the_oracle(pot):
    """With the potentials on and no sextic term the FP32 flow runs on the
    streaming kernel.  Its first energy equals the tile kernel's evaluation of
    the same field, and 50 arrested iterations follow the FP64 oracle: field
    within 1e-4, energy and virial within 1e-5, the same arrests."""
    kw = dict(POTENTIALS[pot], c6=0.0)
    n, h = (40, 40, 40), 0.2
    phi = oracle.seed_rational_map(n, h, 4, 2.0)
    ost = oracle.new_state(phi)
    oreps = oracle.flow(ost, h, model(**kw), 0.05 * h, 50, reports=True)
    lat, st = on_gpu(phi, h, 32, **kw)
    e_tile = sk.energy(lat, st)
    r1 = sk.flow_step(lat, 0.05 * h, 1, sk.ARRESTED, st)
    assert r1["E"] == pytest.approx(e_tile["E"], rel=2e-6)
    assert r1["E0"] == pytest.approx(e_tile["E0"], rel=2e-6)
    rep = sk.flow_step(lat, 0.05 * h, 49, sk.ARRESTED, st)
    assert rep["status"] == 0 and rep["steps"] == 50 and rep["E6"] == 0.0
    assert np.max(np.abs(st.field().double().cpu().numpy() - ost.phi)) < 1e-4
    assert rep["E"] == pytest.approx(oreps[-1]["E"], rel=1e-5)
    assert rep["E0"] == pytest.approx(oreps[-1]["E0"], rel=1e-5)
    assert rep["virial"] == pytest.approx(oreps[-1]["virial"], rel=1e-4, abs=1e-5 * rep["E"])
    assert rep["arrests"] == sum(r["arrested"] for r in oreps)


def test_fp32_sextic_flow_on_the_streaming_kernel_tracks_the_oracle():
    """With the sextic term the FP32 flow runs on the streaming kernel's
    sextic variant.  Its first energy and sextic energy equal the tile
    kernel's evaluation of the same field, and 50 arrested iterations follow
    the FP64 oracle: field within 1e-4, E and E6 within 1e-5, the same
    arrests."""
    n, h = (38, 41, 44), 0.2  # ragged against the 16 x 32 column tile
    phi = oracle.seed_rational_map(n, h, 4, 2.0)
    for kw in (dict(m_y=0.0, m_z=0.0, m_w=0.0), dict()):
        ost = oracle.new_state(phi)
        oreps = oracle.flow(ost, h, model(**kw), 0.05 * h, 50, reports=True)
        lat, st = on_gpu(phi, h, 32, **kw)
        e_tile = sk.energy(lat, st)
        e6_tile = sk.sextic_energy(lat, st)
        r1 = sk.flow_step(lat, 0.05 * h, 1, sk.ARRESTED, st)
        assert r1["E"] == pytest.approx(e_tile["E"], rel=2e-6)
        assert r1["E6"] == pytest.approx(e6_tile, rel=2e-6)
        assert r1["virial"] == pytest.approx(e_tile["virial"], rel=2e-5, abs=2e-6 * r1["E"])
        rep = sk.flow_step(lat, 0.05 * h, 49, sk.ARRESTED, st)
        assert rep["status"] == 0 and rep["steps"] == 50
        assert np.max(np.abs(st.field().double().cpu().numpy() - ost.phi)) < 1e-4
        assert rep["E"] == pytest.approx(oreps[-1]["E"], rel=1e-5)
        assert rep["E6"] == pytest.approx(oreps[-1]["E6"], rel=1e-5)
        assert rep["arrests"] == sum(r["arrested"] for r in oreps)


def test_standard_model_report_has_no_sextic_part_and_vacuum_stays_fixed():
    for prec in (32, 64):
        lat = sk.Lattice((20, 21, 22), 0.2, 1.0, prec)
        st = sk.State(lat, DEV)
        sk.init_field(lat, sk.Seed.rational_map(1, 1.0), st)
        assert sk.flow_step(lat, 0.01, 3, sk.ARRESTED, st)["E6"] == 0.0
        # every extension potential vanishes at the vacuum with zero force
        lat = sk.Lattice((20, 21, 22), 0.2, 1.0, prec, **EXT)
        st = sk.State(lat, DEV)
        sk.init_field(lat, sk.Seed.vacuum(), st)
        rep = sk.flow_step(lat, 0.01, 3, sk.ARRESTED, st)
        f = st.field().double().cpu().numpy()
        assert np.all(f[..., 0] == 1.0) and not f[..., 1:].any()
        assert rep["delta"] == 0.0 and rep["E"] == 0.0


def test_extended_lattices_are_rejected_where_unsupported():
    n, h = (24, 24, 24), 0.25
    lat, st = on_gpu(generic_field(n, h), h, 32)
    with pytest.raises(sk.SkyrmeError) as e:
        sk.observables(lat, st)
    assert e.value.status == 6
