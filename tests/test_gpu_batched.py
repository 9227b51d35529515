"""Batched flow: many FP32 lattices of uneven sizes in one persistent launch
per iteration.  Each lattice must follow the same trajectory as when it is
flowed alone, for every tile shape: the per-site formulas are the same, but
each kernel instantiation may contract multiply-adds differently, so the
comparison is at FP32 rounding level.  The autotuner's dry runs must leave
the flows untouched; a captured batch graph must equal batch_step bit for
bit (same kernels)."""
import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
sk = pytest.importorskip("paper_2604_25876_gb300")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"

SHAPES = [(20, 20, 20), (24, 28, 33), (30, 30, 30), (36, 22, 25), (17, 40, 19)]


def make_states(h=0.2, m=1.0, kind="map"):
    lats, states, fields = [], [], []
    for i, n in enumerate(SHAPES):
        lat = sk.Lattice(n, h, m, 32)
        st = sk.State(lat, DEV)
        if kind == "map":
            phi = oracle.seed_rational_map(n, h, 1 if i % 2 else 4, 1.2)
            sk.load_field(lat, st, phi)
        else:
            sk.init_field(lat, sk.Seed.noise(1.5, 0.6, 1000 + i), st)
        lats.append(lat)
        states.append(st)
    return lats, states


def test_batch_matches_lattices_flowed_alone():
    lats, states = make_states()
    solo_lats, solo = make_states()
    dt = [0.01] * len(lats)
    b = sk.Batch(lats, states, dt)
    b.step(30)
    torch.cuda.synchronize()
    for lat, st, ref in zip(solo_lats, solo, states):
        sk.flow_step(lat, 0.01, 30, sk.ARRESTED, st)
        r0, r1 = sk.read_report(lat, st), sk.read_report(lat, ref)
        assert r1["steps"] == 30 and r1["status"] == 0
        assert r1["E"] == pytest.approx(r0["E"], rel=1e-7)
        assert r1["arrests"] == r0["arrests"]
        np.testing.assert_allclose(ref.field().cpu().numpy(), st.field().cpu().numpy(),
                                   rtol=0, atol=2e-6)
    b.close()


def test_batch_with_potentials_matches_lattices_flowed_alone():
    """Lattices with Section 7.8 potentials (and standard ones) in one batch:
    the batch runs the potentials instantiation for all of them, and each
    lattice follows its solo flow (which runs the single-lattice potentials
    or standard kernel) to FP32 rounding."""
    pots = [dict(), dict(m_w=1.0), dict(m_y=0.5, m_z=0.4), dict(), dict(m_w=0.7)]

    def states():
        lats, sts = [], []
        for i, (n, kw) in enumerate(zip(SHAPES, pots)):
            lat = sk.Lattice(n, 0.2, 1.0, 32, **kw)
            st = sk.State(lat, DEV)
            sk.load_field(lat, st, oracle.seed_rational_map(n, 0.2, 1 if i % 2 else 4, 1.2))
            lats.append(lat)
            sts.append(st)
        return lats, sts

    lats, sts = states()
    solo_lats, solo = states()
    b = sk.Batch(lats, sts, [0.01] * len(lats))
    b.step(30)
    torch.cuda.synchronize()
    for lat, st, ref in zip(solo_lats, solo, sts):
        sk.flow_step(lat, 0.01, 30, sk.ARRESTED, st)
        r0, r1 = sk.read_report(lat, st), sk.read_report(lat, ref)
        assert r1["steps"] == 30 and r1["status"] == 0
        assert r1["E"] == pytest.approx(r0["E"], rel=1e-7)
        assert r1["E0"] == pytest.approx(r0["E0"], rel=1e-6)
        assert r1["arrests"] == r0["arrests"]
        np.testing.assert_allclose(ref.field().cpu().numpy(), st.field().cpu().numpy(),
                                   rtol=0, atol=2e-6)
    b.close()
    # the sextic term is not taken by batches
    lat = sk.Lattice(SHAPES[0], 0.2, 1.0, 32, c6=0.5)
    st = sk.State(lat, DEV)
    with pytest.raises(sk.SkyrmeError) as e:
        sk.Batch([lat], [st], [0.01])
    assert e.value.status == 6


@pytest.mark.parametrize("tile", [0, 4])
def test_batch_tracks_the_oracle_trajectories(tile):
    """Every lattice of a batch of uneven sizes against the FP64 oracle's
    own flow of the same (FP32-rounded) seed: 40 iterations, per site and in
    energy, with the same arrest decisions.  The bounds are those of a single
    FP32 lattice against the oracle (tests/test_gpu_parity.py)."""
    lats, states = make_states()
    seeds = [st.field().double().cpu().numpy() for st in states]
    b = sk.Batch(lats, states, [0.01] * len(lats))
    b.set_tile(tile)
    b.step(40)
    torch.cuda.synchronize()
    for lat, st, phi0 in zip(lats, states, seeds):
        ost = oracle.new_state(phi0)
        oreps = oracle.flow(ost, lat.h, lat.m, 0.01, 40, reports=True)
        rep = sk.read_report(lat, st)
        assert rep["steps"] == 40 and rep["status"] == 0
        assert rep["arrests"] == sum(r["arrested"] for r in oreps)
        assert rep["E"] == pytest.approx(oreps[-1]["E"], rel=1e-5)
        assert rep["B"] == pytest.approx(oreps[-1]["B"], abs=1e-5)
        assert np.max(np.abs(st.field().double().cpu().numpy() - ost.phi)) < 1e-4
    b.close()


@pytest.mark.parametrize("tile", [0, 1, 2, 3, 4])
def test_every_tile_shape_gives_the_same_flow(tile):
    lats, states = make_states(kind="noise")
    ref_lats, refs = make_states(kind="noise")
    b = sk.Batch(lats, states, [0.0075] * len(lats))
    b.set_tile(tile)
    assert b.tile()["tile"] == tile
    b.step(12)
    r = sk.Batch(ref_lats, refs, [0.0075] * len(lats))
    r.step(12)
    torch.cuda.synchronize()
    for lat, a, c in zip(lats, states, refs):
        ra, rc = sk.read_report(lat, a), sk.read_report(lat, c)
        assert ra["E"] == pytest.approx(rc["E"], rel=1e-7)
        np.testing.assert_allclose(a.field().cpu().numpy(), c.field().cpu().numpy(), rtol=0,
                                   atol=2e-6)
    b.close()
    r.close()


@pytest.mark.parametrize("tile", [0, 4])
def test_balanced_and_even_splits_give_the_same_fields(tile):
    """The plane-balanced division of a batch's work among CTAs changes which
    CTA updates a site, not the site's arithmetic: the fields agree bit for
    bit with the even split's, the energies to the rounding of the sums'
    order."""
    lats, states = make_states(kind="noise")
    ref_lats, refs = make_states(kind="noise")
    b = sk.Batch(lats, states, [0.0075] * len(lats))
    b.set_tile(tile)
    b.set_split(True)
    assert b.tile()["balanced"]
    r = sk.Batch(ref_lats, refs, [0.0075] * len(lats))
    r.set_tile(tile)
    r.set_split(False)
    assert not r.tile()["balanced"]
    b.step(12)
    r.step(12)
    torch.cuda.synchronize()
    for lat, a, c in zip(lats, states, refs):
        ra, rc = sk.read_report(lat, a), sk.read_report(lat, c)
        assert ra["arrests"] == rc["arrests"] and ra["status"] == rc["status"] == 0
        assert ra["E"] == pytest.approx(rc["E"], rel=1e-12)
        assert torch.equal(a.field(), c.field())
    b.close()
    r.close()


def test_autotune_is_dry_and_picks_a_tile():
    lats, states = make_states()
    b = sk.Batch(lats, states, [0.01] * len(lats))
    b.step(3)
    torch.cuda.synchronize()
    before = [st.field().clone() for st in states]
    reps = b.reports()
    tile, ms = b.autotune(trials=2)
    assert 0 <= tile < len(sk.TILES) and ms > 0
    torch.cuda.synchronize()
    for st, f, r, lat in zip(states, before, reps, lats):
        assert torch.equal(st.field(), f)
        assert sk.read_report(lat, st)["steps"] == r["steps"] == 3
    b.step(2)
    assert all(r["steps"] == 5 for r in b.reports())
    b.close()


def test_batch_graph_equals_batch_step():
    lats, states = make_states()
    lats2, states2 = make_states()
    b1 = sk.Batch(lats, states, [0.01] * len(lats))
    b2 = sk.Batch(lats2, states2, [0.01] * len(lats))
    b1.step(8)
    g = sk.FlowGraph(nsteps=4, batch=b2)
    g.launch()
    g.launch()
    g.stream.synchronize()
    torch.cuda.synchronize()
    for a, c, la in zip(states, states2, lats):
        assert torch.equal(a.field(), c.field())
        assert sk.read_report(la, a)["E"] == sk.read_report(la, c)["E"]
    g.close()
    b1.close()
    b2.close()


def test_batched_noise_workload_shapes():
    """A slice of the batched workload recipe (uneven sides from the seeded
    draw, smoothed-noise starts) runs and reports finite, decreasing energy."""
    wls = workloads.batched_noise(count=6, steps=40)
    lats, states = [], []
    for w in wls:
        n = tuple(min(v, 80) for v in w.n)
        lat = sk.Lattice(n, w.h, w.m, 32)
        st = sk.State(lat, DEV)
        sk.init_field(lat, sk.Seed.from_spec(w.seed), st)
        lats.append(lat)
        states.append(st)
    e0 = [sk.energy(l, s)["E"] for l, s in zip(lats, states)]
    b = sk.Batch(lats, states, [w.dt for w in wls])
    b.autotune(trials=2)
    b.step(40)
    for r, e in zip(b.reports(), e0):
        assert r["status"] == 0 and np.isfinite(r["E"]) and r["E"] < e
    b.close()


def test_batched_workload_tracks_fp64_flows():
    """Four lattices of the 64-lattice workload at their full sizes, flowed
    200 iterations in one FP32 batch, against each lattice's FP64 flow alone:
    energies and charges agree to 1e-5 relative, arrests are the same."""
    wls = workloads.batched_noise(count=64, steps=200)[:4]
    lats, states = [], []
    for w in wls:
        lat = sk.Lattice(w.n, w.h, w.m, 32)
        st = sk.State(lat, DEV)
        sk.init_field(lat, sk.Seed.from_spec(w.seed), st)
        lats.append(lat)
        states.append(st)
    b = sk.Batch(lats, states, [w.dt for w in wls])
    b.step(200)
    torch.cuda.synchronize()
    for w, lat, st in zip(wls, lats, states):
        r32 = sk.read_report(lat, st)
        l64 = sk.Lattice(w.n, w.h, w.m, 64)
        s64 = sk.State(l64, DEV)
        sk.init_field(l64, sk.Seed.from_spec(w.seed), s64)
        r64 = sk.flow_step(l64, w.dt, 200, sk.ARRESTED, s64)
        assert r32["status"] == 0 and r64["status"] == 0
        assert r32["steps"] == r64["steps"] == 200
        assert r32["E"] == pytest.approx(r64["E"], rel=1e-5), w.n
        assert r32["B"] == pytest.approx(r64["B"], rel=1e-5, abs=1e-6), w.n
        assert r32["arrests"] == r64["arrests"], w.n
    b.close()
