"""GPU-vs-oracle parity of the CUDA library, called through the C ABI.

Tolerances (normwise, since F and the densities vanish in the vacuum region):
  FP64: forces and densities within 1e-12 of the oracle relative to their
        max-norm (the target of the method), energies 1e-12 relative.
  FP32: each stencil value carries a rounding error of about
        eps32 * sum|w| * |phi| / h^2 (sum|w| = 16/3 for the second derivative,
        eps32 = 6e-8), amplified by at most (1 + tr a) in the force, so the
        normwise force error stays below ~1e-5; energies are FP64 sums of FP32
        densities and agree to ~1e-6 relative.
"""
import math

import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

sk = pytest.importorskip("paper_2604_25876_gb300")

DEV = "cuda:0"


def generic_field(n, h, seed=3, K=3, spread=0.9):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(-spread, spread, size=(K, 3))
    q = rng.normal(size=(K, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return oracle.seed_product(n, h, pos, q, 0.9, True)


def gpu_forces(phi, h, m, prec):
    lat = sk.Lattice(phi.shape[:3], h, m, prec)
    st = sk.State(lat, DEV)
    sk.load_field(lat, st, phi)
    F, D = sk.forces(lat, st)
    torch.cuda.synchronize()
    return F.double().cpu().numpy(), D.double().cpu().numpy(), lat, st


CASES = [
    ("hedgehog_ragged", (21, 26, 37), 0.25, 0.0, lambda n, h: oracle.seed_rational_map(n, h, 1, 1.0)),
    ("b4_cube", (40, 40, 40), 0.2, 1.0, lambda n, h: oracle.seed_rational_map(n, h, 4, 2.0)),
    ("product_generic", (30, 33, 36), 0.2, 1.0, lambda n, h: generic_field(n, h)),
]


@pytest.mark.parametrize("name,n,h,m,make", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("prec,tol", [(64, 1e-12), (32, 1e-5)])
def test_forces_and_densities_match_oracle(name, n, h, m, make, prec, tol):
    phi = make(n, h)
    _, Fo, Do = oracle.forces(phi, h, m)
    Fg, Dg, _, _ = gpu_forces(phi, h, m, prec)
    scale = np.max(np.abs(Fo))
    assert scale > 1.0
    assert np.max(np.abs(Fg - Fo)) <= tol * scale
    for q in range(4):
        s = max(np.max(np.abs(Do[..., q])), 1e-300)
        if s > 1e-10:
            assert np.max(np.abs(Dg[..., q] - Do[..., q])) <= tol * s * 4, q
    # boundary layers carry zeros
    assert not Fg[:2].any() and not Fg[-2:].any() and not Fg[:, :, -2:].any()


@pytest.mark.parametrize("prec,tol", [(64, 1e-12), (32, 2e-6)])
def test_energy_baryon_virial_match_oracle(prec, tol):
    n, h, m = (36, 40, 44), 0.2, 1.0
    phi = oracle.seed_rational_map(n, h, 4, 1.5)
    eo = oracle.energy(phi, h, m)
    lat = sk.Lattice(n, h, m, prec)
    st = sk.State(lat, DEV)
    sk.load_field(lat, st, phi)
    eg = sk.energy(lat, st)
    for k in ("E", "E2", "E4", "E0"):
        assert eg[k] == pytest.approx(eo[k], rel=tol), k
    assert eg["B"] == pytest.approx(eo["B"], rel=tol, abs=tol)
    assert eg["virial"] == pytest.approx(eo["virial"], rel=tol * 10, abs=tol * eo["E"])
    assert sk.baryon_number(lat, st) == eg["B"]
    assert sk.virial(lat, st) == eg["virial"]


def seeds_for(n, h):
    wl = workloads.cluster_seed(5, 1.5, 8)
    return [
        ("rational_map_1", sk.Seed.rational_map(1, 1.0), oracle.seed_rational_map(n, h, 1, 1.0)),
        ("rational_map_2", sk.Seed.rational_map(2, 1.5), oracle.seed_rational_map(n, h, 2, 1.5)),
        ("rational_map_3", sk.Seed.rational_map(3, 1.5), oracle.seed_rational_map(n, h, 3, 1.5)),
        ("rational_map_4", sk.Seed.rational_map(4, 2.0), oracle.seed_rational_map(n, h, 4, 2.0)),
        ("product_sym", sk.Seed.product(wl.positions, wl.quaternions, 1.0, True),
         oracle.seed_product(n, h, wl.positions, wl.quaternions, 1.0, True)),
        ("product_plain", sk.Seed.product(wl.positions, wl.quaternions, 1.0, False),
         oracle.seed_product(n, h, wl.positions, wl.quaternions, 1.0, False)),
        ("noise", sk.Seed.noise(2.0, 0.6, 1001), oracle.seed_noise(n, h, 2.0, 0.6, 1001)),
        ("vacuum", sk.Seed.vacuum(), oracle.seed_vacuum(n)),
    ]


@pytest.mark.parametrize("prec,tol", [(64, 1e-12), (32, 2e-6)])
def test_seed_fields_match_oracle(prec, tol):
    n, h = (28, 31, 33), 0.15
    for name, sd, ref in seeds_for(n, h):
        lat = sk.Lattice(n, h, 1.0, prec)
        st = sk.State(lat, DEV)
        sk.init_field(lat, sd, st)
        torch.cuda.synchronize()
        got = st.field().double().cpu().numpy()
        assert np.max(np.abs(got - ref)) <= tol, name
        assert np.array_equal(st.phi[0].cpu().numpy(), st.phi[1].cpu().numpy()), name
        assert not st.vel.any().item(), name


def run_both(phi, h, m, dt, steps, prec, mode=sk.ARRESTED, chunks=1):
    ost = oracle.new_state(phi)
    oreps = oracle.flow(ost, h, m, dt, steps, mode=mode, reports=True)
    lat = sk.Lattice(phi.shape[:3], h, m, prec)
    st = sk.State(lat, DEV)
    sk.load_field(lat, st, phi)
    per = steps // chunks
    for _ in range(chunks):
        rep = sk.flow_step(lat, dt, per, mode, st)
    torch.cuda.synchronize()
    return ost, oreps, st, rep


@pytest.mark.parametrize("mode", [sk.ARRESTED, sk.NEWTON])
def test_fp64_trajectory_matches_oracle(mode):
    n, h, m = (26, 29, 32), 0.25, 1.0
    phi = oracle.seed_rational_map(n, h, 1, 0.9)
    ost, oreps, st, rep = run_both(phi, h, m, 0.05 * h, 60, 64, mode, chunks=3)
    g = st.field().cpu().numpy()
    assert np.max(np.abs(g - ost.phi)) < 1e-11
    assert np.max(np.abs(st.velocity().cpu().numpy() - ost.v)) < 1e-11
    assert rep["E"] == pytest.approx(oreps[-1]["E"], rel=1e-12)
    assert rep["B"] == pytest.approx(oreps[-1]["B"], rel=1e-12)
    assert rep["delta"] == pytest.approx(oreps[-1]["delta"], rel=1e-11)
    assert rep["steps"] == 60
    assert rep["arrests"] == sum(r["arrested"] for r in oreps)


def mispredictions(seq):
    """Mispredicted arrest decisions of the library's documented predictor:
    the last four decisions index 16 two-bit saturating counters (initially
    1); an arrest is predicted when the selected counter is at least 2.
    Returns (predicted free but arrested, predicted arrested but free)."""
    hist, pht, pred, up, down = 0, [1] * 16, 0, 0, 0
    for a in seq:
        if a != pred:
            up, down = (up + 1, down) if a else (up, down + 1)
        pht[hist] = min(pht[hist] + 1, 3) if a else max(pht[hist] - 1, 0)
        hist = ((hist << 1) | a) & 15
        pred = 1 if pht[hist] >= 2 else 0
    return up, down


def test_fp64_arrest_switching_trajectory_exercises_both_fixups():
    """The massless hedgehog on a coarse lattice switches between arrested and
    free iterations many times in its first 160 steps.  Every switch is a
    misprediction of the speculative update, corrected in one direction or the
    other; the corrected trajectory must still match the oracle."""
    n, h, m, dt = (32, 32, 32), 0.3, 0.0, 0.015
    phi = oracle.seed_rational_map(n, h, 1, 1.0)
    ost, oreps, st, rep = run_both(phi, h, m, dt, 160, 64, chunks=4)
    seq = [r["arrested"] for r in oreps]
    ups, downs = mispredictions(seq)
    assert ups >= 3 and downs >= 1
    assert rep["arrests"] == sum(seq)
    assert rep["fixups"] == ups + downs
    assert np.max(np.abs(st.field().cpu().numpy() - ost.phi)) < 1e-11
    assert np.max(np.abs(st.velocity().cpu().numpy() - ost.v)) < 1e-11
    assert rep["E"] == pytest.approx(oreps[-1]["E"], rel=1e-12)


def test_gradient_flow_matches_oracle():
    n, h, m = (24, 24, 24), 0.25, 1.0
    phi = generic_field(n, h)
    ost, oreps, st, rep = run_both(phi, h, m, 5e-5, 20, 64, sk.GRADIENT)
    assert np.max(np.abs(st.field().cpu().numpy() - ost.phi)) < 1e-12
    assert rep["E"] == pytest.approx(oreps[-1]["E"], rel=1e-12)


def test_fp32_short_trajectory_tracks_fp64_oracle():
    n, h, m = (40, 40, 40), 0.2, 1.0
    phi = oracle.seed_rational_map(n, h, 4, 2.0)
    ost, oreps, st, rep = run_both(phi, h, m, 0.05 * h, 50, 32)
    g = st.field().double().cpu().numpy()
    assert np.max(np.abs(g - ost.phi)) < 1e-4
    assert rep["E"] == pytest.approx(oreps[-1]["E"], rel=1e-5)


def test_vacuum_is_fixed_point_on_gpu():
    for prec in (32, 64):
        lat = sk.Lattice((20, 21, 22), 0.2, 1.0, prec)
        st = sk.State(lat, DEV)
        sk.init_field(lat, sk.Seed.vacuum(), st)
        rep = sk.flow_step(lat, 0.01, 5, sk.ARRESTED, st)
        f = st.field().double().cpu().numpy()
        assert np.all(f[..., 0] == 1.0) and not f[..., 1:].any()
        assert rep["delta"] == 0.0 and abs(rep["E"]) < 1e-20


def test_repeated_runs_are_bitwise_identical():
    for prec in (32, 64):
        out = []
        for _ in range(2):
            lat = sk.Lattice((30, 30, 30), 0.2, 1.0, prec)
            st = sk.State(lat, DEV)
            sk.init_field(lat, sk.Seed.rational_map(4, 1.5), st)
            rep = sk.flow_step(lat, 0.01, 25, sk.ARRESTED, st)
            out.append((st.field().cpu().numpy().copy(), rep["E"]))
        assert np.array_equal(out[0][0], out[1][0]) and out[0][1] == out[1][1]


def test_nonfinite_input_is_reported():
    lat = sk.Lattice((16, 16, 16), 0.25, 1.0, 32)
    st = sk.State(lat, DEV)
    phi = oracle.seed_rational_map((16, 16, 16), 0.25, 1, 1.0)
    phi[8, 8, 8, 1] = np.nan
    sk.load_field(lat, st, phi)
    with pytest.raises(sk.SkyrmeError) as ei:
        sk.flow_step(lat, 0.01, 2, sk.ARRESTED, st)
    assert ei.value.status == 4
    with pytest.raises(sk.SkyrmeError):
        sk.energy(lat, st)


def test_bounded_wait_gives_up_and_the_context_stays_usable():
    """The bounded wait of the step kernels, run out on purpose on an
    mbarrier that nothing completes: the kernel returns after the limit with
    SKYRME_ETIMEOUT recorded, flow calls report it until the state is reset,
    and the device keeps working."""
    import time
    lat = sk.Lattice((20, 20, 20), 0.2, 1.0, 32)
    st = sk.State(lat, DEV)
    sk.init_field(lat, sk.Seed.rational_map(1, 1.0), st)
    t0 = time.perf_counter()
    assert sk.selftest_wait(lat, st, 0.05) == 5
    assert 0.04 < time.perf_counter() - t0 < 5.0
    assert sk.read_report(lat, st)["status"] == 5
    with pytest.raises(sk.SkyrmeError) as ei:
        sk.flow_step(lat, 0.01, 2, sk.ARRESTED, st)
    assert ei.value.status == 5
    sk.init_field(lat, sk.Seed.rational_map(1, 1.0), st)  # resets the control block
    rep = sk.flow_step(lat, 0.01, 2, sk.ARRESTED, st)
    assert rep["status"] == 0 and rep["steps"] == 2 and math.isfinite(rep["E"])


def test_graph_replay_equals_flow_step():
    """A captured graph of K iterations replayed twice reproduces 2K calls of
    skyrme_flow_step bit for bit (the flow state lives on the device)."""
    n, h, m, K = (28, 30, 32), 0.2, 1.0, 7
    for prec in (32, 64):
        lat = sk.Lattice(n, h, m, prec)
        a = sk.State(lat, DEV)
        b = sk.State(lat, DEV)
        for st in (a, b):
            sk.init_field(lat, sk.Seed.rational_map(4, 1.5), st)
        ra = sk.flow_step(lat, 0.01, 2 * K, sk.ARRESTED, a)
        g = sk.FlowGraph(lat, b, 0.01, K, sk.ARRESTED)
        g.launch()
        g.launch()
        g.stream.synchronize()
        rb = sk.read_report(lat, b)
        g.close()
        assert rb["steps"] == 2 * K and rb["E"] == ra["E"]
        assert torch.equal(a.field(), b.field()) and torch.equal(a.velocity(), b.velocity())


@pytest.mark.parametrize("prec", [32, 64])
def test_long_flow_step_call_equals_short_calls(prec):
    """A call of 300 iterations runs as replays of a captured 128-iteration
    graph plus 44 direct iterations; it must reproduce three calls of 100
    (launched directly) bit for bit, in every mode."""
    n, h, m = (28, 30, 32), 0.2, 1.0
    for mode in (sk.ARRESTED, sk.NEWTON, sk.GRADIENT):
        lat = sk.Lattice(n, h, m, prec)
        a, b = sk.State(lat, DEV), sk.State(lat, DEV)
        for st in (a, b):
            sk.init_field(lat, sk.Seed.rational_map(4, 1.5), st)
        ra = sk.flow_step(lat, 0.01, 300, mode, a)
        for _ in range(3):
            rb = sk.flow_step(lat, 0.01, 100, mode, b)
        assert ra["steps"] == rb["steps"] == 300
        assert ra["E"] == rb["E"] and ra["arrests"] == rb["arrests"], mode
        assert torch.equal(a.field(), b.field()) and torch.equal(a.velocity(), b.velocity())


def test_long_flow_step_call_inside_a_user_capture_launches_directly():
    """flow_step on a stream that the caller is capturing (here a torch CUDA
    graph) must not start a capture of its own: its launches go into the
    caller's graph, whose replay then equals the same call made directly."""
    n, h, m = (28, 30, 32), 0.2, 1.0
    lat = sk.Lattice(n, h, m, 32)
    a, b = sk.State(lat, DEV), sk.State(lat, DEV)
    for st in (a, b):
        sk.init_field(lat, sk.Seed.rational_map(4, 1.5), st)
    sk.flow_step(lat, 0.01, 1, sk.ARRESTED, a)
    sk.flow_step(lat, 0.01, 1, sk.ARRESTED, b)
    torch.cuda.synchronize()
    s = torch.cuda.Stream(DEV)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        sk.flow_step(lat, 0.01, 300, sk.ARRESTED, b, report=False, stream=s)
    g.replay()
    torch.cuda.synchronize()
    ra = sk.flow_step(lat, 0.01, 300, sk.ARRESTED, a)
    rb = sk.read_report(lat, b)
    assert rb["steps"] == ra["steps"] == 301 and rb["E"] == ra["E"]
    assert torch.equal(a.field(), b.field())


def load_golden(name):
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)
    rows = []
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = line.split()
            rows.append((int(v[0]), [float(t) for t in v[1:7]], int(v[7])))
    return rows


def test_fp64_b1_hedgehog_48_full_run_matches_stored_oracle_trajectory():
    """The 48^3 FP64 workload for its full 1000 iterations against the FP64
    oracle's trajectory stored by tests/golden/make_golden.py."""
    wl = workloads.b1_hedgehog_48()
    lat = sk.Lattice(wl.n, wl.h, wl.m, 64)
    st = sk.State(lat, DEV)
    sk.init_field(lat, sk.Seed.from_spec(wl.seed), st)
    done = 0
    for k, vals, arrests in load_golden("b1_hedgehog_48_trajectory.txt"):
        rep = sk.flow_step(lat, wl.dt, k + 1 - done, sk.ARRESTED, st)
        done = k + 1
        E, E2, E4, E0, B, delta = vals
        assert rep["E"] == pytest.approx(E, rel=1e-12), k
        assert rep["E2"] == pytest.approx(E2, rel=1e-12) and rep["E4"] == pytest.approx(E4, rel=1e-12)
        assert rep["B"] == pytest.approx(B, rel=1e-12)
        assert rep["delta"] == pytest.approx(delta, rel=1e-9)
        assert rep["arrests"] == arrests, k
    assert done == wl.steps
