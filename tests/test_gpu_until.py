"""Run-to-tolerance graphs (skyrme_graph_create_until): a device-side WHILE
node repeats chunks of iterations until delta = max |F| <= tol or the step
cap is reached.  Checked against the same chunks stepped from the host, and
against the FP64 oracle's own delta history."""
import numpy as np
import pytest

import oracle
import paper_2604_25876_gb300 as sk

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
N, H, M = (30, 30, 30), 0.3, 1.0
DT = 0.05 * H
CHUNK = 25


def seeded_state(prec):
    phi = oracle.seed_rational_map(N, H, 1, 1.0)
    lat = sk.Lattice(N, H, M, prec)
    st = sk.State(lat, DEV)
    sk.load_field(lat, st, phi)
    return phi, lat, st


def host_chunks_until(lat, st, tol, max_steps):
    done = 0
    while True:
        rep = sk.flow_step(lat, DT, CHUNK, sk.ARRESTED, st)
        done += CHUNK
        if rep["delta"] <= tol or done >= max_steps:
            return rep


@pytest.mark.parametrize("prec", [64, 32])
def test_until_graph_matches_host_driven_chunks(prec):
    tol = 0.5
    _, lat, st = seeded_state(prec)
    rep = sk.flow_until(lat, DT, sk.ARRESTED, st, tol, 4000, chunk=CHUNK)
    _, lat2, st2 = seeded_state(prec)
    ref = host_chunks_until(lat2, st2, tol, 4000)
    assert rep["steps"] == ref["steps"]
    assert rep["steps"] % CHUNK == 0 and rep["steps"] < 4000
    assert rep["delta"] <= tol
    assert rep["E"] == ref["E"] and rep["delta"] == ref["delta"]  # the same kernels, bitwise
    assert torch.equal(st.field(), st2.field())


def test_until_graph_stops_at_the_step_cap():
    _, lat, st = seeded_state(64)
    rep = sk.flow_until(lat, DT, sk.ARRESTED, st, 0.0, 110, chunk=CHUNK)
    assert rep["steps"] == 125  # the first chunk boundary at or after 110
    # a second launch of a fresh graph counts from where the first stopped
    rep = sk.flow_until(lat, DT, sk.ARRESTED, st, 0.0, 30, chunk=CHUNK)
    assert rep["steps"] == 175


def test_until_graph_stop_step_follows_the_oracle_delta_history():
    tol = 0.5
    phi, lat, st = seeded_state(64)
    rep = sk.flow_until(lat, DT, sk.ARRESTED, st, tol, 4000, chunk=CHUNK)
    steps = rep["steps"]
    ost = oracle.new_state(phi)
    oreps = oracle.flow(ost, H, M, DT, steps, mode=oracle.ARRESTED, reports=True)
    deltas = np.array([r["delta"] for r in oreps])
    # the oracle's delta at every chunk boundary before the stop is above tol,
    # and at the stop it is at or below tol
    ends = np.arange(CHUNK, steps + 1, CHUNK) - 1
    assert np.all(deltas[ends[:-1]] > tol)
    assert deltas[ends[-1]] <= tol
    assert rep["E"] == pytest.approx(oreps[-1]["E"], rel=1e-11)
