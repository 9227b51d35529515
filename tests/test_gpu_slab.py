"""x-slab decomposition on one GPU: a lattice cut into slabs, each held by its
own state, with the records combined and the halos copied on the device
(LocalSlabFlow), must reproduce the whole-lattice flow.

The per-site arithmetic of the slab steps is that of the whole-lattice
kernels, so as long as every arrest decision agrees the fields are equal bit
for bit; the energies differ only by summation order.  The slab path is also
compared with the oracle directly."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
sk = pytest.importorskip("paper_2604_25876_gb300")
from paper_2604_25876_gb300.slab import LocalSlabFlow  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def seed(n, h):
    # an off-centre B=1 Skyrmion: its flow arrests once, at iteration 10, on
    # these lattices at dt = 0.05 h (so both branches of the arrest rule run)
    phi = oracle.rational_map_field(n, h, 1, 1.0, X=(0.6, -0.3, 0.2))
    return oracle.apply_vacuum_boundary(np.ascontiguousarray(phi))


def whole_flow(lat, phi0, dt, steps, mode):
    st = sk.State(lat, DEV)
    sk.load_field(lat, st, phi0)
    rep = sk.flow_step(lat, dt, steps, mode, st)
    return st.field().clone(), rep


def slab_flow(lat, phi0, dt, steps, mode, nslabs):
    f = LocalSlabFlow(lat, nslabs, DEV)
    f.load(torch.as_tensor(phi0, dtype=lat.dtype, device=DEV))
    f.flow(dt, steps, mode)
    out = torch.as_tensor(phi0, dtype=lat.dtype, device=DEV).clone()
    f.whole_field(out)
    reps = [s.st.report() for s in f.slabs]
    return out, reps


H = 0.25
CASES = [
    # precision, lattice, slabs, mode, dt
    (64, (26, 20, 22), 2, sk.ARRESTED, 0.05 * H),
    (64, (27, 20, 22), 3, sk.ARRESTED, 0.05 * H),
    (64, (28, 22, 24), 2, sk.NEWTON, 0.05 * H),
    (32, (26, 20, 22), 2, sk.ARRESTED, 0.05 * H),   # FP32 streaming kernel
    (32, (28, 22, 24), 3, sk.ARRESTED, 0.05 * H),
    (32, (27, 20, 22), 3, sk.GRADIENT, 0.0005),      # first order: a stable step is ~h^2 / 100
]


@pytest.mark.parametrize("prec,n,nslabs,mode,dt", CASES)
def test_slabs_reproduce_the_whole_lattice_flow(prec, n, nslabs, mode, dt):
    m, steps = 1.0, 40
    lat = sk.Lattice(n, H, m, prec)
    phi0 = seed(n, H)
    ref, rep = whole_flow(lat, phi0, dt, steps, mode)
    got, reps = slab_flow(lat, phi0, dt, steps, mode, nslabs)
    # the per-site arithmetic is the whole lattice's: bit for bit
    assert torch.equal(got, ref)
    if mode == sk.ARRESTED:
        assert rep["arrests"] == 1  # the arrest branch ran once (iteration 10)
    for r in reps:
        # every slab made the whole lattice's decisions and reports its
        # energies (to summation order)
        assert r["steps"] == steps and r["status"] == 0
        assert r["arrests"] == rep["arrests"] and r["fixups"] == rep["fixups"]
        for k in ("E", "E2", "E4", "E0"):
            assert r[k] == pytest.approx(rep[k], rel=1e-12), k
        assert r["virial"] == pytest.approx(rep["virial"], abs=1e-12 * rep["E"])
        assert r["B"] == pytest.approx(rep["B"], abs=1e-12)
        assert r["delta"] == rep["delta"]


def test_fp64_slab_flow_matches_the_oracle():
    n, h, m = (27, 20, 22), H, 1.0
    dt, steps = 0.05 * h, 40
    lat = sk.Lattice(n, h, m, 64)
    phi0 = seed(n, h)
    got, reps = slab_flow(lat, phi0, dt, steps, sk.ARRESTED, 2)
    st = oracle.new_state(phi0)
    oreps = oracle.flow(st, h, m, dt, steps, reports=True)
    np.testing.assert_allclose(got.cpu().numpy(), st.phi, rtol=0, atol=1e-11)
    assert reps[0]["E"] == pytest.approx(oreps[-1]["E"], rel=1e-11)
    assert reps[0]["arrests"] == sum(r["arrested"] for r in oreps)


def test_slabs_of_an_extended_model():
    """A potential and the sextic term (the streaming kernel's sextic
    variant in FP32): the slab records carry the sextic sum."""
    n, h = (26, 20, 22), H
    lat = sk.Lattice(n, h, 1.0, 32, m_w=0.5, c6=1.0)
    phi0 = seed(n, h)
    ref, rep = whole_flow(lat, phi0, 0.05 * h, 30, sk.ARRESTED)
    got, reps = slab_flow(lat, phi0, 0.05 * h, 30, sk.ARRESTED, 2)
    assert torch.equal(got, ref)
    assert reps[0]["arrests"] == rep["arrests"]
    assert reps[0]["E6"] == pytest.approx(rep["E6"], rel=1e-12)
