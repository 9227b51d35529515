"""The single-lattice FP32 step under both work splits: every site's
arithmetic is the same whichever CTA streams it, so the lockstep schedule and
the balanced split give the same field and velocity bit for bit, the same
arrest decisions and corrections (the step's own correction walks the CTA's
runs with the same decode), and energies equal up to the FP64 rounding of the
sums' order (Section 3's iteration; the split is not the paper's)."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

sk = pytest.importorskip("paper_2604_25876_gb300")

DEV = "cuda:0"


def flow(n, h, m, dt, nsteps, policy, phi, **model):
    sk.set_single_split(policy)
    try:
        lat = sk.Lattice(n, h, m, 32, **model)
        st = sk.State(lat, torch.device(DEV))
        sk.load_field(lat, st, phi)
        rep = sk.flow_step(lat, dt, nsteps, sk.ARRESTED, st)
        torch.cuda.synchronize()
        return st.field().cpu().numpy(), st.velocity().cpu().numpy(), rep
    finally:
        sk.set_single_split(sk.SPLIT_AUTO)


@pytest.mark.parametrize("n,h,m,dt,nsteps,need_fix", [
    # one wave of columns at most: heads beside tails; the massless hedgehog
    # on a coarse lattice switches between arrested and free iterations, so
    # the step corrects its own mispredictions
    ((32, 68, 100), 0.3, 0.0, 0.015, 160, True),
    # more columns than CTAs: a wave of whole columns, then heads and tails
    ((20, 324, 260), 0.1, 1.0, 0.004, 12, False),
])
def test_lockstep_and_balanced_splits_agree(n, h, m, dt, nsteps, need_fix):
    phi = oracle.seed_rational_map(n, h, 1, 1.0).astype(np.float32)
    runs, chosen = sk.single_split_runs(n, 152, sk.SPLIT_LOCKSTEP)
    assert chosen == sk.SPLIT_LOCKSTEP
    fa, va, ra = flow(n, h, m, dt, nsteps, sk.SPLIT_LOCKSTEP, phi)
    fb, vb, rb = flow(n, h, m, dt, nsteps, sk.SPLIT_BALANCED, phi)
    assert ra["status"] == 0 and rb["status"] == 0 and ra["steps"] == nsteps
    np.testing.assert_array_equal(fa, fb)
    np.testing.assert_array_equal(va, vb)
    assert ra["arrests"] == rb["arrests"] and ra["fixups"] == rb["fixups"]
    if need_fix:
        assert ra["fixups"] > 0
    assert ra["E"] == pytest.approx(rb["E"], rel=1e-13)
    assert ra["B"] == pytest.approx(rb["B"], rel=1e-12, abs=1e-13)


@pytest.mark.parametrize("model", [{"m_w": 1.0}, {"c6": 1.0}], ids=["potentials", "sextic"])
def test_splits_agree_for_the_extension_variants(model):
    """The potentials and sextic instantiations of the step share the run
    decode; a wave of whole columns, then heads and tails."""
    n, h, m, dt, nsteps = (20, 324, 260), 0.1, 1.0, 0.004, 8
    phi = oracle.seed_rational_map(n, h, 1, 1.0).astype(np.float32)
    fa, va, ra = flow(n, h, m, dt, nsteps, sk.SPLIT_LOCKSTEP, phi, **model)
    fb, vb, rb = flow(n, h, m, dt, nsteps, sk.SPLIT_BALANCED, phi, **model)
    assert ra["status"] == 0 and rb["status"] == 0 and ra["steps"] == nsteps
    np.testing.assert_array_equal(fa, fb)
    np.testing.assert_array_equal(va, vb)
    assert ra["arrests"] == rb["arrests"]
    assert ra["E"] == pytest.approx(rb["E"], rel=1e-13)
