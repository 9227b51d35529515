"""skyrme_flow_host: a whole job on host data (upload, load, flow, download)
through the C ABI gives the same field and report, bit for bit, as the
device-side calls it stands for (skyrme_load_field, skyrme_flow_step and a
read of the current buffers).  The iteration count's parity selects the
result buffers, so odd and even counts are both checked."""
import ctypes

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
sk = pytest.importorskip("paper_2604_25876_gb300")

N, H, M, DT = (20, 21, 22), 0.25, 1.0, 0.0125


def seed_field():
    return oracle.seed_rational_map(N, H, 1, 0.9)


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("nsteps", [7, 8])
def test_host_job_equals_the_device_calls(prec, nsteps):
    dev = torch.device("cuda:0")
    lat = sk.Lattice(N, H, M, prec)
    np_dtype = np.float64 if prec == 64 else np.float32
    field_in = np.ascontiguousarray(seed_field().astype(np_dtype))
    field_out = np.zeros_like(field_in)

    a = sk.State(lat, dev)
    rep_a = sk.flow_host(lat, DT, nsteps, sk.ARRESTED, a, field_in, field_out)

    b = sk.State(lat, dev)
    sk.load_field(lat, b, field_in)
    rep_b = sk.flow_step(lat, DT, nsteps, sk.ARRESTED, b)
    torch.cuda.synchronize()
    ref = b.field().cpu().numpy()

    assert rep_a["steps"] == rep_b["steps"] == nsteps and rep_a["status"] == 0
    assert rep_a["cur"] == nsteps % 2
    assert rep_a["E"] == rep_b["E"] and rep_a["arrests"] == rep_b["arrests"]
    np.testing.assert_array_equal(field_out, ref)


def test_pinned_buffers_and_in_place_output():
    dev = torch.device("cuda:0")
    lat = sk.Lattice(N, H, M, 32)
    seed = torch.from_numpy(seed_field().astype(np.float32))
    buf = torch.empty(seed.shape, dtype=torch.float32, pin_memory=True)
    buf.copy_(seed)
    st = sk.State(lat, dev)
    rep = sk.flow_host(lat, DT, 5, sk.NEWTON, st, buf, buf)
    ref = sk.State(lat, dev)
    sk.load_field(lat, ref, seed)
    sk.flow_step(lat, DT, 5, sk.NEWTON, ref)
    torch.cuda.synchronize()
    assert rep["steps"] == 5
    assert torch.equal(buf, ref.field().cpu())


def test_null_host_buffers_are_rejected():
    dev = torch.device("cuda:0")
    lat = sk.Lattice(N, H, M, 32)
    st = sk.State(lat, dev)
    cl, cs = lat.c(), st.c()
    lib = sk.load()
    field = np.zeros(tuple(N) + (4,), dtype=np.float32)
    for fin, fout in ((None, field.ctypes.data), (field.ctypes.data, None)):
        rc = lib.skyrme_flow_host(ctypes.byref(cl), DT, 3, sk.ARRESTED, ctypes.byref(cs),
                                  ctypes.c_void_p(fin), ctypes.c_void_p(fout), None, None)
        assert rc == 1  # SKYRME_EINVAL
