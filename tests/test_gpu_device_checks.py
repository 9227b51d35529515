"""Every entry point works on the current CUDA device and refuses buffers
that the device cannot address (another GPU's, or plain host memory) with
SKYRME_EINVAL, after the other argument checks and before any launch.  On a
one-GPU machine the host-memory case is the one that can be exercised; the check
is the same pointer query for both."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
sk = pytest.importorskip("paper_2604_25876_gb300")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def test_host_memory_buffers_are_rejected_before_any_launch():
    lib = sk.load()
    lat = sk.Lattice((16, 16, 16), 0.2, 1.0, 32)
    st = sk.State(lat, DEV)
    sk.init_field(lat, sk.Seed.rational_map(1, 1.0), st)
    good = st.c()
    host = np.zeros(lat.scratch_bytes() // 4 + 64, dtype=np.float32)
    hp = (host.ctypes.data + 255) // 256 * 256
    for field in ("phi", "vel"):
        cs = st.c()
        arr = getattr(cs, field)
        arr[1] = hp
        rep = sk.c_report()
        rc = lib.skyrme_flow_step(ctypes.byref(lat.c()), 0.01, 1, sk.ARRESTED, ctypes.byref(cs),
                                  ctypes.byref(rep), ctypes.c_void_p(0))
        assert rc == 1, field
    cs = st.c()
    cs.scratch = ctypes.c_void_p(hp)
    out = (ctypes.c_double * 6)()
    assert lib.skyrme_energy(ctypes.byref(lat.c()), ctypes.byref(cs), out, ctypes.c_void_p(0)) == 1
    # nothing was launched: the state flows as before
    rep = sk.flow_step(lat, 0.01, 2, sk.ARRESTED, st)
    assert rep["steps"] == 2 and rep["status"] == 0
    assert lib.skyrme_energy(ctypes.byref(lat.c()), ctypes.byref(good), out, ctypes.c_void_p(0)) == 0
