"""skyrme_energy_static, the allocation-free energy reduction, against
skyrme_energy.

Callers that cannot allocate device memory (their memory is owned by a host
application's pool, or they may only use buffers handed to them) use this
entry point: it takes only the field and keeps its scratch in a fixed array
inside the library.  It must give the same six values as skyrme_energy, on
two calls in a row (the array keeps the previous call's contents), and a
repeated call must not change the device's free memory.  This file is
collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
sk = pytest.importorskip("paper_2604_25876_gb300")

pytestmark = pytest.mark.gpu


def call_static(lib, lat, phi_ptr, stream=None):
    cl = lat.c()
    out = (ctypes.c_double * 6)()
    s = torch.cuda.current_stream() if stream is None else stream
    rc = lib.skyrme_energy_static(ctypes.byref(cl), ctypes.c_void_p(phi_ptr), out,
                                  ctypes.c_void_p(s.cuda_stream))
    return rc, list(out)


@pytest.mark.parametrize("prec,tol", [(64, 1e-12), (32, 2e-6)])
def test_static_energy_matches_energy_entry_point(prec, tol):
    lib = sk.load()
    n, h, m = (30, 35, 41), 0.2, 1.0
    lat = sk.Lattice(n, h, m, prec)
    st = sk.State(lat, "cuda:0")
    sk.load_field(lat, st, oracle.seed_rational_map(n, h, 4, 1.5))
    sk.flow_step(lat, 0.01, 3, sk.ARRESTED, st)  # a field that is not a seed
    ref = sk.energy(lat, st)
    phi = st.field()
    keys = ("E", "E2", "E4", "E0", "B", "virial")
    free = []
    for _ in range(2):  # the array keeps the previous call's contents
        rc, got = call_static(lib, lat, phi.data_ptr())
        assert rc == 0
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        for k, v in zip(keys, got):
            assert v == pytest.approx(ref[k], rel=tol, abs=tol * abs(ref["E"])), k
    assert free[0] == free[1]


def test_static_energy_rejects_lattices_beyond_its_array():
    lib = sk.load()
    lat = sk.Lattice((2053, 8, 8), 0.1, 1.0, 32)
    phi = torch.zeros(16, device="cuda:0")
    rc, _ = call_static(lib, lat, phi.data_ptr())
    assert rc == 1  # SKYRME_EINVAL: 2049 interior x-planes > 2048
    rc, _ = call_static(lib, sk.Lattice((20, 20, 20), 0.1, 1.0, 32), phi.data_ptr() + 4)
    assert rc == 1  # misaligned field pointer


def test_static_energy_rejects_a_field_in_host_memory():
    """The kernel runs on the current device, so a field it cannot address is
    refused before any launch, and the next call works as before."""
    lib = sk.load()
    n = (20, 20, 20)
    lat = sk.Lattice(n, 0.1, 1.0, 32)
    host = np.zeros(n + (4,), dtype=np.float32)
    rc, _ = call_static(lib, lat, host.ctypes.data)
    assert rc == 1  # SKYRME_EINVAL
    phi = torch.zeros(n + (4,), dtype=torch.float32, device="cuda:0")
    phi[..., 0] = 1.0
    rc, got = call_static(lib, lat, phi.data_ptr())
    assert rc == 0 and got[0] == 0.0
