"""Host-side checks of the C ABI (no GPU needed): every function declared in
include/skyrme.h is exported by libskyrme.so, and argument validation
rejects bad input before any CUDA call is made."""
import ctypes
import os
import re

import pytest

import paper_2604_25876_gb300 as sk

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for hdr in os.listdir(os.path.join(ROOT, "include")):
        if not hdr.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(skyrme_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    lib = sk.load()
    names = declared_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name
    # and the binding declares a signature for each of them
    assert set(names) <= set(sk._SIGNATURES), set(names) - set(sk._SIGNATURES)


def test_abi_version_and_status_strings():
    lib = sk.load()
    assert lib.skyrme_abi_version() == 5
    assert lib.skyrme_status_string(0) == b"ok"
    assert lib.skyrme_status_string(4) == b"non-finite value detected"


def test_scratch_bytes_and_lattice_validation():
    lib = sk.load()
    good = sk.Lattice((48, 48, 48), 0.2, 0.0, 64).c()
    assert lib.skyrme_scratch_bytes(ctypes.byref(good)) >= 512
    for bad in (sk.Lattice((4, 48, 48), 0.2, 0.0, 64), sk.Lattice((48, 48, 48), 0.0, 0.0, 64),
                sk.Lattice((48, 48, 48), 0.2, -1.0, 64), sk.Lattice((48, 48, 48), 0.2, 0.0, 16)):
        c = bad.c()
        assert lib.skyrme_scratch_bytes(ctypes.byref(c)) == 0


def test_invalid_arguments_are_rejected_without_cuda():
    lib = sk.load()
    lat = sk.Lattice((16, 16, 16), 0.2, 1.0, 32).c()
    # null state
    assert lib.skyrme_flow_step(ctypes.byref(lat), 0.01, 1, 1, None, None, None) == 1
    # misaligned and too-small buffers (fake addresses: never dereferenced)
    st = sk.c_state((ctypes.c_void_p * 2)(0x10000, 0x20000), (ctypes.c_void_p * 2)(0x30000, 0x40008),
                    ctypes.c_void_p(0x50000), ctypes.c_size_t(1 << 30))
    assert lib.skyrme_flow_step(ctypes.byref(lat), 0.01, 1, 1, ctypes.byref(st), None, None) == 1
    st = sk.c_state((ctypes.c_void_p * 2)(0x10000, 0x20000), (ctypes.c_void_p * 2)(0x30000, 0x40000),
                    ctypes.c_void_p(0x50000), ctypes.c_size_t(16))
    assert lib.skyrme_flow_step(ctypes.byref(lat), 0.01, 1, 1, ctypes.byref(st), None, None) == 2
    st = sk.c_state((ctypes.c_void_p * 2)(0x10000, 0x20000), (ctypes.c_void_p * 2)(0x30000, 0x40000),
                    ctypes.c_void_p(0x50000), ctypes.c_size_t(1 << 30))
    # bad dt / mode / nsteps
    assert lib.skyrme_flow_step(ctypes.byref(lat), 0.0, 1, 1, ctypes.byref(st), None, None) == 1
    assert lib.skyrme_flow_step(ctypes.byref(lat), 0.01, 1, 7, ctypes.byref(st), None, None) == 1
    assert lib.skyrme_flow_step(ctypes.byref(lat), 0.01, -1, 1, ctypes.byref(st), None, None) == 1
    # bad seeds
    for seed in (sk.Seed(sk.SEED_RATIONAL_MAP, B=5, profile_scale=1.0),
                 sk.Seed(sk.SEED_RATIONAL_MAP, B=4, profile_scale=0.0),
                 sk.Seed(sk.SEED_PRODUCT, B=2),  # no arrays
                 sk.Seed(sk.SEED_NOISE, radius=3.0, sigma=100.0, seed=1),  # too wide
                 sk.Seed(9)):
        cs, keep = seed.c()
        assert lib.skyrme_init_field(ctypes.byref(lat), ctypes.byref(cs), ctypes.byref(st),
                                     None) == 1


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    monkeypatch.setattr(sk, "_lib", None)
    monkeypatch.setattr(sk._build, "LIB", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        sk.load(build_if_missing=False)


def test_fma_peak_rejects_bad_arguments_without_cuda():
    lib = sk.load()
    out = ctypes.c_double(0.0)
    assert lib.skyrme_measure_fma_peak(7, ctypes.byref(out), None) == 1
    assert lib.skyrme_measure_fma_peak(sk.PEAK_FP32, None, None) == 1


def test_run_to_tolerance_graph_rejects_bad_arguments_without_cuda():
    lib = sk.load()
    lat = sk.Lattice((16, 16, 16), 0.2, 1.0, 32).c()
    st = sk.c_state((ctypes.c_void_p * 2)(0x10000, 0x20000), (ctypes.c_void_p * 2)(0x30000, 0x40000),
                    ctypes.c_void_p(0x50000), ctypes.c_size_t(1 << 30))
    out = ctypes.c_void_p()
    f = lib.skyrme_graph_create_until
    assert f(ctypes.byref(lat), 0.01, 1, 1e-3, 100, 10, ctypes.byref(st), None, None) == 1
    assert f(ctypes.byref(lat), 0.01, 1, -1.0, 100, 10, ctypes.byref(st), None, ctypes.byref(out)) == 1
    assert f(ctypes.byref(lat), 0.01, 1, float("nan"), 100, 10, ctypes.byref(st), None,
             ctypes.byref(out)) == 1
    assert f(ctypes.byref(lat), 0.01, 1, 1e-3, 0, 10, ctypes.byref(st), None, ctypes.byref(out)) == 1
    assert f(ctypes.byref(lat), 0.01, 1, 1e-3, 100, 0, ctypes.byref(st), None, ctypes.byref(out)) == 1
    assert f(ctypes.byref(lat), 0.0, 1, 1e-3, 100, 10, ctypes.byref(st), None, ctypes.byref(out)) == 1
    assert f(ctypes.byref(lat), 0.01, 9, 1e-3, 100, 10, ctypes.byref(st), None, ctypes.byref(out)) == 1
    assert not out.value


def test_observables_rejects_bad_arguments_without_cuda():
    lib = sk.load()
    lat = sk.Lattice((16, 16, 16), 0.2, 1.0, 64).c()
    st = sk.c_state((ctypes.c_void_p * 2)(0x10000, 0x20000), (ctypes.c_void_p * 2)(0x30000, 0x40000),
                    ctypes.c_void_p(0x50000), ctypes.c_size_t(1 << 30))
    assert lib.skyrme_observables(ctypes.byref(lat), ctypes.byref(st), None, None) == 1
    assert lib.skyrme_observables(ctypes.byref(lat), None, ctypes.byref(sk.c_observables()), None) == 1


def test_render_rejects_bad_arguments_without_cuda():
    lib = sk.load()
    lat = sk.Lattice((16, 20, 24), 0.2, 1.0, 32).c()
    assert lib.skyrme_render_volume_bytes(ctypes.byref(lat)) == 16 * 20 * 24 * 32
    bad_lat = sk.Lattice((4, 20, 24), 0.2, 1.0, 32).c()
    assert lib.skyrme_render_volume_bytes(ctypes.byref(bad_lat)) == 0
    st = sk.c_state((ctypes.c_void_p * 2)(0x10000, 0x20000), (ctypes.c_void_p * 2)(0x30000, 0x40000),
                    ctypes.c_void_p(0x50000), ctypes.c_size_t(1 << 30))
    need = 16 * 20 * 24 * 32
    # volume: null, misaligned, too small
    assert lib.skyrme_render_volume(ctypes.byref(lat), ctypes.byref(st), None, need, None) == 1
    assert lib.skyrme_render_volume(ctypes.byref(lat), ctypes.byref(st), ctypes.c_void_p(0x60010),
                                    need, None) == 1
    assert lib.skyrme_render_volume(ctypes.byref(lat), ctypes.byref(st), ctypes.c_void_p(0x60000),
                                    need - 1, None) == 2
    n = (ctypes.c_int * 3)(16, 20, 24)
    vol, rgba = ctypes.c_void_p(0x60000), ctypes.c_void_p(0x70000)
    good = sk.render_params(32, 24)
    rot = sk.render_params(32, 24, view=[[0, 1, 0], [-1, 0, 0], [0, 0, 1]])
    # a valid call would launch kernels: only invalid ones run here
    for p in (sk.render_params(0, 24), sk.render_params(32, -1), sk.render_params(1 << 14, 1 << 13),
              sk.render_params(32, 24, step=0.0), sk.render_params(32, 24, step=1e-5),
              sk.render_params(32, 24, step=2.0), sk.render_params(32, 24, step=float("nan")),
              sk.render_params(32, 24, levelset=float("inf")),
              sk.render_params(32, 24, brightness=float("nan")),
              sk.render_params(32, 24, view=2 * sk.np.eye(3)),
              sk.render_params(32, 24, view=[[1, 0, 0], [0, 1, 0], [0, 1e-6, 1]]),
              sk.render_params(32, 24, view=sk.np.zeros((3, 3)))):
        assert lib.skyrme_render_rays(n, vol, ctypes.byref(p), rgba, None) == 1
        assert lib.skyrme_render(ctypes.byref(lat), ctypes.byref(st), ctypes.byref(p), vol, need,
                                 rgba, None) == 1
    for p in (good, rot):
        assert lib.skyrme_render_rays(None, vol, ctypes.byref(p), rgba, None) == 1
        assert lib.skyrme_render_rays(n, None, ctypes.byref(p), rgba, None) == 1
        assert lib.skyrme_render_rays(n, vol, ctypes.byref(p), None, None) == 1
        assert lib.skyrme_render_rays(n, ctypes.c_void_p(0x60008), ctypes.byref(p), rgba, None) == 1
        assert lib.skyrme_render_rays(n, vol, ctypes.byref(p), ctypes.c_void_p(0x70004), None) == 1
        assert lib.skyrme_render_rays(n, vol, None, rgba, None) == 1
        assert lib.skyrme_render_rays((ctypes.c_int * 3)(1, 20, 24), vol, ctypes.byref(p), rgba,
                                      None) == 1
        assert lib.skyrme_render(ctypes.byref(lat), None, ctypes.byref(p), vol, need, rgba, None) == 1
        assert lib.skyrme_render(ctypes.byref(lat), ctypes.byref(st), ctypes.byref(p), vol, need - 1,
                                 rgba, None) == 2


def test_extension_coefficients_are_validated_and_gated_without_cuda():
    lib = sk.load()
    base = dict(n=(16, 16, 16), h=0.2, m=1.0, precision=32)
    ok = sk.Lattice(**base, m_y=0.5, m_z=0.3, m_w=0.2, c6=0.4)
    assert ok.extended and not sk.Lattice(**base).extended
    c = ok.c()
    assert lib.skyrme_scratch_bytes(ctypes.byref(c)) > 0
    for bad in (dict(m_y=-0.1), dict(m_z=float("nan")), dict(m_w=float("inf")), dict(c6=-1.0)):
        c = sk.Lattice(**base, **bad).c()
        assert lib.skyrme_scratch_bytes(ctypes.byref(c)) == 0, bad
        out = (ctypes.c_double * 6)()
        assert lib.skyrme_energy_static(ctypes.byref(c), ctypes.c_void_p(0x10000), out, None) == 1
    st = sk.c_state((ctypes.c_void_p * 2)(0x10000, 0x20000), (ctypes.c_void_p * 2)(0x30000, 0x40000),
                    ctypes.c_void_p(0x50000), ctypes.c_size_t(1 << 30))
    c = ok.c()
    # Section 5 observables are those of the standard model
    assert lib.skyrme_observables(ctypes.byref(c), ctypes.byref(st),
                                  ctypes.byref(sk.c_observables()), None) == 6
    # batches take the standard model and the potentials, not the sextic term
    lats = (sk.c_lattice * 1)(c)
    sts = (sk.c_state * 1)(st)
    dts = (ctypes.c_double * 1)(0.01)
    out = ctypes.c_void_p()
    need = lib.skyrme_batch_scratch_bytes(1, lats)
    assert lib.skyrme_batch_create(1, lats, sts, dts, 1, ctypes.c_void_p(0x100000), need,
                                   ctypes.byref(out)) == 6
    assert not out.value
    # a null result pointer
    assert lib.skyrme_sextic_energy(ctypes.byref(c), ctypes.byref(st), None, None) == 1


def test_wait_selftest_rejects_bad_arguments_without_cuda():
    lib = sk.load()
    lat = sk.Lattice((16, 16, 16), 0.2, 1.0, 32).c()
    # fake, well-formed device addresses: the checks run before any CUDA call
    st = sk.c_state((ctypes.c_void_p * 2)(0x10000, 0x20000), (ctypes.c_void_p * 2)(0x30000, 0x40000),
                    ctypes.c_void_p(0x50000), ctypes.c_size_t(1 << 30))
    for limit in (0.0, -1.0, 10.5, float("nan"), float("inf")):
        assert lib.skyrme_selftest_wait(ctypes.byref(lat), ctypes.byref(st), limit, None) == 1
    assert lib.skyrme_selftest_wait(ctypes.byref(lat), None, 0.05, None) == 1
    small = sk.c_state((ctypes.c_void_p * 2)(0x10000, 0x20000), (ctypes.c_void_p * 2)(0x30000, 0x40000),
                       ctypes.c_void_p(0x50000), ctypes.c_size_t(16))
    assert lib.skyrme_selftest_wait(ctypes.byref(lat), ctypes.byref(small), 0.05, None) == 2
