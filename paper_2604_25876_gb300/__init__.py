"""GB300 arrested-Newton-flow library for the 3D Skyrme model (arXiv 2604.25876).

Thin ctypes binding over the C ABI of ``include/skyrme.h``.  Every step of the
flow runs in the library's sm_103a CUDA kernels; this module only marshals
arguments.  PyTorch provides device memory and streams.  There is no CPU
fallback: if ``libskyrme.so`` cannot be loaded (or built with nvcc), importing
the kernels raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

from . import _build

NEWTON, ARRESTED, GRADIENT = 0, 1, 2
SPLIT_AUTO, SPLIT_BALANCED, SPLIT_LOCKSTEP = 0, 1, 2
SEED_VACUUM, SEED_RATIONAL_MAP, SEED_PRODUCT, SEED_NOISE = 0, 1, 2, 3

STATUS = {0: "ok", 1: "invalid argument", 2: "buffer too small", 3: "CUDA error",
          4: "non-finite value", 5: "device wait timed out", 6: "unsupported"}


class c_observables(ctypes.Structure):
    _fields_ = [("B", ctypes.c_double), ("X", ctypes.c_double * 3), ("R", ctypes.c_double),
                ("Q", ctypes.c_double * 9), ("U", ctypes.c_double * 9), ("V", ctypes.c_double * 9),
                ("W", ctypes.c_double * 9), ("D", ctypes.c_double), ("E", ctypes.c_double)]


class c_render_params(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int), ("height", ctypes.c_int), ("view", ctypes.c_double * 9),
                ("levelset", ctypes.c_double), ("transfer_scale", ctypes.c_double),
                ("brightness", ctypes.c_double), ("step", ctypes.c_double)]


class SkyrmeError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        msg = f"{where}: {STATUS.get(status, status)}"
        if detail:
            msg += f" ({detail})"
        super().__init__(msg)


class c_lattice(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("h", ctypes.c_double), ("m", ctypes.c_double),
                ("precision", ctypes.c_int), ("m_y", ctypes.c_double), ("m_z", ctypes.c_double),
                ("m_w", ctypes.c_double), ("c6", ctypes.c_double)]


class c_seed(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("B", ctypes.c_int), ("profile_scale", ctypes.c_double),
                ("positions", ctypes.POINTER(ctypes.c_double)),
                ("quaternions", ctypes.POINTER(ctypes.c_double)),
                ("symmetrise", ctypes.c_int), ("radius", ctypes.c_double),
                ("sigma", ctypes.c_double), ("seed", ctypes.c_uint64)]


class c_state(ctypes.Structure):
    _fields_ = [("phi", ctypes.c_void_p * 2), ("vel", ctypes.c_void_p * 2),
                ("scratch", ctypes.c_void_p), ("scratch_bytes", ctypes.c_size_t)]


class c_report(ctypes.Structure):
    _fields_ = [("E", ctypes.c_double), ("E2", ctypes.c_double), ("E4", ctypes.c_double),
                ("E0", ctypes.c_double), ("B", ctypes.c_double), ("virial", ctypes.c_double),
                ("delta", ctypes.c_double), ("rms_force", ctypes.c_double),
                ("steps", ctypes.c_longlong), ("arrests", ctypes.c_longlong),
                ("fixups", ctypes.c_longlong), ("cur", ctypes.c_int), ("status", ctypes.c_int),
                ("E6", ctypes.c_double)]


# Exported symbols with their ctypes signatures (also checked by the ABI tests).
_P = ctypes.c_void_p
_SIGNATURES = {
    "skyrme_abi_version": (ctypes.c_int, []),
    "skyrme_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "skyrme_last_cuda_error": (ctypes.c_char_p, []),
    "skyrme_scratch_bytes": (ctypes.c_size_t, [ctypes.POINTER(c_lattice)]),
    "skyrme_init_field": (ctypes.c_int, [ctypes.POINTER(c_lattice), ctypes.POINTER(c_seed),
                                         ctypes.POINTER(c_state), _P]),
    "skyrme_load_field": (ctypes.c_int, [ctypes.POINTER(c_lattice), ctypes.POINTER(c_state), _P]),
    "skyrme_flow_step": (ctypes.c_int, [ctypes.POINTER(c_lattice), ctypes.c_double, ctypes.c_int,
                                        ctypes.c_int, ctypes.POINTER(c_state),
                                        ctypes.POINTER(c_report), _P]),
    "skyrme_read_report": (ctypes.c_int, [ctypes.POINTER(c_lattice), ctypes.POINTER(c_state),
                                          ctypes.POINTER(c_report), _P]),
    "skyrme_energy": (ctypes.c_int, [ctypes.POINTER(c_lattice), ctypes.POINTER(c_state),
                                     ctypes.POINTER(ctypes.c_double), _P]),
    "skyrme_baryon_number": (ctypes.c_int, [ctypes.POINTER(c_lattice), ctypes.POINTER(c_state),
                                            ctypes.POINTER(ctypes.c_double), _P]),
    "skyrme_virial": (ctypes.c_int, [ctypes.POINTER(c_lattice), ctypes.POINTER(c_state),
                                     ctypes.POINTER(ctypes.c_double), _P]),
    "skyrme_sextic_energy": (ctypes.c_int, [ctypes.POINTER(c_lattice), ctypes.POINTER(c_state),
                                            ctypes.POINTER(ctypes.c_double), _P]),
    "skyrme_forces": (ctypes.c_int, [ctypes.POINTER(c_lattice), ctypes.POINTER(c_state), _P, _P,
                                     _P]),
    "skyrme_energy_static": (ctypes.c_int, [ctypes.POINTER(c_lattice), _P,
                                            ctypes.POINTER(ctypes.c_double), _P]),
    "skyrme_measure_fma_peak": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double), _P]),
    "skyrme_observables": (ctypes.c_int, [ctypes.POINTER(c_lattice), ctypes.POINTER(c_state),
                                          ctypes.POINTER(c_observables), _P]),
    "skyrme_render_volume_bytes": (ctypes.c_size_t, [ctypes.POINTER(c_lattice)]),
    "skyrme_render_volume": (ctypes.c_int, [ctypes.POINTER(c_lattice), ctypes.POINTER(c_state), _P,
                                            ctypes.c_size_t, _P]),
    "skyrme_render_rays": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int), _P,
                                          ctypes.POINTER(c_render_params), _P, _P]),
    "skyrme_render": (ctypes.c_int, [ctypes.POINTER(c_lattice), ctypes.POINTER(c_state),
                                     ctypes.POINTER(c_render_params), _P, ctypes.c_size_t, _P, _P]),
    "skyrme_graph_create_until": (ctypes.c_int, [ctypes.POINTER(c_lattice), ctypes.c_double,
                                                 ctypes.c_int, ctypes.c_double, ctypes.c_longlong,
                                                 ctypes.c_int, ctypes.POINTER(c_state), _P,
                                                 ctypes.POINTER(ctypes.c_void_p)]),
    "skyrme_batch_scratch_bytes": (ctypes.c_size_t, [ctypes.c_int, ctypes.POINTER(c_lattice)]),
    "skyrme_batch_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(c_lattice),
                                           ctypes.POINTER(c_state), ctypes.POINTER(ctypes.c_double),
                                           ctypes.c_int, _P, ctypes.c_size_t,
                                           ctypes.POINTER(ctypes.c_void_p)]),
    "skyrme_batch_step": (ctypes.c_int, [_P, ctypes.c_int, _P]),
    "skyrme_batch_autotune": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.POINTER(ctypes.c_int),
                                             ctypes.POINTER(ctypes.c_double)]),
    "skyrme_flow_host": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_int, ctypes.c_int, _P, _P, _P,
                                         _P, _P]),
    "skyrme_batch_set_tile": (ctypes.c_int, [_P, ctypes.c_int]),
    "skyrme_batch_set_split": (ctypes.c_int, [_P, ctypes.c_int]),
    "skyrme_batch_split": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int)]),
    "skyrme_set_single_split": (ctypes.c_int, [ctypes.c_int]),
    "skyrme_single_split": (ctypes.c_int, []),
    "skyrme_single_split_runs": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                                ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                                ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "skyrme_batch_tile": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_int)]),
    "skyrme_batch_graph_create": (ctypes.c_int, [_P, ctypes.c_int, _P,
                                                 ctypes.POINTER(ctypes.c_void_p)]),
    "skyrme_batch_destroy": (ctypes.c_int, [_P]),
    "skyrme_graph_create": (ctypes.c_int, [ctypes.POINTER(c_lattice), ctypes.c_double,
                                           ctypes.c_int, ctypes.c_int, ctypes.POINTER(c_state), _P,
                                           ctypes.POINTER(ctypes.c_void_p)]),
    "skyrme_selftest_wait": (ctypes.c_int, [ctypes.POINTER(c_lattice), ctypes.POINTER(c_state),
                                            ctypes.c_double, _P]),
    "skyrme_graph_launch": (ctypes.c_int, [_P, _P]),
    "skyrme_graph_destroy": (ctypes.c_int, [_P]),
    "skyrme_slab_step": (ctypes.c_int, [ctypes.POINTER(c_lattice), ctypes.c_double, ctypes.c_int,
                                        ctypes.POINTER(c_state), _P, _P]),
    "skyrme_slab_finish": (ctypes.c_int, [ctypes.POINTER(c_lattice), ctypes.c_double,
                                          ctypes.c_int, ctypes.POINTER(c_state), _P,
                                          ctypes.c_int, _P]),
    "skyrme_step_densities": (ctypes.c_int, [ctypes.POINTER(c_lattice), ctypes.c_double,
                                             ctypes.c_int, ctypes.POINTER(c_state), _P,
                                             ctypes.POINTER(c_report), _P]),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libskyrme.so (building it with nvcc when absent or stale)."""
    global _lib
    if _lib is None:
        path = _build.build() if build_if_missing else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is missing; run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(rc: int, where: str):
    if rc != 0:
        detail = load().skyrme_last_cuda_error().decode() if rc == 3 else ""
        raise SkyrmeError(rc, where, detail)


def _torch():
    import torch
    return torch


class _On:
    """The library's functions, each called with ``device`` as the current
    CUDA device: the C entry points run on the current device and reject
    buffers of another one."""

    def __init__(self, device):
        self.device = device

    def __getattr__(self, name):
        fn = getattr(load(), name)
        dev = self.device

        def call(*args):
            with _torch().cuda.device(dev):
                return fn(*args)
        return call


def _on(device) -> _On:
    return _On(device)


def _stream_ptr(stream=None, device=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream(device)
    return ctypes.c_void_p(s.cuda_stream)


# --------------------------------------------------------------- lattice
@dataclass
class Lattice:
    """Lattice and model: n sites per axis, spacing h, pion mass m, precision
    32 or 64, and the Section 7.8 extension coefficients m_y (modified pion
    mass), m_z (loosely bound), m_w (lightly bound) and c6 (sextic term)."""
    n: Sequence[int]
    h: float
    m: float = 0.0
    precision: int = 32
    m_y: float = 0.0
    m_z: float = 0.0
    m_w: float = 0.0
    c6: float = 0.0

    def c(self) -> c_lattice:
        return c_lattice((ctypes.c_int * 3)(*[int(v) for v in self.n]), float(self.h),
                         float(self.m), int(self.precision), float(self.m_y), float(self.m_z),
                         float(self.m_w), float(self.c6))

    @property
    def extended(self) -> bool:
        return any(v != 0.0 for v in (self.m_y, self.m_z, self.m_w, self.c6))

    @property
    def dtype(self):
        torch = _torch()
        return torch.float64 if self.precision == 64 else torch.float32

    @property
    def interior_sites(self) -> int:
        return int(np.prod([int(v) - 4 for v in self.n]))

    def scratch_bytes(self) -> int:
        c = self.c()
        return int(load().skyrme_scratch_bytes(ctypes.byref(c)))


@dataclass
class Seed:
    kind: int
    B: int = 1
    profile_scale: float = 1.0
    positions: Optional[np.ndarray] = None
    quaternions: Optional[np.ndarray] = None
    symmetrise: bool = True
    radius: float = 0.0
    sigma: float = 0.0
    seed: int = 0

    @staticmethod
    def vacuum():
        return Seed(SEED_VACUUM)

    @staticmethod
    def rational_map(B: int, profile_scale: float):
        return Seed(SEED_RATIONAL_MAP, B=B, profile_scale=profile_scale)

    @staticmethod
    def product(positions, quaternions, profile_scale: float = 1.0, symmetrise: bool = True):
        pos = np.ascontiguousarray(positions, dtype=np.float64).reshape(-1, 3)
        q = np.ascontiguousarray(quaternions, dtype=np.float64).reshape(-1, 4)
        return Seed(SEED_PRODUCT, B=len(pos), profile_scale=profile_scale, positions=pos,
                    quaternions=q, symmetrise=symmetrise)

    @staticmethod
    def noise(radius: float, sigma: float, seed: int):
        return Seed(SEED_NOISE, radius=radius, sigma=sigma, seed=seed)

    @staticmethod
    def from_spec(spec):
        """Seed from a ``workloads.SeedSpec``."""
        if spec.kind == "rational_map":
            return Seed.rational_map(spec.B, spec.profile_scale)
        if spec.kind == "product":
            return Seed.product(spec.positions, spec.quaternions, spec.profile_scale,
                                spec.symmetrise)
        if spec.kind == "noise":
            return Seed.noise(spec.ball_radius, spec.sigma, spec.seed)
        if spec.kind == "vacuum":
            return Seed.vacuum()
        raise ValueError(spec.kind)

    def c(self):
        pos = self.positions
        q = self.quaternions
        dp = ctypes.POINTER(ctypes.c_double)
        s = c_seed(self.kind, int(self.B), float(self.profile_scale),
                   pos.ctypes.data_as(dp) if pos is not None else dp(),
                   q.ctypes.data_as(dp) if q is not None else dp(),
                   int(bool(self.symmetrise)), float(self.radius), float(self.sigma),
                   int(self.seed) & 0xFFFFFFFFFFFFFFFF)
        return s, (pos, q)  # keep host arrays alive during the call


class State:
    """Device buffers of one lattice: two field and two velocity buffers
    (torch tensors of shape (2, Nx, Ny, Nz, 4)) and the scratch block."""

    def __init__(self, lat: Lattice, device="cuda"):
        torch = _torch()
        self.lat = lat
        self.device = torch.device(device)
        shape = (2,) + tuple(int(v) for v in lat.n) + (4,)
        self.phi = torch.empty(shape, dtype=lat.dtype, device=self.device)
        self.vel = torch.zeros(shape, dtype=lat.dtype, device=self.device)
        self.scratch = torch.zeros(lat.scratch_bytes(), dtype=torch.uint8, device=self.device)

    def c(self) -> c_state:
        return c_state((ctypes.c_void_p * 2)(self.phi[0].data_ptr(), self.phi[1].data_ptr()),
                       (ctypes.c_void_p * 2)(self.vel[0].data_ptr(), self.vel[1].data_ptr()),
                       ctypes.c_void_p(self.scratch.data_ptr()),
                       ctypes.c_size_t(self.scratch.numel()))

    def report(self, stream=None) -> dict:
        return read_report(self.lat, self, stream)

    def field(self, stream=None):
        """Tensor view of the buffer that holds the current field."""
        return self.phi[self.report(stream)["cur"]]

    def velocity(self, stream=None):
        return self.vel[self.report(stream)["cur"]]


def _rep_dict(r: c_report) -> dict:
    return {k: getattr(r, k) for k, _ in c_report._fields_}


def init_field(lat: Lattice, seed: Seed, st: State, stream=None):
    cl, cs = lat.c(), st.c()
    sd, keep = seed.c()
    _check(_on(st.device).skyrme_init_field(ctypes.byref(cl), ctypes.byref(sd), ctypes.byref(cs),
                                    _stream_ptr(stream, st.device)), "skyrme_init_field")
    del keep


def load_field(lat: Lattice, st: State, phi, stream=None):
    """Start a flow from a given field (any device/host tensor or array of
    shape (Nx, Ny, Nz, 4)); its outer layers are replaced by the vacuum."""
    torch = _torch()
    t = torch.as_tensor(np.asarray(phi) if not isinstance(phi, torch.Tensor) else phi)
    st.phi[0].copy_(t.to(device=st.device, dtype=lat.dtype))
    cl, cs = lat.c(), st.c()
    _check(_on(st.device).skyrme_load_field(ctypes.byref(cl), ctypes.byref(cs),
                                    _stream_ptr(stream, st.device)), "skyrme_load_field")


def flow_step(lat: Lattice, dt: float, nsteps: int, mode: int, st: State, report: bool = True,
              stream=None):
    cl, cs = lat.c(), st.c()
    rep = c_report()
    rc = _on(st.device).skyrme_flow_step(ctypes.byref(cl), float(dt), int(nsteps), int(mode),
                                 ctypes.byref(cs), ctypes.byref(rep) if report else None,
                                 _stream_ptr(stream, st.device))
    _check(rc, "skyrme_flow_step")
    return _rep_dict(rep) if report else None


def _host_ptr(buf, nbytes: int, writable: bool):
    """Address of a host buffer (a CPU torch tensor or a NumPy array) of at
    least nbytes contiguous bytes."""
    torch = _torch()
    if isinstance(buf, torch.Tensor):
        if buf.is_cuda or not buf.is_contiguous():
            raise ValueError("host buffers must be contiguous CPU tensors")
        size, ptr = buf.numel() * buf.element_size(), buf.data_ptr()
    else:
        import numpy as np
        if not isinstance(buf, np.ndarray) or not buf.flags["C_CONTIGUOUS"]:
            raise ValueError("host buffers must be contiguous NumPy arrays or CPU tensors")
        if writable and not buf.flags["WRITEABLE"]:
            raise ValueError("the output buffer is read-only")
        size, ptr = buf.nbytes, buf.ctypes.data
    if size < nbytes:
        raise ValueError(f"host buffer of {size} bytes, {nbytes} needed")
    return ctypes.c_void_p(ptr)


def flow_host(lat: Lattice, dt: float, nsteps: int, mode: int, st: State, field_in, field_out,
              report: bool = True, stream=None):
    """skyrme_flow_host: upload the host field `field_in` into the state, run
    nsteps iterations, download the final field into `field_out` (host; may
    be field_in), all on `stream`, which the call synchronises."""
    nbytes = int(np.prod(lat.n)) * 4 * (8 if lat.precision == 64 else 4)
    cl, cs = lat.c(), st.c()
    rep = c_report()
    rc = _on(st.device).skyrme_flow_host(ctypes.byref(cl), float(dt), int(nsteps), int(mode),
                                         ctypes.byref(cs), _host_ptr(field_in, nbytes, False),
                                         _host_ptr(field_out, nbytes, True),
                                         ctypes.byref(rep) if report else None,
                                         _stream_ptr(stream, st.device))
    _check(rc, "skyrme_flow_host")
    return _rep_dict(rep) if report else None


def set_single_split(policy: int):
    """skyrme_set_single_split: the process-wide work split of single FP32
    lattices (SPLIT_AUTO, SPLIT_BALANCED or SPLIT_LOCKSTEP)."""
    _check(load().skyrme_set_single_split(int(policy)), "skyrme_set_single_split")


def single_split() -> int:
    """skyrme_single_split: the policy in force."""
    return int(load().skyrme_single_split())


def single_split_runs(n, grid: int = 152, policy: int = SPLIT_AUTO):
    """skyrme_single_split_runs (host only): the runs `policy` gives an
    n[0] x n[1] x n[2] lattice on `grid` CTAs, as an int array of rows
    (CTA, column, first plane, end plane), and the split taken."""
    nn = (ctypes.c_int * 3)(*[int(v) for v in n])
    chosen = ctypes.c_int(-1)
    lib = load()
    count = lib.skyrme_single_split_runs(nn, int(grid), int(policy), None, 0, ctypes.byref(chosen))
    if count < 0:
        raise ValueError(f"no split for n={tuple(n)}, grid={grid}, policy={policy}")
    buf = (ctypes.c_int * max(1, 4 * count))()
    got = lib.skyrme_single_split_runs(nn, int(grid), int(policy), buf, count, ctypes.byref(chosen))
    assert got == count
    return np.frombuffer(buf, dtype=np.int32)[:4 * count].reshape(count, 4).copy(), chosen.value


def step_densities(lat: Lattice, dt: float, mode: int, st: State, stream=None):
    """One iteration of an FP32 streaming-kernel flow (skyrme_step_densities)
    that also returns, as a float32 device tensor (Nx, Ny, Nz, 4), the
    per-site values {e2, e4, u, det} its energy and charge sums added up
    (interior sites; the rest is zero), with the iteration's report."""
    torch = _torch()
    dens = torch.zeros(tuple(int(v) for v in lat.n) + (4,), dtype=torch.float32,
                       device=st.device)
    cl, cs = lat.c(), st.c()
    rep = c_report()
    _check(_on(st.device).skyrme_step_densities(ctypes.byref(cl), float(dt), int(mode),
                                                ctypes.byref(cs), ctypes.c_void_p(dens.data_ptr()),
                                                ctypes.byref(rep), _stream_ptr(stream, st.device)),
           "skyrme_step_densities")
    return dens, _rep_dict(rep)


def slab_step(lat: Lattice, dt: float, mode: int, st: State, record, stream=None):
    """skyrme_slab_step: one iteration of an x-slab up to the arrest decision;
    ``record`` is a float64 device tensor of 8 values that receives the slab's
    sums."""
    cl, cs = lat.c(), st.c()
    _check(_on(st.device).skyrme_slab_step(ctypes.byref(cl), float(dt), int(mode),
                                           ctypes.byref(cs), ctypes.c_void_p(record.data_ptr()),
                                           _stream_ptr(stream, st.device)), "skyrme_slab_step")


def slab_finish(lat: Lattice, dt: float, mode: int, st: State, records, stream=None):
    """skyrme_slab_finish: the decision over all slabs from ``records`` (a
    float64 device tensor of shape (nslabs, 8), slab order) and the fix-up."""
    if records.dtype != _torch().float64 or records.dim() != 2 or records.shape[1] != 8 or \
            not records.is_contiguous():
        raise ValueError("records must be a contiguous float64 tensor of shape (nslabs, 8)")
    cl, cs = lat.c(), st.c()
    _check(_on(st.device).skyrme_slab_finish(ctypes.byref(cl), float(dt), int(mode),
                                             ctypes.byref(cs), ctypes.c_void_p(records.data_ptr()),
                                             int(records.shape[0]), _stream_ptr(stream, st.device)),
           "skyrme_slab_finish")


def read_report(lat: Lattice, st: State, stream=None) -> dict:
    cl, cs = lat.c(), st.c()
    rep = c_report()
    _check(_on(st.device).skyrme_read_report(ctypes.byref(cl), ctypes.byref(cs), ctypes.byref(rep),
                                     _stream_ptr(stream, st.device)), "skyrme_read_report")
    return _rep_dict(rep)


def energy(lat: Lattice, st: State, stream=None) -> dict:
    cl, cs = lat.c(), st.c()
    out = (ctypes.c_double * 6)()
    _check(_on(st.device).skyrme_energy(ctypes.byref(cl), ctypes.byref(cs), out,
                                _stream_ptr(stream, st.device)), "skyrme_energy")
    return dict(zip(("E", "E2", "E4", "E0", "B", "virial"), list(out)))


def baryon_number(lat: Lattice, st: State, stream=None) -> float:
    cl, cs = lat.c(), st.c()
    out = ctypes.c_double()
    _check(_on(st.device).skyrme_baryon_number(ctypes.byref(cl), ctypes.byref(cs), ctypes.byref(out),
                                       _stream_ptr(stream, st.device)), "skyrme_baryon_number")
    return out.value


def virial(lat: Lattice, st: State, stream=None) -> float:
    cl, cs = lat.c(), st.c()
    out = ctypes.c_double()
    _check(_on(st.device).skyrme_virial(ctypes.byref(cl), ctypes.byref(cs), ctypes.byref(out),
                                _stream_ptr(stream, st.device)), "skyrme_virial")
    return out.value


def energy_static(lat: Lattice, phi, stream=None) -> dict:
    """skyrme_energy_static of a device field tensor (Nx, Ny, Nz, 4) in the
    lattice's precision: E, E2, E4, E0, B and the virial, allocating nothing."""
    if phi.dtype != lat.dtype or not phi.is_contiguous() or tuple(phi.shape) != tuple(
            int(v) for v in lat.n) + (4,):
        raise ValueError("phi must be a contiguous (Nx, Ny, Nz, 4) tensor of the lattice dtype")
    cl = lat.c()
    out = (ctypes.c_double * 6)()
    _check(_on(phi.device).skyrme_energy_static(ctypes.byref(cl), ctypes.c_void_p(phi.data_ptr()), out,
                                       _stream_ptr(stream, phi.device)), "skyrme_energy_static")
    return dict(zip(("E", "E2", "E4", "E0", "B", "virial"), list(out)))


def sextic_energy(lat: Lattice, st: State, stream=None) -> float:
    """E6 = h^3 sum of c6 4 pi^4 (B0)^2 of the current field (skyrme_sextic_energy)."""
    cl, cs = lat.c(), st.c()
    out = ctypes.c_double()
    _check(_on(st.device).skyrme_sextic_energy(ctypes.byref(cl), ctypes.byref(cs), ctypes.byref(out),
                                       _stream_ptr(stream, st.device)), "skyrme_sextic_energy")
    return out.value


def observables(lat: Lattice, st: State, stream=None) -> dict:
    """Section 5 observables of the current field (skyrme_observables): B,
    centre of mass X, RMS radius R, quadrupole Q, inertia tensors U, V, W
    (3x3 lists; W[i][j] with i isospin, j space), D-term D and energy E."""
    o = c_observables()
    cl, cs = lat.c(), st.c()
    _check(_on(st.device).skyrme_observables(ctypes.byref(cl), ctypes.byref(cs), ctypes.byref(o),
                                     _stream_ptr(stream, st.device)), "skyrme_observables")
    mat = lambda a: [list(a[0:3]), list(a[3:6]), list(a[6:9])]
    return {"B": o.B, "X": list(o.X), "R": o.R, "Q": mat(o.Q), "U": mat(o.U), "V": mat(o.V),
            "W": mat(o.W), "D": o.D, "E": o.E}


def forces(lat: Lattice, st: State, want_dens: bool = True, stream=None):
    """(F, dens) of the current field as device tensors of shape (Nx,Ny,Nz,4)."""
    torch = _torch()
    shape = tuple(int(v) for v in lat.n) + (4,)
    F = torch.empty(shape, dtype=lat.dtype, device=st.device)
    D = torch.empty(shape, dtype=lat.dtype, device=st.device) if want_dens else None
    cl, cs = lat.c(), st.c()
    _check(_on(st.device).skyrme_forces(ctypes.byref(cl), ctypes.byref(cs), ctypes.c_void_p(F.data_ptr()),
                                ctypes.c_void_p(D.data_ptr()) if D is not None else None,
                                _stream_ptr(stream, st.device)), "skyrme_forces")
    return F, D


RENDER_MIN_STEP = 1e-4
RENDER_MAX_PIXELS = 1 << 26


def render_params(width: int, height: int, view=None, levelset: float = 0.2,
                  transfer_scale: float = 4.0, brightness: float = 1.0,
                  step: float = 0.01) -> c_render_params:
    """Parameters of the volume render; ``view`` is a row-major 3x3 rotation
    taking view-space vectors to box space (identity by default)."""
    v = np.eye(3) if view is None else np.asarray(view, dtype=np.float64).reshape(3, 3)
    return c_render_params(int(width), int(height), (ctypes.c_double * 9)(*v.ravel().tolist()),
                           float(levelset), float(transfer_scale), float(brightness), float(step))


def render_volume(lat: Lattice, st: State, out=None, stream=None):
    """Per-site volume {B0 / max B0, pion unit vector} of the current field as
    a float64 device tensor of shape (Nx, Ny, Nz, 4) (skyrme_render_volume)."""
    torch = _torch()
    shape = tuple(int(v) for v in lat.n) + (4,)
    vol = out if out is not None else torch.empty(shape, dtype=torch.float64, device=st.device)
    cl, cs = lat.c(), st.c()
    _check(_on(st.device).skyrme_render_volume(ctypes.byref(cl), ctypes.byref(cs),
                                       ctypes.c_void_p(vol.data_ptr()),
                                       ctypes.c_size_t(vol.numel() * vol.element_size()),
                                       _stream_ptr(stream, st.device)), "skyrme_render_volume")
    return vol


def render_rays(vol, params: c_render_params, stream=None):
    """Ray-march a (Nx, Ny, Nz, 4) float64 device volume; returns a float32
    device tensor of shape (height, width, 4), row 0 at the bottom."""
    torch = _torch()
    if vol.dtype != torch.float64 or vol.dim() != 4 or vol.shape[3] != 4 or not vol.is_contiguous():
        raise ValueError("vol must be a contiguous float64 tensor of shape (Nx, Ny, Nz, 4)")
    rgba = torch.empty((params.height, params.width, 4), dtype=torch.float32, device=vol.device)
    n = (ctypes.c_int * 3)(*[int(v) for v in vol.shape[:3]])
    _check(_on(vol.device).skyrme_render_rays(n, ctypes.c_void_p(vol.data_ptr()), ctypes.byref(params),
                                     ctypes.c_void_p(rgba.data_ptr()),
                                     _stream_ptr(stream, vol.device)), "skyrme_render_rays")
    return rgba


def render(lat: Lattice, st: State, params: c_render_params, work=None, stream=None):
    """Volume render of the current field's baryon density (skyrme_render);
    returns a float32 device tensor of shape (height, width, 4)."""
    torch = _torch()
    if work is None:
        work = torch.empty(load().skyrme_render_volume_bytes(ctypes.byref(lat.c())),
                           dtype=torch.uint8, device=st.device)
    rgba = torch.empty((params.height, params.width, 4), dtype=torch.float32, device=st.device)
    cl, cs = lat.c(), st.c()
    _check(_on(st.device).skyrme_render(ctypes.byref(cl), ctypes.byref(cs), ctypes.byref(params),
                                ctypes.c_void_p(work.data_ptr()),
                                ctypes.c_size_t(work.numel() * work.element_size()),
                                ctypes.c_void_p(rgba.data_ptr()), _stream_ptr(stream, st.device)),
           "skyrme_render")
    return rgba


def save_ppm(path: str, rgba) -> None:
    """Write an RGBA image (height, width, 4; row 0 at the bottom, channels in
    [0, 1]) as a binary PPM, top row first, alpha dropped."""
    a = np.asarray(rgba.cpu() if hasattr(rgba, "cpu") else rgba, dtype=np.float64)
    rgb = np.clip(np.rint(a[::-1, :, :3] * 255.0), 0, 255).astype(np.uint8)
    with open(path, "wb") as f:
        f.write(b"P6\n%d %d\n255\n" % (rgb.shape[1], rgb.shape[0]))
        f.write(rgb.tobytes())


PEAK_FP32, PEAK_FP64 = 0, 1


def measure_fma_peak(kind: int, stream=None) -> float:
    """Measured FMA throughput (TFLOP/s) of the current device: packed FP32
    pairs (PEAK_FP32) or FP64 (PEAK_FP64).  Synchronises the stream."""
    out = ctypes.c_double(0.0)
    _check(load().skyrme_measure_fma_peak(int(kind), ctypes.byref(out), _stream_ptr(stream)),
           "skyrme_measure_fma_peak")
    return out.value


def selftest_wait(lat: Lattice, st: State, limit_seconds: float = 0.05, stream=None) -> int:
    """Run the bounded-wait self-test (skyrme_selftest_wait) on the state's
    control block and return its status code (5, SKYRME_ETIMEOUT, when the
    wait gave up as it should)."""
    cl, cs = lat.c(), st.c()
    return int(_on(st.device).skyrme_selftest_wait(ctypes.byref(cl), ctypes.byref(cs),
                                           float(limit_seconds), _stream_ptr(stream, st.device)))


class FlowGraph:
    """A captured CUDA graph of ``nsteps`` flow iterations (skyrme_graph_*).
    ``stream`` must be a capturable (non-default) torch stream.  Pass
    ``batch`` instead of (lat, st, dt, mode) to capture batched iterations.
    Pass ``until=(tol, max_steps)`` for a graph that repeats chunks of
    ``nsteps`` iterations on the device until delta <= tol or max_steps
    iterations have run (skyrme_graph_create_until)."""

    def __init__(self, lat: Lattice = None, st: State = None, dt: float = 0.0, nsteps: int = 1,
                 mode: int = ARRESTED, stream=None, batch=None, until=None):
        torch = _torch()
        dev = st.device if st is not None else batch.states[0].device
        self.stream = stream if stream is not None else torch.cuda.Stream(dev)
        self.nsteps = int(nsteps)
        h = ctypes.c_void_p()
        sp = ctypes.c_void_p(self.stream.cuda_stream)
        if batch is not None:
            _check(_on(dev).skyrme_batch_graph_create(batch._h, self.nsteps, sp, ctypes.byref(h)),
                   "skyrme_batch_graph_create")
        elif until is not None:
            tol, max_steps = until
            cl, cs = lat.c(), st.c()
            _check(_on(dev).skyrme_graph_create_until(ctypes.byref(cl), float(dt), int(mode),
                                                    float(tol), int(max_steps), self.nsteps,
                                                    ctypes.byref(cs), sp, ctypes.byref(h)),
                   "skyrme_graph_create_until")
        else:
            cl, cs = lat.c(), st.c()
            _check(_on(dev).skyrme_graph_create(ctypes.byref(cl), float(dt), self.nsteps, int(mode),
                                              ctypes.byref(cs), sp, ctypes.byref(h)),
                   "skyrme_graph_create")
        self._h = h

    def launch(self, stream=None):
        """Launch the graph on ``stream`` (default: the graph's own stream).
        The launch is ordered after the work already queued on the caller's
        current stream (the state may just have been seeded there), and the
        current stream's later work after the launch, as if the graph ran on
        the current stream."""
        torch = _torch()
        s = stream if stream is not None else self.stream
        cur = torch.cuda.current_stream(s.device)
        if cur != s:
            s.wait_stream(cur)
        _check(load().skyrme_graph_launch(self._h, ctypes.c_void_p(s.cuda_stream)),
               "skyrme_graph_launch")
        if cur != s:
            cur.wait_stream(s)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().skyrme_graph_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


TILES = [(8, 32), (4, 32), (16, 16), (8, 16), (16, 32)]


def flow_until(lat: Lattice, dt: float, mode: int, st: State, tol: float, max_steps: int,
               chunk: int = 64, stream=None) -> dict:
    """Relax the flow on the device until delta = max |F| <= tol (checked
    every ``chunk`` iterations) or ``max_steps`` iterations have run: one
    launch of a run-to-tolerance graph.  Returns the final report."""
    torch = _torch()
    g = FlowGraph(lat, st, dt, chunk, mode, stream=stream, until=(tol, max_steps))
    try:
        g.launch()
        g.stream.synchronize()
        return read_report(lat, st)
    finally:
        g.close()


class Batch:
    """Many independent FP32 lattices advanced by one persistent launch per
    iteration (skyrme_batch_*).  ``states`` keep their own control blocks;
    read each with :func:`read_report`."""

    def __init__(self, lats, states, dts, mode: int = ARRESTED):
        torch = _torch()
        self.lats, self.states = list(lats), list(states)
        n = len(self.lats)
        self._cl = (c_lattice * n)(*[l.c() for l in self.lats])
        self._cs = (c_state * n)(*[st.c() for st in self.states])
        self._dt = (ctypes.c_double * n)(*[float(d) for d in dts])
        nbytes = int(load().skyrme_batch_scratch_bytes(n, self._cl))
        self.scratch = torch.zeros(nbytes, dtype=torch.uint8, device=self.states[0].device)
        h = ctypes.c_void_p()
        _check(_on(self.states[0].device).skyrme_batch_create(n, self._cl, self._cs, self._dt, int(mode),
                                          ctypes.c_void_p(self.scratch.data_ptr()), nbytes,
                                          ctypes.byref(h)), "skyrme_batch_create")
        self._h = h

    def step(self, nsteps: int, stream=None):
        _check(_on(self.states[0].device).skyrme_batch_step(self._h, int(nsteps),
                                        _stream_ptr(stream, self.states[0].device)),
               "skyrme_batch_step")

    def autotune(self, trials: int = 3, stream=None):
        t, ms = ctypes.c_int(), ctypes.c_double()
        _check(_on(self.states[0].device).skyrme_batch_autotune(self._h, int(trials),
                                            _stream_ptr(stream, self.states[0].device),
                                            ctypes.byref(t), ctypes.byref(ms)),
               "skyrme_batch_autotune")
        return t.value, ms.value

    def set_tile(self, tile: int):
        _check(_on(self.states[0].device).skyrme_batch_set_tile(self._h, int(tile)), "skyrme_batch_set_tile")

    def set_split(self, balanced: bool):
        """Divide the work among CTAs by streamed planes (True) or by centres."""
        _check(_on(self.states[0].device).skyrme_batch_set_split(self._h, 1 if balanced else 0),
               "skyrme_batch_set_split")

    def tile(self):
        t, ty, tz, g, sp = (ctypes.c_int() for _ in range(5))
        _check(load().skyrme_batch_tile(self._h, ctypes.byref(t), ctypes.byref(ty),
                                        ctypes.byref(tz), ctypes.byref(g)), "skyrme_batch_tile")
        _check(load().skyrme_batch_split(self._h, ctypes.byref(sp)), "skyrme_batch_split")
        return {"tile": t.value, "ty": ty.value, "tz": tz.value, "grid": g.value,
                "balanced": bool(sp.value)}

    def reports(self):
        return [read_report(l, st) for l, st in zip(self.lats, self.states)]

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().skyrme_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
