"""FP64 CPU oracle of the arrested-Newton-flow step (arXiv 2604.25876).

TEST INFRASTRUCTURE ONLY.  Tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only users; the CUDA library never
imports, links or executes anything here.  The C source ``skyrme_oracle.c``
holds the arithmetic; this module compiles it on first use (gcc, OpenMP,
``-ffp-contract=off`` so that x86 and Arm hosts round identically) and wraps
it with ctypes + NumPy.

Paper passages: Section 2.1 (energy and baryon densities), Section 3 (flow
equation, Euler-Lagrange gradient, stencils, arrest, projection, vacuum box),
Section 4 (rational-map and product ansätze), Section 5.6 (virial), Section
7.8 (extension potentials and the BPS sextic term).

Wherever a mass ``m`` is taken, a ``Model`` may be passed instead to switch on
the extension terms.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "skyrme_oracle.c")
_HDR = os.path.join(_HERE, "skyrme_oracle.h")
_LIB = os.path.join(_HERE, "_build", "libskyrme_oracle.so")
_lock = threading.Lock()
_lib = None

NEWTON, ARRESTED, GRADIENT = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle shared library (idempotent)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    stale = (not os.path.exists(_LIB)) or any(
        os.path.getmtime(p) > os.path.getmtime(_LIB) for p in (_SRC, _HDR))
    if force or stale:
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", "-fno-fast-math", "-Wall", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Report(ctypes.Structure):
    _fields_ = [("E", ctypes.c_double), ("E2", ctypes.c_double),
                ("E4", ctypes.c_double), ("E0", ctypes.c_double),
                ("B", ctypes.c_double), ("virial", ctypes.c_double),
                ("delta", ctypes.c_double), ("arrested", ctypes.c_int),
                ("E6", ctypes.c_double)]


class _Model(ctypes.Structure):
    _fields_ = [("mx", ctypes.c_double), ("my", ctypes.c_double), ("mz", ctypes.c_double),
                ("mw", ctypes.c_double), ("c6", ctypes.c_double)]


@dataclass(frozen=True)
class Model:
    """Section 7.8 extension model: potential 2 mx^2 (1 - phi0) + my^2 (1 - phi0^2)
    + mz^2 (1 - phi0)^2 + mw^2 (1 - phi0)^4 / 2 and the sextic term
    c6 4 pi^4 (B0)^2 in the static energy density."""
    mx: float
    my: float = 0.0
    mz: float = 0.0
    mw: float = 0.0
    c6: float = 0.0

    def c(self) -> _Model:
        return _Model(float(self.mx), float(self.my), float(self.mz), float(self.mw),
                      float(self.c6))


def _model(m) -> _Model:
    return m.c() if isinstance(m, Model) else Model(float(m)).c()


class _Observables(ctypes.Structure):
    _fields_ = [("B", ctypes.c_double), ("X", ctypes.c_double * 3), ("R", ctypes.c_double),
                ("Q", ctypes.c_double * 9), ("U", ctypes.c_double * 9), ("V", ctypes.c_double * 9),
                ("W", ctypes.c_double * 9), ("D", ctypes.c_double), ("E", ctypes.c_double)]


class _RenderParams(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int), ("height", ctypes.c_int), ("view", ctypes.c_double * 9),
                ("levelset", ctypes.c_double), ("transfer_scale", ctypes.c_double),
                ("brightness", ctypes.c_double), ("step", ctypes.c_double)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            D = ctypes.c_double
            P = ctypes.c_void_p
            I3 = ctypes.POINTER(ctypes.c_int)
            lib.orc_site_derivatives.argtypes = [I3, D, P, ctypes.c_int, ctypes.c_int,
                                                 ctypes.c_int, P, P, P]
            lib.orc_site_terms.argtypes = [P, P, P, P, D, P, P, P]
            lib.orc_forces.argtypes = [I3, D, D, P, P, P, P]
            lib.orc_energy.argtypes = [I3, D, D, P, P]
            lib.orc_anf_step.argtypes = [I3, D, D, D, ctypes.c_int, P, P, P, P,
                                         ctypes.POINTER(_Report)]
            lib.orc_anf_step.restype = ctypes.c_int
            lib.orc_flow.argtypes = [I3, D, D, D, ctypes.c_int, ctypes.c_int, P, P, P, P,
                                     ctypes.POINTER(_Report)]
            lib.orc_flow.restype = ctypes.c_longlong
            lib.orc_seed_vacuum.argtypes = [I3, P]
            lib.orc_seed_rational_map.argtypes = [I3, D, ctypes.c_int, D, P]
            lib.orc_seed_rational_map.restype = ctypes.c_int
            lib.orc_seed_product.argtypes = [I3, D, ctypes.c_int, P, P, D, ctypes.c_int, P]
            lib.orc_seed_noise.argtypes = [I3, D, D, D, ctypes.c_uint64, P]
            lib.orc_noise_components.argtypes = [I3, D, D, D, ctypes.c_uint64, P]
            lib.orc_gaussian_smooth.argtypes = [I3, D, D, P, P]
            lib.orc_apply_vacuum_boundary.argtypes = [I3, P]
            lib.orc_rational_map_field.argtypes = [I3, D, ctypes.c_int, D, P, P, P]
            lib.orc_rational_map_field.restype = ctypes.c_int
            lib.orc_field_product.argtypes = [I3, P, P, P]
            PM = ctypes.POINTER(_Model)
            lib.orc_site_terms_model.argtypes = [P, P, P, P, PM, P, P, P]
            lib.orc_forces_model.argtypes = [I3, D, PM, P, P, P, P]
            lib.orc_energy_model.argtypes = [I3, D, PM, P, P]
            lib.orc_anf_step_model.argtypes = [I3, D, PM, D, ctypes.c_int, P, P, P, P,
                                               ctypes.POINTER(_Report)]
            lib.orc_anf_step_model.restype = ctypes.c_int
            lib.orc_flow_model.argtypes = [I3, D, PM, D, ctypes.c_int, ctypes.c_int, P, P, P, P,
                                           ctypes.POINTER(_Report)]
            lib.orc_flow_model.restype = ctypes.c_longlong
            lib.orc_observables.argtypes = [I3, D, D, P, ctypes.POINTER(_Observables)]
            lib.orc_render_volume_from_field.argtypes = [I3, D, P, P]
            lib.orc_render_volume.argtypes = [I3, P, ctypes.POINTER(_RenderParams), P]
            lib.orc_render_sample.argtypes = [I3, P, P, P]
            lib.orc_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.orc_splitmix64.restype = ctypes.c_uint64
            lib.orc_normal.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.orc_normal.restype = ctypes.c_double
            _lib = lib
    return _lib


def _dims(n):
    n = tuple(int(v) for v in n)
    if len(n) != 3:
        raise ValueError("lattice dims must be (Nx, Ny, Nz)")
    return (ctypes.c_int * 3)(*n)


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.c_void_p)


def _field(n):
    return np.zeros(tuple(n) + (4,), dtype=np.float64)


# ---------------------------------------------------------------- site level
def site_derivatives(phi: np.ndarray, h: float, x: int, y: int, z: int):
    """(d1, d2, dm) at one interior site: shapes (3,4) each; dm pairs xy, xz, yz."""
    lib = _load()
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    d1, d2, dm = (np.zeros((3, 4)) for _ in range(3))
    lib.orc_site_derivatives(_dims(phi.shape[:3]), h, _ptr(phi), x, y, z,
                             _ptr(d1), _ptr(d2), _ptr(dm))
    return d1, d2, dm


def site_terms(phi0, d1, d2, dm, m):
    """(G, F, dens) at one site from its value and derivatives; dens =
    (e2, e4, e0, b) for a mass m, (e2, e4, e0, b, e6) for a ``Model``."""
    lib = _load()
    args = [np.ascontiguousarray(a, dtype=np.float64) for a in (phi0, d1, d2, dm)]
    G, F = np.zeros(4), np.zeros(4)
    if isinstance(m, Model):
        dens = np.zeros(5)
        md = m.c()
        lib.orc_site_terms_model(*[_ptr(a) for a in args], ctypes.byref(md), _ptr(G), _ptr(F),
                                 _ptr(dens))
    else:
        dens = np.zeros(4)
        lib.orc_site_terms(*[_ptr(a) for a in args], m, _ptr(G), _ptr(F), _ptr(dens))
    return G, F, dens


# ------------------------------------------------------------- lattice level
def forces(phi: np.ndarray, h: float, m):
    """(G, F, dens) arrays of shape (Nx,Ny,Nz,4); zero on boundary layers.
    dens = (e2, e4, e0, b) per site; ``m`` a mass or a ``Model``."""
    lib = _load()
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    G, F, dens = (np.zeros_like(phi) for _ in range(3))
    md = _model(m)
    lib.orc_forces_model(_dims(phi.shape[:3]), h, ctypes.byref(md), _ptr(phi), _ptr(G), _ptr(F),
                         _ptr(dens))
    return G, F, dens


def observables(phi: np.ndarray, h: float, m: float) -> dict:
    """Section 5 observables of a static field (see orc_observables):
    B, centre of mass X, RMS radius R, quadrupole Q, inertia tensors U, V, W
    (3x3 arrays; W[i, j] with i isospin and j space), D-term D and energy E."""
    lib = _load()
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    o = _Observables()
    lib.orc_observables(_dims(phi.shape[:3]), h, m, _ptr(phi), ctypes.byref(o))
    mat = lambda a: np.array(list(a)).reshape(3, 3)
    return {"B": o.B, "X": np.array(list(o.X)), "R": o.R, "Q": mat(o.Q), "U": mat(o.U),
            "V": mat(o.V), "W": mat(o.W), "D": o.D, "E": o.E}


def render_volume_from_field(phi: np.ndarray, h: float) -> np.ndarray:
    """(n0, n1, n2, 4) volume {B0 / max B0, unit pions} (orc_render_volume_from_field)."""
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    vol = np.zeros_like(phi)
    _load().orc_render_volume_from_field(_dims(phi.shape[:3]), h, _ptr(phi), _ptr(vol))
    return vol


def render_volume(vol: np.ndarray, width: int, height: int, view=None, levelset: float = 0.2,
                  transfer_scale: float = 4.0, brightness: float = 1.0,
                  step: float = 0.01) -> np.ndarray:
    """(height, width, 4) RGBA image of a volume (orc_render_volume)."""
    vol = np.ascontiguousarray(vol, dtype=np.float64)
    rp = _RenderParams(int(width), int(height),
                       (ctypes.c_double * 9)(*np.asarray(view if view is not None else np.eye(3),
                                                         dtype=np.float64).ravel()),
                       levelset, transfer_scale, brightness, step)
    out = np.zeros((int(height), int(width), 4))
    _load().orc_render_volume(_dims(vol.shape[:3]), _ptr(vol), ctypes.byref(rp), _ptr(out))
    return out


def render_sample(vol: np.ndarray, g) -> np.ndarray:
    """Trilinear sample of the volume at lattice coordinates g (orc_render_sample)."""
    vol = np.ascontiguousarray(vol, dtype=np.float64)
    gg = np.ascontiguousarray(g, dtype=np.float64)
    out = np.zeros(4)
    _load().orc_render_sample(_dims(vol.shape[:3]), _ptr(vol), _ptr(gg), _ptr(out))
    return out


def energy(phi: np.ndarray, h: float, m) -> dict:
    """E, E2, E4, E0, E6, B and the virial of a field; ``m`` a mass or a ``Model``."""
    lib = _load()
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    out = np.zeros(7)
    md = _model(m)
    lib.orc_energy_model(_dims(phi.shape[:3]), h, ctypes.byref(md), _ptr(phi), _ptr(out))
    return dict(zip(("E", "E2", "E4", "E0", "E6", "B", "virial"), out.tolist()))


@dataclass
class FlowState:
    """Field, velocity and the previous energy of an oracle flow."""
    phi: np.ndarray
    v: np.ndarray
    E_prev: float = float("inf")
    steps: int = 0
    arrests: int = 0


def new_state(phi: np.ndarray) -> FlowState:
    phi = np.ascontiguousarray(phi, dtype=np.float64).copy()
    return FlowState(phi=phi, v=np.zeros_like(phi))


def flow(st: FlowState, h: float, m, dt: float, nsteps: int,
         mode: int = ARRESTED, reports: bool = False):
    """Advance ``st`` by ``nsteps`` iterations; returns a list of per-step dicts
    when ``reports`` is true, else None.  Raises on a non-finite value."""
    lib = _load()
    n = st.phi.shape[:3]
    work = np.zeros_like(st.phi)
    e_prev = np.array([st.E_prev])
    reps = (_Report * max(nsteps, 1))()
    md = _model(m)
    got = lib.orc_flow_model(_dims(n), h, ctypes.byref(md), dt, mode, nsteps, _ptr(st.phi),
                             _ptr(st.v), _ptr(work), _ptr(e_prev), reps)
    st.E_prev = float(e_prev[0])
    if got < 0:
        raise FloatingPointError("oracle flow produced a non-finite value")
    st.steps += nsteps
    st.arrests += int(got)
    if reports:
        return [dict(E=r.E, E2=r.E2, E4=r.E4, E0=r.E0, E6=r.E6, B=r.B, virial=r.virial,
                     delta=r.delta, arrested=r.arrested) for r in reps[:nsteps]]
    return None


# --------------------------------------------------------------------- seeds
def seed_vacuum(n):
    phi = _field(n)
    _load().orc_seed_vacuum(_dims(n), _ptr(phi))
    return phi


def seed_rational_map(n, h: float, B: int, profile_scale: float):
    phi = _field(n)
    if _load().orc_seed_rational_map(_dims(n), h, B, profile_scale, _ptr(phi)) != 0:
        raise ValueError("rational maps of degree 1 to 4 only")
    return phi


def seed_product(n, h: float, positions, quats, profile_scale: float, symmetrise: bool):
    pos = np.ascontiguousarray(positions, dtype=np.float64).reshape(-1, 3)
    q = np.ascontiguousarray(quats, dtype=np.float64).reshape(-1, 4)
    assert len(pos) == len(q)
    phi = _field(n)
    _load().orc_seed_product(_dims(n), h, len(pos), _ptr(pos), _ptr(q), profile_scale,
                             int(bool(symmetrise)), _ptr(phi))
    return phi


def rational_map_field(n, h: float, B: int, profile_scale: float, X=(0.0, 0.0, 0.0), R=None):
    """Rational-map Skyrmion moved to X and rotated by R: U_B(R^T (x - X))
    (orc_rational_map_field); no vacuum boundary applied."""
    phi = _field(n)
    Xa = np.ascontiguousarray(X, dtype=np.float64)
    Ra = np.ascontiguousarray(np.eye(3) if R is None else R, dtype=np.float64).reshape(9)
    if _load().orc_rational_map_field(_dims(n), h, B, profile_scale, _ptr(Xa), _ptr(Ra),
                                      _ptr(phi)) != 0:
        raise ValueError("rational maps of degree 1 to 4 only")
    return phi


def field_product(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Ordered product ansatz a b, site by site (orc_field_product)."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    out = np.zeros_like(a)
    _load().orc_field_product(_dims(a.shape[:3]), _ptr(a), _ptr(b), _ptr(out))
    return out


def seed_noise(n, h: float, radius: float, sigma: float, seed: int):
    phi = _field(n)
    _load().orc_seed_noise(_dims(n), h, radius, sigma, int(seed), _ptr(phi))
    return phi


def noise_components(n, h: float, radius: float, sigma: float, seed: int):
    """The smoothed-noise seed's noise field before it is added to the vacuum."""
    out = _field(n)
    _load().orc_noise_components(_dims(n), h, radius, sigma, int(seed), _ptr(out))
    return out


def gaussian_smooth(field: np.ndarray, h: float, sigma: float):
    """The noise seed's separable Gaussian smoothing applied to a 4-component field."""
    a = np.ascontiguousarray(field, dtype=np.float64)
    out = np.zeros_like(a)
    _load().orc_gaussian_smooth(_dims(a.shape[:3]), h, sigma, _ptr(a), _ptr(out))
    return out


def apply_vacuum_boundary(phi: np.ndarray):
    _load().orc_apply_vacuum_boundary(_dims(phi.shape[:3]), _ptr(phi))
    return phi


def splitmix64(seed: int, i: int) -> int:
    return int(_load().orc_splitmix64(seed, i))


def normal(seed: int, i: int) -> float:
    return float(_load().orc_normal(seed, i))
