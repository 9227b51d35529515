"""Relaxed-Skyrmion pins of the oracle's arrested Newton flow (Section 3).

The massless B=1 Skyrmion has E = 1.232 x 12 pi^2 in these units (no
1/12 pi^2 in Eq. SkyrmeEnergy_phi).  Two independent routes are checked:
the 1D radial Euler-Lagrange boundary-value problem (solved with SciPy) and
the 3D oracle flow from the hedgehog seed on the 48^3, h = 0.2 lattice.
"""
import math

import numpy as np
import pytest
from scipy.integrate import quad, solve_bvp

import oracle

PI = math.pi
LITERATURE_B1 = 1.232  # E / (12 pi^2) of the massless B = 1 Skyrmion


def radial_solution(m, R=30.0, delta=1e-3):
    """Profile ODE from the radial energy density
    r^2 f'^2 + 2 sin^2 f (1 + f'^2) + sin^4 f / r^2 + 2 m^2 r^2 (1 - cos f):
    (r^2 + 2 sin^2 f) f'' + 2 r f' + sin 2f (f'^2 - 1 - sin^2 f / r^2) - m^2 r^2 sin f = 0,
    f(0) = pi, f(R) = 0."""
    def ode(r, y, p):
        f, g = y
        s = np.sin(f)
        fpp = -(2 * r * g + np.sin(2 * f) * (g * g - 1 - s * s / (r * r))
                - m * m * r * r * s) / (r * r + 2 * s * s)
        return np.vstack([g, fpp])

    def bc(ya, yb, p):
        return np.array([ya[0] - (PI + p[0] * delta), ya[1] - p[0], yb[0]])

    r = np.linspace(delta, R, 3000)
    f0 = PI * np.exp(-r)
    sol = solve_bvp(ode, bc, r, np.vstack([f0, -f0]), p=[-2.0], tol=1e-10,
                    max_nodes=200000)

    def dens(rr):
        F, P = sol.sol(rr)
        s = math.sin(F)
        return 4 * PI * (rr * rr * P * P + 2 * s * s * (1 + P * P) + s ** 4 / (rr * rr)
                         + 2 * m * m * rr * rr * (1 - math.cos(F)))
    return sol, quad(dens, delta, R, limit=1000, epsrel=1e-12)[0]


def test_radial_minimum_is_literature_value():
    sol, E = radial_solution(0.0)
    assert E / (12 * PI ** 2) == pytest.approx(LITERATURE_B1, abs=1e-3)
    assert sol.p[0] == pytest.approx(-2.008, abs=2e-3)  # f'(0)


@pytest.fixture(scope="module")
def relaxed_b1():
    N, h = 48, 0.2
    st = oracle.new_state(oracle.seed_rational_map((N, N, N), h, 1, 1.0))
    seed = oracle.energy(st.phi, h, 0.0)
    reps = oracle.flow(st, h, 0.0, 0.05 * h, 500, reports=True)
    return st, h, seed, reps


def test_relaxed_massless_b1_energy(relaxed_b1):
    st, h, seed, reps = relaxed_b1
    e = oracle.energy(st.phi, h, 0.0)
    ratio = e["E"] / (12 * PI ** 2)
    # the vacuum box at |x| = 4.7 squeezes the massless tail: E sits slightly above
    assert LITERATURE_B1 <= ratio < LITERATURE_B1 * 1.01, ratio
    assert e["B"] == pytest.approx(1.0, abs=5e-3)
    # relaxation lowered the energy, the residual and the virial
    assert e["E"] < seed["E"] - 2.0
    assert reps[-1]["delta"] < 0.1 * reps[0]["delta"]
    assert abs(e["virial"]) < 0.3 * abs(seed["virial"])


def test_relaxed_hedgehog_keeps_o3_symmetry(relaxed_b1):
    st, h, _, _ = relaxed_b1
    N = st.phi.shape[0]
    ax = (np.arange(N) - 0.5 * (N - 1)) * h
    X, Y, Z = np.meshgrid(ax, ax, ax, indexing="ij")
    r = np.sqrt(X * X + Y * Y + Z * Z)
    inner = (slice(2, -2),) * 3
    phi, r, X, Y, Z = st.phi[inner], r[inner], X[inner], Y[inner], Z[inner]
    # phi^0 is a function of r alone: residuals about a smooth fit in r are
    # small away from the cubic box (whose walls break O(3) at large r)
    sel = r < 3.0
    rs, p0 = r[sel], phi[..., 0][sel]
    fit = np.polynomial.Chebyshev.fit(rs, p0, 14)
    resid = p0 - fit(rs)
    assert np.sqrt(np.mean(resid ** 2)) < 2e-3 and np.max(np.abs(resid)) < 1e-2
    # the pion vector points along +r (hedgehog orientation is kept)
    pion = phi[..., 1:]
    rhat = np.stack([X, Y, Z], axis=-1) / r[..., None]
    norm = np.linalg.norm(pion, axis=-1)
    sel = (r > 0.4) & (r < 3.0)
    cosang = np.sum(pion * rhat, axis=-1)[sel] / norm[sel]
    assert cosang.min() > 0.999
