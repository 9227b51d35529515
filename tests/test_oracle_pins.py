"""Pins of the FP64 CPU oracle against what the paper and mathematics fix.

None of these tests re-types the oracle's own formulas: each compares it with
an independent route (exact polynomial calculus, the Euler-Lagrange operator
applied symbolically to the energy density, a 1D radial reduction, Derrick
scaling, symmetry, topology, brute-force differences of the discrete energy).
A plausible slip in the oracle (a dropped term, wrong sign, transposed pair,
wrong stencil weight) fails at least one of them.
"""
import math

import numpy as np
import pytest
from scipy.integrate import quad

import oracle

PI = math.pi


# ----------------------------------------------------------------- helpers
def coords(n, h):
    ax = [(np.arange(N) - 0.5 * (N - 1)) * h for N in n]
    return np.meshgrid(*ax, indexing="ij")


def tanh_hedgehog(n, h, s=0.8, lam=1.0, centre=(0.0, 0.0, 0.0)):
    """Smooth B=1 hedgehog phi = (cos f, sin f rhat), f = pi (1 - tanh(lam r / s)).
    f - pi is odd in r, so the field is analytic at the origin (the exponential
    profile is not)."""
    X, Y, Z = coords(n, h)
    X, Y, Z = X - centre[0], Y - centre[1], Z - centre[2]
    r = np.sqrt(X * X + Y * Y + Z * Z)
    f = PI * (1.0 - np.tanh(lam * r / s))
    with np.errstate(invalid="ignore", divide="ignore"):
        sr = np.where(r > 0, np.sin(f) / np.where(r > 0, r, 1.0), 0.0)
    phi = np.stack([np.cos(f), sr * X, sr * Y, sr * Z], axis=-1)
    return np.ascontiguousarray(phi)


def radial_energy(fun, dfun, m):
    """E = 4 pi int [r^2 f'^2 + 2 sin^2 f (1 + f'^2) + sin^4 f / r^2 + 2 m^2 r^2 (1 - cos f)] dr,
    the reduction of Eq. SkyrmeEnergy_phi for phi = (cos f, sin f rhat)
    (a_ij has eigenvalues f'^2 and sin^2 f / r^2 twice)."""
    def g(r):
        F, P = fun(r), dfun(r)
        s = math.sin(F)
        t4 = s ** 4 / (r * r) if r > 0 else 0.0
        return 4 * PI * (r * r * P * P + 2 * s * s * (1 + P * P) + t4
                         + 2 * m * m * r * r * (1 - math.cos(F)))
    return quad(g, 0, 40, limit=500, epsabs=1e-12, epsrel=1e-13)[0]


def random_rotation(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def generic_field(n, h, seed=3):
    """A smooth unit field with no symmetry: symmetrised product of three
    isorotated hedgehogs at scattered positions."""
    rng = np.random.default_rng(seed)
    pos = rng.uniform(-0.9, 0.9, size=(3, 3))
    q = rng.normal(size=(3, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return oracle.seed_product(n, h, pos, q, 0.9, True)


# ------------------------------------------------- 1. stencils (Section 3)
def poly_field(n, h, rng, degree):
    """Unconstrained R^4-valued polynomial of total degree <= degree, with its
    exact first and second derivatives."""
    X, Y, Z = coords(n, h)
    terms = [(a, b, c) for a in range(degree + 1) for b in range(degree + 1)
             for c in range(degree + 1) if a + b + c <= degree]
    coef = rng.uniform(-0.4, 0.4, size=(4, len(terms)))

    def mono(a, b, c):
        def p(V, k):
            return V ** k if k >= 0 else np.zeros_like(V)
        return p(X, a) * p(Y, b) * p(Z, c)

    val = np.zeros(X.shape + (4,))
    d1 = np.zeros((3,) + X.shape + (4,))
    d2 = np.zeros((3,) + X.shape + (4,))
    dm = np.zeros((3,) + X.shape + (4,))
    for t, (a, b, c) in enumerate(terms):
        for A in range(4):
            k = coef[A, t]
            val[..., A] += k * mono(a, b, c)
            d1[0, ..., A] += k * a * mono(a - 1, b, c)
            d1[1, ..., A] += k * b * mono(a, b - 1, c)
            d1[2, ..., A] += k * c * mono(a, b, c - 1)
            d2[0, ..., A] += k * a * (a - 1) * mono(a - 2, b, c)
            d2[1, ..., A] += k * b * (b - 1) * mono(a, b - 2, c)
            d2[2, ..., A] += k * c * (c - 1) * mono(a, b, c - 2)
            dm[0, ..., A] += k * a * b * mono(a - 1, b - 1, c)
            dm[1, ..., A] += k * a * c * mono(a - 1, b, c - 1)
            dm[2, ..., A] += k * b * c * mono(a, b - 1, c - 1)
    return np.ascontiguousarray(val), d1, d2, dm


def test_stencils_exact_on_degree4_polynomials():
    rng = np.random.default_rng(0)
    n, h = (9, 10, 11), 0.3
    phi, d1x, d2x, dmx = poly_field(n, h, rng, 4)
    for (x, y, z) in [(2, 2, 2), (4, 5, 6), (6, 7, 8), (3, 6, 4)]:
        d1, d2, dm = oracle.site_derivatives(phi, h, x, y, z)
        np.testing.assert_allclose(d1, d1x[:, x, y, z], rtol=0, atol=1e-11)
        np.testing.assert_allclose(d2, d2x[:, x, y, z], rtol=0, atol=1e-10)
        np.testing.assert_allclose(dm, dmx[:, x, y, z], rtol=0, atol=1e-10)


def test_first_derivative_truncation_term():
    """For f = x^5 the 5-point first derivative is exactly 5x^4 - 4h^4
    (leading error -h^4 f^(5)/30), and the second derivative 20x^3 exactly."""
    n, h = (9, 5, 5), 0.25
    X, _, _ = coords(n, h)
    phi = np.zeros(n + (4,))
    phi[..., 1] = X ** 5
    for x in range(2, 7):
        d1, d2, _ = oracle.site_derivatives(phi, h, x, 2, 2)
        xv = X[x, 2, 2]
        assert d1[0, 1] == pytest.approx(5 * xv ** 4 - 4 * h ** 4, abs=1e-12)
        assert d2[0, 1] == pytest.approx(20 * xv ** 3, abs=1e-11)


# ------------------- 2. Euler-Lagrange gradient is dE/dphi (Section 2.1, 3)
def test_el_gradient_is_variational_derivative_of_energy_density():
    sp = pytest.importorskip("sympy")
    x, y, z = sp.symbols("x y z")
    rng = np.random.default_rng(5)
    # cubic polynomial field with rational coefficients (stencils are exact)
    mons = [x ** a * y ** b * z ** c for a in range(4) for b in range(4) for c in range(4)
            if a + b + c <= 3]
    comps = []
    for A in range(4):
        cs = rng.integers(-4, 5, size=len(mons))
        comps.append(sum(sp.Rational(int(c), 7) * mm for c, mm in zip(cs, mons)))
    m = sp.Rational(3, 4)
    # energy density written with independent symbols for phi^A and d_i phi^A
    P = sp.symbols("p0:4")
    D = [[sp.Symbol(f"d{i}{A}") for A in range(4)] for i in range(3)]
    a = [[sum(D[i][B] * D[j][B] for B in range(4)) for j in range(3)] for i in range(3)]
    tra = a[0][0] + a[1][1] + a[2][2]
    dens = tra + sp.Rational(1, 2) * (tra ** 2 - sum(a[i][j] ** 2 for i in range(3)
                                                      for j in range(3))) \
        + 2 * m ** 2 * (1 - P[0])
    X = (x, y, z)
    subs = {P[A]: comps[A] for A in range(4)}
    subs.update({D[i][A]: sp.diff(comps[A], X[i]) for i in range(3) for A in range(4)})
    n, h = (11, 11, 11), sp.Rational(1, 4)
    site = (4, 6, 5)
    pt = {X[k]: (site[k] - sp.Rational(n[k] - 1, 2)) * h for k in range(3)}
    G_exact = []
    for A in range(4):
        # Euler-Lagrange operator: dL/dphi - d_i (dL/d(d_i phi))
        term = sp.diff(dens, P[A]).subs(subs)
        for i in range(3):
            term -= sp.diff(sp.diff(dens, D[i][A]).subs(subs), X[i])
        G_exact.append(float(term.subs(pt)))
    f = sp.lambdify((x, y, z), comps, "numpy")
    Xs, Ys, Zs = coords(n, float(h))
    phi = np.ascontiguousarray(np.stack(f(Xs, Ys, Zs), axis=-1).astype(np.float64))
    d1, d2, dm = oracle.site_derivatives(phi, float(h), *site)
    G, F, _ = oracle.site_terms(phi[site], d1, d2, dm, float(m))
    np.testing.assert_allclose(G, G_exact, rtol=1e-10, atol=1e-9)


def test_force_is_tangent_projection():
    n, h = (12, 12, 12), 0.25
    phi = generic_field(n, h)
    G, F, _ = oracle.forces(phi, h, 1.0)
    inner = slice(2, 10)
    ph, Gi, Fi = (a[inner, inner, inner] for a in (phi, G, F))
    # tangent to S^3 ...
    assert np.max(np.abs(np.sum(Fi * ph, axis=-1))) < 1e-12 * np.max(np.abs(Gi))
    # ... and equal to -G minus its normal part
    Gt = Gi - np.sum(Gi * ph, axis=-1, keepdims=True) * ph
    np.testing.assert_allclose(Fi, -Gt, rtol=0, atol=1e-12 * np.max(np.abs(Gi)))


# ----------------------- 3. energy: 1D radial reduction (Section 2.1 energy)
@pytest.mark.parametrize("m", [0.0, 1.0])
def test_energy_converges_to_radial_integral_at_fourth_order(m):
    s = 0.8
    fun = lambda r: PI * (1 - math.tanh(r / s))
    dfun = lambda r: -PI / s / math.cosh(r / s) ** 2
    exact = radial_energy(fun, dfun, m)
    errs = []
    for N, h in ((40, 0.24), (80, 0.12), (120, 0.08)):
        e = oracle.energy(tanh_hedgehog((N, N, N), h, s), h, m)
        errs.append(abs(e["E"] - exact) / exact)
    # the steep core gives a large error constant; the order is what is pinned
    assert errs[0] > errs[1] > errs[2] and errs[2] < 2.5e-3, errs
    order = math.log(errs[1] / errs[2]) / math.log(1.5)
    assert 3.5 < order < 4.5, (errs, order)


def test_bogomolny_bound_and_vacuum_is_fixed_point():
    n, h = (14, 14, 14), 0.3
    vac = oracle.seed_vacuum(n)
    G, F, dens = oracle.forces(vac, h, 1.0)
    # F vanishes exactly (the projection removes the mass-term gradient); the
    # densities only carry the rounding residue of the stencil weights
    assert np.all(F == 0.0) and np.max(np.abs(dens)) < 1e-28
    e = oracle.energy(vac, h, 1.0)
    assert abs(e["E"]) < 1e-25 and abs(e["B"]) < 1e-25
    st = oracle.new_state(vac)
    oracle.flow(st, h, 1.0, 0.01, 5)
    assert np.array_equal(st.phi, vac) and not st.v.any()
    # E >= 12 pi^2 |B| for a generic field (the sigma-model form has no 1/12pi^2)
    phi = tanh_hedgehog((48, 48, 48), 0.2, 0.5)
    e = oracle.energy(phi, 0.2, 0.0)
    assert e["E"] >= 12 * PI ** 2 * abs(e["B"])


# -------------------------- 4. baryon number (Section 2, Eq. B0_components)
def test_baryon_number_is_topological_degree():
    N, h = 80, 0.12
    # hedgehog with f(0) = pi and R = z: B = +1 (Table 1) -- pins the sign;
    # the lattice deficit shrinks as h falls
    b1c = oracle.energy(oracle.seed_rational_map((40, 40, 40), 0.24, 1, 0.8), 0.24, 0.0)["B"]
    b1 = oracle.energy(oracle.seed_rational_map((N, N, N), h, 1, 0.8), h, 0.0)["B"]
    assert abs(b1 - 1.0) < 5e-3 and abs(b1 - 1.0) < abs(b1c - 1.0) / 8
    # the B = 4 cubic map of Table 1 (the rest of the deficit is the box tail)
    b4c = oracle.energy(oracle.seed_rational_map((40, 40, 40), 0.24, 4, 1.5), 0.24, 0.0)["B"]
    b4 = oracle.energy(oracle.seed_rational_map((N, N, N), h, 4, 1.5), h, 0.0)["B"]
    assert abs(b4 - 4.0) < 2e-2 and abs(b4 - 4.0) < abs(b4c - 4.0)
    # a spatial reflection reverses orientation: B -> -B
    phi = oracle.seed_rational_map((N, N, N), h, 1, 0.8)
    bm = oracle.energy(np.ascontiguousarray(phi[::-1]), h, 0.0)["B"]
    assert bm == pytest.approx(-b1, rel=1e-12)


def test_baryon_density_is_determinant_form():
    """eps^{ijk} eps_{ABCD} phi^A d_i phi^B d_j phi^C d_k phi^D = 6 det[phi, d1 phi, d2 phi, d3 phi]."""
    rng = np.random.default_rng(11)
    n, h = (10, 10, 10), 0.3
    phi, _, _, _ = poly_field(n, h, rng, 3)
    for site in [(3, 4, 5), (6, 2, 7)]:
        d1, d2, dm = oracle.site_derivatives(phi, h, *site)
        _, _, dens = oracle.site_terms(phi[site], d1, d2, dm, 0.0)
        M = np.stack([phi[site], d1[0], d1[1], d1[2]])
        assert dens[3] == pytest.approx(-np.linalg.det(M) / (2 * PI ** 2), rel=1e-11)


def test_baryon_number_is_additive_for_separated_product():
    N, h = 72, 0.15
    pos = np.array([[-2.2, 0.3, 0.0], [2.2, -0.3, 0.1]])
    rng = np.random.default_rng(2)
    q = rng.normal(size=(2, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    # the lattice deficit of one constituent, measured on the same lattice
    one = oracle.energy(oracle.seed_product((N, N, N), h, pos[:1], q[:1], 0.6, False),
                        h, 1.0)["B"]
    assert abs(one - 1.0) < 0.03
    for sym in (False, True):
        phi = oracle.seed_product((N, N, N), h, pos, q, 0.6, sym)
        assert np.allclose(np.linalg.norm(phi, axis=-1), 1.0, atol=1e-13)
        assert oracle.energy(phi, h, 1.0)["B"] == pytest.approx(2.0 * one, abs=2e-3)


# ----------------------------------------- 5. symmetries (Section 2, 3)
def test_isospin_rotation_covariance():
    n, h = (14, 14, 14), 0.25
    phi = generic_field(n, h)
    R = random_rotation(np.random.default_rng(7))
    rot = phi.copy()
    rot[..., 1:] = phi[..., 1:] @ R.T
    G0, F0, d0 = oracle.forces(phi, h, 1.0)
    G1, F1, d1 = oracle.forces(np.ascontiguousarray(rot), h, 1.0)
    scale = np.max(np.abs(F0))
    np.testing.assert_allclose(F1[..., 0], F0[..., 0], atol=1e-12 * scale)
    np.testing.assert_allclose(F1[..., 1:], F0[..., 1:] @ R.T, atol=1e-12 * scale)
    np.testing.assert_allclose(d1, d0, atol=1e-11)


def test_chiral_so4_covariance_when_massless():
    n, h = (14, 14, 14), 0.25
    phi = generic_field(n, h)
    Q, _ = np.linalg.qr(np.random.default_rng(9).normal(size=(4, 4)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] = -Q[:, 0]
    rot = np.ascontiguousarray(phi @ Q.T)
    _, F0, d0 = oracle.forces(phi, h, 0.0)
    _, F1, d1 = oracle.forces(rot, h, 0.0)
    np.testing.assert_allclose(F1, F0 @ Q.T, atol=1e-12 * np.max(np.abs(F0)))
    np.testing.assert_allclose(d1, d0, atol=1e-11)


@pytest.mark.parametrize("op", ["swap_xy", "swap_yz", "cycle", "reflect_x", "reflect_z"])
def test_cubic_lattice_symmetry(op):
    N, h = 14, 0.25
    phi = generic_field((N, N, N), h)
    _, F0, d0 = oracle.forces(phi, h, 1.0)

    def T(a):
        if op == "swap_xy":
            return np.ascontiguousarray(np.swapaxes(a, 0, 1))
        if op == "swap_yz":
            return np.ascontiguousarray(np.swapaxes(a, 1, 2))
        if op == "cycle":
            return np.ascontiguousarray(np.transpose(a, (1, 2, 0, 3)))
        if op == "reflect_x":
            return np.ascontiguousarray(a[::-1])
        return np.ascontiguousarray(a[:, :, ::-1])

    orient = -1.0 if op in ("swap_xy", "swap_yz", "reflect_x", "reflect_z") else 1.0
    _, F1, d1 = oracle.forces(T(phi), h, 1.0)
    scale = np.max(np.abs(F0))
    np.testing.assert_allclose(F1, T(F0), atol=1e-12 * scale)
    np.testing.assert_allclose(d1[..., :3], T(d0)[..., :3], atol=1e-11)
    np.testing.assert_allclose(d1[..., 3], orient * T(d0)[..., 3], atol=1e-12)


# ------------------ 6. force = gradient of the discrete energy, 4th order
def test_force_matches_energy_gradient_at_fourth_order():
    L = 2.6
    errs = []
    for h in (0.2, 0.1):
        N = int(round(2 * L / h)) + 1
        n = (N, N, N)
        phi = tanh_hedgehog(n, h, 0.9, centre=(0.13, -0.07, 0.05))
        X, Y, Z = coords(n, h)
        bump = np.exp(-((X - 0.3) ** 2 + (Y + 0.2) ** 2 + Z ** 2) / 0.35)
        eta = np.zeros_like(phi)
        eta[..., 1] = bump * np.cos(X)
        eta[..., 2] = 0.5 * bump
        eta[..., 3] = -0.3 * bump * Y
        m, eps = 1.0, 1e-4
        Ep = oracle.energy(np.ascontiguousarray(phi + eps * eta), h, m)["E"]
        Em = oracle.energy(np.ascontiguousarray(phi - eps * eta), h, m)["E"]
        G, _, _ = oracle.forces(phi, h, m)
        lhs = (Ep - Em) / (2 * eps)
        rhs = h ** 3 * np.sum(G * eta)
        errs.append(abs(lhs - rhs) / abs(lhs))
    assert errs[1] < 5e-3, errs
    assert 3.3 < math.log2(errs[0] / errs[1]) < 4.7, errs


# ----------------------------- 7. Derrick scaling = virial (Section 5.6)
def test_virial_is_derivative_of_energy_under_dilation():
    """E(lambda) of phi(lambda x) is E2/lambda + lambda E4 + E0/lambda^3, so
    dE/dlambda at 1 is -E2 + E4 - 3 E0 = V.  On the lattice the two sides
    differ by a truncation error that must vanish at fourth order."""
    m, s, eps = 1.0, 1.0, 1e-4
    gaps, V = [], None
    for N, h in ((80, 0.12), (120, 0.08)):
        n = (N, N, N)
        e1 = oracle.energy(tanh_hedgehog(n, h, s), h, m)
        Ep = oracle.energy(tanh_hedgehog(n, h, s, lam=1 + eps), h, m)["E"]
        Em = oracle.energy(tanh_hedgehog(n, h, s, lam=1 - eps), h, m)["E"]
        gaps.append(abs(e1["virial"] - (Ep - Em) / (2 * eps)))
        V = e1["virial"]
    assert abs(V) > 10.0  # a non-stationary field: the check is not vacuous
    assert gaps[1] < 0.01 * abs(V), gaps
    order = math.log(gaps[0] / gaps[1]) / math.log(1.5)
    assert 3.4 < order < 4.6, (gaps, order)


# ------------------------------------- 8. the flow itself (Section 3)
def test_arrest_rule_direction_and_update_order():
    n, h, dt, m = (12, 12, 12), 0.25, 0.01, 1.0
    phi = generic_field(n, h)
    _, F, _ = oracle.forces(phi, h, m)
    v0 = np.ascontiguousarray(0.3 * np.roll(F, 1, axis=0))
    v0[:2] = v0[-2:] = 0
    v0[:, :2] = v0[:, -2:] = 0
    v0[:, :, :2] = v0[:, :, -2:] = 0
    # energy rose (previous energy -inf): velocity zeroed first, v' = dt F
    st = oracle.FlowState(phi=phi.copy(), v=v0.copy(), E_prev=-math.inf)
    r = oracle.flow(st, h, m, dt, 1, reports=True)[0]
    assert r["arrested"] == 1
    np.testing.assert_array_equal(st.v, dt * F)
    t = phi + dt * (dt * F)
    inner = (slice(2, -2),) * 3
    np.testing.assert_allclose(st.phi[inner],
                               (t / np.linalg.norm(t, axis=-1, keepdims=True))[inner],
                               rtol=0, atol=1e-15)
    # energy fell (previous energy +inf): v' = v + dt F
    st = oracle.FlowState(phi=phi.copy(), v=v0.copy(), E_prev=math.inf)
    r = oracle.flow(st, h, m, dt, 1, reports=True)[0]
    assert r["arrested"] == 0
    np.testing.assert_allclose(st.v, v0 + dt * F, rtol=0, atol=1e-15)
    # equal energy does not arrest (strict comparison)
    e = oracle.energy(phi, h, m)["E"]
    st = oracle.FlowState(phi=phi.copy(), v=v0.copy(), E_prev=e)
    assert oracle.flow(st, h, m, dt, 1, reports=True)[0]["arrested"] == 0
    # the unit-length constraint holds after every update (Section 3)
    assert np.allclose(np.linalg.norm(st.phi, axis=-1), 1.0, atol=1e-14)


def test_newton_flow_is_first_order_consistent_in_time():
    """Symplectic Euler with projection is a first-order integrator of the flow
    equation: over a fixed fictitious time T, halving dt halves the distance to
    the dt -> 0 trajectory (differences between successive halvings fall by 2)."""
    N, h, m, T = 24, 0.25, 1.0, 0.2
    base = tanh_hedgehog((N, N, N), h, 0.9, centre=(0.2, 0.1, -0.1))
    finals = []
    for k in range(3):
        dt = 0.01 / 2 ** k
        st = oracle.new_state(base)
        oracle.flow(st, h, m, dt, int(round(T / dt)), mode=oracle.NEWTON)
        finals.append(st.phi.copy())
    d1 = np.max(np.abs(finals[0] - finals[1]))
    d2 = np.max(np.abs(finals[1] - finals[2]))
    assert d1 > 1e-6  # the field moved
    assert 1.7 < d1 / d2 < 2.3, (d1, d2)


def test_newton_flow_total_energy_is_bounded_without_secular_drift():
    """With the arrest off, H = E(phi_n) + h^3 sum |v_n|^2 / 2 of the flow
    (symplectic Euler, Section 3) stays bounded: a transient of about 1% while
    the renormalisation absorbs the centripetal part of the motion (the same
    at dt and dt/2), then no drift beyond 0.2% over the rest of the run.
    A wrong sign, a missing dt or an unstable step makes H run away."""
    N, h, m = 28, 0.25, 1.0
    phi = tanh_hedgehog((N, N, N), h, 0.9)
    for dt in (0.05 * h, 0.025 * h):
        st = oracle.new_state(phi)
        H = []
        for _ in range(600):
            K = 0.5 * h ** 3 * np.sum(st.v[2:-2, 2:-2, 2:-2] ** 2)
            r = oracle.flow(st, h, m, dt, 1, mode=oracle.NEWTON, reports=True)[0]
            H.append(r["E"] + K)
        H = np.array(H)
        assert np.all(np.abs(H - H[0]) < 0.05 * H[0]), (H.min(), H.max())
        assert abs(H[-100:].mean() - H[300:400].mean()) < 2e-3 * H[0]
        assert r["E"] < H[0] and r["B"] > 0.95  # the Skyrmion is still there


def test_gradient_flow_decreases_energy_monotonically():
    # first-order flow: explicit stability needs dt of order h^2 / stiffness
    N, h, m, dt = 24, 0.25, 1.0, 5e-5
    st = oracle.new_state(generic_field((N, N, N), h))
    E = [oracle.energy(st.phi, h, m)["E"]]
    for _ in range(6):
        oracle.flow(st, h, m, dt, 5, mode=oracle.GRADIENT)
        E.append(oracle.energy(st.phi, h, m)["E"])
    assert np.all(np.diff(E) < 0), E


# --------------------------------- 9. seeds and random inputs (Section 4)
PAULI = np.array([[[0, 1], [1, 0]], [[0, -1j], [1j, 0]], [[1, 0], [0, -1]]])


def to_su2(phi):
    """U = phi^0 1 + i phi^a tau^a as 2x2 complex matrices (Section 2.1)."""
    return phi[..., 0, None, None] * np.eye(2) + 1j * np.einsum("...a,aij->...ij",
                                                               phi[..., 1:], PAULI)


def from_su2(U):
    phi0 = np.real(np.trace(U, axis1=-2, axis2=-1)) / 2
    pa = [np.real(np.trace(-1j * U @ PAULI[a], axis1=-2, axis2=-1)) / 2 for a in range(3)]
    return np.stack([phi0] + pa, axis=-1)


def test_product_ansatz_matches_su2_matrix_products():
    """Eq. "Product ansatz" with explicit 2x2 matrices: U = prod_k A_k U_k A_k^dagger."""
    N, h = 16, 0.3
    X, Y, Z = coords((N, N, N), h)
    rng = np.random.default_rng(4)
    K = 3
    q = rng.normal(size=(K, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    pos = rng.uniform(-0.8, 0.8, size=(K, 3))
    Ufwd = np.broadcast_to(np.eye(2, dtype=complex), X.shape + (2, 2)).copy()
    Urev = Ufwd.copy()
    mats = []
    for k in range(K):
        d = np.stack([X - pos[k, 0], Y - pos[k, 1], Z - pos[k, 2]], axis=-1)
        r = np.linalg.norm(d, axis=-1)
        f = PI * np.exp(-r / 0.9)
        hh = np.concatenate([np.cos(f)[..., None], (np.sin(f) / r)[..., None] * d], -1)
        A = to_su2(q[k])
        mats.append(A @ to_su2(hh) @ A.conj().T)
    for k in range(K):
        Ufwd = Ufwd @ mats[k]
        Urev = Urev @ mats[K - 1 - k]
    fwd = from_su2(Ufwd)
    sym = from_su2(Ufwd + Urev)
    sym /= np.linalg.norm(sym, axis=-1, keepdims=True)
    for symmetrise, expect in ((False, fwd), (True, sym)):
        phi = oracle.seed_product((N, N, N), h, pos, q, 0.9, symmetrise)
        expect = np.ascontiguousarray(expect)
        oracle.apply_vacuum_boundary(expect)
        np.testing.assert_allclose(phi, expect, atol=1e-13)


def test_b4_rational_map_has_cubic_symmetry():
    """The energy density of the O_h-symmetric B=4 map is invariant under the
    cubic rotations (x,y,z) -> (y,-x,z) and (x,y,z) -> (z,x,y)."""
    N, h = 40, 0.2
    phi = oracle.seed_rational_map((N, N, N), h, 4, 1.5)
    _, _, d = oracle.forces(phi, h, 1.0)
    e = d[..., 0] + d[..., 1] + d[..., 2]
    rot90 = np.transpose(e, (1, 0, 2))[::-1]  # x' = y, y' = -x (as array ops)
    np.testing.assert_allclose(rot90, e, atol=1e-10 * e.max())
    cyc = np.transpose(e, (2, 0, 1))
    np.testing.assert_allclose(cyc, e, atol=1e-10 * e.max())


def test_noise_generator_statistics():
    from scipy import stats
    vals = np.array([oracle.normal(1234, i) for i in range(20000)])
    assert abs(vals.mean()) < 0.03 and abs(vals.std() - 1) < 0.03
    assert stats.kstest(vals, "norm").pvalue > 1e-3
    u = np.array([oracle.splitmix64(7, i) >> 11 for i in range(20000)], dtype=np.float64) / 2.0 ** 53
    assert stats.kstest(u, "uniform").pvalue > 1e-3
    assert oracle.splitmix64(7, 0) != oracle.splitmix64(8, 0)


def test_noise_seed_properties():
    N, h, R, sigma = 40, 0.15, 2.0, 0.6
    phi = oracle.seed_noise((N, N, N), h, R, sigma, 1001)
    assert np.allclose(np.linalg.norm(phi, axis=-1), 1.0, atol=1e-13)
    assert np.all(phi[:2, ..., 0] == 1) and np.all(phi[-2:, ..., 0] == 1)
    X, Y, Z = coords((N, N, N), h)
    ball = X * X + Y * Y + Z * Z <= R * R
    # the field differs from the vacuum at O(1) inside the ball
    assert np.mean(np.abs(phi[ball][:, 1:])) > 0.2
    again = oracle.seed_noise((N, N, N), h, R, sigma, 1001)
    assert np.array_equal(phi, again)
    other = oracle.seed_noise((N, N, N), h, R, sigma, 1002)
    assert not np.array_equal(phi, other)
