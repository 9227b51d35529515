"""Pins of the oracle's extension models (Section 7.8): the modified-pion,
loosely bound and lightly bound potentials and the BPS sextic term.

Independent routes, as for the standard model: the Euler-Lagrange operator
applied symbolically to the energy density (with B0 written in the paper's
double-epsilon form, not the oracle's cofactors), 1D radial reductions of the
hedgehog, Derrick scaling, brute-force differences of the discrete energy,
chiral SO(4) covariance and a planar field, which has no baryon density."""
import math

import numpy as np
import pytest
from scipy.integrate import quad

import oracle

from test_oracle_pins import coords, generic_field, tanh_hedgehog

PI = math.pi
MODEL = oracle.Model(mx=0.7, my=0.9, mz=0.6, mw=1.1, c6=0.35)


def levi(*p):
    p = list(p)
    if len(set(p)) < len(p):
        return 0
    s = 1
    for i in range(len(p)):
        for j in range(i + 1, len(p)):
            if p[i] > p[j]:
                s = -s
    return s


def test_extended_el_gradient_is_variational_derivative_of_energy_density():
    """EL_A = dL/dphi^A - d_i dL/d(d_i phi^A), the second term expanded by the
    chain rule with the symbolic Hessian of L, on a cubic polynomial field
    (the stencils are exact on it)."""
    sp = pytest.importorskip("sympy")
    x, y, z = sp.symbols("x y z")
    X = (x, y, z)
    rng = np.random.default_rng(11)
    mons = [x ** a * y ** b * z ** c for a in range(4) for b in range(4) for c in range(4)
            if a + b + c <= 3]
    comps = []
    for A in range(4):
        cs = rng.integers(-4, 5, size=len(mons))
        comps.append(sum(sp.Rational(int(c), 9) * mm for c, mm in zip(cs, mons)))
    mx, my, mz, mw, c6 = (sp.Rational(7, 10), sp.Rational(9, 10), sp.Rational(3, 5),
                          sp.Rational(11, 10), sp.Rational(7, 20))
    P = sp.symbols("p0:4")
    D = [[sp.Symbol(f"d{i}{A}") for A in range(4)] for i in range(3)]
    a = [[sum(D[i][B] * D[j][B] for B in range(4)) for j in range(3)] for i in range(3)]
    tra = a[0][0] + a[1][1] + a[2][2]
    u = 1 - P[0]
    # Eq. B0_components: -(1/12 pi^2) eps^{ijk} eps_{ABCD} phi^A d_i phi^B d_j phi^C d_k phi^D
    S = 0
    for i in range(3):
        for j in range(3):
            for k in range(3):
                e3 = levi(i, j, k)
                if not e3:
                    continue
                for A in range(4):
                    for B in range(4):
                        for C in range(4):
                            for Dd in range(4):
                                e4 = levi(A, B, C, Dd)
                                if e4:
                                    S += e3 * e4 * P[A] * D[i][B] * D[j][C] * D[k][Dd]
    B0sq_times_4pi4 = sp.expand(S * S) / 36  # 4 pi^4 (S / (12 pi^2))^2
    L = (tra + sp.Rational(1, 2) * (tra ** 2 - sum(a[i][j] ** 2 for i in range(3) for j in range(3)))
         + 2 * mx ** 2 * u + my ** 2 * (1 - P[0] ** 2) + mz ** 2 * u ** 2
         + sp.Rational(1, 2) * mw ** 2 * u ** 4 + c6 * B0sq_times_4pi4)
    n, h = (11, 11, 11), sp.Rational(1, 4)
    site = (4, 6, 5)
    pt = {X[k]: (site[k] - sp.Rational(n[k] - 1, 2)) * h for k in range(3)}
    val = {P[A]: comps[A].subs(pt) for A in range(4)}
    val.update({D[i][A]: sp.diff(comps[A], X[i]).subs(pt) for i in range(3) for A in range(4)})
    second = [[[sp.diff(comps[B], X[i], X[j]).subs(pt) for B in range(4)] for j in range(3)]
              for i in range(3)]
    G_exact = []
    for A in range(4):
        term = sp.diff(L, P[A]).subs(val)
        for i in range(3):
            dLd = sp.diff(L, D[i][A])
            for B in range(4):
                term -= sp.diff(dLd, P[B]).subs(val) * val[D[i][B]]
                for j in range(3):
                    term -= sp.diff(dLd, D[j][B]).subs(val) * second[i][j][B]
        G_exact.append(float(term))
    f = sp.lambdify((x, y, z), comps, "numpy")
    Xs, Ys, Zs = coords(n, float(h))
    phi = np.ascontiguousarray(np.stack(f(Xs, Ys, Zs), axis=-1).astype(np.float64))
    d1, d2, dm = oracle.site_derivatives(phi, float(h), *site)
    model = oracle.Model(0.7, 0.9, 0.6, 1.1, 0.35)
    G, F, dens = oracle.site_terms(phi[site], d1, d2, dm, model)
    np.testing.assert_allclose(G, G_exact, rtol=1e-10, atol=1e-9 * max(1.0, max(map(abs, G_exact))))
    # the densities at the same point
    e0 = float((2 * mx ** 2 * u + my ** 2 * (1 - P[0] ** 2) + mz ** 2 * u ** 2
                + sp.Rational(1, 2) * mw ** 2 * u ** 4).subs(val))
    e6 = float((c6 * B0sq_times_4pi4).subs(val))
    assert dens[2] == pytest.approx(e0, rel=1e-12)
    assert dens[4] == pytest.approx(e6, rel=1e-10)
    assert dens[3] == pytest.approx(float(-S.subs(val)) / (12 * PI ** 2), rel=1e-10)


def radial_terms(fun, dfun, md):
    """Hedgehog phi = (cos f, sin f rhat): E0 of the four potentials and
    E6 = c6 4 pi^4 int (B0)^2 = 4 pi c6 int f'^2 sin^4 f / r^2 dr, using
    B0 = -f' sin^2 f / (2 pi^2 r^2)."""
    def e0(r):
        c = math.cos(fun(r))
        return 4 * PI * r * r * (2 * md.mx ** 2 * (1 - c) + md.my ** 2 * (1 - c * c)
                                 + md.mz ** 2 * (1 - c) ** 2 + 0.5 * md.mw ** 2 * (1 - c) ** 4)

    def e6(r):
        if r == 0:
            return 0.0
        return 4 * PI * md.c6 * dfun(r) ** 2 * math.sin(fun(r)) ** 4 / (r * r)

    E0 = quad(e0, 0, 40, limit=500, epsabs=1e-12, epsrel=1e-13)[0]
    E6 = quad(e6, 0, 40, limit=500, epsabs=1e-12, epsrel=1e-13)[0]
    return E0, E6


def test_extension_energies_converge_to_radial_integrals_at_fourth_order():
    s = 0.8
    fun = lambda r: PI * (1 - math.tanh(r / s))
    dfun = lambda r: -PI / s / math.cosh(r / s) ** 2
    E0x, E6x = radial_terms(fun, dfun, MODEL)
    e0s, e6s = [], []
    for N, h in ((40, 0.24), (80, 0.12), (120, 0.08)):
        e = oracle.energy(tanh_hedgehog((N, N, N), h, s), h, MODEL)
        e0s.append(abs(e["E0"] - E0x) / E0x)
        e6s.append(abs(e["E6"] - E6x) / E6x)
        assert e["E"] == pytest.approx(e["E2"] + e["E4"] + e["E0"] + e["E6"], rel=1e-14)
    # the potentials carry no derivatives: a lattice sum of a smooth decaying
    # function, exact up to the box truncation (~1e-8 here) once h resolves it
    assert e0s[1] < 5e-8 and e0s[2] < 5e-8, e0s
    # the sextic density is built from the 4th-order first derivatives
    assert e6s[0] > e6s[1] > e6s[2] and e6s[2] < 5e-3, e6s
    order = math.log(e6s[1] / e6s[2]) / math.log(1.5)
    assert 3.4 < order < 4.6, (e6s, order)


def test_extended_virial_is_derivative_of_energy_under_dilation():
    """E(lambda) of phi(lambda x): E2/lambda + lambda E4 + E0/lambda^3 +
    lambda^3 E6, so dE/dlambda at 1 is -E2 + E4 - 3 E0 + 3 E6 = V."""
    s, eps = 1.0, 1e-4
    gaps, V, E6 = [], None, None
    for N, h in ((80, 0.12), (120, 0.08)):
        n = (N, N, N)
        e1 = oracle.energy(tanh_hedgehog(n, h, s), h, MODEL)
        Ep = oracle.energy(tanh_hedgehog(n, h, s, lam=1 + eps), h, MODEL)["E"]
        Em = oracle.energy(tanh_hedgehog(n, h, s, lam=1 - eps), h, MODEL)["E"]
        gaps.append(abs(e1["virial"] - (Ep - Em) / (2 * eps)))
        V, E6 = e1["virial"], e1["E6"]
    assert abs(V) > 10.0 and E6 > 1.0  # not vacuous; the sextic part matters
    assert gaps[1] < 0.01 * abs(V), gaps
    order = math.log(gaps[0] / gaps[1]) / math.log(1.5)
    assert 3.4 < order < 4.6, (gaps, order)
    # dropping the 3 E6 term would miss by far more than the truncation gap
    assert 3 * E6 > 20 * gaps[1]


def test_extended_force_matches_energy_gradient_at_fourth_order():
    L = 2.6
    errs = []
    for h in (0.2, 0.1):
        N = int(round(2 * L / h)) + 1
        n = (N, N, N)
        phi = tanh_hedgehog(n, h, 0.9, centre=(0.13, -0.07, 0.05))
        X, Y, Z = coords(n, h)
        bump = np.exp(-((X - 0.3) ** 2 + (Y + 0.2) ** 2 + Z ** 2) / 0.35)
        eta = np.zeros_like(phi)
        eta[..., 0] = 0.4 * bump * np.sin(Y)
        eta[..., 1] = bump * np.cos(X)
        eta[..., 2] = 0.5 * bump
        eta[..., 3] = -0.3 * bump * Y
        eps = 1e-4
        Ep = oracle.energy(np.ascontiguousarray(phi + eps * eta), h, MODEL)["E"]
        Em = oracle.energy(np.ascontiguousarray(phi - eps * eta), h, MODEL)["E"]
        G, _, _ = oracle.forces(phi, h, MODEL)
        lhs = (Ep - Em) / (2 * eps)
        rhs = h ** 3 * np.sum(G * eta)
        errs.append(abs(lhs - rhs) / abs(lhs))
    assert errs[1] < 5e-3, errs
    assert 3.3 < math.log2(errs[0] / errs[1]) < 4.7, errs


def test_sextic_term_vanishes_for_a_planar_field():
    """A field independent of z has d_z phi = 0, so D, B0 and every sextic
    contribution vanish: the forces equal those without the term."""
    n, h = (14, 15, 9), 0.3
    X, Y, _ = coords(n, h)
    r = np.sqrt(X * X + Y * Y)
    f = PI * np.exp(-r / 0.9)
    with np.errstate(invalid="ignore", divide="ignore"):
        c = np.where(r > 0, X / np.where(r > 0, r, 1), 1.0)
        s_ = np.where(r > 0, Y / np.where(r > 0, r, 1), 0.0)
    phi = np.ascontiguousarray(np.stack([np.cos(f), np.sin(f) * c, np.sin(f) * s_,
                                         np.zeros_like(f)], axis=-1))
    with_six = oracle.forces(phi, h, oracle.Model(0.5, c6=2.0))
    without = oracle.forces(phi, h, oracle.Model(0.5))
    for a, b in zip(with_six, without):
        np.testing.assert_array_equal(a, b)
    assert oracle.energy(phi, h, oracle.Model(0.5, c6=2.0))["E6"] == 0.0


def test_sextic_term_is_chirally_covariant():
    """det[phi, d phi...] is SO(4) invariant: without potentials, G(R phi) = R G(phi)."""
    n, h = (13, 13, 13), 0.25
    phi = generic_field(n, h)
    rng = np.random.default_rng(8)
    Q, _ = np.linalg.qr(rng.normal(size=(4, 4)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] = -Q[:, 0]
    md = oracle.Model(0.0, c6=1.3)
    G, _, d = oracle.forces(phi, h, md)
    G2, _, d2 = oracle.forces(np.ascontiguousarray(phi @ Q.T), h, md)
    scale = np.max(np.abs(G))
    np.testing.assert_allclose(G2, G @ Q.T, atol=1e-11 * scale, rtol=0)
    np.testing.assert_allclose(d2, d, atol=1e-11 * np.max(np.abs(d)), rtol=0)


def test_standard_model_entry_points_agree_with_the_model_ones_bitwise():
    n, h = (12, 12, 12), 0.25
    phi = generic_field(n, h)
    d1, d2, dm = oracle.site_derivatives(phi, h, 5, 6, 7)
    G, F, dens = oracle.site_terms(phi[5, 6, 7], d1, d2, dm, 0.8)
    Gm, Fm, densm = oracle.site_terms(phi[5, 6, 7], d1, d2, dm, oracle.Model(0.8))
    assert np.array_equal(G, Gm) and np.array_equal(F, Fm) and np.array_equal(dens, densm[:4])
    assert densm[4] == 0.0


def test_flow_reports_the_model_energy_and_virial():
    """The flow's per-step E (the arrest's comparand) and virial are those of
    the model's static energy, sextic part included."""
    n, h = (14, 13, 15), 0.25
    phi = generic_field(n, h)
    st = oracle.new_state(phi)
    reps = oracle.flow(st, h, MODEL, 0.01, 2, reports=True)
    e0 = oracle.energy(phi, h, MODEL)
    assert e0["E6"] > 0.01 * e0["E"]
    for k in ("E", "E2", "E4", "E0", "E6", "B", "virial"):
        assert reps[0][k] == e0[k], k
    # the second step starts from the first step's field
    assert reps[1]["E"] != reps[0]["E"]
