"""Pins of the oracle's Section 5 observables (centre of mass, RMS radius,
quadrupole, inertia tensors U, V, W, D-term), which the oracle evaluates in
the paper's su(2) notation (2x2 complex matrices, traces of currents).

Independent references used here:
  - closed forms for the B=1 hedgehog, from the 4-vector reduction of the
    same formulas with the exact derivatives of the profile, summed over the
    same lattice sites (so only the finite-difference error remains, which
    must fall as h^4);
  - exact covariance under a 90-degree lattice rotation, an isorotation and
    a whole-site translation;
  - brute-force kinetic energies: U, V, W are defined by
    T = a U a / 2 + b V b / 2 - a W b for a field isorotating with angular
    velocity a and rotating with b, where T is the kinetic energy of the
    Lagrangian whose static part is Eq. SkyrmeEnergy_phi,
    T = h^3 sum |phi_t|^2 + sum_i (|phi_t|^2 |d_i phi|^2 - (phi_t . d_i phi)^2).
"""
import math

import numpy as np
import pytest

import oracle

PI = math.pi


def coords(n, h):
    ax = [(np.arange(N) - 0.5 * (N - 1)) * h for N in n]
    return np.meshgrid(*ax, indexing="ij")


def hedgehog(X, Y, Z, s=0.8):
    """phi = (cos f, sin f rhat), f = pi (1 - tanh(r / s)), and f'."""
    r = np.sqrt(X * X + Y * Y + Z * Z)
    f = PI * (1.0 - np.tanh(r / s))
    fp = -PI / s / np.cosh(r / s) ** 2
    sr = np.where(r > 0, np.sin(f) / np.where(r > 0, r, 1.0), 0.0)
    phi = np.stack([np.cos(f), sr * X, sr * Y, sr * Z], axis=-1)
    return np.ascontiguousarray(phi), r, f, fp


def interior(a):
    return a[2:-2, 2:-2, 2:-2]


def fd1(phi, h, axis):
    """4th-order first derivative along axis (interior sites only)."""
    sl = lambda k: np.take(phi, np.arange(2 + k, phi.shape[axis] - 2 + k), axis=axis)
    d = (8.0 * (sl(1) - sl(-1)) - (sl(2) - sl(-2))) / (12.0 * h)
    idx = [slice(2, -2)] * 3
    idx[axis] = slice(None)
    return d[tuple(idx)]


def kinetic(phi, phidot, h):
    """Kinetic energy with the tangent part of the lattice derivative (the
    su(2) current L_i of a lattice field)."""
    p = interior(phi)
    d = [fd1(phi, h, i) for i in range(3)]
    d = [di - np.sum(p * di, axis=-1, keepdims=True) * p for di in d]
    v = interior(phidot)
    v2 = np.sum(v * v, axis=-1)
    t = v2.copy()
    for i in range(3):
        t += v2 * np.sum(d[i] * d[i], axis=-1) - np.sum(v * d[i], axis=-1) ** 2
    return h ** 3 * float(np.sum(t))


def closed_form_hedgehog(n, h, m, s=0.8):
    """Lattice sums of the hedgehog's observable densities, exact derivatives."""
    X, Y, Z = coords(n, h)
    _, r, f, fp = hedgehog(X, Y, Z, s)
    X, Y, Z, r, f, fp = (interior(a) for a in (X, Y, Z, r, f, fp))
    sn2 = np.sin(f) ** 2
    q = sn2 / r ** 2  # the two transverse eigenvalues of a_ij
    rh = np.stack([X / r, Y / r, Z / r], axis=-1)
    delta = np.eye(3)
    P = rh[..., :, None] * rh[..., None, :]  # rhat rhat
    a = fp[..., None, None] ** 2 * P + q[..., None, None] * (delta - P)
    tra = fp ** 2 + 2 * q
    e2, e4, e0 = tra, 2 * fp ** 2 * q + q * q, 2 * m * m * (1 - np.cos(f))
    b = -sn2 * fp / (2 * PI ** 2 * r ** 2)
    lam = 2 * sn2 * (1 + fp ** 2 + q)  # U = V = W density / (delta - rhat rhat)
    inertia = lam[..., None, None] * (delta - P)
    a2 = np.einsum("...ik,...kj->...ij", a, a)
    T = 2 * a * (1 + tra)[..., None, None] - 2 * a2 - (e2 + e4 + e0)[..., None, None] * delta
    rv = np.stack([X, Y, Z], axis=-1)
    r2 = r ** 2
    dint = np.einsum("...i,...j,...ij->...", rv, rv, T) - r2 * np.trace(T, axis1=-2, axis2=-1) / 3
    h3 = h ** 3
    E = h3 * np.sum(e2 + e4 + e0)
    B = h3 * np.sum(b)
    return {"B": B, "R": math.sqrt(h3 * np.sum(r2 * b) / B), "E": E,
            "I": h3 * np.sum(inertia, axis=(0, 1, 2)), "D": -2 * E / 5 * h3 * np.sum(dint)}


@pytest.mark.parametrize("m", [0.0, 1.0])
def test_hedgehog_observables_match_closed_forms_at_fourth_order(m):
    errs = []
    for N, h in ((32, 0.2), (62, 0.1)):
        n = (N, N, N)
        X, Y, Z = coords(n, h)
        phi = hedgehog(X, Y, Z)[0]
        o = oracle.observables(phi, h, m)
        c = closed_form_hedgehog(n, h, m)
        lam = c["I"][0, 0]
        assert np.allclose(c["I"], lam * np.eye(3), atol=1e-12 * lam)
        # symmetric lattice and cubic symmetry: centre 0, no quadrupole, isotropic tensors
        assert np.max(np.abs(o["X"])) < 1e-12
        assert np.max(np.abs(o["Q"])) < 1e-12
        for k in ("U", "V", "W"):
            t = o[k]
            assert np.max(np.abs(t - np.diag(np.diag(t)))) < 1e-10 * lam, k
            assert np.ptp(np.diag(t)) < 1e-10 * lam, k
        # the paper's remark that W vanishes for B = 1 does not follow from
        # its Eq. "W inertia tensor": the hedgehog's grand-spin symmetry makes
        # U = V = W (a rotation combined with the same isorotation is no motion)
        errs.append(max(abs(o["U"][0, 0] / lam - 1), abs(o["V"][0, 0] / lam - 1),
                        abs(o["W"][0, 0] / lam - 1), abs(o["B"] / c["B"] - 1),
                        abs(o["R"] / c["R"] - 1), abs(o["E"] / c["E"] - 1),
                        abs(o["D"] / c["D"] - 1)))
    # steep core (f' = -pi/0.8 at r = 0): a few per cent at h = 0.2, and the
    # error falls by 2^4 (within rounding of the order) when h halves
    assert errs[1] < 5e-3, errs
    assert errs[0] / errs[1] > 2 ** 3.5, errs


def lattice_rot_z(phi):
    """phi'(x) = phi(R^-1 x) for R the +90 degree rotation about z."""
    return np.ascontiguousarray(np.flip(phi, axis=1).transpose(1, 0, 2, 3))


def generic_field(n, h, seed=5):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(-0.8, 0.8, size=(2, 3))
    q = rng.normal(size=(2, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return oracle.seed_product(n, h, pos, q, 0.9, False)


def test_observables_covariant_under_lattice_rotation_and_isorotation():
    n, h, m = (28, 28, 28), 0.25, 1.0
    phi = generic_field(n, h)
    o = oracle.observables(phi, h, m)
    R = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    o2 = oracle.observables(lattice_rot_z(phi), h, m)
    tol = 1e-10 * np.max(np.abs(o["V"]))
    for k in ("B", "R", "D", "E"):
        assert o2[k] == pytest.approx(o[k], rel=1e-12, abs=1e-12), k
    assert np.allclose(o2["X"], R @ o["X"], atol=1e-12)
    assert np.allclose(o2["Q"], R @ o["Q"] @ R.T, atol=tol)
    assert np.allclose(o2["V"], R @ o["V"] @ R.T, atol=tol)
    assert np.allclose(o2["U"], o["U"], atol=tol)
    assert np.allclose(o2["W"], o["W"] @ R.T, atol=tol)
    # isorotation of the pion components by S
    S = np.array([[0.0, 0.0, 1.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    iso = phi.copy()
    iso[..., 1:] = phi[..., 1:] @ S.T
    o3 = oracle.observables(iso, h, m)
    for k in ("B", "R", "D", "E"):
        assert o3[k] == pytest.approx(o[k], rel=1e-12, abs=1e-12), k
    assert np.allclose(o3["Q"], o["Q"], atol=tol)
    assert np.allclose(o3["V"], o["V"], atol=tol)
    assert np.allclose(o3["U"], S @ o["U"] @ S.T, atol=tol)
    assert np.allclose(o3["W"], S @ o["W"], atol=tol)
    assert abs(np.trace(o["Q"])) < tol
    # a generic field has no isotropy
    assert np.max(np.abs(o["Q"])) > 1e-3 and np.max(np.abs(o["W"] - o["W"].T)) > 1e-3


def test_observables_under_whole_site_translation():
    n, h, m = (30, 30, 30), 0.25, 1.0
    X, Y, Z = coords(n, h)
    # a compactly supported field, exactly vacuum beyond the ellipsoid r = 1.8,
    # which stays inside the interior (with its stencil) after the shift
    r = np.sqrt((X / 1.2) ** 2 + Y ** 2 + (Z / 0.9) ** 2)
    f = np.where(r < 1.8, PI * (1 - r / 1.8) ** 3, 0.0)
    rr = np.sqrt(X * X + Y * Y + Z * Z)
    sr = np.where(rr > 0, np.sin(f) / np.where(rr > 0, rr, 1.0), 0.0)
    phi = np.ascontiguousarray(np.stack([np.cos(f), sr * X, sr * Y, sr * Z], axis=-1))
    o = oracle.observables(phi, h, m)
    shift = (2, -2, 1)
    o2 = oracle.observables(np.ascontiguousarray(np.roll(phi, shift, axis=(0, 1, 2))), h, m)
    assert np.allclose(o2["X"], o["X"] + h * np.array(shift), atol=1e-10)
    for k in ("B", "R", "D", "E"):
        assert o2[k] == pytest.approx(o[k], rel=1e-9), k
    for k in ("Q", "U", "V", "W"):
        assert np.allclose(o2[k], o[k], rtol=1e-9, atol=1e-9 * np.max(np.abs(o[k]))), k


def rotation(axis, angle):
    c, s = math.cos(angle), math.sin(angle)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + s * K + (1 - c) * (K @ K)


def deformed_hedgehog(X, Y, Z, s0=0.8):
    """B=1, not spherical: f of an ellipsoidal radius, pions along rhat."""
    s = np.sqrt((X / 1.25) ** 2 + Y ** 2 + (Z / 0.85) ** 2)
    f = PI * (1.0 - np.tanh(s / s0))
    r = np.sqrt(X * X + Y * Y + Z * Z)
    sr = np.where(r > 0, np.sin(f) / np.where(r > 0, r, 1.0), 0.0)
    return np.stack([np.cos(f), sr * X, sr * Y, sr * Z], axis=-1)


def test_inertia_tensors_are_the_kinetic_energy_of_rotations_and_isorotations():
    """T(phi_t) for phi_t = a.K + b.G, with K_a = (0, e_a x pi) the
    isorotation and G_b = -(e_b x r) . grad phi the rotation generator on the
    lattice (tangent lattice derivative), equals a U a/2 + b V b/2 - a W b to
    rounding, for every pair of axes."""
    n, h, m = (30, 30, 30), 0.2, 1.0
    X, Y, Z = coords(n, h)
    phi = np.ascontiguousarray(deformed_hedgehog(X, Y, Z))
    o = oracle.observables(phi, h, m)
    assert np.max(np.abs(o["X"])) < 1e-12  # reflection symmetric: rotations about X_c = 0
    p = interior(phi)
    d = [fd1(phi, h, i) for i in range(3)]
    d = [di - np.sum(p * di, axis=-1, keepdims=True) * p for di in d]
    rv = [interior(X), interior(Y), interior(Z)]
    e = np.eye(3)

    def pad(v):  # kinetic() takes full-lattice velocities
        out = np.zeros_like(phi)
        out[2:-2, 2:-2, 2:-2] = v
        return out

    def K(a):
        v = np.zeros_like(phi)
        v[..., 1:] = np.cross(a, phi[..., 1:])
        return v

    def G(b):  # -(b x r) . grad phi
        bxr = np.cross(b, np.stack(rv, axis=-1))
        return pad(-sum(bxr[..., l:l + 1] * d[l] for l in range(3)))

    for i in range(3):
        for j in range(3):
            a = e[i] + e[j]
            assert kinetic(phi, K(a), h) == pytest.approx(0.5 * a @ o["U"] @ a, rel=1e-10), (i, j)
            assert kinetic(phi, G(a), h) == pytest.approx(0.5 * a @ o["V"] @ a, rel=1e-10), (i, j)
            T = kinetic(phi, K(e[i]) + G(e[j]), h)
            assert 0.5 * o["U"][i, i] + 0.5 * o["V"][j, j] - T == pytest.approx(
                o["W"][i, j], abs=1e-10 * np.max(np.abs(o["V"]))), (i, j)
    # the deformation splits the spin tensor's eigenvalues
    ev = np.linalg.eigvalsh(0.5 * (o["V"] + o["V"].T))
    assert ev[-1] - ev[0] > 0.05 * ev[-1]


def test_lattice_rotation_generator_is_the_derivative_of_a_rotated_field():
    """b V b / 2 against the kinetic energy of the exactly rotated analytic
    field phi(R(-t b) x): equal up to the lattice derivative's error."""
    n, h, m = (36, 36, 36), 0.2, 1.0
    X, Y, Z = coords(n, h)
    pts = np.stack([X, Y, Z], axis=-1)
    phi = np.ascontiguousarray(deformed_hedgehog(X, Y, Z, s0=1.5))
    o = oracle.observables(phi, h, m)
    eps = 1e-4
    for b in (np.array([1.0, 0, 0]), np.array([0, 1.0, 1.0]), np.array([1.0, -1.0, 0.5])):
        nb = np.linalg.norm(b)
        fwd = deformed_hedgehog(*np.moveaxis(pts @ rotation(b / nb, -eps * nb).T, -1, 0), s0=1.5)
        bwd = deformed_hedgehog(*np.moveaxis(pts @ rotation(b / nb, eps * nb).T, -1, 0), s0=1.5)
        T = kinetic(phi, (fwd - bwd) / (2 * eps), h)
        assert T == pytest.approx(0.5 * b @ o["V"] @ b, rel=2e-3), b
