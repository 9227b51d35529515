"""Pins of the oracle's placed rational-map Skyrmions and ordered product
(Section 4.1, Section 4.2 Eq. "Product ansatz", and the position and Euler-angle
placement of the configuration files, Section 7.3)."""
import math

import numpy as np
import pytest

import oracle


def euler_zyz(a1, a2, a3):
    """Rotation about z by a1, then about y by a2, then about z by a3."""
    def rz(t):
        c, s = math.cos(t), math.sin(t)
        return np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]])

    def ry(t):
        c, s = math.cos(t), math.sin(t)
        return np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]])
    return rz(a3) @ ry(a2) @ rz(a1)


def test_unplaced_map_is_the_seed():
    n, h = (17, 19, 21), 0.3
    for B, s in ((1, 0.9), (4, 1.5)):
        got = oracle.rational_map_field(n, h, B, s)
        oracle.apply_vacuum_boundary(got)
        assert np.array_equal(got, oracle.seed_rational_map(n, h, B, s))


def test_translation_by_whole_sites_shifts_the_array():
    n, h, k = (30, 24, 26), 0.25, (3, -2, 1)
    base = oracle.rational_map_field(n, h, 4, 1.5)
    moved = oracle.rational_map_field(n, h, 4, 1.5, X=np.array(k) * h)
    # moved[i] = base[i - k] wherever both are on the lattice
    sl_new = tuple(slice(max(0, kk), n_ + min(0, kk)) for kk, n_ in zip(k, n))
    sl_old = tuple(slice(max(0, -kk), n_ - max(0, kk)) for kk, n_ in zip(k, n))
    np.testing.assert_allclose(moved[sl_new], base[sl_old], rtol=0, atol=1e-14)


def test_quarter_turn_about_z_rotates_the_array():
    n, h = (23, 23, 21), 0.3   # equal x and y sides: the turn maps sites to sites
    R = euler_zyz(math.pi / 2, 0.0, 0.0)
    base = oracle.rational_map_field(n, h, 4, 1.5)
    turned = oracle.rational_map_field(n, h, 4, 1.5, R=R)
    # U_rot(x) = U(R^T x): the site (i, j) takes the value of (j, N-1-i)
    expect = np.empty_like(base)
    N = n[0]
    for i in range(N):
        for j in range(N):
            expect[i, j] = base[j, N - 1 - i]
    np.testing.assert_allclose(turned, expect, rtol=0, atol=1e-13)
    # a turn by (a1, 0, 0) equals one by (0, 0, a1) (the second angle vanishing)
    np.testing.assert_allclose(oracle.rational_map_field(n, h, 4, 1.5, R=euler_zyz(0, 0, math.pi / 2)),
                               turned, rtol=0, atol=1e-15)


def test_ordered_product_identity_associativity_and_charge():
    n, h = (56, 40, 40), 0.2
    a = oracle.rational_map_field(n, h, 4, 0.8, X=(-2.0, 0, 0))
    b = oracle.rational_map_field(n, h, 4, 0.8, X=(2.0, 0, 0), R=euler_zyz(1.2, 0.7, -0.4))
    c = oracle.rational_map_field(n, h, 1, 0.8, X=(0, 1.0, 0))
    vac = oracle.seed_vacuum(n)
    assert np.array_equal(oracle.field_product(a, vac), a)
    assert np.array_equal(oracle.field_product(vac, b), b)
    ab_c = oracle.field_product(oracle.field_product(a, b), c)
    a_bc = oracle.field_product(a, oracle.field_product(b, c))
    np.testing.assert_allclose(ab_c, a_bc, rtol=0, atol=1e-14)
    # unit quaternions stay unit
    assert np.max(np.abs(np.linalg.norm(ab_c, axis=-1) - 1)) < 1e-14
    # the product is not commutative where the constituents overlap ...
    assert np.max(np.abs(oracle.field_product(a, c) - oracle.field_product(c, a))) > 1e-3
    # ... and its charge is the sum of the charges (Section 4.2).  On this
    # coarse lattice each cube carries about 3.3 of its 4 units; the sum rule
    # holds to the lattice error of the overlap region.
    charge = lambda f: oracle.energy(oracle.apply_vacuum_boundary(f.copy()), h, 1.0)["B"]
    Ba, Bb, Bab = charge(a), charge(b), charge(oracle.field_product(a, b))
    assert 3.0 < Ba < 4.0 and 3.0 < Bb < 4.0
    assert abs(Bab - (Ba + Bb)) < 2e-3, (Ba, Bb, Bab)
