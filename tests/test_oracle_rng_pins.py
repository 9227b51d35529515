"""Pins of the oracle's random-number and noise-seed steps against values
fixed outside the oracle.

The smoothed-noise start of the batched workload (i.i.d. normal noise in a
ball, Gaussian smoothing, per-component rescale, phi = normalise(vacuum +
noise)) draws its numbers from SplitMix64 (Steele, Lea and Flood, OOPSLA
2014) in counter form and turns pairs of them into normals by Box-Muller.
Each step is checked here against something the oracle does not compute:

* SplitMix64: the first outputs of the published generator from two states
  (state 0, and the 1234567 sequence of the public SplitMix64 task);
* Box-Muller: the closed form evaluated in the test on the uniforms that
  those published outputs give;
* smoothing: a unit spike must come out as the outer product of three
  normalised 1D Gaussian weight vectors truncated at ceil(4 sigma / h), and a
  random field must match SciPy's separable correlation with zero fill;
* rescale: unit standard deviation per component over the ball sites, and the
  whole noise field rebuilt from the normals with SciPy.

Each pin is also shown to reject the plausible mistakes (a truncation radius
off by one, a skipped axis, a missing rescale).
"""
import math

import numpy as np
import pytest
from scipy import ndimage

import oracle

# First outputs of SplitMix64 from state 0 (the generator's reference
# implementation: x += 0x9E3779B97F4A7C15, then the two xor-shift-multiply
# rounds and a final xor-shift).
SPLITMIX_STATE0 = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F,
                   0xF88BB8A8724C81EC, 0x1B39896A51A8749B]
# ... and from state 1234567.
SPLITMIX_1234567 = [6457827717110365317, 3203168211198807973, 9817491932198370423,
                    4593380528125082431, 16408922859458223821]


@pytest.mark.parametrize("state,expect", [(0, SPLITMIX_STATE0), (1234567, SPLITMIX_1234567)])
def test_splitmix64_matches_published_outputs(state, expect):
    got = [oracle.splitmix64(state, i) for i in range(len(expect))]
    assert got == expect


def box_muller(o1: int, o2: int) -> float:
    """Normal from two 64-bit outputs: u1 in (0, 1] and u2 in [0, 1) from the
    top 53 bits, z = sqrt(-2 ln u1) cos(2 pi u2)."""
    u1 = ((o1 >> 11) + 1) / 2.0 ** 53
    u2 = (o2 >> 11) / 2.0 ** 53
    return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)


def test_normal_is_box_muller_of_published_outputs():
    # normal i of a stream uses outputs 2i and 2i + 1
    for i in range(2):
        expect = box_muller(SPLITMIX_1234567[2 * i], SPLITMIX_1234567[2 * i + 1])
        assert oracle.normal(1234567, i) == pytest.approx(expect, rel=1e-15, abs=1e-15)
    expect = box_muller(SPLITMIX_STATE0[2], SPLITMIX_STATE0[3])
    assert oracle.normal(0, 1) == pytest.approx(expect, rel=1e-15, abs=1e-15)


def weights(h, sigma, K):
    k = np.arange(-K, K + 1)
    w = np.exp(-(k * h) ** 2 / (2.0 * sigma ** 2))
    return w / w.sum()


# 4 sigma / h = 6.4: ceil gives 7, floor and round give 6
H, SIGMA = 0.25, 0.4
K = math.ceil(4 * SIGMA / H)


def test_smoothing_of_a_spike_is_the_truncated_gaussian_product():
    n = (21, 19, 23)
    c = (10, 9, 11)
    field = np.zeros(n + (4,))
    field[c + (2,)] = 1.0
    out = oracle.gaussian_smooth(field, H, SIGMA)

    def product(Kt):
        w = weights(H, SIGMA, Kt)
        expect = np.zeros(n)
        sl = tuple(slice(ci - Kt, ci + Kt + 1) for ci in c)
        expect[sl] = np.einsum("i,j,k->ijk", w, w, w)
        return expect

    np.testing.assert_allclose(out[..., 2], product(K), rtol=0, atol=1e-16)
    assert np.all(out[..., [0, 1, 3]] == 0.0)
    # the pin rejects a truncation radius off by one either way: the 4-sigma
    # tail weights are small (e^-8 of the centre), but far above the pin's
    # 1e-16 tolerance
    for Kt in (K - 1, K + 1):
        assert np.max(np.abs(out[..., 2] - product(Kt))) > 1e-9


def test_smoothing_matches_scipy_separable_correlation_with_zero_fill():
    rng = np.random.default_rng(5)
    n = (17, 14, 19)  # smaller than 2K + 1 along every axis: the box edges matter everywhere
    field = rng.standard_normal(n + (4,))
    out = oracle.gaussian_smooth(field, H, SIGMA)
    w = weights(H, SIGMA, K)
    expect = field
    for axis in range(3):
        expect = ndimage.correlate1d(expect, w, axis=axis, mode="constant", cval=0.0)
    np.testing.assert_allclose(out, expect, rtol=0, atol=1e-13)
    # a skipped axis is caught
    for skip in range(3):
        wrong = field
        for axis in range(3):
            if axis != skip:
                wrong = ndimage.correlate1d(wrong, w, axis=axis, mode="constant", cval=0.0)
        assert np.max(np.abs(out - wrong)) > 1e-2


def ball_mask(n, h, radius):
    ax = [(np.arange(m) - 0.5 * (m - 1)) * h for m in n]
    X, Y, Z = np.meshgrid(*ax, indexing="ij")
    return X * X + Y * Y + Z * Z <= radius * radius


def test_noise_components_rebuilt_from_normals_with_scipy():
    n, h, radius, sigma, seed = (22, 20, 18), 0.3, 2.0, 0.5, 1003
    got = oracle.noise_components(n, h, radius, sigma, seed)
    ball = ball_mask(n, h, radius)
    # i.i.d. normals at ball sites: counter 4 s + c at site s
    raw = np.zeros(n + (4,))
    for s in np.flatnonzero(ball.ravel()):
        idx = np.unravel_index(s, n)
        for c in range(4):
            raw[idx + (c,)] = oracle.normal(seed, 4 * int(s) + c)
    w = weights(h, sigma, math.ceil(4 * sigma / h))
    sm = raw
    for axis in range(3):
        sm = ndimage.correlate1d(sm, w, axis=axis, mode="constant", cval=0.0)
    sd = sm[ball].std(axis=0)  # population standard deviation over ball sites
    expect = sm / sd
    np.testing.assert_allclose(got, expect, rtol=1e-12, atol=1e-14)
    # unit standard deviation per component over the ball sites
    np.testing.assert_allclose(got[ball].std(axis=0), 1.0, rtol=1e-12)
    # without the rescale the smoothed noise is far below unit size
    assert np.all(sm[ball].std(axis=0) < 0.5)


def test_noise_seed_is_normalised_vacuum_plus_noise():
    n, h, radius, sigma, seed = (20, 20, 20), 0.3, 2.0, 0.5, 1004
    noise = oracle.noise_components(n, h, radius, sigma, seed)
    t = noise.copy()
    t[..., 0] += 1.0
    expect = t / np.linalg.norm(t, axis=-1, keepdims=True)
    oracle.apply_vacuum_boundary(expect)
    np.testing.assert_allclose(oracle.seed_noise(n, h, radius, sigma, seed), expect,
                               rtol=0, atol=1e-15)
