"""Pins of the oracle's headless volume render of the baryon density
(Section 6.2): the sampler, the transfer function and the front-to-back
compositing against closed forms, and invariances of the camera model."""
import math

import numpy as np
import pytest

import oracle


def slab_volume(n, b, pion=(1.0, 0.0, 0.0)):
    vol = np.zeros(tuple(n) + (4,))
    vol[..., 0] = b
    vol[..., 1:] = pion
    return vol


def test_sampler_is_exact_on_lattice_points_and_multilinear_fields_and_clamps():
    n = (7, 9, 8)
    rng = np.random.default_rng(1)
    vol = rng.normal(size=tuple(n) + (4,))
    for idx in [(0, 0, 0), (6, 8, 7), (3, 4, 5), (1, 7, 2)]:
        assert np.array_equal(oracle.render_sample(vol, idx), vol[idx])
    # trilinear interpolation reproduces any function linear in each coordinate
    gx, gy, gz = np.meshgrid(*[np.arange(k, dtype=float) for k in n], indexing="ij")
    c = rng.normal(size=(8, 4))

    def f(x, y, z):  # linear in each coordinate, 4 components
        x, y, z = (np.asarray(v, dtype=float)[..., None] for v in (x, y, z))
        return (c[0] + c[1] * x + c[2] * y + c[3] * z + c[4] * x * y + c[5] * x * z
                + c[6] * y * z + c[7] * x * y * z)

    lin = f(gx, gy, gz)
    for g in rng.uniform(0, 1, size=(20, 3)) * (np.array(n) - 1):
        assert np.allclose(oracle.render_sample(lin, g), f(*g), rtol=1e-12, atol=1e-12)
    # outside the lattice the sample is that of the nearest face
    assert np.array_equal(oracle.render_sample(vol, (-3.0, 4.0, 5.0)), vol[0, 4, 5])
    assert np.array_equal(oracle.render_sample(vol, (6.0, 40.0, 7.5)), vol[6, 8, 7])


@pytest.mark.parametrize("b,step", [(0.3, 0.01), (0.45, 0.02), (0.9, 0.005)])
def test_uniform_slab_matches_the_compositing_closed_form(b, step):
    n = (17, 17, 17)
    W = H = 9  # the centre pixel's ray runs along -z through the box centre
    level, scale = 0.2, 4.0
    img = oracle.render_volume(slab_volume(n, b), W, H, levelset=level, transfer_scale=scale,
                               step=step)
    inp = (b - level) * scale
    # the centre ray enters the box [-1, 1]^3 at t = 3 (eye at z = 4) and leaves at t = 5
    nsamples = int(math.floor((5.0 - 3.0) / step + 1e-9)) + 1
    alpha, red = 0.0, 0.0
    for _ in range(nsamples):
        red += inp * inp * (1 - alpha)
        alpha += inp * (1 - alpha)
        if alpha > 0.95:
            break
    px = img[H // 2, W // 2]
    assert px[3] == pytest.approx(min(alpha, 1.0), rel=1e-12)
    assert px[0] == pytest.approx(min(red, 1.0), rel=1e-12)
    assert px[1] == 0.0 and px[2] == 0.0
    # closed form of the same recursion before termination: alpha_k = 1 - (1 - inp)^k
    k = next((j for j in range(1, nsamples + 1) if 1 - (1 - inp) ** j > 0.95), nsamples)
    assert px[3] == pytest.approx(min(1 - (1 - inp) ** k, 1.0), rel=1e-9)


def test_density_below_the_levelset_is_not_rendered_and_brightness_scales():
    n = (12, 12, 12)
    assert not oracle.render_volume(slab_volume(n, 0.19), 16, 16, levelset=0.2).any()
    vol = slab_volume(n, 0.22, pion=(0.6, 0.0, 0.8))
    a = oracle.render_volume(vol, 16, 16, brightness=1.0)
    b = oracle.render_volume(vol, 16, 16, brightness=0.5)
    assert np.allclose(b, 0.5 * a, rtol=1e-14, atol=0.0) and a.max() < 1.0


def rot_z_volume(vol):
    """vol'(g) = vol(R^-1 g) for R the +90 degree rotation about z."""
    return np.ascontiguousarray(np.flip(vol, axis=1).transpose(1, 0, 2, 3))


def test_rotating_volume_and_camera_together_leaves_the_image_unchanged():
    n, h = (24, 24, 24), 0.3
    rng = np.random.default_rng(2)
    pos = rng.uniform(-1.0, 1.0, size=(3, 3))
    q = rng.normal(size=(3, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    phi = oracle.seed_product(n, h, pos, q, 1.0, False)
    vol = oracle.render_volume_from_field(phi, h)
    c, s = math.cos(0.4), math.sin(0.4)
    view = np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]])  # a tilted camera
    R = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    img = oracle.render_volume(vol, 40, 32, view=view, levelset=0.1)
    img2 = oracle.render_volume(rot_z_volume(vol), 40, 32, view=R @ view, levelset=0.1)
    assert img[..., 3].max() > 0.5
    assert np.allclose(img2, img, rtol=0, atol=1e-12)


def test_volume_from_field_is_the_normalised_baryon_density_and_unit_pions():
    n, h = (20, 22, 18), 0.3
    phi = oracle.seed_rational_map(n, h, 1, 1.0)
    vol = oracle.render_volume_from_field(phi, h)
    _, _, d = oracle.forces(phi, h, 0.0)
    b = d[..., 3]
    assert vol[..., 0].max() == 1.0
    assert np.allclose(vol[..., 0], b / b.max(), rtol=1e-14, atol=1e-15)
    pion = phi[..., 1:]
    norm = np.linalg.norm(pion, axis=-1)
    mask = norm > 0
    assert np.allclose(vol[mask][:, 1:], pion[mask] / norm[mask][:, None], atol=1e-15)
    assert not vol[~mask][:, 1:].any()
    # the vacuum renders nothing
    vac = oracle.render_volume_from_field(oracle.seed_vacuum(n), h)
    assert not vac[..., 0].any()
