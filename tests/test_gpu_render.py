"""GPU volume render of the baryon density (Section 6.2) against the oracle:
the per-site volume, the ray-march on the same volume (bit for bit) and the
whole render from a field."""
import numpy as np
import pytest

import oracle
import paper_2604_25876_gb300 as sk
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def rotation(seed):
    q = np.random.default_rng(seed).normal(size=4)
    a, b, c, d = q / np.linalg.norm(q)
    return np.array([[a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
                     [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
                     [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d]])


def field_on_gpu(phi, h, prec):
    lat = sk.Lattice(phi.shape[:3], h, 1.0, prec)
    st = sk.State(lat, DEV)
    sk.load_field(lat, st, phi)
    return lat, st


def generic_field(n, h, seed=3):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(-0.7, 0.7, size=(3, 3))
    q = rng.normal(size=(3, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return oracle.seed_product(n, h, pos, q, 0.8, False)


@pytest.mark.parametrize("prec", [64, 32])
def test_volume_matches_oracle(prec):
    n, h = (27, 33, 30), 0.25  # ragged: no side a multiple of a warp or tile
    phi = generic_field(n, h)
    if prec == 32:
        phi = phi.astype(np.float32).astype(np.float64)  # the values the GPU holds
    lat, st = field_on_gpu(phi, h, prec)
    vol = sk.render_volume(lat, st).cpu().numpy()
    ref = oracle.render_volume_from_field(phi, h)
    # the pion unit vector takes the same IEEE operations on both sides
    assert np.array_equal(vol[..., 1:], ref[..., 1:])
    # B0 / max B0: lattice derivatives summed in another order
    assert np.max(np.abs(vol[..., 0] - ref[..., 0])) <= 1e-12
    assert np.max(vol[..., 0]) == pytest.approx(1.0, abs=1e-15)
    assert np.all(vol[:2, ..., 0] == 0) and np.all(vol[-2:, ..., 0] == 0)
    assert np.all(vol[:, :, :2, 0] == 0) and np.all(vol[:, :, -2:, 0] == 0)


CASES = [
    dict(width=64, height=48),
    dict(width=37, height=53, view=rotation(1), levelset=0.1, step=0.013),
    dict(width=1, height=1, view=rotation(2)),
    dict(width=80, height=20, view=rotation(3), levelset=0.5, transfer_scale=9.0, brightness=1.7,
         step=0.004),
    dict(width=45, height=45, view=rotation(4), levelset=-0.05, transfer_scale=2.0, step=0.03),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_rays_match_oracle_bit_for_bit_on_the_same_volume(case):
    p = CASES[case]
    n, h = (27, 33, 30), 0.25
    vol = oracle.render_volume_from_field(generic_field(n, h, seed=10 + case), h)
    img = sk.render_rays(torch.from_numpy(vol).to(DEV), sk.render_params(**p)).cpu().numpy()
    ref = oracle.render_volume(vol, **p).astype(np.float32)
    # no contraction on either side: the same rounding, the same decisions
    bad = np.argwhere(img != ref)
    assert bad.size == 0, (len(bad), bad[:5], img[tuple(bad[0][:2])], ref[tuple(bad[0][:2])])
    assert np.all((img >= 0) & (img <= 1))


def test_render_from_the_128_cubed_b4_field_matches_oracle():
    wl = workloads.b4_cubic_128()
    lat = sk.Lattice(wl.n, wl.h, wl.m, 32)
    st = sk.State(lat, DEV)
    sk.init_field(lat, sk.Seed.from_spec(wl.seed), st)
    sk.flow_step(lat, wl.dt, 40, sk.ARRESTED, st, report=False)
    p = dict(width=96, height=72, view=rotation(7), step=0.008)
    img = sk.render(lat, st, sk.render_params(**p)).cpu().numpy()
    phi = st.field().cpu().numpy().astype(np.float64)
    ref = oracle.render_volume(oracle.render_volume_from_field(phi, wl.h), **p)
    # volumes agree to ~1e-15: a skip or stop decision flips only at a value
    # within rounding of its threshold
    assert np.max(np.abs(img - ref)) <= 1e-6
    assert np.max(img[..., 3]) > 0.5  # the skyrmion is in the picture


def test_vacuum_renders_black_and_a_repeated_render_is_identical():
    lat = sk.Lattice((20, 20, 20), 0.3, 1.0, 64)
    st = sk.State(lat, DEV)
    sk.init_field(lat, sk.Seed.vacuum(), st)
    img = sk.render(lat, st, sk.render_params(16, 16))
    assert torch.count_nonzero(img).item() == 0
    # a field with baryon density: two renders are bitwise the same
    phi = generic_field((24, 26, 28), 0.3, seed=9)
    lat, st = field_on_gpu(phi, 0.3, 64)
    p = sk.render_params(33, 17, view=rotation(5))
    a = sk.render(lat, st, p)
    assert torch.equal(a, sk.render(lat, st, p)) and torch.count_nonzero(a).item() > 0
