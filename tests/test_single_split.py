"""The work split of a single FP32 lattice (skyrme_single_split_runs, host
only): every (column, x-plane) unit is streamed exactly once, every launched
CTA streams at least one plane, and the lockstep schedule has the structure
that lets neighbouring columns share their halo rows through L2 (waves of
whole columns, then equal heads beside the tails, all starting together).
No GPU is needed: the runs come from the planner and the per-CTA decode the
step kernel uses."""
import numpy as np
import pytest

sk = pytest.importorskip("paper_2604_25876_gb300")

FILL = 4  # pipeline fill planes of a run

SIZES = [(128, 128, 128), (256, 256, 256), (512, 512, 512), (20, 324, 260), (32, 68, 100),
         (32, 32, 32), (20, 21, 22), (9, 5, 5), (300, 100, 40), (60, 500, 36), (1028, 36, 68)]


def geometry(n):
    nyt, nzt, nix = -(-(n[1] - 4) // 16), -(-(n[2] - 4) // 32), n[0] - 4
    return nyt * nzt, nix


def plane_counts(runs):
    counts = np.zeros(runs[:, 0].max() + 1, dtype=np.int64)
    for b, _, x0, x1 in runs:
        counts[b] += x1 - x0 + FILL
    return counts


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("policy", [sk.SPLIT_AUTO, sk.SPLIT_BALANCED, sk.SPLIT_LOCKSTEP])
@pytest.mark.parametrize("grid", [152, 37])
def test_every_unit_is_streamed_once(n, policy, grid):
    ncol, nix = geometry(n)
    runs, chosen = sk.single_split_runs(n, grid, policy)
    assert chosen in (sk.SPLIT_BALANCED, sk.SPLIT_LOCKSTEP)
    if policy == sk.SPLIT_BALANCED:
        assert chosen == sk.SPLIT_BALANCED
    seen = np.zeros((ncol, nix), dtype=np.int64)
    for b, col, x0, x1 in runs:
        assert 0 <= col < ncol and 0 <= x0 < x1 <= nix
        seen[col, x0:x1] += 1
    assert (seen == 1).all()
    ctas = runs[:, 0].max() + 1
    assert ctas <= min(grid, ncol * nix)
    assert set(runs[:, 0]) == set(range(ctas))  # every launched CTA streams
    # each CTA's runs come in streaming order and do not overlap in time
    assert (np.diff(runs[:, 0]) >= 0).all()


@pytest.mark.parametrize("n", SIZES)
def test_auto_is_the_balanced_split(n):
    bal, _ = sk.single_split_runs(n, 152, sk.SPLIT_BALANCED)
    auto, chosen = sk.single_split_runs(n, 152, sk.SPLIT_AUTO)
    assert chosen == sk.SPLIT_BALANCED
    assert np.array_equal(auto, bal)


@pytest.mark.parametrize("n", SIZES)
def test_lockstep_streams_no_more_planes_than_balanced_in_one_wave(n):
    """Where the columns fit in one wave, the heads and tails are balanced as
    well as the balanced split itself (the lockstep schedule costs no planes)."""
    ncol, nix = geometry(n)
    bal, _ = sk.single_split_runs(n, 152, sk.SPLIT_BALANCED)
    lk, chosen = sk.single_split_runs(n, 152, sk.SPLIT_LOCKSTEP)
    if chosen == sk.SPLIT_LOCKSTEP and ncol <= 152:
        assert plane_counts(lk).max() <= plane_counts(bal).max()


@pytest.mark.parametrize("n,G", [((512, 512, 512), 152), ((20, 324, 260), 152),
                                 ((256, 256, 256), 152), ((256, 308, 260), 152),
                                 ((300, 100, 40), 37)])
def test_lockstep_structure(n, G):
    """W = ncol // G waves: CTA b's first W runs are the whole columns
    b, b + G, ...; then CTA b < R = ncol % G streams the head [0, a) of
    column W G + b (one length a for all heads) and the other CTAs the tails
    [a, nix) of those columns, in column order."""
    ncol, nix = geometry(n)
    runs, chosen = sk.single_split_runs(n, G, sk.SPLIT_LOCKSTEP)
    assert chosen == sk.SPLIT_LOCKSTEP
    W, R = divmod(ncol, G)
    by_cta = {}
    for b, col, x0, x1 in runs:
        by_cta.setdefault(int(b), []).append((int(col), int(x0), int(x1)))
    heads = set()
    for b, rs in by_cta.items():
        for w in range(W):
            assert rs[w] == (w * G + b, 0, nix)
        rest = rs[W:]
        if b < R:
            assert len(rest) == 1 and rest[0][0] == W * G + b and rest[0][1] == 0
            heads.add(rest[0][2])
        else:
            for col, x0, x1 in rest:
                assert W * G <= col < ncol and x1 <= nix
    if R:
        assert len(heads) == 1  # every head ends at the same plane a
        a = heads.pop()
        tails = [(c, x0, x1) for b, rs in by_cta.items() if b >= R for (c, x0, x1) in rs[W:]]
        assert all(x0 >= a for _, x0, _ in tails)
        flat = [(c, x) for c, x0, x1 in tails for x in range(x0, x1)]
        assert flat == sorted(flat)  # tail units in column order across the CTAs
    else:
        assert all(len(rs) == W for rs in by_cta.values())


def test_policy_setting_round_trips_and_rejects_unknown_values():
    assert sk.single_split() == sk.SPLIT_AUTO
    try:
        sk.set_single_split(sk.SPLIT_LOCKSTEP)
        assert sk.single_split() == sk.SPLIT_LOCKSTEP
        with pytest.raises(sk.SkyrmeError):
            sk.set_single_split(7)
        assert sk.single_split() == sk.SPLIT_LOCKSTEP
    finally:
        sk.set_single_split(sk.SPLIT_AUTO)
    assert sk.single_split() == sk.SPLIT_AUTO


def test_invalid_geometry_is_rejected():
    with pytest.raises(ValueError):
        sk.single_split_runs((4, 40, 40), 152, sk.SPLIT_AUTO)
    with pytest.raises(ValueError):
        sk.single_split_runs((40, 40, 40), 0, sk.SPLIT_AUTO)
    with pytest.raises(ValueError):
        sk.single_split_runs((40, 40, 40), 152, 5)
