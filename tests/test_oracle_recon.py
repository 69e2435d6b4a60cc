"""Pins of the oracle's reconstruction by dilation and h-dome (Table I,
ReconToNuclei; Vincent's MR).  The oracle uses Vincent's hybrid
sweep+queue algorithm; the pins are the plain definition iterated to
stability, the order invariants, idempotence and closed forms."""
import numpy as np
import pytest

import oracle
from tests import brute


def _rand_pair(rng, H, W, levels=256, smooth=False):
    mask = rng.integers(0, levels, (H, W)).astype(np.uint8)
    if smooth:
        mask = np.minimum(255, mask // 8 + 100).astype(np.uint8)
    marker = np.minimum(mask, rng.integers(0, levels, (H, W))).astype(np.uint8)
    return marker, mask


@pytest.mark.parametrize("seed", range(12))
def test_equals_iterated_definition_random(seed):
    rng = np.random.default_rng(seed)
    H, W = int(rng.integers(1, 17)), int(rng.integers(1, 17))
    marker, mask = _rand_pair(rng, H, W, levels=int(rng.choice([2, 4, 256])))
    ref, _ = brute.recon_iterated(marker, mask)
    assert np.array_equal(oracle.recon(marker, mask), ref)


@pytest.mark.parametrize("seed", range(4))
def test_equals_iterated_definition_128(seed):
    rng = np.random.default_rng(100 + seed)
    mask = rng.integers(0, 256, (128, 128)).astype(np.uint8)
    marker = np.where(rng.random((128, 128)) < 0.01, mask, 0).astype(np.uint8)
    ref, it = brute.recon_iterated(marker, mask)
    assert it > 3
    got = oracle.recon(marker, mask)
    assert np.array_equal(got, ref)
    plain, it2 = oracle.recon_plain(marker, mask)
    assert np.array_equal(plain, ref) and it2 == it


def test_invariants_and_idempotence():
    rng = np.random.default_rng(7)
    for _ in range(20):
        marker, mask = _rand_pair(rng, 24, 31)
        R = oracle.recon(marker, mask)
        assert np.all(marker <= R) and np.all(R <= mask)
        assert np.array_equal(oracle.recon(R, mask), R)


def test_diagonal_only_connection_propagates():
    # two bright cells touching only at a corner: 8-connectivity must join them
    mask = np.zeros((4, 4), np.uint8)
    mask[0:2, 0:2] = 50
    mask[2:4, 2:4] = 50
    marker = np.zeros_like(mask)
    marker[0, 0] = 50
    R = oracle.recon(marker, mask)
    assert np.all(R[2:4, 2:4] == 50)


def test_flat_plateaus_are_constant():
    mask = np.zeros((20, 20), np.uint8)
    mask[3:9, 3:9] = 120
    mask[12:18, 10:17] = 80
    mask[2, 15] = 200
    marker = np.maximum(mask.astype(int) - 20, 0).astype(np.uint8)
    R = oracle.recon(marker, mask)
    assert len(np.unique(R[3:9, 3:9])) == 1 and R[4, 4] == 100
    assert len(np.unique(R[12:18, 10:17])) == 1 and R[13, 13] == 60


@pytest.mark.parametrize("W,h", [(40, 20), (300, 20), (25, 7)])
def test_ramp_closed_form(W, h):
    # mask(x) = x on a monotone ramp; the best source is the top end, so
    # R(x) = min(x, W-1-h) and the dome is max(0, x-(W-1-h))
    mask = np.tile(np.minimum(np.arange(W), 255), (3, 1)).astype(np.uint8)
    hem = mask
    R, fg = oracle.hdome(hem, h=h, thr=10)
    x = np.minimum(np.arange(W), 255)
    top = x.max()
    assert np.array_equal(R[1], np.minimum(x, top - h))
    assert np.array_equal(fg[1], (x - np.minimum(x, top - h) >= 10).astype(np.uint8))


def test_marker_above_mask_rejected():
    with pytest.raises(ValueError):
        oracle.recon(np.full((2, 2), 5, np.uint8), np.full((2, 2), 4, np.uint8))


@pytest.mark.parametrize("seed", range(4))
def test_hdome_matches_brute(seed):
    rng = np.random.default_rng(40 + seed)
    hem = rng.integers(0, 256, (20, 23)).astype(np.uint8)
    R, fg = oracle.hdome(hem, h=20, thr=10)
    bR, bfg = brute.hdome_fg(hem, 20, 10)
    assert np.array_equal(R, bR) and np.array_equal(fg, bfg)


def test_hdome_threshold_is_inclusive():
    # a plateau exactly 10 above its surround with h=10 has dome 10 -> foreground
    hem = np.full((9, 9), 30, np.uint8)
    hem[3:6, 3:6] = 40
    _, fg = oracle.hdome(hem, h=10, thr=10)
    assert fg[4, 4] == 1 and fg.sum() == 9
    _, fg = oracle.hdome(hem, h=10, thr=11)
    assert fg.sum() == 0


# ---- the front-distance instrument (plain iteration, evaluated where it can change)

@pytest.mark.parametrize("seed", range(8))
def test_rounds_equals_iterated_definition(seed):
    rng = np.random.default_rng(300 + seed)
    H, W = int(rng.integers(1, 48)), int(rng.integers(1, 48))
    mask = rng.integers(0, 256, (H, W)).astype(np.uint8)
    if seed % 2:
        mask = (rng.integers(0, 3, (H, W)) * 100).astype(np.uint8)
    marker = np.where(rng.random((H, W)) < 0.05, mask, 0).astype(np.uint8)
    ref, it = brute.recon_iterated(marker, mask)
    got, steps, evals = oracle.recon_rounds(marker, mask)
    assert np.array_equal(got, ref)
    assert steps == it
    assert evals >= H * W


@pytest.mark.parametrize("N", [1, 2, 9, 40])
def test_rounds_front_distance_closed_form(N):
    """One seed in the corner of a flat square mask: the front needs the
    chessboard distance to the far corner, N-1 steps (2N-2 if propagation
    were 4-connected); along a single row it needs W-1 steps."""
    mask = np.full((N, N), 100, np.uint8)
    marker = np.zeros((N, N), np.uint8)
    marker[0, 0] = 100
    R, steps, _ = oracle.recon_rounds(marker, mask)
    assert (R == 100).all() and steps == N - 1
    row = np.full((1, 3 * N), 7, np.uint8)
    mrow = np.zeros_like(row)
    mrow[0, -1] = 7
    R, steps, _ = oracle.recon_rounds(mrow, row)
    assert (R == 7).all() and steps == 3 * N - 1


def test_worst_case_front_travels_beyond_2000px():
    """Acceptance of the worst-case workload: in its h-dome reconstruction
    (h = 20) the slowest front travels more than 2000 px, and the result
    equals Vincent's."""
    import synth
    hem8 = oracle.deconv(synth.cfg4(0))
    marker = np.maximum(hem8.astype(np.int32) - 20, 0).astype(np.uint8)
    R, steps, _ = oracle.recon_rounds(marker, hem8)
    assert steps > 2000, steps
    assert np.array_equal(R, oracle.recon(marker, hem8))
