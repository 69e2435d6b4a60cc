"""Pins of the oracle's RBC detection (Table I "RBC detection": OpenCV colour
operations and Vincent's MR; our reading: red dominance d = R - max(G, B),
markers d >= t_hi grown through the mask d >= t_lo by 8-connected binary
reconstruction).  Checked against the iterated geodesic dilation and
union-find / SciPy components (tests/brute.py, independent of oracle.c),
hand colours, inclusive thresholds, connectivity cases and invariants."""
import numpy as np
import pytest

import oracle
import synth
from tests import brute


def red(rgb):
    r = rgb.astype(np.int32)
    return r[..., 0] - np.maximum(r[..., 1], r[..., 2])


def rand_rgb(rng, H, W):
    """Random tiles with red blobs: smooth red dominance so that the mask
    has components with and without markers."""
    rgb = rng.integers(0, 256, (H, W, 3)).astype(np.int32)
    base = rng.integers(0, 160, (H, W))
    rgb[..., 0] = np.clip(base + rng.integers(-30, 200, (H, W)), 0, 255)
    rgb[..., 1] = np.clip(base + rng.integers(-20, 20, (H, W)), 0, 255)
    rgb[..., 2] = np.clip(base + rng.integers(-20, 20, (H, W)), 0, 255)
    return rgb.astype(np.uint8)


@pytest.mark.parametrize("seed", range(6))
def test_equals_iterated_binary_reconstruction(seed):
    rng = np.random.default_rng(seed)
    H, W = int(rng.integers(1, 40)), int(rng.integers(1, 40))
    rgb = rand_rgb(rng, H, W)
    d = red(rgb)
    for t_lo, t_hi in ((40, 100), (0, 0), (60, 60), (10, 200), (120, 255)):
        got = oracle.rbc(rgb, t_lo, t_hi)
        want, _ = brute.recon_iterated((d >= t_hi).astype(np.uint8), (d >= t_lo).astype(np.uint8))
        assert np.array_equal(got, want), (t_lo, t_hi)


@pytest.mark.parametrize("seed", range(4))
def test_equals_mask_components_holding_a_marker(seed):
    rng = np.random.default_rng(100 + seed)
    rgb = rand_rgb(rng, 48, 37)
    d = red(rgb)
    t_lo, t_hi = 40, 100
    root = brute.components(d >= t_lo, 8)
    keep = set(root[(d >= t_hi)].tolist())
    want = np.isin(root, list(keep)) & (root >= 0)
    assert np.array_equal(oracle.rbc(rgb, t_lo, t_hi), want.astype(np.uint8))
    ndi = pytest.importorskip("scipy.ndimage")
    lab, n = ndi.label(d >= t_lo, structure=np.ones((3, 3), int))
    hit = np.unique(lab[d >= t_hi])
    assert np.array_equal(oracle.rbc(rgb, t_lo, t_hi), np.isin(lab, hit[hit > 0]).astype(np.uint8))


def test_red_dominance_of_the_workload_colours():
    cols = {(200, 60, 70): 130, (225, 215, 228): -3, (90, 60, 140): -50, (200, 150, 190): 10, (0, 0, 0): 0,
            (255, 0, 0): 255, (0, 255, 255): -255}
    rgb = np.array([list(cols)], np.uint8)
    _, d = oracle.rbc(rgb, detail=True)
    assert d[0].tolist() == list(cols.values())
    assert oracle.rbc(np.full((9, 7, 3), (200, 60, 70), np.uint8)).all()
    for c in ((225, 215, 228), (90, 60, 140), (200, 150, 190)):
        assert not oracle.rbc(np.full((9, 7, 3), c, np.uint8)).any()


def plane(d):
    """An RGB tile whose red dominance is d (>= 0): R = d, G = B = 0."""
    d = np.asarray(d, np.int32)
    rgb = np.zeros(d.shape + (3,), np.uint8)
    rgb[..., 0] = d
    return rgb


def test_thresholds_are_inclusive():
    # a marker at exactly t_hi; its neighbours at t_lo join, at t_lo - 1 do not
    d = np.array([[0, 39, 0, 0, 0],
                  [0, 100, 40, 0, 0],
                  [0, 0, 0, 0, 40]])
    got = oracle.rbc(plane(d), 40, 100)
    assert got.tolist() == [[0, 0, 0, 0, 0], [0, 1, 1, 0, 0], [0, 0, 0, 0, 0]]
    d[1, 1] = 99                                      # below t_hi: no marker, nothing kept
    assert not oracle.rbc(plane(d), 40, 100).any()


def test_connectivity_is_8_and_a_gap_stops_the_flood():
    d = np.zeros((7, 7), np.int32)
    d[0, 0] = 120                                     # marker
    for k in range(1, 5):
        d[k, k] = 50                                  # a diagonal-only chain: joins
    d[6, 6] = 50                                      # beyond a gap at (5, 5): stays out
    d[0, 3] = d[0, 4] = 60                            # a mask run without a marker: stays out
    got = oracle.rbc(plane(d), 40, 100)
    want = np.zeros_like(got)
    for k in range(5):
        want[k, k] = 1
    assert np.array_equal(got, want)


@pytest.mark.parametrize("seed", range(3))
def test_invariants(seed):
    rng = np.random.default_rng(200 + seed)
    rgb = rand_rgb(rng, 64, 64)
    d = red(rgb)
    out = oracle.rbc(rgb, 40, 100).astype(bool)
    assert ((d >= 100) <= out).all() and (out <= (d >= 40)).all()     # marker <= out <= mask
    looser = oracle.rbc(rgb, 20, 100).astype(bool)
    stricter = oracle.rbc(rgb, 40, 140).astype(bool)
    assert (out <= looser).all() and (stricter <= out).all()          # monotone in both thresholds
    # idempotence: reconstructing again under the result changes nothing
    again, _ = brute.recon_iterated(out.astype(np.uint8), out.astype(np.uint8))
    assert np.array_equal(again.astype(bool), out)


def test_workload_tiles():
    """No pixel of the RBC-free workloads (background, nuclei, stroma, the
    ramp corridor) is detected; on a tile with red blood cells, the
    detected components number between 40% of the cells and the cell count
    (the generator starts a clump of 2-5 touching cells on 30% of its
    draws, about 1.75 cells per draw, and a clump is one component)."""
    assert oracle.rbc(synth.cfg0()).sum() == 0
    assert oracle.rbc(synth.tile(1024, 1024, 1000, n_nuclei=190, frac_cluster=0.2, n_stroma=10)).sum() == 0
    assert oracle.rbc(synth.tile(1024, 1024, 4000, n_nuclei=500, frac_chain=0.5, corridor=True)).sum() == 0
    t = synth.tile(1024, 1024, 77, n_nuclei=200, frac_cluster=0.2, n_stroma=10, n_rbc=150)
    out = oracle.rbc(t)
    root = brute.components(out, 8)
    n = len(np.unique(root[root >= 0]))
    assert 0.4 * 150 <= n <= 150, n


def test_bad_arguments():
    rgb = np.zeros((4, 4, 3), np.uint8)
    for lo, hi in ((-1, 10), (50, 40), (0, 256)):
        with pytest.raises(ValueError):
            oracle.rbc(rgb, lo, hi)
