"""Pins of fill-holes (Table I FillHoles) and labelling with the area filter
(Table I BWLabel, AreaThreshold): union-find restatements, scipy's labelling
as a library special case, and hand cases."""
import numpy as np
import pytest
from scipy import ndimage

import oracle
from tests import brute


def test_fill_hand_cases():
    ring = np.zeros((7, 7), np.uint8)
    ring[1:6, 1:6] = 1
    ring[2:5, 2:5] = 0
    assert oracle.fill_holes(ring)[3, 3] == 1
    # diamond joined only diagonally: background inside is 4-enclosed -> hole
    d = np.zeros((5, 5), np.uint8)
    d[1, 2] = d[2, 1] = d[2, 3] = d[3, 2] = 1
    f = oracle.fill_holes(d)
    assert f[2, 2] == 1 and f[0, 0] == 0
    # a hole that touches the image border is not a hole
    u = np.zeros((5, 5), np.uint8)
    u[:, 1] = u[:, 3] = u[4, :] = 1
    assert oracle.fill_holes(u)[0, 2] == 0 and oracle.fill_holes(u)[2, 2] == 0
    assert oracle.fill_holes(np.ones((4, 6), np.uint8)).all()
    assert not oracle.fill_holes(np.zeros((4, 6), np.uint8)).any()


@pytest.mark.parametrize("seed", range(20))
def test_fill_random_vs_unionfind(seed):
    rng = np.random.default_rng(seed)
    H, W = int(rng.integers(1, 17)), int(rng.integers(1, 17))
    fg = (rng.random((H, W)) < rng.uniform(0.2, 0.8)).astype(np.uint8)
    assert np.array_equal(oracle.fill_holes(fg), brute.fill_holes(fg))


def test_fill_vs_scipy_4conn():
    rng = np.random.default_rng(3)
    fg = (rng.random((200, 150)) < 0.55).astype(np.uint8)
    lab, n = ndimage.label(fg == 0, structure=ndimage.generate_binary_structure(2, 1))
    border = set(np.unique(np.concatenate([lab[0], lab[-1], lab[:, 0], lab[:, -1]]))) - {0}
    holes = (lab > 0) & ~np.isin(lab, list(border))
    assert np.array_equal(oracle.fill_holes(fg), (fg.astype(bool) | holes).astype(np.uint8))


@pytest.mark.parametrize("seed", range(20))
def test_label_random_vs_unionfind(seed):
    rng = np.random.default_rng(seed)
    H, W = int(rng.integers(1, 20)), int(rng.integers(1, 20))
    m = (rng.random((H, W)) < rng.uniform(0.2, 0.7)).astype(np.uint8)
    amin, amax = int(rng.integers(1, 4)), int(rng.integers(3, 30))
    lab, K = oracle.label(m, amin, amax)
    blab, bK = brute.label(m, amin, amax)
    assert K == bK and np.array_equal(lab, blab)


def test_label_vs_scipy_and_order():
    rng = np.random.default_rng(11)
    m = (rng.random((300, 257)) < 0.45).astype(np.uint8)
    lab, K = oracle.label(m, 20, 1500)
    slab, n = ndimage.label(m, structure=np.ones((3, 3)))
    areas = ndimage.sum(np.ones_like(slab), slab, index=np.arange(1, n + 1))
    keep = [i + 1 for i in range(n) if 20 <= areas[i] <= 1500]
    first = {c: np.flatnonzero(slab.ravel() == c)[0] for c in keep}
    order = sorted(keep, key=lambda c: first[c])
    ref = np.zeros_like(lab)
    for k, c in enumerate(order):
        ref[slab == c] = k + 1
    assert K == len(keep) and np.array_equal(lab, ref)
    # first pixels are increasing in label order
    firsts = [np.flatnonzero(lab.ravel() == k)[0] for k in range(1, K + 1)]
    assert firsts == sorted(firsts)


def test_label_area_bounds_inclusive():
    m = np.zeros((10, 30), np.uint8)
    m[1, 0:20] = 1       # area 20: kept
    m[4, 0:19] = 1       # area 19: dropped
    m[7, 0:21] = 1       # area 21 with amax 21: kept
    lab, K = oracle.label(m, 20, 21)
    assert K == 2 and lab[1, 0] == 1 and lab[4, 0] == 0 and lab[7, 0] == 2
