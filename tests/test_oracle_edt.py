"""Pins of the exact squared EDT (Table I, Pre-Watershed distance
transform): all-pairs minimum on small masks, special cases, and scipy's
exact EDT as a library special case."""
import numpy as np
import pytest
from scipy import ndimage

import oracle
from tests import brute

IMAX = 2 ** 31 - 1


@pytest.mark.parametrize("seed", range(16))
def test_allpairs_random(seed):
    rng = np.random.default_rng(seed)
    H, W = int(rng.integers(1, 65)), int(rng.integers(1, 65))
    lab = (rng.random((H, W)) < rng.choice([0.5, 0.9, 0.99])).astype(np.int32)
    if lab.all():
        lab[rng.integers(0, H), rng.integers(0, W)] = 0
    assert np.array_equal(oracle.edt(lab), brute.edt_allpairs(lab))


def test_special_cases():
    lab = np.ones((9, 13), np.int32)
    lab[4, 6] = 0
    gy, gx = np.mgrid[0:9, 0:13]
    assert np.array_equal(oracle.edt(lab), (gy - 4) ** 2 + (gx - 6) ** 2)
    assert (oracle.edt(np.zeros((5, 7), np.int32)) == 0).all()
    assert (oracle.edt(np.ones((5, 7), np.int32)) == IMAX).all()
    row = np.ones((1, 40), np.int32)
    row[0, 0] = 0
    assert np.array_equal(oracle.edt(row)[0], np.arange(40) ** 2)
    col = np.ones((40, 1), np.int32)
    col[-1, 0] = 0
    assert np.array_equal(oracle.edt(col)[:, 0], (39 - np.arange(40)) ** 2)
    one = np.array([[3]], np.int32)
    assert oracle.edt(one)[0, 0] == IMAX


def test_zero_iff_background_and_vs_scipy():
    rng = np.random.default_rng(5)
    lab = (rng.random((333, 211)) < 0.97).astype(np.int32)
    d = oracle.edt(lab)
    assert np.array_equal(d == 0, lab == 0)
    ref = ndimage.distance_transform_edt(lab != 0)
    assert np.array_equal(d, np.rint(ref ** 2).astype(np.int64))
