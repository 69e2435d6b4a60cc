"""Pins of the oracle's morphological opening by a disk (Table I "Morph.
Open", by a 19x19 disk) to things other than itself: SciPy's grey
morphology with the same footprint, the Gauss circle counts of the disk,
duality, and the algebraic properties of an opening."""
import numpy as np
import pytest

import oracle


def disk(r):
    d = np.arange(-r, r + 1)
    return (d[:, None] ** 2 + d[None, :] ** 2) <= r * r


@pytest.mark.parametrize("r", [1, 3, 9])
def test_matches_scipy_grey_morphology(r):
    """Out-of-image pixels take no part: that is constant padding with 255
    for the erosion and 0 for the dilation."""
    ndi = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(100 + r)
    a = rng.integers(0, 256, (67, 91), dtype=np.uint8)
    fp = disk(r)
    e = ndi.grey_erosion(a, footprint=fp, mode="constant", cval=255)
    d = ndi.grey_dilation(a, footprint=fp, mode="constant", cval=0)
    assert np.array_equal(oracle.morph_erode(a, r), e)
    assert np.array_equal(oracle.morph_dilate(a, r), d)
    o = ndi.grey_dilation(e, footprint=fp, mode="constant", cval=0)
    assert np.array_equal(oracle.morph_open(a, r), o)


@pytest.mark.parametrize("r,count", [(1, 5), (2, 13), (3, 29), (5, 81), (9, 253)])
def test_disk_cardinality_is_the_gauss_circle_count(r, count):
    """A lone dark pixel spreads, under erosion, onto exactly the disk: the
    number of lattice points with x^2 + y^2 <= r^2."""
    a = np.full((41, 41), 255, np.uint8)
    a[20, 20] = 0
    assert int((oracle.morph_erode(a, r) == 0).sum()) == count


def test_duality_and_opening_properties():
    rng = np.random.default_rng(7)
    a = rng.integers(0, 256, (53, 77), dtype=np.uint8)
    b = np.maximum(a, rng.integers(0, 256, a.shape, dtype=np.uint8))  # b >= a
    r = 9
    assert np.array_equal(oracle.morph_erode(a, r), 255 - oracle.morph_dilate(255 - a, r))
    o = oracle.morph_open(a, r)
    assert (o <= a).all()                                  # anti-extensive
    assert np.array_equal(oracle.morph_open(o, r), o)      # idempotent
    assert (oracle.morph_open(b, r) >= o).all()            # increasing
    c = np.full((30, 40), 77, np.uint8)
    assert np.array_equal(oracle.morph_open(c, r), c)      # constants are open


def test_unions_of_the_disk_survive_and_small_features_vanish():
    r = 9
    fp = disk(r)
    a = np.full((64, 80), 40, np.uint8)
    a[10:29, 12:31][fp] = 200           # one translate of the disk
    a[14:33, 20:39][fp] = 200           # an overlapping one
    a[40:59, 50:69][fp] = 150           # a separate one, another level
    assert np.array_equal(oracle.morph_open(a, r), a)
    s = np.full((50, 50), 30, np.uint8)
    s[20:25, 20:25] = 220               # a 5x5 square fits no disk of radius 9
    s[5, 40] = 0                        # a dark pinhole is not opened away
    o = oracle.morph_open(s, r)
    assert int(o[20:25, 20:25].max()) == 30
    assert o[5, 40] == 0
