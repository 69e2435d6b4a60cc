"""Pins of the oracle's watershed split (Table I "Pre-Watershed" +
"Watershed") to closed forms and invariants: single convex objects stay
whole, symmetric pairs split on their bisector, chains split into their
discs, the marker height h removes shallow necks, and on a workload tile
every basin is an 8-connected part of exactly one object."""
import numpy as np
import pytest

import oracle
import synth


def discs(H, W, centres, r):
    yy, xx = np.mgrid[:H, :W]
    m = np.zeros((H, W), bool)
    for cy, cx in centres:
        m |= (yy - cy) ** 2 + (xx - cx) ** 2 <= r * r
    return m


def split(mask, h=1):
    lab, K = oracle.label(mask.astype(np.uint8), 1, 10 ** 9)
    out, n = oracle.watershed(lab, oracle.edt(lab), h)
    return lab, K, out, n


@pytest.mark.parametrize("r", [3, 7, 12, 20])
def test_a_disc_stays_whole(r):
    lab, K, out, n = split(discs(2 * r + 9, 2 * r + 11, [(r + 4, r + 5)], r))
    assert (K, n) == (1, 1)
    assert np.array_equal(out, lab)


def test_separate_objects_keep_their_labels():
    lab, K, out, n = split(discs(40, 90, [(20, 15), (20, 45), (20, 75)], 9))
    assert K == n == 3
    assert np.array_equal(out, lab)


@pytest.mark.parametrize("gap", [14, 16, 17, 20])
def test_a_symmetric_pair_splits_on_its_bisector(gap):
    """Centres (20, 20) and (20, 20 + gap), radius 12: pixels left of the
    bisector x = 20 + gap/2 go to the left disc, right of it to the right
    one.  A pixel on it (even gaps) is reached from both sides in the same
    wave, by neighbours of equal squared distance (mirror images), so the
    tie goes to the smaller name: the left disc's marker, whose first pixel
    comes first in raster order (basin 1)."""
    H, W, cx = 41, 20 + gap + 20, 20 + gap / 2
    lab, K, out, n = split(discs(H, W, [(20, 20), (20, 20 + gap)], 12))
    assert (K, n) == (1, 2)
    xx = np.mgrid[:H, :W][1]
    obj = lab > 0
    left, right = obj & (xx < cx), obj & (xx > cx)
    assert set(np.unique(out[left])) == {1}
    assert set(np.unique(out[right])) == {2}
    on = obj & (xx == cx)
    if gap % 2 == 0:
        assert set(np.unique(out[on])) == {1}


def test_a_chain_splits_into_its_discs():
    lab, K, out, n = split(discs(40, 100, [(20, 18), (20, 38), (20, 58), (20, 78)], 12))
    assert (K, n) == (1, 4)
    for b, cx in zip(range(1, 5), (18, 38, 58, 78)):
        assert out[20, cx] == b


def test_the_marker_height_removes_shallow_necks():
    """Centres 14 apart, radius 12: the integer distance falls from 12 at
    the centres to 10 at the neck, a dome of height 2: it survives h = 1 and
    merges at h = 2.  Centres 8 apart leave no saddle at all."""
    m = discs(41, 50, [(20, 20), (20, 34)], 12)
    assert split(m, h=1)[3] == 2
    assert split(m, h=2)[3] == 1
    assert split(discs(41, 50, [(20, 20), (20, 28)], 12), h=0)[3] == 1


def test_thin_objects_are_one_basin():
    m = np.zeros((20, 60), bool)
    m[9:11, 5:55] = True            # a 2-pixel-wide bar: distance 1 everywhere
    m[3:17, 30] = True
    assert split(m)[3] == 1


def test_invariants_on_a_workload_tile():
    rgb = synth.tile(768, 640, 77, n_nuclei=150, frac_cluster=0.4, n_stroma=4)
    r = oracle.seg(rgb)
    lab, K = r["labels"], r["K"]
    out, n = oracle.watershed(lab, r["edt"], 1)
    assert n >= K
    assert np.array_equal(out > 0, lab > 0)
    # every basin lies in one object, and objects own consecutive basin numbers
    pairs = np.unique(np.stack([out[lab > 0], lab[lab > 0]], 1), axis=0)
    assert len(np.unique(pairs[:, 0])) == len(pairs) == n
    assert np.all(np.diff(pairs[:, 1]) >= 0) and np.array_equal(pairs[:, 0], np.arange(1, n + 1))
    # every basin is 8-connected: relabelling the basins' pixels finds one component each
    for b in range(1, n + 1):
        comp, kb = oracle.label((out == b).astype(np.uint8), 1, 10 ** 9)
        assert kb == 1, b
    # clusters of touching nuclei were split somewhere
    assert n > K


def test_basins_are_numbered_by_their_first_pixel_within_each_object():
    """Within every object the basin numbers increase with the raster
    position of each basin's first pixel (not of its marker), and objects
    take consecutive ranges in label order; checked on a tile with many
    split clusters."""
    rgb = synth.tile(768, 768, 91, n_nuclei=300, frac_cluster=0.6, frac_overlap=0.3, n_stroma=2)
    r = oracle.seg(rgb, amax=6000)
    lab = r["labels"]
    out, n = oracle.watershed(lab, r["edt"], 1)
    flat_out, flat_lab = out.ravel(), lab.ravel()
    first = {}
    for i in np.flatnonzero(flat_out):
        first.setdefault(int(flat_out[i]), i)
    split = 0
    for k in range(1, int(lab.max()) + 1):
        basins = sorted(set(np.unique(flat_out[flat_lab == k]).tolist()))
        assert basins == list(range(basins[0], basins[-1] + 1))
        assert [first[b] for b in basins] == sorted(first[b] for b in basins)
        split += len(basins) > 1
    assert split >= 5
    assert n == max(first)
