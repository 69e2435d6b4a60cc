"""Pins of the oracle's Canny edges (Sec. V-A feature-stage transform; Table I
"Features comp.") and per-object edge counts (Sec. II "edge" features):
closed forms of ideal vertical, horizontal and diagonal steps worked out by
hand from the definition, the Sobel magnitude against SciPy's Sobel filter,
the hysteresis against SciPy's connected components and the oracle's own
reconstruction, the strict thresholds, hysteresis reach, and the edge counts
against a SciPy disk dilation."""
import numpy as np
import pytest
from scipy import ndimage

import oracle
import synth


def step_x(H, W, c, a, b):
    img = np.full((H, W), a, np.uint8)
    img[:, c:] = b
    return img


@pytest.mark.parametrize("c", [1, 5, 17])
def test_vertical_step_gives_the_column_left_of_it(c):
    """I = a left of column c, b from c on: gx = 4(b - a) on columns c-1 and c,
    gy = 0; non-maximum suppression keeps c-1 (m > left, m >= right) and
    drops c (m == left)."""
    a, b = 20, 200
    img = step_x(23, 30, c, a, b)
    e, m, cls = oracle.canny(img, 40, 120, detail=True)
    want_m = np.zeros_like(m)
    want_m[:, c - 1:c + 1] = 4 * (b - a)
    assert np.array_equal(m, want_m)
    want = np.zeros_like(e)
    want[:, c - 1] = 1
    assert np.array_equal(e, want)
    assert np.array_equal(oracle.canny(img.T.copy(), 40, 120), want.T)   # horizontal step: row c - 1


def test_diagonal_step_keeps_two_lines():
    """I = a where x + y < c, else b.  Per unit of (b - a), with s = x + y:
    gx = gy = 1, 3, 3, 1 at s = c-2 .. c+1, so m = 2, 6, 6, 2; the sector is
    the (+x,+y) diagonal (ax = ay); s = c-1 survives (6 > 0, 6 >= 2), s = c
    survives (6 > 2, 6 >= 0), s = c-2 (2 < 6 ahead) and s = c+1 (2 < 6
    behind) do not.  Checked away from the image border."""
    H = W = 40
    c = 40
    yy, xx = np.mgrid[:H, :W]
    a, b = 10, 60
    img = np.where(xx + yy < c, a, b).astype(np.uint8)
    e, m, _ = oracle.canny(img, 40, 120, detail=True)
    inner = (yy > 3) & (yy < H - 4) & (xx > 3) & (xx < W - 4)
    s = xx + yy
    unit = {c - 2: 2, c - 1: 6, c: 6, c + 1: 2}
    for k, v in unit.items():
        assert np.all(m[inner & (s == k)] == v * (b - a))
    assert np.all(m[inner & ((s < c - 2) | (s > c + 1))] == 0)
    assert np.array_equal(e[inner], ((s == c - 1) | (s == c))[inner].astype(np.uint8))


def test_sobel_magnitude_is_scipys_with_nearest_border():
    rng = np.random.default_rng(3)
    img = rng.integers(0, 256, (37, 53), dtype=np.uint8)
    _, m, _ = oracle.canny(img, 0, 0, detail=True)
    f = img.astype(np.int64)
    want = np.abs(ndimage.sobel(f, axis=1, mode="nearest")) + np.abs(ndimage.sobel(f, axis=0, mode="nearest"))
    assert np.array_equal(m, want)


@pytest.mark.parametrize("seed", range(4))
def test_hysteresis_is_the_strong_components_of_the_candidates(seed):
    """Edges = the 8-connected components of the candidates that hold a
    strong pixel (SciPy labelling), = the reconstruction by dilation of the
    strong pixels under the candidates (the oracle's Vincent reconstruction)."""
    rgb = synth.tile(160, 120, 50 + seed, n_nuclei=12, frac_cluster=0.3)
    hem = oracle.deconv(rgb)
    rng = np.random.default_rng(seed)
    hem = np.clip(hem.astype(int) + rng.integers(-25, 26, hem.shape), 0, 255).astype(np.uint8)
    e, m, cls = oracle.canny(hem, 40, 120, detail=True)
    comp, n = ndimage.label(cls > 0, structure=np.ones((3, 3)))
    strong = np.unique(comp[cls == 2])
    want = np.isin(comp, strong[strong > 0]).astype(np.uint8)
    assert np.array_equal(e, want)
    rec = oracle.recon((cls == 2).astype(np.uint8), (cls > 0).astype(np.uint8))
    assert np.array_equal(e, rec)
    assert e.sum() > 0 and (cls == 1).any()


def test_thresholds_are_strict():
    img = step_x(9, 12, 6, 50, 80)          # m = 4 * 30 = 120 on the kept column
    assert not oracle.canny(img, 120, 200).any()          # m == low: not a candidate
    assert not oracle.canny(img, 100, 120).any()          # a candidate, but m == high: not strong
    assert oracle.canny(img, 100, 119)[:, 5].all()        # strong


def test_hysteresis_reaches_along_weak_pixels():
    """A vertical step of contrast 40 (m = 160: weak for thresholds 100 / 200)
    whose top rows have contrast 80 (m = 320: strong): its whole column is
    kept, the weak part reached through the junction at the contrast change
    (rows 4-5, where the horizontal step of the block takes column 9 itself).
    A second step of contrast 40 over the full height, with no corner (its
    L1 magnitude would exceed 200 there), is dropped."""
    img = np.full((30, 48), 20, np.uint8)
    img[:, 10:] = 60
    img[:5, 10:25] = 100
    img[:, 35:] = 100
    e = oracle.canny(img, 100, 200)
    assert e[:4, 9].all() and e[6:, 9].all()
    assert not e[:, 30:].any()
    weak_only = img.copy()
    weak_only[:5, 10:25] = 60
    assert not oracle.canny(weak_only, 100, 200).any()


def test_constant_and_degenerate_planes():
    assert not oracle.canny(np.full((7, 9), 123, np.uint8)).any()
    assert not oracle.canny(np.zeros((1, 1), np.uint8)).any()
    assert oracle.canny(np.array([[0, 255]], np.uint8), 10, 20).tolist() == [[1, 0]]
    with pytest.raises(ValueError):
        oracle.canny(np.zeros((4, 4), np.uint8), 50, 40)


@pytest.mark.parametrize("r", [0, 1, 3, 4])
def test_edge_counts_are_the_edges_in_each_objects_disk_dilation(r):
    rgb = synth.tile(256, 200, 9, n_nuclei=25, frac_cluster=0.4)
    seg = oracle.seg(rgb)
    lab, K = seg["labels"], seg["K"]
    e = oracle.canny(seg["hem8"])
    yy, xx = np.mgrid[-r:r + 1, -r:r + 1]
    disk = xx * xx + yy * yy <= r * r
    want = [int(e[ndimage.binary_dilation(lab == k, structure=disk)].sum()) for k in range(1, K + 1)]
    assert oracle.edge_counts(e, lab, K, r).tolist() == want
    if r == 3:
        assert sum(want) > 10 * K


def _nms_by_angle(img):
    """Non-maximum suppression restated with SciPy's Sobel and
    floating-point angles (atan2) instead of the oracle's exact integer
    sector tests: horizontal below 22.5 degrees, vertical above 67.5,
    otherwise the diagonal of the gradient's sign."""
    f = img.astype(np.int64)
    gx = ndimage.sobel(f, axis=1, mode="nearest")
    gy = ndimage.sobel(f, axis=0, mode="nearest")
    m = np.abs(gx) + np.abs(gy)
    H, W = img.shape
    mp = np.zeros((H + 2, W + 2), np.int64)
    mp[1:-1, 1:-1] = m
    ang = np.degrees(np.arctan2(np.abs(gy), np.abs(gx)))
    keep = np.zeros((H, W), bool)
    for y in range(H):
        for x in range(W):
            if ang[y, x] < 22.5:
                a, b = (0, -1), (0, 1)
            elif ang[y, x] > 67.5:
                a, b = (-1, 0), (1, 0)
            elif gx[y, x] * gy[y, x] > 0:
                a, b = (-1, -1), (1, 1)
            else:
                a, b = (-1, 1), (1, -1)
            v = m[y, x]
            keep[y, x] = v > mp[y + 1 + a[0], x + 1 + a[1]] and v >= mp[y + 1 + b[0], x + 1 + b[1]]
    return m, keep


@pytest.mark.parametrize("seed", range(3))
def test_suppression_matches_angles_computed_in_floating_point(seed):
    """Planes whose gradients fall near the 22.5 and 67.5 degree sector
    boundaries (linear ramps at slopes around tan 22.5 = 0.414 and
    tan 67.5 = 2.414, with noise), plus a random plane: with thresholds 0,
    the candidates are exactly the survivors with m > 0."""
    rng = np.random.default_rng(seed)
    H, W = 40, 48
    yy, xx = np.mgrid[:H, :W]
    planes = [rng.integers(0, 256, (H, W), dtype=np.uint8)]
    for slope in (0.38, 0.41, 0.42, 0.45, 2.3, 2.41, 2.42, 2.6):
        ramp = 3.0 * xx + 3.0 * slope * yy + rng.normal(0, 4, (H, W))
        ramp = ramp if seed % 2 == 0 else -ramp
        planes.append(np.clip(ramp - ramp.min(), 0, 255).astype(np.uint8))
    checked = 0
    for img in planes:
        _, m, cls = oracle.canny(img, 0, 0, detail=True)
        mref, keep = _nms_by_angle(img)
        assert np.array_equal(m, mref)
        assert np.array_equal(cls > 0, keep & (mref > 0))
        checked += int(keep.sum())
    assert checked > 500
