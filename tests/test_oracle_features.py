"""Pins of the per-object features (Sec. II feature families; Sec. V-A
gradient): a numpy restatement of every formula on random small label maps,
and closed-form hand cases."""
import math

import numpy as np
import pytest

import oracle
from tests import brute


@pytest.mark.parametrize("seed", range(8))
def test_random_objects_vs_numpy(seed):
    rng = np.random.default_rng(seed)
    H, W = int(rng.integers(3, 30)), int(rng.integers(3, 30))
    hem = rng.integers(0, 256, (H, W)).astype(np.uint8)
    if seed % 2:
        hem = (hem // 64 * 64 + 10).astype(np.uint8)  # few grey levels
    lab = rng.integers(0, 4, (H, W)).astype(np.int32)
    K = int(lab.max())
    got = oracle.features(hem, lab, K)
    ref = brute.features(hem, lab, K)
    assert np.allclose(got, ref, rtol=1e-9, atol=1e-12)


def test_one_pixel_object():
    hem = np.full((5, 5), 77, np.uint8)
    lab = np.zeros((5, 5), np.int32)
    lab[2, 2] = 1
    f = oracle.features(hem, lab, 1)[0]
    assert f[0] == 1 and f[1] == 4 and f[2] == 77 and f[3] == 0 and f[4] == f[5] == 77
    assert f[6] == 0 and f[7] == 0 and all(f[10:] == 0)


def test_square_perimeter_and_constant_texture():
    hem = np.full((6, 6), 100, np.uint8)
    lab = np.zeros((6, 6), np.int32)
    lab[2:4, 2:4] = 1
    f = oracle.features(hem, lab, 1)[0]
    assert f[0] == 4 and f[1] == 8
    # constant object: contrast 0, energy 1, homogeneity 1, entropy 0, correlation 0
    assert list(f[10:]) == [0.0, 1.0, 1.0, 0.0, 0.0]
    # constant image: zero gradient everywhere
    assert f[6] == f[7] == f[8] == f[9] == 0


def test_object_at_image_corner_counts_outside_as_boundary():
    hem = np.zeros((3, 3), np.uint8)
    lab = np.ones((3, 3), np.int32)
    assert oracle.features(hem, lab, 1)[0][1] == 12


def test_checkerboard_closed_form():
    # 4x4 object, levels 0 and 1 (hem8 0 and 32) in a checkerboard
    y, x = np.mgrid[0:4, 0:4]
    hem = (((x + y) % 2) * 32).astype(np.uint8)
    lab = np.ones((4, 4), np.int32)
    f = oracle.features(hem, lab, 1)[0]
    # (1,0),(0,1): 12 pairs each, all between levels 0/1 in equal number ->
    #   contrast 1, energy 1/2, homogeneity 1/2, entropy ln2, correlation -1
    # (1,1): 9 pairs, same level; starts on level 0 at 5 of them -> P00=5/9
    # (1,-1): 9 pairs, same level; P00=4/9
    e = lambda p: -(p * math.log(p) + (1 - p) * math.log(1 - p))
    con = (1 + 1 + 0 + 0) / 4
    ene = (0.5 + 0.5 + (25 + 16) / 81 + (16 + 25) / 81) / 4
    hom = (0.5 + 0.5 + 1 + 1) / 4
    ent = (math.log(2) * 2 + e(5 / 9) + e(4 / 9)) / 4
    cor = (-1 - 1 + 1 + 1) / 4
    assert np.allclose(f[10:], [con, ene, hom, ent, cor], rtol=1e-12, atol=1e-15)


def test_offset_direction_anisotropic():
    # vertical stripes: only the horizontal offset (1,0) and diagonals see
    # changes of level; (0,1) sees constant pairs
    y, x = np.mgrid[0:5, 0:6]
    hem = ((x % 2) * 64).astype(np.uint8)   # levels 0 and 2
    lab = np.ones((5, 6), np.int32)
    f = oracle.features(hem, lab, 1)[0]
    # contrast per offset: (1,0): 4, (0,1): 0, (1,1): 4, (1,-1): 4
    assert abs(f[10] - 3.0) < 1e-12


def test_ramp_gradient_with_replicated_border():
    # hem8 = 8*x: interior gx = 4*(8*(x+1) - 8*(x-1)) = 64; border columns 32
    hem = np.tile(np.arange(0, 80, 8), (4, 1)).astype(np.uint8)
    lab = np.ones(hem.shape, np.int32)
    f = oracle.features(hem, lab, 1)[0]
    n = hem.size
    mags = np.array([32] + [64] * 8 + [32], float)
    assert math.isclose(f[6], mags.mean(), rel_tol=1e-12)
    assert math.isclose(f[7], mags.std(), rel_tol=1e-12)
    assert f[8] == 32 and f[9] == 64 and f[0] == n


def test_std_is_population():
    hem = np.array([[10, 20]], np.uint8)
    lab = np.ones((1, 2), np.int32)
    f = oracle.features(hem, lab, 1)[0]
    assert f[2] == 15 and f[3] == 5
