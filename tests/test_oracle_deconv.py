"""Pins of the oracle's colour deconvolution (Sec. V-A, 'Color deconvolution').

The paper names the transform only; the stain vectors, fixed point and
scaling are the reading documented with the oracle.  Pinned by: the constant
tables rebuilt independently, hand values of the stated colours, and an
exhaustive sweep over all 2^24 RGB triples against the formula in integers.
"""
import math

import numpy as np

import oracle
from tests import brute


def test_tables_match_independent_rebuild():
    lut, wq, w = oracle.deconv_tables()
    blut, bwq, bw = brute.deconv_constants()
    assert np.array_equal(lut, blut)
    assert np.array_equal(wq, bwq)
    assert np.allclose(w, bw, rtol=1e-12, atol=0)
    assert list(wq) == [304962, -33310, 104952]
    assert lut[255] == 0 and lut[0] == 1420
    # no table entry sits within 1e-6 of a rounding tie, so the integer
    # tables do not depend on the last bit of log()
    for v in range(256):
        x = -math.log((v + 1) / 256.0) * 256.0 + 0.5
        assert abs(x - round(x)) > 1e-6 or abs(x - math.floor(x)) > 1e-6
    for k in range(3):
        x = 100.0 * w[k] * 2048.0
        assert abs(abs(x - math.floor(x)) - 0.5) > 1e-6


def test_inverse_stain_matrix_recovers_pure_hematoxylin():
    _, _, w = oracle.deconv_tables()
    H = np.array([0.650, 0.704, 0.286])
    H /= np.linalg.norm(H)
    E = np.array([0.072, 0.990, 0.105])
    E /= np.linalg.norm(E)
    # an optical density made only of stain H has unit H concentration and none of E
    assert abs(H @ w - 1.0) < 1e-12
    assert abs(E @ w) < 1e-12


def test_hand_values():
    cases = {(225, 215, 228): 22, (90, 60, 140): 161, (200, 150, 190): 42,
             (255, 255, 255): 0, (0, 0, 0): 255}
    rgb = np.array([list(k) for k in cases], np.uint8).reshape(1, -1, 3)
    got = oracle.deconv(rgb)[0]
    assert list(got) == list(cases.values())


def test_exhaustive_all_rgb_triples():
    v = np.arange(1 << 24, dtype=np.uint32)
    rgb = np.stack([(v >> 16) & 255, (v >> 8) & 255, v & 255], -1).astype(np.uint8)
    rgb = rgb.reshape(4096, 4096, 3)
    got = oracle.deconv(rgb)
    ref = brute.deconv(rgb.astype(np.int64))
    assert np.array_equal(got, ref)


def test_int32_accumulator_bound():
    lut, wq, _ = oracle.deconv_tables()
    hi = sum(int(w) * (int(lut.max()) if w > 0 else 0) for w in wq)
    lo = sum(int(w) * (int(lut.max()) if w < 0 else 0) for w in wq)
    assert hi + (1 << 18) < 2 ** 31 and lo > -(2 ** 31)
