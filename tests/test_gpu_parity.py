"""Parity of the CUDA path (through the C ABI) with the CPU oracle: every
integer plane and the object count bit for bit, every feature within 1e-4
relative or 1e-6 absolute of the FP64 oracle."""
import numpy as np
import pytest

import synth
from tests.gpu_util import assert_feats_close, assert_planes_equal, oracle_all, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pipe():
    import torch
    import paper_1209_3332_gb300 as P
    from paper_1209_3332_gb300 import build
    build.build()
    torch.cuda.init()
    p = P.Pipe(0)
    yield p
    assert p.status() == P.PIPE_OK
    p.close()


def check(pipe, rgb, **kw):
    g = run_gpu(pipe, rgb)
    r = oracle_all(rgb, **kw)
    assert_planes_equal(g, r)
    assert_feats_close(g["feats"], r["feats"])
    return g, r


def test_cfg0_512(pipe):
    g, r = check(pipe, synth.cfg0())
    assert r["K"] > 20


@pytest.mark.parametrize("W,H,n", [(77, 133, 6), (33, 65, 3), (1, 1, 0), (1, 300, 0), (300, 1, 0),
                                   (1000, 999, 120), (2049, 1025, 300), (31, 32, 1), (64, 64, 2)])
def test_ragged_sizes(pipe, W, H, n):
    rgb = synth.tile(W, H, 7 + W + H, n_nuclei=n, frac_overlap=0.1, frac_cluster=0.2, n_stroma=n // 20)
    check(pipe, rgb)


def test_empty_tile(pipe):
    rgb = synth.tile(700, 500, 3, n_nuclei=0)
    g, r = check(pipe, rgb)
    assert g["K"] == 0


def test_all_foreground_small_tile_has_no_background(pipe):
    rgb = np.zeros((30, 30, 3), np.uint8)  # hem8 = 255 everywhere -> one object, no background
    g, r = check(pipe, rgb)
    assert g["K"] == 1 and (g["edt"] == 2 ** 31 - 1).all()


def test_uniform_random_rgb(pipe):
    rng = np.random.default_rng(0)
    rgb = rng.integers(0, 256, (257, 300, 3)).astype(np.uint8)
    check(pipe, rgb)


def test_dense_chains_and_corridor(pipe):
    rgb = synth.tile(1536, 1280, 99, n_nuclei=1500, frac_chain=0.5, corridor=True)
    check(pipe, rgb)


def test_cfg1_full_4096(pipe):
    g, r = check(pipe, synth.cfg1())
    assert r["K"] > 1000


def test_repeat_is_deterministic(pipe):
    rgb = synth.tile(900, 700, 5, n_nuclei=200, frac_cluster=0.3)
    a = run_gpu(pipe, rgb)
    b = run_gpu(pipe, rgb)
    for k in ("hem8", "R", "labels", "edt"):
        assert np.array_equal(a[k], b[k])
    assert np.array_equal(a["feats"], b["feats"])


def test_all_rgb_triples_through_the_whole_path(pipe):
    # every 24-bit colour once: hem8 must match the oracle exactly everywhere,
    # and the rest of the path must agree on this far-from-natural image too
    v = np.arange(1 << 24, dtype=np.uint32)
    rgb = np.stack([(v >> 16) & 255, (v >> 8) & 255, v & 255], -1).astype(np.uint8).reshape(4096, 4096, 3)
    check(pipe, rgb)


def ring_tile(W=620, H=530):
    """White tile with black annuli: each annulus is a flat dome of the
    hematoxylin plane, so it is foreground and its inside a hole -- holes of
    2 to 230 pixels across, inside one 32x32 labelling block or spanning
    many, nested rings, and rings cut by the tile border (their inside
    touches the border and is no hole)."""
    yy, xx = np.mgrid[:H, :W]
    rgb = np.full((H, W, 3), 255, np.uint8)
    rings = [(40, 40, 2, 4), (31, 95, 5, 3), (100, 63, 9, 4), (160, 160, 14, 5), (300, 120, 30, 4),
             (300, 120, 12, 3), (420, 330, 115, 6), (420, 330, 60, 5), (420, 330, 20, 3), (5, 300, 25, 4),
             (600, 500, 40, 5), (250, 480, 33, 4), (96, 400, 31, 2)]
    for cx, cy, r, t in rings:
        d2 = (xx - cx) ** 2 + (yy - cy) ** 2
        rgb[(d2 >= r * r) & (d2 < (r + t) ** 2)] = 0
    return rgb


def test_holes_of_every_size(pipe):
    rgb = ring_tile()
    g, r = check(pipe, rgb)
    holes = int(r["filled"].sum()) - int(r["fg"].sum())
    assert holes > 20000  # the rings' insides were filled
