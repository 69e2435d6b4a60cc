"""Parity of the CUDA watershed split (Table I "Pre-Watershed" + "Watershed")
with the oracle, bit for bit on the split label plane and the basin count:
closed-form shapes (discs, symmetric pairs, chains, necks at several marker
heights), random unions of discs, objects whose box exceeds the shared-memory
stage (the global-memory path), image edges, a tile without background,
labels above n_objects, workload tiles through the whole GPU path up to the
full 4096^2 benchmark tile, determinism, the batched form (equal to the
oracle per tile, and to the plain form on four 4096^2 tiles), and the
argument checks."""
import numpy as np
import pytest

import oracle
import synth

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


def gpu_ws(pipe, lab, edt, K, h):
    import torch
    dev = torch.device("cuda", 0)
    L = torch.from_numpy(np.ascontiguousarray(lab, np.int32)).to(dev)
    E = torch.from_numpy(np.ascontiguousarray(edt, np.int32)).to(dev)
    out = torch.full_like(L, -7)
    n = torch.full((1,), -7, dtype=torch.int32, device=dev)
    pipe.watershed(L, E, K, out, n, h=h)
    torch.cuda.synchronize()
    return out.cpu().numpy(), int(n.item())


def check(pipe, lab, h=1, K=None):
    lab = np.ascontiguousarray(lab, np.int32)
    K = int(lab.max()) if K is None else K
    edt = oracle.edt(lab)
    want, n = oracle.watershed(np.where(lab <= K, lab, 0), edt, h)
    got, gn = gpu_ws(pipe, lab, edt, K, h)
    assert gn == n
    assert np.array_equal(got, want), np.argwhere(got != want)[:5]
    return n


def discs(H, W, centres, r):
    yy, xx = np.mgrid[:H, :W]
    m = np.zeros((H, W), bool)
    for cy, cx in centres:
        m |= (yy - cy) ** 2 + (xx - cx) ** 2 <= r * r
    return m


def lab_of(mask):
    return oracle.label(mask.astype(np.uint8), 1, 10 ** 9)[0]


@pytest.mark.parametrize("h", [0, 1, 2, 3])
def test_closed_form_shapes(pipe, h):
    for r in (3, 7, 12, 20):
        check(pipe, lab_of(discs(2 * r + 9, 2 * r + 11, [(r + 4, r + 5)], r)), h)
    for gap in (14, 17, 20):
        check(pipe, lab_of(discs(41, 40 + gap, [(20, 20), (20, 20 + gap)], 12)), h)
    check(pipe, lab_of(discs(41, 50, [(20, 20), (20, 34)], 12)), h)
    check(pipe, lab_of(discs(40, 100, [(20, 18), (20, 38), (20, 58), (20, 78)], 12)), h)


@pytest.mark.parametrize("seed", range(6))
def test_random_unions_of_discs(pipe, seed):
    rng = np.random.default_rng(seed)
    H, W = int(rng.integers(60, 200)), int(rng.integers(60, 260))
    m = np.zeros((H, W), bool)
    for _ in range(int(rng.integers(5, 40))):
        m |= discs(H, W, [(rng.integers(0, H), rng.integers(0, W))], int(rng.integers(2, 15)))
    for h in (0, 1, 2):
        check(pipe, lab_of(m), h)


def test_large_boxes_take_the_global_path(pipe):
    """Objects whose box with margin exceeds the 1024-pixel stage: a long
    chain of discs, a diagonal band, a ring and a comb, beside small ones."""
    H, W = 300, 420
    m = discs(H, W, [(40, 20 + 22 * i) for i in range(12)], 12)
    yy, xx = np.mgrid[:H, :W]
    m |= (np.abs((yy - 80) - (xx - 20) * 0.6) < 3) & (xx > 20) & (xx < 300)
    rr = (yy - 210) ** 2 + (xx - 90) ** 2
    m |= (rr <= 70 ** 2) & (rr >= 60 ** 2)
    m[150:290, 250:254] = True
    for x in range(250, 400, 12):
        m[280:284, 250:x + 3] = True
        m[200:284, x:x + 3] = True
    m |= discs(H, W, [(230, 380), (100, 380)], 9)
    n = check(pipe, lab_of(m), 1)
    assert n >= 14


def test_edges_degenerate_and_out_of_range_labels(pipe):
    check(pipe, lab_of(discs(30, 40, [(15, 20)], 25)), 1)     # touches all four edges
    check(pipe, np.ones((20, 25), np.int32), 1)                  # no background: edt INT32_MAX
    check(pipe, np.ones((1, 1), np.int32), 1)
    z = np.zeros((33, 65), np.int32)
    got, n = gpu_ws(pipe, z, oracle.edt(z), 0, 1)
    assert n == 0 and not got.any()
    lab = lab_of(discs(40, 100, [(20, 15), (20, 45), (20, 80)], 9))
    check(pipe, lab, 1, K=2)                                    # label 3 is above n_objects: 0
    m = np.zeros((40, 40), bool)
    m[5, 5] = True
    m[10:30, 10] = True
    for i in range(25):
        m[10 + i, 15 + i] = True
    check(pipe, lab_of(m), 1)


def test_workload_tiles_through_the_gpu_path(pipe):
    """seg_tile's own labels and EDT feed the split; everything is compared
    with the oracle's segmentation and split of the same tile."""
    import torch
    from tests.gpu_util import run_gpu
    for rgb, amax in ((synth.tile(512, 512, 0, n_nuclei=60, frac_overlap=0.1), 1500),
                      (synth.tile(768, 640, 77, n_nuclei=150, frac_cluster=0.4, n_stroma=4), 1500),
                      (synth.tile(333, 517, 9, n_nuclei=90, frac_cluster=0.5, frac_overlap=0.2), 6000)):
        r = oracle.seg(rgb, amax=amax)
        g = run_gpu(pipe, rgb) if amax == 1500 else None
        if g is not None:
            assert np.array_equal(g["labels"], r["labels"]) and np.array_equal(g["edt"], r["edt"])
        for h in (1, 2):
            check(pipe, r["labels"], h)
    torch.cuda.synchronize()


def test_full_4096_benchmark_tile(pipe):
    import bench
    rgb = synth.tile(4096, 4096, bench.tile_seed(0, 0), n_nuclei=3000, frac_cluster=0.2, n_stroma=150)
    r = oracle.seg(rgb)
    n = check(pipe, r["labels"], 1)
    assert n > r["K"]
    # determinism: a second run gives the same plane
    a, na = gpu_ws(pipe, r["labels"], r["edt"], r["K"], 1)
    b, nb = gpu_ws(pipe, r["labels"], r["edt"], r["K"], 1)
    assert na == nb and np.array_equal(a, b)


def _ws_batch(pipe, labs, Ks, h):
    import torch
    dev = torch.device("cuda", 0)
    tiles = []
    for lab, K in zip(labs, Ks):
        L = torch.from_numpy(np.ascontiguousarray(lab, np.int32)).to(dev)
        tiles.append(dict(labels=L, edt=torch.from_numpy(oracle.edt(lab)).to(dev), out=torch.full_like(L, -7),
                          n_objects=K, n_basins=torch.full((1,), -7, dtype=torch.int32, device=dev)))
    pipe.watershed_batch(tiles, h=h)
    torch.cuda.synchronize()
    return [(t["out"].cpu().numpy(), int(t["n_basins"].item())) for t in tiles]


@pytest.mark.parametrize("h", [1, 2])
def test_batched_form_equals_the_oracle_per_tile(pipe, h):
    """Tiles of ragged sizes in one batch: workload tiles with clusters (one
    with labels above n_objects), a chain of discs whose box exceeds the
    stage, a 1x1 tile, empty tiles."""
    labs = []
    for seed, (W, H) in enumerate(((300, 200), (64, 33), (420, 300), (17, 90), (513, 257))):
        rgb = synth.tile(W, H, 500 + seed, n_nuclei=max(1, W * H // 900), frac_cluster=0.5)
        labs.append(oracle.seg(rgb, amax=6000)["labels"])
    labs.append(lab_of(discs(300, 420, [(40, 20 + 22 * i) for i in range(12)], 12)))
    labs.append(np.ones((1, 1), np.int32))
    labs.append(np.zeros((5, 7), np.int32))
    Ks = [int(x.max()) for x in labs]
    Ks[0] -= 2
    got = _ws_batch(pipe, labs, Ks, h)
    for lab, K, (out, n) in zip(labs, Ks, got):
        want, wn = oracle.watershed(np.where(lab <= K, lab, 0), oracle.edt(lab), h)
        assert n == wn and np.array_equal(out, want)


def test_batched_form_equals_the_plain_form_on_4096_tiles(pipe):
    import bench
    labs = []
    for i in range(4):
        rgb = synth.tile(4096, 4096, bench.tile_seed(0, i), n_nuclei=3000, frac_cluster=0.2, n_stroma=150)
        labs.append(oracle.seg(rgb)["labels"])
    Ks = [int(x.max()) for x in labs]
    got = _ws_batch(pipe, labs, Ks, 1)
    for lab, K, (out, n) in zip(labs, Ks, got):
        plain, pn = gpu_ws(pipe, lab, oracle.edt(lab), K, 1)
        assert n == pn and np.array_equal(out, plain)


def test_argument_checks(pipe):
    import torch
    import paper_1209_3332_gb300 as P
    dev = torch.device("cuda", 0)
    L = torch.zeros((8, 8), dtype=torch.int32, device=dev)
    E = torch.zeros_like(L)
    out = torch.zeros_like(L)
    n = torch.zeros(1, dtype=torch.int32, device=dev)
    for kw in ({"h": -1}, {"h": 256}):
        with pytest.raises(P.PipeError):
            pipe.watershed(L, E, 0, out, n, **kw)
    with pytest.raises(P.PipeError):
        pipe.watershed(L, E, 0, L, n)            # out overlaps labels
    with pytest.raises(P.PipeError):
        pipe.watershed(L, E, -1, out, n)
