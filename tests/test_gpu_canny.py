"""Parity of the CUDA Canny edges (Sec. V-A feature-stage transform; Table I
"Features comp.") and per-object edge counts (Sec. II "edge" features) with
the oracle, bit for bit: random planes of ragged sizes at several
thresholds, ideal steps, hem8 and labels of workload tiles at every radius,
a large ring beside a small disc, disks holding many objects at once, the
full 4096^2 benchmark tile, the batched form (canny_batch: every tile equal
to canny_tile alone and to the oracle), and the argument checks of the C
ABI."""
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


def gpu_canny(pipe, img, lab=None, K=0, low=40, high=120, r=3):
    import torch
    dev = torch.device("cuda", 0)
    I = torch.from_numpy(np.ascontiguousarray(img, np.uint8)).to(dev)
    E = torch.full_like(I, 7)
    L = torch.from_numpy(np.ascontiguousarray(lab, np.int32)).to(dev) if lab is not None else None
    C = torch.full((max(K, 1),), -7, dtype=torch.int32, device=dev)
    pipe.canny(I, E, labels=L, n_objects=K, counts=C if K else None, low=low, high=high, radius=r)
    torch.cuda.synchronize()
    return E.cpu().numpy(), C.cpu().numpy()[:K]


def check(pipe, img, lab=None, K=0, low=40, high=120, r=3):
    want = oracle.canny(img, low, high)
    got, cnt = gpu_canny(pipe, img, lab, K, low, high, r)
    assert np.array_equal(got, want), np.argwhere(got != want)[:5]
    if K:
        assert np.array_equal(cnt, oracle.edge_counts(want, lab, K, r))
    return want


@pytest.mark.parametrize("W,H", [(1, 1), (2, 1), (7, 300), (33, 65), (64, 64), (65, 63), (200, 131), (517, 389)])
def test_random_planes(pipe, W, H):
    rng = np.random.default_rng(W * 7919 + H)
    img = rng.integers(0, 256, (H, W), dtype=np.uint8)
    for low, high in ((40, 120), (0, 0), (300, 900), (100, 100)):
        check(pipe, img, low=low, high=high)


def test_ideal_steps(pipe):
    H = W = 40
    yy, xx = np.mgrid[:H, :W]
    check(pipe, np.where(xx < 17, 20, 200).astype(np.uint8))
    check(pipe, np.where(yy < 5, 20, 200).astype(np.uint8))
    check(pipe, np.where(xx + yy < 40, 10, 60).astype(np.uint8))
    check(pipe, np.full((30, 31), 99, np.uint8))


@pytest.mark.parametrize("r", [0, 1, 2, 3, 4])
def test_workload_tiles_with_counts(pipe, r):
    for rgb in (synth.tile(512, 512, 0, n_nuclei=60, frac_overlap=0.1),
                synth.tile(768, 640, 77, n_nuclei=150, frac_cluster=0.4, n_stroma=4)):
        seg = oracle.seg(rgb)
        e = check(pipe, seg["hem8"], seg["labels"], seg["K"], r=r)
        assert e.any()
    seg = oracle.seg(synth.tile(333, 517, 9, n_nuclei=90, frac_cluster=0.5))
    check(pipe, seg["hem8"], seg["labels"], seg["K"] - 3, low=20, high=60, r=r)   # labels above n_objects


def test_large_ring_beside_a_small_disc(pipe):
    """A ring with a 141 x 141 box beside a small disc."""
    H, W = 200, 260
    yy, xx = np.mgrid[:H, :W]
    rr = (yy - 100) ** 2 + (xx - 100) ** 2
    m = ((rr <= 70 ** 2) & (rr >= 60 ** 2)) | (((yy - 40) ** 2 + (xx - 220) ** 2) <= 100)
    lab, K = oracle.label(m.astype(np.uint8), 1, 10 ** 9)
    img = np.where(m, 200, 20).astype(np.uint8)
    for r in (0, 1, 3, 4):
        check(pipe, img, lab, K, r=r)


def test_full_4096_benchmark_tile(pipe):
    import bench
    rgb = synth.tile(4096, 4096, bench.tile_seed(0, 0), n_nuclei=3000, frac_cluster=0.2, n_stroma=150)
    seg = oracle.seg(rgb)
    e = check(pipe, seg["hem8"], seg["labels"], seg["K"])
    assert e.sum() > 10 * seg["K"]


def test_argument_checks(pipe):
    import torch
    import paper_1209_3332_gb300 as P
    dev = torch.device("cuda", 0)
    I = torch.zeros((8, 8), dtype=torch.uint8, device=dev)
    E = torch.zeros_like(I)
    L = torch.zeros((8, 8), dtype=torch.int32, device=dev)
    C = torch.zeros(4, dtype=torch.int32, device=dev)
    for kw in ({"low": -1}, {"low": 50, "high": 40}, {"radius": 5}, {"radius": -1}):
        with pytest.raises(P.PipeError):
            pipe.canny(I, E, **kw)
    with pytest.raises(P.PipeError):
        pipe.canny(I, I)                                   # edges overlaps img
    with pytest.raises(P.PipeError):
        pipe.canny(I, E, labels=None, n_objects=2, counts=C)  # objects without labels


def many_objects(H=97, W=131, seed=5):
    """A one-pixel object at every other pixel of every other row (a disk of
    radius 4 holds up to about 13 of them) under a random plane."""
    rng = np.random.default_rng(seed)
    img = rng.integers(0, 256, (H, W), dtype=np.uint8)
    yy, xx = np.mgrid[:H, :W]
    lab = np.where((yy % 2 == 0) & (xx % 2 == 0), (yy // 2) * ((W + 1) // 2) + xx // 2 + 1, 0).astype(np.int32)
    return img, lab, int(lab.max())


@pytest.mark.parametrize("r", [1, 3, 4])
def test_disks_holding_many_objects(pipe, r):
    img, lab, K = many_objects()
    check(pipe, img, lab, K, low=30, high=90, r=r)


def batch_tiles():
    rng = np.random.default_rng(11)
    out = [(rng.integers(0, 256, (389, 517), dtype=np.uint8), None, 0)]          # no objects
    for rgb in (synth.tile(512, 512, 0, n_nuclei=60, frac_overlap=0.1),
                synth.tile(1024, 768, 78, n_nuclei=250, frac_cluster=0.3, n_stroma=6)):
        seg = oracle.seg(rgb)
        out.append((seg["hem8"], seg["labels"], seg["K"]))
    seg = oracle.seg(synth.tile(333, 517, 9, n_nuclei=90, frac_cluster=0.5))
    out.append((seg["hem8"], seg["labels"], seg["K"] - 3))                        # labels above n_objects
    out.append((np.array([[77]], np.uint8), np.array([[1]], np.int32), 1))        # 1 x 1
    out.append((np.full((70, 90), 50, np.uint8), np.zeros((70, 90), np.int32), 0))  # constant plane
    out.append(many_objects(61, 75, 9))
    return out


@pytest.mark.parametrize("r", [0, 3, 4])
def test_batch_equals_plain_and_oracle(pipe, r):
    import torch
    dev = torch.device("cuda", 0)
    tiles = batch_tiles()
    jobs = []
    for img, lab, K in tiles:
        jobs.append(dict(img=torch.from_numpy(np.ascontiguousarray(img)).to(dev),
                         edges=torch.full(img.shape, 7, dtype=torch.uint8, device=dev),
                         labels=torch.from_numpy(np.ascontiguousarray(lab)).to(dev) if lab is not None else None,
                         n_objects=K, counts=torch.full((max(K, 1),), -7, dtype=torch.int32, device=dev)))
    for _ in range(2):                       # a second call: flags, queue and counts start fresh
        pipe.canny_batch(jobs, low=40, high=120, radius=r)
        torch.cuda.synchronize()
        for (img, lab, K), j in zip(tiles, jobs):
            want = oracle.canny(img, 40, 120)
            got = j["edges"].cpu().numpy()
            assert np.array_equal(got, want), (img.shape, np.argwhere(got != want)[:5])
            cnt = j["counts"].cpu().numpy()[:K]
            if K:
                assert np.array_equal(cnt, oracle.edge_counts(want, lab, K, r))
            alone, c_alone = gpu_canny(pipe, img, lab, K, r=r)
            assert np.array_equal(alone, got) and np.array_equal(c_alone, cnt)


def test_batch_argument_checks(pipe):
    import torch
    import paper_1209_3332_gb300 as P
    dev = torch.device("cuda", 0)
    I = torch.zeros((8, 8), dtype=torch.uint8, device=dev)
    E = torch.zeros_like(I)
    C = torch.zeros(4, dtype=torch.int32, device=dev)
    ok = dict(img=I, edges=E)
    for kw in ({"low": -1}, {"low": 50, "high": 40}, {"radius": 5}):
        with pytest.raises(P.PipeError):
            pipe.canny_batch([ok], **kw)
    with pytest.raises(P.PipeError):
        pipe.canny_batch([ok, dict(img=I, edges=I)])                          # overlap in one tile
    with pytest.raises(P.PipeError):
        pipe.canny_batch([dict(img=I, edges=E, n_objects=2, counts=C)])       # objects without labels
    with pytest.raises(P.PipeError):
        pipe.canny_batch([])
