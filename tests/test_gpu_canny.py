"""Parity of the CUDA Canny edges (Sec. V-A feature-stage transform; Table I
"Features comp.") and per-object edge counts (Sec. II "edge" features) with
the oracle, bit for bit: random planes of ragged sizes at several
thresholds, ideal steps, hem8 and labels of workload tiles at every radius,
an object whose box exceeds the count kernel's mask stage, the full 4096^2
benchmark tile, and the argument checks of the C ABI."""
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


def test_objects_whose_box_exceeds_the_count_stage(pipe):
    """A ring with a 141 x 141 box (beyond the 4096-pixel mask stage of the
    count kernel: the label plane is read instead) beside a small disc."""
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
