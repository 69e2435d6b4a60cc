"""RBC detection (Table I "RBC detection") on the GPU through the C ABI,
bit for bit against the oracle: random tiles of ragged sizes at several
threshold pairs, pitched rows, a mask that snakes through many work tiles
from one marker (the reconstruction starts from the flagged tiles only, so
the rest must be reached on demand), markers on work-tile seams, workload
tiles with and without red blood cells, the full 4096^2 tile, repeated
calls, and the argument checks."""
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


def gpu_rbc(pipe, rgb, t_lo=40, t_hi=100, pad=0):
    """rbc_tile on a copy of rgb whose rows are `pad` bytes longer than 3W."""
    import torch
    H, W = rgb.shape[:2]
    dev = torch.device("cuda", 0)
    if pad:
        buf = torch.zeros((H, 3 * W + pad), dtype=torch.uint8, device=dev)
        buf[:, :3 * W] = torch.from_numpy(np.ascontiguousarray(rgb).reshape(H, 3 * W)).to(dev)
        src = buf.view(torch.uint8)
        out = torch.full((H, W), 7, dtype=torch.uint8, device=dev)
        import paper_1209_3332_gb300 as P
        rc = P.lib().rbc_tile(pipe.h, src.data_ptr(), W, H, 3 * W + pad, t_lo, t_hi, out.data_ptr(),
                              P._stream_ptr(None))
        assert rc == P.PIPE_OK
    else:
        src = torch.from_numpy(np.ascontiguousarray(rgb)).to(dev)
        out = torch.full((H, W), 7, dtype=torch.uint8, device=dev)
        pipe.rbc(src, out, t_lo, t_hi)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def rand_rgb(rng, H, W):
    rgb = rng.integers(0, 256, (H, W, 3)).astype(np.int32)
    base = rng.integers(0, 160, (H, W))
    rgb[..., 0] = np.clip(base + rng.integers(-30, 200, (H, W)), 0, 255)
    rgb[..., 1] = np.clip(base + rng.integers(-20, 20, (H, W)), 0, 255)
    rgb[..., 2] = np.clip(base + rng.integers(-20, 20, (H, W)), 0, 255)
    return rgb.astype(np.uint8)


def assert_same(got, want, what=""):
    if not np.array_equal(got, want):
        bad = np.argwhere(got != want)
        y, x = bad[0]
        raise AssertionError("%s: %d pixels differ; first (%d,%d) gpu %d oracle %d"
                             % (what, len(bad), y, x, got[y, x], want[y, x]))


@pytest.mark.parametrize("shape", [(1, 1), (1, 300), (300, 1), (33, 65), (77, 133), (64, 64), (65, 129),
                                   (517, 389), (999, 1000)])
def test_random_ragged(pipe, shape):
    rng = np.random.default_rng(shape[0] * 1009 + shape[1])
    rgb = rand_rgb(rng, *shape)
    for t_lo, t_hi in ((40, 100), (0, 0), (60, 60), (10, 200), (120, 255)):
        assert_same(gpu_rbc(pipe, rgb, t_lo, t_hi), oracle.rbc(rgb, t_lo, t_hi), "%s %d/%d" % (shape, t_lo, t_hi))


@pytest.mark.parametrize("pad", [1, 5, 16, 37])
def test_pitched_rows(pipe, pad):
    rng = np.random.default_rng(pad)
    rgb = rand_rgb(rng, 131, 250)
    assert_same(gpu_rbc(pipe, rgb, pad=pad), oracle.rbc(rgb), "pad %d" % pad)


def snake(H, W, step, seed_at_end):
    """A one-pixel-wide serpentine mask (d = 50) with one marker pixel
    (d = 150) at one end: the flood must cross every work tile it passes."""
    d = np.zeros((H, W), np.int32)
    y, going_right = 1, True
    path = []
    while y < H - 1:
        xs = range(1, W - 1) if going_right else range(W - 2, 0, -1)
        path += [(y, x) for x in xs]
        end_x = W - 2 if going_right else 1
        for yy in range(y + 1, min(y + step, H - 1)):
            path.append((yy, end_x))
        y += step
        going_right = not going_right
    for (yy, xx) in path:
        d[yy, xx] = 50
    yy, xx = path[-1] if seed_at_end else path[0]
    d[yy, xx] = 150
    rgb = np.zeros((H, W, 3), np.uint8)
    rgb[..., 0] = d
    return rgb


@pytest.mark.parametrize("seed_at_end", [False, True])
def test_snake_through_unseeded_tiles(pipe, seed_at_end):
    rgb = snake(700, 530, 6, seed_at_end)
    want = oracle.rbc(rgb)
    assert want.sum() > 50000
    assert_same(gpu_rbc(pipe, rgb), want, "snake")


def test_markers_on_tile_seams(pipe):
    """Marker pixels on the rows and columns either side of the 64-pixel
    work-tile seams, each with mask that runs into the neighbouring tile."""
    H = W = 256
    d = np.zeros((H, W), np.int32)
    for c in (63, 64, 127, 128, 191, 192):
        d[:, c] = 45                       # mask lines across the seams
        d[c, :] = 45
    for (y, x) in ((63, 10), (64, 70), (10, 127), (200, 128), (63, 63), (64, 64), (127, 192), (192, 191)):
        d[y, x] = 101
    rgb = np.zeros((H, W, 3), np.uint8)
    rgb[..., 0] = d
    assert_same(gpu_rbc(pipe, rgb), oracle.rbc(rgb), "seams")


def test_workload_tiles(pipe):
    with_rbc = synth.tile(1024, 768, 91, n_nuclei=200, frac_cluster=0.2, n_stroma=10, n_rbc=300)
    want = oracle.rbc(with_rbc)
    assert want.sum() > 10000
    assert_same(gpu_rbc(pipe, with_rbc), want, "tile with red blood cells")
    without = synth.tile(1024, 768, 91, n_nuclei=200, frac_cluster=0.2, n_stroma=10)
    assert not gpu_rbc(pipe, without).any()
    for _ in range(2):                    # repeated calls: the seed flags and queue start fresh
        assert_same(gpu_rbc(pipe, with_rbc), want, "repeat")


def test_full_4096_tile(pipe):
    t = synth.tile(4096, 4096, 1000, n_nuclei=3000, frac_cluster=0.2, n_stroma=150, n_rbc=800)
    assert_same(gpu_rbc(pipe, t), oracle.rbc(t), "4096^2")


def test_argument_checks(pipe):
    import torch
    import paper_1209_3332_gb300 as P
    dev = torch.device("cuda", 0)
    rgb = torch.zeros((8, 8, 3), dtype=torch.uint8, device=dev)
    out = torch.zeros((8, 8), dtype=torch.uint8, device=dev)
    for lo, hi in ((-1, 10), (50, 40), (0, 256)):
        with pytest.raises(P.PipeError):
            pipe.rbc(rgb, out, lo, hi)
    L = P.lib()
    s = P._stream_ptr(None)
    assert L.rbc_tile(pipe.h, rgb.data_ptr(), 8, 8, 23, 40, 100, out.data_ptr(), s) == P.PIPE_EINVAL  # pitch < 3W
    assert L.rbc_tile(pipe.h, rgb.data_ptr(), 0, 8, 24, 40, 100, out.data_ptr(), s) == P.PIPE_EINVAL
    assert L.rbc_tile(pipe.h, rgb.data_ptr(), 8, 8, 24, 40, 100, rgb.data_ptr() + 8, s) == P.PIPE_EINVAL  # overlap
    assert L.rbc_tile(pipe.h, None, 8, 8, 24, 40, 100, out.data_ptr(), s) == P.PIPE_EINVAL
