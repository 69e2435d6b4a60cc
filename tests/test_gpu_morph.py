"""Parity of the CUDA opening by a disk (Table I "Morph. Open", 19x19 disk)
with the oracle, bit for bit: random planes of ragged sizes and every radius
class, a deconvolved tile of the benchmark workload, full 4096^2 planes on
sampled row bands, and the argument checks of the C ABI."""
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


def gpu_open(pipe, a, r):
    import torch
    dev = torch.device("cuda", 0)
    src = torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    dst = torch.full_like(src, 7)
    pipe.morph_open(src, dst, radius=r)
    torch.cuda.synchronize()
    return dst.cpu().numpy()


@pytest.mark.parametrize("W,H", [(1, 1), (64, 64), (65, 63), (200, 131), (7, 300), (517, 389)])
@pytest.mark.parametrize("r", [0, 1, 4, 9, 15])
def test_random_planes(pipe, W, H, r):
    rng = np.random.default_rng(W * 1000 + H + r)
    a = rng.integers(0, 256, (H, W), dtype=np.uint8)
    assert np.array_equal(gpu_open(pipe, a, r), oracle.morph_open(a, r))


def test_hem8_of_a_workload_tile(pipe):
    """The plane the opening would see in the pipeline: hem8 of a seeded
    1024^2 tile with nuclei, clusters and stroma."""
    rgb = synth.tile(1024, 768, 4242, n_nuclei=250, frac_cluster=0.2, n_stroma=12)
    hem8 = oracle.deconv(rgb)
    assert np.array_equal(gpu_open(pipe, hem8, 9), oracle.morph_open(hem8, 9))


def test_full_4096_on_row_bands(pipe):
    """A full 4096^2 hem8 plane of the benchmark workload.  The opening at a
    pixel depends on input within 2r, so the oracle on rows y0-2r..y1+2r
    gives rows y0..y1 exactly; three bands plus the two image edges."""
    import bench
    rgb = synth.tile(4096, 4096, bench.tile_seed(0, 0), n_nuclei=3000, frac_cluster=0.2, n_stroma=150)
    hem8 = oracle.deconv(rgb)
    got = gpu_open(pipe, hem8, 9)
    r = 9
    for y0, y1 in [(0, 24), (1000, 1040), (2047, 2080), (4071, 4096)]:
        a0, a1 = max(0, y0 - 2 * r), min(4096, y1 + 2 * r)
        ref = oracle.morph_open(hem8[a0:a1], r)
        assert np.array_equal(got[y0:y1], ref[y0 - a0:y1 - a0]), (y0, y1)


def test_argument_checks(pipe):
    import torch
    import paper_1209_3332_gb300 as P
    dev = torch.device("cuda", 0)
    a = torch.zeros((32, 48), dtype=torch.uint8, device=dev)
    b = torch.zeros_like(a)
    L = P.lib()
    assert L.morph_open_tile(pipe.h, a.data_ptr(), 48, 32, 16, b.data_ptr(), None) == P.PIPE_EINVAL
    assert L.morph_open_tile(pipe.h, a.data_ptr(), 48, 32, -1, b.data_ptr(), None) == P.PIPE_EINVAL
    assert L.morph_open_tile(pipe.h, a.data_ptr(), 48, 32, 9, a.data_ptr() + 100, None) == P.PIPE_EINVAL
    assert L.morph_open_tile(pipe.h, a.data_ptr(), 0, 32, 9, b.data_ptr(), None) == P.PIPE_EINVAL
    assert L.morph_open_tile(pipe.h, a.data_ptr(), 48, 32, 9, b.data_ptr(), None) == P.PIPE_OK
