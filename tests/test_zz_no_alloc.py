"""features_tile_noalloc: the feature pass for callers that cannot allocate
device memory (for example code running under a framework's caching
allocator, or a serving loop that must avoid the synchronisation an
allocation can bring).  Its scratch is a static device array, so this test
checks it against features_tile on two calls in a row (the second call must
not be disturbed by what the first left in the shared array).  Both entry
points run the same kernels, so they must agree bit for bit; each result is
also checked against the FP64 oracle within the parity tests' tolerance.
It lives in its own file, collected last, and passes alone in a fresh
process or after the other tests."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_noalloc_matches_features_tile_twice():
    import torch
    import paper_1209_3332_gb300 as P
    from paper_1209_3332_gb300 import build
    from tests.gpu_util import assert_feats_close, assert_same_feats, oracle_all
    build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    pipe = P.Pipe(0)
    tiles = [synth.tile(1024, 768, 51, n_nuclei=250, frac_cluster=0.2, n_stroma=8),
             synth.tile(700, 900, 52, n_nuclei=120, frac_overlap=0.1)]
    for rgb_np in tiles:
        H, W = rgb_np.shape[:2]
        rgb = torch.from_numpy(rgb_np).to(dev)
        hem8 = torch.empty((H, W), dtype=torch.uint8, device=dev)
        labels = torch.empty((H, W), dtype=torch.int32, device=dev)
        edt = torch.empty((H, W), dtype=torch.int32, device=dev)
        nobj = torch.zeros(1, dtype=torch.int32, device=dev)
        pipe.seg_tile(rgb, hem8, labels, edt, nobj)
        torch.cuda.synchronize()
        K = int(nobj.item())
        assert 0 < K <= P.NOALLOC_MAX_OBJECTS
        ref = torch.zeros((K, 15), dtype=torch.float32, device=dev)
        pipe.features_tile(hem8, labels, K, ref)
        got = torch.full((K, 15), -1.0, dtype=torch.float32, device=dev)
        P.features_tile_noalloc(hem8, labels, K, got)
        torch.cuda.synchronize()
        a, b = got.cpu().numpy(), ref.cpu().numpy()
        assert_same_feats(a, b, "noalloc vs features_tile")
        o = oracle_all(rgb_np)
        assert o["K"] == K
        assert np.array_equal(labels.cpu().numpy(), o["labels"])
        assert_feats_close(a, o["feats"])
    with pytest.raises(P.PipeError):
        P.features_tile_noalloc(hem8, labels, P.NOALLOC_MAX_OBJECTS + 1, got)
    assert pipe.status() == P.PIPE_OK
    pipe.close()
