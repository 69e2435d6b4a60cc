"""Helpers for the GPU parity tests: run the CUDA path through the C ABI on
torch buffers and compare with the oracle on the same seeded input."""
import numpy as np

import oracle

TOL_REL, TOL_ABS = 1e-4, 1e-6


def run_gpu(pipe, rgb_np, want_planes=True, stream=None):
    import torch
    H, W = rgb_np.shape[:2]
    dev = torch.device("cuda", pipe.device)
    rgb = torch.from_numpy(np.ascontiguousarray(rgb_np)).to(dev)
    hem8 = torch.empty((H, W), dtype=torch.uint8, device=dev)
    labels = torch.empty((H, W), dtype=torch.int32, device=dev)
    edt = torch.empty((H, W), dtype=torch.int32, device=dev)
    nobj = torch.zeros(1, dtype=torch.int32, device=dev)
    pipe.seg_tile(rgb, hem8, labels, edt, nobj, stream=stream)
    out = {}
    if want_planes:
        for k, name in enumerate(("R", "fg", "filled")):
            buf = torch.empty((H, W), dtype=torch.uint8, device=dev)
            pipe.debug_plane(k, buf, stream=stream)
            out[name] = buf
    torch.cuda.synchronize()
    K = int(nobj.item())
    feats = torch.zeros((max(K, 1), 15), dtype=torch.float32, device=dev)
    pipe.features_tile(hem8, labels, K, feats, stream=stream)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res.update(hem8=hem8.cpu().numpy(), labels=labels.cpu().numpy(), edt=edt.cpu().numpy(), K=K,
               feats=feats.cpu().numpy()[:K])
    return res


def oracle_all(rgb_np, h=20, thr=10, amin=20, amax=1500):
    r = oracle.seg(rgb_np, h=h, thr=thr, amin=amin, amax=amax, planes=True)
    r["feats"] = oracle.features(r["hem8"], r["labels"], r["K"])
    return r


def assert_feats_close(got, ref):
    assert got.shape == ref.shape, (got.shape, ref.shape)
    err = np.abs(got.astype(np.float64) - ref)
    ok = (err <= TOL_REL * np.abs(ref)) | (err <= TOL_ABS)
    if not ok.all():
        i, j = np.argwhere(~ok)[0]
        raise AssertionError("feature [%d][%d]: gpu %r oracle %r (%d bad of %d)"
                             % (i, j, got[i, j], ref[i, j], int((~ok).sum()), ok.size))


def assert_planes_equal(g, r, planes=("hem8", "R", "fg", "filled", "labels", "edt")):
    for k in planes:
        if k not in g:
            continue
        a, b = g[k], r[k]
        if not np.array_equal(a, b):
            bad = np.argwhere(a != b)
            y, x = bad[0]
            raise AssertionError("%s differs at %d pixels; first (%d,%d): gpu %r oracle %r"
                                 % (k, len(bad), y, x, a[y, x], b[y, x]))
    assert g["K"] == r["K"], (g["K"], r["K"])


# ---- many tiles: oracle outputs computed in a process pool ------------------

def plane_digest(a):
    import hashlib
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def make_tile(spec):
    """spec: ("cfg2"|"cfg3"|"cfg4", i) for the synth presets, or
    ("bench", seed) for a tile of the 4096^2 benchmark workload."""
    import synth
    kind, i = spec
    if kind == "bench":
        return synth.tile(4096, 4096, i, n_nuclei=3000, frac_cluster=0.2, n_stroma=150)
    return getattr(synth, kind)(i)


def oracle_digest(spec):
    """Oracle result of one seeded tile: K, FP64 features and a SHA-256
    digest of each integer plane (compared bit for bit with the GPU's)."""
    rgb = make_tile(spec)
    r = oracle.seg(rgb, planes=False)
    feats = oracle.features(r["hem8"], r["labels"], r["K"])
    return dict(K=r["K"], feats=feats, hem8=plane_digest(r["hem8"]), labels=plane_digest(r["labels"]),
                edt=plane_digest(r["edt"]))


def oracle_digests(specs):
    """oracle_digest over a spawn-started process pool (fork after CUDA
    initialisation is unsafe)."""
    import concurrent.futures
    import multiprocessing
    import os
    n = max(1, min(len(specs), os.cpu_count() or 1))
    with concurrent.futures.ProcessPoolExecutor(n, mp_context=multiprocessing.get_context("spawn")) as ex:
        return list(ex.map(oracle_digest, specs))


def assert_matches_digest(got, ref, rgb=None, what=""):
    """got: dict with K, feats and (optionally) hem8/labels/edt planes."""
    assert got["K"] == ref["K"], (what, got["K"], ref["K"])
    for k in ("hem8", "labels", "edt"):
        if k in got and got[k] is not None and plane_digest(got[k]) != ref[k]:
            if rgb is not None:  # locate the first difference
                assert_planes_equal(got, oracle_all(rgb), planes=(k,))
            raise AssertionError("%s: plane %s differs from the oracle" % (what, k))
    assert_feats_close(got["feats"], ref["feats"])


def assert_same_feats(a, b, what=""):
    """Bit-identical feature rows (two forms of the CUDA path)."""
    assert a.shape == b.shape, (what, a.shape, b.shape)
    if not np.array_equal(a, b):
        bad = np.argwhere(a != b)
        i, j = bad[0]
        raise AssertionError("%s feature [%d][%d]: %r vs %r (%d differ)" % (what, i, j, a[i, j], b[i, j], len(bad)))
