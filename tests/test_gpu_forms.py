"""Batched and served forms: each tile's result equals the plain form's on
the same tile alone (bit for bit, features included) and the oracle's, while
tiles of uneven size and density share launches and run concurrently."""
import time

import numpy as np
import pytest

import synth
from tests.gpu_util import assert_feats_close, assert_planes_equal, assert_same_feats, oracle_all, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pipe():
    import torch
    import paper_1209_3332_gb300 as P
    from paper_1209_3332_gb300 import build
    build.build()
    torch.cuda.init()
    p = P.Pipe(0, max_slots=4)
    yield p
    assert p.status() == P.PIPE_OK
    p.close()


def mixed_tiles():
    tiles = [synth.tile(640, 480, 21, n_nuclei=0),                                    # empty
             synth.tile(1024, 1024, 22, n_nuclei=300, frac_cluster=0.2, n_stroma=10),  # dense
             synth.tile(333, 517, 23, n_nuclei=40, frac_overlap=0.1),                 # ragged
             synth.tile(1, 77, 24),
             synth.tile(2048, 1536, 25, n_nuclei=700, frac_chain=0.5, corridor=True)]
    return tiles


def run_batched(pipe, tiles, caps=None):
    import torch
    dev = torch.device("cuda", 0)
    bufs = []
    for i, t in enumerate(tiles):
        H, W = t.shape[:2]
        cap = caps[i] if caps else max(1, W * H // 20 + 1)
        bufs.append(dict(rgb=torch.from_numpy(t).to(dev), hem8=torch.empty((H, W), dtype=torch.uint8, device=dev),
                         labels=torch.empty((H, W), dtype=torch.int32, device=dev),
                         edt=torch.empty((H, W), dtype=torch.int32, device=dev),
                         n_objects=torch.zeros(1, dtype=torch.int32, device=dev),
                         feats=torch.zeros((cap, 15), dtype=torch.float32, device=dev)))
    pipe.seg_features_batch(bufs)
    torch.cuda.synchronize()
    out = []
    for b in bufs:
        K = int(b["n_objects"].item())
        out.append(dict(hem8=b["hem8"].cpu().numpy(), labels=b["labels"].cpu().numpy(),
                        edt=b["edt"].cpu().numpy(), K=K, feats=b["feats"][:min(K, b["feats"].shape[0])].cpu().numpy()))
    return out


def test_batched_equals_plain_and_oracle(pipe):
    tiles = mixed_tiles()
    got = run_batched(pipe, tiles)
    for t, g in zip(tiles, got):
        alone = run_gpu(pipe, t, want_planes=False)
        assert_planes_equal(g, alone, planes=("hem8", "labels", "edt"))
        assert_same_feats(g["feats"], alone["feats"], "batched vs plain")
        r = oracle_all(t)
        assert_planes_equal(g, r, planes=("hem8", "labels", "edt"))
        assert_feats_close(g["feats"], r["feats"])


def test_batched_graph_replay_and_shape_change(pipe):
    tiles = mixed_tiles()[:3]
    a = run_batched(pipe, tiles)
    b = run_batched(pipe, tiles)          # replayed from the captured graph
    c = run_batched(pipe, tiles[::-1])    # another shape -> another graph
    for x, y in zip(a, b):
        assert_planes_equal(x, y, planes=("hem8", "labels", "edt"))
        assert_same_feats(x["feats"], y["feats"], "graph replay")
    for x, y in zip(a, c[::-1]):
        assert_planes_equal(x, y, planes=("hem8", "labels", "edt"))


def test_batched_feature_capacity_overflow_is_reported(pipe):
    import paper_1209_3332_gb300 as P
    t = synth.tile(512, 512, 31, n_nuclei=80)
    got = run_batched(pipe, [t], caps=[3])
    assert got[0]["K"] > 3
    assert pipe.status() == P.PIPE_EOVERFLOW
    r = oracle_all(t)
    assert_feats_close(got[0]["feats"], r["feats"][:3])


def wait(pipe, tk, timeout=60):
    t0 = time.time()
    while True:
        r = pipe.poll(tk)
        if r is not None:
            return r
        assert time.time() - t0 < timeout
        time.sleep(0.001)


def test_served_alone_and_in_the_mix(pipe):
    import torch
    tiles = mixed_tiles()
    alone = []
    for t in tiles:
        tk = pipe.submit([t], want_planes=True)
        alone.append(wait(pipe, tk)[0])
    # in the mix: several groups in flight at once, pinned and pageable inputs
    pinned = [torch.from_numpy(t).pin_memory() for t in tiles[:2]]
    tks = [pipe.submit(pinned, want_planes=True), pipe.submit(tiles[2:4], want_planes=True),
           pipe.submit([tiles[4]], want_planes=True)]
    assert all(tk is not None for tk in tks)
    mixed = []
    for tk in tks:
        mixed.extend(wait(pipe, tk))
    for t, a, m in zip(tiles, alone, mixed):
        assert a["status"] == 0 and m["status"] == 0
        for k in ("hem8", "labels", "edt"):
            assert np.array_equal(a[k], m[k]), k
        assert a["n_objects"] == m["n_objects"]
        assert_same_feats(a["feats"], m["feats"], "served alone vs mix")
        r = oracle_all(t)
        assert a["n_objects"] == r["K"]
        for k in ("hem8", "labels", "edt"):
            assert np.array_equal(a[k], r[k]), k
        assert_feats_close(a["feats"], r["feats"])
        assert m["t_done_ms"] >= m["t_arrive_ms"]


def test_served_admission_refused_when_slots_full(pipe):
    t = synth.tile(256, 256, 41, n_nuclei=10)
    tks = []
    for _ in range(4):
        tk = pipe.submit([t])
        assert tk is not None
        tks.append(tk)
    assert pipe.submit([t]) is None       # max_slots=4 contexts are busy until polled
    for tk in tks:
        wait(pipe, tk)
    tk = pipe.submit([t])
    assert tk is not None
    assert wait(pipe, tk)[0]["status"] == 0


def test_autotune_keeps_results_and_cache_file_round_trip(tmp_path):
    """Launch shapes change no result; a second pipe reads the tuned shapes
    from the cache file instead of tuning again."""
    import paper_1209_3332_gb300 as P
    tiles = mixed_tiles()[:3]
    cache = str(tmp_path / "shapes.txt")
    a = P.Pipe(0, autotune=1, autotune_cache=cache)
    got_a = run_batched(a, tiles)
    info_a = a.autotune_info()
    assert info_a["tune_runs"] > 0
    a.close()
    lines = open(cache).read().splitlines()
    assert len(lines) == 1 and lines[0].split(" ")[0].endswith("640x480;1024x1024;333x517;")
    b = P.Pipe(0, autotune=0)
    got_b = run_batched(b, tiles)
    assert b.autotune_info()["tune_runs"] == 0
    b.close()
    c = P.Pipe(0, autotune=1, autotune_cache=cache)
    got_c = run_batched(c, tiles)
    info_c = c.autotune_info()
    assert info_c["tune_runs"] == 0
    assert {k: info_c[k] for k in ("recon_workers", "edt_rows", "feat_blocks")} == \
        {k: info_a[k] for k in ("recon_workers", "edt_rows", "feat_blocks")}
    assert c.status() == P.PIPE_OK
    c.close()
    for x, y, z in zip(got_a, got_b, got_c):
        for k in ("hem8", "labels", "edt"):
            assert np.array_equal(x[k], y[k]) and np.array_equal(x[k], z[k]), k
        assert np.array_equal(x["feats"], y["feats"]) and np.array_equal(x["feats"], z["feats"])


def test_served_budget_counts_idle_contexts():
    """The HBM budget bounds the device memory of every served context, busy
    or idle: groups of alternating sizes, up to two in flight, never leave
    more than hbm_budget_bytes allocated, and every result equals the tile's
    result alone."""
    import paper_1209_3332_gb300 as P
    small = [synth.tile(512, 384, 61, n_nuclei=40)]
    big = [synth.tile(1024, 1024, 62 + i, n_nuclei=250, frac_cluster=0.2) for i in range(3)]
    probe = P.Pipe(0, max_slots=3)
    ref = {}
    for grp in (small, big):
        for t, r in zip(grp, wait(probe, probe.submit(grp))):
            ref[id(t)] = r
    probe.close()
    one_big = P.Pipe(0, max_slots=1)
    wait(one_big, one_big.submit(big))
    need_big = one_big.serve_memory()["allocated"]
    one_big.close()
    budget = int(1.5 * need_big)
    p = P.Pipe(0, max_slots=3, hbm_budget_bytes=budget)
    # a context stays busy until its ticket is polled, so a second big group
    # submitted before any poll cannot fit beside the first
    tk = p.submit(big)
    assert tk is not None
    assert p.submit(big) is None
    assert p.serve_memory()["allocated"] <= budget
    seq = [small, big[:2], small, big, big[:1], small + big[:1], big]
    inflight, k = [(tk, big)], 0
    t0 = time.time()
    while k < len(seq) or inflight:
        if k < len(seq) and len(inflight) < 2:
            tk = p.submit(seq[k])
            assert p.serve_memory()["allocated"] <= budget
            if tk is not None:
                inflight.append((tk, seq[k]))
                k += 1
        still = []
        for tk, grp in inflight:
            res = p.poll(tk)
            if res is None:
                still.append((tk, grp))
                continue
            for t, r in zip(grp, res):
                assert r["status"] == 0
                assert r["n_objects"] == ref[id(t)]["n_objects"]
                assert_same_feats(r["feats"], ref[id(t)]["feats"], "served under a small budget")
        inflight = still
        assert p.serve_memory()["allocated"] <= budget
        assert time.time() - t0 < 120
    m = p.serve_memory()
    assert m["in_flight"] == 0 and m["allocated"] <= budget
    assert p.status() == P.PIPE_OK
    p.close()


def test_served_concurrent_polls_keep_each_tickets_results(pipe):
    """Two threads poll their own tickets at once: a poll never releases
    another ticket's results (they stay until that ticket is released)."""
    import threading
    tiles = [synth.tile(768, 512, 71 + i, n_nuclei=120, frac_cluster=0.2) for i in range(4)]
    ref = [wait(pipe, pipe.submit([t]))[0] for t in tiles]
    tks = [pipe.submit([t]) for t in tiles]
    assert all(tk is not None for tk in tks)
    got = [None] * 4
    errs = []

    def worker(idx):
        try:
            for i in idx:
                got[i] = wait(pipe, tks[i])[0]
        except Exception as e:  # reported by the main thread
            errs.append(e)
    th = [threading.Thread(target=worker, args=(idx,)) for idx in ((0, 2), (1, 3))]
    for t in th:
        t.start()
    for t in th:
        t.join(120)
    assert not errs, errs
    for a, b in zip(got, ref):
        assert a["n_objects"] == b["n_objects"]
        assert_same_feats(a["feats"], b["feats"], "concurrent polls")
