"""Benchmark: 4096x4096 tiles per second through the segmentation + feature path.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--batch B]
                    [--impl ours|reference] [--no-cpu] [--no-extra] [--no-configs]

One step is one pass of the whole path -- colour deconvolution, h-dome
reconstruction, fill holes, labelling + area filter + relabel, EDT and
per-object features -- over one batch of B synthetic 4096x4096 tiles in the
batched form (one launch per pass over all tiles, replayed from a CUDA
graph).  Tiles are generated like the 4096^2 workload (~3000 nuclei, 20% in
touching clusters of 2-6, 150 stroma discs), each with its own seed.  Inputs
are resident in HBM when the timed region starts; a batch's inputs alone
(B x 48 MiB) and its planes exceed the 129 MB L2.

Reported beside the batched value: the plain form (seg_tile + features_tile,
one tile per call) on the same tiles; the served form (batch_submit /
batch_poll under Poisson arrivals at 80% and at 125% of the batched rate,
with p50/p99 latency); an end-to-end figure (whole batches submitted from
pinned host memory through the served API and polled to completion);
per-kernel CUDA event times; the roofline of the dominant kernel; the steps
beside the path (RBC detection, opening, watershed, Canny); the other workloads -- the
64-tile mixed batch (batched vs plain), the served pool (2000 Poisson
requests at 80% of the mixed batch's rate under the 40 GiB budget) and the
stress stream (4096 worst-case tiles from pinned host memory, against the
batched and plain forms), each result checked bit for bit against the
batched form; and the CPU oracle.

N>1: every rank is an independent replica on its own tiles (the path shards
by tile; there is no data exchange), value = all tiles / max time.  Under
torchrun the ranks come from the environment; with --gpus N and no
WORLD_SIZE, bench.py starts the N ranks itself under torch.distributed.run.

--impl reference times the CPU oracle (the plain C program written from the
paper's definitions) on this host's cores on full tiles of the same
workload; rank 0 only.
"""
import argparse
import hashlib
import json
import math
import os
import random
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "4Kx4K tiles/sec/GB300 (batched+served vs plain) at bit-exact seg; p50/p99 ms"
WORKLOAD = ("4096x4096 RGB uint8 tiles, ~3000 nuclei (20% in touching clusters of 2-6) + 150 stroma "
            "discs r40-120; h=20, dome>=10, area [20,1500], 8-level GLCM x4 offsets")
# algorithmic HBM bytes per pixel of each step (each step reads its inputs and
# writes its outputs once)
BYTES_PER_PX = {"deconv": 4, "recon": 2, "fill": 2, "label": 13, "edt": 16, "features": 5}
KERNEL_STAGE = {"recon": "recon", "deconv": "deconv", "edt_rows": "edt", "relabel": "label",
                "feat_objects": "features", "fill_local": "fill", "label_local": "label"}
PATH_BYTES_PER_PX = 42
IO_BYTES_PER_PX = 12  # compulsory: RGB in (3) + hem8 (1), labels (4), edt (4) out
H = W = 4096


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_traffic(name):
    """DRAM bytes per 4096^2 launch from the committed ncu summary, if the
    kernel's source is unchanged since the capture (else None)."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            d = json.load(f)
        ent = d[name]
        src = os.path.join(ROOT, "paper_1209_3332_gb300", "csrc", ent["source"])
        if hashlib.sha256(open(src, "rb").read()).hexdigest() != ent["source_sha256"]:
            return None
        return float(ent["dram_bytes_per_launch"])
    except Exception:
        return None


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, v):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def tile_seed(rank, i):
    """Seed of tile i of rank `rank`; rank 0's first tile is the 4096^2 workload tile."""
    return 1000 if (rank == 0 and i == 0) else 1000 + 7919 * (rank * 256 + i)


def gen_tiles(n, rank):
    import synth
    return [synth.tile(W, H, tile_seed(rank, i), n_nuclei=3000, frac_cluster=0.2, n_stroma=150)
            for i in range(n)]


def _oracle_worker_init(shm_name, shape):
    global _ORACLE_TILE, _ORACLE_SHM
    from multiprocessing import shared_memory
    import numpy as np
    _ORACLE_SHM = shared_memory.SharedMemory(name=shm_name)
    _ORACLE_TILE = np.ndarray(shape, dtype=np.uint8, buffer=_ORACLE_SHM.buf)


def _oracle_worker_run(n):
    """Runs the whole oracle path (segmentation + features) n times on the
    shared tile; returns the seconds it took."""
    import oracle
    t0 = time.perf_counter()
    for _ in range(n):
        r = oracle.seg(_ORACLE_TILE)
        oracle.features(r["hem8"], r["labels"], r["K"])
    return time.perf_counter() - t0


class OraclePool:
    """The CPU oracle as a bag of tasks over this host's cores: one
    single-threaded oracle process per core, each working on its own copy of
    a full tile (the paper's multi-core CPU runs are a bag of independent
    tiles too).  Processes are started with spawn, before or after CUDA
    initialisation alike."""

    def __init__(self, tile, procs=None):
        import concurrent.futures
        import multiprocessing
        from multiprocessing import shared_memory
        import numpy as np
        import oracle
        oracle.build()
        self.procs = procs or os.cpu_count() or 1
        self.shm = shared_memory.SharedMemory(create=True, size=tile.nbytes)
        np.ndarray(tile.shape, dtype=np.uint8, buffer=self.shm.buf)[...] = tile
        self.ex = concurrent.futures.ProcessPoolExecutor(
            self.procs, mp_context=multiprocessing.get_context("spawn"),
            initializer=_oracle_worker_init, initargs=(self.shm.name, tile.shape))

    def step(self):
        """One tile per process, all at once; returns wall seconds."""
        t0 = time.perf_counter()
        list(self.ex.map(_oracle_worker_run, [1] * self.procs))
        return time.perf_counter() - t0

    def close(self):
        self.ex.shutdown()
        self.shm.close()
        self.shm.unlink()


def cpu_baseline(tile, steps=2):
    """The oracle as it stands on this host's cores: a bag-of-tasks warm-up
    step then `steps` timed steps of one full tile per core, and one tile on
    a single core."""
    import oracle
    pool = OraclePool(tile)
    try:
        pool.step()
        el = sum(pool.step() for _ in range(steps))
    finally:
        pool.close()
    t0 = time.perf_counter()
    r = oracle.seg(tile)
    oracle.features(r["hem8"], r["labels"], r["K"])
    single = time.perf_counter() - t0
    return {"value": steps * pool.procs / el, "unit": "tiles/s", "cores": pool.procs, "kind": "oracle",
            "sample": "%d steps x %d processes, each the single-threaded C oracle (segmentation + features) "
                      "on one full 4096x4096 tile of the benchmark workload, %.1f s" % (steps, pool.procs, el),
            "single_core_tiles_per_s": 1.0 / single}


def run_reference(args, world, rank):
    if rank != 0:
        return
    tile = gen_tiles(1, 0)[0]
    pool = OraclePool(tile)
    try:
        for _ in range(args.warmup):
            pool.step()
        times = [pool.step() for _ in range(args.steps)]
    finally:
        pool.close()
    ms = 1000.0 * statistics.mean(times)
    val = pool.procs * 1000.0 / ms
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "tiles/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": WORKLOAD, "form": "CPU oracle, bag of tasks: one tile per host core per step",
                       "tiles_per_step": pool.procs},
            "cpu_baseline": {"value": val, "unit": "tiles/s", "cores": pool.procs, "kind": "oracle",
                             "sample": "%d steps, each one full 4096x4096 tile on each of %d single-threaded "
                                       "oracle processes" % (args.steps, pool.procs)},
            "e2e": {"value": val, "unit": "tiles/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def device_buffers(torch, dev, host, feats_cap):
    bufs = []
    for h in host:
        bufs.append(dict(rgb=torch.from_numpy(h).to(dev), hem8=torch.empty((H, W), dtype=torch.uint8, device=dev),
                         labels=torch.empty((H, W), dtype=torch.int32, device=dev),
                         edt=torch.empty((H, W), dtype=torch.int32, device=dev),
                         n_objects=torch.zeros(1, dtype=torch.int32, device=dev),
                         feats=torch.empty((feats_cap, 15), dtype=torch.float32, device=dev)))
    return bufs


def timed(torch, stream, fn, steps):
    """CUDA-event time of `steps` calls of fn on `stream`, ms."""
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


MORPH_R = 9                      # the 19x19 disk of Table I "Morph. Open"
# instruction issue of the GB300: 152 SMs x 4 schedulers, one warp instruction each per clock
ISSUE_PER_CLK = 152 * 4


def kernel_instructions(name):
    """Warp instructions per 4096^2 plane from the committed ncu capture, if
    the kernel's source is unchanged since the capture (else None)."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            ent = json.load(f)[name]
        src = os.path.join(ROOT, "paper_1209_3332_gb300", "csrc", ent["source"])
        if hashlib.sha256(open(src, "rb").read()).hexdigest() != ent["source_sha256"]:
            return None
        return float(ent["warp_instructions_per_plane"])
    except Exception:
        return None


def morph_open_run(torch, pipe, stream, planes, steps, hbm_peak, want_cpu):
    """The opening by the 19x19 disk (Table I "Morph. Open") of every hem8
    plane of the batch through morph_open_tile, timed with CUDA events on the
    launching stream (planes larger than L2 in all).  The passes are bound by
    instruction issue (ncu: issue active 66%, ALU and load/store pipes near
    55%, DRAM 4%), so the roofline is the SMs' issue rate, against the warp
    instructions the committed ncu capture counted per plane."""
    outs = [torch.empty_like(p) for p in planes]

    def step():
        for a, b in zip(planes, outs):
            pipe.morph_open(a, b, MORPH_R, stream=stream)
    for _ in range(3):
        step()
    ms = timed(torch, stream, step, steps) / steps
    n = len(planes)
    px = n * planes[0].numel()
    mhz = peaks_clock()
    gbs = 2.0 * px / (ms / 1000.0) / 1e9                       # read once, write once
    out = {"radius": MORPH_R, "planes_per_step": n, "plane": list(planes[0].shape), "ms_per_step": ms,
           "planes_per_s": n * 1000.0 / ms,
           "hbm": {"achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                   "alg_bytes_per_px": 2},
           "parity": "bit-exact with the oracle (tests/test_gpu_morph.py)"}
    inst = kernel_instructions("morph_stream")
    if inst is not None and tuple(planes[0].shape) == (H, W):
        issue_peak = ISSUE_PER_CLK * mhz * 1e6 / 1e9                  # G warp-instructions/s
        ach = inst * n / (ms / 1000.0) / 1e9
        out["roofline"] = {"bound": "issue", "achieved": ach, "peak": issue_peak, "unit": "G warp-inst/s",
                           "frac": ach / issue_peak, "warp_instructions_per_plane": inst,
                           "peak_source": "derived: 152 SMs x 4 schedulers x 1 warp instruction per clock x %.0f "
                                          "MHz; instructions executed from the committed ncu capture "
                                          "(profiles/k_morph_stream_4096.md)" % mhz}
    if want_cpu:
        import time
        import oracle
        a = planes[0][:128 + 4 * MORPH_R].cpu().numpy()     # a band of 128 output rows plus its halo
        t = time.perf_counter()
        oracle.morph_open(a, MORPH_R)
        s = time.perf_counter() - t
        out["cpu_oracle"] = {"planes_per_s": (a.shape[0] * a.shape[1]) / planes[0].numel() / s, "cores": 1,
                             "sample": "the oracle on one band of %d x %d pixels of plane 0, %.2f s, scaled"
                                       % (a.shape[0], a.shape[1], s)}
    return out


WS_H = 1                  # marker height of the watershed split (h-maxima of the integer distance)
WS_BYTES_PER_PX = 12      # minimal pass: labels and EDT read once, the split plane written once


def watershed_run(torch, pipe, stream, bufs, steps, hbm_peak, want_cpu):
    """The watershed split (Table I "Pre-Watershed" + "Watershed") of every
    tile of the batch, on the labels and EDT the batched step wrote: the
    batched form (watershed_batch) as the figure, one watershed_tile call per
    tile beside it; timed with CUDA events on the launching stream (the
    planes of the batch are far larger than L2).  Per-kernel times (batched
    form) come from the pipe's own events around each launch."""
    ks = [int(b["n_objects"].item()) for b in bufs]
    outs = [torch.empty_like(b["labels"]) for b in bufs]
    nb = torch.zeros(len(bufs), dtype=torch.int32, device=bufs[0]["labels"].device)

    def plain():
        for i, b in enumerate(bufs):
            pipe.watershed(b["labels"], b["edt"], ks[i], outs[i], nb[i:i + 1], h=WS_H, stream=stream)
    batch = [dict(labels=b["labels"], edt=b["edt"], out=outs[i], n_objects=ks[i], n_basins=nb[i:i + 1])
             for i, b in enumerate(bufs)]

    def step():
        pipe.watershed_batch(batch, h=WS_H, stream=stream)
    for _ in range(3):
        plain()
    plain_ms = timed(torch, stream, plain, steps) / steps
    for _ in range(3):
        step()
    ms = timed(torch, stream, step, steps) / steps
    before = pipe.profile_read()
    pipe.profile(True)
    step()
    torch.cuda.synchronize()
    after = pipe.profile_read()
    pipe.profile(False)
    kern = {}
    for k, (c, t) in after.items():
        c0, t0 = before.get(k, (0, 0.0))
        if c > c0 and (k.startswith("ws_") or k.startswith("feat_bbox")):
            kern[k] = round((t - t0) / (c - c0), 4)
    n = len(bufs)
    px = sum(b["labels"].numel() for b in bufs)
    gbs = WS_BYTES_PER_PX * px / (ms / 1000.0) / 1e9
    out = {"h": WS_H, "form": "batched (watershed_batch: the objects of all tiles in one launch per pass)",
           "tiles_per_step": n, "tile": list(bufs[0]["labels"].shape), "ms_per_step": ms,
           "tiles_per_s": n * 1000.0 / ms,
           "plain": {"form": "watershed_tile per tile", "ms_per_step": plain_ms, "tiles_per_s": n * 1000.0 / plain_ms},
           "objects_per_step": sum(ks),
           "basins_per_step": int(nb.sum().item()), "kernels_ms": kern,
           "hbm": {"achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                   "alg_bytes_per_px": WS_BYTES_PER_PX,
                   "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)"},
           "parity": "bit-exact with the oracle (tests/test_gpu_watershed.py)"}
    if want_cpu:
        import time
        import oracle
        rows = 512                                              # a band of the first tile
        lab = bufs[0]["labels"][:rows].cpu().numpy()
        edt = bufs[0]["edt"][:rows].cpu().numpy()
        t = time.perf_counter()
        oracle.watershed(lab, edt, WS_H)
        sec = time.perf_counter() - t
        out["cpu_oracle"] = {"tiles_per_s": lab.size / bufs[0]["labels"].numel() / sec, "cores": 1,
                             "sample": "the oracle on the first %d rows of tile 0 (%d x %d pixels), %.2f s, scaled"
                                       % (rows, lab.shape[0], lab.shape[1], sec)}
    return out


CANNY_LOW, CANNY_HIGH, EDGE_R = 40, 120, 3   # thresholds on the L1 Sobel magnitude; disk radius of the counts
CANNY_BYTES_PER_PX = 2                        # minimal pass: the plane read once, the edge map written once


def canny_run(torch, pipe, stream, bufs, steps, hbm_peak, want_cpu):
    """Canny edges of every hem8 plane of the batch and the edge counts of
    its objects (Sec. V-A feature-stage transform, Sec. II edge features):
    the batched form (canny_batch: one launch per pass over all tiles) as the
    figure, one canny_tile call per tile beside it; timed with CUDA events on
    the launching stream (the planes of the batch are far larger than L2)."""
    ks = [int(b["n_objects"].item()) for b in bufs]
    edges = [torch.empty_like(b["hem8"]) for b in bufs]
    counts = [torch.empty(max(k, 1), dtype=torch.int32, device=b["hem8"].device) for k, b in zip(ks, bufs)]
    jobs = [dict(img=b["hem8"], edges=edges[i], labels=b["labels"], n_objects=ks[i], counts=counts[i])
            for i, b in enumerate(bufs)]

    def plain():
        for i, b in enumerate(bufs):
            pipe.canny(b["hem8"], edges[i], labels=b["labels"], n_objects=ks[i], counts=counts[i],
                       low=CANNY_LOW, high=CANNY_HIGH, radius=EDGE_R, stream=stream)

    def step():
        pipe.canny_batch(jobs, low=CANNY_LOW, high=CANNY_HIGH, radius=EDGE_R, stream=stream)
    for _ in range(3):
        plain()
    plain_ms = timed(torch, stream, plain, steps) / steps
    ref = [(e.clone(), c.clone()) for e, c in zip(edges, counts)]
    for _ in range(3):
        step()
    ms = timed(torch, stream, step, steps) / steps
    for (e0, c0), e, c in zip(ref, edges, counts):
        if not torch.equal(e0, e) or not torch.equal(c0, c):
            raise RuntimeError("canny_batch differs from canny_tile")
    before = pipe.profile_read()
    pipe.profile(True)
    step()
    torch.cuda.synchronize()
    after = pipe.profile_read()
    pipe.profile(False)
    kern = {}
    for k, (c, t) in after.items():
        c0, t0 = before.get(k, (0, 0.0))
        if c > c0:
            kern[k] = round((t - t0) / (c - c0), 4)
    n = len(bufs)
    px = sum(b["hem8"].numel() for b in bufs)
    out = {"low": CANNY_LOW, "high": CANNY_HIGH, "radius": EDGE_R, "tiles_per_step": n,
           "form": "batched (canny_batch: one launch per pass over all tiles)",
           "tile": list(bufs[0]["hem8"].shape), "ms_per_step": ms, "tiles_per_s": n * 1000.0 / ms,
           "plain": {"form": "canny_tile per tile", "ms_per_step": plain_ms, "tiles_per_s": n * 1000.0 / plain_ms},
           "edge_px_per_step": int(sum(int(e.sum().item()) for e in edges)), "kernels_ms": kern,
           "hbm": {"achieved": CANNY_BYTES_PER_PX * px / (ms / 1000.0) / 1e9, "peak": hbm_peak, "unit": "GB/s",
                   "alg_bytes_per_px": CANNY_BYTES_PER_PX,
                   "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)"},
           "parity": "batched == plain bit for bit in this run; bit-exact with the oracle (tests/test_gpu_canny.py)"}
    out["hbm"]["frac"] = out["hbm"]["achieved"] / hbm_peak
    nms_ms = kern.get("canny_nms", 0.0)
    if nms_ms > 0:  # the stencil pass alone: the planes read once, strong and candidate planes written
        gbs = 3.0 * px / (nms_ms / 1000.0) / 1e9
        out["nms_kernel"] = {"achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                             "alg_bytes_per_px": 3}
    cnt_ms = kern.get("canny_counts", 0.0)
    if cnt_ms > 0:  # the counts pass alone: edges and labels read once
        gbs = 5.0 * px / (cnt_ms / 1000.0) / 1e9
        out["counts_kernel"] = {"achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                                "alg_bytes_per_px": 5}
    if want_cpu:
        import time
        import oracle
        rows = 1024
        img = bufs[0]["hem8"][:rows].cpu().numpy()
        lab = bufs[0]["labels"][:rows].cpu().numpy()
        t = time.perf_counter()
        e = oracle.canny(img, CANNY_LOW, CANNY_HIGH)
        oracle.edge_counts(e, lab, ks[0], EDGE_R)
        sec = time.perf_counter() - t
        out["cpu_oracle"] = {"tiles_per_s": img.size / bufs[0]["hem8"].numel() / sec, "cores": 1,
                             "sample": "the oracle on the first %d rows of tile 0 (%d x %d pixels), %.2f s, scaled"
                                       % (rows, img.shape[0], img.shape[1], sec)}
    return out


RBC_LO, RBC_HI = 40, 100       # red-dominance thresholds of the RBC mask and markers
RBC_BYTES_PER_PX = 4           # minimal pass: RGB read once, the mask written once
RBC_TILES, RBC_CELLS = 8, 800  # 4096^2 tiles of the workload with red blood cells painted in


def rbc_run(torch, pipe, stream, steps, hbm_peak, want_cpu):
    """RBC detection (Table I "RBC detection") of 4096^2 workload tiles with
    red blood cells through rbc_tile, one call per tile, timed with CUDA
    events on the launching stream (the RGB planes exceed L2); tile 0 is
    checked against the oracle bit for bit."""
    import numpy as np
    import synth
    dev = torch.device("cuda", torch.cuda.current_device())
    host = [synth.tile(W, H, 5000 + i, n_nuclei=3000, frac_cluster=0.2, n_stroma=150, n_rbc=RBC_CELLS)
            for i in range(RBC_TILES)]
    rgb = [torch.from_numpy(h).to(dev) for h in host]
    outs = [torch.empty((H, W), dtype=torch.uint8, device=dev) for _ in host]

    def step():
        for a, b in zip(rgb, outs):
            pipe.rbc(a, b, RBC_LO, RBC_HI, stream=stream)
    for _ in range(3):
        step()
    ms = timed(torch, stream, step, steps) / steps
    before = pipe.profile_read()
    pipe.profile(True)
    step()
    torch.cuda.synchronize()
    after = pipe.profile_read()
    pipe.profile(False)
    kern = {}
    for k, (c, t) in after.items():
        c0, t0 = before.get(k, (0, 0.0))
        if c > c0:
            kern[k] = round((t - t0) / (c - c0), 4)
    import oracle
    t0 = time.perf_counter()
    want = oracle.rbc(host[0], RBC_LO, RBC_HI)
    cpu_s = time.perf_counter() - t0
    if not np.array_equal(outs[0].cpu().numpy(), want):
        raise RuntimeError("rbc_tile differs from the oracle on tile 0")
    px = RBC_TILES * H * W
    gbs = RBC_BYTES_PER_PX * px / (ms / 1000.0) / 1e9
    out = {"t_lo": RBC_LO, "t_hi": RBC_HI, "tiles_per_step": RBC_TILES, "tile": [H, W],
           "workload": "4096x4096 tiles as the benchmark's, plus %d red blood cells (discs r 3.5-5.5, RGB ~(200,60,70), "
                       "30%% of draws in clumps of 2-5)" % RBC_CELLS,
           "ms_per_step": ms, "tiles_per_s": RBC_TILES * 1000.0 / ms,
           "rbc_px_tile0": int(want.sum()), "kernels_ms": kern,
           "hbm": {"achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                   "alg_bytes_per_px": RBC_BYTES_PER_PX, "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)"},
           "parity": "tile 0 equals the oracle bit for bit in this run; tests/test_gpu_rbc.py"}
    pl = kern.get("rbc_planes")
    if pl:   # the planes pass alone: RGB read, marker and mask written
        g = 5.0 * H * W / (pl / 1000.0) / 1e9
        out["planes_kernel"] = {"achieved": g, "peak": hbm_peak, "unit": "GB/s", "frac": g / hbm_peak,
                                "alg_bytes_per_px": 5}
    if want_cpu:
        out["cpu_oracle"] = {"tiles_per_s": 1.0 / cpu_s, "cores": 1, "sample": "the oracle on tile 0, %.2f s" % cpu_s}
    return out


def peaks_clock():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f).get("sm_max_mhz", 2070.0))
    except (OSError, ValueError):
        return 2070.0


def h2d_gbs(torch, dev, nbytes=256 << 20, reps=4):
    """Pinned host-to-device copy bandwidth (best of reps), GB/s."""
    src = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    dst = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    s = torch.cuda.Stream(dev)
    best = 0.0
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(s)
        with torch.cuda.stream(s):
            dst.copy_(src, non_blocking=True)
        e1.record(s)
        torch.cuda.synchronize()
        best = max(best, nbytes / (e0.elapsed_time(e1) / 1000.0) / 1e9)
    del src, dst
    return best


def serve_run(pipe, pinned, n_requests, rate, seed=3999, max_group=16, max_inflight=2, limit_s=120.0, costs=None,
              check=None):
    """Poisson arrivals at `rate` tiles/s; each request is one pool tile.
    Continuous batching: whenever fewer than max_inflight groups are on the
    device, the requests that have arrived (up to max_group) are admitted as
    the next group, so one group uploads while the previous one computes.
    Without `costs` the group takes them in order of arrival; with `costs`
    (an estimate per pool tile) they wait in the dispatcher's queue
    (P.Sched) and the group takes the most expensive first.  check(pool
    index, result) is called on every result (it raises on a mismatch).
    Also reports the served contexts' peak device memory."""
    import paper_1209_3332_gb300 as P
    rng = random.Random(seed)
    arrivals, t = [], 0.0
    for _ in range(n_requests):
        t += rng.expovariate(rate)
        arrivals.append(t)
    sched = P.Sched(1, max_group * max_inflight) if costs is not None else None
    waiting, inflight, lat, done_t, sizes = [], [], [], [], []
    i, peak_mem = 0, 0
    t0 = time.monotonic()

    def queued():
        return sched.counts()[0] if sched else len(waiting)
    while len(lat) < n_requests:
        now = time.monotonic() - t0
        while i < n_requests and arrivals[i] <= now:
            if sched:
                sched.push(i, costs[i % len(pinned)])
            else:
                waiting.append(i)
            i += 1
        while queued() and len(inflight) < max_inflight:
            if sched:
                group = []
                while len(group) < max_group:
                    r = sched.request(0)
                    if r is None:
                        break
                    group.append(r)
            else:
                group = waiting[:max_group]
            tk = pipe.submit([pinned[r % len(pinned)] for r in group])
            if tk is None:
                if sched:                        # not admitted: back to the queue
                    for r in group:
                        sched.done(0, r)
                        sched.push(r, costs[r % len(pinned)])
                break
            inflight.append((tk, group))
            sizes.append(len(group))
            if not sched:
                waiting = waiting[len(group):]
        if time.monotonic() - t0 > limit_s:
            raise RuntimeError("served leg exceeded %.0f s" % limit_s)
        still = []
        for tk, reqs in inflight:
            res = pipe.poll(tk)
            if res is None:
                still.append((tk, reqs))
                continue
            for r, out in zip(reqs, res):
                if out["status"] != 0:
                    raise RuntimeError("served tile status %d" % out["status"])
                if check is not None:
                    check(r % len(pinned), out)
                if sched:
                    sched.done(0, r)
                done_ms = out["t_done_ms"] - t0 * 1000.0
                lat.append(done_ms - arrivals[r] * 1000.0)
                done_t.append(done_ms / 1000.0)
        inflight = still
        peak_mem = max(peak_mem, pipe.serve_memory()["allocated"])
        if not queued() and not inflight and i < n_requests:
            time.sleep(max(0.0, min(0.0005, arrivals[i] - (time.monotonic() - t0))))
    lat.sort()
    span = max(done_t) - arrivals[0]

    def pct(p):
        return lat[min(len(lat) - 1, int(math.ceil(p / 100.0 * len(lat))) - 1)]
    return {"value": n_requests / span, "unit": "tiles/s", "p50_ms": pct(50), "p99_ms": pct(99),
            "requests": n_requests, "arrival_rate": rate, "pool_tiles": len(pinned),
            "policy": "continuous batching: <= %d groups in flight, <= %d tiles per group, %s"
                      % (max_inflight, max_group, "most expensive first (Sched)" if sched else "arrival order"),
            "groups": len(sizes), "mean_group": sum(sizes) / max(1, len(sizes)),
            "peak_device_bytes": peak_mem, "hbm_budget_bytes": pipe.params.hbm_budget_bytes,
            "checked": check is not None}


def dispatch_compare(torch, pipe, n_requests, batched_rate):
    """The served form on a pool of 16 tiles of the served workload (sides
    2048-4096, 0-5000 nuclei per 4096^2), the same Poisson stream fed in
    arrival order and through the dispatcher's cost-sorted queue (the PATS
    order of Sec. IV-B reduced to tile cost; window of Sec. III-B).  The
    arrival rate is the batched 4096^2 rate scaled by the pool's mean area,
    so that requests queue up."""
    import paper_1209_3332_gb300 as P
    import synth
    host = [synth.cfg3(i) for i in range(16)]
    pool = [torch.from_numpy(h).pin_memory() for h in host]
    costs = [P.tile_cost(h) for h in host]
    mean_px = sum(h.shape[0] * h.shape[1] for h in host) / len(host)
    rate = batched_rate * 4096.0 * 4096.0 / mean_px
    serve_run(pipe, pool, 64, rate)                         # warm the contexts for these shapes
    fifo = serve_run(pipe, pool, n_requests, rate)
    lpt = serve_run(pipe, pool, n_requests, rate, costs=costs)
    return {"pool": "16 served-workload tiles (synth.cfg3), sides %d-%d"
                    % (min(h.shape[0] for h in host), max(h.shape[0] for h in host)),
            "arrival_rate": rate, "arrival_order": fifo, "most_expensive_first": lpt,
            "cost": "tile_cost: W*H*(1 + 8 * dark fraction on a 1-in-64 sample)"}


def feats_cap_of(W, H):
    """The served form's feature capacity of a W x H tile."""
    return max(1, min(W * H // 20 + 1, 65536))


def tile_buffers(torch, dev, host):
    """Device buffers of the batched / plain forms for host tiles of any sizes."""
    bufs = []
    for h in host:
        Ht, Wt = h.shape[:2]
        bufs.append(dict(rgb=torch.from_numpy(h).to(dev), hem8=torch.empty((Ht, Wt), dtype=torch.uint8, device=dev),
                         labels=torch.empty((Ht, Wt), dtype=torch.int32, device=dev),
                         edt=torch.empty((Ht, Wt), dtype=torch.int32, device=dev),
                         n_objects=torch.zeros(1, dtype=torch.int32, device=dev),
                         feats=torch.empty((feats_cap_of(Wt, Ht), 15), dtype=torch.float32, device=dev)))
    return bufs


def px4k(host):
    """Pixels of the tiles in 4096 x 4096 tile equivalents."""
    return sum(h.shape[0] * h.shape[1] for h in host) / float(H * W)


def batched_vs_plain(torch, pipe, stream, bufs, steps):
    """The batched form over all of `bufs` in one launch per pass, timed
    with CUDA events, and the plain form (seg_tile + features_tile per
    tile) on the same tiles; the plain outputs must equal the batched ones
    bit for bit (labels, K, feature rows).  Returns ms per step of each and
    the batched results (K and feature rows per tile, on the host)."""
    def batched():
        pipe.seg_features_batch(bufs, stream=stream)
    for _ in range(3):
        batched()                       # the first call tunes this batch shape
    stream.synchronize()
    ms_b = timed(torch, stream, batched, steps) / steps
    ref = [(int(b["n_objects"].item()), b["labels"].clone(), b["feats"].clone()) for b in bufs]

    def plain():
        for b in bufs:
            pipe.seg_tile(b["rgb"], b["hem8"], b["labels"], b["edt"], b["n_objects"], stream=stream)
            stream.synchronize()        # the plain feature call takes K from the host
            pipe.features_tile(b["hem8"], b["labels"], int(b["n_objects"].item()), b["feats"], stream=stream)
    plain()
    n_plain = max(1, steps // 2)
    ms_p = timed(torch, stream, plain, n_plain) / n_plain
    out = []
    for b, (K, lab, ft) in zip(bufs, ref):
        k2 = int(b["n_objects"].item())
        rows = min(K, ft.shape[0])
        if k2 != K or not torch.equal(lab, b["labels"]) or not torch.equal(ft[:rows], b["feats"][:rows]):
            raise RuntimeError("plain and batched forms differ on a tile")
        out.append((K, ft[:rows].cpu().numpy()))
    st = pipe.status()
    if st != 0:
        raise RuntimeError("device status %d" % st)
    return ms_b, ms_p, out


def make_check(ref):
    """check(pool index, served result): K and every feature row equal the
    batched form's on that pool tile, bit for bit."""
    import numpy as np

    def check(i, out):
        K, ft = ref[i]
        if out["n_objects"] != K or not np.array_equal(out["feats"], ft):
            raise RuntimeError("served result of pool tile %d differs from the batched form" % i)
    return check


def cfg2_run(torch, pipe, stream, steps):
    """The 64-tile mixed batch (sides 1024-4096, 0-5000 nuclei per 4096^2,
    tile 0 empty, tile 1 at 5000): the batched form in one launch per pass
    against the plain form on the same tiles."""
    import synth
    host = [synth.cfg2(i) for i in range(64)]
    bufs = tile_buffers(torch, torch.device("cuda", torch.cuda.current_device()), host)
    ms_b, ms_p, _ = batched_vs_plain(torch, pipe, stream, bufs, steps)
    eq = px4k(host)
    n = len(host)
    out = {"workload": "64 tiles, sides uniform in {1024,2048,3072,4096}, 0-5000 nuclei per 4096^2 "
                       "(synth.cfg2, seeds 2000+i)", "tiles_per_step": n, "4k_equivalents_per_step": eq,
           "batched": {"ms_per_step": ms_b, "tiles_per_s": n * 1000.0 / ms_b, "4k_equiv_per_s": eq * 1000.0 / ms_b},
           "plain": {"ms_per_step": ms_p, "tiles_per_s": n * 1000.0 / ms_p, "4k_equiv_per_s": eq * 1000.0 / ms_p},
           "parity": "plain == batched bit for bit on every tile in this run; oracle parity in "
                     "tests/test_gpu_configs.py"}
    out["batched_over_plain"] = ms_p / ms_b
    del bufs
    torch.cuda.empty_cache()
    return out


def cfg3_run(torch, pipe, stream, cfg2_rate, n_requests, steps):
    """Config 3: Poisson arrivals over the 64-tile served pool (sides
    2048-4096 in steps of 256, densities as config 2) at 80% of the config-2
    batched rate, through batch_submit / batch_poll under the pipe's 40 GiB
    HBM budget; every result is checked against the batched form on its
    pool tile."""
    import synth
    host = [synth.cfg3(i) for i in range(64)]
    dev = torch.device("cuda", torch.cuda.current_device())
    bufs = tile_buffers(torch, dev, host)
    ms_b, _, ref = batched_vs_plain(torch, pipe, stream, bufs, max(2, steps // 4))
    del bufs
    torch.cuda.empty_cache()
    pinned = [torch.from_numpy(h).pin_memory() for h in host]
    rate = 0.8 * cfg2_rate
    serve_run(pipe, pinned, 64, rate)                     # warm the contexts for these shapes
    r = serve_run(pipe, pinned, n_requests, rate, check=make_check(ref))
    pool_rate = len(host) * 1000.0 / ms_b
    r.update(workload="%d requests cycling 64 tiles of synth.cfg3 (sides 2048-4096, 0-5000 nuclei per 4096^2), "
                      "Poisson arrivals at 0.8 x the config-2 batched tiles/s" % n_requests,
             batched_pool_tiles_per_s=pool_rate, offered_load_vs_batched=rate / pool_rate,
             parity="every served result equals the batched form on its pool tile, bit for bit")
    return r


def stream_run(pipe, pinned, n_tiles, group=16, inflight=2, limit_s=300.0, check=None):
    """n_tiles requests cycling the pinned pool, submitted in groups of
    `group` with up to `inflight` groups on the device (a closed loop that
    keeps the device busy); returns tiles/s and group latencies."""
    t0 = time.monotonic()
    q, sent, done, lat = [], 0, 0, []
    while done < n_tiles:
        while len(q) < inflight and sent < n_tiles:
            idx = [(sent + k) % len(pinned) for k in range(min(group, n_tiles - sent))]
            tk = pipe.submit([pinned[i] for i in idx])
            if tk is None:
                break
            q.append((tk, idx, time.monotonic()))
            sent += len(idx)
        if not q:
            continue
        res = pipe.poll(q[0][0])
        if res is None:
            if time.monotonic() - t0 > limit_s:
                raise RuntimeError("stream not done within %.0f s" % limit_s)
            continue
        tk, idx, ts = q.pop(0)
        for i, out in zip(idx, res):
            if out["status"] != 0:
                raise RuntimeError("streamed tile status %d" % out["status"])
            if check is not None:
                check(i, out)
        lat.append(1000.0 * (time.monotonic() - ts))
        done += len(idx)
    el = time.monotonic() - t0
    lat.sort()
    return {"tiles": n_tiles, "seconds": el, "tiles_per_s": n_tiles / el, "group": group, "groups_in_flight": inflight,
            "group_latency_p50_ms": lat[len(lat) // 2], "group_latency_p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))]}


def cfg4_run(torch, pipe, stream, n_tiles, steps, link_gbs):
    """Config 4, the stress workload: worst-case 4096^2 tiles (8000 nuclei,
    half in chains, a serpentine ramp corridor) from a pool of 32, streamed
    from pinned host memory through batch_submit / batch_poll (batched +
    served), against the batched and plain forms on 16 tiles resident in
    HBM; every streamed result is checked against the batched form."""
    import synth
    host = [synth.cfg4(i) for i in range(32)]
    dev = torch.device("cuda", torch.cuda.current_device())
    ref, resident = [], None
    for half in (host[:16], host[16:]):
        bufs = tile_buffers(torch, dev, half)
        ms_b, ms_p, r = batched_vs_plain(torch, pipe, stream, bufs, max(2, steps // 4))
        ref.extend(r)
        if resident is None:
            resident = {"batched": {"tiles_per_s": 16 * 1000.0 / ms_b, "ms_per_step": ms_b},
                        "plain": {"tiles_per_s": 16 * 1000.0 / ms_p, "ms_per_step": ms_p}}
        del bufs
        torch.cuda.empty_cache()
    pinned = [torch.from_numpy(h).pin_memory() for h in host]
    stream_run(pipe, pinned, 64)                           # warm
    r = stream_run(pipe, pinned, n_tiles, check=make_check(ref))
    link_bound = link_gbs * 1e9 / (3.0 * H * W)
    return {"workload": "%d worst-case 4096x4096 tiles cycling a pool of 32 (synth.cfg4: 8000 nuclei, half in "
                        "chains of 10-30, serpentine ramp corridor)" % n_tiles,
            "streamed": r, "resident": resident,
            "streamed_over_plain": r["tiles_per_s"] / resident["plain"]["tiles_per_s"],
            "link_bound_tiles_per_s": link_bound, "streamed_frac_of_link": r["tiles_per_s"] / link_bound,
            "parity": "every streamed result equals the batched form on its pool tile, bit for bit"}


def run_ours(args, world, rank, local):
    import torch
    import paper_1209_3332_gb300 as P
    from paper_1209_3332_gb300 import build
    build.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(dev)
    pipe = P.Pipe(local)
    B = args.batch
    feats_cap = 20000
    host = gen_tiles(B, rank)
    bufs = device_buffers(torch, dev, host, feats_cap)
    torch.cuda.synchronize()

    def step_batched():
        pipe.seg_features_batch(bufs, stream=stream)

    def plain_tile(b):
        pipe.seg_tile(b["rgb"], b["hem8"], b["labels"], b["edt"], b["n_objects"], stream=stream)
        stream.synchronize()  # the plain feature call takes K from the host
        pipe.features_tile(b["hem8"], b["labels"], int(b["n_objects"].item()), b["feats"], stream=stream)

    def step_plain():
        for b in bufs:
            plain_tile(b)

    # ---- batched form: the timed region -----------------------------------
    for _ in range(args.warmup):
        step_batched()
    stream.synchronize()
    st = pipe.status()
    if st != P.PIPE_OK:
        raise RuntimeError("device status %d after warm-up" % st)
    clocks = Clocks(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    l0 = pipe.launch_count()
    ms_total = timed(torch, stream, step_batched, args.steps)
    barrier(world)
    launches = pipe.launch_count() - l0
    ck = clocks.stop()
    shapes = pipe.autotune_info()
    ms_total = max_over_ranks(world, ms_total)
    ms_step = ms_total / args.steps
    value = world * B * args.steps / (ms_total / 1000.0)
    st = pipe.status()
    if st != P.PIPE_OK:
        raise RuntimeError("device status %d" % st)
    line = {"metric": METRIC, "value": value, "unit": "tiles/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": WORKLOAD, "form": "batched (one launch per pass over the batch, CUDA graph)",
                       "tiles_per_step": B, "l2": "inputs larger than L2 (%d x 48 MiB RGB per step)" % B,
                       "parallelism": "replicas" if world > 1 else "1 GPU",
                       "launch_shapes": {"recon_workers": shapes["recon_workers"], "edt_rows": shapes["edt_rows"],
                                         "feat_blocks": shapes["feat_blocks"],
                                         "tuned_in_warmup_passes": shapes["tune_runs"]}},
            "gpu_launches": int(launches), "clocks": ck}
    if args.no_extra:
        if rank == 0:
            print(json.dumps(line), flush=True)
        pipe.close()
        return

    # ---- per-kernel times (events around every launch, same stream) ---------
    pipe.profile(True)
    for _ in range(args.steps):
        step_batched()
    torch.cuda.synchronize()
    prof = pipe.profile_read()
    pipe.profile(False)

    # ---- plain form on the same tiles ---------------------------------------
    step_plain()
    n_plain = max(1, args.steps // 2)
    ms_plain = timed(torch, stream, step_plain, n_plain)
    line["plain"] = {"value": world * B * n_plain / (max_over_ranks(world, ms_plain) / 1000.0), "unit": "tiles/s",
                     "form": "seg_tile + features_tile per tile (host reads K between them)"}
    plain_tile(bufs[0])
    line["plain"]["recon_tile_visits_per_work_tile"] = pipe.recon_visits() / float(
        ((W + 63) // 64) * ((H + 63) // 64))

    # ---- end to end through the served API with host buffers ----------------
    pinned = [torch.from_numpy(h).pin_memory() for h in host]
    h2d = B * H * W * 3

    def e2e_run(steps, inflight=2, limit_s=120.0):
        """`steps` steps through the served API with up to `inflight` in
        flight: every step uploads its B tiles from pinned host memory and
        reads back counts and feature rows, in order.  Returns the seconds
        taken and the D2H bytes of one step."""
        t0 = time.monotonic()
        q, n, done, d2h = [], 0, 0, 0
        while done < steps:
            while len(q) < inflight and n < steps:
                tk = pipe.submit(pinned)
                if tk is None:
                    break
                q.append(tk)
                n += 1
            res = pipe.poll(q[0]) if q else None
            if res is None:
                if time.monotonic() - t0 > limit_s:
                    raise RuntimeError("e2e steps not done within %.0f s" % limit_s)
                continue
            q.pop(0)
            done += 1
            d2h = sum(4 * 3 + r["n_objects"] * 15 * 4 for r in res)
        return time.monotonic() - t0, d2h
    e2e_run(2)
    lat_s, _ = e2e_run(1, inflight=1)
    barrier(world)
    e2e_s, d2h = e2e_run(args.steps)
    e2e_s = max_over_ranks(world, e2e_s)
    line["e2e"] = {"value": world * B * args.steps / e2e_s, "unit": "tiles/s", "h2d_bytes_per_step": h2d,
                   "d2h_bytes_per_step": d2h,
                   "path": "batch_submit (pinned host RGB) -> batch_poll (count + feature rows), "
                           "two steps in flight",
                   "single_step_latency_ms": 1000.0 * lat_s}

    # ---- served form: Poisson arrivals at 80% and 125% of the batched rate ---
    rate = 0.8 * value / world
    serve_run(pipe, pinned, min(32, 4 * B), rate)  # warm the contexts
    line["served"] = serve_run(pipe, pinned, args.requests, rate)
    line["served_saturated"] = serve_run(pipe, pinned, args.requests, 1.25 * value / world)
    line["served_saturated"]["offered_load_vs_batched"] = 1.25

    # ---- dispatch order on a mixed pool: arrival order vs most expensive first
    if not args.no_extra:
        line["dispatch"] = dispatch_compare(torch, pipe, args.requests, value / world)

    # ---- roofline of the dominant kernel ------------------------------------
    peak, peak_kind = peaks()
    name, (cnt, tot) = max(prof.items(), key=lambda kv: kv[1][1])
    stage = KERNEL_STAGE.get(name)
    if stage:
        avg_ms = tot / cnt
        alg = BYTES_PER_PX[stage] * B * H * W
        ach = alg / (avg_ms / 1000.0) / 1e9
        tr = kernel_traffic(name)
        line["roofline"] = {"bound": "hbm", "kernel": name, "achieved": ach, "peak": peak, "unit": "GB/s",
                            "frac": ach / peak, "traffic": tr * B if tr is not None else None,
                            "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)",
                            "alg_bytes_per_launch": alg, "avg_launch_ms": avg_ms}
    path_gbs = PATH_BYTES_PER_PX * H * W * value / world / 1e9
    line["path_roofline"] = {"bytes_per_tile": PATH_BYTES_PER_PX * H * W, "achieved": path_gbs, "peak": peak,
                             "unit": "GB/s", "frac": path_gbs / peak,
                             "bound_tiles_per_s": peak * 1e9 / (PATH_BYTES_PER_PX * H * W),
                             "io_bytes_per_tile": IO_BYTES_PER_PX * H * W,
                             "io_bound_tiles_per_s": peak * 1e9 / (IO_BYTES_PER_PX * H * W)}
    link = h2d_gbs(torch, dev)
    link_tiles = link * 1e9 / (3 * H * W)
    bound = min(link_tiles, line["path_roofline"]["bound_tiles_per_s"])
    line["link_roofline"] = {"h2d_gbs": link, "h2d_bytes_per_tile": 3 * H * W, "link_bound_tiles_per_s": link_tiles,
                             "e2e_bound_tiles_per_s": bound, "e2e_frac": line["e2e"]["value"] / world / bound}
    line["kernels_ms"] = {k: round(v[1] / max(v[0], 1), 4)
                          for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])}
    # ---- the step before the path: opening by the 19x19 disk ------------------
    line["morph_open"] = morph_open_run(torch, pipe, stream, [b["hem8"] for b in bufs], max(3, args.steps // 2),
                                        peak, rank == 0 and world == 1 and not args.no_cpu)
    # ---- the step after the path: watershed split of the objects -------------
    line["watershed"] = watershed_run(torch, pipe, stream, bufs, max(3, args.steps // 2), peak,
                                      rank == 0 and world == 1 and not args.no_cpu)
    # ---- the feature-stage edge transform: Canny and per-object edge counts --
    line["canny"] = canny_run(torch, pipe, stream, bufs, max(3, args.steps // 2), peak,
                              rank == 0 and world == 1 and not args.no_cpu)
    # ---- the first step of the segmentation stage: RBC detection -------------
    line["rbc"] = rbc_run(torch, pipe, stream, max(3, args.steps // 2), peak,
                          rank == 0 and world == 1 and not args.no_cpu)
    # ---- the other workloads: mixed batch, served pool, worst-case stream ----
    if world == 1 and not args.no_configs:
        line["cfg2"] = cfg2_run(torch, pipe, stream, max(3, args.steps // 2))
        line["cfg3"] = cfg3_run(torch, pipe, stream, line["cfg2"]["batched"]["tiles_per_s"], args.cfg3_requests,
                                args.steps)
        line["cfg4"] = cfg4_run(torch, pipe, stream, args.cfg4_tiles, args.steps, link)
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(host[0])
    if rank == 0:
        print(json.dumps(line), flush=True)
    pipe.close()


def relaunch(n):
    """Runs this command again under torch.distributed.run with n local
    ranks (rendezvous on 127.0.0.1); returns its exit code."""
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", str(n),
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__)] + sys.argv[1:]
    return subprocess.call(cmd)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=16, help="4096^2 tiles per batched step")
    ap.add_argument("--requests", type=int, default=400, help="requests in the served leg")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline leg")
    ap.add_argument("--no-extra", action="store_true", help="timed region only")
    ap.add_argument("--no-configs", action="store_true", help="skip the mixed-batch, served-pool and stress legs")
    ap.add_argument("--cfg3-requests", type=int, default=2000, help="requests of the served-pool leg")
    ap.add_argument("--cfg4-tiles", type=int, default=4096, help="tiles streamed in the stress leg")
    args = ap.parse_args()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        # one process per GPU: start the ranks here rather than run one replica
        sys.exit(relaunch(args.gpus))
    world, rank, local = dist_setup()
    if world != args.gpus:
        sys.exit("bench.py: --gpus %d but WORLD_SIZE is %d" % (args.gpus, world))
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
