"""The demand-driven dispatcher (host only, no GPU): the most expensive queued
tile first with ties in arrival order (the PATS sorted queue, Sec. IV-B),
the window of tiles a worker may hold (Sec. III-B), argument checks, many
threads at once, the tile cost estimate, and the Manager/Worker protocol
over gloo with three ranks."""
import os
import threading

import numpy as np
import pytest

import paper_1209_3332_gb300 as P
import synth


def test_most_expensive_first_ties_in_arrival_order():
    s = P.Sched(1, 100)
    costs = [5.0, 9.0, 1.0, 9.0, 0.0, 5.0, 7.5]
    for i, c in enumerate(costs):
        s.push(i, c)
    got = [s.request(0) for _ in costs]
    assert got == [1, 3, 6, 0, 5, 2, 4]
    assert s.request(0) is None
    assert s.counts() == (0, 7, 0)


def test_window_limits_the_tiles_a_worker_holds():
    s = P.Sched(2, 2)
    for i in range(6):
        s.push(i, float(i))
    assert [s.request(0), s.request(0)] == [5, 4]
    with pytest.raises(P.PipeError) as e:
        s.request(0)
    assert e.value.code == P.PIPE_EBUSY
    assert s.request(1) == 3                     # the other worker is not blocked
    s.done(0, 5)
    assert s.request(0) == 2
    assert s.counts() == (2, 3, 1)


def test_argument_checks():
    s = P.Sched(2, 1)
    s.push(7, 1.0)
    for bad in ((7, 2.0), (8, -1.0), (9, float("nan")), (10, float("inf"))):
        with pytest.raises(P.PipeError):
            s.push(*bad)
    with pytest.raises(P.PipeError):
        s.request(2)
    t = s.request(0)
    with pytest.raises(P.PipeError):
        s.done(1, t)                             # held by worker 0, not 1
    s.done(0, t)
    with pytest.raises(P.PipeError):
        s.done(0, t)                             # already done
    s.push(7, 3.0)                               # a finished id may be queued again
    with pytest.raises(P.PipeError):
        P.Sched(0, 1)
    with pytest.raises(P.PipeError):
        P.Sched(1, 0)


def test_many_threads_each_task_granted_once():
    n_workers, n_tasks = 8, 5000
    s = P.Sched(n_workers, 3)
    rng = np.random.default_rng(0)
    for i in range(n_tasks):
        s.push(i, float(rng.integers(0, 50)))
    seen = [[] for _ in range(n_workers)]

    def run(w):
        held = []
        while True:
            try:
                t = s.request(w)
            except P.PipeError:
                t = -1                            # window full: finish one first
            if t is None and not held:
                return
            if t is not None and t >= 0:
                held.append(t)
                seen[w].append(t)
            if t is None or t < 0 or len(held) >= 3:
                s.done(w, held.pop(0))
    th = [threading.Thread(target=run, args=(w,)) for w in range(n_workers)]
    for x in th:
        x.start()
    for x in th:
        x.join()
    allt = sorted(t for v in seen for t in v)
    assert allt == list(range(n_tasks))
    assert s.counts() == (0, 0, n_tasks)


def test_tile_cost_follows_area_and_density():
    empty = synth.tile(512, 256, 1, n_nuclei=0)
    assert P.tile_cost(empty) == 512 * 256
    sparse = synth.tile(512, 512, 2, n_nuclei=20)
    dense = synth.tile(512, 512, 2, n_nuclei=400)
    assert 512 * 512 < P.tile_cost(sparse) < P.tile_cost(dense) < 9 * 512 * 512
    assert P.tile_cost(synth.tile(1024, 1024, 2, n_nuclei=1600)) > 3 * P.tile_cost(dense)
    # a pitched view costs the same as its contiguous copy
    big = synth.tile(600, 300, 3, n_nuclei=50)
    assert P.tile_cost(big[:, :512]) == P.tile_cost(np.ascontiguousarray(big[:, :512]))


def _dispatch_rank(rank, world, port, tasks, costs, window, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1209_3332_gb300 import dispatch
    if rank == 0:
        out = ("log", dispatch.manager(tasks, costs, window))
    else:
        out = ("done", rank, dispatch.worker(lambda t: None, window))
    q.put(out)
    dist.barrier()
    dist.destroy_process_group()


def test_manager_worker_over_gloo_three_ranks():
    """Rank 0 manages, ranks 1 and 2 work with a window of 2: every tile is
    processed exactly once, tiles are granted most expensive first (all are
    queued before the first request), and no worker ever holds more than
    its window (the grant log is consistent with the done reports)."""
    import multiprocessing as mp
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    rng = np.random.default_rng(5)
    tasks = list(range(60))
    costs = [float(c) for c in rng.integers(0, 1000, len(tasks))]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_dispatch_rank, args=(r, 3, port, tasks, costs, 2, q)) for r in range(3)]
    for p in ps:
        p.start()
    res = [q.get(timeout=120) for _ in range(3)]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    log = next(r[1] for r in res if r[0] == "log")
    done = {r[1]: r[2] for r in res if r[0] == "done"}
    assert sorted(t for v in done.values() for t in v) == tasks
    granted = [t for _, t in log]
    assert [costs[t] for t in granted] == sorted(costs, reverse=True)
    for w, ts in done.items():
        assert [t for r, t in log if r == w] == ts   # each worker processes its tiles in grant order
