"""The demand-driven dispatcher (host only, no GPU): the most expensive queued
tile first with ties in arrival order (the PATS sorted queue, Sec. IV-B),
the window of tiles a worker may hold (Sec. III-B), release of a failed
worker's tiles, argument checks, many threads at once, the tile cost
estimate, and the Manager/Worker protocol across processes over a
TCPStore, with a stalled worker detected and its tiles served again."""
import os
import threading
import time

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


def test_the_manager_gives_up_at_its_deadline():
    """No Worker ever asks: with deadline_s the Manager closes and raises."""
    import socket
    import time
    from datetime import timedelta
    import torch.distributed as dist
    from paper_1209_3332_gb300 import dispatch
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    st = dist.TCPStore("127.0.0.1", port, 1, True, timeout=timedelta(seconds=10), wait_for_workers=False)
    t0 = time.monotonic()
    with pytest.raises(TimeoutError):
        dispatch.manager(st, [0, 1], [1.0, 2.0], 1, 1, deadline_s=0.2)
    assert time.monotonic() - t0 < 5 and st.check(["dispatch/closed"])


def test_release_returns_a_workers_tiles_to_the_queue():
    s = P.Sched(2, 3)
    for i, c in enumerate([1.0, 5.0, 3.0, 4.0]):
        s.push(i, c)
    assert [s.request(0), s.request(0), s.request(1)] == [1, 3, 2]
    assert s.release(0) == 2
    assert s.counts() == (3, 1, 0)
    with pytest.raises(P.PipeError):
        s.done(0, 1)                             # released: no longer held by worker 0
    assert [s.request(1), s.request(1)] == [1, 3]  # back in cost order
    assert s.release(0) == 0


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


def _dispatch_rank(role, port, tasks, costs, window, n_workers, stall, q, heartbeat_s=None):
    import time as _t
    from datetime import timedelta
    import torch.distributed as dist
    from paper_1209_3332_gb300 import dispatch
    store = dist.TCPStore("127.0.0.1", port, n_workers + 1, role == "manager", timeout=timedelta(seconds=60))
    if role == "manager":
        q.put(("manager", dispatch.manager(store, tasks, costs, n_workers, window,
                                           timeout_s=0.3 if stall is not None else None, deadline_s=60)))
        # this process hosts the store: it stays until every Worker has left
        store.wait(["test/bye/%d" % w for w in range(n_workers)], timedelta(seconds=60))
    else:
        first = [True]

        def process(t):
            if role == stall and first[0]:          # this worker hangs on its first tile
                first[0] = False
                _t.sleep(2.0)
        q.put(("worker", role, dispatch.worker(store, role, process, window, heartbeat_s=heartbeat_s)))
        store.set("test/bye/%d" % role, "1")


def _run_dispatch(tasks, costs, window, n_workers, stall=None, heartbeat_s=None):
    import multiprocessing as mp
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    roles = ["manager"] + list(range(n_workers))
    ps = [ctx.Process(target=_dispatch_rank, args=(r, port, tasks, costs, window, n_workers, stall, q, heartbeat_s))
          for r in roles]
    for p in ps:
        p.start()
    res = [q.get(timeout=120) for _ in roles]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    m = next(r[1] for r in res if r[0] == "manager")
    done = {r[1]: r[2] for r in res if r[0] == "worker"}
    return m, done


def test_manager_worker_three_processes():
    """A Manager and three Workers (separate processes sharing a TCPStore),
    window 2: every tile is completed exactly once, tiles are granted most
    expensive first (all are queued before the first request), and each
    Worker processes its tiles in grant order."""
    rng = np.random.default_rng(5)
    tasks = list(range(60))
    costs = [float(c) for c in rng.integers(0, 1000, len(tasks))]
    m, done = _run_dispatch(tasks, costs, 2, 3)
    assert sorted(t for _, t in m["completed"]) == tasks and not m["failed"]
    assert [costs[t] for _, t in m["grants"]] == sorted(costs, reverse=True)
    for w, ts in done.items():
        assert [t for r, t in m["grants"] if r == w] == ts


def test_a_stalled_worker_is_detected_and_its_tiles_served_again():
    """Worker 1 hangs for 2 s on its first tile while holding two (its
    window): after 0.3 s without a word the Manager declares it failed and
    returns both tiles to the queue; the other Workers complete every tile
    exactly once; the stalled Worker's late reports are ignored and it is
    told there is no more work (or finds the Manager closed)."""
    tasks = list(range(40))
    costs = [float(40 - t) for t in tasks]
    m, done = _run_dispatch(tasks, costs, 2, 3, stall=1)
    assert m["failed"] == [1]
    assert len(m["requeued"]) == 2
    assert sorted(t for _, t in m["completed"]) == tasks
    assert all(w != 1 for w, _ in m["completed"])
    assert set(m["requeued"]) <= set(t for w, t in m["completed"])
    assert set(m["requeued"]) <= set(done[1])           # it did process them, late


def test_a_worker_that_stops_for_good_is_detected():
    """In-process (threads over one TCPStore): Worker 1 takes its window of
    tiles and then never speaks again; the Manager declares it failed after
    the deadline and Worker 0 completes every tile."""
    import socket
    import threading
    import time
    from datetime import timedelta
    import torch.distributed as dist
    from paper_1209_3332_gb300 import dispatch
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    master = dist.TCPStore("127.0.0.1", port, 1, True, timeout=timedelta(seconds=30), wait_for_workers=False)
    res = {}

    def run1():  # Worker 1 by hand: two requests, each awaited, then silence
        st = dist.TCPStore("127.0.0.1", port, 1, False, timeout=timedelta(seconds=30))
        for i in range(2):
            st.set("dispatch/req/1/%d" % i, "1")
            st.wait(["dispatch/grant/1/%d" % i], timedelta(seconds=30))
        res[1] = True

    def run0():
        st = dist.TCPStore("127.0.0.1", port, 1, False, timeout=timedelta(seconds=30))
        time.sleep(0.05)                          # let Worker 1 take its tiles first
        res[0] = dispatch.worker(st, 0, lambda t: time.sleep(0.002), 2)
    ths = [threading.Thread(target=f, daemon=True) for f in (run1, run0)]
    for t in ths:
        t.start()
    m = dispatch.manager(master, list(range(30)), [float(30 - t) for t in range(30)], 2, 2, timeout_s=0.3,
                         deadline_s=60)
    for t in ths:
        t.join(30)
    assert res.get(1) and m["failed"] == [1] and len(m["requeued"]) == 2
    assert sorted(t for _, t in m["completed"]) == list(range(30))
    assert all(w == 0 for w, _ in m["completed"]) and sorted(res[0]) == list(range(30))


def test_a_slow_tile_under_a_heartbeat_is_not_a_failure():
    """Worker 1 takes 2 s on its first tile, far past the Manager's 0.3 s
    timeout, but its heartbeat thread keeps beating every 0.05 s: no Worker
    is declared failed, nothing is served twice, and every tile is completed
    exactly once."""
    tasks = list(range(30))
    costs = [float(30 - t) for t in tasks]
    m, done = _run_dispatch(tasks, costs, 2, 3, stall=1, heartbeat_s=0.05)
    assert m["failed"] == [] and m["requeued"] == []
    assert sorted(t for _, t in m["completed"]) == tasks
    assert sorted(sum(done.values(), [])) == tasks


def test_workers_return_when_the_manager_raises():
    """The Manager's queue refuses a request (the Worker runs with a larger
    window than the Manager's, so its second request finds its window full):
    the Manager raises, but sets the closed key first, so the Worker still
    returns."""
    import socket
    import threading
    from datetime import timedelta
    import torch.distributed as dist
    import paper_1209_3332_gb300 as P
    from paper_1209_3332_gb300 import dispatch
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    master = dist.TCPStore("127.0.0.1", port, 1, True, timeout=timedelta(seconds=30), wait_for_workers=False)
    res = {}

    def run0():
        st = dist.TCPStore("127.0.0.1", port, 1, False, timeout=timedelta(seconds=30))
        res[0] = dispatch.worker(st, 0, lambda t: time.sleep(0.05), 2)
    th = threading.Thread(target=run0, daemon=True)
    th.start()
    with pytest.raises(P.PipeError):
        dispatch.manager(master, list(range(10)), [1.0] * 10, 1, 1, deadline_s=30)
    assert master.check(["dispatch/closed"])
    th.join(30)
    assert not th.is_alive() and len(res[0]) >= 1
