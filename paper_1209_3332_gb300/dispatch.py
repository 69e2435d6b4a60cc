"""Manager/Worker tile dispatch across processes (Sec. III-B), over a
torch.distributed key-value store (``TCPStore``), with failure detection.

The Manager holds the cost-sorted queue (``Sched``, the native dispatcher of
libpipe) and answers requests.  A Worker asks for a tile whenever it holds
fewer than ``window`` (the paper's window of stage instances per Worker, so
that the next assignment and its input overlap the processing of the
current one), processes the oldest tile it holds, and reports it done.  The
Manager grants the most expensive queued tile (the PATS order of Sec. IV-B,
reduced to tile cost for GPU-only Workers).  Only tile ids travel; tile data
stays with the ranks.

Messages are store keys, which the Manager polls without blocking, so it can
keep a deadline: a Worker that holds tiles and has not been heard from for
``timeout_s`` is declared failed and its tiles go back to the queue for the
others (the paper's Manager re-serves work on demand).  A Worker is heard
from through its requests and reports, and, when it runs with
``heartbeat_s``, through a heartbeat key that a thread of its own advances
while a tile is being processed; without the heartbeat, ``timeout_s`` must
exceed the longest time one tile takes.  A failed Worker that
comes back is told there is no more work, and its late reports are
ignored.  When every live Worker has been told so and has reported every
tile it holds, the Manager sets the closed key, which also ends any Worker
still waiting.

The store must outlive every Worker (the process hosting a ``TCPStore``
server keeps it): a failed Worker that comes back after it has gone gets a
connection error instead of the closed key.

Keys (prefix ``dispatch/``): ``req/<w>/<i>`` is Worker w's i-th request;
``grant/<w>/<i>`` the answer (a tile id, or -1: no more work); ``done/<w>/<j>``
Worker w's j-th report (a tile id); ``alive/<w>`` Worker w's heartbeat
counter; ``closed`` the end, set on every exit of the Manager (also when it
raises), so that no Worker waits for it forever.
"""
import collections
import threading
import time

from . import Sched

_P = "dispatch/"


def _has(store, key):
    return store.check([key])


def manager(store, tasks, costs, n_workers, window, timeout_s=None, poll_s=0.0005, deadline_s=None):
    """Serve Workers 0..n_workers-1 through `store` until the work is done.
    Returns a dict: "grants" [(worker, task)] in grant order, "completed"
    [(worker, task)] in report order (exactly one entry per task), "failed"
    the Workers declared failed, "requeued" the tiles returned by them.

    A request that finds the queue empty while another live Worker holds
    tiles is left unanswered until it can be answered (those tiles may still
    come back); only then is a Worker told there is no more work.  With
    deadline_s, the whole run is bounded: past it the Manager closes and
    raises TimeoutError.  Whatever ends the loop (completion, the deadline,
    an error), the closed key is set and the queue is freed."""
    s = Sched(n_workers, window)
    try:
        return _serve(store, s, tasks, costs, n_workers, timeout_s, poll_s, deadline_s)
    finally:
        store.set(_P + "closed", "1")
        s.close()


def _serve(store, s, tasks, costs, n_workers, timeout_s, poll_s, deadline_s):
    for t, c in zip(tasks, costs):
        s.push(int(t), float(c))
    nreq = [0] * n_workers
    ndone = [0] * n_workers
    held = [set() for _ in range(n_workers)]
    told = [False] * n_workers
    failed, requeued = [], []
    grants, completed = [], []
    now = time.monotonic()
    seen = [now] * n_workers
    noticed = [-1] * n_workers     # the last request index counted as a sign of life
    beat = [None] * n_workers      # the last heartbeat value read
    end = None if deadline_s is None else now + deadline_s
    while True:
        if end is not None and time.monotonic() > end:
            raise TimeoutError("dispatch did not finish within %.1f s" % deadline_s)
        busy = False
        for w in range(n_workers):
            # a Worker writes each report before its next request, so once a
            # request is visible every older report is too: look for the
            # request, then drain the reports, then answer the request
            asked = not told[w] and _has(store, "%sreq/%d/%d" % (_P, w, nreq[w]))
            while True:
                k = "%sdone/%d/%d" % (_P, w, ndone[w])
                if not _has(store, k):
                    break
                busy = True
                seen[w] = time.monotonic()
                t = int(store.get(k))
                ndone[w] += 1
                if w not in failed and t in held[w]:
                    s.done(w, t)
                    held[w].discard(t)
                    completed.append((w, t))
            if not asked:
                continue
            if noticed[w] != nreq[w]:  # a deferred request is not a new sign of life
                noticed[w] = nreq[w]
                seen[w] = time.monotonic()
            t = None if w in failed else s.request(w)
            if t is None and w not in failed and any(held[v] for v in range(n_workers) if v != w):
                continue                                  # wait: tiles held elsewhere may come back
            busy = True
            store.set("%sgrant/%d/%d" % (_P, w, nreq[w]), str(-1 if t is None else t))
            nreq[w] += 1
            if t is None:
                told[w] = True
            else:
                held[w].add(t)
                grants.append((w, t))
        if timeout_s is not None:
            now = time.monotonic()
            for w in range(n_workers):
                if w not in failed and held[w] and now - seen[w] > timeout_s:
                    hb = "%salive/%d" % (_P, w)
                    if _has(store, hb):        # silent but beating: busy with a long tile
                        v = store.get(hb)
                        if v != beat[w]:
                            beat[w] = v
                            seen[w] = now
                            continue
                    failed.append(w)
                    requeued.extend(sorted(held[w]))
                    s.release(w)
                    held[w].clear()
        if all(told[w] or w in failed for w in range(n_workers)) and not any(held):
            break
        if not busy:
            time.sleep(poll_s)
    return {"grants": grants, "completed": completed, "failed": failed, "requeued": requeued}


class _Heartbeat:
    """Advances the key alive/<w> every period seconds from a thread of its
    own while the Worker runs."""

    def __init__(self, store, w, period):
        self.store, self.key, self.period = store, "%salive/%d" % (_P, w), period
        self.stop = threading.Event()
        self.th = threading.Thread(target=self._run, daemon=True)
        self.th.start()

    def _run(self):
        n = 0
        while not self.stop.is_set():
            n += 1
            try:
                self.store.set(self.key, str(n))
            except Exception:              # the store has gone: the run is over
                return
            self.stop.wait(self.period)

    def close(self):
        self.stop.set()
        self.th.join()


def worker(store, w, process, window, poll_s=0.0005, heartbeat_s=None):
    """Worker w: keeps one request outstanding while it holds fewer than
    `window` tiles, processes the tiles it holds meanwhile (oldest first),
    and reports each; ends when told there is no more work (or the Manager
    has closed) and nothing is left.  process(task id) does the work.
    With heartbeat_s, a thread advances the Worker's heartbeat key every
    heartbeat_s seconds, so that a tile longer than the Manager's timeout_s
    does not get a live Worker declared failed.  Returns the task ids
    processed, in order."""
    hb = _Heartbeat(store, w, heartbeat_s) if heartbeat_s else None
    try:
        return _work(store, w, process, window, poll_s)
    finally:
        if hb:
            hb.close()


def _work(store, w, process, window, poll_s):
    held = collections.deque()
    done = []
    nreq = ndone = 0
    more = True
    asking = False
    while True:
        if more and not asking and len(held) < window:
            store.set("%sreq/%d/%d" % (_P, w, nreq), "1")
            asking = True
        if asking:
            key = "%sgrant/%d/%d" % (_P, w, nreq)
            if _has(store, key):
                t = int(store.get(key))
                nreq += 1
                asking = False
                if t < 0:
                    more = False
                else:
                    held.append(t)
                continue
            if _has(store, _P + "closed"):
                more = asking = False
        if held:
            t = held.popleft()
            process(t)
            done.append(t)
            store.set("%sdone/%d/%d" % (_P, w, ndone), str(t))
            ndone += 1
            continue
        if not more and not asking:
            return done
        time.sleep(poll_s)
