"""Manager/Worker tile dispatch across processes (Sec. III-B), over
torch.distributed point-to-point messages.

Rank 0 is the Manager: it holds the cost-sorted queue (``Sched``, the native
dispatcher of libpipe) and answers requests.  Every other rank is a Worker:
it asks for a tile whenever it holds fewer than ``window`` (the paper's
window of stage instances per Worker, so that the next assignment and its
input overlap the processing of the current one), processes the oldest tile
it holds, and reports it done.  The Manager grants the most expensive queued
tile (the PATS order of Sec. IV-B, reduced to tile cost for GPU-only
Workers).  Messages between a pair of ranks arrive in order, so a Worker's
report of a finished tile always reaches the Manager before its next
request.  The messages carry only tile ids; tile data stays with the ranks.
"""
import collections

import torch
import torch.distributed as dist

from . import Sched

_REQUEST, _DONE = 0, 1


def manager(tasks, costs, window, world_size=None):
    """Serve the Workers (ranks 1..world_size-1) until every Worker has been
    told there is no more work and has reported every tile it held.  Returns
    the grant log: (worker rank, task id) in grant order."""
    world = world_size or dist.get_world_size()
    s = Sched(world - 1, window)
    for t, c in zip(tasks, costs):
        s.push(int(t), float(c))
    msg = torch.zeros(2, dtype=torch.int64)
    active = set(range(1, world))
    log = []
    while active or s.counts()[1] > 0:
        src = dist.recv(msg)
        op, task = int(msg[0]), int(msg[1])
        if op == _DONE:
            s.done(src - 1, task)
            continue
        t = s.request(src - 1)
        dist.send(torch.tensor([-1 if t is None else t], dtype=torch.int64), src)
        if t is None:
            active.discard(src)
        else:
            log.append((src, t))
    s.close()
    return log


def worker(process, window):
    """Request, process and report tiles until the Manager has none left;
    process(task id) does the work.  Returns the task ids processed, in
    order."""
    held = collections.deque()
    done = []
    more = True
    reply = torch.zeros(1, dtype=torch.int64)
    while True:
        while more and len(held) < window:
            dist.send(torch.tensor([_REQUEST, 0], dtype=torch.int64), 0)
            dist.recv(reply, 0)
            t = int(reply[0])
            if t < 0:
                more = False
            else:
                held.append(t)
        if not held:
            return done
        t = held.popleft()
        process(t)
        done.append(t)
        dist.send(torch.tensor([_DONE, t], dtype=torch.int64), 0)
