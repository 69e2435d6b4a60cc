"""Host logic of the benchmark's served leg, with a fake pipe (no GPU): in
arrival order and in the dispatcher's cost order, every request completes
exactly once, groups respect their size and the limit of groups in flight,
refused admissions are retried, and with a backlog the cost order takes the
most expensive pool tiles first."""
import random
import types
import time

import numpy as np

import bench


class FakePipe:
    """Admits up to two groups; a group 'runs' for a time proportional to its
    pixels; one submission in ten is refused."""

    def __init__(self, seed):
        self.params = types.SimpleNamespace(hbm_budget_bytes=2 << 20)  # room for the two groups
        self.rng = random.Random(seed)
        self.n = 0
        self.running = {}
        self.groups = []

    def submit(self, tiles):
        if len(self.running) >= 2 or self.rng.random() < 0.1:
            return None
        self.n += 1
        px = sum(t.shape[0] * t.shape[1] for t in tiles)
        self.running[self.n] = (time.monotonic() + px * 2e-12, len(tiles))
        self.groups.append([t.shape[0] for t in tiles])
        return self.n

    def poll(self, ticket):
        due, k = self.running[ticket]
        if time.monotonic() < due:
            return None
        del self.running[ticket]
        return [{"status": 0, "t_done_ms": time.monotonic() * 1000.0} for _ in range(k)]

    def serve_memory(self):
        # contexts of the groups in flight, 1 MB each
        return {"allocated": len(self.running) << 20, "in_flight": len(self.running) << 20,
                "contexts": len(self.running)}


def pool():
    sides = (256, 512, 128, 384)
    return [np.zeros((s, s, 3), np.uint8) for s in sides] * 3


def test_arrival_order_completes_every_request_once():
    p = FakePipe(1)
    r = bench.serve_run(p, pool(), 300, 20000.0, max_group=8)
    assert r["requests"] == 300 and r["groups"] == len(p.groups)
    assert sum(len(g) for g in p.groups) == 300
    assert max(len(g) for g in p.groups) <= 8
    assert "arrival order" in r["policy"] and r["p50_ms"] <= r["p99_ms"]


def test_cost_order_takes_the_most_expensive_first():
    tiles = pool()
    costs = [float(t.shape[0] * t.shape[1]) for t in tiles]
    p = FakePipe(2)
    r = bench.serve_run(p, tiles, 300, 1e9, max_group=8, costs=costs)   # all arrive at once: a backlog
    assert sum(len(g) for g in p.groups) == 300
    assert "most expensive first" in r["policy"]
    # every group is sorted by decreasing size, and the first groups hold the largest tiles
    assert all(g == sorted(g, reverse=True) for g in p.groups)
    assert p.groups[0][0] == 512 and p.groups[-1][-1] == 128
