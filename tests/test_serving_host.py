"""Host logic of the continuous serving loop (paper_1501_03358_gb300/serving.py)
on the CPU: slots that start queued requests while others are still
running, admission under the memory budget with the footprint of a first
solve counted before it runs, least-recently-used eviction of idle problems
with the recycle space spilled and restored, and per-problem arrival order.
The library calls are replaced by stand-ins that keep only byte counts and
whose solves finish when the test releases them; the GPU test of the same
loop (test_gpu_batch.py) checks the numbers."""
import threading
import time

import pytest

torch = pytest.importorskip("torch")

from paper_1501_03358_gb300 import serving

BASE, FULL = 10, 100
GATES = {}   # right-hand side -> threading.Event that its solve waits for
STARTED = {}  # right-hand side -> threading.Event set when its solve starts


class Blob:
    def __init__(self, owner, gen):
        self.owner, self.gen = owner, gen

    def cpu(self):
        return self

    def pin_memory(self):
        return self

    def cuda(self, non_blocking=False):
        return self


class FakeProblem:
    def __init__(self, ctx, grid, coef):
        self.name = grid
        self.bytes = BASE
        self.k = 0
        self.gen = 0
        self.imported = []
        self.solved = []
        self.lock = threading.Lock()

    def memory(self):
        return self.bytes

    def footprint(self, **kw):
        return max(self.bytes, FULL)

    def stats(self):
        return {"recycle_dim": self.k}

    def export_recycle(self):
        return Blob(self.name, self.gen)

    def import_recycle(self, blob):
        assert blob.owner == self.name
        self.imported.append(blob.gen)
        self.k, self.gen = 4, blob.gen
        self.bytes = FULL

    def release(self):
        self.bytes, self.k = BASE, 0

    def solve(self, b, stream=None, **kw):
        assert self.lock.acquire(blocking=False), "one problem solved in two slots at once"
        try:
            if b in STARTED:
                STARTED[b].set()
            if b in GATES:
                assert GATES[b].wait(10), b
            self.bytes = FULL
            self.k = 4
            self.gen += 1
            self.solved.append(b)
            return b, {"status": 0}
        finally:
            self.lock.release()

    def close(self):
        pass


@pytest.fixture
def make_server(monkeypatch):
    monkeypatch.setattr(serving, "Problem", FakeProblem)
    made = []

    def mk(budget, slots, names=("p0", "p1", "p2")):
        srv = serving.Server(ctx=None, budget_bytes=budget, solve_kw={}, slots=slots, device=None)
        for n in names:
            srv.add(n, n, None)
        made.append(srv)
        return srv

    yield mk
    for s in made:
        s.close()
    GATES.clear()
    STARTED.clear()


def gate(*bs):
    for b in bs:
        GATES[b] = threading.Event()
        STARTED[b] = threading.Event()


def test_requests_arriving_mid_solve_start_as_slots_free(make_server):
    srv = make_server(budget=10_000, slots=2)
    gate("p0-0", "p1-0", "p2-0")
    srv.submit("p0", "p0-0")
    srv.submit("p1", "p1-0")
    assert srv.poll() == 2 and STARTED["p0-0"].wait(5) and STARTED["p1-0"].wait(5)
    # p2's request arrives while both slots are busy: it waits
    srv.submit("p2", "p2-0")
    assert srv.poll() == 0 and srv.in_flight() == 2
    GATES["p1-0"].set()  # one slot frees; p0's solve is still running
    srv.wait_any(5)
    assert srv.poll() == 1 and STARTED["p2-0"].wait(5)
    assert srv.in_flight() == 2 and "p0" in srv.busy and "p2" in srv.busy
    GATES["p0-0"].set()
    GATES["p2-0"].set()
    srv.drain()
    assert [r.b for r in srv.done][0] == "p1-0"
    assert sorted(r.b for r in srv.done) == ["p0-0", "p1-0", "p2-0"]
    assert srv.max_in_flight == 2


def test_first_solve_footprint_counts_against_the_budget(make_server):
    # three problems of 10 bytes each; a solve needs 100. Budget 230: two
    # solves in flight reserve 200 + 10 idle = 210; the third first solve
    # would need 90 more and must wait although its problem has never run
    srv = make_server(budget=230, slots=3)
    gate("p0-0", "p1-0", "p2-0")
    for n in ("p0", "p1", "p2"):
        srv.submit(n, f"{n}-0")
    assert srv.poll() == 2
    assert srv.committed_bytes() <= 230
    assert [r.name for r in srv.queue] == ["p2"]
    GATES["p0-0"].set()
    srv.wait_any(5)
    # p0 is idle at 100 bytes: admitting p2 (90 more) needs p0 evicted
    assert srv.poll() == 1 and srv.evictions == 1 and "p0" in srv.released and "p0" in srv.spilled
    assert srv.committed_bytes() <= 230
    GATES["p1-0"].set()
    GATES["p2-0"].set()
    srv.drain()
    # p0's next request restores its space before it solves
    srv.submit("p0", "p0-1")
    srv.drain()
    assert srv.problems["p0"].imported == [1]
    assert srv.restores == 1
    assert srv.committed_bytes() <= 230


def test_requests_of_one_problem_stay_in_order(make_server):
    srv = make_server(budget=10_000, slots=3)
    for i in range(5):
        srv.submit("p1", f"p1-{i}")
    srv.submit("p0", "p0-0")
    srv.drain()
    assert srv.problems["p1"].solved == [f"p1-{i}" for i in range(5)]
    assert srv.problems["p0"].solved == ["p0-0"]
    assert len(srv.done) == 6


def test_request_larger_than_the_budget_raises(make_server):
    srv = make_server(budget=50, slots=2, names=("a",))
    srv.submit("a", "a-0")
    with pytest.raises(RuntimeError):
        srv.poll()  # its first solve needs 100 bytes > 50


def test_latency_is_completion_minus_arrival(make_server):
    srv = make_server(budget=10_000, slots=1, names=("a",))
    t0 = time.perf_counter()
    srv.submit("a", "a-0", arrival=t0 - 1.0)
    srv.drain()
    r = srv.done[0]
    assert r.finish - r.arrival >= 1.0 and r.start >= t0 - 1.0
