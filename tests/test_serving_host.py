"""Host logic of the serving loop (paper_1501_03358_gb300/serving.py) on the
CPU: batching of distinct problems in arrival order, admission under the
memory budget, least-recently-used eviction with the recycle space spilled
and restored. The library calls are replaced by stand-ins that only keep the
byte counts; the GPU test of the same loop (test_gpu_batch.py) checks the
numbers."""
import pytest

torch = pytest.importorskip("torch")

from paper_1501_03358_gb300 import serving

BASE, FULL = 10, 100


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

    def memory(self):
        return self.bytes

    def stats(self):
        return {"recycle_dim": self.k}

    def export_recycle(self):
        return Blob(self.name, self.gen)

    def import_recycle(self, blob):
        assert blob.owner == self.name
        self.imported.append(blob.gen)
        self.k, self.gen = 4, blob.gen

    def release(self):
        self.bytes, self.k = BASE, 0

    def close(self):
        pass


def fake_solve_batch(problems, bs, nthreads=0, **kw):
    xs, infos = [], []
    for p, b in zip(problems, bs):
        p.bytes = FULL
        p.k = 4
        p.gen += 1
        p.solved.append(b)
        xs.append(b)
        infos.append({"status": 0})
    return xs, infos


@pytest.fixture
def server(monkeypatch):
    monkeypatch.setattr(serving, "Problem", FakeProblem)
    monkeypatch.setattr(serving, "solve_batch", fake_solve_batch)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    srv = serving.Server(ctx=None, budget_bytes=250, solve_kw={}, max_batch=3)
    for n in ("p0", "p1", "p2"):
        srv.add(n, n, None)
    return srv


def test_batches_admission_and_lru_eviction(server):
    for rnd in range(2):
        for n in ("p0", "p1", "p2"):
            server.submit(n, f"{n}-{rnd}")
    # first batch: footprints unknown, all three admitted
    assert [r.name for r in server.step()] == ["p0", "p1", "p2"]
    # second: 3 x 100 bytes exceed 250; p2 waits, nothing outside the batch
    # can be evicted until it shrinks, then p2 (least recently used) goes
    assert [r.name for r in server.step()] == ["p0", "p1"]
    assert server.evictions == 1 and "p2" in server.released and "p2" in server.spilled
    # third: p2 needs 90 more bytes; p0 (now least recently used) is evicted,
    # p2's recycle space comes back from its spill before it solves
    assert [r.name for r in server.step()] == ["p2"]
    assert server.evictions == 2 and server.restores == 1
    assert server.problems["p2"].imported == [1]  # the space its first solve left
    assert not server.queue
    assert server.resident_bytes() <= 250


def test_requests_of_one_problem_stay_in_order(server):
    for i in range(4):
        server.submit("p1", f"p1-{i}")
    server.submit("p0", "p0-0")
    server.drain()
    assert server.problems["p1"].solved == [f"p1-{i}" for i in range(4)]
    assert server.problems["p0"].solved == ["p0-0"]
    assert len(server.done) == 5


def test_request_larger_than_the_budget_raises(monkeypatch):
    monkeypatch.setattr(serving, "Problem", FakeProblem)
    monkeypatch.setattr(serving, "solve_batch", fake_solve_batch)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    srv = serving.Server(ctx=None, budget_bytes=50, solve_kw={}, max_batch=2)
    srv.add("a", "a", None)
    srv.submit("a", "a-0")
    srv.step()  # first solve: footprint unknown, admitted
    srv.submit("a", "a-1")
    with pytest.raises(RuntimeError):
        srv.step()  # now known to need 100 bytes > 50
