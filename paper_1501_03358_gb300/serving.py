"""Serving many resident problems (the serving-loop workload of the recycling
solver): requests (one new right-hand side of one problem each) queue in
arrival order; the server takes up to ``max_batch`` of them for distinct
problems, admits them under a device-memory budget, and solves them together
with rk_solve_batch. Each problem keeps its recycle space between requests
(the time-step sequence of Sec. 2.4 carried per problem). When the budget is
exceeded, least recently used idle problems are evicted: their recycle space
is copied to pinned host memory (rk_export_recycle, the stored double-float
columns) and their basis/workspace memory released (rk_problem_release); the
next request for such a problem restores the space bit-for-bit
(rk_import_recycle) before solving, so its sequence continues exactly as if
it had never been evicted.

The budget counts the library's own buffers (rk_problem_memory) plus, for a
problem about to be solved, the footprint it had after its last solve
(which is what it will reallocate). The paper has no counterpart to this
layer; it only orchestrates calls into librk."""
import collections
import time

import torch

from .solver import Problem, solve_batch


class Request:
    __slots__ = ("rid", "name", "b", "arrival", "start", "finish", "x", "info")

    def __init__(self, rid, name, b, arrival):
        self.rid, self.name, self.b, self.arrival = rid, name, b, arrival
        self.start = self.finish = None
        self.x = self.info = None


class Server:
    def __init__(self, ctx, budget_bytes: int, solve_kw: dict, max_batch: int = 16, nthreads: int = 0):
        self.ctx = ctx
        self.budget = int(budget_bytes)
        self.solve_kw = dict(solve_kw)
        self.max_batch = max_batch
        self.nthreads = nthreads
        self.problems = {}                      # name -> Problem
        self.footprint = {}                     # name -> bytes after its last solve
        self.spilled = {}                       # name -> recycle blob in pinned host memory
        self.released = set()                   # names whose workspace is freed
        self.lru = collections.OrderedDict()   # name -> None, least recent first
        self.queue = collections.deque()
        self.done = []
        self._next = 0
        self.evictions = 0
        self.restores = 0

    # -- problems and requests
    def add(self, name, grid, coef):
        if name in self.problems:
            raise ValueError(f"problem {name!r} exists")
        self.problems[name] = Problem(self.ctx, grid, coef)
        self.lru[name] = None

    def submit(self, name, b, arrival=None):
        if name not in self.problems:
            raise KeyError(name)
        r = Request(self._next, name, b, time.perf_counter() if arrival is None else arrival)
        self._next += 1
        self.queue.append(r)
        return r.rid

    def resident_bytes(self):
        return sum(p.memory() for p in self.problems.values())

    # -- memory management
    def _evict(self, name):
        p = self.problems[name]
        if p.stats()["recycle_dim"] > 0:
            self.spilled[name] = p.export_recycle().cpu().pin_memory()
        p.release()
        self.released.add(name)
        self.evictions += 1

    def _restore(self, name):
        self.released.discard(name)
        if name in self.spilled:
            self.problems[name].import_recycle(self.spilled.pop(name).cuda(non_blocking=True))
            self.restores += 1

    def _admit(self, names):
        """Evict LRU problems outside ``names`` until the batch fits."""
        need = sum(max(self.footprint.get(n, 0) - self.problems[n].memory(), 0) for n in names)
        for victim in list(self.lru):
            if self.resident_bytes() + need <= self.budget:
                break
            if victim in names or victim in self.released:
                continue
            self._evict(victim)
        return self.resident_bytes() + need <= self.budget

    # -- one round: a batch of queued requests for distinct problems
    def step(self):
        if not self.queue:
            return []
        picked, names, rest = [], set(), collections.deque()
        while self.queue and len(picked) < self.max_batch:
            r = self.queue.popleft()
            if r.name in names:
                rest.append(r)
            else:
                picked.append(r)
                names.add(r.name)
        # admission: shrink the batch until it fits the budget
        while picked and not self._admit(names):
            r = picked.pop()
            names.discard(r.name)
            rest.appendleft(r)
        self.queue.extendleft(reversed(rest))
        if not picked:
            raise RuntimeError("a single request does not fit the memory budget")
        for r in picked:
            self._restore(r.name)
            self.lru.move_to_end(r.name)
        t0 = time.perf_counter()
        for r in picked:
            r.start = t0
        xs, infos = solve_batch([self.problems[r.name] for r in picked], [r.b for r in picked],
                                nthreads=self.nthreads, **self.solve_kw)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for r, x, info in zip(picked, xs, infos):
            r.finish, r.x, r.info = t1, x, info
            self.footprint[r.name] = max(self.footprint.get(r.name, 0), self.problems[r.name].memory())
            self.done.append(r)
        return picked

    def drain(self):
        while self.queue:
            self.step()

    def close(self):
        for p in self.problems.values():
            p.close()
        self.problems.clear()
