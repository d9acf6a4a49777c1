"""Serving many resident problems with continuous admission (the serving-loop
workload of the recycling solver). A request is one new right-hand side of
one problem (the next time step of its sequence, Sec. 2.4). The server owns
``slots`` worker threads, each driving its own CUDA stream; whenever a slot
is free, the dispatcher starts the earliest queued request whose problem is
idle and whose memory fits the budget, while the other slots keep solving:
requests that arrive while others are on the GPU are admitted as slots and
memory free up, and their work overlaps on the device. A problem is in at
most one slot at a time, so its requests run in arrival order and its
recycle space carries from one to the next.

Memory: the budget counts the library's own buffers. An idle problem counts
its current bytes (rk_problem_memory); a problem in a slot counts the bytes
reserved for it at admission, the bound rk_problem_footprint gives for the
solve (its first solve included, before any buffer exists). When a request
does not fit, least recently used idle problems are evicted: their recycle
space is copied to pinned host memory (rk_export_recycle, exact) and their
basis/workspace released (rk_problem_release); the next request for such a
problem restores the space bit for bit (rk_import_recycle) before solving,
so its sequence continues exactly as if it had never been evicted.

The paper has no counterpart to this layer; it orchestrates calls into
librk from the host and computes nothing itself."""
import collections
import threading
import time

import torch

from .solver import Problem


class Request:
    __slots__ = ("rid", "name", "b", "arrival", "start", "finish", "x", "info", "ready", "slot")

    def __init__(self, rid, name, b, arrival, ready):
        self.rid, self.name, self.b, self.arrival, self.ready = rid, name, b, arrival, ready
        self.start = self.finish = None
        self.x = self.info = None
        self.slot = None


class _Slot:
    """One worker thread with its own CUDA stream; runs one solve at a time."""

    def __init__(self, server, index, device):
        self.server, self.index, self.device = server, index, device
        self.stream = torch.cuda.Stream(device=device) if device is not None else None
        self.job = None
        self.cv = threading.Condition()
        self.stop = False
        self.th = threading.Thread(target=self._run, name=f"rk-serve-slot{index}", daemon=True)
        self.th.start()

    def give(self, req):
        with self.cv:
            self.job = req
            self.cv.notify()

    def close(self):
        with self.cv:
            self.stop = True
            self.cv.notify()
        self.th.join(timeout=60)

    def _run(self):
        if self.device is not None:
            torch.cuda.set_device(self.device)
        while True:
            with self.cv:
                while self.job is None and not self.stop:
                    self.cv.wait()
                if self.stop and self.job is None:
                    return
                req = self.job
            srv = self.server
            err = None
            try:
                prob = srv.problems[req.name]
                if self.stream is not None:
                    if req.ready is not None:
                        self.stream.wait_event(req.ready)
                    with torch.cuda.stream(self.stream):
                        req.x, req.info = prob.solve(req.b, stream=self.stream, **srv.solve_kw)
                else:
                    req.x, req.info = prob.solve(req.b, **srv.solve_kw)
                mem = prob.memory()
            except Exception as e:  # reported to the dispatcher, which re-raises
                err, mem = e, None
            req.finish = time.perf_counter()
            with self.cv:
                self.job = None
            srv._finished(self, req, mem, err)


class Server:
    def __init__(self, ctx, budget_bytes: int, solve_kw: dict, slots: int = 4, device=None):
        self.ctx = ctx
        self.budget = int(budget_bytes)
        self.solve_kw = dict(solve_kw)
        if device is None and torch.cuda.is_available():
            device = torch.cuda.current_device()
        self.device = device
        self.problems = {}                      # name -> Problem
        self.bytes = {}                         # name -> device bytes when idle (its last solve's)
        self.reserved = {}                      # name -> bytes reserved while in a slot
        self.spilled = {}                       # name -> recycle blob in pinned host memory
        self.released = set()                   # names whose workspace is freed
        self.lru = collections.OrderedDict()   # name -> None, least recently used first
        self.queue = collections.deque()
        self.done = []
        self.busy = {}                          # name -> Request in a slot
        self._next = 0
        self.evictions = 0
        self.restores = 0
        self.max_in_flight = 0
        self.errors = []
        self._lock = threading.Lock()
        self._cv = threading.Condition(self._lock)
        self._slots = [_Slot(self, i, device) for i in range(max(1, int(slots)))]
        self._free = list(self._slots)

    # -- problems and requests
    def add(self, name, grid, coef):
        if name in self.problems:
            raise ValueError(f"problem {name!r} exists")
        p = Problem(self.ctx, grid, coef)
        self.problems[name] = p
        self.bytes[name] = p.memory()
        self.lru[name] = None

    def submit(self, name, b, arrival=None):
        if name not in self.problems:
            raise KeyError(name)
        ready = None
        if torch.cuda.is_available() and torch.is_tensor(b) and b.is_cuda:
            ready = torch.cuda.Event()
            ready.record()  # b is complete on the submitting stream
        with self._lock:
            r = Request(self._next, name, b, time.perf_counter() if arrival is None else arrival, ready)
            self._next += 1
            self.queue.append(r)
        return r.rid

    def in_flight(self):
        with self._lock:
            return len(self.busy)

    def committed_bytes(self):
        """Idle problems at their current bytes, problems in a slot at their
        reservation."""
        return sum(self.reserved[n] if n in self.busy else self.bytes[n] for n in self.problems)

    # -- memory management (dispatcher thread, lock held; idle problems only)
    def _evict(self, name):
        p = self.problems[name]
        if p.stats()["recycle_dim"] > 0:
            self.spilled[name] = p.export_recycle().cpu().pin_memory()
        p.release()
        self.released.add(name)
        self.bytes[name] = p.memory()
        self.evictions += 1

    def _restore(self, name):
        self.released.discard(name)
        if name in self.spilled:
            self.problems[name].import_recycle(self.spilled.pop(name).cuda(non_blocking=True))
            self.bytes[name] = self.problems[name].memory()
            self.restores += 1

    def _admit(self, name):
        """Reserve the request's footprint, evicting least recently used idle
        problems until it fits; False if it does not fit now."""
        need = self.problems[name].footprint(**self.solve_kw)
        # a released problem reallocates its recycle space on restore; the
        # footprint of a released problem already counts its whole basis
        extra = max(need - self.bytes[name], 0)
        if self.committed_bytes() + extra > self.budget:
            for victim in list(self.lru):
                if self.committed_bytes() + extra <= self.budget:
                    break
                if victim == name or victim in self.busy or victim in self.released:
                    continue
                self._evict(victim)
        if self.committed_bytes() + extra > self.budget:
            return False
        self.reserved[name] = max(need, self.bytes[name])
        return True

    # -- dispatch
    def poll(self):
        """Start queued requests on free slots (earliest first, one per idle
        problem, within the budget). Returns the number started. Raises if a
        request can never fit the budget."""
        started = 0
        with self._lock:
            if self.errors:
                raise self.errors[0]
            blocked = set()
            for r in list(self.queue):
                if not self._free:
                    break
                if r.name in self.busy or r.name in blocked:
                    blocked.add(r.name)  # keep the problem's requests in arrival order
                    continue
                if not self._admit(r.name):
                    if not self.busy:
                        raise RuntimeError(f"request for {r.name!r} does not fit the memory budget")
                    blocked.add(r.name)
                    continue
                self.queue.remove(r)
                self._restore(r.name)
                self.lru.move_to_end(r.name)
                slot = self._free.pop()
                r.start = time.perf_counter()
                r.slot = slot.index
                self.busy[r.name] = r
                self.max_in_flight = max(self.max_in_flight, len(self.busy))
                slot.give(r)
                started += 1
        return started

    def _finished(self, slot, req, mem, err):
        with self._cv:
            del self.busy[req.name]
            self.reserved.pop(req.name, None)
            if err is not None:
                self.errors.append(err)
            else:
                self.bytes[req.name] = mem
                self.done.append(req)
            self._free.append(slot)
            self._cv.notify_all()

    def wait_any(self, timeout=None):
        """Block until a slot finishes (or the timeout passes)."""
        with self._cv:
            if not self.busy:
                return
            n = len(self.done) + len(self.errors)
            self._cv.wait_for(lambda: len(self.done) + len(self.errors) > n, timeout=timeout)

    def drain(self):
        """Serve until the queue is empty and every slot is idle."""
        while True:
            self.poll()
            with self._lock:
                if not self.queue and not self.busy:
                    if self.errors:
                        raise self.errors[0]
                    return
            self.wait_any(timeout=1.0)

    def close(self):
        for s in self._slots:
            s.close()
        for p in self.problems.values():
            p.close()
        self.problems.clear()
