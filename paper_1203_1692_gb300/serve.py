"""Continuous-batching server for chains of SpAMM squarings.

A request is a matrix X0 and a threshold tau; the server computes the chain
X_{k+1} = SpAMM(X_k, X_k; tau) for a fixed number of squarings (the
McWeeny-style X <- X^2 of density-matrix purification, the paper's test
operation of Sec. IV).  Requests arrive over time.  Each scheduler
iteration

  1. admits waiting requests in arrival order while the device-memory
     budget has room for them (X, X^2 and the norm tree with its packs, as
     the library reports them) and a slot is free;
  2. runs ONE squaring of every active request as one batch: the norm trees
     of all of them are rebuilt with spamm_tree_rebuild_batched and the
     products run through spamm_multiply_batched (culls of all products in
     shared launches, leaf products of all products in one persistent
     tensor-core launch), so requests of different n and tau overlap on the
     device;
  3. retires the requests whose chain is complete and frees their memory.

With an executor that can launch a batch without waiting for it
(``launch``/``ready``/``collect``, as ``GpuChainExecutor`` does), the
squaring runs asynchronously: while it is on the device the server keeps
taking arrivals, admits them and makes them resident (their copies and
norm trees queue behind the batch), and it picks up the batch's results
once its completion event has fired.  Admission counts the executor's own
scratch (the triple pools of its batch slots) against the budget as well.

A request's norm tree, pack arrays and triple lists stay resident on the
device for its whole chain.  Every product of a batch gives the same C, bit
for bit, as the same product run alone, so a request's result does not
depend on what it was batched with.

The scheduler is host logic over an executor object; ``GpuChainExecutor``
is the one that drives the CUDA library.  Tests drive the scheduler with a
fake executor on the CPU.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field


@dataclass
class Request:
    rid: int
    n: int
    tau: float
    squarings: int = 8
    arrival: float = 0.0          # seconds on the server clock
    X0: object = None             # device matrix, copied at admission, or a
                                  # callable that makes it at admission
    # filled in by the server
    admitted: float | None = None
    finished: float | None = None
    result: object = None
    kept_flops: float = 0.0
    done_steps: int = 0
    state: object = field(default=None, repr=False)

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


class AdmissionError(RuntimeError):
    pass


class Server:
    """Continuous batching over an executor (see module docstring).

    ``executor`` provides ``footprint(req) -> bytes``, ``start(req)`` (make
    the request resident), ``step(reqs)`` (one squaring of each, returns the
    kept flops per request), ``finish(req)`` (release it, set req.result) and
    ``now()`` (the server clock, seconds)."""

    def __init__(self, executor, budget_bytes: int, max_active: int = 64):
        self.ex = executor
        self.budget = int(budget_bytes)
        self.max_active = max_active
        self.waiting: list[Request] = []
        self.active: list[Request] = []
        self.done: list[Request] = []
        self.used = 0
        self.iterations = 0
        self.peak_used = 0
        self.batch_sizes: list[int] = []
        self.joining: list[Request] = []   # admitted while a batch is on the device

    def submit(self, req: Request) -> None:
        if self.ex.footprint(req) > self.budget:
            raise AdmissionError(f"request {req.rid} (n={req.n}) exceeds the memory budget")
        self.waiting.append(req)

    def _scratch(self) -> int:
        f = getattr(self.ex, "scratch_bytes", None)
        return int(f()) if f else 0

    def _admit(self, into=None) -> None:
        active = self.active if into is None else into
        while self.waiting and len(self.active) + len(self.joining) < self.max_active:
            req = self.waiting[0]
            need = self.ex.footprint(req)
            if self.used + need + self._scratch() > self.budget:
                break                      # arrival order: no overtaking
            self.waiting.pop(0)
            self.used += need
            self.peak_used = max(self.peak_used, self.used)
            self.ex.start(req)
            req.admitted = self.ex.now()
            active.append(req)

    def _retire(self, batch, flops, t) -> None:
        still = []
        for req, f in zip(batch, flops):
            req.kept_flops += f
            req.done_steps += 1
            if req.done_steps >= req.squarings:
                req.finished = t
                self.ex.finish(req)
                self.used -= self.ex.footprint(req)
                self.done.append(req)
            else:
                still.append(req)
        self.active = still

    def step(self) -> bool:
        """One scheduler iteration; False when there was nothing to run."""
        self._admit()
        if not self.active:
            return False
        batch = list(self.active)
        flops = self.ex.step(batch)
        self.iterations += 1
        self.batch_sizes.append(len(batch))
        self._retire(batch, flops, self.ex.now())
        return True

    def step_async(self, pending, cursor: int) -> tuple[bool, int]:
        """One iteration with the batch on the device while arrivals are
        taken and admitted; returns (ran, new cursor into pending)."""
        self._admit()
        if not self.active:
            return False, cursor
        batch = list(self.active)
        handle = self.ex.launch(batch)
        self.iterations += 1
        self.batch_sizes.append(len(batch))
        self.joining = []
        while True:
            now = self.ex.now()
            while cursor < len(pending) and pending[cursor].arrival <= now:
                self.submit(pending[cursor])
                cursor += 1
            self._admit(into=self.joining)
            if self.ex.ready(handle):
                break
            self.ex.idle()
        flops = self.ex.collect(handle, batch)
        self._retire(batch, flops, self.ex.now())
        self.active += self.joining
        self.joining = []
        return True, cursor

    def run(self, requests, idle_wait=None) -> list[Request]:
        """Serve ``requests`` (sorted by arrival) in real time on the
        executor's clock: a request is submitted once the clock passes its
        arrival time; when nothing is active the server waits for the next
        arrival."""
        pending = sorted(requests, key=lambda r: (r.arrival, r.rid))
        asynchronous = getattr(self.ex, "asynchronous", False) and hasattr(self.ex, "launch")
        i = 0
        while i < len(pending) or self.waiting or self.active:
            now = self.ex.now()
            while i < len(pending) and pending[i].arrival <= now:
                self.submit(pending[i])
                i += 1
            if asynchronous:
                ran, i = self.step_async(pending, i)
            else:
                ran = self.step()
            if not ran:
                if i < len(pending):
                    (idle_wait or self.ex.wait_until)(pending[i].arrival)
        return self.done


class GpuChainExecutor:
    """Runs chains of squarings on the CUDA library: per request a copy X of
    X0, a buffer Y for X^2 and a norm tree (with its packs) on the device.

    With ``asynchronous`` (the default) a batch is launched unchecked and
    an event recorded behind it; ``ready`` polls the event and ``collect``
    reads the batch's statuses.  A batch whose triple pools overflowed is
    run again in checked mode (which grows the pools); its inputs are
    untouched until ``collect`` swaps X and X^2, so the rerun gives the same
    result.  ``step`` is the synchronous form (launch, wait, collect)."""

    def __init__(self, leaf: int = 16, precision: str = "tf32x3", keep_results: bool = True,
                 tier_bits: int = 0, slice: int = 0, asynchronous: bool = True):
        import torch
        from . import Context
        self.torch = torch
        self.ctx = Context(leaf=leaf, precision=precision, checked=not asynchronous,
                           tier_bits=tier_bits, slice=slice)
        self.asynchronous = asynchronous
        self.keep_results = keep_results
        self.t0 = time.perf_counter()
        self._foot = {}
        self._scratch = 0
        self.reruns = 0

    def now(self) -> float:
        return time.perf_counter() - self.t0

    def wait_until(self, t: float) -> None:
        while self.now() < t:
            time.sleep(min(1e-3, max(0.0, t - self.now())))

    def footprint(self, req: Request) -> int:
        if req.n not in self._foot:
            self._foot[req.n] = self.ctx.tree_footprint(req.n) + 2 * 4 * req.n * req.n
        return self._foot[req.n]

    def start(self, req: Request) -> None:
        torch = self.torch
        X = req.X0() if callable(req.X0) else req.X0.detach().clone()
        Y = torch.empty_like(X)
        tree = self.ctx.build_norms(X)
        req.state = {"X": X, "Y": Y, "tree": tree, "fresh": True}

    def _note_device_use(self) -> None:
        free, total = self.torch.cuda.mem_get_info()
        self.device_used_peak = max(getattr(self, "device_used_peak", 0), total - free)

    def scratch_bytes(self) -> int:
        """Device bytes of the triple pools of the batch slots (they only grow)."""
        return self._scratch

    def _run(self, reqs, checked: bool):
        trees = [r.state["tree"] for r in reqs]
        Ys = [r.state["Y"] for r in reqs]
        stale = [r for r in reqs if not r.state["fresh"]]
        if stale:
            self.ctx.rebuild_batched([r.state["tree"] for r in stale], [r.state["X"] for r in stale])
        self.ctx.set_checked(checked)
        self.ctx.multiply_batched(trees, trees, [r.tau for r in reqs], None, None, Ys)

    def launch(self, reqs):
        """Queue one squaring of every request; returns an event behind it."""
        self._run(reqs, checked=False)
        ev = self.torch.cuda.Event()
        ev.record(self.ctx.stream)
        return ev

    def ready(self, handle) -> bool:
        return handle.query()

    def idle(self) -> None:
        pass                                  # poll the event again at once

    def collect(self, handle, reqs):
        """Statuses of the finished batch (rerun checked if a pool
        overflowed), kept flops per request, X <- X^2."""
        handle.synchronize()
        st = self.ctx.stats(raise_on_error=False)
        if st["status"] != 0:
            self.reruns += 1
            for r in reqs:
                if not r.state["fresh"]:
                    r.state["fresh"] = True   # the trees already hold X's norms
            self._run(reqs, checked=True)     # raises on anything but overflow
            st = self.ctx.stats()
        self._scratch = max(self._scratch, int(st["pool_bytes"]))
        self._collected = getattr(self, "_collected", 0) + 1
        if self._collected % 8 == 1:
            self._note_device_use()
        flops = [f for f in self.ctx.per_product_flops(len(reqs))]
        for r in reqs:
            s = r.state
            s["X"], s["Y"] = s["Y"], s["X"]     # X <- X^2
            s["fresh"] = False
        return flops

    def step(self, reqs):
        if self.asynchronous:
            return self.collect(self.launch(reqs), reqs)
        self._run(reqs, checked=True)
        self._scratch = max(self._scratch, int(self.ctx.stats()["pool_bytes"]))
        flops = self.ctx.per_product_flops(len(reqs))
        for r in reqs:
            st = r.state
            st["X"], st["Y"] = st["Y"], st["X"]     # X <- X^2
            st["fresh"] = False
        return flops

    def finish(self, req: Request) -> None:
        st = req.state
        req.result = st["X"] if self.keep_results else None
        st["tree"].close()
        req.state = None

    def close(self):
        self.ctx.close()
