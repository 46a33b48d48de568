"""The continuous-batching scheduler (paper_1203_1692_gb300.serve.Server)
driven by a fake executor on the CPU: admission by memory budget in arrival
order, requests joining while others are mid-chain, every chain completed
with the right number of squarings."""
import pytest

from paper_1203_1692_gb300.serve import AdmissionError, Request, Server


class FakeExec:
    """Clock advances by a cost per squaring proportional to n^2."""

    def __init__(self, rate=1e9):
        self.t = 0.0
        self.rate = rate
        self.log = []          # (time, rids of the batch)
        self.resident = set()

    def now(self):
        return self.t

    def wait_until(self, t):
        self.t = max(self.t, t)

    def footprint(self, req):
        return 16 * req.n * req.n

    def start(self, req):
        assert req.rid not in self.resident
        self.resident.add(req.rid)

    def step(self, reqs):
        assert all(r.rid in self.resident for r in reqs)
        self.log.append((self.t, [r.rid for r in reqs]))
        self.t += sum(r.n * r.n for r in reqs) / self.rate
        return [2.0 * r.n ** 3 for r in reqs]

    def finish(self, req):
        self.resident.discard(req.rid)
        req.result = ("done", req.rid, req.done_steps)


def _trace(ns, gap):
    return [Request(rid=i, n=n, tau=1e-6, squarings=8, arrival=i * gap) for i, n in enumerate(ns)]


def test_all_chains_complete_with_eight_squarings():
    ex = FakeExec()
    srv = Server(ex, budget_bytes=10 ** 12)
    done = srv.run(_trace([1000, 2000, 500, 4000, 1500], gap=0.001))
    assert sorted(r.rid for r in done) == list(range(5))
    assert all(r.done_steps == 8 and r.result == ("done", r.rid, 8) for r in done)
    assert all(r.finished >= r.admitted >= r.arrival for r in done)
    assert not ex.resident


def test_budget_is_never_exceeded_and_admission_keeps_arrival_order():
    ns = [3000, 1000, 3000, 500, 2000, 3000, 700]
    ex = FakeExec()
    budget = 16 * 3000 * 3000 + 16 * 1000 * 1000     # room for one 3000 and one 1000
    srv = Server(ex, budget_bytes=budget)
    peak = []
    orig = srv._admit

    def admit():
        orig()
        peak.append(srv.used)
    srv._admit = admit
    done = srv.run(_trace(ns, gap=0.0))
    assert max(peak) <= budget and srv.peak_used <= budget
    admitted = sorted(done, key=lambda r: (r.admitted, r.rid))
    assert [r.rid for r in admitted] == sorted(r.rid for r in done)


def test_requests_join_while_others_are_mid_chain():
    ex = FakeExec(rate=1e8)
    srv = Server(ex, budget_bytes=10 ** 12)
    reqs = _trace([2000, 2000, 2000], gap=0.05)      # arrivals during the first chain
    srv.run(reqs)
    sizes = [len(b) for _, b in ex.log]
    assert max(sizes) >= 2                             # batches mixed requests
    first = next(t for t, b in ex.log if 1 in b)
    last0 = max(t for t, b in ex.log if 0 in b)
    assert first < last0                               # 1 joined before 0 finished


def test_slot_limit_and_oversized_request():
    ex = FakeExec()
    srv = Server(ex, budget_bytes=10 ** 12, max_active=2)
    srv.run(_trace([100] * 6, gap=0.0))
    assert max(len(b) for _, b in ex.log) == 2
    srv2 = Server(FakeExec(), budget_bytes=100)
    with pytest.raises(AdmissionError):
        srv2.submit(Request(rid=0, n=1000, tau=1e-6))


class FakeAsyncExec(FakeExec):
    """A batch runs on a simulated device while the server keeps admitting:
    launch returns the batch's completion time, ready compares the clock
    with it, idle advances the clock."""

    asynchronous = True

    def __init__(self, rate=1e9, scratch=0):
        super().__init__(rate)
        self.scratch = scratch
        self.admitted_during = []      # rids made resident while a batch ran
        self.busy_until = None

    def scratch_bytes(self):
        return self.scratch

    def start(self, req):
        super().start(req)
        if self.busy_until is not None:
            self.admitted_during.append(req.rid)

    def launch(self, reqs):
        self.log.append((self.t, [r.rid for r in reqs]))
        self.busy_until = self.t + sum(r.n * r.n for r in reqs) / self.rate
        return self.busy_until

    def ready(self, handle):
        return self.t >= handle

    def idle(self):
        self.t += 1e-4

    def collect(self, handle, reqs):
        self.busy_until = None
        return [2.0 * r.n ** 3 for r in reqs]


def test_async_batches_admit_arrivals_while_the_device_runs():
    """Requests arriving while a batch is on the device are admitted and
    made resident during it, join the next batch, and every chain still
    completes with its eight squarings."""
    ex = FakeAsyncExec(rate=1e8)
    srv = Server(ex, budget_bytes=10 ** 12)
    done = srv.run(_trace([4000, 1000, 500, 2000, 800], gap=0.01))
    assert sorted(r.rid for r in done) == list(range(5))
    assert all(r.done_steps == 8 for r in done)
    assert ex.admitted_during                     # admission overlapped a batch
    for t, rids in ex.log:                        # a request never runs twice in a batch
        assert len(rids) == len(set(rids))
    assert not ex.resident


def test_admission_counts_the_executor_scratch():
    """The executor's own scratch (its batch slots' triple pools) comes out of
    the budget before any request is admitted."""
    ns = [1000, 1000, 1000]
    scratch = 16 * 1000 * 1000
    budget = 2 * 16 * 1000 * 1000 + scratch        # room for two requests beside the scratch
    ex = FakeAsyncExec(rate=1e8, scratch=scratch)
    srv = Server(ex, budget_bytes=budget)
    done = srv.run([Request(rid=i, n=n, tau=1e-6, squarings=2, arrival=0.0)
                    for i, n in enumerate(ns)])
    assert len(done) == 3
    assert srv.peak_used + scratch <= budget
    assert max(len(r) for _, r in ex.log) == 2
