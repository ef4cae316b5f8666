"""Host-side scheduling of the continuous-batching server, with the C ABI replaced by a
fake batch (no GPU): admission order, waiting at the memory cap, retirement."""
import numpy as np
import pytest

from paper_2308_11469_gb300 import binding, serve


class FakeBatch:
    """Each solve needs `cost[rid]` bytes and finishes after `steps[rid]` outer steps."""

    def __init__(self, cap, cost, steps):
        self.cap, self.cost, self.steps = cap, cost, steps
        self.live = {}
        self.next = 1
        self.log = []

    def submit(self, rid):
        used = sum(self.cost[r] for r, _ in self.live.values())
        if used + self.cost[rid] > self.cap:
            return None
        t = self.next
        self.next += 1
        self.live[t] = (rid, 0)
        self.log.append(("admit", rid))
        return t

    def step(self, k):
        for t, (rid, s) in list(self.live.items()):
            self.live[t] = (rid, s + k)

    def poll(self, t):
        rid, s = self.live[t]
        if s >= self.steps[rid]:
            del self.live[t]
            self.log.append(("done", rid))
            return (0, self.steps[rid], np.ones(self.steps[rid] + 1))
        return None

    def submit_many(self, jobs):
        out = []
        for job in jobs:
            t = self.submit(job[4])          # the job's f carries its request id here
            if t is None:
                break
            out.append(t)
        return out

    def peek(self, t):
        rid, s = self.live[t]
        return (1, 0, self.steps[rid]) if s >= self.steps[rid] else (0, 0, 0)


@pytest.fixture
def fake(monkeypatch):
    holder = {}

    def create(cap, stream=None):
        return holder["batch"]

    monkeypatch.setattr(binding, "helm_batch_create", create)
    monkeypatch.setattr(binding, "helm_batch_set_cycle", lambda b, *a: None)
    monkeypatch.setattr(binding, "helm_batch_submit_geom",
                        lambda b, D, n, h, k, prec, f, g, u, tol, mo: b.submit(f))
    monkeypatch.setattr(binding, "helm_batch_step", lambda b, k: b.step(k))
    monkeypatch.setattr(binding, "helm_batch_poll", lambda b, t, mo: b.poll(t))
    monkeypatch.setattr(binding, "helm_batch_submit_many", lambda b, jobs, prec, tol, mo: b.submit_many(jobs))
    monkeypatch.setattr(binding, "helm_batch_poll_many",
                        lambda b, ts, release=True: [b.peek(t) for t in ts])
    monkeypatch.setattr(binding, "helm_batch_info",
                        lambda b: (len(b.live), sum(b.cost[r] for r, _ in b.live.values())))
    monkeypatch.setattr(binding, "helm_batch_destroy", lambda b: None)
    return holder


def _jobs(n):
    # f carries the request id into the fake batch
    return [serve.Job(i, 2, 7, 0.125, 1.0, i, None, None, t_arrival=0.0) for i in range(n)]


def test_admission_waits_at_the_cap_and_keeps_arrival_order(fake):
    cost = {i: 10 for i in range(6)}
    steps = {0: 3, 1: 12, 2: 5, 3: 2, 4: 7, 5: 1}
    fake["batch"] = FakeBatch(cap=25, cost=cost, steps=steps)
    srv = serve.Server(25, chunk=2)
    done = srv.run(_jobs(6), realtime=False)
    log = fake["batch"].log
    admits = [r for ev, r in log if ev == "admit"]
    assert admits == list(range(6))                        # FIFO admission
    # never more than two solves resident (cap 25, 10 bytes each)
    live = 0
    for ev, r in log:
        live += 1 if ev == "admit" else -1
        assert live <= 2
    assert sorted(j.rid for j in done) == list(range(6))
    assert all(j.status == 0 and j.iters == steps[j.rid] for j in done)
    assert srv.max_in_use <= 25


def test_late_arrivals_join_while_others_run(fake):
    cost = {i: 1 for i in range(3)}
    steps = {0: 20, 1: 4, 2: 4}
    fake["batch"] = FakeBatch(cap=100, cost=cost, steps=steps)
    srv = serve.Server(100, chunk=4)
    jobs = _jobs(3)
    srv.submit(jobs[0])
    srv.admit()
    srv.step()                                             # job 0 mid-flight
    srv.submit(jobs[1])
    srv.submit(jobs[2])
    srv.admit()
    assert len(srv.active) == 3
    fin = srv.step()
    assert sorted(j.rid for j in fin) == [1, 2]            # the short late arrivals finish first
    while srv.active:
        srv.step()
    assert {j.rid for j in srv.done} == {0, 1, 2}


def test_latency_stats():
    js = [serve.Job(i, 2, 7, 0.1, 1.0, None, None, None, t_arrival=float(i)) for i in range(4)]
    for i, j in enumerate(js):
        j.t_done = j.t_arrival + 0.01 * (i + 1)
    st = serve.latency_stats(js)
    assert st["count"] == 4
    assert abs(st["p50_ms"] - 25.0) < 1e-9
    assert st["p99_ms"] <= 40.0 + 1e-9
