"""Continuous-batching server for streams of Helmholtz solves (host scheduling only).

Requests of different dimension, grid size and k arrive over time; the server keeps the
solves resident on the device in one ``helm_batch`` (one engine per kernel class, its
plans, multigrid hierarchies and iterates in device memory), admits arrivals whenever
the batch's device-memory cap allows, advances every active solve together a few outer
steps at a time, and retires solves as they converge.  A solve admitted while others are
mid-flight shares their launches from the next chunk on; its arithmetic depends only on
its own data, so its result is the same alone and in the mix.

Latency of a request = completion time - arrival time, on the host clock.  All
arithmetic runs in the CUDA library through the C ABI (``binding``); this module only
orders admissions, steps and polls.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import binding as B


@dataclass
class Job:
    """One request: a problem (device tensors f, g, u) and its bookkeeping."""
    rid: int
    D: int
    n: int
    h: float
    k: float
    f: object
    g: object
    u: object
    t_arrival: float
    tol: float = 1e-8
    max_outer: int = 2000
    ticket: int | None = None
    t_admit: float | None = None
    t_done: float | None = None
    status: int | None = None
    iters: int | None = None
    hist: np.ndarray | None = field(default=None, repr=False)


class Server:
    """Admission queue + batch stepping + retirement.

    hbm_cap_bytes  cap on the workspace the batch may hold (HELM_ENOMEM beyond it:
                   the request waits in the queue until solves retire).
    chunk          outer steps per batch launch between admission / retirement checks.
    prec           inner precision of every solve (HELM_PREC_MIXED by default).
    schedule       (nu1, nu2, cycles) of every solve (None: the library's default V(2,2)).
    class_schedules  {ndim: (nu1, nu2, cycles)}: a schedule per dimension (2D and 3D solves
                   run in separate kernel classes, each with its own tuned cycle).
    """

    def __init__(self, hbm_cap_bytes: int, chunk: int = 4, prec: int = B.HELM_PREC_MIXED,
                 schedule=None, clock=time.perf_counter, class_schedules=None):
        self.batch = B.helm_batch_create(hbm_cap_bytes)
        if schedule is not None:
            B.helm_batch_set_cycle(self.batch, *schedule)
        for ndim, sch in (class_schedules or {}).items():
            B.helm_batch_set_cycle_class(self.batch, ndim, prec, *sch)
        self.chunk = chunk
        self.prec = prec
        self.clock = clock
        self.queue: deque[Job] = deque()
        self.active: dict[int, Job] = {}
        self.done: list[Job] = []
        self.max_in_use = 0

    def submit(self, job: Job) -> None:
        self.queue.append(job)

    def admit(self) -> int:
        """Admit queued jobs in arrival order while the memory cap allows (one library call
        per run of jobs sharing a tolerance and step budget)."""
        n = 0
        while self.queue:
            head = self.queue[0]
            run = []
            for job in self.queue:
                if job.tol != head.tol or job.max_outer != head.max_outer:
                    break
                run.append(job)
            ts = B.helm_batch_submit_many(self.batch, [(j.D, j.n, j.h, j.k, j.f, j.g, j.u) for j in run],
                                          self.prec, head.tol, head.max_outer)
            now = self.clock()
            for job, t in zip(run, ts):
                job.ticket = t
                job.t_admit = now
                self.active[t] = job
                self.queue.popleft()
            n += len(ts)
            if len(ts) < len(run):
                break                       # over the cap: wait for retirements
        a, used = B.helm_batch_info(self.batch)
        self.max_in_use = max(self.max_in_use, used)
        return n

    def step(self) -> list[Job]:
        """Advance every active solve by up to `chunk` outer steps; return the finished."""
        if not self.active:
            return []
        B.helm_batch_step(self.batch, self.chunk)
        now = self.clock()
        fin = []
        tickets = list(self.active)
        for t, (done, _, _) in zip(tickets, B.helm_batch_poll_many(self.batch, tickets, release=False)):
            if not done:
                continue
            job = self.active.pop(t)
            job.status, job.iters, job.hist = B.helm_batch_poll(self.batch, t, job.max_outer)
            job.t_done = now
            fin.append(job)
        self.done.extend(fin)
        return fin

    def run(self, jobs: list[Job], realtime: bool = True) -> list[Job]:
        """Serve `jobs` (sorted by arrival time, seconds from the start) to completion."""
        pending = deque(sorted(jobs, key=lambda j: j.t_arrival))
        t0 = self.clock()
        if realtime:
            for j in pending:
                j.t_arrival += t0
        while pending or self.queue or self.active:
            now = self.clock()
            while pending and (not realtime or pending[0].t_arrival <= now):
                job = pending.popleft()
                if not realtime:
                    job.t_arrival = now
                self.submit(job)
            self.admit()
            if self.active:
                self.step()
            elif pending and realtime:
                time.sleep(max(0.0, min(pending[0].t_arrival - self.clock(), 0.001)))
        return self.done

    def close(self) -> None:
        B.helm_batch_destroy(self.batch)


def solve_host_batch(batch, plans, f_host, g_host, u_host, tol: float, max_outer: int):
    """Solve problems whose data live in host memory through the library's host entry
    point (``helm_batch_submit_host``: the library uploads f and g, solves from zero and
    copies each result into u_host[i] as soon as that solve ends).

    plans[i], f_host[i], g_host[i] (complex128 CPU tensors, page-locked for asynchronous
    copies) describe problem i; u_host[i] receives its padded solution.  The solves are
    submitted in decreasing order of the closed-form spectral radius rho (the most outer
    steps first): the library uploads in submission order on its own stream and starts each
    solve once its data are on the device, so the longest solve runs while the others
    upload.  Returns [(status, iters, relres history)] in input order.
    """
    m = len(plans)
    order = sorted(range(m), key=lambda i: -B.helm_plan_info(plans[i])[2])
    tickets = {}
    for i in order:
        t = B.helm_batch_submit_host(batch, plans[i], f_host[i], g_host[i], u_host[i], tol, max_outer)
        if t is None:
            raise RuntimeError("solve_host_batch: the batch's memory cap does not admit every solve")
        tickets[i] = t
    B.helm_batch_step(batch, 0)
    out = [None] * m
    for i, t in tickets.items():
        out[i] = B.helm_batch_poll(batch, t, max_outer)
    return out


def latency_stats(jobs: list[Job]) -> dict:
    lat = np.array([j.t_done - j.t_arrival for j in jobs if j.t_done is not None])
    if lat.size == 0:
        return {"count": 0}
    span = max(j.t_done for j in jobs) - min(j.t_arrival for j in jobs)
    return {"count": int(lat.size), "p50_ms": float(1e3 * np.percentile(lat, 50)),
            "p99_ms": float(1e3 * np.percentile(lat, 99)), "mean_ms": float(1e3 * lat.mean()),
            "solves_per_s": float(lat.size / span) if span > 0 else None}


def _pool_key(req):
    p = req.problem
    return (p.D, p.n, p.meta["kind"])


def make_jobs(reqs, dev, pool=None, tol: float = 1e-8, max_outer: int = 2000):
    """Jobs of a request stream drawn with ``materialise=False``.  Device data: one
    materialised source / wall-data pair per (D, n, kind), built from the first request
    of that key and shared by the later ones (each request keeps its own k and its own
    solution buffer).  Returns (jobs, pool); `pool` maps the key to (f, g, problem)."""
    import torch

    from . import inputs
    pool = {} if pool is None else pool
    jobs = []
    for i, r in enumerate(reqs):
        key = _pool_key(r)
        if key not in pool:
            p = inputs.materialise(r.problem)
            pool[key] = (torch.from_numpy(p.f).to(dev), torch.from_numpy(p.g).to(dev), p)
        f, g, _ = pool[key]
        p = r.problem
        jobs.append(Job(i, p.D, p.n, p.h, p.k, f, g, torch.zeros_like(g), r.t_arrival, tol, max_outer))
    return jobs, pool


def main(argv=None) -> int:
    """Serve a seeded stream of mixed 2D / 3D requests and print latency / throughput."""
    import argparse
    import json

    import torch

    from . import build, inputs

    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--rate", type=float, default=100.0, help="mean arrivals per second")
    ap.add_argument("--count", type=int, default=200)
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--cap-gb", type=float, default=120.0)
    ap.add_argument("--chunk", type=int, default=4)
    ap.add_argument("--sizes-2d", default="127,255,511,1023,2047")
    ap.add_argument("--sizes-3d", default="63,127,255")
    ap.add_argument("--sched-2d", default="0,1,1", help="nu1,nu2,cycles of the 2D solves")
    ap.add_argument("--sched-3d", default="0,2,1", help="nu1,nu2,cycles of the 3D solves")
    args = ap.parse_args(argv)
    build.build()
    B.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    reqs = inputs.served_stream(args.rate, args.count, seed=args.seed,
                                sizes_2d=tuple(int(x) for x in args.sizes_2d.split(",")),
                                sizes_3d=tuple(int(x) for x in args.sizes_3d.split(",")),
                                materialise=False)
    jobs, _ = make_jobs(reqs, dev)
    torch.cuda.synchronize()
    scheds = {2: tuple(int(x) for x in args.sched_2d.split(",")),
              3: tuple(int(x) for x in args.sched_3d.split(","))}
    srv = Server(int(args.cap_gb * (1 << 30)), chunk=args.chunk, class_schedules=scheds)
    done = srv.run(jobs, realtime=True)
    stats = latency_stats(done)
    stats.update({"rate": args.rate, "requests": args.count, "chunk": args.chunk,
                  "converged": sum(j.status == B.HELM_CONVERGED for j in done),
                  "max_workspace_gb": srv.max_in_use / (1 << 30)})
    srv.close()
    print(json.dumps(stats))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
