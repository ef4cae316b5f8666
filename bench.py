"""Benchmark: solves/s of the FP Poisson iteration on the 1023x1023 Gaussian cavity.

Workload (one "step"): the four solves k in {1, 2, 3, 4} of the 1023x1023 unit-square
Dirichlet cavity (h = 1/1024, g = 0, f = 8 seeded Gaussians of width 0.02) to
relres 1e-8.

* headline (``value``): mixed precision -- complex64 multigrid V-cycles, complex128
  residual and solution (iterative refinement) -- the four solves advanced together as
  one batch in two concurrent lanes: the k = 4 solve alone on the highest-priority
  stream (the latency form of its step), the three shorter ones in the other lane (each
  of its launches covers their active instances); each solve retires when it converges,
  and each lane's run is one CUDA-graph launch.
* ``fp64_single``: the plain FP64 form, each solve alone (complex128 everywhere).
* ``e2e``: the headline measured through the C ABI's host entry point
  (``helm_batch_submit_host`` via ``serve.solve_host_batch``): pinned host -> device
  copies of f and g by the library, the solves,
  device -> host copy of u, every step; the uploads of the shorter solves overlap the
  first outer steps of the longest one, which starts as soon as its own data are on the
  device.
* ``roofline``: the kernel with the largest device-time share, from a replay of one
  step with every launch bracketed by CUDA events on the launching stream.
* ``cpu_baseline``: the CPU oracle (exact sine-basis Poisson solves, all host cores).
  The same leg states every result's error against the oracle's exact discrete solution
  (``accuracy`` and each leg's ``accuracy``).

Other configurations, as bounded legs of the same run (each with its own clock sample;
``--legs`` picks them, ``--legs none`` skips them):

* ``cavity63``: the 63x63 plane-wave cavity (h = 1/64, theta = pi/6), k = 2 to relres
  1e-10 and k = 5 > k_max (must diverge), mixed and FP64 single solves: microseconds per
  solve, status against the closed-form prediction, O(h^2) error against the continuum
  plane wave.
* ``cube255``: the 255^3 plane-wave + sine cube, k = 4, relres 1e-8, mixed and FP64
  single solves (autotuned schedules): solves/s.
* ``batch512``: 512 uneven 2D cavities (n in {63..511}), mixed batch to completion, and
  the plain FP64 form solving its first 64 alone: solves/s beside the byte-model
  ceiling.
* ``served``: Poisson arrivals of mixed 2D (127^2..2047^2) / 3D (63^3..255^3) requests
  at several rates through the continuous-batching server (HBM cap 120 GB): request
  latency p50 / p99 (completion - arrival) and solves/s per rate.

Under torchrun each rank solves its own copy of the workload (weak scaling, no
collective on the data path).  ``--impl reference`` times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

KS = (1.0, 2.0, 3.0, 4.0)
# concurrent engines of the 4-solve batch: the k = 4 solve (75 of the 129 outer steps) in
# one lane, the three shorter ones together in the other; measured 6.42 against 6.53 (3
# lanes) and 6.63 ms (4, the library's default) per step of four solves
LANES = 2
N_GRID = 1023
TOL = 1e-8
MAX_OUTER = 2000
METRIC = "solves/s & stencil HBM GB/s (%peak) at relres 1e-8, mixed vs FP64; p50/p99"
WORKLOAD = "gaussian_cavity_2d_1023_k1234"
FP64_PEAK_TFLOPS = 1.25          # GB300 nominal FP64 rate (FMA = 2 flops)
# DRAM bytes (read + write) per point of the residual kernels, from one ncu capture each,
# scaled below to the points of an average launch; None where the kernel changed after its
# capture (the bench's top kernel is the fused one)
RESIDUAL_DRAM_BYTES_PER_POINT = None
# the finest level's ascent fused with the residual (fixed-point numerator, loops flattened
# over the CTA's threads): one ncu capture of the paired replay's launch (two instances,
# 73.21 MB read + 17.23 MB written)
UPRES_DRAM_BYTES_PER_POINT = (73.205760e6 + 17.231104e6) / (2 * 1023 ** 2)
# the same kernel forming level 1's ascent too (the latency lane's form, level 1's words
# as their own copy group): one capture of the single-solve replay's launch (44.66 MB read
# + 1.07 MB written)
UPRES_L1_DRAM_BYTES_PER_POINT = (44.662016e6 + 1.065728e6) / (1023 ** 2)


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _dist():
    from paper_2308_11469_gb300 import dist as wsd
    return wsd.world()


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 50 ms while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        t0 = time.time()                      # sampling is live before the timed region
        while not self.lines and time.time() - t0 < 5.0 and self.proc.poll() is None:
            time.sleep(0.01)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def cpu_oracle_workload(problems, max_seconds: float = 60.0):
    """The oracle on the bench workload: exact sine-basis inner solves on every host
    core; also the exact discrete solutions used to state each result's error."""
    from oracle import fd, iteration as it
    workers = os.cpu_count() or 1
    t0 = time.perf_counter()
    iters = []
    times = []
    for p in problems:
        t = time.perf_counter()
        r = it.paper_iteration(p.f, p.g, p.h, p.k, tol=TOL, max_outer=MAX_OUTER, poisson="dst",
                               workers=workers)
        times.append(time.perf_counter() - t)
        iters.append(r.iters)
        if time.perf_counter() - t0 > max_seconds:
            break
    exact = [fd.solve_exact_dst(p.f, p.g, p.h, p.k, workers=workers) for p in problems]
    return times, iters, exact, workers


def run_reference(args):
    """CPU oracle arm: each timed step is the whole workload (the four solves k = 1..4 to
    relres 1e-8, exact sine-basis inner solves on every host core); each warm-up step is
    the cheapest solve (k = 1) alone, so the run stays within a few minutes.
    solves/s = 4 x steps / the timed steps' total time."""
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    from oracle import iteration as it
    from paper_2308_11469_gb300 import inputs
    problems = [inputs.gaussian_cavity_2d(k) for k in KS]
    workers = os.cpu_count() or 1
    for w in range(args.warmup):
        p = problems[0]
        it.paper_iteration(p.f, p.g, p.h, p.k, tol=TOL, max_outer=MAX_OUTER, poisson="dst",
                           workers=workers)
    times = []
    for s in range(args.steps):
        t = time.perf_counter()
        for p in problems:
            it.paper_iteration(p.f, p.g, p.h, p.k, tol=TOL, max_outer=MAX_OUTER, poisson="dst",
                               workers=workers)
        times.append(time.perf_counter() - t)
    t_work = float(np.sum(times))
    value = len(KS) * args.steps / t_work
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t_work / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": N_GRID, "k": list(KS), "tol": TOL,
                   "solves_per_step": len(KS)},
        "latency_ms": {"p50": float(1e3 * np.percentile(times, 50)),
                       "p99": float(1e3 * np.percentile(times, 99)), "per": "step of 4 solves"},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": workers, "kind": "oracle",
                         "sample": f"{args.steps} steps of the four solves k = {list(KS)} (exact "
                                   f"sine-basis inner solves); warm-up steps solve k = 1 alone"},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# bounded legs for the other configurations (GPU side; their errors against the
# oracle are formed in the cpu_baseline leg, errors_vs_oracle below)
# ---------------------------------------------------------------------------

def _ev_ms(torch, fn):
    s = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    s.record()
    out = fn()
    e.record()
    e.synchronize()
    return s.elapsed_time(e), out


def bytes_per_point_step(nu1: int, nu2: int, cycles: int, eb: int) -> float:
    """Algorithmic bytes per fine point of one outer step: the FP64 residual + update
    (u, f in, u out: 48 B; e in, r out: 2 inner elements) and per V(nu1, nu2) cycle, on
    every level (x 4/3 for the 2D hierarchy), 3 inner elements per sweep and 2 + 1/4 for
    each of the restriction and the prolongation (mixed V(2,2): 240 B)."""
    return 48 + 2 * eb + cycles * 4.0 / 3.0 * (3 * eb * (nu1 + nu2) + 2 * (2 * eb + eb / 4))


def leg_cavity63(B, torch, dev):
    from paper_2308_11469_gb300 import inputs
    rows, keep = [], {}
    for k, tol in ((2.0, 1e-10), (5.0, 1e-10)):
        p = inputs.plane_wave_cavity_2d(k)
        f = torch.from_numpy(p.f).to(dev)
        g = torch.from_numpy(p.g).to(dev)
        u = torch.zeros_like(g)
        for prec, name in ((B.HELM_PREC_MIXED, "mixed"), (B.HELM_PREC_FP64, "fp64")):
            plan = B.helm_plan_create(2, p.n, p.h, k, prec=prec)
            rho = B.helm_plan_info(plan)[2]

            def run():
                u.zero_()
                return B.helm_solve(plan, f, g, u, tol, 400)
            for _ in range(3):
                run()
            ts = []
            for _ in range(10):
                t, (st, it, hist) = _ev_ms(torch, run)
                ts.append(t)
            B.helm_plan_destroy(plan)
            status = B.helm_status_str(st)
            row = {"k": k, "form": name, "tol": tol, "status": status, "iters": it,
                   "relres_last": float(hist[-1]), "us_per_solve_median": 1e3 * float(np.median(ts)),
                   "rho_closed_form": rho,
                   "predicted": "converges" if rho < 1 else "diverges",
                   "status_matches_prediction": (status == "HELM_CONVERGED") == (rho < 1)}
            if k == 2.0:
                uh = u.cpu().numpy()
                keep[("cavity63", name)] = (p, uh)
                cont = inputs.plane_wave(2, p.n, p.h, k, p.meta["direction"])
                row["max_err_vs_continuum_plane_wave"] = float(np.max(np.abs(uh - cont)))
            rows.append(row)
    return {"rows": rows}, keep


def leg_cube255(B, torch, dev, flush):
    from paper_2308_11469_gb300 import inputs
    p = inputs.plane_wave_sine_cube(4.0, seed=3, n=255)
    f = torch.from_numpy(p.f).to(dev)
    g = torch.from_numpy(p.g).to(dev)
    u = torch.zeros_like(g)
    out, keep = {"n": p.n, "k": p.k, "tol": TOL}, {}
    npts = float(p.n) ** 3
    for prec, name in ((B.HELM_PREC_MIXED, "mixed"), (B.HELM_PREC_FP64, "fp64")):
        plan = B.helm_plan_create(3, p.n, p.h, p.k, prec=prec)
        u.zero_()                             # the tuning solves start from the zero iterate
        sched = B.helm_plan_autotune(plan, f, g, u, TOL, MAX_OUTER)

        def run():
            u.zero_()
            return B.helm_solve(plan, f, g, u, TOL, MAX_OUTER)
        run()
        ts = []
        for _ in range(3):
            flush.fill_(1)
            t, (st, it, hist) = _ev_ms(torch, run)
            ts.append(t)
        B.helm_plan_destroy(plan)
        ms = float(np.mean(ts))
        eb = 8 if prec == B.HELM_PREC_MIXED else 16
        # 3D: the hierarchy adds 1/7 instead of 1/3
        bpp = 48 + 2 * eb + sched[2] * 8.0 / 7.0 * (3 * eb * (sched[0] + sched[1]) + 2 * (2 * eb + eb / 8))
        out[name] = {"solves_per_s": 1e3 / ms, "ms_per_solve": ms, "ms_best": float(min(ts)),
                     "status": B.helm_status_str(st), "iters": it, "relres_last": float(hist[-1]),
                     "schedule": {"nu1": sched[0], "nu2": sched[1], "cycles": sched[2]},
                     "model_bytes_per_solve": bpp * npts * it,
                     "model_GBs": bpp * npts * it / (ms / 1e3) / 1e9}
        keep[("cube255", name)] = (p, u.cpu().numpy())
    out["mixed_over_fp64"] = out["mixed"]["solves_per_s"] / out["fp64"]["solves_per_s"]
    return out, keep


def leg_batch512(B, torch, dev, peak_gbs):
    from paper_2308_11469_gb300 import inputs
    probs = inputs.batched_instances(count=512, seed=4)
    F = [torch.from_numpy(q.f).to(dev) for q in probs]
    G = [torch.from_numpy(q.g).to(dev) for q in probs]
    # the solutions as views of one buffer: one fill clears every starting iterate
    Uall = torch.zeros(sum(x.numel() for x in G), dtype=torch.complex128, device=dev)
    U, off = [], 0
    for x in G:
        U.append(Uall[off:off + x.numel()].view(x.shape))
        off += x.numel()
    big = max(range(len(probs)), key=lambda i: (probs[i].n, probs[i].k))
    q = probs[big]
    scheds, tiles = {}, {}
    for prec in (B.HELM_PREC_MIXED, B.HELM_PREC_FP64):
        pl = B.helm_plan_create(2, q.n, q.h, q.k, prec=prec)
        U[big].zero_()
        scheds[prec] = B.helm_plan_autotune(pl, F[big], G[big], U[big], TOL, 3000)[:3]
        tiles[prec] = B.helm_plan_tiles(pl)
        B.helm_plan_destroy(pl)
    batch = B.helm_batch_create(120 << 30)
    B.helm_batch_set_cycle(batch, *scheds[B.HELM_PREC_MIXED])
    B.helm_batch_set_tiles(batch, tiles[B.HELM_PREC_MIXED])

    jobs = [(2, q.n, q.h, q.k, F[i], G[i], U[i]) for i, q in enumerate(probs)]

    def run_batch():
        Uall.zero_()
        ts = B.helm_batch_submit_many(batch, jobs, B.HELM_PREC_MIXED, TOL, 3000)
        assert len(ts) == len(jobs)
        B.helm_batch_step(batch, 0)
        return [(st, it) for _, st, it in B.helm_batch_poll_many(batch, ts)]
    run_batch()
    ts = []
    for _ in range(3):
        t, res = _ev_ms(torch, run_batch)
        ts.append(t)
    B.helm_batch_destroy(batch)
    ms = float(np.mean(ts))
    its = [r[1] for r in res]
    pts_steps = float(sum(q.n ** 2 * r[1] for q, r in zip(probs, res)))
    nu1, nu2, cyc = scheds[B.HELM_PREC_MIXED]
    b_run = bytes_per_point_step(nu1, nu2, cyc, 8) * pts_steps
    b_v22 = bytes_per_point_step(2, 2, 1, 8) * pts_steps
    out = {"instances": len(probs), "ms_per_batch": ms, "solves_per_s": 512e3 / ms,
           "converged": int(sum(r[0] == B.HELM_CONVERGED for r in res)),
           "iters_mean": float(np.mean(its)), "iters_max": int(max(its)),
           "schedule": dict(zip(("nu1", "nu2", "cycles"), scheds[B.HELM_PREC_MIXED])),
           "tiles": ("auto", "large", "small")[tiles[B.HELM_PREC_MIXED]],
           "model_bytes_per_batch": b_run, "model_GBs": b_run / (ms / 1e3) / 1e9,
           "ceiling_solves_per_s_at_peak": 512 / (b_run / (peak_gbs * 1e9)),
           "ceiling_solves_per_s_v22_model": 512 / (b_v22 / (peak_gbs * 1e9))}
    keep = {("batch512", "mixed", i): (probs[i], U[i].cpu().numpy()) for i in range(len(probs))}
    tot, cnt = 0.0, 64
    its64 = []
    for i in range(cnt):
        q = probs[i]
        pl = B.helm_plan_create(2, q.n, q.h, q.k, prec=B.HELM_PREC_FP64)
        B.helm_plan_set_cycle(pl, *scheds[B.HELM_PREC_FP64])
        B.helm_plan_set_tiles(pl, tiles[B.HELM_PREC_FP64])

        def one():
            U[i].zero_()
            return B.helm_solve(pl, F[i], G[i], U[i], TOL, 3000)
        one()
        t, r = _ev_ms(torch, one)
        its64.append(r[1])
        tot += t
        B.helm_plan_destroy(pl)
        keep[("batch512", "fp64", i)] = (q, U[i].cpu().numpy())
    out["fp64_single_first64"] = {"solves_per_s": cnt * 1e3 / tot, "iters_mean": float(np.mean(its64)),
                                  "schedule": dict(zip(("nu1", "nu2", "cycles"), scheds[B.HELM_PREC_FP64]))}
    mixed64 = float(sum(its[:cnt]))
    out["note"] = ("fp64_single_first64: each of the first 64 instances alone, device time summed; "
                   f"their mixed outer steps {mixed64:.0f}, fp64 {float(sum(its64)):.0f}")
    return out, keep


SERVED_RATES = (10.0, 100.0, 300.0, 1000.0, 2000.0)


def served_count(rate: float) -> int:
    """Requests per rate: about two seconds of arrivals, at least 30 and at most 400."""
    return int(min(400, max(30, round(2.0 * rate))))


def leg_served(B, torch, dev, schedules, rates=SERVED_RATES, seed: int = 5):
    """schedules: {ndim: (nu1, nu2, cycles)}, the tuned schedule of each dimension's solves."""
    from paper_2308_11469_gb300 import inputs, serve
    pool = {}
    # warm-up: one request of every (dimension, size) class, all at once (engines, plans
    # and graphs of every class are built outside the measured streams)
    warm = []
    rng = np.random.default_rng(seed + 1000)
    for D, sizes in ((2, (127, 255, 511, 1023, 2047)), (3, (63, 127, 255))):
        for n in sizes:
            h = 1.0 / (n + 1)
            k = 0.5 * inputs.dirichlet_kmax(D, n, h)
            c, a = inputs.draw_gaussian_params(D, rng)
            warm.append(inputs.Request(0.0, inputs.Problem(D, n, h, k, None, None,
                                                           {"kind": "gauss", "centres": c, "amps": a})))
    jobs, pool = serve.make_jobs(warm, dev, pool)
    srv = serve.Server(120 << 30, chunk=4, class_schedules=schedules)
    srv.run(jobs, realtime=False)
    srv.close()
    del jobs
    rows, keep = [], {}
    for rate in rates:
        count = served_count(rate)
        reqs = inputs.served_stream(rate, count, seed=seed, materialise=False)
        jobs, pool = serve.make_jobs(reqs, dev, pool, tol=TOL, max_outer=MAX_OUTER)
        torch.cuda.synchronize()
        srv = serve.Server(120 << 30, chunk=4, class_schedules=schedules)
        done = srv.run(jobs, realtime=True)
        st = serve.latency_stats(done)
        pts_steps = float(sum((j.n ** j.D) * j.iters for j in done))
        st.update({"rate_req_per_s": rate, "requests": count,
                   "converged": int(sum(j.status == B.HELM_CONVERGED for j in done)),
                   "max_workspace_gb": srv.max_in_use / (1 << 30),
                   "outer_steps_mean": float(np.mean([j.iters for j in done])),
                   "point_steps": pts_steps})
        srv.close()
        rows.append(st)
        # a seeded sample of three results per rate, kept for the error check
        pick = np.random.default_rng(int(rate)).choice(len(done), size=min(3, len(done)), replace=False)
        for i in pick:
            j = done[int(i)]
            key = (j.D, j.n, reqs[j.rid].problem.meta["kind"])
            keep[("served", rate, j.rid)] = (pool[key][2], j.k, j.u.cpu().numpy())
        del jobs, done
        torch.cuda.synchronize()
    return {"rates": rows, "hbm_cap_gb": 120, "chunk": 4,
            "schedules": {f"{d}D": dict(zip(("nu1", "nu2", "cycles"), v)) for d, v in schedules.items()},
            "mix": "2D n in {127..2047} (70 %) / 3D n in {63, 127, 255}; Gaussian sources or "
                   "plane-wave wall data (50/50); k ~ U[0.5, 0.9 k_max]; source / wall data "
                   "materialised once per (D, n, kind), each request its own k and solution"}, keep


def errors_vs_oracle(keep, workers: int, budget_s: float = 60.0):
    """Relative L2 error of each kept result against the oracle's exact discrete
    solution (sine-basis direct solve), within a CPU-time budget; the served sample is
    checked last, smallest grids first."""
    from oracle import fd
    t0 = time.perf_counter()
    errs = {}

    def exact_for(p, k):
        return fd.solve_exact_dst(p.f, p.g, p.h, k, workers=workers)

    order = sorted(keep, key=lambda key: (key[0] == "served",
                                          keep[key][0].n ** keep[key][0].D if key[0] == "served" else 0))
    skipped = 0
    for key in order:
        if key[0] == "served":
            p, k, u = keep[key]
        else:
            p, u = keep[key]
            k = p.k
        if key[0] == "served" and time.perf_counter() - t0 > budget_s:
            skipped += 1
            continue
        ex = exact_for(p, k)
        errs[key] = float(np.linalg.norm(u - ex) / np.linalg.norm(ex))
    return errs, skipped, time.perf_counter() - t0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--legs", default="cavity63,cube255,batch512,served",
                    help="other configurations run after the headline ('none' to skip)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        dist = None
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_2308_11469_gb300 import binding as B
    from paper_2308_11469_gb300 import build as _build
    from paper_2308_11469_gb300 import inputs
    _build.build()
    B.load()

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    from paper_2308_11469_gb300 import dist as wsd

    def max_over_ranks(x: float) -> float:
        return wsd.max_over_ranks(x, dist, dev)

    def job_throughput(units: float, ms: float) -> float:
        # units summed over the ranks / the slowest rank's time
        return wsd.throughput(units, ms / 1e3, dist, dev)

    problems = [inputs.gaussian_cavity_2d(k) for k in KS]
    n = N_GRID
    h = problems[0].h
    F = [torch.from_numpy(p.f).to(dev) for p in problems]
    G = [torch.from_numpy(p.g).to(dev) for p in problems]
    U = [torch.zeros_like(g) for g in G]
    mixed_plans = [B.helm_plan_create(2, n, h, k, prec=B.HELM_PREC_MIXED) for k in KS]
    fp64_plans = [B.helm_plan_create(2, n, h, k, prec=B.HELM_PREC_FP64) for k in KS]
    batch = B.helm_batch_create(120 << 30)
    B.helm_batch_set_lanes(batch, LANES)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2

    # autotuned inner schedule (smoother sweeps, cycles per outer step), chosen on the
    # costliest solve of the step (k = 4) and used by every solve of each form
    U[-1].zero_()
    sched_mixed = B.helm_plan_autotune(mixed_plans[-1], F[-1], G[-1], U[-1], TOL, MAX_OUTER)
    tiles_mixed = B.helm_plan_tiles(mixed_plans[-1])
    B.helm_batch_set_cycle(batch, *sched_mixed[:3])
    B.helm_batch_set_tiles(batch, tiles_mixed)
    sched_fp64 = None
    if not args.no_fp64:
        sched_fp64 = B.helm_plan_autotune(fp64_plans[-1], F[-1], G[-1], U[-1], TOL, MAX_OUTER)
        tiles_fp64 = B.helm_plan_tiles(fp64_plans[-1])
        for pl in fp64_plans:
            B.helm_plan_set_cycle(pl, *sched_fp64[:3])
            B.helm_plan_set_tiles(pl, tiles_fp64)

    def mixed_step(Fs=F, Gs=G, Us=U):
        for u in Us:
            u.zero_()
        # longest predicted solve first (rho grows with k): the batch spreads its lanes
        # longest-job-first
        tickets = [None] * len(KS)
        for i in sorted(range(len(KS)), key=lambda j: -KS[j]):
            tickets[i] = B.helm_batch_submit(batch, mixed_plans[i], Fs[i], Gs[i], Us[i], TOL, MAX_OUTER)
        B.helm_batch_step(batch, 0)
        out = [B.helm_batch_poll(batch, t, MAX_OUTER) for t in tickets]
        return out

    def fp64_step():
        out = []
        for i in range(len(KS)):
            U[i].zero_()
            out.append(B.helm_solve(fp64_plans[i], F[i], G[i], U[i], TOL, MAX_OUTER))
        return out

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        barrier()
        times = []
        last = None
        for _ in range(steps):
            flush.fill_(1)                          # evict L2 between timed steps
            s = torch.cuda.Event(enable_timing=True)
            e = torch.cuda.Event(enable_timing=True)
            s.record()
            last = fn()
            e.record()
            e.synchronize()
            times.append(s.elapsed_time(e))
        barrier()
        return times, last

    # ---- headline: mixed batch ----
    sampler = ClockSampler(local)
    sampler.start()
    l0 = B.helm_launch_count()
    t_mixed, res_mixed = timed(mixed_step, args.steps, args.warmup)
    launches = (B.helm_launch_count() - l0)
    clocks = sampler.stop()
    l1 = B.helm_launch_count()
    mixed_step()
    launches_per_step = B.helm_launch_count() - l1
    total_ms = max_over_ranks(float(np.sum(t_mixed)))
    value = job_throughput(len(KS) * args.steps, float(np.sum(t_mixed)))
    mixed_u = [u.cpu().numpy() for u in U]
    mixed_iters = [r[1] for r in res_mixed]
    mixed_status = [B.helm_status_str(r[0]) for r in res_mixed]

    # ---- plain FP64, each solve alone ----
    fp64 = None
    fp64_u = None
    if not args.no_fp64:
        t_fp64, res_fp64 = timed(fp64_step, max(2, args.steps // 2), min(args.warmup, 2))
        tot64 = max_over_ranks(float(np.sum(t_fp64)))
        fp64 = {"value": job_throughput(len(KS) * len(t_fp64), float(np.sum(t_fp64))),
                "unit": "solves/s",
                "ms_per_step": tot64 / len(t_fp64),
                "iters": [r[1] for r in res_fp64],
                "status": [B.helm_status_str(r[0]) for r in res_fp64]}
        fp64_u = [u.cpu().numpy() for u in U]

    # ---- end to end through the public API with host buffers ----
    Fh = [torch.from_numpy(p.f).pin_memory() for p in problems]
    Gh = [torch.from_numpy(p.g).pin_memory() for p in problems]
    Uh = [torch.empty(g.shape, dtype=g.dtype).pin_memory() for g in Gh]

    from paper_2308_11469_gb300 import serve

    def e2e_step():
        # the C ABI's host entry point (helm_batch_submit_host): the library uploads f and
        # g (in submission order, the costliest solve first, which starts while the others
        # upload), solves from zero and copies every result back to pinned host memory
        return serve.solve_host_batch(batch, mixed_plans, Fh, Gh, Uh, TOL, MAX_OUTER)

    t_e2e, _ = timed(e2e_step, args.steps, args.warmup)
    e2e_value = job_throughput(len(KS) * len(t_e2e), float(np.sum(t_e2e)))
    h2d = sum(f.numel() * 16 + g.numel() * 16 for f, g in zip(Fh, Gh))
    d2h = sum(u.numel() * 16 for u in Uh)
    e2e = {"value": e2e_value, "unit": "solves/s",
           "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

    # ---- per-kernel replay of one step (events around every launch) ----
    for u in U:
        u.zero_()
    # submitted as the timed step submits them (longest first), so the lanes hold the same
    # solves and run the same forms of their steps
    tickets = [B.helm_batch_submit(batch, mixed_plans[i], F[i], G[i], U[i], TOL, MAX_OUTER)
               for i in sorted(range(len(KS)), key=lambda j: -KS[j])]
    prof = B.helm_batch_profile(batch, 0)
    for t in tickets:
        B.helm_batch_poll(batch, t, MAX_OUTER)
    total_kernel_ms = sum(v[1] for v in prof.values())
    peak, peak_kind = _peaks()
    # Roofline of the kernel with the largest device-time share.  The FP64 residual is
    # bound by the FP64 pipe (GB300 runs FP64 at a small fraction of its FP32 rate): its
    # algorithmic work is 16 FP64 flops per point (u + e: 2 adds; per component of
    # f - (sum of 4 neighbours / h^2 + cdiag u): 3 adds, 1 multiply, 1 FMA (2 flops),
    # 1 subtract) against the nominal 1.25 TFLOP/s FP64 rate.  The multigrid kernels are
    # reported against the measured HBM copy bandwidth.
    eb = 8
    top = max(prof.items(), key=lambda kv: kv[1][1])
    name, (nl, ms, by) = top
    # the FP64 peak the residual kernels are measured against: this device's own FMA rate
    fp64_tflops, fp64_probe_ms = B.helm_measure_fp64_rate()

    def hbm_line(nm, v):
        n_l, m_s, b_y = v
        ach = (b_y / n_l) / ((m_s / n_l) / 1e3) / 1e9 if n_l else 0.0
        return {"bound": "hbm", "kernel": nm, "achieved": ach, "peak": peak, "unit": "GB/s",
                "frac": ach / peak, "peak_kind": f"{peak_kind} hbm_gbs (burst)", "traffic": None,
                "share": m_s / total_kernel_ms, "bytes_per_launch": b_y / n_l if n_l else 0,
                "avg_launch_us": 1e3 * m_s / n_l if n_l else 0}

    fused = ("helmholtz_residual_update", "ascent_residual_update_2d", "ascent_l1_residual_update_2d")

    def roofline_of(name, nl, ms, by):
        if name in fused:
            if name == "helmholtz_residual_update":
                pts = by / (48 + 2 * eb)
                per_pt = RESIDUAL_DRAM_BYTES_PER_POINT
            else:
                # the instance-steps a kind's launches covered, from its algorithmic bytes (the
                # library's model per 1023^2 instance-step: e2 (zero without pre-smoothing), r_N,
                # u_N, f in and u', r out at level 0, level 1's e; with level 1 fused, level 1's
                # rhs instead of its e plus level 2's e)
                n1, n2 = (n - 1) // 2, (n - 3) // 4
                per_is = n * n * ((1 if sched_mixed[0] == 0 else 2) * eb + 48 + eb) + n1 * n1 * eb
                if name == "ascent_l1_residual_update_2d":
                    per_is += n2 * n2 * eb
                pts = float(n) ** 2 * round(by / per_is)
                per_pt = UPRES_L1_DRAM_BYTES_PER_POINT if name == "ascent_l1_residual_update_2d" \
                    else UPRES_DRAM_BYTES_PER_POINT
            flops = 16.0 * pts
            ach = (flops / nl) / ((ms / nl) / 1e3) / 1e12
            traffic = per_pt * pts / nl if per_pt else None
            hv = hbm_line(name, (nl, ms, by))
            hv["traffic"] = traffic
            hv["bytes_note"] = "fused minimum: every array the fused kernel must read or write, once"
            roofline = {"bound": "alu", "kernel": name, "achieved": ach, "peak": fp64_tflops,
                        "unit": "TFLOP/s", "frac": ach / fp64_tflops,
                        "peak_kind": "measured FP64 FMA rate of this device (helm_measure_fp64_rate: "
                                     f"8 FMA chains per thread on every SM, best launch {fp64_probe_ms:.3f} ms); "
                                     f"nominal {FP64_PEAK_TFLOPS} TFLOP/s",
                        "traffic": traffic,
                        "traffic_source": "ncu DRAM bytes per point of one launch x the average "
                                          "launch's points",
                        "share": ms / total_kernel_ms,
                        "flops_per_launch": flops / nl, "avg_launch_us": 1e3 * ms / nl,
                        "hbm_view": hv}
            if name in ("ascent_residual_update_2d", "ascent_l1_residual_update_2d"):
                # the unfused steps' bytes: residual + update (64 B/pt), prolongation +
                # correction (2e + e/4 = 18 B/pt), one red-black sweep (3e = 24 B/pt); with
                # level 1 fused, its prolongation, correction and sweep on a quarter of the
                # points (10.5 B/pt)
                b106 = (116.5 if name == "ascent_l1_residual_update_2d" else 106.0) * pts / nl
                a106 = b106 / ((ms / nl) / 1e3) / 1e9
                roofline["hbm_view_unfused_steps"] = {"bound": "hbm", "bytes_per_launch": b106,
                                                      "achieved": a106, "peak": peak, "unit": "GB/s",
                                                      "frac": a106 / peak,
                                                      "peak_kind": f"{peak_kind} hbm_gbs (burst)"}
        else:
            roofline = hbm_line(name, (nl, ms, by))
        return roofline

    roofline = roofline_of(name, nl, ms, by)
    # the other form of the fused finest kernel, where the step ran both (the latency form
    # in the critical-path lane, the throughput form covering the other lane's solves)
    other_fused = [k for k in fused[1:] if k != name and prof.get(k, (0,))[0]]
    roofline_other = roofline_of(other_fused[0], *prof[other_fused[0]]) if other_fused else None
    mg = {k: v for k, v in prof.items() if k in ("smooth_restrict_2d", "prolong_smooth_2d") and v[0]}
    roofline_mg = None
    if mg:
        n_l = sum(v[0] for v in mg.values())
        m_s = sum(v[1] for v in mg.values())
        b_y = sum(v[2] for v in mg.values())
        roofline_mg = hbm_line("smooth_restrict_2d + prolong_smooth_2d", (n_l, m_s, b_y))
    kernels = {k: {"launches": v[0], "ms": round(v[1], 4), "GBs": (v[2] / (v[1] / 1e3) / 1e9) if v[1] else 0}
               for k, v in prof.items() if v[0]}
    model_bytes = sum(v[2] for v in prof.values())
    step_ms = total_ms / args.steps
    stencil_gbs = model_bytes / (step_ms / 1e3) / 1e9

    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c64/c128",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n, "h": h, "k": list(KS), "tol": TOL,
                   "solves_per_step": len(KS), "lanes": LANES,
                   "form": "mixed complex64 V-cycles + FP64 refinement, 4-instance batch",
                   "schedule_mixed": {"nu1": sched_mixed[0], "nu2": sched_mixed[1], "cycles": sched_mixed[2],
                                      "tiles": ("auto", "large", "small")[tiles_mixed]},
                   "schedule_fp64": (None if sched_fp64 is None else
                                     {"nu1": sched_fp64[0], "nu2": sched_fp64[1], "cycles": sched_fp64[2],
                                      "tiles": ("auto", "large", "small")[tiles_fp64]}),
                   "l2": "flushed between timed steps (256 MB write)"},
        "latency_ms": {"p50": float(np.percentile(t_mixed, 50)), "p99": float(np.percentile(t_mixed, 99)),
                       "per": "step of 4 solves"},
        "iters": mixed_iters, "status": mixed_status,
        "fp64_single": fp64,
        "stencil_GBs": stencil_gbs, "stencil_frac_of_peak": stencil_gbs / peak,
        "model_bytes_per_step": model_bytes,
        "roofline": roofline, "roofline_fused_other_form": roofline_other,
        "roofline_multigrid": roofline_mg, "kernels": kernels,
        "e2e": e2e, "clocks": clocks, "gpu_launches": int(launches_per_step * args.steps),
    }

    line["fp64_rate_measured_tflops"] = fp64_tflops

    # ---- other configurations: bounded legs, each with its own clock sample ----
    legs = [] if args.legs in ("", "none") else args.legs.split(",")
    kept = {}
    for leg in legs:
        smp = ClockSampler(local)
        smp.start()
        t_leg = time.perf_counter()
        if leg == "cavity63":
            res, kp = leg_cavity63(B, torch, dev)
        elif leg == "cube255":
            res, kp = leg_cube255(B, torch, dev, flush)
        elif leg == "batch512":
            res, kp = leg_batch512(B, torch, dev, peak)
        elif leg == "served":
            # each dimension's solves on its tuned schedule: the headline's for 2D, the cube
            # leg's for 3D (V(0,2), the cube's tuned schedule, when that leg did not run)
            s3 = line.get("cube255", {}).get("mixed", {}).get("schedule")
            scheds = {2: tuple(sched_mixed[:3]),
                      3: (s3["nu1"], s3["nu2"], s3["cycles"]) if s3 else (0, 2, 1)}
            res, kp = leg_served(B, torch, dev, scheds)
        else:
            raise SystemExit(f"unknown leg {leg}")
        res["clocks"] = smp.stop()
        res["wall_s"] = time.perf_counter() - t_leg
        line[leg] = res
        kept.update(kp)
        torch.cuda.synchronize()
        torch.cuda.empty_cache()

    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        times, iters, exact, workers = cpu_oracle_workload(problems)
        done = len(times)
        cpu_val = done / float(np.sum(times))
        line["cpu_baseline"] = {"value": cpu_val, "unit": "solves/s", "cores": workers, "kind": "oracle",
                                "sample": f"{done} of the step's {len(KS)} solves, each to relres {TOL} "
                                          f"with exact sine-basis inner solves (iters {iters})"}
        acc = {"mixed_rel_l2_vs_exact": [], "fp64_rel_l2_vs_exact": []}
        for i in range(len(KS)):
            nrm = np.linalg.norm(exact[i])
            acc["mixed_rel_l2_vs_exact"].append(float(np.linalg.norm(mixed_u[i] - exact[i]) / nrm))
            if fp64_u is not None:
                acc["fp64_rel_l2_vs_exact"].append(float(np.linalg.norm(fp64_u[i] - exact[i]) / nrm))
        line["accuracy"] = acc
        if kept:
            errs, skipped, t_err = errors_vs_oracle(kept, workers)
            if "cavity63" in line:
                for row in line["cavity63"]["rows"]:
                    e = errs.get(("cavity63", row["form"])) if row["k"] == 2.0 else None
                    if e is not None:
                        row["rel_l2_vs_exact"] = e
            if "cube255" in line:
                for form in ("mixed", "fp64"):
                    if ("cube255", form) in errs:
                        line["cube255"][form]["rel_l2_vs_exact"] = errs[("cube255", form)]
            if "batch512" in line:
                for form in ("mixed", "fp64"):
                    ev = [v for kk, v in errs.items() if kk[0] == "batch512" and kk[1] == form]
                    if ev:
                        line["batch512"][f"{form}_rel_l2_vs_exact"] = {
                            "max": float(max(ev)), "median": float(np.median(ev)), "count": len(ev)}
            if "served" in line:
                ev = {kk: v for kk, v in errs.items() if kk[0] == "served"}
                line["served"]["sample_rel_l2_vs_exact"] = {
                    "max": float(max(ev.values())) if ev else None, "count": len(ev),
                    "skipped_for_time": skipped,
                    "sample": "three seeded requests per rate, smallest grids first within a 60 s budget"}
            line["accuracy_check_s"] = t_err
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    B.helm_batch_destroy(batch)
    return 0


if __name__ == "__main__":
    sys.exit(main())
