"""Timings of the method's other workloads on one GPU (one JSON line each).

    python -m paper_2308_11469_gb300.workloads [--only cavity63,cube255,batch512,damped1023,exit1023,spectral1023,annulus1024,annulus_spectrum]
    python -m paper_2308_11469_gb300.workloads --replay cube255|cavity1023 [--steps 4] [--fp64] [--pair]

* cavity63  63x63 unit-square cavity, plane-wave wall data (theta = pi/6), f = 0:
            k = 2 to relres 1e-10 and k = 5 (above k_max: the iteration diverges), mixed
            and FP64 single solves; device ms per solve.
* cube255   255^3 cube, plane-wave wall data + sine source, k = 4, relres 1e-8, mixed and
            FP64 single solves with autotuned inner schedules; solves/s.
* batch512  512 2D cavities, n in {63, 127, 255, 511}, k ~ U[0.5, 0.9 k_max], relres 1e-8:
            one mixed batch (graph run to completion) against the plain FP64 form solving
            the first 64 alone (per-solve rate).
* damped1023  the 1023^2 Gaussian cavity at k = 4 with damping p in {0, 4, 8} (general
            cavity iteration, alpha = k^2 and the rho-minimising alpha), mixed.
* exit1023  mean exit time and k_*^C of the 1023^2 square and the 255^3 cube.
* spectral1023  rho(G) against k by GPU power iteration on the 1023^2 cavity.
* annulus1024  the annular problem (square with a square hole, Robin outer edge) on a
            1024-interval grid, k = 0.8: mixed and FP64 solves; exit / local time, k_*^A.
* annulus_spectrum  rho(G) and cond(G) of that problem's iteration against k on grids of
            16 ... 1024 intervals, and the k where rho(G) = 1.

Device time comes from CUDA events on the current stream around each call.  The inputs
are the seeded generators of ``inputs``; result accuracy against exact discrete
solutions is checked by the GPU test-suite, not here.
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from . import binding as B
from . import inputs


def _dev_ms(fn, reps: int = 3):
    import torch
    best, out = None, None
    for _ in range(reps):
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record()
        out = fn()
        e.record()
        e.synchronize()
        t = s.elapsed_time(e)
        best = t if best is None else min(best, t)
    return best, out


def cavity63(dev):
    import torch
    rows = []
    for k, tol in ((2.0, 1e-10), (5.0, 1e-10)):
        p = inputs.plane_wave_cavity_2d(k)
        f = torch.from_numpy(p.f).to(dev)
        g = torch.from_numpy(p.g).to(dev)
        u = torch.zeros_like(g)
        for prec, name in ((B.HELM_PREC_MIXED, "mixed"), (B.HELM_PREC_FP64, "fp64")):
            plan = B.helm_plan_create(2, p.n, p.h, k, prec=prec)

            def run():
                u.zero_()
                return B.helm_solve(plan, f, g, u, tol, 400)
            run()
            ms, (st, it, hist) = _dev_ms(run, 5)
            rows.append({"workload": "cavity63", "k": k, "form": name, "tol": tol,
                         "status": B.helm_status_str(st), "iters": it, "ms_per_solve": ms,
                         "rho_pred": B.helm_plan_info(plan)[2]})
            B.helm_plan_destroy(plan)
    return rows


def cube255(dev):
    import torch
    rows = []
    p = inputs.plane_wave_sine_cube(4.0, seed=3, n=255)
    f = torch.from_numpy(p.f).to(dev)
    g = torch.from_numpy(p.g).to(dev)
    u = torch.zeros_like(g)
    for prec, name in ((B.HELM_PREC_MIXED, "mixed"), (B.HELM_PREC_FP64, "fp64")):
        plan = B.helm_plan_create(3, p.n, p.h, p.k, prec=prec)
        u.zero_()                      # the tuning solves start from u: the paper's zero start
        sched = B.helm_plan_autotune(plan, f, g, u, 1e-8, 2000)

        def run():
            u.zero_()
            return B.helm_solve(plan, f, g, u, 1e-8, 2000)
        ms, (st, it, hist) = _dev_ms(run, 3)
        rows.append({"workload": "cube255", "k": p.k, "form": name, "status": B.helm_status_str(st),
                     "iters": it, "ms_per_solve": ms, "solves_per_s": 1e3 / ms,
                     "schedule": {"nu1": sched[0], "nu2": sched[1], "cycles": sched[2]}})
        B.helm_plan_destroy(plan)
    return rows


def batch512(dev):
    import torch
    probs = inputs.batched_instances(count=512, seed=4)
    F = [torch.from_numpy(q.f).to(dev) for q in probs]
    G = [torch.from_numpy(q.g).to(dev) for q in probs]
    U = [torch.zeros_like(x) for x in G]
    # inner schedules tuned on the largest instance of the set
    big = max(range(len(probs)), key=lambda i: (probs[i].n, probs[i].k))
    q = probs[big]
    scheds = {}
    for prec in (B.HELM_PREC_MIXED, B.HELM_PREC_FP64):
        pl = B.helm_plan_create(2, q.n, q.h, q.k, prec=prec)
        scheds[prec] = B.helm_plan_autotune(pl, F[big], G[big], U[big], 1e-8, 3000)[:3]
        B.helm_plan_destroy(pl)
    batch = B.helm_batch_create(120 << 30)
    B.helm_batch_set_cycle(batch, *scheds[B.HELM_PREC_MIXED])

    def run_batch():
        for x in U:
            x.zero_()
        ts = [B.helm_batch_submit_geom(batch, 2, q.n, q.h, q.k, B.HELM_PREC_MIXED, F[i], G[i], U[i],
                                       1e-8, 3000) for i, q in enumerate(probs)]
        B.helm_batch_step(batch, 0)
        return [B.helm_batch_poll(batch, t, 3000) for t in ts]
    run_batch()
    ms, res = _dev_ms(run_batch, 3)
    B.helm_batch_destroy(batch)
    its = [r[1] for r in res]
    rows = [{"workload": "batch512", "form": "mixed batch", "ms_per_batch": ms,
             "solves_per_s": 512 * 1e3 / ms, "converged": int(sum(r[0] == B.HELM_CONVERGED for r in res)),
             "iters_mean": float(np.mean(its)), "iters_max": int(max(its)),
             "schedule": dict(zip(("nu1", "nu2", "cycles"), scheds[B.HELM_PREC_MIXED]))}]
    tot, cnt = 0.0, 64
    for i in range(cnt):
        q = probs[i]
        pl = B.helm_plan_create(2, q.n, q.h, q.k, prec=B.HELM_PREC_FP64)
        B.helm_plan_set_cycle(pl, *scheds[B.HELM_PREC_FP64])

        def one():
            U[i].zero_()
            return B.helm_solve(pl, F[i], G[i], U[i], 1e-8, 3000)
        one()
        t, _ = _dev_ms(one, 1)
        tot += t
        B.helm_plan_destroy(pl)
    rows.append({"workload": "batch512", "form": "fp64 single (first 64 instances)",
                 "solves_per_s": cnt * 1e3 / tot,
                 "schedule": dict(zip(("nu1", "nu2", "cycles"), scheds[B.HELM_PREC_FP64]))})
    return rows


def replay(dev, which: str, steps: int, prec: int = B.HELM_PREC_MIXED, pair: bool = False):
    """Per-kernel device time of `steps` outer steps of one solve, every launch made
    directly between CUDA events (so a profiler sees each kernel; the graph's
    conditional loop hides them): the 255^3 cube or the 1023^2 Gaussian cavity (k = 4).
    A solve alone is a critical path and runs the latency form of its step; `pair` submits
    two copies of it to one engine, whose launches then each cover both instances in the
    throughput form (2D: level 1's ascent in its own launch)."""
    import torch
    p = (inputs.plane_wave_sine_cube(4.0, seed=3, n=255) if which == "cube255"
         else inputs.gaussian_cavity_2d(4.0))
    f = torch.from_numpy(p.f).to(dev)
    g = torch.from_numpy(p.g).to(dev)
    u = torch.zeros_like(g)
    plan = B.helm_plan_create(p.D, p.n, p.h, p.k, prec=prec)
    sched = B.helm_plan_autotune(plan, f, g, u, 1e-8, 2000)[:3]
    batch = B.helm_batch_create(0)
    B.helm_batch_set_cycle(batch, *sched)
    B.helm_batch_set_lanes(batch, 1)
    us = [u] + ([torch.zeros_like(g)] if pair else [])
    for x in us:
        x.zero_()
        B.helm_batch_submit(batch, plan, f, g, x, 1e-8, 2000)
    prof = B.helm_batch_profile(batch, steps)
    B.helm_batch_destroy(batch)
    B.helm_plan_destroy(plan)
    rows = []
    for kind, (nl, ms, by) in prof.items():
        if nl:
            rows.append({"workload": f"replay_{which}" + ("_pair" if pair else ""),
                         "prec": "mixed" if prec else "fp64",
                         "schedule": dict(zip(("nu1", "nu2", "cycles"), sched)), "kernel": kind,
                         "launches": nl, "us_per_launch": 1e3 * ms / nl,
                         "model_GBs": by / (ms / 1e3) / 1e9})
    return rows


def damped1023(dev):
    """The 1023^2 Gaussian cavity, k = 4, with damping p (Eq. (2.4)) and alpha = k^2 or the
    alpha minimising rho, max(k^2, p^2 / (lambda_min - k^2)) (Section 2.2 allows any
    alpha >= k^2): mixed single solves, autotuned schedule."""
    import torch
    q = inputs.gaussian_cavity_2d(4.0)
    f = torch.from_numpy(q.f).to(dev)
    g = torch.from_numpy(q.g).to(dev)
    u = torch.zeros_like(g)
    rows = []
    for p in (0.0, 4.0, 8.0):
        plan = B.helm_plan_create(2, q.n, q.h, q.k, prec=B.HELM_PREC_MIXED)
        lam = B.helm_plan_info(plan)[0]
        for alpha in sorted({q.k ** 2, max(q.k ** 2, p * p / (lam - q.k ** 2))}):
            B.helm_plan_set_cavity(plan, alpha, p)
            u.zero_()
            sched = B.helm_plan_autotune(plan, f, g, u, 1e-8, 3000)

            def run():
                u.zero_()
                return B.helm_solve(plan, f, g, u, 1e-8, 3000)
            ms, (st, it, hist) = _dev_ms(run, 3)
            rows.append({"workload": "damped1023", "k": q.k, "p": p, "alpha": alpha, "form": "mixed",
                         "status": B.helm_status_str(st), "iters": it, "ms_per_solve": ms,
                         "solves_per_s": 1e3 / ms, "rho_pred": B.helm_plan_info(plan)[2],
                         "schedule": {"nu1": sched[0], "nu2": sched[1], "cycles": sched[2]}})
        B.helm_plan_destroy(plan)
    return rows


def exit1023(dev):
    """Mean exit time of the 1023^2 square and 255^3 cube (Delta_h E = -1) and k_*^C."""
    import torch  # noqa: F401  (device context)
    rows = []
    for D, n in ((2, 1023), (3, 255)):
        for prec, name, tol in ((B.HELM_PREC_MIXED, "mixed", 1e-8), (B.HELM_PREC_FP64, "fp64", 1e-10)):
            plan = B.helm_plan_create(D, n, 1.0 / (n + 1), 1.0, prec=prec)
            B.helm_exit_time(plan, tol, 200)
            ms, (st, emax, kstar) = _dev_ms(lambda: B.helm_exit_time(plan, tol, 200), 3)
            rows.append({"workload": "exit_time", "D": D, "n": n, "form": name, "tol": tol,
                         "status": B.helm_status_str(st), "max_E": emax, "k_star_C": kstar,
                         "ms": ms})
            B.helm_plan_destroy(plan)
    return rows


def spectral1023(dev):
    """rho(G) against k by GPU power iteration on the 1023^2 cavity (mixed, V(2,2) x 8 per
    application of M^{-1}), beside the closed form k^2 / lambda_min."""
    import torch  # noqa: F401
    rows = []
    n = 1023
    h = 1.0 / (n + 1)
    plan0 = B.helm_plan_create(2, n, h, 1.0, prec=B.HELM_PREC_MIXED)
    km = B.helm_plan_info(plan0)[1]
    B.helm_plan_destroy(plan0)
    for frac in (0.25, 0.5, 0.75, 0.9, 1.0, 1.1):
        k = frac * km
        plan = B.helm_plan_create(2, n, h, k, prec=B.HELM_PREC_MIXED)
        B.helm_plan_set_cycle(plan, 2, 2, 1)
        ms, (st, rho, its) = _dev_ms(lambda: B.helm_spectral_radius(plan, 100, 1e-7, 8), 1)
        rows.append({"workload": "spectral_radius", "n": n, "k": k, "k_over_kmax": frac,
                     "rho_power_iteration": rho, "rho_closed_form": B.helm_plan_info(plan)[2],
                     "iterations": its, "status": B.helm_status_str(st), "ms": ms})
        B.helm_plan_destroy(plan)
    return rows


def annulus1024(dev):
    """The annular problem (square [-1/2, 1/2]^2 with the hole [-0.15, 0.15]^2, Section 2.3's
    scattering data) on a 1024-interval grid at k = 0.8: single solves to relres 1e-8, mixed
    and FP64; exit time, local time and k_*^A (both normalisations of E)."""
    import torch
    N, k = 1024, 0.8
    d = torch.from_numpy(inputs.annulus_scattering(N, k)).to(dev)
    u = torch.empty_like(d)
    rows = []
    for prec, name in ((B.HELM_PREC_MIXED, "mixed"), (B.HELM_PREC_FP64, "fp64")):
        plan = B.helm_annulus_create(N, 1.0, 0.15, k, prec)
        B.helm_annulus_solve(plan, d, u, 1e-8, 2000)
        ms, (st, it, hist) = _dev_ms(lambda: B.helm_annulus_solve(plan, d, u, 1e-8, 2000), 3)
        # algorithmic bytes per fine node and outer step: FP64 step (U in/out 32, data 16, e and
        # rhs one inner element each) + V(2,2) on level 0 (4 half-sweep pairs reading e, rhs and
        # writing e: 3 elements each; restriction 2 elements; prolongation 2) x 4/3 for the levels
        eb = 8 if prec == B.HELM_PREC_MIXED else 16
        per_node = 48 + 2 * eb + (4 * 3 * eb + 2 * eb + 2 * eb) * 4 / 3
        bytes_step = per_node * (N + 1) ** 2
        rows.append({"workload": "annulus1024", "N": N, "k": k, "form": name, "status": B.helm_status_str(st),
                     "iters": it, "ms_per_solve": ms, "solves_per_s": 1e3 / ms, "us_per_step": 1e3 * ms / max(it, 1),
                     "model_bytes_per_step": bytes_step,
                     "model_GBs": bytes_step / (ms / max(it, 1) / 1e3) / 1e9})
        B.helm_annulus_destroy(plan)
    E = torch.empty((N + 1, N + 1), dtype=torch.float64, device=dev)
    L = torch.empty_like(E)
    plan = B.helm_annulus_create(N, 1.0, 0.15, k, B.HELM_PREC_MIXED)
    for c_tau in (1.0, 2.0):
        ms, (st, ks) = _dev_ms(lambda: B.helm_annulus_exit_times(plan, E, L, c_tau=c_tau, tol=1e-8), 1)
        rows.append({"workload": "annulus1024_exit", "N": N, "c_tau": c_tau, "status": B.helm_status_str(st),
                     "k_star_A": ks, "max_E": float(E.max()), "max_L": float(L.max()), "ms": ms})
    B.helm_annulus_destroy(plan)
    return rows


def annulus_spectrum(dev):
    """Section 2.4's figure on the GPU: rho(G) and cond(G) against k for the square
    [-1/2, 1/2]^2 with the hole [-0.15, 0.15]^2 on grids of 16 ... 1024 intervals (power
    iteration and Lanczos with multigrid cycles as A^{-1}), and the k where rho(G) crosses 1
    (bisection on the power-iteration estimate)."""
    import torch  # noqa: F401
    rows = []
    for N, prec, cyc in ((16, B.HELM_PREC_FP64, 24), (32, B.HELM_PREC_FP64, 24), (64, B.HELM_PREC_FP64, 24),
                         (256, B.HELM_PREC_MIXED, 12), (1024, B.HELM_PREC_MIXED, 12)):
        for k in (0.25, 0.5, 0.75, 1.0, 1.25, 1.5):
            plan = B.helm_annulus_create(N, 1.0, 0.15, k, prec)
            tol = 1e-8 if prec == B.HELM_PREC_FP64 else 1e-6     # complex64 cycles: ~1e-6 floor
            ms, (st, rho, lam, its) = _dev_ms(lambda: B.helm_annulus_spectral_radius(plan, 300, tol, cyc), 1)
            row = {"workload": "annulus_spectrum", "N": N, "h": 1.0 / N, "k": k,
                   "prec": "fp64" if prec == B.HELM_PREC_FP64 else "mixed", "cycles": cyc,
                   "rho": rho, "lambda": [lam.real, lam.imag], "rho_iters": its,
                   "rho_status": B.helm_status_str(st), "rho_ms": ms}
            if N <= 64:                 # FP64 grids: both singular values converge
                ms2, (st2, smax, smin, cond, its2) = _dev_ms(
                    lambda: B.helm_annulus_condition(plan, 3000, tol, cyc), 1)
                row.update({"sigma_max": smax, "sigma_min": smin, "cond": cond, "cond_iters": its2,
                            "cond_status": B.helm_status_str(st2), "cond_ms": ms2})
            B.helm_annulus_destroy(plan)
            rows.append(row)
        # crossing of rho = 1 by bisection in k
        lo, hi = 0.5, 2.0
        for _ in range(20 if N <= 256 else 12):
            mid = 0.5 * (lo + hi)
            plan = B.helm_annulus_create(N, 1.0, 0.15, mid, prec)
            st, rho, _, _ = B.helm_annulus_spectral_radius(plan, 300, 1e-8 if prec == B.HELM_PREC_FP64 else 1e-6, cyc)
            B.helm_annulus_destroy(plan)
            if rho < 1.0:
                lo = mid
            else:
                hi = mid
        rows.append({"workload": "annulus_spectrum_crossing", "N": N, "h": 1.0 / N,
                     "k_rho_eq_1": 0.5 * (lo + hi), "bracket": [lo, hi]})
    return rows


WORKLOADS = {"cavity63": cavity63, "cube255": cube255, "batch512": batch512,
             "damped1023": damped1023, "exit1023": exit1023, "spectral1023": spectral1023,
             "annulus1024": annulus1024, "annulus_spectrum": annulus_spectrum}


def main(argv=None) -> int:
    import torch

    from . import build
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--only", default=",".join(WORKLOADS))
    ap.add_argument("--replay", default=None, choices=["cube255", "cavity1023"],
                    help="per-kernel replay of a few outer steps of one solve instead")
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--fp64", action="store_true", help="replay the plain FP64 form")
    ap.add_argument("--pair", action="store_true",
                    help="replay two copies of the solve in one engine (the throughput form)")
    args = ap.parse_args(argv)
    build.build()
    B.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    if args.replay:
        for row in replay(dev, args.replay, args.steps,
                          B.HELM_PREC_FP64 if args.fp64 else B.HELM_PREC_MIXED, args.pair):
            print(json.dumps(row), flush=True)
        return 0
    for name in args.only.split(","):
        for row in WORKLOADS[name](dev):
            print(json.dumps(row), flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
