"""GPU batch / serving path: each result is the same alone and in the mix.

Instances in a batch share every launch, but each one's arithmetic depends only on its
own data (fixed tile partials, no cross-instance reduction), so results must be
bit-identical to the single-solve path; admission respects the memory cap.
"""
import numpy as np
import pytest

from oracle import fd
from paper_2308_11469_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
DEV = "cuda:0"


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_11469_gb300 import binding, build
    build.build()
    binding.load()
    return binding


def _solo(B, p, prec, tol, max_outer):
    plan = B.helm_plan_create(p.D, p.n, p.h, p.k, prec=prec)
    f = torch.from_numpy(p.f).to(DEV)
    g = torch.from_numpy(p.g).to(DEV)
    u = torch.zeros_like(g)
    st, iters, hist = B.helm_solve(plan, f, g, u, tol, max_outer)
    B.helm_plan_destroy(plan)
    return st, iters, hist, u.cpu().numpy()


def _mix():
    probs = inputs.batched_instances(count=10, seed=4, sizes=(15, 31, 63, 127, 255),
                                      probs=(0.2, 0.2, 0.2, 0.2, 0.2))
    probs.append(inputs.plane_wave_sine_cube(3.0, seed=3, n=15))
    probs.append(inputs.plane_wave_sine_cube(4.0, seed=5, n=31))
    probs.append(inputs.plane_wave_cavity_2d(2.0))
    return probs


@pytest.mark.parametrize("prec", [1, 0])
def test_batch_equals_solo(B, prec):
    probs = _mix()
    tol, max_outer = 1e-8, 2000
    batch = B.helm_batch_create(0)
    keep = []
    tickets = []
    for p in probs:
        plan = B.helm_plan_create(p.D, p.n, p.h, p.k, prec=prec)
        f = torch.from_numpy(p.f).to(DEV)
        g = torch.from_numpy(p.g).to(DEV)
        u = torch.zeros_like(g)
        keep.append((f, g, u))
        tickets.append(B.helm_batch_submit(batch, plan, f, g, u, tol, max_outer))
        B.helm_plan_destroy(plan)          # the batch copied what it needs
    assert all(t is not None for t in tickets)
    results = [None] * len(probs)
    for _ in range(10000):
        B.helm_batch_step(batch, 7)
        for i, t in enumerate(tickets):
            if results[i] is None:
                r = B.helm_batch_poll(batch, t, max_outer)
                if r is not None:
                    results[i] = r
        if all(r is not None for r in results):
            break
    assert B.helm_batch_info(batch) == (0, 0)
    B.helm_batch_destroy(batch)
    for i, p in enumerate(probs):
        st, iters, hist = results[i]
        s2, it2, h2, u2 = _solo(B, p, prec, tol, max_outer)
        assert st == s2 == B.HELM_CONVERGED
        assert iters == it2
        assert np.array_equal(hist, h2)
        assert np.array_equal(keep[i][2].cpu().numpy(), u2)
        exact = fd.solve_exact_dst(p.f, p.g, p.h, p.k)
        err = np.linalg.norm(u2 - exact) / np.linalg.norm(exact)
        # relres 1e-8 leaves ~1e-7 relative error in either precision
        assert err <= 1e-6, (i, err)


def test_admission_cap(B):
    p = inputs.gaussian_cavity_2d(2.0, n=255)
    plan = B.helm_plan_create(2, 255, p.h, p.k, prec=1)
    lm, km, rho, ws = B.helm_plan_info(plan)
    f = torch.from_numpy(p.f).to(DEV)
    g = torch.from_numpy(p.g).to(DEV)
    us = [torch.zeros_like(g) for _ in range(3)]
    batch = B.helm_batch_create(int(ws * 2.5))
    t0 = B.helm_batch_submit(batch, plan, f, g, us[0], 1e-8, 200)
    t1 = B.helm_batch_submit(batch, plan, f, g, us[1], 1e-8, 200)
    t2 = B.helm_batch_submit(batch, plan, f, g, us[2], 1e-8, 200)
    assert t0 is not None and t1 is not None and t2 is None       # over the cap
    active, used = B.helm_batch_info(batch)
    assert active == 2 and 0 < used <= ws * 2.5
    B.helm_batch_step(batch, 0)
    assert B.helm_batch_poll(batch, t0, 200) is not None
    assert B.helm_batch_poll(batch, t1, 200) is not None
    t2 = B.helm_batch_submit(batch, plan, f, g, us[2], 1e-8, 200)  # room again
    assert t2 is not None
    B.helm_batch_step(batch, 0)
    r2 = B.helm_batch_poll(batch, t2, 200)
    assert r2 is not None and r2[0] == B.HELM_CONVERGED
    assert torch.equal(us[0], us[2])
    B.helm_batch_destroy(batch)
    B.helm_plan_destroy(plan)


def test_late_arrivals_join_running_batch(B):
    # continuous batching: a solve submitted while another is mid-flight gives the
    # same result as alone
    a = inputs.gaussian_cavity_2d(4.0, n=127)
    b = inputs.gaussian_cavity_2d(3.0, seed=9, n=63)
    batch = B.helm_batch_create(0)
    bufs = []
    for p in (a, b):
        f = torch.from_numpy(p.f).to(DEV)
        g = torch.from_numpy(p.g).to(DEV)
        bufs.append((f, g, torch.zeros_like(g)))
    pa = B.helm_plan_create(2, a.n, a.h, a.k, prec=1)
    pb = B.helm_plan_create(2, b.n, b.h, b.k, prec=1)
    ta = B.helm_batch_submit(batch, pa, *bufs[0], 1e-8, 500)
    B.helm_batch_step(batch, 5)
    assert B.helm_batch_poll(batch, ta, 500) is None
    tb = B.helm_batch_submit(batch, pb, *bufs[1], 1e-8, 500)
    B.helm_batch_step(batch, 0)
    ra = B.helm_batch_poll(batch, ta, 500)
    rb = B.helm_batch_poll(batch, tb, 500)
    for p, r, buf in ((a, ra, bufs[0]), (b, rb, bufs[1])):
        st, iters, hist, u = _solo(B, p, 1, 1e-8, 500)
        assert r[0] == st and r[1] == iters
        assert np.array_equal(r[2], hist)
        assert np.array_equal(buf[2].cpu().numpy(), u)
    B.helm_batch_destroy(batch)


def test_lanes_do_not_change_results(B):
    # the same submissions spread over 1, 2 or 4 concurrent lanes give the same results
    probs = [inputs.gaussian_cavity_2d(k, seed=3, n=127) for k in (1.0, 2.0, 3.0, 4.0)]
    out = {}
    for lanes in (1, 2, 4):
        batch = B.helm_batch_create(0)
        B.helm_batch_set_lanes(batch, lanes)
        us, ts, keep = [], [], []
        for p in probs:
            plan = B.helm_plan_create(2, p.n, p.h, p.k, prec=1)
            # the batch reads f and g when it steps: they must outlive the submission
            f, g = torch.from_numpy(p.f).to(DEV), torch.from_numpy(p.g).to(DEV)
            u = torch.zeros((p.n + 2,) * 2, dtype=torch.complex128, device=DEV)
            ts.append(B.helm_batch_submit(batch, plan, f, g, u, 1e-8, 2000))
            B.helm_plan_destroy(plan)
            keep.append((f, g))
            us.append(u)
        B.helm_batch_step(batch, 0)
        out[lanes] = [(B.helm_batch_poll(batch, t, 2000), u.cpu().numpy()) for t, u in zip(ts, us)]
        B.helm_batch_destroy(batch)
    for lanes in (2, 4):
        for (r1, u1), (r2, u2) in zip(out[1], out[lanes]):
            assert r1[0] == r2[0] == B.HELM_CONVERGED and r1[1] == r2[1]
            assert np.array_equal(r1[2], r2[2]) and np.array_equal(u1, u2)
    batch = B.helm_batch_create(0)
    for bad in (0, 5):
        with pytest.raises(B.HelmError):
            B.helm_batch_set_lanes(batch, bad)
    B.helm_batch_destroy(batch)


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("chunk", [0, 5])
def test_host_result_copy(B, chunk, pinned):
    # the result also lands in host memory: behind the lane's last step when the step runs
    # to completion (chunk 0, page-locked buffers), at retirement otherwise
    probs = [inputs.gaussian_cavity_2d(k, seed=2, n=127) for k in (1.0, 2.5, 4.0)]
    batch = B.helm_batch_create(0)
    F = [torch.from_numpy(p.f).to(DEV) for p in probs]
    G = [torch.from_numpy(p.g).to(DEV) for p in probs]
    U = [torch.zeros_like(g) for g in G]
    UH = [torch.full(tuple(g.shape), complex(7.0, 7.0), dtype=torch.complex128) for g in G]
    if pinned:
        UH = [x.pin_memory() for x in UH]
    plans = [B.helm_plan_create(2, p.n, p.h, p.k, prec=1) for p in probs]
    tickets = [B.helm_batch_submit(batch, plans[i], F[i], G[i], U[i], 1e-8, 2000) for i in range(3)]
    for t, uh in zip(tickets, UH):
        B.helm_batch_set_host_result(batch, t, uh)
    with pytest.raises(B.HelmError):
        B.helm_batch_set_host_result(batch, 10 ** 9, UH[0])          # unknown ticket
    with pytest.raises(ValueError):
        B.helm_batch_set_host_result(batch, tickets[0], U[0])       # a device tensor
    res = [None] * 3
    while any(r is None for r in res):
        B.helm_batch_step(batch, chunk)
        for i, t in enumerate(tickets):
            if res[i] is None:
                res[i] = B.helm_batch_poll(batch, t, 2000)
    torch.cuda.synchronize()
    for i, p in enumerate(probs):
        st, it, hist, u = _solo(B, p, 1, 1e-8, 2000)
        assert res[i][0] == st == B.HELM_CONVERGED and res[i][1] == it
        assert np.array_equal(UH[i].numpy(), u)
        assert np.array_equal(U[i].cpu().numpy(), u)
    B.helm_batch_destroy(batch)
    for pl in plans:
        B.helm_plan_destroy(pl)


def test_tile_policies_give_the_same_solutions(B):
    """The 2D tile-shape policy changes only how the levels are cut into tiles (each shape is
    its own kernel instantiation, so the FP32 cycle may round differently in the last bit):
    a batch of uneven sizes converges under each policy to the same solutions within the
    mixed-precision tolerance, and the autotuner keeps one of the policies."""
    probs = inputs.batched_instances(count=12, seed=9)
    outs = []
    for pol in (B.HELM_TILES_AUTO, B.HELM_TILES_LARGE, B.HELM_TILES_SMALL):
        batch = B.helm_batch_create(0)
        B.helm_batch_set_tiles(batch, pol)
        bufs, tickets = [], []
        for q in probs:
            f = torch.from_numpy(q.f).to(DEV)
            g = torch.from_numpy(q.g).to(DEV)
            u = torch.zeros_like(g)
            tickets.append(B.helm_batch_submit_geom(batch, 2, q.n, q.h, q.k, B.HELM_PREC_MIXED, f, g, u,
                                                    1e-8, 3000))
            bufs.append(u)
        B.helm_batch_step(batch, 0)
        res = [B.helm_batch_poll(batch, t, 3000) for t in tickets]
        assert all(r[0] == B.HELM_CONVERGED for r in res)
        outs.append([u.cpu().numpy() for u in bufs])
        B.helm_batch_destroy(batch)
    for other in outs[1:]:
        for a, b in zip(outs[0], other):
            assert np.linalg.norm(a - b) <= 1e-6 * np.linalg.norm(a)
    q = max(probs, key=lambda p: p.n)
    plan = B.helm_plan_create(2, q.n, q.h, q.k, prec=B.HELM_PREC_MIXED)
    f = torch.from_numpy(q.f).to(DEV)
    g = torch.from_numpy(q.g).to(DEV)
    u = torch.zeros_like(g)
    B.helm_plan_autotune(plan, f, g, u, 1e-8, 3000)
    assert B.helm_plan_tiles(plan) in (B.HELM_TILES_AUTO, B.HELM_TILES_LARGE, B.HELM_TILES_SMALL)
    with pytest.raises(B.HelmError):
        B.helm_plan_set_tiles(plan, 7)
    B.helm_plan_destroy(plan)


def test_class_schedules_equal_solo_solves(B):
    """A batch mixing 2D and 3D solves with a schedule per dimension gives each solve the
    iterates of a single solve on that schedule, bit for bit."""
    probs = _mix()
    sched = {2: (0, 1, 1), 3: (0, 2, 1)}
    tol, max_outer = 1e-8, 2000
    batch = B.helm_batch_create(0)
    for d, sc in sched.items():
        B.helm_batch_set_cycle_class(batch, d, B.HELM_PREC_MIXED, *sc)
    keep, tickets = [], []
    for p in probs:
        f = torch.from_numpy(p.f).to(DEV)
        g = torch.from_numpy(p.g).to(DEV)
        u = torch.zeros_like(g)
        keep.append((f, g, u))
        tickets.append(B.helm_batch_submit_geom(batch, p.D, p.n, p.h, p.k, B.HELM_PREC_MIXED, f, g, u, tol,
                                                max_outer))
    B.helm_batch_step(batch, 0)
    results = [B.helm_batch_poll(batch, t, max_outer) for t in tickets]
    B.helm_batch_destroy(batch)
    for i, p in enumerate(probs):
        plan = B.helm_plan_create(p.D, p.n, p.h, p.k, prec=B.HELM_PREC_MIXED)
        B.helm_plan_set_cycle(plan, *sched[p.D])
        f, g, _ = keep[i]
        u = torch.zeros_like(g)
        st, it, hist = B.helm_solve(plan, f, g, u, tol, max_outer)
        B.helm_plan_destroy(plan)
        assert results[i][0] == st == B.HELM_CONVERGED
        assert results[i][1] == it
        assert np.array_equal(results[i][2], hist)
        assert np.array_equal(keep[i][2].cpu().numpy(), u.cpu().numpy())
    with pytest.raises(B.HelmError):
        B.helm_batch_set_cycle_class(B.helm_batch_create(0), 4, B.HELM_PREC_MIXED, 0, 1, 1)


@pytest.mark.parametrize("sizes", [(127, 255), (63, 127, 255, 511), (511, 1023)])
def test_mixed_sizes_v01_equal_solo_solves(B, sizes):
    """Instances of different sizes in one launch sequence on V(0, 1) (descent steps paired
    per launch where every instance shares both levels, the cluster tail where all are at
    least 511): each result is that of a single solve, bit for bit."""
    probs = []
    for i, n in enumerate(sizes):
        probs += inputs.batched_instances(count=1, seed=60 + i, sizes=(n,), probs=(1.0,))
    tol, max_outer = 1e-8, 3000
    batch = B.helm_batch_create(0)
    B.helm_batch_set_cycle(batch, 0, 1, 1)
    B.helm_batch_set_lanes(batch, 1)
    keep, tickets = [], []
    for p in probs:
        f = torch.from_numpy(p.f).to(DEV)
        g = torch.from_numpy(p.g).to(DEV)
        u = torch.zeros_like(g)
        keep.append((f, g, u))
        tickets.append(B.helm_batch_submit_geom(batch, p.D, p.n, p.h, p.k, B.HELM_PREC_MIXED, f, g, u, tol,
                                                max_outer))
    B.helm_batch_step(batch, 0)
    results = [B.helm_batch_poll(batch, t, max_outer) for t in tickets]
    B.helm_batch_destroy(batch)
    for i, p in enumerate(probs):
        plan = B.helm_plan_create(p.D, p.n, p.h, p.k, prec=B.HELM_PREC_MIXED)
        B.helm_plan_set_cycle(plan, 0, 1, 1)
        f, g, _ = keep[i]
        u = torch.zeros_like(g)
        st, it, hist = B.helm_solve(plan, f, g, u, tol, max_outer)
        B.helm_plan_destroy(plan)
        assert results[i][0] == st == B.HELM_CONVERGED, (p.n, results[i][0], st)
        assert results[i][1] == it
        assert np.array_equal(results[i][2], hist)
        assert np.array_equal(keep[i][2].cpu().numpy(), u.cpu().numpy())


def test_submit_many_equals_single_submissions(B):
    """Bulk submission and polling give the results of one-by-one submission bit for bit,
    and a memory cap admits a prefix (the rest wait)."""
    probs = inputs.batched_instances(count=16, seed=13)
    tol, max_outer = 1e-8, 3000
    data = [(torch.from_numpy(q.f).to(DEV), torch.from_numpy(q.g).to(DEV)) for q in probs]
    U1 = [torch.zeros_like(g) for _, g in data]
    batch = B.helm_batch_create(0)
    ts = [B.helm_batch_submit_geom(batch, 2, q.n, q.h, q.k, B.HELM_PREC_MIXED, f, g, u, tol, max_outer)
          for q, (f, g), u in zip(probs, data, U1)]
    B.helm_batch_step(batch, 0)
    r1 = [B.helm_batch_poll(batch, t, max_outer) for t in ts]
    B.helm_batch_destroy(batch)
    U2 = [torch.zeros_like(g) for _, g in data]
    batch = B.helm_batch_create(0)
    jobs = [(2, q.n, q.h, q.k, f, g, u) for q, (f, g), u in zip(probs, data, U2)]
    ts = B.helm_batch_submit_many(batch, jobs, B.HELM_PREC_MIXED, tol, max_outer)
    assert len(ts) == len(jobs)
    B.helm_batch_step(batch, 0)
    r2 = B.helm_batch_poll_many(batch, ts)
    assert B.helm_batch_info(batch) == (0, 0)
    B.helm_batch_destroy(batch)
    for a, b, u1, u2 in zip(r1, r2, U1, U2):
        assert b[0] == 1 and (a[0], a[1]) == (b[1], b[2])
        assert torch.equal(u1, u2)
    # a cap below the whole set: a prefix is admitted, the rest after retirements (each
    # solve's reservation read from a batch holding it alone)
    need = []
    for q, (f, g) in zip(probs[:3], data[:3]):
        b1 = B.helm_batch_create(0)
        u = torch.zeros_like(g)
        t = B.helm_batch_submit_geom(b1, 2, q.n, q.h, q.k, B.HELM_PREC_MIXED, f, g, u, tol, max_outer)
        need.append(B.helm_batch_info(b1)[1])
        B.helm_batch_step(b1, 0)
        B.helm_batch_poll(b1, t, max_outer)
        B.helm_batch_destroy(b1)
    batch = B.helm_batch_create(int(need[0] + need[1] + need[2] // 2))
    U3 = [torch.zeros_like(g) for _, g in data[:3]]
    ts = B.helm_batch_submit_many(batch, [(2, q.n, q.h, q.k, f, g, u) for q, (f, g), u in
                                         zip(probs[:3], data[:3], U3)], B.HELM_PREC_MIXED, tol, max_outer)
    assert len(ts) == 2
    B.helm_batch_step(batch, 0)
    assert all(d == 1 for d, _, _ in B.helm_batch_poll_many(batch, ts))
    B.helm_batch_destroy(batch)


def test_latency_lane_fuses_level_1_and_equals_solo(B):
    # four 1023^2 cavities, k = 1..4, in two lanes, submitted longest first: the k = 4
    # solve alone in the highest-priority lane runs the latency form of its step (level 1's
    # ascent inside the fused finest kernel, one launch per outer step), the three shorter
    # ones share the other lane in the throughput form; every result is that of the solve
    # alone, bit for bit
    ks = (4.0, 3.0, 2.0, 1.0)
    probs = [inputs.gaussian_cavity_2d(k) for k in ks]
    tol, max_outer = 1e-6, 400
    batch = B.helm_batch_create(0)
    B.helm_batch_set_cycle(batch, 0, 1, 1)
    B.helm_batch_set_lanes(batch, 2)
    # the batch reads f, g and u through their device pointers: the tensors stay alive
    fs = [torch.from_numpy(p.f).to(DEV) for p in probs]
    gs = [torch.from_numpy(p.g).to(DEV) for p in probs]
    us = [torch.zeros_like(g) for g in gs]
    plans, tickets = [], []
    for i, p in enumerate(probs):
        pl = B.helm_plan_create(2, p.n, p.h, p.k, prec=B.HELM_PREC_MIXED)
        B.helm_plan_set_cycle(pl, 0, 1, 1)
        plans.append(pl)
        tickets.append(B.helm_batch_submit(batch, pl, fs[i], gs[i], us[i], tol, max_outer))
    prof = B.helm_batch_profile(batch, 0)
    res = [B.helm_batch_poll(batch, t, max_outer) for t in tickets]
    B.helm_batch_destroy(batch)
    iters = [r[1] for r in res]
    assert all(r[0] == B.HELM_CONVERGED for r in res) and min(iters) > 0
    assert prof["ascent_l1_residual_update_2d"][0] == iters[0]
    assert prof["ascent_residual_update_2d"][0] == max(iters[1:])
    for i, p in enumerate(probs):
        u = torch.zeros_like(us[i])
        st, it, hist = B.helm_solve(plans[i], fs[i], gs[i], u, tol, max_outer)
        assert st == B.HELM_CONVERGED and it == iters[i] and np.array_equal(hist, res[i][2])
        assert np.array_equal(u.cpu().numpy(), us[i].cpu().numpy())
    for pl in plans:
        B.helm_plan_destroy(pl)
