"""Parity at the full sizes of the workloads (through the C ABI), against the oracle's
exact discrete solutions (sine-basis solves), and the k_max status at those sizes.

* 1023^2 Gaussian cavity, k in {1, 2, 3, 4}: mixed and FP64 at relres 1e-8 (the bench
  workload, solved as the bench solves it: one four-instance batch / single plans).
* 255^3 plane-wave + sine-source cube, k = 4: mixed at relres 1e-8.
* 512-instance batch of 2D cavities N in {63, 127, 255, 511}: every result checked
  against the exact solution (a seeded sample of 64 by the oracle), all converged.
"""
import numpy as np
import pytest

from oracle import fd, iteration as it
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


def _relerr(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _batch_solve(B, probs, prec, tol=1e-8, max_outer=3000, cap=0):
    batch = B.helm_batch_create(cap)
    bufs, tickets = [], []
    for p in probs:
        plan = B.helm_plan_create(p.D, p.n, p.h, p.k, prec=prec)
        f = torch.from_numpy(p.f).to(DEV)
        g = torch.from_numpy(p.g).to(DEV)
        u = torch.zeros_like(g)
        t = B.helm_batch_submit(batch, plan, f, g, u, tol, max_outer)
        assert t is not None
        B.helm_plan_destroy(plan)
        bufs.append((f, g, u))
        tickets.append(t)
    B.helm_batch_step(batch, 0)
    out = []
    for t, (f, g, u) in zip(tickets, bufs):
        r = B.helm_batch_poll(batch, t, max_outer)
        assert r is not None
        out.append((r[0], r[1], r[2], u.cpu().numpy()))
    B.helm_batch_destroy(batch)
    return out


def test_gaussian_cavity_1023_mixed_batch_and_fp64(B):
    probs = [inputs.gaussian_cavity_2d(k) for k in (1.0, 2.0, 3.0, 4.0)]
    mixed = _batch_solve(B, probs, B.HELM_PREC_MIXED)
    for p, (st, iters, hist, u) in zip(probs, mixed):
        assert st == B.HELM_CONVERGED and hist[-1] <= 1e-8
        assert it.predicted_status(2, p.n, p.h, p.k) == it.CONVERGED
        exact = fd.solve_exact_dst(p.f, p.g, p.h, p.k)
        assert _relerr(u, exact) <= 1e-6
    # plain FP64 single solve.  At 1023^2 FP64 itself limits the attainable residual:
    # each residual entry carries rounding ~eps * 8/h^2 |u| ~ 1e-9 |u|, a relres floor near
    # 1e-10, so the FP64 check here is taken at tol 1e-9 (error ~ 1e-8); the 1e-10 FP64
    # parity is checked on the grids where rounding allows it (test_gpu_parity.py).
    p = probs[1]
    plan = B.helm_plan_create(2, p.n, p.h, p.k, prec=B.HELM_PREC_FP64)
    f = torch.from_numpy(p.f).to(DEV)
    g = torch.from_numpy(p.g).to(DEV)
    u = torch.zeros_like(g)
    st, iters, hist = B.helm_solve(plan, f, g, u, 1e-9, 3000)
    B.helm_plan_destroy(plan)
    assert st == B.HELM_CONVERGED
    exact = fd.solve_exact_dst(p.f, p.g, p.h, p.k)
    assert _relerr(u.cpu().numpy(), exact) <= 1e-8


def test_plane_wave_sine_cube_255_mixed(B):
    # With plane-wave wall data ||r_0|| = ||b|| is dominated by the lifted wall values
    # (g / h^2 next to the wall), so relres 1e-8 only bounds the error to ~1e-5 of ||u||
    # (||u - u*|| <= ||r|| / (lambda_min - k^2)); parity is taken at relres 1e-10 (mixed
    # precision reaches it: the residual is FP64) and the 1e-8 error is checked to be
    # within that bound.
    p = inputs.plane_wave_sine_cube(4.0, seed=3, n=255)
    exact = fd.solve_exact_dst(p.f, p.g, p.h, p.k)
    (st, iters, hist, u), = _batch_solve(B, [p], B.HELM_PREC_MIXED, tol=1e-10)
    assert st == B.HELM_CONVERGED
    assert _relerr(u, exact) <= 1e-6
    (st, iters, hist, u), = _batch_solve(B, [p], B.HELM_PREC_MIXED, tol=1e-8)
    assert st == B.HELM_CONVERGED
    lam = fd.lambda_min(3, p.n, p.h)
    r0 = np.linalg.norm(fd.lifted_rhs(p.f, p.g, p.h))
    bound = hist[-1] * r0 / (lam - p.k ** 2) / np.linalg.norm(exact)
    assert _relerr(u, exact) <= bound


def test_batched_512_instances(B):
    probs = inputs.batched_instances(count=512, seed=4)
    res = _batch_solve(B, probs, B.HELM_PREC_MIXED, cap=120 << 30)
    assert all(r[0] == B.HELM_CONVERGED for r in res)
    rng = np.random.default_rng(40)
    for i in rng.choice(len(probs), size=64, replace=False):
        p = probs[i]
        exact = fd.solve_exact_dst(p.f, p.g, p.h, p.k)
        assert _relerr(res[i][3], exact) <= 1e-6, i
