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


# ---------------------------------------------------------------------------
# FP64 at full size: the attainable relres floor, and 1e-10 parity below it
# ---------------------------------------------------------------------------

def _fp64_to_floor(B, p, max_outer):
    """Plain FP64 solve run past its rounding floor (tol 0): the outer loop stops at
    max_outer (or by the stagnation rule).  Returns (status, hist, u)."""
    plan = B.helm_plan_create(p.D, p.n, p.h, p.k, prec=B.HELM_PREC_FP64)
    f = torch.from_numpy(p.f).to(DEV)
    g = torch.from_numpy(p.g).to(DEV)
    u = torch.zeros_like(g)
    st, iters, hist = B.helm_solve(plan, f, g, u, 0.0, max_outer)
    B.helm_plan_destroy(plan)
    return st, hist, u.cpu().numpy()


@pytest.mark.parametrize("k", [2.0, 4.0])
def test_fp64_floor_and_parity_1023(B, k):
    # The FP64 residual of a 1023^2 iterate carries rounding ~ eps 8/h^2 |u| per entry, so
    # relres stalls near 1e-10 (measured, printed), while the increments it drives are
    # divided by ~8/h^2 again: the iterate itself keeps converging, to ~1e-13.
    p = inputs.gaussian_cavity_2d(k)
    st, hist, u = _fp64_to_floor(B, p, 200 if k == 2.0 else 400)
    assert st in (B.HELM_MAXITER, B.HELM_DIVERGED)
    exact = fd.solve_exact_dst(p.f, p.g, p.h, p.k)
    err = _relerr(u, exact)
    floor = float(np.min(hist))
    print(f"FP64 1023^2 k={k}: relres floor {floor:.3e} (last {hist[-1]:.3e}, {len(hist) - 1} steps), "
          f"rel. L2 error vs exact {err:.3e}")
    assert floor < 1e-9
    assert err <= 1e-10, err


def test_fp64_floor_and_parity_cube_255(B):
    p = inputs.plane_wave_sine_cube(4.0, seed=3, n=255)
    st, hist, u = _fp64_to_floor(B, p, 120)
    assert st in (B.HELM_MAXITER, B.HELM_DIVERGED)
    exact = fd.solve_exact_dst(p.f, p.g, p.h, p.k)
    err = _relerr(u, exact)
    floor = float(np.min(hist))
    print(f"FP64 255^3 k=4: relres floor {floor:.3e} (last {hist[-1]:.3e}, {len(hist) - 1} steps), "
          f"rel. L2 error vs exact {err:.3e}")
    assert floor < 1e-10
    assert err <= 1e-10, err


@pytest.mark.parametrize("D,n,k", [(2, 255, 3.0), (2, 511, 2.0), (3, 63, 4.0)])
def test_fp64_iterates_match_exact_solve_iterates_large(B, D, n, k):
    # enough V(2,2) cycles per outer step that each inner solve is exact to rounding: the
    # GPU iterates are the paper's partial sums, step by step (sine-basis inner solves)
    h = 1.0 / (n + 1)
    rng = np.random.default_rng(21 + n)
    f = rng.standard_normal((n,) * D) + 1j * rng.standard_normal((n,) * D)
    g = rng.standard_normal((n + 2,) * D) + 1j * rng.standard_normal((n + 2,) * D)
    N = 5
    ora = it.paper_iteration(f, g, h, k, tol=0.0, max_outer=N, keep_iterates=True, poisson="dst")
    plan = B.helm_plan_create(D, n, h, k, prec=B.HELM_PREC_FP64)
    B.helm_plan_set_cycle(plan, 2, 2, 14)
    ft = torch.from_numpy(f).to(DEV)
    gt = torch.from_numpy(g).to(DEV)
    for steps in (1, 3, N):
        u = torch.zeros_like(gt)
        st, iters, hist, einf = B.helm_solve_ex(plan, ft, gt, u, 0.0, steps)
        assert st == B.HELM_MAXITER and iters == steps
        err = _relerr(u.cpu().numpy(), ora.iterates[steps])
        assert err <= 1e-10, (steps, err)
    B.helm_plan_destroy(plan)
    assert np.allclose(hist, ora.relres, rtol=1e-8, atol=1e-14)
    assert np.allclose(einf, ora.einf, rtol=1e-8, atol=0)
