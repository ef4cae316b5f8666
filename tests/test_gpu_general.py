"""GPU parity of the general cavity iteration (shift alpha >= k^2, damping p >= 0;
Section 2.2, Eq. (2.4)-(2.8)) against the oracle, through the C ABI.

* single shifted V-cycles element by element (FP64 1e-12, complex64 1e-4 of the max);
* FP64 iterates = the oracle's exact-solve iterates (1e-10) with enough cycles per step;
* converged results against the exact discrete solution of (Delta_h + k^2 + i p) u = f
  (FP64 1e-10 at tol 1e-12, mixed 1e-6 at relres 1e-8), 2D and 3D;
* the CONVERGED / DIVERGED status across the k limit of the damped iteration;
* plan closed forms, argument checks, batch = single solve bit for bit.
"""
import numpy as np
import pytest

from oracle import fd, general as gen, iteration as it, multigrid as mg
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


def _rand_c(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _t(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a)).to(DEV)
    return t if dtype is None else t.to(dtype)


def _relerr(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _plan(B, D, n, h, k, prec, alpha, p, cycle=None):
    plan = B.helm_plan_create(D, n, h, k, prec=prec)
    B.helm_plan_set_cavity(plan, alpha, p)
    if cycle:
        B.helm_plan_set_cycle(plan, *cycle)
    return plan


def _solve(B, D, n, h, k, f, g, prec, alpha, p, tol, max_outer, cycle=None):
    plan = _plan(B, D, n, h, k, prec, alpha, p, cycle)
    u = torch.zeros((n + 2,) * D, dtype=torch.complex128, device=DEV)
    st, iters, hist, einf = B.helm_solve_ex(plan, _t(f), _t(g), u, tol, max_outer)
    B.helm_plan_destroy(plan)
    return st, iters, hist, einf, u.cpu().numpy()


@pytest.mark.parametrize("D,n", [(2, 31), (2, 63), (2, 255), (2, 1023), (3, 15), (3, 63)])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("nus", [(2, 2), (0, 1)])
def test_shifted_vcycle_elementwise(B, D, n, prec, nus):
    h = 1.0 / (n + 1)
    k = 2.0
    alpha, p = k * k + 3.0e4 * h, 7.0          # sigma large enough to matter on every level
    rng = np.random.default_rng(300 + n + D)
    r = _rand_c(rng, (n,) * D)
    e0 = _rand_c(rng, (n,) * D) * 0.01
    plan = _plan(B, D, n, h, k, prec, alpha, p)
    _, exact_n = B.helm_plan_coarse(plan)
    E = fd.padded_from(e0.copy())
    mg.vcycle(E, r, h, *nus, exact_n=exact_n or None, sigma=alpha - k * k)
    expect = fd.interior(E)
    dt = torch.complex128 if prec == 0 else torch.complex64
    et = _t(e0, dt)
    B.poisson_vcycle(plan, _t(r, dt), et, *nus)
    got = et.cpu().numpy().astype(np.complex128)
    B.helm_plan_destroy(plan)
    scale = np.max(np.abs(expect))
    tol = 1e-12 if prec == 0 else 1e-4 * max(1.0, (n + 1) / 256)
    assert np.max(np.abs(got - expect)) <= tol * scale


@pytest.mark.parametrize("D,n,k,dalpha,p", [(2, 31, 3.0, 5.0, 4.0), (2, 127, 2.5, 0.0, 6.0),
                                           (3, 15, 3.0, 8.0, 2.0)])
def test_iterates_match_the_papers_v_w_iteration(B, D, n, k, dalpha, p):
    # enough cycles per step make the inner solves exact to rounding: the GPU iterates are
    # the oracle's v_n + i w_n partial sums of Eq. (2.6)
    h = 1.0 / (n + 1)
    alpha = k * k + dalpha
    rng = np.random.default_rng(40 + n)
    f = _rand_c(rng, (n,) * D)
    g = _rand_c(rng, (n + 2,) * D)
    N = 6
    ora = gen.general_iteration(f, g, h, k, alpha, p, tol=0.0, max_outer=N, keep_iterates=True)
    for steps in range(1, N + 1):
        st, iters, hist, einf, u = _solve(B, D, n, h, k, f, g, 0, alpha, p, 0.0, steps, (2, 2, 12))
        assert st == B.HELM_MAXITER and iters == steps
        assert _relerr(u, ora.iterates[steps]) <= 1e-10
    assert np.allclose(hist, ora.relres, rtol=1e-8, atol=1e-14)
    assert np.allclose(einf, ora.einf, rtol=1e-8, atol=0)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("dalpha,p", [(0.0, 5.0), (20.0, 0.0), (10.0, 15.0)])
def test_gaussian_cavity_255_damped(B, prec, dalpha, p):
    q = inputs.gaussian_cavity_2d(3.0, seed=2, n=255)
    alpha = q.k ** 2 + dalpha
    exact = gen.solve_exact(q.f, q.g, q.h, q.k, p)
    tol = 1e-12 if prec == 0 else 1e-8
    st, iters, hist, einf, u = _solve(B, 2, q.n, q.h, q.k, q.f, q.g, prec, alpha, p, tol, 3000)
    assert st == B.HELM_CONVERGED
    assert _relerr(u, exact) <= (1e-10 if prec == 0 else 1e-6)
    assert gen.predicted_status(2, q.n, q.h, q.k, alpha, p) == it.CONVERGED


def test_sine_cube_63_damped(B):
    q = inputs.plane_wave_sine_cube(4.0, seed=3, n=63)
    alpha, p = q.k ** 2 + 4.0, 3.0
    exact = gen.solve_exact(q.f, q.g, q.h, q.k, p)
    for prec, tol, bound in [(0, 1e-12, 1e-10), (1, 1e-10, 1e-6)]:
        st, iters, hist, einf, u = _solve(B, 3, q.n, q.h, q.k, q.f, q.g, prec, alpha, p, tol, 3000)
        assert st == B.HELM_CONVERGED
        assert _relerr(u, exact) <= bound


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("p", [4.0, 12.0])
def test_status_follows_the_damped_k_limit(B, prec, p):
    D, n = 2, 63
    h = 1.0 / (n + 1)
    lam = fd.lambda_min(D, n, h)
    alpha = lam + 8.0
    klim = gen.k_limit(D, n, h, alpha, p)
    rng = np.random.default_rng(21)
    f = _rand_c(rng, (n, n))
    g = np.zeros((n + 2, n + 2), dtype=np.complex128)
    for frac, want in [(0.9, B.HELM_CONVERGED), (1.1, B.HELM_DIVERGED)]:
        k = frac * klim
        st, iters, *_ = _solve(B, D, n, h, k, f, g, prec, alpha, p, 1e-8, 4000)
        assert st == want, (frac, B.helm_status_str(st), iters)
        assert gen.predicted_status(D, n, h, k, alpha, p) == (it.CONVERGED if want == 0 else it.DIVERGED)


def test_plan_closed_forms(B):
    D, n = 2, 127
    h = 1.0 / (n + 1)
    for k, alpha, p in [(2.0, 4.0, 0.0), (2.0, 10.0, 0.0), (3.0, 9.0, 5.0), (1.0, 40.0, 30.0)]:
        plan = _plan(B, D, n, h, k, 1, alpha, p)
        lam, kmax, rho, _ = B.helm_plan_info(plan)
        assert lam == pytest.approx(fd.lambda_min(D, n, h), rel=1e-14)
        assert rho == pytest.approx(gen.rho_pred(D, n, h, k, alpha, p), rel=1e-14)
        want_k = fd.k_max(D, n, h) if p == 0 else gen.k_limit(D, n, h, alpha, p)
        assert kmax == pytest.approx(want_k, rel=1e-14)
        B.helm_plan_destroy(plan)


def test_set_cavity_rejects_bad_values(B):
    plan = B.helm_plan_create(2, 31, 1 / 32, 2.0)
    for alpha, p in [(3.9, 0.0), (5.0, -1.0), (float("nan"), 0.0), (5.0, float("inf"))]:
        with pytest.raises(B.HelmError):
            B.helm_plan_set_cavity(plan, alpha, p)
    B.helm_plan_set_cavity(plan, 4.0, 0.0)                # alpha = k^2 exactly is allowed
    B.helm_plan_destroy(plan)


def test_batch_equals_single_solve(B):
    q = inputs.gaussian_cavity_2d(2.0, seed=2, n=127)
    alpha, p = q.k ** 2 + 6.0, 4.0
    st, iters, hist, einf, u_single = _solve(B, 2, q.n, q.h, q.k, q.f, q.g, 1, alpha, p, 1e-8, 2000)
    plan = _plan(B, 2, q.n, q.h, q.k, 1, alpha, p)
    batch = B.helm_batch_create(0)
    B.helm_batch_set_cycle(batch, 2, 2, 1)
    u = torch.zeros((q.n + 2,) * 2, dtype=torch.complex128, device=DEV)
    t = B.helm_batch_submit(batch, plan, _t(q.f), _t(q.g), u, 1e-8, 2000)
    B.helm_batch_step(batch, 0)
    r = B.helm_batch_poll(batch, t, 2000)
    B.helm_batch_destroy(batch)
    B.helm_plan_destroy(plan)
    assert r[0] == st and r[1] == iters
    assert np.array_equal(u.cpu().numpy(), u_single)


def test_batch_slot_reused_by_a_damped_solve(B):
    # an undamped solve retires, a damped one of the same size takes its slot: the launch
    # plan must switch to the residual that carries the damping term
    q = inputs.gaussian_cavity_2d(2.0, seed=2, n=127)
    alpha, p = q.k ** 2 + 6.0, 4.0
    st_ref, it_ref, _, _, u_ref = _solve(B, 2, q.n, q.h, q.k, q.f, q.g, 1, alpha, p, 1e-8, 2000)
    batch = B.helm_batch_create(0)
    plain = B.helm_plan_create(2, q.n, q.h, q.k, prec=1)
    damped = _plan(B, 2, q.n, q.h, q.k, 1, alpha, p)
    for plan, want in ((plain, None), (damped, u_ref)):
        u = torch.zeros((q.n + 2,) * 2, dtype=torch.complex128, device=DEV)
        t = B.helm_batch_submit(batch, plan, _t(q.f), _t(q.g), u, 1e-8, 2000)
        B.helm_batch_step(batch, 0)
        r = B.helm_batch_poll(batch, t, 2000)
        assert r[0] == B.HELM_CONVERGED
        if want is not None:
            assert r[1] == it_ref
            assert np.array_equal(u.cpu().numpy(), want)
    B.helm_batch_destroy(batch)
    B.helm_plan_destroy(plain)
    B.helm_plan_destroy(damped)


def test_batch_starts_damped_and_undamped_together(B):
    # solves of one size started together by one engine: those without a damping term and
    # those with one take separate initial-residual launches (the kernel variant differs);
    # every result is that of the solve alone, bit for bit
    q = inputs.gaussian_cavity_2d(2.0, seed=2, n=127)
    cases = [(q.k ** 2, 0.0), (q.k ** 2 + 6.0, 4.0), (q.k ** 2, 0.0), (q.k ** 2 + 3.0, 2.0)]
    refs = [_solve(B, 2, q.n, q.h, q.k, q.f, q.g, 1, a, p, 1e-8, 2000) for a, p in cases]
    batch = B.helm_batch_create(0)
    B.helm_batch_set_lanes(batch, 1)
    f, g = _t(q.f), _t(q.g)                      # alive until the batch has run
    plans = [_plan(B, 2, q.n, q.h, q.k, 1, a, p) for a, p in cases]
    us = [torch.zeros((q.n + 2,) * 2, dtype=torch.complex128, device=DEV) for _ in cases]
    tickets = [B.helm_batch_submit(batch, pl, f, g, u, 1e-8, 2000) for pl, u in zip(plans, us)]
    B.helm_batch_step(batch, 0)
    for i, t in enumerate(tickets):
        r = B.helm_batch_poll(batch, t, 2000)
        st, iters, hist, _, u_ref = refs[i]
        assert r[0] == st == B.HELM_CONVERGED and r[1] == iters
        assert np.array_equal(r[2], hist)
        assert np.array_equal(us[i].cpu().numpy(), u_ref)
    B.helm_batch_destroy(batch)
    for pl in plans:
        B.helm_plan_destroy(pl)
