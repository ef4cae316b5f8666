"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances: FP64 results within 1e-10 relative L2 of the oracle (exact discrete solution
or exact-solve iterates), mixed precision (complex64 V-cycles + FP64 outer refinement)
within 1e-6 relative L2 at relres 1e-8; single multigrid cycles element by element
(1e-12 FP64; complex64 1e-4 relative to the array's max, times (n+1)/256 above 255).
"""
import numpy as np
import pytest

from oracle import fd, iteration as it, multigrid as mg
from paper_2308_11469_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_11469_gb300 import binding, build
    build.build()
    binding.load()
    return binding


DEV = "cuda:0"


def _rand_c(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _t(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a)).to(DEV)
    return t if dtype is None else t.to(dtype)


def _relerr(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# ---------------------------------------------------------------------------
# single V-cycles, element by element
# ---------------------------------------------------------------------------
VC_CASES = [(2, 15), (2, 31), (2, 63), (2, 127), (2, 255), (3, 7), (3, 15), (3, 31), (3, 63), (2, 1),
            (3, 1)]


@pytest.mark.parametrize("D,n", VC_CASES)
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("nus", [(2, 2), (1, 1), (0, 2), (3, 1)])
def test_vcycle_elementwise(B, D, n, prec, nus):
    h = 1.0 / (n + 1)
    rng = np.random.default_rng(100 + n + D)
    r = _rand_c(rng, (n,) * D)
    e0 = _rand_c(rng, (n,) * D) * 0.01
    plan = B.helm_plan_create(D, n, h, 1.0, prec=prec)
    _, exact_n = B.helm_plan_coarse(plan)      # the level solved exactly, if any
    E = fd.padded_from(e0.copy())
    mg.vcycle(E, r, h, *nus, exact_n=exact_n or None)
    expect = fd.interior(E)
    dt = torch.complex128 if prec == 0 else torch.complex64
    rt = _t(r, dt)
    et = _t(e0, dt)
    B.poisson_vcycle(plan, rt, et, *nus)
    got = et.cpu().numpy().astype(np.complex128)
    B.helm_plan_destroy(plan)
    scale = np.max(np.abs(expect))
    # complex64: the fine residual rhs - Delta_h e cancels terms ~|e|/h^2 down to ~|rhs|,
    # so one cycle's rounding grows with the grid (~2e-5 at 255, ~1.2e-4 at 1023)
    tol = 1e-12 if prec == 0 else 1e-4 * max(1.0, (n + 1) / 256)
    assert np.max(np.abs(got - expect)) <= tol * scale


@pytest.mark.parametrize("n", [127, 255])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("nus", [(5, 5), (6, 1)])
def test_vcycle_elementwise_generic_2d(B, n, prec, nus):
    # more than four sweeps per side: the 2D levels run on the generic per-sweep kernels
    test_vcycle_elementwise(B, 2, n, prec, nus)


@pytest.mark.parametrize("D,n,prec,want", [
    (2, 1023, 1, (63, 31)), (2, 1023, 0, (31, 15)), (2, 31, 1, (31, 31)), (2, 15, 1, (15, 0)),
    (2, 15, 0, (15, 15)), (2, 7, 0, (7, 0)),
    (3, 255, 1, (15, 15)), (3, 255, 0, (7, 0)), (3, 15, 1, (15, 15)), (3, 7, 1, (7, 0))])
def test_plan_coarse_hierarchy(B, D, n, prec, want):
    plan = B.helm_plan_create(D, n, 1.0 / (n + 1), 1.0, prec=prec)
    assert B.helm_plan_coarse(plan) == want
    B.helm_plan_destroy(plan)


@pytest.mark.parametrize("D,n", [(2, 1023), (2, 511), (3, 127)])
@pytest.mark.parametrize("prec", [0, 1])
def test_vcycle_elementwise_full_size(B, D, n, prec):
    # the bench's 1023^2 grid (10 levels, ragged 64 x 32 tiles) and the 3D 127^3 grid
    test_vcycle_elementwise(B, D, n, prec, (2, 2))


@pytest.mark.parametrize("D,n", [(2, 255), (3, 63)])
def test_vcycles_converge_to_direct_solve(B, D, n):
    h = 1.0 / (n + 1)
    rng = np.random.default_rng(7)
    r = _rand_c(rng, (n,) * D)
    exact = fd.dst_poisson(r, h)
    plan = B.helm_plan_create(D, n, h, 1.0, prec=0)
    et = torch.zeros((n,) * D, dtype=torch.complex128, device=DEV)
    rt = _t(r)
    errs = []
    for _ in range(16):
        B.poisson_vcycle(plan, rt, et, 2, 2)
        errs.append(_relerr(et.cpu().numpy(), exact))
    B.helm_plan_destroy(plan)
    factors = np.asarray(errs[1:6]) / np.asarray(errs[:5])
    assert np.all(factors < (0.1 if D == 2 else 0.15)), factors
    assert errs[-1] < 1e-12


# ---------------------------------------------------------------------------
# whole solves
# ---------------------------------------------------------------------------
def _solve(B, p, prec, tol, max_outer, cycles=1, nus=(2, 2)):
    plan = B.helm_plan_create(p.D, p.n, p.h, p.k, prec=prec)
    if cycles != 1 or nus != (2, 2):
        B.helm_plan_set_cycle(plan, nus[0], nus[1], cycles)
    f = _t(p.f)
    g = _t(p.g)
    u = torch.zeros_like(g)
    st, iters, hist, einf = B.helm_solve_ex(plan, f, g, u, tol, max_outer)
    B.helm_plan_destroy(plan)
    return st, iters, hist, einf, u.cpu().numpy()


@pytest.mark.parametrize("prec", [0, 1])
def test_plane_wave_cavity_63(B, prec):
    p = inputs.plane_wave_cavity_2d(2.0)
    exact = fd.solve_exact_dst(p.f, p.g, p.h, p.k)
    tol = 1e-13 if prec == 0 else 1e-8
    st, iters, hist, einf, u = _solve(B, p, prec, tol, 300)
    assert st == B.HELM_CONVERGED
    assert hist[0] == 1.0 and hist[-1] <= tol and len(hist) == iters + 1
    err = _relerr(u, exact)
    assert err <= (1e-10 if prec == 0 else 1e-6), err
    # wall ring carries g exactly
    ring = u.copy()
    ring[1:-1, 1:-1] = p.g[1:-1, 1:-1]
    assert np.array_equal(ring, p.g)
    # O(h^2) against the continuum plane wave, as the oracle gives
    cont = inputs.plane_wave(2, p.n, p.h, p.k, p.meta["direction"])
    assert 1.5e-5 < np.max(np.abs(u - cont)) < 2.0e-5


@pytest.mark.parametrize("prec", [0, 1])
def test_above_kmax_diverges(B, prec):
    p = inputs.plane_wave_cavity_2d(5.0)
    st, iters, hist, einf, u = _solve(B, p, prec, 1e-10, 400)
    assert st == B.HELM_DIVERGED
    ora = it.paper_iteration(p.f, p.g, p.h, p.k, tol=1e-10, max_outer=400)
    assert ora.status == it.DIVERGED


@pytest.mark.parametrize("D,n", [(2, 63), (3, 15)])
@pytest.mark.parametrize("prec", [0, 1])
def test_status_follows_kmax(B, D, n, prec):
    h = 1.0 / (n + 1)
    rng = np.random.default_rng(11)
    f = _rand_c(rng, (n,) * D)
    g = np.zeros((n + 2,) * D, dtype=np.complex128)
    km = fd.k_max(D, n, h)
    for frac, want in [(0.9, B.HELM_CONVERGED), (1.05, B.HELM_DIVERGED)]:
        p = inputs.Problem(D, n, h, frac * km, f, g)
        st, iters, hist, einf, u = _solve(B, p, prec, 1e-8, 3000)
        assert st == want, (frac, B.helm_status_str(st), iters)
        assert it.predicted_status(D, n, h, frac * km) == (it.CONVERGED if want == 0 else it.DIVERGED)


@pytest.mark.parametrize("D,n,k", [(2, 31, 3.0), (2, 127, 2.5), (3, 15, 3.0), (3, 31, 4.0)])
def test_iterates_match_exact_solve_iterates(B, D, n, k):
    # with enough V-cycles per outer step the inner solves are exact to rounding, so the
    # GPU iterates are the paper's partial sums: compare u^(N) and relres_N step by step
    h = 1.0 / (n + 1)
    rng = np.random.default_rng(12 + n)
    f = _rand_c(rng, (n,) * D)
    g = _rand_c(rng, (n + 2,) * D)
    p = inputs.Problem(D, n, h, k, f, g)
    N = 6
    ora = it.paper_iteration(f, g, h, k, tol=0.0, max_outer=N, keep_iterates=True)
    for steps in range(1, N + 1):
        st, iters, hist, einf, u = _solve(B, p, 0, 0.0, steps, cycles=12)
        assert st == B.HELM_MAXITER and iters == steps
        assert _relerr(u, ora.iterates[steps]) <= 1e-10
    assert np.allclose(hist, ora.relres, rtol=1e-8, atol=1e-14)
    assert np.allclose(einf, ora.einf, rtol=1e-8, atol=0)


def test_discrete_plane_wave_to_roundoff(B):
    D, n, k = 2, 127, 3.0
    h = 1.0 / (n + 1)
    d = (0.6, 0.8)
    kap = fd.discrete_wavenumber(k, h, d)
    w = inputs.plane_wave(D, n, h, kap, d)
    p = inputs.Problem(D, n, h, k, np.zeros((n, n), complex), w)
    st, iters, hist, einf, u = _solve(B, p, 0, 1e-14, 500)
    assert st == B.HELM_CONVERGED
    assert np.max(np.abs(u - w)) < 1e-11


@pytest.mark.parametrize("k", [1.0, 4.0])
@pytest.mark.parametrize("prec", [0, 1])
def test_gaussian_cavity_255(B, k, prec):
    # the 1023^2 Gaussian workload at 255^2 (same source recipe)
    p = inputs.gaussian_cavity_2d(k, seed=2, n=255)
    exact = fd.solve_exact_dst(p.f, p.g, p.h, p.k)
    tol = 1e-12 if prec == 0 else 1e-8
    st, iters, hist, einf, u = _solve(B, p, prec, tol, 2000)
    assert st == B.HELM_CONVERGED
    err = _relerr(u, exact)
    assert err <= (1e-10 if prec == 0 else 1e-6), err


def test_sine_source_cube_31(B):
    D, n, k = 3, 31, 4.0
    p = inputs.plane_wave_sine_cube(k, seed=3, n=n)
    exact = fd.solve_exact_dst(p.f, p.g, p.h, p.k)
    for prec, tol, bound in [(0, 1e-12, 1e-10), (1, 1e-8, 1e-6)]:
        st, iters, hist, einf, u = _solve(B, p, prec, tol, 2000)
        assert st == B.HELM_CONVERGED
        assert _relerr(u, exact) <= bound


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("D,n", [(2, 1), (2, 3), (3, 1), (3, 3)])
def test_tiny_grids(B, D, n):
    h = 1.0 / (n + 1)
    rng = np.random.default_rng(13)
    p = inputs.Problem(D, n, h, 1.3, _rand_c(rng, (n,) * D), _rand_c(rng, (n + 2,) * D))
    exact = fd.solve_exact_splu(p.f, p.g, p.h, p.k)
    st, iters, hist, einf, u = _solve(B, p, 0, 1e-13, 500)
    assert st == B.HELM_CONVERGED
    assert _relerr(u, exact) <= 1e-10


def test_zero_data_and_zero_steps(B):
    n = 31
    p = inputs.Problem(2, n, 1 / 32, 2.0, np.zeros((n, n), complex), np.zeros((n + 2, n + 2), complex))
    st, iters, hist, einf, u = _solve(B, p, 1, 1e-8, 100)
    assert st == B.HELM_CONVERGED and iters == 0 and hist[0] == 0.0
    q = inputs.gaussian_cavity_2d(2.0, n=31)
    st, iters, hist, einf, u = _solve(B, q, 1, 1e-8, 0)
    assert st == B.HELM_MAXITER and iters == 0 and hist[0] == 1.0


def test_nonfinite_input_is_reported(B):
    q = inputs.gaussian_cavity_2d(2.0, n=63)
    q.f[10, 10] = np.nan
    st, iters, hist, einf, u = _solve(B, q, 1, 1e-8, 50)
    assert st == B.HELM_ENONFINITE


def test_invalid_arguments(B):
    with pytest.raises(B.HelmError):
        B.helm_plan_create(2, 100, 0.01, 1.0)          # not 2^m - 1
    with pytest.raises(B.HelmError):
        B.helm_plan_create(4, 7, 0.1, 1.0)
    plan = B.helm_plan_create(2, 7, 1 / 8, 1.0)
    with pytest.raises(B.HelmError):
        B.helm_plan_set_cycle(plan, 0, 0, 1)
    f = torch.zeros((7, 7), dtype=torch.complex128, device=DEV)
    g = torch.zeros((9, 9), dtype=torch.complex128, device=DEV)
    with pytest.raises(B.HelmError):                    # u aliases g
        B.helm_solve(plan, f, g, g, 1e-8, 10)
    with pytest.raises(TypeError):
        B.helm_solve(plan, f.to(torch.complex64), g, g.clone(), 1e-8, 10)
    B.helm_plan_destroy(plan)


def test_plan_info_closed_forms(B):
    plan = B.helm_plan_create(2, 63, 1 / 64, 2.0)
    lmin, kmax, rho, ws = B.helm_plan_info(plan)
    assert abs(lmin - fd.lambda_min(2, 63, 1 / 64)) < 1e-9 * lmin
    assert abs(kmax - fd.k_max(2, 63, 1 / 64)) < 1e-12
    assert abs(rho - fd.rho_pred(2, 63, 1 / 64, 2.0)) < 1e-12
    assert ws > 0
    B.helm_plan_destroy(plan)


def test_repeated_solves_are_deterministic(B):
    p = inputs.gaussian_cavity_2d(3.0, n=127)
    a = _solve(B, p, 1, 1e-8, 500)
    b = _solve(B, p, 1, 1e-8, 500)
    assert a[1] == b[1]
    assert np.array_equal(a[2], b[2])
    assert np.array_equal(a[4], b[4])


def test_integer_pipe_conversions_match_hardware(B):
    # the complex64 residual path converts with integer operations; they must agree with
    # the GPU's own IEEE conversions (round to nearest even) outside the subnormal range
    assert B.helm_selftest_conversions(1 << 22, 12345) == 0


def test_autotuner_picks_a_converging_schedule_and_restores_u(B):
    p = inputs.gaussian_cavity_2d(3.0, n=255)
    plan = B.helm_plan_create(2, p.n, p.h, p.k, prec=1)
    f = _t(p.f)
    g = _t(p.g)
    u0 = _t(np.random.default_rng(3).standard_normal((p.n + 2, p.n + 2)) * 0.0 + 0j)
    u = u0.clone()
    nu1, nu2, cyc, ms = B.helm_plan_autotune(plan, f, g, u, 1e-8, 2000)
    assert (nu1, nu2, cyc) in [(1, 0, 1), (0, 1, 1), (1, 1, 1), (2, 1, 1), (1, 2, 1), (2, 2, 1),
                               (3, 3, 1), (1, 1, 2)]
    assert ms > 0
    assert torch.equal(u, u0)
    st, iters, hist = B.helm_solve(plan, f, g, u, 1e-8, 2000)
    assert st == B.HELM_CONVERGED
    exact = fd.solve_exact_dst(p.f, p.g, p.h, p.k)
    assert _relerr(u.cpu().numpy(), exact) <= 1e-6
    B.helm_plan_destroy(plan)


@pytest.mark.parametrize("prec", [0, 1])
def test_resume_from_a_saved_iterate(B, prec):
    # relres is measured against ||b||: resuming from an interrupted solve continues where
    # it stopped, and resuming from a converged solve stops at once
    p = inputs.gaussian_cavity_2d(3.0, n=127)
    plan = B.helm_plan_create(2, p.n, p.h, p.k, prec=prec)
    f = _t(p.f)
    g = _t(p.g)
    u = torch.zeros_like(g)
    st, it_full, h_full = B.helm_solve(plan, f, g, u, 1e-8, 500)
    assert st == B.HELM_CONVERGED
    st, it0, h0 = B.helm_solve(plan, f, g, u, 1e-8, 500)
    assert st == B.HELM_CONVERGED and it0 == 0 and h0[0] <= 1e-8
    u.zero_()
    st, it_a, h_a = B.helm_solve(plan, f, g, u, 1e-8, 6)
    assert st == B.HELM_MAXITER and it_a == 6
    st, it_b, h_b = B.helm_solve(plan, f, g, u, 1e-8, 500)
    assert st == B.HELM_CONVERGED
    assert abs(h_b[0] - h_a[-1]) <= 1e-6 * h_a[-1]
    assert it_a + it_b <= it_full + 1
    B.helm_plan_destroy(plan)
