"""GPU parity of the annular problem (square with a square hole, Dirichlet hole, Robin outer
edge; Section 2.3, Section 2.4) against the oracle, through the C ABI.

* converged solutions against the oracle's direct FD solution (FP64 1e-10 relative L2 at
  tol 1e-12; mixed 1e-6 at relres 1e-8), with and without a shift alpha > k^2;
* FP64 iterates and relres history against the oracle's exact-solve iteration (enough
  multigrid cycles per step);
* the status on both sides of rho(G) = 1 (dense eigenvalues of the oracle's G);
* exit time, local time and k_*^A against the oracle;
* argument checks.
"""
import numpy as np
import pytest

from oracle import annulus as an
from oracle import iteration as it

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


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _solve(B, N, k, data, prec, tol, max_outer, alpha=None, cycle=None, hole=0.15):
    plan = B.helm_annulus_create(N, 1.0, hole, k, prec)
    if alpha is not None:
        B.helm_annulus_set_shift(plan, alpha)
    if cycle:
        B.helm_annulus_set_cycle(plan, *cycle)
    d = torch.from_numpy(np.ascontiguousarray(data)).to(DEV)
    u = torch.empty_like(d)
    st, iters, hist = B.helm_annulus_solve(plan, d, u, tol, max_outer)
    B.helm_annulus_destroy(plan)
    return st, iters, hist, u.cpu().numpy()


@pytest.mark.parametrize("N", [32, 64, 256])
@pytest.mark.parametrize("prec", [0, 1])
def test_converged_solution_matches_the_direct_solve(B, N, prec):
    k = 0.8
    g = an.geometry(N)
    data = an.scattering_data(g, k)
    exact = an.solve_direct(g, k, data)
    tol = 1e-12 if prec == 0 else 1e-8
    st, iters, hist, u = _solve(B, N, k, data, prec, tol, 2000)
    assert st == B.HELM_CONVERGED, (st, iters)
    # the error left at a given relres is up to cond(B) times it, and cond(B) of the Robin
    # problem grows like N^2: the bounds scale from N = 128
    grow = max(1.0, (N / 128) ** 2)
    assert _rel(u, exact) <= (1e-10 if prec == 0 else 1e-6) * grow
    assert hist[0] == 1.0 and hist[-1] <= tol


@pytest.mark.parametrize("prec", [0, 1])
def test_shifted_iteration_and_general_data(B, prec):
    N, k = 64, 1.1
    g = an.geometry(N)
    rng = np.random.default_rng(7)
    data = rng.standard_normal((N + 1, N + 1)) + 1j * rng.standard_normal((N + 1, N + 1))
    exact = an.solve_direct(g, k, data)
    tol = 1e-12 if prec == 0 else 1e-8
    st, iters, hist, u = _solve(B, N, k, data, prec, tol, 3000, alpha=k * k + 2.0)
    assert st == B.HELM_CONVERGED
    assert _rel(u, exact) <= (1e-10 if prec == 0 else 1e-6)


def test_iterates_match_the_papers_iteration(B):
    N, k = 32, 0.9
    g = an.geometry(N)
    data = an.scattering_data(g, k)
    ora = an.annulus_iteration(g, k, data, tol=0.0, max_outer=5, keep_iterates=True)
    # 16 V(2,2) cycles per step, each contracting the increment's error by <= 0.3 here,
    # leave <= 0.3^16 ~ 4e-9 of each increment: the iterates agree to 1e-8
    for steps in range(1, 6):
        st, iters, hist, u = _solve(B, N, k, data, 0, 0.0, steps, cycle=(2, 2, 16))
        assert st == B.HELM_MAXITER and iters == steps
        assert _rel(u, ora.iterates[steps]) <= 1e-8
    assert np.allclose(hist, ora.relres, rtol=1e-8, atol=1e-14)


@pytest.mark.parametrize("prec", [0, 1])
def test_status_follows_the_spectral_radius(B, prec):
    N = 16
    g = an.geometry(N)
    for k in (0.9, 1.6):
        rho = an.spectral_radius(g, k)
        st, iters, hist, u = _solve(B, N, k, an.scattering_data(g, k), prec, 1e-8, 3000)
        assert st == (B.HELM_CONVERGED if rho < 1 else B.HELM_DIVERGED), (k, rho, st, iters)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("c_tau", [1.0, 2.0])
def test_exit_time_local_time_and_k_star(B, prec, c_tau):
    N = 64
    g = an.geometry(N)
    E_o, L_o = an.exit_times(g, c_tau)
    plan = B.helm_annulus_create(N, 1.0, 0.15, 1.0, prec)
    E = torch.empty((N + 1, N + 1), dtype=torch.float64, device=DEV)
    L = torch.empty_like(E)
    # relres 1e-11 (FP64): the edge-only data of L put the rounding floor of the residual
    # near 1e-12 at N = 64
    tol = 1e-11 if prec == 0 else 1e-9
    st, ks = B.helm_annulus_exit_times(plan, E, L, c_tau=c_tau, tol=tol)
    B.helm_annulus_destroy(plan)
    assert st == B.HELM_CONVERGED
    bound = 1e-9 if prec == 0 else 1e-6
    assert _rel(E.cpu().numpy(), E_o) <= bound and _rel(L.cpu().numpy(), L_o) <= bound
    assert ks == pytest.approx(an.k_star_A(g, c_tau), rel=(1e-9 if prec == 0 else 1e-6))


def test_argument_checks(B):
    for args in ((12, 1.0, 0.15, 1.0, 1), (64, 1.0, 0.45, 1.0, 1), (64, 1.0, 0.15, -1.0, 1),
                 (64, 1.0, 0.15, 1.0, 7), (64, -1.0, 0.15, 1.0, 1)):
        with pytest.raises(B.HelmError):
            B.helm_annulus_create(*args)
    plan = B.helm_annulus_create(64, 1.0, 0.15, 2.0, 1)
    with pytest.raises(B.HelmError):
        B.helm_annulus_set_shift(plan, 3.9)
    B.helm_annulus_set_shift(plan, 4.0)
    with pytest.raises(B.HelmError):
        B.helm_annulus_set_cycle(plan, 0, 0, 1)
    B.helm_annulus_destroy(plan)


@pytest.mark.parametrize("cycle", [(2, 2, 1), (0, 1, 2), (1, 0, 1)])
def test_repeated_solve_is_bit_identical(B, cycle):
    # the tile kernels stage overlapping windows while other CTAs write their swept nodes:
    # any read of a neighbour's output would show up as run-to-run differences
    N, k = 512, 0.8
    g = an.geometry(N)
    data = an.scattering_data(g, k)
    runs = [_solve(B, N, k, data, 1, 1e-8, 3000, cycle=cycle) for _ in range(3)]
    for st, iters, hist, u in runs[1:]:
        assert st == runs[0][0] and iters == runs[0][1]
        assert np.array_equal(hist, runs[0][2])
        assert np.array_equal(u, runs[0][3])


# ---------------------------------------------------------------------------
# spectrum of G (Section 2.4's figure) against the oracle's dense matrices
# ---------------------------------------------------------------------------

def _dense_dominant(geo, k, alpha=None):
    ev = np.linalg.eigvals(an.iteration_matrix(geo, k, alpha))
    return ev[np.argmax(np.abs(ev))]


@pytest.mark.parametrize("N", [16, 32])
@pytest.mark.parametrize("k", [0.5, 1.0, 1.3])
def test_spectral_radius_against_dense(B, N, k):
    geo = an.geometry(N)
    lam = _dense_dominant(geo, k)
    plan = B.helm_annulus_create(N, 1.0, 0.15, k, B.HELM_PREC_FP64)
    st, rho, lam_gpu, its = B.helm_annulus_spectral_radius(plan, 400, 1e-11, 24)
    B.helm_annulus_destroy(plan)
    assert st == B.HELM_OK, its
    assert abs(rho - abs(lam)) <= 1e-6 * abs(lam), (rho, abs(lam))
    assert abs(lam_gpu - lam) <= 1e-5 * abs(lam), (lam_gpu, lam)


def test_spectral_radius_with_shift_and_mixed(B):
    N, k = 32, 1.0
    geo = an.geometry(N)
    alpha = 1.5
    want = abs(_dense_dominant(geo, k, alpha))
    plan = B.helm_annulus_create(N, 1.0, 0.15, k, B.HELM_PREC_FP64)
    B.helm_annulus_set_shift(plan, alpha)
    st, rho, _, _ = B.helm_annulus_spectral_radius(plan, 400, 1e-11, 24)
    B.helm_annulus_destroy(plan)
    assert st == B.HELM_OK and abs(rho - want) <= 1e-6 * want
    # complex64 cycles: the operator is applied to ~1e-7, rho to a few 1e-6
    want = abs(_dense_dominant(geo, k))
    plan = B.helm_annulus_create(N, 1.0, 0.15, k, B.HELM_PREC_MIXED)
    st, rho, _, _ = B.helm_annulus_spectral_radius(plan, 400, 1e-7, 24)
    B.helm_annulus_destroy(plan)
    assert abs(rho - want) <= 2e-5 * want, (rho, want)


@pytest.mark.parametrize("N", [16, 32])
@pytest.mark.parametrize("k", [0.5, 1.2])
def test_condition_number_against_dense(B, N, k):
    geo = an.geometry(N)
    smax, smin = an.singular_extremes(geo, k)
    plan = B.helm_annulus_create(N, 1.0, 0.15, k, B.HELM_PREC_FP64)
    st, gmax, gmin, cond, its = B.helm_annulus_condition(plan, 2000, 1e-11, 24)
    B.helm_annulus_destroy(plan)
    assert st == B.HELM_OK, its
    assert abs(gmax - smax) <= 1e-6 * smax, (gmax, smax)
    assert abs(gmin - smin) <= 1e-6 * smin, (gmin, smin)
    assert abs(cond - smax / smin) <= 2e-6 * smax / smin


def test_spectral_radius_crossing_follows_dense(B):
    # the k where rho(G) = 1 on the 16-interval grid: the GPU's status on either side of the
    # dense crossing
    geo = an.geometry(16)
    lo, hi = 0.5, 2.0
    for _ in range(40):
        mid = 0.5 * (lo + hi)
        if abs(_dense_dominant(geo, mid)) < 1.0:
            lo = mid
        else:
            hi = mid
    kc = 0.5 * (lo + hi)
    for k, below in ((0.97 * kc, True), (1.03 * kc, False)):
        plan = B.helm_annulus_create(16, 1.0, 0.15, k, B.HELM_PREC_MIXED)
        st, rho, _, _ = B.helm_annulus_spectral_radius(plan, 400, 1e-8, 16)
        B.helm_annulus_destroy(plan)
        assert (rho < 1.0) == below, (k, kc, rho)


def test_spectral_arguments(B):
    plan = B.helm_annulus_create(16, 1.0, 0.15, 0.0, B.HELM_PREC_FP64)
    with pytest.raises(B.HelmError):
        B.helm_annulus_condition(plan, 10, 1e-8, 4)          # k = 0: G is singular
    with pytest.raises(B.HelmError):
        B.helm_annulus_spectral_radius(plan, 10, 1e-8, 0)    # no cycle
    B.helm_annulus_destroy(plan)
