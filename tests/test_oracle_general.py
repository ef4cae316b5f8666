"""Pins of the general cavity oracle (shift alpha >= k^2, damping p >= 0; Section 2.2).

Each pin is fixed by something other than the oracle's own code: a hand-worked one-node
example, dense linear algebra (matrix powers, eigenvalues, a dense solve), the reduction
to the alpha = k^2, p = 0 iteration, and the shifted multigrid's exactness properties.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import fd, general as gen, iteration as it, multigrid as mg
from paper_2308_11469_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "general_cavity_hand.json")


def _rand_c(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _problem(D, n, seed):
    rng = np.random.default_rng(seed)
    f = _rand_c(rng, (n,) * D)
    g = fd.padded_from(np.zeros((n,) * D, dtype=np.complex128), _rand_c(rng, (n + 2,) * D))
    return f, g


def _dense_laplacian(D, n, h):
    T = (np.diag(-2.0 * np.ones(n)) + np.diag(np.ones(n - 1), 1) + np.diag(np.ones(n - 1), -1)) / h ** 2
    I = np.eye(n)
    if D == 2:
        return np.kron(I, T) + np.kron(T, I)
    return np.kron(I, np.kron(I, T)) + np.kron(I, np.kron(T, I)) + np.kron(T, np.kron(I, I))


def test_hand_worked_one_node():
    case = json.load(open(GOLDEN))["cases"][0]
    D, n, h, k, alpha, p = case["D"], case["n"], case["h"], case["k"], case["alpha"], case["p"]
    f = np.array([[complex(*case["f"])]])
    g = np.full((3, 3), complex(*case["ring"]["all_sides"]))
    r = gen.general_iteration(f, g, h, k, alpha, p, tol=1e-30, max_outer=3, keep_iterates=True)
    assert r.iterates[1][1, 1] == pytest.approx(complex(*case["u1"]), abs=1e-15)
    assert r.iterates[2][1, 1] == pytest.approx(complex(*case["u2"]), abs=1e-15)
    assert np.allclose(r.relres, case["relres_first"], rtol=1e-13, atol=0)
    assert gen.rho_pred(D, n, h, k, alpha, p) == pytest.approx(case["rho"], rel=1e-15)
    ex = gen.solve_exact(f, g, h, k, p)
    assert ex[1, 1] == pytest.approx(complex(*case["u_exact"]), abs=1e-15)


@pytest.mark.parametrize("D,n", [(2, 3), (2, 5), (3, 3)])
def test_iterates_are_partial_sums_of_the_dense_series(D, n):
    # u^(N) = sum_{j<N} G^j M^{-1} b with M = Delta_h - sigma, G = -(alpha + i p) M^{-1}
    h = 1.0 / (n + 1)
    k, alpha, p = 1.5, 1.5 ** 2 + 3.0, 2.5
    f, g = _problem(D, n, 20 + n + D)
    b = fd.lifted_rhs(f, g, h).reshape(-1)
    M = _dense_laplacian(D, n, h) - (alpha - k * k) * np.eye(n ** D)
    Minv = np.linalg.inv(M)
    G = -(alpha + 1j * p) * Minv
    r = gen.general_iteration(f, g, h, k, alpha, p, tol=1e-30, max_outer=6, keep_iterates=True)
    term = Minv @ b
    acc = np.zeros_like(term)
    for N in range(1, 7):
        acc = acc + term
        term = G @ term
        assert np.allclose(fd.interior(r.iterates[N]).reshape(-1), acc, rtol=0,
                           atol=1e-12 * np.max(np.abs(acc))), N


@pytest.mark.parametrize("D,n", [(2, 7), (3, 5)])
def test_spectral_radius_matches_dense_eigenvalues(D, n):
    h = 1.0 / (n + 1)
    for k, alpha, p in ((2.0, 4.0, 0.0), (2.0, 9.0, 3.0), (1.0, 1.0, 7.5), (3.0, 20.0, 40.0)):
        M = _dense_laplacian(D, n, h) - (alpha - k * k) * np.eye(n ** D)
        ev = np.linalg.eigvals(-(alpha + 1j * p) * np.linalg.inv(M))
        assert np.max(np.abs(ev)) == pytest.approx(gen.rho_pred(D, n, h, k, alpha, p), rel=1e-10)


def test_converged_result_is_the_dense_solution():
    D, n = 2, 15
    h = 1.0 / (n + 1)
    k, alpha, p = 2.0, 6.0, 3.0
    f, g = _problem(D, n, 5)
    r = gen.general_iteration(f, g, h, k, alpha, p, tol=1e-13, max_outer=500)
    assert r.status == it.CONVERGED
    A = _dense_laplacian(D, n, h) + (k * k + 1j * p) * np.eye(n ** D)
    want = np.linalg.solve(A, fd.lifted_rhs(f, g, h).reshape(-1)).reshape((n,) * D)
    assert np.linalg.norm(fd.interior(r.u) - want) <= 1e-11 * np.linalg.norm(want)
    ex = gen.solve_exact(f, g, h, k, p)
    assert np.linalg.norm(fd.interior(ex) - want) <= 1e-12 * np.linalg.norm(want)


def test_alpha_k2_without_damping_is_the_plain_iteration():
    p_ = inputs.plane_wave_cavity_2d(2.0)
    a = it.paper_iteration(p_.f, p_.g, p_.h, p_.k, tol=1e-10, max_outer=100)
    b = gen.general_iteration(p_.f, p_.g, p_.h, p_.k, p_.k ** 2, 0.0, tol=1e-10, max_outer=100)
    assert a.iters == b.iters and a.status == b.status
    assert np.allclose(a.relres, b.relres, rtol=1e-12, atol=1e-15)
    assert np.allclose(a.u, b.u, rtol=0, atol=1e-12)


def test_residual_ratio_tends_to_rho():
    D, n = 2, 31
    h = 1.0 / (n + 1)
    k, alpha, p = 3.0, 12.0, 6.0
    f, g = _problem(D, n, 9)
    rho = gen.rho_pred(D, n, h, k, alpha, p)
    r = gen.general_iteration(f, g, h, k, alpha, p, tol=1e-300, max_outer=22)
    ratios = np.asarray(r.relres[1:]) / np.asarray(r.relres[:-1])
    # G is normal, so ||r_{N+1}|| <= rho ||r_N|| (up to rounding), and the ratio tends to rho
    assert np.all(ratios[1:] <= rho * (1 + 1e-8))
    assert ratios[-1] == pytest.approx(rho, rel=1e-6)


@pytest.mark.parametrize("p", [0.0, 5.0, 15.0])
def test_status_follows_the_spectral_radius(p):
    # fix alpha and p, move k across the limit k^2 = lambda_min + alpha - sqrt(alpha^2+p^2)
    D, n = 2, 15
    h = 1.0 / (n + 1)
    lam = fd.lambda_min(D, n, h)
    alpha = lam + 10.0                    # alpha >= k^2 for every k tried
    klim = gen.k_limit(D, n, h, alpha, p)
    assert klim ** 2 <= lam + 1e-12       # damping only lowers the limit
    f, g = _problem(D, n, 3)
    for frac, want in ((0.9, it.CONVERGED), (1.1, it.DIVERGED)):
        k = frac * klim
        assert gen.predicted_status(D, n, h, k, alpha, p) == want
        r = gen.general_iteration(f, g, h, k, alpha, p, tol=1e-10, max_outer=3000)
        assert r.status == want, (frac, r.status, r.iters)


def test_needs_alpha_at_least_k2():
    f, g = _problem(2, 3, 1)
    with pytest.raises(ValueError):
        gen.general_iteration(f, g, 0.25, 2.0, 3.0, 0.0)
    with pytest.raises(ValueError):
        gen.general_iteration(f, g, 0.25, 1.0, 3.0, -1.0)


# ---------------------------------------------------------------------------
# the shifted multigrid
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("D", [2, 3])
def test_shifted_half_sweep_solves_its_nodes(D):
    n, sigma = 7, 37.0
    h = 1.0 / (n + 1)
    rng = np.random.default_rng(4)
    r = _rand_c(rng, (n,) * D)
    E = fd.padded_from(_rand_c(rng, (n,) * D))
    for color in (0, 1):
        mg.rbgs_half_sweep(E, r, h, color, sigma)
        res = mg.poisson_residual(E, r, h, sigma)
        mask = mg.color_mask(D, n, color)
        assert np.max(np.abs(res[mask])) <= 1e-10 * np.max(np.abs(r))


@pytest.mark.parametrize("D,n,xn", [(2, 63, None), (2, 63, 31), (3, 15, None)])
def test_shifted_vcycle_converges_to_the_shifted_solve(D, n, xn):
    sigma = 250.0
    h = 1.0 / (n + 1)
    rng = np.random.default_rng(8)
    r = _rand_c(rng, (n,) * D)
    exact = gen.dst_shifted_poisson(r, h, sigma)
    lu = gen.ShiftedSolver(D, n, h, sigma)
    assert np.allclose(exact, lu(r.real) + 1j * lu(r.imag), rtol=0, atol=1e-12 * np.max(np.abs(exact)))
    E = np.zeros((n + 2,) * D, dtype=np.complex128)
    errs = []
    for _ in range(12):
        mg.vcycle(E, r, h, 2, 2, exact_n=xn, sigma=sigma)
        errs.append(np.linalg.norm(fd.interior(E) - exact) / np.linalg.norm(exact))
    factors = np.asarray(errs[1:6]) / np.asarray(errs[:5])
    assert np.all(factors < (0.1 if D == 2 else 0.15)), factors
    assert errs[-1] < 1e-11


def test_shift_only_helps_the_smoother():
    # a positive shift makes every local solve more diagonally dominant: one cycle
    # reduces the error at least as much as without it
    n = 63
    h = 1.0 / (n + 1)
    rng = np.random.default_rng(2)
    r = _rand_c(rng, (n, n))
    out = []
    for sigma in (0.0, 500.0):
        exact = gen.dst_shifted_poisson(r, h, sigma)
        E = np.zeros((n + 2, n + 2), dtype=np.complex128)
        mg.vcycle(E, r, h, 1, 1, sigma=sigma)
        out.append(np.linalg.norm(fd.interior(E) - exact) / np.linalg.norm(exact))
    assert out[1] <= out[0] * 1.01


def test_sufficient_condition_of_the_theorem_implies_contraction():
    # (alpha + p) max E < 1, E the exit time (Delta_h E = -1), implies rho < 1: the sup
    # norm of -Delta_h^{-1} bounds its spectral radius, so 1/lambda_min <= max E
    D, n = 2, 31
    h = 1.0 / (n + 1)
    Emax = float(np.max(fd.dst_poisson(-np.ones((n, n)), h)))
    assert 1.0 / fd.lambda_min(D, n, h) <= Emax
    for alpha, p in ((5.0, 2.0), (10.0, 3.0), (12.0, 1.0)):
        if (alpha + p) * Emax < 1.0:
            k = math.sqrt(alpha)
            assert gen.rho_pred(D, n, h, k, alpha, p) < 1.0
